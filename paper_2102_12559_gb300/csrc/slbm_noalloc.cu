// slbm_noalloc.cu -- slbm_audit_dense_noalloc: the FP64 conservation audit
// for a dense, caller-owned population field, with no allocation at all.
//
// The audit is a two-pass reduction whose per-block partial sums need
// scratch memory.  Here that scratch is a file-scope device array of fixed
// size, so callers that must not allocate (inside a stream capture, in a
// real-time loop, or under a framework that owns all device memory) can
// still run it.  Host code cannot hand the array's name to a kernel (on the
// host it is only a stand-in symbol), so the first call on each device looks
// up its device address with cudaGetSymbolAddress, with that device current.
#include <mutex>

#include "../../include/slbm.h"
#include "slbm_impl.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kBlocks = SLBM_NOALLOC_MAX_BLOCKS;
constexpr int kMaxDevices = 64;

// Per-block partial sums {rho, rho u_x, rho u_y, rho E}.  Every call writes
// the entries of the blocks it launches before reading them, so nothing has
// to start at zero; calls that overlap on the GPU share it and race.
static __device__ __align__(256) double g_partials[4 * kBlocks];

struct DeviceScratch {
  std::once_flag once;
  double* ptr = nullptr;
  cudaError_t err = cudaSuccess;
};
DeviceScratch g_scratch[kMaxDevices];

struct Velocities {
  double c[slbm::kMaxN];
};

__global__ void __launch_bounds__(kThreads)
k_audit_dense_partial(const float* __restrict__ f, int n, long long ncell, Velocities v,
                      double* partials) {
  __shared__ double sh[4][kThreads];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * kThreads)
    for (int iy = 0; iy < n; ++iy)
      for (int ix = 0; ix < n; ++ix) {
        const double fi = (double)f[(size_t)(ix + n * iy) * ncell + c];
        const double cx = v.c[ix], cy = v.c[iy];
        a[0] += fi;
        a[1] += cx * fi;
        a[2] += cy * fi;
        a[3] += 0.5 * (cx * cx + cy * cy) * fi;
      }
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) partials[4 * blockIdx.x + q] = sh[q][0];
}

__global__ void __launch_bounds__(kThreads)
k_audit_dense_final(const double* partials, int nparts, double* out) {
  __shared__ double sh[4][kThreads];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nparts; b += kThreads)
    for (int q = 0; q < 4; ++q) a[q] += partials[4 * b + q];
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 4; ++q) out[q] = sh[q][0];
}

}  // namespace

extern "C" int slbm_audit_dense_noalloc(const float* f, int lattice, int nx, int ny, double* out,
                                        void* cuda_stream) {
  if (!f || !out || lattice < SLBM_D2Q9 || lattice > SLBM_D2Q25 || nx < 1 || ny < 1)
    return SLBM_EINVAL;
  const long long ncell = (long long)nx * ny;
  if (ncell > SLBM_NOALLOC_MAX_CELLS) return SLBM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SLBM_ECUDA;
  }
  DeviceScratch& s = g_scratch[dev];
  std::call_once(s.once, [&s] {
    s.err = cudaGetSymbolAddress(reinterpret_cast<void**>(&s.ptr), g_partials);
  });
  if (s.err != cudaSuccess || !s.ptr) return SLBM_ECUDA;
  Velocities v{};
  double w[slbm::kMaxN];
  slbm::host_gauss_hermite(lattice, v.c, w);
  const long long want = (ncell + kThreads - 1) / kThreads;
  const int blocks = (int)(want < kBlocks ? want : kBlocks);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  k_audit_dense_partial<<<blocks, kThreads, 0, st>>>(f, lattice, ncell, v, s.ptr);
  k_audit_dense_final<<<1, kThreads, 0, st>>>(s.ptr, blocks, out);
  return cudaGetLastError() == cudaSuccess ? SLBM_OK : SLBM_ECUDA;
}
