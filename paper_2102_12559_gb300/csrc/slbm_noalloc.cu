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
// A failed lookup is not remembered: the next call tries again.
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

// Device address of g_partials per device ordinal, cached once found.
std::mutex g_scratch_mu;
double* g_scratch[kMaxDevices] = {};

// g_partials' address on the current device `dev`, or null if the lookup
// failed (its error is cleared from the runtime's last-error state, which
// belongs to the caller).
double* scratch_on(int dev) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return nullptr;
    }
    g_scratch[dev] = static_cast<double*>(p);
  }
  return g_scratch[dev];
}

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
  double* partials = scratch_on(dev);
  if (!partials) return SLBM_ECUDA;
  Velocities v{};
  double w[slbm::kMaxN];
  slbm::host_gauss_hermite(lattice, v.c, w);
  const long long want = (ncell + kThreads - 1) / kThreads;
  int blocks = (int)(want < kBlocks ? want : kBlocks);
  int n = lattice;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // each launch's own status (an error left by an earlier call of the caller
  // is neither reported nor cleared here)
  void* a1[] = {(void*)&f, (void*)&n, (void*)&ncell, (void*)&v, (void*)&partials};
  cudaError_t e = cudaLaunchKernel((const void*)k_audit_dense_partial, dim3(blocks),
                                   dim3(kThreads), a1, 0, st);
  if (e == cudaSuccess) {
    void* a2[] = {(void*)&partials, (void*)&blocks, (void*)&out};
    e = cudaLaunchKernel((const void*)k_audit_dense_final, dim3(1), dim3(kThreads), a2, 0, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();  // this call's own launch error
    return SLBM_ECUDA;
  }
  return SLBM_OK;
}
