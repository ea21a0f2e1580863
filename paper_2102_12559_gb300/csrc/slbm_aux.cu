// slbm_aux.cu -- setup ghost / boundary fill, equilibrium initialisation,
// macroscopic moments, Mach criterion, FP64 audit and host packing kernels.  S = storage type, R = arithmetic type (float for the FP32
// path: GB300's FP64 rate is a small fraction of its FP32 rate, so doubles
// appear only in moment sums and the audit).
#include "../../include/slbm.h"
#include "slbm_ghost.cuh"

namespace slbm {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <class S, class R>
__device__ __forceinline__ void load_dev(const LatTab<R>& L, const S* f, long long plane, int base,
                                         R (*s)[kMaxN]) {
  for (int iy = 0; iy < L.n; ++iy)
    for (int ix = 0; ix < L.n; ++ix)
      s[iy][ix] = from_s<R>(f[(size_t)(ix + L.n * iy) * plane + base], L.sc[ix + L.n * iy]);
}

template <class S, class R>
__device__ __forceinline__ void store_dev(const LatTab<R>& L, S* f, long long plane, int base,
                                          const R (*s)[kMaxN]) {
  for (int iy = 0; iy < L.n; ++iy)
    for (int ix = 0; ix < L.n; ++ix)
      f[(size_t)(ix + L.n * iy) * plane + base] = to_s<S, R>(s[iy][ix], L.isc[ix + L.n * iy]);
}

// rho of an interior cell from its own lattice (FP64 sum of 1 + deviations).
template <class S, class R>
__device__ double cell_rho(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                           int x, int y) {
  const int k = flag[x + p.nx * y];
  const int n = p.lat[k].n;
  const S* f = k ? f1 : f0;
  const int base = (y + p.G) * p.pitch + (x + kOX);
  double r = 1.0;
  for (int i = 0; i < n * n; ++i) r += (double)from_s<R>(f[(size_t)i * p.plane + base], p.lat[k].sc[i]);
  return r;
}

template <class S, class R>
__device__ void write_eq_both(const Params<R>& p, S* f0, S* f1, int base, double rho, double ux,
                              double uy) {
  R e[kMaxN][kMaxN];
  for (int k = 0; k < 2; ++k) {
    eq_dev<R>(p.lat[k], p.lat[k].n, (R)(rho - 1.0), (R)ux, (R)uy, e);
    store_dev<S, R>(p.lat[k], k ? f1 : f0, p.plane, base, e);
  }
}

// Ghost ring: periodic images, or the boundary state of a non-periodic side
// in both lattices (OUTFLOW copies the nearest interior cell, DIRICHLET /
// INLET write the lattice equilibrium).  A non-periodic y side wins at corners.
template <class S, class R>
__global__ void k_ghosts(const Params<R> p, S* f0, S* f1, const uint8_t* __restrict__ flag,
                         const BcDev bc) {
  const int G = p.G;
  const int total = 2 * G * (p.nx + 2 * G) + 2 * G * p.ny + bc.nwall;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int gx, gy, sx, sy, side = 0, bidx = 0;
  const int kind = ghost_cell(G, p.nx, p.ny, p.periodic_x, p.periodic_y, bc, idx, gx, gy, sx, sy,
                              side, bidx);
  const int gbase = (gy + G) * p.pitch + (gx + kOX);
  const int sbase = (sy + G) * p.pitch + (sx + kOX);
  if (kind == 1 || kind == 2) {
    const double er = kind == 1 ? cell_rho<S, R>(p, f0, f1, flag, sx, sy) : bc.rho[side][bidx];
    write_eq_both<S, R>(p, f0, f1, gbase, er, bc.ux[side][bidx], bc.uy[side][bidx]);
  } else if (kind == 3) {
    // diffuse wall, both lattices, every population
    const R uwx = (R)ghost_ux(bc, side, bidx), uwy = (R)ghost_uy(bc, side, bidx);
    for (int k = 0; k < 2; ++k) {
      S* f = k ? f1 : f0;
      const int n = p.lat[k].n;
      for (int i = 0; i < n * n; ++i) {
        R v;
        if (n == 3) v = diffuse_value<3, S, R>(p.lat[k], f, p.plane, sbase, side, uwx, uwy, i);
        else if (n == 4) v = diffuse_value<4, S, R>(p.lat[k], f, p.plane, sbase, side, uwx, uwy, i);
        else v = diffuse_value<5, S, R>(p.lat[k], f, p.plane, sbase, side, uwx, uwy, i);
        f[(size_t)i * p.plane + gbase] = to_s<S, R>(v, p.lat[k].isc[i]);
      }
    }
  } else {
    const int q0 = p.lat[0].n * p.lat[0].n, q1 = p.lat[1].n * p.lat[1].n;
    S v[kMaxN * kMaxN];  // loads first, then stores (no serialised round trips)
    for (int i = 0; i < q0; ++i) v[i] = f0[(size_t)i * p.plane + sbase];
    for (int i = 0; i < q0; ++i) f0[(size_t)i * p.plane + gbase] = v[i];
    for (int i = 0; i < q1; ++i) v[i] = f1[(size_t)i * p.plane + sbase];
    for (int i = 0; i < q1; ++i) f1[(size_t)i * p.plane + gbase] = v[i];
  }
}

template <class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_init_eq(const Params<R> p, S* f0, S* f1, const double* __restrict__ rho,
          const double* __restrict__ ux, const double* __restrict__ uy) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = x + p.nx * y;
  write_eq_both<S, R>(p, f0, f1, (y + p.G) * p.pitch + (x + kOX), rho[c], ux[c], uy[c]);
}

// rho, momentum and total energy (sum v^2/2 f, plus sum g in the
// two-population model) of a cell's own lattice, in FP64.  lam (three frame
// planes of stride nx*ny, or null for the lattice frame) gives the co-moving
// frame {u, T} the populations live in: v_i = sqrt(T) c_i + u.  e0 / e1: the g
// planes (g / T - (C_v - 1) W_i), or null.
template <class S, class R>
__device__ void cell_moments(const Params<R>& p, const S* f0, const S* f1, int k, int base,
                             double& r, double& jx, double& jy, double& e,
                             const S* lam = nullptr, long long c = 0, const S* e0 = nullptr,
                             const S* e1 = nullptr) {
  if (k == kFlagGap) {  // no fluid: zero in every sum
    r = jx = jy = e = 0.0;
    return;
  }
  const LatTab<R>& L = p.lat[k];
  const S* f = k ? f1 : f0;
  r = 1.0;
  jx = jy = 0.0;
  e = 1.0;  // sum W_i |c_i|^2 / 2 = D T_L / 2 = 1
  for (int iy = 0; iy < L.n; ++iy)
    for (int ix = 0; ix < L.n; ++ix) {
      const double v =
          (double)from_s<R>(f[(size_t)(ix + L.n * iy) * p.plane + base], L.sc[ix + L.n * iy]);
      const double cx = (double)L.c[ix], cy = (double)L.c[iy];
      r += v;
      jx += cx * v;
      jy += cy * v;
      e += 0.5 * (cx * cx + cy * cy) * v;
    }
  if constexpr (!is_fx16<S>())  // co-moving frames (lam) never store fixed point
  if (lam) {
    const long long nc = (long long)p.nx * p.ny;
    const double ux = (double)lam[c], uy = (double)lam[nc + c], T = (double)lam[2 * nc + c];
    const double st = sqrt(T);
    // sum v f = rho u + sqrt(T) sum c f; sum |v|^2/2 f likewise expanded
    e = T * e + st * (ux * jx + uy * jy) + 0.5 * r * (ux * ux + uy * uy);
    jx = r * ux + st * jx;
    jy = r * uy + st * jy;
    const S* g = k ? e1 : e0;
    if (g) {  // sum g = T (sum e + C_v - 1)
      double sg = p.cv - 1.0;
      for (int i = 0; i < L.n * L.n; ++i) sg += (double)from_s<R>(g[(size_t)i * p.plane + base], R(1));
      e += T * sg;
    }
  }
}

template <class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_moments(const Params<R> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
          double* rho, double* ux, double* uy, double* T, const S* lam, const S* e0,
          const S* e1) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = x + p.nx * y;
  double r, jx, jy, e;
  cell_moments<S, R>(p, f0, f1, flag[c], (y + p.G) * p.pitch + (x + kOX), r, jx, jy, e, lam, c,
                     e0, e1);
  if (r == 0.0) {  // a gap cell between channels: no fluid, every moment 0
    if (rho) rho[c] = 0.0;
    if (ux) ux[c] = 0.0;
    if (uy) uy[c] = 0.0;
    if (T) T[c] = 0.0;
    return;
  }
  const double u = jx / r, v = jy / r;
  if (rho) rho[c] = r;
  if (ux) ux[c] = u;
  if (uy) uy[c] = v;
  if (T) T[c] = e0 ? (e / r - 0.5 * (u * u + v * v)) / p.cv : (2.0 * e / r - u * u - v * v) / 2.0;
}

// Mach criterion of Sec. IV.A on the current state (flag = |u| > thr, c_s = 1).
template <class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_criterion(const Params<R> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
            uint8_t* __restrict__ flag_new) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = x + p.nx * y;
  if (flag[c] == kFlagGap) {
    flag_new[c] = kFlagGap;
    return;
  }
  double r, jx, jy, e;
  cell_moments<S, R>(p, f0, f1, flag[c], (y + p.G) * p.pitch + (x + kOX), r, jx, jy, e);
  const R u = (R)(jx / r), v = (R)(jy / r);
  flag_new[c] = sqrt(u * u + v * v) > p.thr ? 1 : 0;
}

// FP64 conservation audit: per-block partial sums, then one block adds the
// partials in a fixed order (deterministic result).
template <class S, class R>
__global__ void __launch_bounds__(kThreads)
k_audit_partial(const Params<R> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
                double* partials, const S* lam, const S* e0, const S* e1) {
  __shared__ double sh[4][kThreads];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  const long long ncell = (long long)p.nx * p.ny;
  for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * kThreads) {
    const int x = (int)(c % p.nx), y = (int)(c / p.nx);
    double r, jx, jy, e;
    cell_moments<S, R>(p, f0, f1, flag[c], (y + p.G) * p.pitch + (x + kOX), r, jx, jy, e, lam, c,
                       e0, e1);
    a[0] += r; a[1] += jx; a[2] += jy; a[3] += e;
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

__global__ void __launch_bounds__(kThreads) k_audit_final(const double* partials, int nparts,
                                                          double* out4) {
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
    for (int q = 0; q < 4; ++q) out4[q] = sh[q][0];
}

// Planes i0 .. i0+cnt-1 of lattice k's interior to / from a plane-major array
// of full populations f = s + W.
template <class S, class R>
__global__ void k_pack(const Params<R> p, int k, int i0, int cnt, const S* f, double* out,
                       int unpack, S* fw, const double* in) {
  const LatTab<R>& L = p.lat[k];
  const long long ncell = (long long)p.nx * p.ny;
  const long long total = ncell * cnt;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = i0 + (int)(t / ncell);
    const double Wi = (double)L.w1[i % L.n] * (double)L.w1[i / L.n];
    const long long c = t % ncell;
    const int x = (int)(c % p.nx), y = (int)(c / p.nx);
    const size_t e = (size_t)i * p.plane + (y + p.G) * p.pitch + (x + kOX);
    if (unpack)
      fw[e] = to_s<S, R>((R)(in[t] - Wi), L.isc[i]);
    else
      out[t] = (double)from_s<R>(f[e], L.sc[i]) + Wi;
  }
}

template <class R>
dim3 tile_grid(const Params<R>& p) {
  return dim3((p.nx + kTX - 1) / kTX, (p.ny + kTY - 1) / kTY);
}

}  // namespace

int audit_parts(int nx, int ny) {
  const long long ncell = (long long)nx * ny;
  const long long b = (ncell + kThreads - 1) / kThreads;
  return (int)(b < 1024 ? b : 1024);
}

// One CTA per 32 x 8 tile: bits (1 << new flag) | 4 if the flag flipped,
// OR-reduced over the tile; thread q < 9 adds the tile's part to the work word
// of neighbour q of its 3 x 3 tile neighbourhood (lattices from all nine, the
// flip bit only to the tile itself), listing the tiles that become work.
__global__ void __launch_bounds__(kTX * kTY)
k_tile_work(int nx, int ny, int periodic_x, int periodic_y, const uint8_t* __restrict__ flag_old,
            const uint8_t* __restrict__ flag_new, uint8_t* __restrict__ mask, int* work,
            int* wlist, int* wcount, int half) {
  const int x = blockIdx.x * kTX + threadIdx.x, y = blockIdx.y * kTY + threadIdx.y;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  int bit = 0;
  if (x < nx && y < ny) {
    const long long c = x + (long long)nx * y;
    const int o = flag_old[c], n = flag_new[c];
    if (n != kFlagGap) bit = (1 << n) | (o != n ? 4 : 0);  // gap cells are no work
  }
  __shared__ int acc;
  if (tid == 0) acc = 0;
  __syncthreads();
  const int w = __reduce_or_sync(0xffffffffu, bit);
  if (threadIdx.x == 0 && w) atomicOr(&acc, w);
  __syncthreads();
  if (tid < 9) {
    const int ntx = (int)gridDim.x, nty = (int)gridDim.y;
    const int m = acc;
    if (tid == 0) mask[blockIdx.x + ntx * blockIdx.y] = (uint8_t)m;
    int tx = (int)blockIdx.x + tid % 3 - 1, ty = (int)blockIdx.y + tid / 3 - 1;
    bool ok = true;
    if (tx < 0 || tx >= ntx) {
      if (periodic_x) tx = tx < 0 ? tx + ntx : tx - ntx;
      else ok = false;
    }
    if (ty < 0 || ty >= nty) {
      if (periodic_y) ty = ty < 0 ? ty + nty : ty - nty;
      else ok = false;
    }
    const int contrib = (m & 3) | (tid == 4 ? (m & 4) : 0);
    if (ok && contrib) add_work(work, wlist, wcount, half, ntx * nty, ty * ntx + tx, contrib);
  }
}

// Source tile of every ghost cell (set-up of the post-step kernel's per-tile
// ghost lists): the same ghost rule as every ghost writer.  -1 (in no list):
// DIRICHLET ghosts (constant) and, with skip_y, the y ghost rows, which the
// stream kernel then never reads (it wraps those rows).
__global__ void k_ghost_src(int G, int nx, int ny, int periodic_x, int periodic_y, int skip_y,
                            const BcDev bc, int* __restrict__ out, int ring) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ring) return;
  int gx, gy, sx, sy, side = 0, idx = 0;
  const int kind = ghost_cell(G, nx, ny, periodic_x, periodic_y, bc, g, gx, gy, sx, sy, side, idx);
  const int ntx = (nx + kTX - 1) / kTX;
  const bool dead = skip_y && (gy < 0 || gy >= ny);
  out[g] = (kind == 2 || dead) ? -1 : (sy / kTY) * ntx + sx / kTX;
}

cudaError_t launch_ghost_src(int G, int nx, int ny, int periodic_x, int periodic_y, int skip_y,
                             const BcDev& bc, int* out, cudaStream_t st) {
  const int ring = 2 * G * (nx + 2 * G) + 2 * G * ny + bc.nwall;
  if (ring == 0) return cudaSuccess;
  k_ghost_src<<<(ring + 127) / 128, 128, 0, st>>>(G, nx, ny, periodic_x, periodic_y, skip_y, bc,
                                                  out, ring);
  return cudaGetLastError();
}

cudaError_t launch_tile_work(int nx, int ny, int periodic_x, int periodic_y,
                             const uint8_t* flag_old, const uint8_t* flag_new, uint8_t* mask,
                             int* work, int* wlist, int* wcount, int half, cudaStream_t st) {
  const dim3 grid((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY);
  k_tile_work<<<grid, dim3(kTX, kTY), 0, st>>>(nx, ny, periodic_x, periodic_y, flag_old, flag_new,
                                               mask, work, wlist, wcount, half);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_ghosts(const Params<R>& p, S* f0, S* f1, const uint8_t* flag, const BcDev& bc,
                          cudaStream_t st) {
  const long long total = 2LL * p.G * (p.nx + 2 * p.G) + 2LL * p.G * p.ny + bc.nwall;
  if (total == 0) return cudaSuccess;
  k_ghosts<S, R><<<(unsigned)((total + 127) / 128), 128, 0, st>>>(p, f0, f1, flag, bc);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_init_eq(const Params<R>& p, S* f0, S* f1, const double* rho, const double* ux,
                           const double* uy, cudaStream_t st) {
  k_init_eq<S, R><<<tile_grid(p), dim3(kTX, kTY), 0, st>>>(p, f0, f1, rho, ux, uy);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_moments(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                           double* rho, double* ux, double* uy, double* T, const S* lam,
                           cudaStream_t st, const S* e0, const S* e1) {
  k_moments<S, R><<<tile_grid(p), dim3(kTX, kTY), 0, st>>>(p, f0, f1, flag, rho, ux, uy, T, lam,
                                                           e0, e1);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_criterion(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                             uint8_t* flag_new, cudaStream_t st) {
  k_criterion<S, R><<<tile_grid(p), dim3(kTX, kTY), 0, st>>>(p, f0, f1, flag, flag_new);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_audit(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                         double* partials, int nparts, double* out4, const S* lam,
                         cudaStream_t st, const S* e0, const S* e1) {
  k_audit_partial<S, R><<<nparts, kThreads, 0, st>>>(p, f0, f1, flag, partials, lam, e0, e1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_audit_final<<<1, kThreads, 0, st>>>(partials, nparts, out4);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_pack(const Params<R>& p, int k, int i0, int cnt, const S* f, double* out,
                        int unpack, S* fw, const double* in, cudaStream_t st) {
  k_pack<S, R><<<1024, kThreads, 0, st>>>(p, k, i0, cnt, f, out, unpack, fw, in);
  return cudaGetLastError();
}

// Largest |f^L_i(rho, u) - W_i| of every plane i of both lattices over the
// cells' equilibria, into out[k * 25 + i] as float bits (nonnegative floats
// order like their bit patterns; out zeroed by the caller).
__global__ void __launch_bounds__(kThreads)
k_fx_range(const Params<float> p, const double* __restrict__ rho, const double* __restrict__ ux,
           const double* __restrict__ uy, unsigned* __restrict__ out) {
  constexpr int Q = kMaxN * kMaxN;
  float m[2][Q];
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < Q; ++i) m[k][i] = 0.f;
  const long long nc = (long long)p.nx * p.ny;
  for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < nc;
       c += (long long)gridDim.x * kThreads) {
    for (int k = 0; k < 2; ++k) {
      float e[kMaxN][kMaxN];
      const int n = p.lat[k].n;
      eq_dev<float>(p.lat[k], n, (float)(rho[c] - 1.0), (float)ux[c], (float)uy[c], e);
#pragma unroll
      for (int iy = 0; iy < kMaxN; ++iy)
#pragma unroll
        for (int ix = 0; ix < kMaxN; ++ix)
          if (iy < n && ix < n) m[k][ix + n * iy] = fmaxf(m[k][ix + n * iy], fabsf(e[iy][ix]));
    }
  }
#pragma unroll
  for (int k = 0; k < 2; ++k)
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const unsigned b = __reduce_max_sync(0xffffffffu, __float_as_uint(m[k][i]));
      if ((threadIdx.x & 31) == 0 && b) atomicMax(out + k * Q + i, b);
    }
}

cudaError_t launch_fx_range(const Params<float>& p, const double* rho, const double* ux,
                            const double* uy, unsigned* out, cudaStream_t st) {
  const long long nc = (long long)p.nx * p.ny;
  long long blocks = (nc + kThreads - 1) / kThreads;
  if (blocks > 8LL * p.nsm) blocks = 8LL * p.nsm;
  k_fx_range<<<(unsigned)(blocks > 0 ? blocks : 1), kThreads, 0, st>>>(p, rho, ux, uy, out);
  return cudaGetLastError();
}

#define SLBM_AUX_INST(S, R)                                                                  \
  template cudaError_t launch_ghosts<S, R>(const Params<R>&, S*, S*, const uint8_t*,         \
                                           const BcDev&, cudaStream_t);                      \
  template cudaError_t launch_init_eq<S, R>(const Params<R>&, S*, S*, const double*,         \
                                            const double*, const double*, cudaStream_t);     \
  template cudaError_t launch_moments<S, R>(const Params<R>&, const S*, const S*,            \
                                            const uint8_t*, double*, double*, double*,       \
                                            double*, const S*, cudaStream_t, const S*,       \
                                            const S*);                                       \
  template cudaError_t launch_criterion<S, R>(const Params<R>&, const S*, const S*,          \
                                              const uint8_t*, uint8_t*, cudaStream_t);       \
  template cudaError_t launch_audit<S, R>(const Params<R>&, const S*, const S*,              \
                                          const uint8_t*, double*, int, double*, const S*,   \
                                          cudaStream_t, const S*, const S*);                 \
  template cudaError_t launch_pack<S, R>(const Params<R>&, int, int, int, const S*, double*, \
                                         int, S*, const double*, cudaStream_t);
SLBM_AUX_INST(float, float)
SLBM_AUX_INST(double, double)
SLBM_AUX_INST(__half, float)
SLBM_AUX_INST(fx16, float)
#undef SLBM_AUX_INST

}  // namespace slbm
