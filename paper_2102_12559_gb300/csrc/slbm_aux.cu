// slbm_aux.cu -- interface conversion, ghost / boundary fill, equilibrium
// initialisation, macroscopic moments, FP64 audit and host packing kernels.
#include "slbm_impl.cuh"

#include "../../include/slbm.h"

namespace slbm {

namespace {

constexpr int kThreads = 256;

// Raw Gaussian moments h_m(u) = E[(u + Z)^m], m < 5, T = T_L = 1.
__device__ __forceinline__ void gauss_moments(double u, double* h) {
  const double u2 = u * u;
  h[0] = 1.0;
  h[1] = u;
  h[2] = 1.0 + u2;
  h[3] = u * (u2 + 3.0);
  h[4] = u2 * u2 + 6.0 * u2 + 3.0;
}

// 1-D lattice-equilibrium factors phi_j = sum_m vinv[j][m] h_m, j < n.
__device__ __forceinline__ void factors(const double (*vinv)[kMaxN], int n, const double* h,
                                        double* phi) {
  for (int j = 0; j < n; ++j) {
    double s = 0.0;
    for (int m = 0; m < n; ++m) s += vinv[j][m] * h[m];
    phi[j] = s;
  }
}

template <class S>
__device__ __forceinline__ double ld(const S* p) { return static_cast<double>(*p); }

// Lattice-frame equilibrium of lattice k (eq. feqL0) written to planes at `base`.
template <class S>
__device__ void write_eq(const ConvTab& t, int k, S* f, long long plane, int base, double rho,
                         double ux, double uy) {
  const int n = k ? t.nQ : t.nq;
  const double(*vinv)[kMaxN] = k ? t.vinvQ : t.vinvq;
  double hx[kMaxN], hy[kMaxN], px[kMaxN], py[kMaxN];
  gauss_moments(ux, hx);
  gauss_moments(uy, hy);
  factors(vinv, n, hx, px);
  factors(vinv, n, hy, py);
  for (int jy = 0; jy < n; ++jy)
    for (int jx = 0; jx < n; ++jx)
      f[(size_t)(jx + n * jy) * plane + base] = static_cast<S>(rho * py[jy] * px[jx]);
}

// Lifting f_q -> f_Q (Sec. III.B): the q x q moments are kept and the rest are
// those of the Q-lattice equilibrium at the cell's rho, u.  In tensor form the
// lifted vector is f^L_Q(rho, u) + L (f_q - f^L_q) L^T with the fixed nQ x nq
// matrix L = VQ^-1[:, :nq] Vq, which carries the non-equilibrium part with its
// moments intact and zero higher moments.  Accumulated in FP64.
template <class S>
__device__ void lift_cell(const ConvTab& t, const S* src, S* dst, long long plane, int base) {
  const int nq = t.nq, nQ = t.nQ;
  double F[kMaxN][kMaxN];
  double rho = 0.0, mx = 0.0, my = 0.0;
  for (int jy = 0; jy < nq; ++jy)
    for (int jx = 0; jx < nq; ++jx) {
      const double v = ld(src + (size_t)(jx + nq * jy) * plane + base);
      F[jy][jx] = v;
      rho += v;
      mx += t.cq[jx] * v;
      my += t.cq[jy] * v;
    }
  const double ux = mx / rho, uy = my / rho;
  double hx[kMaxN], hy[kMaxN], pqx[kMaxN], pqy[kMaxN], pQx[kMaxN], pQy[kMaxN];
  gauss_moments(ux, hx);
  gauss_moments(uy, hy);
  factors(t.vinvq, nq, hx, pqx);
  factors(t.vinvq, nq, hy, pqy);
  factors(t.vinvQ, nQ, hx, pQx);
  factors(t.vinvQ, nQ, hy, pQy);
  for (int jy = 0; jy < nq; ++jy)
    for (int jx = 0; jx < nq; ++jx) F[jy][jx] -= rho * pqy[jy] * pqx[jx];
  double A[kMaxN][kMaxN];  // A[ay][jx] = sum_jy L[ay][jy] D[jy][jx]
  for (int ay = 0; ay < nQ; ++ay)
    for (int jx = 0; jx < nq; ++jx) {
      double s = 0.0;
      for (int jy = 0; jy < nq; ++jy) s += t.lift[ay][jy] * F[jy][jx];
      A[ay][jx] = s;
    }
  for (int ay = 0; ay < nQ; ++ay)
    for (int ax = 0; ax < nQ; ++ax) {
      double s = rho * pQy[ay] * pQx[ax];
      for (int jx = 0; jx < nq; ++jx) s += t.lift[ax][jx] * A[ay][jx];
      dst[(size_t)(ax + nQ * ay) * plane + base] = static_cast<S>(s);
    }
}

// Projection f_Q -> f_q (Sec. III.C): f_q keeps the first q x q moments of f_Q;
// per axis that is Lagrange interpolation of the Q nodes onto the q nodes,
// f_q = P F_Q P^T with P[j][a] = l^q_j(c^Q_a).  Accumulated in FP64.
template <class S>
__device__ void project_cell(const ConvTab& t, const S* src, S* dst, long long plane, int base) {
  const int nq = t.nq, nQ = t.nQ;
  double F[kMaxN][kMaxN];
  for (int ay = 0; ay < nQ; ++ay)
    for (int ax = 0; ax < nQ; ++ax) F[ay][ax] = ld(src + (size_t)(ax + nQ * ay) * plane + base);
  double A[kMaxN][kMaxN];  // A[jy][ax] = sum_ay P[jy][ay] F[ay][ax]
  for (int jy = 0; jy < nq; ++jy)
    for (int ax = 0; ax < nQ; ++ax) {
      double s = 0.0;
      for (int ay = 0; ay < nQ; ++ay) s += t.proj[jy][ay] * F[ay][ax];
      A[jy][ax] = s;
    }
  for (int jy = 0; jy < nq; ++jy)
    for (int jx = 0; jx < nq; ++jx) {
      double s = 0.0;
      for (int ax = 0; ax < nQ; ++ax) s += t.proj[jx][ax] * A[jy][ax];
      dst[(size_t)(jx + nq * jy) * plane + base] = static_cast<S>(s);
    }
}

__device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Interface conversion (step 2 of Sec. III.D, done once per node per step).
// A cell needs its other-lattice representation when a cell of the other
// lattice lies within the stencil reach (band), and a cell whose flag changed
// needs its new lattice.  Both are "convert from the lattice the cell was
// computed in (flag_old) to the other one".
template <class S>
__global__ void __launch_bounds__(kTX * kTY)
k_convert(const Params<double> p, S* f0, S* f1, const uint8_t* __restrict__ flag_old,
          const uint8_t* __restrict__ flag_new) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = x + p.nx * y;
  const int old = flag_old[c], nw = flag_new[c];
  bool need = old != nw;
  for (int dy = -p.band; dy <= p.band && !need; ++dy) {
    int yy = y + dy;
    if (yy < 0 || yy >= p.ny) {
      if (!p.periodic_y) continue;
      yy = wrap(yy, p.ny);
    }
    for (int dx = -p.band; dx <= p.band; ++dx) {
      int xx = x + dx;
      if (xx < 0 || xx >= p.nx) {
        if (!p.periodic_x) continue;
        xx = wrap(xx, p.nx);
      }
      if (flag_new[xx + p.nx * yy] != nw) { need = true; break; }
    }
  }
  if (!need) return;
  const int base = (y + p.G) * p.pitch + (x + kOX);
  if (old == 0)
    lift_cell<S>(p.conv, f0, f1, p.plane, base);
  else
    project_cell<S>(p.conv, f1, f0, p.plane, base);
}

template <class S>
__device__ double cell_rho(const Params<double>& p, const S* f0, const S* f1,
                           const uint8_t* flag, int x, int y) {
  const int k = flag[x + p.nx * y];
  const int Q = k ? p.conv.nQ * p.conv.nQ : p.conv.nq * p.conv.nq;
  const S* f = k ? f1 : f0;
  const int base = (y + p.G) * p.pitch + (x + kOX);
  double r = 0.0;
  for (int i = 0; i < Q; ++i) r += ld(f + (size_t)i * p.plane + base);
  return r;
}

// Ghost ring: periodic images, or the boundary state of a non-periodic side
// in both lattices (OUTFLOW copies the nearest interior cell, DIRICHLET /
// INLET write the lattice equilibrium).  A non-periodic y side wins at corners.
template <class S>
__global__ void k_ghosts(const Params<double> p, S* f0, S* f1, const uint8_t* __restrict__ flag,
                         const BcDev bc) {
  const int G = p.G, W = p.nx + 2 * G;
  const long long nstrip = (long long)G * W;
  const long long total = 2 * nstrip + 2LL * G * p.ny;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  int gx, gy;
  if (idx < nstrip) {
    gy = -G + (int)(idx / W); gx = -G + (int)(idx % W);
  } else if (idx < 2 * nstrip) {
    const long long j = idx - nstrip;
    gy = p.ny + (int)(j / W); gx = -G + (int)(j % W);
  } else if (idx < 2 * nstrip + (long long)G * p.ny) {
    const long long j = idx - 2 * nstrip;
    gy = (int)(j / G); gx = -G + (int)(j % G);
  } else {
    const long long j = idx - 2 * nstrip - (long long)G * p.ny;
    gy = (int)(j / G); gx = p.nx + (int)(j % G);
  }
  int sx = gx, sy = gy;
  bool eq = false;
  double er = 1.0, eu = 0.0, ev = 0.0;
  if (sy < 0 || sy >= p.ny) {
    if (p.periodic_y) {
      sy = wrap(sy, p.ny);
    } else {
      const int side = sy < 0 ? SLBM_SIDE_YMIN : SLBM_SIDE_YMAX;
      const int xi = min(max(sx, 0), p.nx - 1), yi = sy < 0 ? 0 : p.ny - 1;
      const int kind = bc.kind[side];
      if (kind == SLBM_BC_OUTFLOW) {
        sy = yi;
      } else {
        eq = true;
        er = kind == SLBM_BC_INLET ? cell_rho<S>(p, f0, f1, flag, xi, yi) : bc.rho[side][xi];
        eu = bc.ux[side][xi];
        ev = bc.uy[side][xi];
      }
    }
  }
  if (!eq && (sx < 0 || sx >= p.nx)) {
    if (p.periodic_x) {
      sx = wrap(sx, p.nx);
    } else {
      const int side = sx < 0 ? SLBM_SIDE_XMIN : SLBM_SIDE_XMAX;
      const int xi = sx < 0 ? 0 : p.nx - 1;
      const int kind = bc.kind[side];
      if (kind == SLBM_BC_OUTFLOW) {
        sx = xi;
      } else {
        eq = true;
        er = kind == SLBM_BC_INLET ? cell_rho<S>(p, f0, f1, flag, xi, sy) : bc.rho[side][sy];
        eu = bc.ux[side][sy];
        ev = bc.uy[side][sy];
      }
    }
  }
  const int gbase = (gy + G) * p.pitch + (gx + kOX);
  if (eq) {
    write_eq<S>(p.conv, 0, f0, p.plane, gbase, er, eu, ev);
    write_eq<S>(p.conv, 1, f1, p.plane, gbase, er, eu, ev);
  } else {
    const int sbase = (sy + G) * p.pitch + (sx + kOX);
    const int q0 = p.conv.nq * p.conv.nq, q1 = p.conv.nQ * p.conv.nQ;
    for (int i = 0; i < q0; ++i) f0[(size_t)i * p.plane + gbase] = f0[(size_t)i * p.plane + sbase];
    for (int i = 0; i < q1; ++i) f1[(size_t)i * p.plane + gbase] = f1[(size_t)i * p.plane + sbase];
  }
}

template <class S>
__global__ void __launch_bounds__(kTX * kTY)
k_init_eq(const Params<double> p, S* f0, S* f1, const double* __restrict__ rho,
          const double* __restrict__ ux, const double* __restrict__ uy) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = x + p.nx * y;
  const int base = (y + p.G) * p.pitch + (x + kOX);
  write_eq<S>(p.conv, 0, f0, p.plane, base, rho[c], ux[c], uy[c]);
  write_eq<S>(p.conv, 1, f1, p.plane, base, rho[c], ux[c], uy[c]);
}

// Per-cell rho, u, kinetic T and (for the audit) momentum and energy sums.
template <class S>
__device__ void cell_moments(const Params<double>& p, const S* f0, const S* f1, int k, int base,
                             double& r, double& jx, double& jy, double& e) {
  const int n = k ? p.conv.nQ : p.conv.nq;
  const double* c = k ? p.conv.cQ : p.conv.cq;
  const S* f = k ? f1 : f0;
  r = jx = jy = e = 0.0;
  for (int iy = 0; iy < n; ++iy)
    for (int ix = 0; ix < n; ++ix) {
      const double v = ld(f + (size_t)(ix + n * iy) * p.plane + base);
      r += v;
      jx += c[ix] * v;
      jy += c[iy] * v;
      e += 0.5 * (c[ix] * c[ix] + c[iy] * c[iy]) * v;
    }
}

template <class S>
__global__ void __launch_bounds__(kTX * kTY)
k_moments(const Params<double> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
          double* rho, double* ux, double* uy, double* T) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = x + p.nx * y;
  const int base = (y + p.G) * p.pitch + (x + kOX);
  double r, jx, jy, e;
  cell_moments<S>(p, f0, f1, flag[c], base, r, jx, jy, e);
  const double u = jx / r, v = jy / r;
  if (rho) rho[c] = r;
  if (ux) ux[c] = u;
  if (uy) uy[c] = v;
  if (T) T[c] = (2.0 * e / r - u * u - v * v) / 2.0;
}

// Mach criterion of Sec. IV.A on the current state (flag = |u| > thr, c_s = 1).
template <class S>
__global__ void __launch_bounds__(kTX * kTY)
k_criterion(const Params<double> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
            uint8_t* __restrict__ flag_new) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int c = x + p.nx * y;
  const int base = (y + p.G) * p.pitch + (x + kOX);
  double r, jx, jy, e;
  cell_moments<S>(p, f0, f1, flag[c], base, r, jx, jy, e);
  const double u = jx / r, v = jy / r;
  flag_new[c] = sqrt(u * u + v * v) > p.thr ? 1 : 0;
}

// FP64 conservation audit: per-block partial sums, then one block adds the
// partials in a fixed order (deterministic result).
template <class S>
__global__ void __launch_bounds__(kThreads)
k_audit_partial(const Params<double> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
                double* partials) {
  __shared__ double sh[4][kThreads];
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  const long long ncell = (long long)p.nx * p.ny;
  for (long long c = (long long)blockIdx.x * kThreads + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * kThreads) {
    const int x = (int)(c % p.nx), y = (int)(c / p.nx);
    const int base = (y + p.G) * p.pitch + (x + kOX);
    double r, jx, jy, e;
    cell_moments<S>(p, f0, f1, flag[c], base, r, jx, jy, e);
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

// Copy planes i0 .. i0+cnt-1 of one lattice's interior to / from a
// plane-major double array.
template <class S>
__global__ void k_pack(const Params<double> p, int i0, int cnt, const S* f, double* out,
                       int unpack, S* fw, const double* in) {
  const long long ncell = (long long)p.nx * p.ny;
  const long long total = ncell * cnt;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = i0 + (int)(t / ncell);
    const long long c = t % ncell;
    const int x = (int)(c % p.nx), y = (int)(c / p.nx);
    const size_t e = (size_t)i * p.plane + (y + p.G) * p.pitch + (x + kOX);
    if (unpack)
      fw[e] = static_cast<S>(in[t]);
    else
      out[t] = static_cast<double>(f[e]);
  }
}

dim3 tile_grid(const Params<double>& p) {
  return dim3((p.nx + kTX - 1) / kTX, (p.ny + kTY - 1) / kTY);
}

}  // namespace

int audit_parts(const Params<double>& p) {
  const long long ncell = (long long)p.nx * p.ny;
  long long b = (ncell + kThreads - 1) / kThreads;
  return (int)(b < 1024 ? b : 1024);
}

template <class S>
cudaError_t launch_convert(const Params<double>& pd, S* f0, S* f1, const uint8_t* flag_old,
                           const uint8_t* flag_new, cudaStream_t st) {
  k_convert<S><<<tile_grid(pd), dim3(kTX, kTY), 0, st>>>(pd, f0, f1, flag_old, flag_new);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_ghosts(const Params<double>& pd, S* f0, S* f1, const uint8_t* flag,
                          const BcDev& bc, cudaStream_t st) {
  const long long total = 2LL * pd.G * (pd.nx + 2 * pd.G) + 2LL * pd.G * pd.ny;
  if (total == 0) return cudaSuccess;
  k_ghosts<S><<<(unsigned)((total + kThreads - 1) / kThreads), kThreads, 0, st>>>(pd, f0, f1,
                                                                                  flag, bc);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_init_eq(const Params<double>& pd, S* f0, S* f1, const double* rho,
                           const double* ux, const double* uy, cudaStream_t st) {
  k_init_eq<S><<<tile_grid(pd), dim3(kTX, kTY), 0, st>>>(pd, f0, f1, rho, ux, uy);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_moments(const Params<double>& pd, const S* f0, const S* f1,
                           const uint8_t* flag, double* rho, double* ux, double* uy, double* T,
                           cudaStream_t st) {
  k_moments<S><<<tile_grid(pd), dim3(kTX, kTY), 0, st>>>(pd, f0, f1, flag, rho, ux, uy, T);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_criterion(const Params<double>& pd, const S* f0, const S* f1,
                             const uint8_t* flag, uint8_t* flag_new, cudaStream_t st) {
  k_criterion<S><<<tile_grid(pd), dim3(kTX, kTY), 0, st>>>(pd, f0, f1, flag, flag_new);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_audit(const Params<double>& pd, const S* f0, const S* f1, const uint8_t* flag,
                         double* partials, int nparts, double* out4, cudaStream_t st) {
  k_audit_partial<S><<<nparts, kThreads, 0, st>>>(pd, f0, f1, flag, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_audit_final<<<1, kThreads, 0, st>>>(partials, nparts, out4);
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_pack(const Params<double>& pd, int i0, int cnt, const S* f, double* out,
                        int unpack, S* fw, const double* in, cudaStream_t st) {
  k_pack<S><<<1024, kThreads, 0, st>>>(pd, i0, cnt, f, out, unpack, fw, in);
  return cudaGetLastError();
}

#define SLBM_AUX_INST(S)                                                                     \
  template cudaError_t launch_convert<S>(const Params<double>&, S*, S*, const uint8_t*,      \
                                         const uint8_t*, cudaStream_t);                      \
  template cudaError_t launch_ghosts<S>(const Params<double>&, S*, S*, const uint8_t*,       \
                                        const BcDev&, cudaStream_t);                         \
  template cudaError_t launch_init_eq<S>(const Params<double>&, S*, S*, const double*,       \
                                         const double*, const double*, cudaStream_t);        \
  template cudaError_t launch_moments<S>(const Params<double>&, const S*, const S*,          \
                                         const uint8_t*, double*, double*, double*, double*, \
                                         cudaStream_t);                                      \
  template cudaError_t launch_criterion<S>(const Params<double>&, const S*, const S*,       \
                                           const uint8_t*, uint8_t*, cudaStream_t);          \
  template cudaError_t launch_audit<S>(const Params<double>&, const S*, const S*,            \
                                       const uint8_t*, double*, int, double*, cudaStream_t); \
  template cudaError_t launch_pack<S>(const Params<double>&, int, int, const S*, double*, int, \
                                      S*, const double*, cudaStream_t);
SLBM_AUX_INST(float)
SLBM_AUX_INST(double)
#undef SLBM_AUX_INST

}  // namespace slbm
