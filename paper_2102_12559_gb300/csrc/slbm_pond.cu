// slbm_pond.cu -- the co-moving (PonD) frame of Sec. II.C on sm_103a.
//
// Every cell keeps its populations in its own frame lambda = {u, T}, with
// particle velocities v_i = sqrt(theta) c_i + u, theta = T / T_L (eq. vi).
// One cell update (one thread):
//   predictor  lambda_0 = the cell's frame of the previous step;
//   repeat     reconstruct every population at x - v_i dt (eq. advectionPond)
//              from the collocation nodes, each node's vector first carried
//              into the target frame by the transfer matrix of eq. (fll);
//              the moments of the result (eqs. correctorfieldsrho-u) are the
//              next frame, until they agree with the one used to tol;
//   collide    BGK (eq. Pond_f_equation, omega_1 = omega_2) towards the
//              equilibrium at those moments, expressed in the frame used
//              (rho W_i itself once converged, eq. feqPond).
//
// Transfer between frames in tensor form.  For one axis, the populations in
// frame lambda that reproduce the moments of order < n of a node's
// populations in frame lambda_s are G[a][j] = l_a(xi_j): the Lagrange basis
// polynomial of the target's nodes evaluated at the source's nodes.  In the
// target's units, xi_j = r c_j + d with r = sqrt(T_s / T) and
// d = (u_s - u) / sqrt(T); the 2-D transfer is G_x (x) G_y.
//
// Deviation form.  Stored values are s_i = f_i - W_i.  A node's vector in the
// target frame is G s_s + G W; G W is the rest-state equilibrium of the node
// (rho = 1, u_s, T_s) seen from the target frame, i.e. the product
// phi_a(d_x, r^2) phi_b(d_y, r^2) of the 1-D equilibria at relative velocity d
// and temperature r^2, so G W - W follows from the small differences
// dphi = phi - w without cancellation.  The equilibria use the raw Gaussian
// moments h_m(u, T) of N(u, T), orders < n.
//
// Wrapping: the grid is periodic and departure points may move several cells
// (|v| dt grows with u and T), so node indices wrap with a modulo instead of
// reading a ghost ring.
#include "../../include/slbm.h"
#include "slbm_impl.cuh"

namespace slbm {

namespace {

constexpr int kThreads = kTX * kTY;

__device__ __forceinline__ int wrapm(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// h_m(u, T) - h_m(0, 1) for m < 5: raw moments of N(u, T) minus those of the
// rest state.
template <class R>
__device__ __forceinline__ void gauss_dev_t(R u, R dT, R* dh) {
  const R T = R(1) + dT;
  const R u2 = u * u;
  dh[0] = R(0);
  dh[1] = u;
  dh[2] = u2 + dT;
  dh[3] = u * (u2 + R(3) * T);
  dh[4] = u2 * (u2 + R(6) * T) + R(3) * dT * (R(2) + dT);
}

// dphi_a = phi_a(u, 1 + dT) - w_a, a < N.
template <int N, class R>
__device__ __forceinline__ void dphi_t(const PondLat<R>& L, R u, R dT, R* d) {
  R dh[kMaxN];
  gauss_dev_t<R>(u, dT, dh);
#pragma unroll
  for (int a = 0; a < N; ++a) {
    R s = R(0);
#pragma unroll
    for (int m = 1; m < N; ++m) s += L.vinv[a][m] * dh[m];
    d[a] = s;
  }
}

// One component of dphi_t.
template <int N, class R>
__device__ __forceinline__ R dphi1(const PondLat<R>& L, int a, R u, R dT) {
  R dh[kMaxN];
  gauss_dev_t<R>(u, dT, dh);
  R s = R(0);
#pragma unroll
  for (int m = 1; m < N; ++m) s += L.vinv[a][m] * dh[m];
  return s;
}

// Lagrange basis polynomial a of the lattice's 1-D nodes, at xi.
template <int N, class R>
__device__ __forceinline__ R basis(const PondLat<R>& L, int a, R xi) {
  R v = R(1);
#pragma unroll
  for (int m = 0; m < N; ++m)
    if (m != a) v *= (xi - L.c[m]) * L.inv[a][m];
  return v;
}

// Lagrange interpolation functions on P equispaced points x0 .. x0+P-1 at xd
// (first point floor(xd - (P-1)/2 + 1/2), ties rounding up).
template <class R>
__device__ __forceinline__ int stencil(int P, R xd, R* a) {
  const int x0 = (int)floor(xd - R(0.5) * (R)(P - 1) + R(0.5));
#pragma unroll
  for (int s = 0; s < kMaxP; ++s) {
    if (s >= P) break;
    R v = R(1);
#pragma unroll
    for (int r = 0; r < kMaxP; ++r) {
      if (r >= P) break;
      if (r != s) v *= (xd - (R)(x0 + r)) / (R)(s - r);
    }
    a[s] = v;
  }
  return x0;
}

// One co-moving update of cell (x, y) whose populations (and those of every
// collocation node it reads) are in lattice L with N nodes per axis.
template <int N, class S, class R>
__device__ void pond_cell(const PondParams<R>& p, const PondLat<R>& L, const S* __restrict__ f,
                          const S* __restrict__ lam, S* __restrict__ g, S* __restrict__ lam_out,
                          int x, int y, int* err) {
  const long long c = (long long)x + (long long)p.nx * y;
  R ux = (R)lam[c], uy = (R)lam[p.nc + c], T = (R)lam[2 * p.nc + c];
  R d[N][N];                    // reconstructed deviations, [b][a]
  for (int b = 0; b < N; ++b)
    for (int a = 0; a < N; ++a) d[b][a] = R(0);
  R dr = R(0), s1x = R(0), s1y = R(0), dT = R(0);
  bool ok = true, conv = false;
  for (int it = 0; it < p.maxit; ++it) {
    if (!(T > R(0)) || !isfinite(ux) || !isfinite(uy)) { ok = false; break; }
    const R st = sqrt(T), ist = R(1) / st;
#pragma unroll 1
    for (int b = 0; b < N; ++b) {
      const R vy = st * L.c[b] + uy;
      if (fabs(vy * p.dt) > p.reach) ok = false;
      R ay[kMaxP];
      const int y0 = stencil<R>(p.P, (R)y - vy * p.dt, ay);
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        const R vx = st * L.c[a] + ux;
        if (fabs(vx * p.dt) > p.reach) ok = false;
        R ax[kMaxP];
        const int x0 = stencil<R>(p.P, (R)x - vx * p.dt, ax);
        R acc = R(0);
#pragma unroll 1
        for (int t = 0; t < p.P; ++t) {
          const int yi = wrapm(y0 + t, p.ny);
          R acc_t = R(0);
#pragma unroll 1
          for (int u = 0; u < p.P; ++u) {
            const int xi = wrapm(x0 + u, p.nx);
            const long long cs = (long long)xi + (long long)p.nx * yi;
            const R sux = (R)lam[cs], suy = (R)lam[p.nc + cs], sT = (R)lam[2 * p.nc + cs];
            const R r = sqrt(sT) * ist;
            const R dx = (sux - ux) * ist, dy = (suy - uy) * ist;
            const R dTs = (sT - T) / T;                   // r^2 - 1
            R gx[N], gy[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
              gx[j] = basis<N, R>(L, a, r * L.c[j] + dx);
              gy[j] = basis<N, R>(L, b, r * L.c[j] + dy);
            }
            // G s_s
            const size_t base = (size_t)(yi + p.G) * p.pitch + (xi + kOX);
            R v = R(0);
#pragma unroll
            for (int k = 0; k < N; ++k) {
              R row = R(0);
#pragma unroll
              for (int j = 0; j < N; ++j) row += gx[j] * (R)f[(size_t)(j + N * k) * p.plane + base];
              v += gy[k] * row;
            }
            // G W - W
            const R pxa = dphi1<N, R>(L, a, dx, dTs), pyb = dphi1<N, R>(L, b, dy, dTs);
            v += L.w[a] * pyb + pxa * L.w[b] + pxa * pyb;
            acc_t += ax[u] * v;
          }
          acc += ay[t] * acc_t;
        }
        d[b][a] = acc;
      }
    }
    // moments in the frame used: rho = 1 + sum d, relative velocity S1 / rho,
    // relative temperature 1 + dT (sum W c^2 = 1 per axis)
    R s0 = R(0), sx = R(0), sy = R(0), s2 = R(0);
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const R v = d[b][a];
        s0 += v;
        sx += L.c[a] * v;
        sy += L.c[b] * v;
        s2 += (L.c[a] * L.c[a] + L.c[b] * L.c[b] - R(2)) * v;
      }
    dr = s0;
    const R rho = R(1) + s0;
    s1x = sx / rho;
    s1y = sy / rho;
    dT = p.thermal ? (s2 - rho * (s1x * s1x + s1y * s1y)) / (R(2) * rho) : R(0);
    const R dux = st * s1x, duy = st * s1y, dTabs = T * dT;
    const R diff = fmax(fabs(dux), fmax(fabs(duy), fabs(dTabs)));
    if (!(diff == diff)) { ok = false; break; }
    if (diff <= p.tol) { conv = true; break; }
    if (it + 1 < p.maxit) {
      ux += dux;
      uy += duy;
      T += dTabs;
    }
  }
  if (!ok) atomicOr(err, kErrFrame);
  else if (!conv) atomicOr(err, kErrNoConv);
  // BGK towards the equilibrium at (rho, relative velocity s1, relative
  // temperature 1 + dT), in the frame used
  R ex[N], ey[N];
  dphi_t<N, R>(L, s1x, dT, ex);
  dphi_t<N, R>(L, s1y, dT, ey);
  const size_t base = (size_t)(y + p.G) * p.pitch + (x + kOX);
#pragma unroll
  for (int b = 0; b < N; ++b)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const R pa = L.w[a] + ex[a], pb = L.w[b] + ey[b];
      const R eq = dr * pa * pb + L.w[a] * ey[b] + ex[a] * L.w[b] + ex[a] * ey[b];
      g[(size_t)(a + N * b) * p.plane + base] = (S)(d[b][a] + p.omega * (eq - d[b][a]));
    }
  lam_out[c] = (S)ux;
  lam_out[p.nc + c] = (S)uy;
  lam_out[2 * p.nc + c] = (S)T;
}

template <int NL, int NH, class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_step(const PondParams<R> p, const S* __restrict__ f0, const S* __restrict__ f1,
            const S* __restrict__ lam, S* __restrict__ g0, S* __restrict__ g1,
            S* __restrict__ lam_out, const uint8_t* __restrict__ flag, int* err) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  if (flag[(long long)x + (long long)p.nx * y])
    pond_cell<NH, S, R>(p, p.lat[1], f1, lam, g1, lam_out, x, y, err);
  else
    pond_cell<NL, S, R>(p, p.lat[0], f0, lam, g0, lam_out, x, y, err);
}

// Rest-frame equilibrium of both lattices (s = (rho - 1) W_i) and the frame.
template <class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_init(const PondParams<R> p, S* f0, S* f1, S* lam, const double* __restrict__ rho,
            const double* __restrict__ ux, const double* __restrict__ uy,
            const double* __restrict__ T) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long c = (long long)x + (long long)p.nx * y;
  const size_t base = (size_t)(y + p.G) * p.pitch + (x + kOX);
  const double dr = rho[c] - 1.0;
  for (int k = 0; k < 2; ++k) {
    const PondLat<R>& L = p.lat[k];
    S* f = k ? f1 : f0;
    for (int b = 0; b < L.n; ++b)
      for (int a = 0; a < L.n; ++a)
        f[(size_t)(a + L.n * b) * p.plane + base] = (S)(dr * (double)L.w[a] * (double)L.w[b]);
  }
  lam[c] = (S)ux[c];
  lam[p.nc + c] = (S)uy[c];
  lam[2 * p.nc + c] = (S)(T ? T[c] : 1.0);
}

// Per 32 x 8 tile: bit 0 = a low-order cell, bit 1 = a high-order cell.
__global__ void __launch_bounds__(kThreads)
k_pond_masks(int nx, int ny, const uint8_t* __restrict__ flag, uint8_t* __restrict__ mask) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  const bool in = x < nx && y < ny;
  const int bit = in ? (flag[(long long)x + (long long)nx * y] ? 2 : 1) : 0;
  __shared__ int acc;
  if (threadIdx.x == 0 && threadIdx.y == 0) acc = 0;
  __syncthreads();
  const int w = __reduce_or_sync(0xffffffffu, bit);
  if (threadIdx.x == 0 && w) atomicOr(&acc, w);
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) mask[blockIdx.x + gridDim.x * blockIdx.y] = (uint8_t)acc;
}

// Lifting matrix of one axis in the frame {u, T = s^2} (Sec. III.B, App. C).
// The lift keeps the raw moments sum v^m f (v = s c + u, the frame's particle
// velocities, eq. momf) of orders < nq and takes the others from the
// equilibrium, so per axis f_Q - f^eq_Q = Lm (f_q - f^eq_q) with
// Lm = M_Q^-1[:, :nq] M_q in the frame's raw-moment matrices:
// Lm[A][j] = sum_{m < nq} coef_A[m] v_j^m, where coef_A are the monomial
// coefficients (in v) of the Q-lattice Lagrange basis polynomial
// l_A((v - u) / s).  At u = 0 this is the lattice-frame L.  FP64: the
// expansion in powers of v cancels for large |u|.
template <int NQ, int NQQ, class R>
__device__ void lift_matrix(const PondLat<R>& Lq, const PondLat<R>& LQ, double s, double u,
                            R (*Lm)[NQ]) {
  double binom[NQQ][NQQ];
#pragma unroll
  for (int k = 0; k < NQQ; ++k)
#pragma unroll
    for (int m = 0; m < NQQ; ++m)
      binom[k][m] = (m == 0 || m == k) ? 1.0 : (m > k ? 0.0 : binom[k - 1][m - 1] + binom[k - 1][m]);
  const double is = 1.0 / s;
  double pis[NQQ], pu[NQQ];      // s^-k, (-u)^k
  pis[0] = 1.0;
  pu[0] = 1.0;
#pragma unroll
  for (int k = 1; k < NQQ; ++k) {
    pis[k] = pis[k - 1] * is;
    pu[k] = pu[k - 1] * (-u);
  }
#pragma unroll
  for (int A = 0; A < NQQ; ++A) {
    double coef[NQ];
#pragma unroll
    for (int m = 0; m < NQ; ++m) {
      double acc = 0.0;
#pragma unroll
      for (int k = m; k < NQQ; ++k) acc += (double)LQ.vinv[A][k] * pis[k] * binom[k][m] * pu[k - m];
      coef[m] = acc;
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const double v = s * (double)Lq.c[j] + u;
      double acc = 0.0, vm = 1.0;
#pragma unroll
      for (int m = 0; m < NQ; ++m) {
        acc += coef[m] * vm;
        vm *= v;
      }
      Lm[A][j] = (R)acc;
    }
  }
}

// Lift q -> Q (flag 0) or project Q -> q (flag 1) of one cell in its own
// frame (Sec. III.B-C, App. C).  Projection keeps the moments of orders < nq,
// a set the change of velocity variable v = s c + u maps onto itself, so it
// is the lattice-frame P F P^T.  Lifting uses the frame's lifting matrices;
// its completing equilibrium is taken at the vector's own relative velocity
// and temperature (T_L when isothermal).
template <int NQ, int NQQ, class S, class R>
__device__ void pond_convert_cell(const PondParams<R>& p, S* f0, S* f1, int k, size_t base,
                                  const S* lam, long long c) {
  const PondLat<R>& Lq = p.lat[0];
  const PondLat<R>& LQ = p.lat[1];
  if (k == 0) {
    R s[NQ][NQ];
    double m0 = 0.0, mx = 0.0, my = 0.0, m2 = 0.0;
#pragma unroll
    for (int b = 0; b < NQ; ++b)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        const R v = (R)f0[(size_t)(a + NQ * b) * p.plane + base];
        s[b][a] = v;
        m0 += (double)v;
        mx += (double)Lq.c[a] * (double)v;
        my += (double)Lq.c[b] * (double)v;
        m2 += ((double)Lq.c[a] * (double)Lq.c[a] + (double)Lq.c[b] * (double)Lq.c[b] - 2.0) *
              (double)v;
      }
    const double rho = 1.0 + m0;
    const R ux = (R)(mx / rho), uy = (R)(my / rho);
    const R dT = p.thermal ? (R)((m2 - rho * ((mx / rho) * (mx / rho) + (my / rho) * (my / rho))) /
                                 (2.0 * rho))
                           : R(0);
    const R dr = (R)m0;
    R qx[NQ], qy[NQ], Qx[NQQ], Qy[NQQ];
    dphi_t<NQ, R>(Lq, ux, dT, qx);
    dphi_t<NQ, R>(Lq, uy, dT, qy);
    dphi_t<NQQ, R>(LQ, ux, dT, Qx);
    dphi_t<NQQ, R>(LQ, uy, dT, Qy);
    // non-equilibrium part of the q vector
#pragma unroll
    for (int b = 0; b < NQ; ++b)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        const R pa = Lq.w[a] + qx[a], pb = Lq.w[b] + qy[b];
        s[b][a] -= dr * pa * pb + Lq.w[a] * qy[b] + qx[a] * Lq.w[b] + qx[a] * qy[b];
      }
    // L_x (f_q - f^eq_q) L_y^T + f^eq_Q
    const double sq = sqrt((double)lam[2 * p.nc + c]);
    R Lx[NQQ][NQ], Ly[NQQ][NQ];
    lift_matrix<NQ, NQQ, R>(Lq, LQ, sq, (double)lam[c], Lx);
    lift_matrix<NQ, NQQ, R>(Lq, LQ, sq, (double)lam[p.nc + c], Ly);
    R t[NQ][NQQ];
#pragma unroll
    for (int b = 0; b < NQ; ++b)
#pragma unroll
      for (int A = 0; A < NQQ; ++A) {
        R v = R(0);
#pragma unroll
        for (int a = 0; a < NQ; ++a) v += Lx[A][a] * s[b][a];
        t[b][A] = v;
      }
#pragma unroll
    for (int B = 0; B < NQQ; ++B)
#pragma unroll
      for (int A = 0; A < NQQ; ++A) {
        R v = R(0);
#pragma unroll
        for (int b = 0; b < NQ; ++b) v += Ly[B][b] * t[b][A];
        const R pa = LQ.w[A] + Qx[A], pb = LQ.w[B] + Qy[B];
        v += dr * pa * pb + LQ.w[A] * Qy[B] + Qx[A] * LQ.w[B] + Qx[A] * Qy[B];
        f1[(size_t)(A + NQQ * B) * p.plane + base] = (S)v;
      }
  } else {
    // P s_Q P^T (P W_Q P^T = W_q: projection keeps the moments of order < nq)
    R t[NQQ][NQ];
#pragma unroll
    for (int B = 0; B < NQQ; ++B)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        R v = R(0);
#pragma unroll
        for (int A = 0; A < NQQ; ++A)
          v += p.proj[a][A] * (R)f1[(size_t)(A + NQQ * B) * p.plane + base];
        t[B][a] = v;
      }
#pragma unroll
    for (int b = 0; b < NQ; ++b)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        R v = R(0);
#pragma unroll
        for (int B = 0; B < NQQ; ++B) v += p.proj[b][B] * t[B][a];
        f0[(size_t)(a + NQ * b) * p.plane + base] = (S)v;
      }
  }
}

template <int NQ, int NQQ, class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_convert(const PondParams<R> p, S* f0, S* f1, const S* __restrict__ lam,
               const uint8_t* __restrict__ flag, const uint8_t* __restrict__ mask) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (mask) {
    // 3 x 3 tile neighbourhood (periodic) must hold both lattices
    const int tx = blockIdx.x, ty = blockIdx.y, ntx = gridDim.x, nty = gridDim.y;
    int bits = 0;
    for (int j = -1; j <= 1; ++j)
      for (int i = -1; i <= 1; ++i)
        bits |= mask[wrapm(tx + i, ntx) + ntx * wrapm(ty + j, nty)];
    if (bits != 3) return;
  }
  if (x >= p.nx || y >= p.ny) return;
  const long long c = (long long)x + (long long)p.nx * y;
  const int k = flag[c] ? 1 : 0;
  pond_convert_cell<NQ, NQQ, S, R>(p, f0, f1, k, (size_t)(y + p.G) * p.pitch + (x + kOX), lam, c);
}

template <class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_frame_io(const PondParams<R> p, S* lam, double* ux, double* uy, double* T, int unpack) {
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (c >= p.nc) return;
  double* h[3] = {ux, uy, T};
  for (int q = 0; q < 3; ++q) {
    if (unpack) lam[q * p.nc + c] = (S)h[q][c];
    else h[q][c] = (double)lam[q * p.nc + c];
  }
}

dim3 tile_grid(int nx, int ny) { return dim3((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY); }

template <int NL, int NH, class S, class R>
cudaError_t step_pair(const PondParams<R>& p, const S* f0, const S* f1, const S* lam, S* g0, S* g1,
                      S* lam_out, const uint8_t* flag, int* err, cudaStream_t st) {
  k_pond_step<NL, NH, S, R><<<tile_grid(p.nx, p.ny), dim3(kTX, kTY), 0, st>>>(
      p, f0, f1, lam, g0, g1, lam_out, flag, err);
  return cudaGetLastError();
}

template <int NL, int NH, class S, class R>
cudaError_t convert_pair(const PondParams<R>& p, S* f0, S* f1, const S* lam, const uint8_t* flag,
                         const uint8_t* mask, cudaStream_t st) {
  k_pond_convert<NL, NH, S, R><<<tile_grid(p.nx, p.ny), dim3(kTX, kTY), 0, st>>>(p, f0, f1, lam,
                                                                                 flag, mask);
  return cudaGetLastError();
}

}  // namespace

template <class S, class R>
cudaError_t launch_pond_init(const PondParams<R>& p, S* f0, S* f1, S* lam, const double* rho,
                             const double* ux, const double* uy, const double* T,
                             cudaStream_t st) {
  k_pond_init<S, R><<<tile_grid(p.nx, p.ny), dim3(kTX, kTY), 0, st>>>(p, f0, f1, lam, rho, ux, uy,
                                                                      T);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_pond_step(const PondParams<R>& p, const S* f0, const S* f1, const S* lam,
                             S* g0, S* g1, S* lam_out, const uint8_t* flag, int* err,
                             cudaStream_t st) {
  const int lo = p.lat[0].n, hi = p.lat[1].n;
  if (lo == 3 && hi == 4) return step_pair<3, 4, S, R>(p, f0, f1, lam, g0, g1, lam_out, flag, err, st);
  if (lo == 3 && hi == 5) return step_pair<3, 5, S, R>(p, f0, f1, lam, g0, g1, lam_out, flag, err, st);
  if (lo == 4 && hi == 5) return step_pair<4, 5, S, R>(p, f0, f1, lam, g0, g1, lam_out, flag, err, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_pond_masks(int nx, int ny, const uint8_t* flag, uint8_t* mask,
                              cudaStream_t st) {
  k_pond_masks<<<tile_grid(nx, ny), dim3(kTX, kTY), 0, st>>>(nx, ny, flag, mask);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_pond_convert(const PondParams<R>& p, S* f0, S* f1, const S* lam,
                                const uint8_t* flag, const uint8_t* mask, cudaStream_t st) {
  const int lo = p.lat[0].n, hi = p.lat[1].n;
  if (lo == 3 && hi == 4) return convert_pair<3, 4, S, R>(p, f0, f1, lam, flag, mask, st);
  if (lo == 3 && hi == 5) return convert_pair<3, 5, S, R>(p, f0, f1, lam, flag, mask, st);
  if (lo == 4 && hi == 5) return convert_pair<4, 5, S, R>(p, f0, f1, lam, flag, mask, st);
  return cudaErrorInvalidValue;
}

template <class S, class R>
cudaError_t launch_pond_frame_io(const PondParams<R>& p, S* lam, double* ux, double* uy,
                                 double* T, int unpack, cudaStream_t st) {
  const unsigned blocks = (unsigned)((p.nc + kThreads - 1) / kThreads);
  k_pond_frame_io<S, R><<<blocks, kThreads, 0, st>>>(p, lam, ux, uy, T, unpack);
  return cudaGetLastError();
}

#define SLBM_POND_INST(S, R)                                                                    \
  template cudaError_t launch_pond_init<S, R>(const PondParams<R>&, S*, S*, S*, const double*, \
                                              const double*, const double*, const double*,     \
                                              cudaStream_t);                                   \
  template cudaError_t launch_pond_step<S, R>(const PondParams<R>&, const S*, const S*,        \
                                              const S*, S*, S*, S*, const uint8_t*, int*,      \
                                              cudaStream_t);                                   \
  template cudaError_t launch_pond_convert<S, R>(const PondParams<R>&, S*, S*, const S*,       \
                                                 const uint8_t*, const uint8_t*, cudaStream_t); \
  template cudaError_t launch_pond_frame_io<S, R>(const PondParams<R>&, S*, double*, double*,  \
                                                  double*, int, cudaStream_t);
SLBM_POND_INST(float, float)
SLBM_POND_INST(double, double)
#undef SLBM_POND_INST

}  // namespace slbm
