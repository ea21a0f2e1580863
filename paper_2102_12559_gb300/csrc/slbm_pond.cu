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
// Two-population model (Sec. II.B, eqs. Pond_f_equation / Pond_g_equation):
// the g populations are kept as e_i = g_i / T_frame - (C_v - 1) W_i, so the
// node's rest state is e = 0 like s = 0 for f.  Carried into a target frame
// with r^2 = T_s / T they become r^2 G e_s + (C_v - 1)(r^2 (G W - W) +
// (r^2 - 1) W).  T follows from the total energy (eq. E) with the g sum, and
// the collision adds (omega_1 - omega_2)(f* - f^eq) and (omega_1 - omega_2)
// (g* - g^eq) with the quasi-equilibria of eqs. (fqeq, gqeq) formed in the
// frame used (the co-moving frame to the predictor-corrector tolerance):
// f* - f^eq = W_i / 6 A:He3(c_i), A = sum c c c (f - f^eq); g* - g^eq = W_i q.c_i
// with q = sum c (g - g^eq), in the frame's units.
//
// Wrapping: the grid is periodic and departure points may move several cells
// (|v| dt grows with u and T), so node indices wrap with a modulo instead of
// reading a ghost ring.
#include "../../include/slbm.h"
#include "slbm_eq.cuh"

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
template <int N, bool ROWS, bool TWO, class S, class R>
__device__ void pond_cell(const PondParams<R>& p, const PondLat<R>& L, const S* __restrict__ f,
                          const S* __restrict__ e, const S* __restrict__ lam, S* __restrict__ g,
                          S* __restrict__ eo, S* __restrict__ lam_out, int x, int y, int* err) {
  const long long c = (long long)x + (long long)p.nx * y;
  R ux = (R)lam[c], uy = (R)lam[p.nc + c], T = (R)lam[2 * p.nc + c];
  // batched rows: the instance is uniform in y (the y interpolation of a
  // constant is the constant) and has fixed end states beyond 0 and len
  const int len = p.rows ? p.row_len[y] : p.nx;
  const double* ends = p.rows ? p.row_ends + 8 * y : nullptr;
  // the row's end states in the arithmetic type, converted once per cell
  R endv[2][4] = {{R(0), R(0), R(0), R(0)}, {R(0), R(0), R(0), R(0)}};
  if (p.rows)
#pragma unroll
    for (int q = 0; q < 8; ++q) endv[q / 4][q % 4] = (R)ends[q];
  const int Py = p.rows ? 1 : p.P;
  R d[N][N];                    // reconstructed deviations, [b][a]
  R dg[N][N];                   // g deviations (two-population model)
  for (int b = 0; b < N; ++b)
    for (int a = 0; a < N; ++a) d[b][a] = dg[b][a] = R(0);
  R dr = R(0), s1x = R(0), s1y = R(0), dT = R(0);
  bool ok = true, conv = false;
  for (int it = 0; it < p.maxit; ++it) {
    if (!(T > R(0)) || !isfinite(ux) || !isfinite(uy)) { ok = false; break; }
    const R st = sqrt(T), ist = R(1) / st;
    if constexpr (ROWS) {
      // batched rows: the collocation nodes of population (a, b) lie on the
      // cell's row and depend on a only, so per (a, node) the node's frame
      // terms, the x basis and the x contraction sum_j G_x[j] s[j][k] are
      // shared by every b (same arithmetic, fewer evaluations)
#pragma unroll 1
      for (int b = 0; b < N; ++b)
        if (fabs((st * L.c[b] + uy) * p.dt) > p.reach) ok = false;
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        const R vx = st * L.c[a] + ux;
        if (fabs(vx * p.dt) > p.reach) ok = false;
        R ax[kMaxP];
        const int x0 = stencil<R>(p.P, (R)x - vx * p.dt, ax);
        R accf[N], accg[N];
#pragma unroll
        for (int b = 0; b < N; ++b) accf[b] = accg[b] = R(0);
#pragma unroll 1
        for (int u = 0; u < p.P; ++u) {
          const int xi = x0 + u;
          const int side = xi < 0 ? 0 : (xi >= len ? 1 : -1);  // an end state, or a cell
          const bool E = side >= 0;
          const long long cs = E ? 0 : (long long)xi + (long long)p.nx * y;
          R sux, suy, sT, erho = R(0);
          if (E) {
            erho = endv[side][0];
            sux = endv[side][1];
            suy = endv[side][2];
            sT = endv[side][3];
          } else {
            sux = (R)lam[cs];
            suy = (R)lam[p.nc + cs];
            sT = (R)lam[2 * p.nc + cs];
          }
          const R r = sqrt(sT) * ist;
          const R dx = (sux - ux) * ist, dy = (suy - uy) * ist;
          const R dTs = (sT - T) / T;
          const R r2 = r * r;
          R gx[N];
#pragma unroll
          for (int j = 0; j < N; ++j) gx[j] = basis<N, R>(L, a, r * L.c[j] + dx);
          const R pxa = dphi1<N, R>(L, a, dx, dTs);
          const size_t base = (size_t)(y + p.G) * p.pitch + (xi + kOX);
          R rowf[N], rowg[N];
#pragma unroll
          for (int k = 0; k < N; ++k) {
            R rf = R(0), rg = R(0);
            if (!E) {
#pragma unroll
              for (int j = 0; j < N; ++j) {
                rf += gx[j] * (R)f[(size_t)(j + N * k) * p.plane + base];
                if constexpr (TWO) rg += gx[j] * (R)e[(size_t)(j + N * k) * p.plane + base];
              }
            }
            rowf[k] = rf;
            rowg[k] = rg;
          }
#pragma unroll
          for (int b = 0; b < N; ++b) {
            R gy[N];
#pragma unroll
            for (int j = 0; j < N; ++j) gy[j] = basis<N, R>(L, b, r * L.c[j] + dy);
            const R pyb = dphi1<N, R>(L, b, dy, dTs);
            const R gw = L.w[a] * pyb + pxa * L.w[b] + pxa * pyb;
            const R Wab = L.w[a] * L.w[b];
            R v = R(0);
            if (E) {
              v = (erho - R(1)) * (Wab + gw);
            } else {
#pragma unroll
              for (int k = 0; k < N; ++k) v += gy[k] * rowf[k];
            }
            v += gw;
            accf[b] += ax[u] * v;
            if constexpr (TWO) {
              R vg = R(0);
              if (E) {
                vg = p.cvm1 * (erho - R(1)) * (Wab + gw);
              } else {
#pragma unroll
                for (int k = 0; k < N; ++k) vg += gy[k] * rowg[k];
              }
              vg = r2 * vg + p.cvm1 * (r2 * gw + dTs * Wab);
              accg[b] += ax[u] * vg;
            }
          }
        }
#pragma unroll
        for (int b = 0; b < N; ++b) {
          d[b][a] = accf[b];
          dg[b][a] = accg[b];
        }
      }
    } else {
#pragma unroll 1
    for (int b = 0; b < N; ++b) {
      const R vy = st * L.c[b] + uy;
      if (fabs(vy * p.dt) > p.reach) ok = false;
      R ay[kMaxP];
      int y0 = stencil<R>(p.P, (R)y - vy * p.dt, ay);
      if (p.rows) {
        y0 = y;
        ay[0] = R(1);
      }
#pragma unroll 1
      for (int a = 0; a < N; ++a) {
        const R vx = st * L.c[a] + ux;
        if (fabs(vx * p.dt) > p.reach) ok = false;
        R ax[kMaxP];
        const int x0 = stencil<R>(p.P, (R)x - vx * p.dt, ax);
        R acc = R(0), gacc = R(0);
#pragma unroll 1
        for (int t = 0; t < Py; ++t) {
          const int yi = p.rows ? y : wrapm(y0 + t, p.ny);
          R acc_t = R(0), gacc_t = R(0);
#pragma unroll 1
          for (int u = 0; u < p.P; ++u) {
            int xi = x0 + u;
            const double* E = nullptr;  // fixed end state of a node beyond the instance
            if (p.rows) {
              if (xi < 0) E = ends;
              else if (xi >= len) E = ends + 4;
            } else {
              xi = wrapm(xi, p.nx);
            }
            const long long cs = E ? 0 : (long long)xi + (long long)p.nx * yi;
            const R sux = E ? (R)E[1] : (R)lam[cs], suy = E ? (R)E[2] : (R)lam[p.nc + cs];
            const R sT = E ? (R)E[3] : (R)lam[2 * p.nc + cs];
            const R r = sqrt(sT) * ist;
            const R dx = (sux - ux) * ist, dy = (suy - uy) * ist;
            const R dTs = (sT - T) / T;                   // r^2 - 1
            R gx[N], gy[N];
#pragma unroll
            for (int j = 0; j < N; ++j) {
              gx[j] = basis<N, R>(L, a, r * L.c[j] + dx);
              gy[j] = basis<N, R>(L, b, r * L.c[j] + dy);
            }
            // G W - W
            const R pxa = dphi1<N, R>(L, a, dx, dTs), pyb = dphi1<N, R>(L, b, dy, dTs);
            const R gw = L.w[a] * pyb + pxa * L.w[b] + pxa * pyb;
            const R Wab = L.w[a] * L.w[b];
            // G s_s; an end state is rho_b W, so G s_s = (rho_b - 1)(W + G W - W)
            const size_t base = (size_t)(yi + p.G) * p.pitch + (xi + kOX);
            R v = R(0);
            if (E) {
              v = ((R)E[0] - R(1)) * (Wab + gw);
            } else {
#pragma unroll
              for (int k = 0; k < N; ++k) {
                R row = R(0);
#pragma unroll
                for (int j = 0; j < N; ++j) row += gx[j] * (R)f[(size_t)(j + N * k) * p.plane + base];
                v += gy[k] * row;
              }
            }
            v += gw;
            acc_t += ax[u] * v;
            if constexpr (TWO) {  // r^2 G e_s + (C_v - 1)(r^2 (G W - W) + (r^2 - 1) W)
              R vg = R(0);
              if (E) {
                vg = p.cvm1 * ((R)E[0] - R(1)) * (Wab + gw);
              } else {
#pragma unroll
                for (int k = 0; k < N; ++k) {
                  R row = R(0);
#pragma unroll
                  for (int j = 0; j < N; ++j) row += gx[j] * (R)e[(size_t)(j + N * k) * p.plane + base];
                  vg += gy[k] * row;
                }
              }
              const R r2 = r * r;
              vg = r2 * vg + p.cvm1 * (r2 * gw + dTs * Wab);
              gacc_t += ax[u] * vg;
            }
          }
          acc += ay[t] * acc_t;
          gacc += ay[t] * gacc_t;
        }
        d[b][a] = acc;
        dg[b][a] = gacc;
      }
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
    if constexpr (TWO) {
      // rho C_v T / T_frame = 1 + s2'/2 - rho s1^2/2 + sum g / T_frame (eq. E)
      R sg = R(0);
#pragma unroll
      for (int b = 0; b < N; ++b)
#pragma unroll
        for (int a = 0; a < N; ++a) sg += dg[b][a];
      dT = (R(0.5) * s2 - R(0.5) * rho * (s1x * s1x + s1y * s1y) + sg - p.cvm1 * s0) /
           (rho * p.cv);
    } else {
      dT = p.thermal ? (s2 - rho * (s1x * s1x + s1y * s1y)) / (R(2) * rho) : R(0);
    }
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
  auto feq = [&](int a, int b) {
    const R pa = L.w[a] + ex[a], pb = L.w[b] + ey[b];
    return dr * pa * pb + L.w[a] * ey[b] + ex[a] * L.w[b] + ex[a] * ey[b];
  };
  if constexpr (!TWO) {
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const R eq = feq(a, b);
        g[(size_t)(a + N * b) * p.plane + base] = (S)(d[b][a] + p.omega * (eq - d[b][a]));
      }
  } else {
    // g^eq = (C_v - 1) (T / T_frame) f^eq (eq. geqPond), as a deviation; the
    // non-equilibrium tensors A = sum c c c (f - f^eq), q = sum c (g - g^eq)
    R Axxx = R(0), Axxy = R(0), Axyy = R(0), Ayyy = R(0), qx = R(0), qy = R(0);
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const R eq = feq(a, b);
        const R ca = L.c[a], cb = L.c[b];
        const R nf = d[b][a] - eq;
        Axxx += ca * ca * ca * nf;
        Axxy += ca * ca * cb * nf;
        Axyy += ca * cb * cb * nf;
        Ayyy += cb * cb * cb * nf;
        const R eg = p.cvm1 * ((R(1) + dT) * eq + dT * L.w[a] * L.w[b]);
        const R ng = dg[b][a] - eg;
        qx += ca * ng;
        qy += cb * ng;
      }
    const R Bx = Axxx + Axyy, By = Axxy + Ayyy;  // A_x.., A_y.. contracted
    R w1 = p.omega, w2 = p.omega2;
    if (p.hs) {  // mu = (1/omega_1 - 1/2) rho T dt with mu from the viscosity law
      const R Tabs = T * (R(1) + dT), rho = R(1) + dr;
      const R mu1 = (R)p.row_visc[2 * y], T1 = (R)p.row_visc[2 * y + 1];
      const R mu = mu1 * pow(Tabs / T1, p.s_exp);
      const R tau1 = mu / (rho * Tabs * p.dt) + R(0.5);
      w1 = R(1) / tau1;
      w2 = R(1) / ((tau1 - R(0.5)) * p.inv_pr + R(0.5));
    }
    const R w12 = w1 - w2;
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int a = 0; a < N; ++a) {
        const R eq = feq(a, b);
        const R ca = L.c[a], cb = L.c[b], W = L.w[a] * L.w[b];
        // eq. (fqeq): W/6 A:(c c c - sym(c (x) 1)); eq. (gqeq): W q.c
        const R fst = W * (Axxx * ca * ca * ca + R(3) * Axxy * ca * ca * cb +
                           R(3) * Axyy * ca * cb * cb + Ayyy * cb * cb * cb -
                           R(3) * (Bx * ca + By * cb)) / R(6);
        const R gst = W * (qx * ca + qy * cb);
        const R eg = p.cvm1 * ((R(1) + dT) * eq + dT * W);
        const size_t o = (size_t)(a + N * b) * p.plane + base;
        g[o] = (S)(d[b][a] + w1 * (eq - d[b][a]) + w12 * fst);
        eo[o] = (S)(dg[b][a] + w1 * (eg - dg[b][a]) + w12 * gst);
      }
  }
  lam_out[c] = (S)ux;
  lam_out[p.nc + c] = (S)uy;
  lam_out[2 * p.nc + c] = (S)T;
}

template <int NL, int NH, bool ROWS, bool TWO, int ONLY, class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_step(const PondParams<R> p, const S* __restrict__ f0, const S* __restrict__ f1,
            const S* __restrict__ e0, const S* __restrict__ e1, const S* __restrict__ lam,
            S* __restrict__ g0, S* __restrict__ g1, S* __restrict__ eo0, S* __restrict__ eo1,
            S* __restrict__ lam_out, const uint8_t* __restrict__ flag, int* err) {
  // one thread per cell; the block shape is a tuning choice (p.bx x p.by).
  // ONLY = 0 / 1: only the cells of that lattice (the other lattice's code is
  // not in the kernel); -1: both.
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  if (p.rows && x >= p.row_len[y]) return;  // beyond the row's instance
  const int k = flag[(long long)x + (long long)p.nx * y] ? 1 : 0;
  if constexpr (ONLY == 1) {
    if (k == 1) pond_cell<NH, ROWS, TWO, S, R>(p, p.lat[1], f1, e1, lam, g1, eo1, lam_out, x, y, err);
  } else if constexpr (ONLY == 0) {
    if (k == 0) pond_cell<NL, ROWS, TWO, S, R>(p, p.lat[0], f0, e0, lam, g0, eo0, lam_out, x, y, err);
  } else if (k) {
    pond_cell<NH, ROWS, TWO, S, R>(p, p.lat[1], f1, e1, lam, g1, eo1, lam_out, x, y, err);
  } else {
    pond_cell<NL, ROWS, TWO, S, R>(p, p.lat[0], f0, e0, lam, g0, eo0, lam_out, x, y, err);
  }
}

// Rest-frame equilibrium of both lattices (s = (rho - 1) W_i) and the frame.
template <class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_init(const PondParams<R> p, S* f0, S* f1, S* e0, S* e1, S* lam,
            const double* __restrict__ rho, const double* __restrict__ ux,
            const double* __restrict__ uy, const double* __restrict__ T) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long c = (long long)x + (long long)p.nx * y;
  const size_t base = (size_t)(y + p.G) * p.pitch + (x + kOX);
  const double dr = rho[c] - 1.0;
  for (int k = 0; k < 2; ++k) {
    const PondLat<R>& L = p.lat[k];
    S* f = k ? f1 : f0;
    S* e = k ? e1 : e0;  // g = (C_v - 1) T rho W_i in the cell's own frame (eq. geqPond)
    for (int b = 0; b < L.n; ++b)
      for (int a = 0; a < L.n; ++a) {
        const double w = (double)L.w[a] * (double)L.w[b];
        f[(size_t)(a + L.n * b) * p.plane + base] = (S)(dr * w);
        if (p.twopop) e[(size_t)(a + L.n * b) * p.plane + base] = (S)((double)p.cvm1 * dr * w);
      }
  }
  lam[c] = (S)ux[c];
  lam[p.nc + c] = (S)uy[c];
  lam[2 * p.nc + c] = (S)(T ? T[c] : 1.0);
}

// Per 32 x 8 tile: bit 0 = a low-order cell, bit 1 = a high-order cell.
__global__ void __launch_bounds__(kThreads)
k_pond_masks(int nx, int ny, const uint8_t* __restrict__ flag, const uint8_t* __restrict__ flag_old,
             uint8_t* __restrict__ mask) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  const bool in = x < nx && y < ny;
  const long long c = (long long)x + (long long)nx * y;
  int bit = in ? (flag[c] ? 2 : 1) : 0;
  if (in && flag_old && (flag_old[c] ? 1 : 0) != (flag[c] ? 1 : 0)) bit |= 4;
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
// l_A((v - u) / s).  At u = 0 this is the lattice-frame L.  Expanding in
// powers of v cancels for large |u|, so it is computed in closed form.  With
// w = u / s and v_j = s (c_j + w) the q-lattice velocities of the frame, the
// polynomial P_A(v) = l_A((v - u) / s) has P_A(v_j) = l_A(c_j), so the
// truncation to degrees < nq is
//   Lm[A][j] = l_A(c_j) - sum_{m = nq}^{nQ - 1} k_A[m] (c_j + w)^m,
//   k_A[m] = sum_{k >= m} V_Q^-1[A][k] binom(k, m) (-w)^(k - m),
// the coefficients of P_A in powers of v / s.  Every term is of the size of
// the result, so the arithmetic type suffices.
template <int NQ, int NQQ, class R>
__device__ __forceinline__ void lift_matrix_w(const PondLat<R>& Lq, const PondLat<R>& LQ, R w,
                                              R (*Lm)[NQ]) {
#pragma unroll
  for (int A = 0; A < NQQ; ++A) {
    R kA[NQQ];
#pragma unroll
    for (int m = NQ; m < NQQ; ++m) {
      R acc = R(0), pw = R(1), bin = R(1);  // (-w)^(k-m), binom(k, m) for k = m, m+1, ...
#pragma unroll
      for (int k = m; k < NQQ; ++k) {
        acc += LQ.vinv[A][k] * bin * pw;
        pw *= -w;
        bin = bin * R(k + 1) / R(k + 1 - m);
      }
      kA[m] = acc;
    }
#pragma unroll
    for (int j = 0; j < NQ; ++j) {
      const R x = Lq.c[j] + w;
      R v = basis<NQQ, R>(LQ, A, Lq.c[j]), xm = R(1);
#pragma unroll
      for (int m = 1; m < NQQ; ++m) {
        xm *= x;
        if (m >= NQ) v -= kA[m] * xm;
      }
      Lm[A][j] = v;
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
__device__ void pond_convert_cell(const PondParams<R>& p, S* f0, S* f1, S* e0, S* e1, int k,
                                  size_t base, const S* lam, long long c) {
  const PondLat<R>& Lq = p.lat[0];
  const PondLat<R>& LQ = p.lat[1];
  if (k == 0) {
    R s[NQ][NQ];
    // moment sums in twice the working precision for FP32 (MomentAcc)
    MomentAcc<R> a0, ax, ay, a2, ag;
#pragma unroll
    for (int b = 0; b < NQ; ++b)
#pragma unroll
      for (int a = 0; a < NQ; ++a) {
        const R v = (R)f0[(size_t)(a + NQ * b) * p.plane + base];
        s[b][a] = v;
        a0.add(v);
        ax.add_product(Lq.c[a], v);
        ay.add_product(Lq.c[b], v);
        a2.add_product(Lq.c[a] * Lq.c[a] + Lq.c[b] * Lq.c[b] - R(2), v);
        if (p.twopop) ag.add((R)e0[(size_t)(a + NQ * b) * p.plane + base]);
      }
    const R m0 = a0.value(), m2 = a2.value(), mg = ag.value();
    const R rho = R(1) + m0;
    const R ux = ax.value() / rho, uy = ay.value() / rho;
    const R u2 = ux * ux + uy * uy;
    R dT = R(0);
    if (p.twopop)  // the node's T from the total energy (eq. E), as in the step
      dT = (R(0.5) * m2 - R(0.5) * rho * u2 + mg - p.cvm1 * m0) / (rho * p.cv);
    else if (p.thermal)
      dT = (m2 - rho * u2) / (R(2) * rho);
    const R dr = m0;
    R qx[NQ], qy[NQ], Qx[NQQ], Qy[NQQ];
    dphi_t<NQ, R>(Lq, ux, dT, qx);
    dphi_t<NQ, R>(Lq, uy, dT, qy);
    dphi_t<NQQ, R>(LQ, ux, dT, Qx);
    dphi_t<NQQ, R>(LQ, uy, dT, Qy);
    const double sq = sqrt((double)lam[2 * p.nc + c]);
    R Lx[NQQ][NQ], Ly[NQQ][NQ];
    lift_matrix_w<NQ, NQQ, R>(Lq, LQ, (R)((double)lam[c] / sq), Lx);
    lift_matrix_w<NQ, NQQ, R>(Lq, LQ, (R)((double)lam[p.nc + c] / sq), Ly);
    // pass 0: f; pass 1: g, whose equilibrium is (C_v - 1)(1 + dT) f^eq (eq.
    // geqPond, in units of the frame temperature) as a deviation
    for (int pass = 0; pass < (p.twopop ? 2 : 1); ++pass) {
      const R sc = pass ? p.cvm1 * (R(1) + dT) : R(1), sw = pass ? p.cvm1 * dT : R(0);
      if (pass)
#pragma unroll
        for (int b = 0; b < NQ; ++b)
#pragma unroll
          for (int a = 0; a < NQ; ++a) s[b][a] = (R)e0[(size_t)(a + NQ * b) * p.plane + base];
      // non-equilibrium part of the q vector
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
          const R pa = Lq.w[a] + qx[a], pb = Lq.w[b] + qy[b];
          const R eq = dr * pa * pb + Lq.w[a] * qy[b] + qx[a] * Lq.w[b] + qx[a] * qy[b];
          s[b][a] -= sc * eq + sw * Lq.w[a] * Lq.w[b];
        }
      // L_x (f_q - f^eq_q) L_y^T + f^eq_Q
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
      S* out = pass ? e1 : f1;
#pragma unroll
      for (int B = 0; B < NQQ; ++B)
#pragma unroll
        for (int A = 0; A < NQQ; ++A) {
          R v = R(0);
#pragma unroll
          for (int b = 0; b < NQ; ++b) v += Ly[B][b] * t[b][A];
          const R pa = LQ.w[A] + Qx[A], pb = LQ.w[B] + Qy[B];
          const R eq = dr * pa * pb + LQ.w[A] * Qy[B] + Qx[A] * LQ.w[B] + Qx[A] * Qy[B];
          v += sc * eq + sw * LQ.w[A] * LQ.w[B];
          out[(size_t)(A + NQQ * B) * p.plane + base] = (S)v;
        }
    }
  } else {
    // P s_Q P^T (P W_Q P^T = W_q: projection keeps the moments of order < nq);
    // the same for the g planes
    for (int pass = 0; pass < (p.twopop ? 2 : 1); ++pass) {
      const S* in = pass ? e1 : f1;
      S* out = pass ? e0 : f0;
      R t[NQQ][NQ];
#pragma unroll
      for (int B = 0; B < NQQ; ++B)
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
          R v = R(0);
#pragma unroll
          for (int A = 0; A < NQQ; ++A)
            v += p.proj[a][A] * (R)in[(size_t)(A + NQQ * B) * p.plane + base];
          t[B][a] = v;
        }
#pragma unroll
      for (int b = 0; b < NQ; ++b)
#pragma unroll
        for (int a = 0; a < NQ; ++a) {
          R v = R(0);
#pragma unroll
          for (int B = 0; B < NQQ; ++B) v += p.proj[b][B] * t[B][a];
          out[(size_t)(a + NQ * b) * p.plane + base] = (S)v;
        }
    }
  }
}

// Screening for a conversion, one thread per cell of a 32 x 8 tile (few
// registers, so many tiles are resident): flag_to given, the cells whose
// lattice changes; else mask null, every cell; else the cells of tiles whose
// 3 x 3 tile neighbourhood holds both lattices (and, with near_change, a
// changed cell), on batched rows only those that read the other lattice.
// Selected cells are appended per warp to the lift or the projection list.
template <class R>
__global__ void __launch_bounds__(kThreads)
k_pond_screen(const PondParams<R> p, const uint8_t* __restrict__ flag,
              const uint8_t* __restrict__ mask, const uint8_t* __restrict__ flag_to,
              int near_change, ConvLists L) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  bool sel = x < p.nx && y < p.ny && !(p.rows && x >= p.row_len[y]);
  const long long c = (long long)x + (long long)p.nx * y;
  const int k = sel ? (flag[c] ? 1 : 0) : 0;
  if (flag_to) {
    if (sel) sel = (flag_to[c] ? 1 : 0) != k;
  } else if (mask) {
    // 3 x 3 tile neighbourhood (periodic) must hold both lattices (the same
    // answer for the whole block)
    const int tx = blockIdx.x, ty = blockIdx.y, ntx = gridDim.x, nty = gridDim.y;
    int bits = 0;
    for (int j = -1; j <= 1; ++j)
      for (int i = -1; i <= 1; ++i)
        bits |= mask[wrapm(tx + i, ntx) + ntx * wrapm(ty + j, nty)];
    if ((bits & 3) != 3 || (near_change && !(bits & 4))) sel = false;
    if (sel && p.rows) {
      // a row reads only itself: only cells that a cell of the other lattice
      // within the largest departure plus the stencil half-width reads
      const int B = (int)p.reach + (p.P + 1) / 2;
      const int lo = max(0, x - B), hi = min(p.row_len[y] - 1, x + B);
      bool other = false;
      for (int xi = lo; xi <= hi && !other; ++xi)
        other = (flag[(long long)xi + (long long)p.nx * y] ? 1 : 0) != k;
      sel = other;
    }
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int kk = 0; kk < 2; ++kk) {
    const bool mine = sel && k == kk;
    const unsigned b = __ballot_sync(0xffffffffu, mine);
    if (!b) continue;
    const int leader = __ffs(b) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(L.count + kk, __popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (mine) (kk ? L.proj : L.lift)[base + __popc(b & ((1u << lane) - 1u))] = (int)c;
  }
}

constexpr int kConvThreads = 128;

// The listed conversions, one thread per cell.
template <int NQ, int NQQ, class S, class R>
__global__ void __launch_bounds__(kConvThreads)
k_pond_convert_list(const PondParams<R> p, S* f0, S* f1, S* e0, S* e1, const S* __restrict__ lam,
                    ConvLists L) {
  const int nc = (int)p.nc;
  const int n0 = min(max(L.count[0], 0), nc), n1 = min(max(L.count[1], 0), nc);
  for (int i = blockIdx.x * kConvThreads + threadIdx.x; i < n0 + n1;
       i += gridDim.x * kConvThreads) {
    const int k = i < n0 ? 0 : 1;
    const int c = k ? L.proj[i - n0] : L.lift[i];
    if (c < 0 || c >= nc) continue;
    const int x = c % p.nx, y = c / p.nx;
    pond_convert_cell<NQ, NQQ, S, R>(p, f0, f1, e0, e1, k, (size_t)(y + p.G) * p.pitch + (x + kOX),
                                     lam, c);
  }
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

// rho and absolute T of a cell from its own lattice (N nodes per axis), its
// g planes (two-population model) and its frame (as the step's moments).
template <int N, class S, class R>
__device__ __forceinline__ void cell_rho_T(const PondParams<R>& p, const PondLat<R>& L,
                                           const S* f, const S* e, const S* lam, long long c,
                                           size_t base, R& rho, R& T) {
  R s0 = R(0), sx = R(0), sy = R(0), s2 = R(0), sg = R(0);
#pragma unroll
  for (int b = 0; b < N; ++b)
#pragma unroll
    for (int a = 0; a < N; ++a) {
      const size_t o = (size_t)(a + N * b) * p.plane + base;
      const R v = (R)f[o];
      s0 += v;
      sx += L.c[a] * v;
      sy += L.c[b] * v;
      s2 += (L.c[a] * L.c[a] + L.c[b] * L.c[b] - R(2)) * v;
      if (p.twopop) sg += (R)e[o];
    }
  rho = R(1) + s0;
  const R s1x = sx / rho, s1y = sy / rho;
  const R dT = p.twopop ? (R(0.5) * s2 - R(0.5) * rho * (s1x * s1x + s1y * s1y) + sg - p.cvm1 * s0) /
                              (rho * p.cv)
                        : (s2 - rho * (s1x * s1x + s1y * s1y)) / (R(2) * rho);
  T = (R)lam[2 * p.nc + c] * (R(1) + dT);
}

// Knudsen refinement criterion of Sec. IV.C on batched rows: Kn = lambda / L,
// L = |rho / (d rho / dx)| by central differences (the end states' density
// beyond the ends), lambda = 16 / (5 sqrt(2 pi gamma)) mu a / p of hard
// spheres with the row's viscosity law, a = sqrt(gamma T), p = rho T; the new
// flag is Kn > thr or the old flag (refinement only: a cell once high-order
// stays so; cells beyond the instance keep theirs).
template <int NL, int NH, class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_kn(const PondParams<R> p, const S* __restrict__ f0, const S* __restrict__ f1,
          const S* __restrict__ e0, const S* __restrict__ e1, const S* __restrict__ lam,
          const uint8_t* __restrict__ flag, R thr, uint8_t* __restrict__ out) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long c = (long long)x + (long long)p.nx * y;
  const int len = p.row_len[y];
  if (x >= len) {
    out[c] = flag[c];
    return;
  }
  auto state = [&](int xi, R& rho, R& T) {
    const long long ci = (long long)xi + (long long)p.nx * y;
    const size_t base = (size_t)(y + p.G) * p.pitch + (xi + kOX);
    if (flag[ci]) cell_rho_T<NH, S, R>(p, p.lat[1], f1, e1, lam, ci, base, rho, T);
    else cell_rho_T<NL, S, R>(p, p.lat[0], f0, e0, lam, ci, base, rho, T);
  };
  R rho, T, rl, rr, Tn;
  state(x, rho, T);
  if (x > 0) state(x - 1, rl, Tn);
  else rl = (R)p.row_ends[8 * y];
  if (x < len - 1) state(x + 1, rr, Tn);
  else rr = (R)p.row_ends[8 * y + 4];
  const R gam = (p.cv + R(1)) / p.cv;
  const R mu = (R)p.row_visc[2 * y] * pow(T / (R)p.row_visc[2 * y + 1], p.s_exp);
  const R lmf = R(16) / (R(5) * sqrt(R(2) * R(3.14159265358979323846) * gam)) * mu *
                sqrt(gam * T) / (rho * T);
  const R kn = lmf * fabs(R(0.5) * (rr - rl)) / rho;
  out[c] = (kn > thr || flag[c]) ? 1 : 0;
}

// Plane i of lattice k's g planes to / from absolute g (cell-major doubles).
template <class S, class R>
__global__ void __launch_bounds__(kThreads)
k_pond_gio(const PondParams<R> p, int k, int i, S* e, const S* __restrict__ lam, double* buf,
           int unpack) {
  const long long c = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (c >= p.nc) return;
  const PondLat<R>& L = p.lat[k];
  const int x = (int)(c % p.nx), y = (int)(c / p.nx);
  const size_t o = (size_t)i * p.plane + (size_t)(y + p.G) * p.pitch + (x + kOX);
  const double W = (double)L.w[i % L.n] * (double)L.w[i / L.n];
  const double T = (double)lam[2 * p.nc + c];
  if (unpack) e[o] = (S)(buf[c] / T - (double)p.cvm1 * W);
  else buf[c] = T * ((double)e[o] + (double)p.cvm1 * W);
}

dim3 tile_grid(int nx, int ny) { return dim3((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY); }

template <int NL, int NH, bool ROWS, bool TWO, class S, class R>
cudaError_t step_launch(const PondParams<R>& p, dim3 grid, dim3 block, const S* f0, const S* f1,
                        const S* e0, const S* e1, const S* lam, S* g0, S* g1, S* eo0, S* eo1,
                        S* lam_out, const uint8_t* flag, int* err, int split, cudaStream_t st) {
  if (!split) {
    k_pond_step<NL, NH, ROWS, TWO, -1, S, R><<<grid, block, 0, st>>>(
        p, f0, f1, e0, e1, lam, g0, g1, eo0, eo1, lam_out, flag, err);
    return cudaGetLastError();
  }
  // one launch per lattice, each carrying only its lattice's code: with both
  // lattices in one kernel, warps running either path stall on instruction
  // fetch (the batched shocks with 14 % D2Q25 cells: 0.99 ms, against 0.60 ms
  // all-D2Q16 and 1.13 ms all-D2Q25).  The launches write disjoint cells.
  k_pond_step<NL, NH, ROWS, TWO, 0, S, R><<<grid, block, 0, st>>>(
      p, f0, f1, e0, e1, lam, g0, g1, eo0, eo1, lam_out, flag, err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pond_step<NL, NH, ROWS, TWO, 1, S, R><<<grid, block, 0, st>>>(
      p, f0, f1, e0, e1, lam, g0, g1, eo0, eo1, lam_out, flag, err);
  return cudaGetLastError();
}

template <int NL, int NH, class S, class R>
cudaError_t step_pair(const PondParams<R>& p, const S* f0, const S* f1, const S* e0, const S* e1,
                      const S* lam, S* g0, S* g1, S* eo0, S* eo1, S* lam_out, const uint8_t* flag,
                      int* err, int split, cudaStream_t st) {
  const int bx = p.bx > 0 ? p.bx : kTX, by = p.bx > 0 ? p.by : kTY;
  if (bx * by != kThreads) return cudaErrorInvalidConfiguration;
  const dim3 grid((p.nx + bx - 1) / bx, (p.ny + by - 1) / by), block(bx, by);
  // batched rows and the two-population model get their own instantiations
  // (each kernel carries only the code it runs: less instruction fetch)
#define SLBM_POND_STEP(ROWS, TWO)                                                              \
  return step_launch<NL, NH, ROWS, TWO, S, R>(p, grid, block, f0, f1, e0, e1, lam, g0, g1, eo0, \
                                              eo1, lam_out, flag, err, split, st)
  if (p.rows && p.twopop) SLBM_POND_STEP(true, true);
  if (p.rows) SLBM_POND_STEP(true, false);
  if (p.twopop) SLBM_POND_STEP(false, true);
  SLBM_POND_STEP(false, false);
#undef SLBM_POND_STEP
}

template <int NL, int NH, class S, class R>
cudaError_t convert_pair(const PondParams<R>& p, S* f0, S* f1, S* e0, S* e1, const S* lam,
                         const ConvLists& L, cudaStream_t st) {
  k_pond_convert_list<NL, NH, S, R><<<2 * (p.nsm > 0 ? p.nsm : 1), kConvThreads, 0, st>>>(
      p, f0, f1, e0, e1, lam, L);
  return cudaGetLastError();
}

}  // namespace

template <class S, class R>
cudaError_t launch_pond_init(const PondParams<R>& p, S* f0, S* f1, S* e0, S* e1, S* lam,
                             const double* rho, const double* ux, const double* uy,
                             const double* T, cudaStream_t st) {
  k_pond_init<S, R><<<tile_grid(p.nx, p.ny), dim3(kTX, kTY), 0, st>>>(p, f0, f1, e0, e1, lam, rho,
                                                                      ux, uy, T);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_pond_step(const PondParams<R>& p, const S* f0, const S* f1, const S* e0,
                             const S* e1, const S* lam, S* g0, S* g1, S* eo0, S* eo1,
                             S* lam_out, const uint8_t* flag, int* err, int split,
                             cudaStream_t st) {
  const int lo = p.lat[0].n, hi = p.lat[1].n;
  if (lo == 3 && hi == 4)
    return step_pair<3, 4, S, R>(p, f0, f1, e0, e1, lam, g0, g1, eo0, eo1, lam_out, flag, err,
                                 split, st);
  if (lo == 3 && hi == 5)
    return step_pair<3, 5, S, R>(p, f0, f1, e0, e1, lam, g0, g1, eo0, eo1, lam_out, flag, err,
                                 split, st);
  if (lo == 4 && hi == 5)
    return step_pair<4, 5, S, R>(p, f0, f1, e0, e1, lam, g0, g1, eo0, eo1, lam_out, flag, err,
                                 split, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_pond_masks(int nx, int ny, const uint8_t* flag, const uint8_t* flag_old,
                              uint8_t* mask, cudaStream_t st) {
  k_pond_masks<<<tile_grid(nx, ny), dim3(kTX, kTY), 0, st>>>(nx, ny, flag, flag_old, mask);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_pond_convert(const PondParams<R>& p, S* f0, S* f1, S* e0, S* e1, const S* lam,
                                const uint8_t* flag, const uint8_t* mask, const uint8_t* flag_to,
                                int near_change, const ConvLists& lists, cudaStream_t st) {
  const int lo = p.lat[0].n, hi = p.lat[1].n;
  if (!((lo == 3 && hi == 4) || (lo == 3 && hi == 5) || (lo == 4 && hi == 5)))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(lists.count, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_pond_screen<R><<<tile_grid(p.nx, p.ny), dim3(kTX, kTY), 0, st>>>(p, flag, mask, flag_to,
                                                                     near_change, lists);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (lo == 3 && hi == 4) return convert_pair<3, 4, S, R>(p, f0, f1, e0, e1, lam, lists, st);
  if (lo == 3 && hi == 5) return convert_pair<3, 5, S, R>(p, f0, f1, e0, e1, lam, lists, st);
  return convert_pair<4, 5, S, R>(p, f0, f1, e0, e1, lam, lists, st);
}

template <class S, class R>
cudaError_t launch_pond_kn(const PondParams<R>& p, const S* f0, const S* f1, const S* e0,
                           const S* e1, const S* lam, const uint8_t* flag, double thr,
                           uint8_t* out, cudaStream_t st) {
  const int lo = p.lat[0].n, hi = p.lat[1].n;
  const dim3 g = tile_grid(p.nx, p.ny), b(kTX, kTY);
  if (lo == 3 && hi == 4) k_pond_kn<3, 4, S, R><<<g, b, 0, st>>>(p, f0, f1, e0, e1, lam, flag, (R)thr, out);
  else if (lo == 3 && hi == 5) k_pond_kn<3, 5, S, R><<<g, b, 0, st>>>(p, f0, f1, e0, e1, lam, flag, (R)thr, out);
  else if (lo == 4 && hi == 5) k_pond_kn<4, 5, S, R><<<g, b, 0, st>>>(p, f0, f1, e0, e1, lam, flag, (R)thr, out);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_pond_gio(const PondParams<R>& p, int k, int i, S* e, const S* lam, double* buf,
                            int unpack, cudaStream_t st) {
  const unsigned blocks = (unsigned)((p.nc + kThreads - 1) / kThreads);
  k_pond_gio<S, R><<<blocks, kThreads, 0, st>>>(p, k, i, e, lam, buf, unpack);
  return cudaGetLastError();
}

template <class S, class R>
cudaError_t launch_pond_frame_io(const PondParams<R>& p, S* lam, double* ux, double* uy,
                                 double* T, int unpack, cudaStream_t st) {
  const unsigned blocks = (unsigned)((p.nc + kThreads - 1) / kThreads);
  k_pond_frame_io<S, R><<<blocks, kThreads, 0, st>>>(p, lam, ux, uy, T, unpack);
  return cudaGetLastError();
}

#define SLBM_POND_INST(S, R)                                                                    \
  template cudaError_t launch_pond_init<S, R>(const PondParams<R>&, S*, S*, S*, S*, S*,         \
                                              const double*, const double*, const double*,     \
                                              const double*, cudaStream_t);                    \
  template cudaError_t launch_pond_step<S, R>(const PondParams<R>&, const S*, const S*,        \
                                              const S*, const S*, const S*, S*, S*, S*, S*,    \
                                              S*, const uint8_t*, int*, int, cudaStream_t);    \
  template cudaError_t launch_pond_convert<S, R>(const PondParams<R>&, S*, S*, S*, S*,         \
                                                 const S*, const uint8_t*, const uint8_t*,     \
                                                 const uint8_t*, int, const ConvLists&,        \
                                                 cudaStream_t);                                \
  template cudaError_t launch_pond_frame_io<S, R>(const PondParams<R>&, S*, double*, double*,  \
                                                  double*, int, cudaStream_t);                 \
  template cudaError_t launch_pond_gio<S, R>(const PondParams<R>&, int, int, S*, const S*,     \
                                             double*, int, cudaStream_t);                     \
  template cudaError_t launch_pond_kn<S, R>(const PondParams<R>&, const S*, const S*,          \
                                            const S*, const S*, const S*, const uint8_t*,      \
                                            double, uint8_t*, cudaStream_t);
SLBM_POND_INST(float, float)
SLBM_POND_INST(double, double)
#undef SLBM_POND_INST

}  // namespace slbm
