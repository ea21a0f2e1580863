// slbm_stream.cuh -- fused stream-collide kernel (sm_103a).
//
// One time step of every cell, lattice frame (Sec. II.C "Lattice reference
// frame" and Sec. III.D):
//   1. semi-Lagrangian streaming: f_i(x) = sum_{a,b} w^x_{i,a} w^y_{i,b}
//      f_i(x + o_i + (a, b)) -- eqs. (reconstructionPond), (advectionPond)
//      with the departure point x - c_i dt.  In the lattice frame every shift
//      c_i dt is a constant, so each population plane is a separable
//      constant-coefficient stencil; shifts that are integers (the rest node
//      and the CFL = 1 outer node) are single taps.  Collocation points of the
//      other lattice were converted beforehand by the interface kernel, so
//      every tap reads the target lattice's own planes.
//   2. rho, rho u (Sec. II.B), the lattice equilibrium in product form
//      f^L_i = rho phi_ix(u_x) phi_iy(u_y), phi = V^-1 h(u) with the Gaussian
//      moments h_m(u) = E[(u + Z)^m] (eq. feqL0 restated for a tensor-product
//      Gauss-Hermite lattice), and BGK: f <- f + omega (f^L - f)
//      (eq. Pond_f_equation with omega_1 = omega_2), all on the stored
//      deviations s_i = f_i - W_i.
//   3. optionally the Mach criterion of Sec. IV.A for the next step's flag.
//
// A CTA owns a 32 x 8 tile, one cell per thread; a warp is one 32-cell row
// segment.  A warp runs the low-order pass for its low-order lanes, then the
// high-order pass for its high-order lanes: inside a pass all active lanes
// execute the same Q-specific code, so no warp diverges on Q; a warp whose
// lanes are all of one lattice skips the other pass entirely.
#pragma once

#include "slbm_eq.cuh"

namespace slbm {

template <class S, class R>
__device__ __forceinline__ R ldg_as(const S* p) { return static_cast<R>(__ldg(p)); }

// Interpolate along x over one row: node jx's stencil starting at `row`
// (differential form v[k] + sum_a w[a] (v[a] - v[k]), see LatTab).
template <int P, class S, class R>
__device__ __forceinline__ R row_interp(const S* __restrict__ row, const LatTab<R>& L, int jx) {
  if (L.ntap[jx] == 1) return ldg_as<S, R>(row);
  R v[P];
#pragma unroll
  for (int a = 0; a < P; ++a) v[a] = ldg_as<S, R>(row + a);
  const int k = L.kref[jx];
  R vk = v[0];
#pragma unroll
  for (int a = 1; a < P; ++a) vk = a == k ? v[a] : vk;
  R t = vk;
#pragma unroll
  for (int a = 0; a < P; ++a) t += L.w[jx][a] * (v[a] - vk);
  return t;
}

// Stream + collide one cell of lattice L (N nodes per axis), on deviations
// s_i = f_i - W_i (streaming is affine in the shift; the collision uses the
// deviation form of the product equilibrium, see slbm_eq.cuh).
template <int N, int P, class S, class R>
__device__ __forceinline__ void stream_collide_cell(const Params<R>& p, const LatTab<R>& L,
                                                    const S* __restrict__ fin,
                                                    S* __restrict__ fout, int base, R& ux,
                                                    R& uy) {
  R f[N * N];
#pragma unroll
  for (int jy = 0; jy < N; ++jy) {
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const S* pl = fin + (size_t)(jx + N * jy) * p.plane + base + L.off[jx];
      R acc;
      if (L.ntap[jy] == 1) {
        acc = row_interp<P, S, R>(pl + L.off[jy] * p.pitch, L, jx);
      } else {
        R r[P];
#pragma unroll
        for (int b = 0; b < P; ++b) r[b] = row_interp<P, S, R>(pl + (L.off[jy] + b) * p.pitch, L, jx);
        const int k = L.kref[jy];
        R rk = r[0];
#pragma unroll
        for (int b = 1; b < P; ++b) rk = b == k ? r[b] : rk;
        acc = rk;
#pragma unroll
        for (int b = 0; b < P; ++b) acc += L.w[jy][b] * (r[b] - rk);
      }
      f[jx + N * jy] = acc;
    }
  }
  // density deviation and momentum through row / column sums of the N x N block
  R dr = R(0), mx = R(0), my = R(0);
#pragma unroll
  for (int jy = 0; jy < N; ++jy) {
    R rs = R(0);
#pragma unroll
    for (int jx = 0; jx < N; ++jx) rs += f[jx + N * jy];
    dr += rs;
    my += L.c[jy] * rs;
  }
#pragma unroll
  for (int jx = 0; jx < N; ++jx) {
    R cs = R(0);
#pragma unroll
    for (int jy = 0; jy < N; ++jy) cs += f[jx + N * jy];
    mx += L.c[jx] * cs;
  }
  const R inv = R(1) / (R(1) + dr);
  ux = mx * inv;
  uy = my * inv;
  R dx[N], dy[N];
  dphi<R>(L, N, ux, dx);
  dphi<R>(L, N, uy, dy);
#pragma unroll
  for (int jy = 0; jy < N; ++jy) {
    const R py = L.w1[jy] + dy[jy];
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const int i = jx + N * jy;
      const R px = L.w1[jx] + dx[jx];
      const R feq = dr * px * py + L.w1[jx] * dy[jy] + dx[jx] * L.w1[jy] + dx[jx] * dy[jy];
      fout[(size_t)i * p.plane + base] = static_cast<S>(f[i] + p.omega * (feq - f[i]));
    }
  }
}

template <int NL, int NH, int P, class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_stream_collide(const Params<R> p, const S* __restrict__ fin0, const S* __restrict__ fin1,
                 S* __restrict__ fout0, S* __restrict__ fout1,
                 const uint8_t* __restrict__ flag_cur, uint8_t* __restrict__ flag_nxt) {
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const int cell = x + p.nx * y;
  const int fl = flag_cur[cell];
  const int base = (y + p.G) * p.pitch + (x + kOX);
  R ux = R(0), uy = R(0);
  if (fl == 0)
    stream_collide_cell<NL, P, S, R>(p, p.lat[0], fin0, fout0, base, ux, uy);
  else
    stream_collide_cell<NH, P, S, R>(p, p.lat[1], fin1, fout1, base, ux, uy);
  if (p.crit == 1) flag_nxt[cell] = sqrt(ux * ux + uy * uy) > p.thr ? 1 : 0;
}

template <class S, class R>
cudaError_t launch_stream_collide_impl(const Params<R>& p, int P, const S* fin0, const S* fin1,
                                       S* fout0, S* fout1, const uint8_t* flag_cur,
                                       uint8_t* flag_nxt, cudaStream_t st) {
  const dim3 blk(kTX, kTY);
  const dim3 grd((p.nx + kTX - 1) / kTX, (p.ny + kTY - 1) / kTY);
  const int nl = p.lat[0].n, nh = p.lat[1].n;
#define SLBM_SC_CASE(NL, NH, PP)                                                            \
  if (nl == NL && nh == NH && P == PP) {                                                    \
    k_stream_collide<NL, NH, PP, S, R>                                                      \
        <<<grd, blk, 0, st>>>(p, fin0, fin1, fout0, fout1, flag_cur, flag_nxt);             \
    return cudaGetLastError();                                                              \
  }
#define SLBM_SC_PAIR(NL, NH) \
  SLBM_SC_CASE(NL, NH, 2) SLBM_SC_CASE(NL, NH, 3) SLBM_SC_CASE(NL, NH, 4) SLBM_SC_CASE(NL, NH, 5) SLBM_SC_CASE(NL, NH, 6)
  SLBM_SC_PAIR(3, 4)
  SLBM_SC_PAIR(3, 5)
  SLBM_SC_PAIR(4, 5)
#undef SLBM_SC_PAIR
#undef SLBM_SC_CASE
  return cudaErrorInvalidValue;
}

}  // namespace slbm
