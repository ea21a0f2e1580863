// slbm_eq.cuh -- device arithmetic of the lattice equilibrium in deviation
// form, shared by the streaming and the interface / boundary kernels.
//
// Lattice-frame equilibrium of a tensor-product Gauss-Hermite lattice (eq.
// feqL0): f^L_i = rho phi_ix(u_x) phi_iy(u_y), where phi = V^-1 h(u) and
// h_m(u) = E[(u + Z)^m] are the raw Gaussian moments at T = T_L = 1 (the
// moment conditions sum_j c_j^m phi_j = h_m, m < n).  At rest phi = w (the 1-D
// weights), so with rho = 1 + dr and phi = w + dphi, dphi = V^-1 (h(u) - h(0)),
//   f^L_i - W_i = dr phi_x phi_y + w_x dphi_y + dphi_x w_y + dphi_x dphi_y,
// a sum of small terms that FP32 evaluates without cancellation.
#pragma once

#include "slbm_impl.cuh"

namespace slbm {

// h_m(u) - h_m(0), m < 5.
template <class R>
__device__ __forceinline__ void gauss_dev(R u, R* dh) {
  const R u2 = u * u;
  dh[0] = R(0);
  dh[1] = u;
  dh[2] = u2;
  dh[3] = u * (u2 + R(3));
  dh[4] = u2 * (u2 + R(6));
}

// dphi_j(u) for j < n.
template <class R>
__device__ __forceinline__ void dphi(const LatTab<R>& L, int n, R u, R* d) {
  R dh[kMaxN];
  gauss_dev<R>(u, dh);
#pragma unroll
  for (int j = 0; j < kMaxN; ++j) {
    if (j >= n) break;
    R s = R(0);
#pragma unroll
    for (int m = 1; m < kMaxN; ++m)
      if (m < n) s += L.vinv[j][m] * dh[m];
    d[j] = s;
  }
}

// Equilibrium deviation e[iy][ix] = f^L - W at (rho = 1 + dr, u).
template <class R>
__device__ __forceinline__ void eq_dev(const LatTab<R>& L, int n, R dr, R ux, R uy,
                                       R (*e)[kMaxN]) {
  R dx[kMaxN], dy[kMaxN];
  dphi<R>(L, n, ux, dx);
  dphi<R>(L, n, uy, dy);
#pragma unroll
  for (int iy = 0; iy < kMaxN; ++iy) {
    if (iy >= n) break;
    const R py = L.w1[iy] + dy[iy];
#pragma unroll
    for (int ix = 0; ix < kMaxN; ++ix) {
      if (ix >= n) break;
      const R px = L.w1[ix] + dx[ix];
      e[iy][ix] = dr * px * py + L.w1[ix] * dy[iy] + dx[ix] * L.w1[iy] + dx[ix] * dy[iy];
    }
  }
}

// Accumulator of the lifting's moment sums.  In FP32 it is the compensated
// dot product Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005): each product is split exactly with an FMA,
// each addition with TwoSum, and the error terms are summed alongside, so the
// result is as accurate as an accumulation in twice the working precision --
// at FP32 rates, where GB300's FP64 rate is a small fraction of its FP32 rate.
// In FP64 it sums plainly.
template <class R>
struct MomentAcc {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R a) {
    if constexpr (sizeof(R) == 8) {
      s += a;
    } else {
      const R t = s + a, z = t - s;
      c += (s - (t - z)) + (a - z);
      s = t;
    }
  }
  __device__ __forceinline__ void add_product(R x, R y) {
    if constexpr (sizeof(R) == 8) {
      s = fma(x, y, s);
    } else {
      const R pr = x * y, pe = fmaf(x, y, -pr);
      add(pr);
      c += pe;
    }
  }
  __device__ __forceinline__ R value() const { return s + c; }
};

}  // namespace slbm
