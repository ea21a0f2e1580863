// slbm_indicator.cu -- learned refinement indicator: per-cell features from the
// local moments and their gradients, and a small MLP (16 -> 32 -> 32 -> 1,
// ReLU, FP16 weights, FP32 accumulation) evaluated on the tensor cores with
// warp-level mma.sync (m16n8k16, FP16 x FP16 -> FP32).  The flag is
// logit > threshold.  The paper refines by the plain Mach / Knudsen criteria
// (Sec. IV); this indicator is trained to reproduce such a criterion from the
// state of all-high-order runs, and the plain criterion stays its fallback.
//
// Features (lattice frame, the cell's own lattice; each multiplied by a fixed
// scale so the FP16 inputs are O(1)):
//   0 rho - 1, 1-2 u, 3 T - 1 (kinetic), 4-6 the non-equilibrium stress
//   sum c_a c_b (f - f^L) (xx, xy, yy), 7-8 the non-equilibrium energy flux
//   1/2 sum c_a |c|^2 (f - f^L), 9-14 central differences of rho, u_x, u_y
//   along x and y (periodic wrap, else the edge cell repeated), 15 |u|.
#include "../../include/slbm.h"
#include "slbm_eq.cuh"

namespace slbm {

namespace {

constexpr int kFeat = 16;
constexpr int kHid = 32;
constexpr int kIndThreads = 128;  // 4 warps, 32 cells per warp per pass

__constant__ float c_scale[kFeat] = {10.f,  3.f,   3.f,   10.f,  100.f, 100.f, 100.f, 100.f,
                                     100.f, 100.f, 100.f, 100.f, 100.f, 100.f, 100.f, 3.f};

__device__ __forceinline__ int clampwrap(int v, int n, int periodic) {
  if (v < 0) return periodic ? v + n : 0;
  if (v >= n) return periodic ? v - n : n - 1;
  return v;
}

// Features of cell (x, y) from its own lattice (N nodes per axis).
template <int N, class S, class R>
__device__ void cell_features_n(const Params<R>& p, const LatTab<R>& L, const S* f, int x, int y,
                                const R* mrho, const R* mux, const R* muy, float* out) {
  const size_t base = (size_t)(y + p.G) * p.pitch + (x + kOX);
  R s[N * N];
  R dr = R(0), jx = R(0), jy = R(0), e2 = R(0);
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix) {
      const R v = static_cast<R>(f[(size_t)(ix + N * iy) * p.plane + base]);
      s[ix + N * iy] = v;
      dr += v;
      jx += L.c[ix] * v;
      jy += L.c[iy] * v;
      e2 += (L.c[ix] * L.c[ix] + L.c[iy] * L.c[iy]) * v;
    }
  const R rho = R(1) + dr;
  const R ux = jx / rho, uy = jy / rho;
  const R T = ((R(2) + e2) / rho - ux * ux - uy * uy) / R(2);
  R dx[N], dy[N];
  dphi<R>(L, N, ux, dx);
  dphi<R>(L, N, uy, dy);
  R pxx = R(0), pxy = R(0), pyy = R(0), qx = R(0), qy = R(0);
#pragma unroll
  for (int iy = 0; iy < N; ++iy) {
    const R py = L.w1[iy] + dy[iy];
#pragma unroll
    for (int ix = 0; ix < N; ++ix) {
      const R px = L.w1[ix] + dx[ix];
      const R e = dr * px * py + L.w1[ix] * dy[iy] + dx[ix] * py;
      const R ne = s[ix + N * iy] - e;
      const R cx = L.c[ix], cy = L.c[iy], c2 = cx * cx + cy * cy;
      pxx += cx * cx * ne;
      pxy += cx * cy * ne;
      pyy += cy * cy * ne;
      qx += R(0.5) * cx * c2 * ne;
      qy += R(0.5) * cy * c2 * ne;
    }
  }
  const int xm = clampwrap(x - 1, p.nx, p.periodic_x), xp = clampwrap(x + 1, p.nx, p.periodic_x);
  const int ym = clampwrap(y - 1, p.ny, p.periodic_y), yp = clampwrap(y + 1, p.ny, p.periodic_y);
  const long long cxm = xm + (long long)p.nx * y, cxp = xp + (long long)p.nx * y;
  const long long cym = x + (long long)p.nx * ym, cyp = x + (long long)p.nx * yp;
  out[0] = (float)dr;
  out[1] = (float)ux;
  out[2] = (float)uy;
  out[3] = (float)(T - R(1));
  out[4] = (float)pxx;
  out[5] = (float)pxy;
  out[6] = (float)pyy;
  out[7] = (float)qx;
  out[8] = (float)qy;
  out[9] = (float)(R(0.5) * (mrho[cxp] - mrho[cxm]));
  out[10] = (float)(R(0.5) * (mrho[cyp] - mrho[cym]));
  out[11] = (float)(R(0.5) * (mux[cxp] - mux[cxm]));
  out[12] = (float)(R(0.5) * (mux[cyp] - mux[cym]));
  out[13] = (float)(R(0.5) * (muy[cxp] - muy[cxm]));
  out[14] = (float)(R(0.5) * (muy[cyp] - muy[cym]));
  out[15] = (float)sqrt(ux * ux + uy * uy);
#pragma unroll
  for (int q = 0; q < kFeat; ++q) out[q] *= c_scale[q];
}

template <class S, class R>
__device__ void cell_features(const Params<R>& p, const S* f0, const S* f1, int k, int x, int y,
                              const R* mrho, const R* mux, const R* muy, float* out) {
  const LatTab<R>& L = p.lat[k];
  const S* f = k ? f1 : f0;
  switch (L.n) {
    case 3: cell_features_n<3, S, R>(p, L, f, x, y, mrho, mux, muy, out); break;
    case 4: cell_features_n<4, S, R>(p, L, f, x, y, mrho, mux, muy, out); break;
    default: cell_features_n<5, S, R>(p, L, f, x, y, mrho, mux, muy, out); break;
  }
}

// rho, u_x, u_y of one cell from its own lattice, in the arithmetic type
// (the values the gradient features difference).
template <int N, class S, class R>
__device__ __forceinline__ void cell_ru(const Params<R>& p, const LatTab<R>& L, const S* f,
                                        size_t base, R* out) {
  R dr = R(0), jx = R(0), jy = R(0);
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix) {
      const R v = static_cast<R>(f[(size_t)(ix + N * iy) * p.plane + base]);
      dr += v;
      jx += L.c[ix] * v;
      jy += L.c[iy] * v;
    }
  const R rho = R(1) + dr;
  out[0] = rho;
  out[1] = jx / rho;
  out[2] = jy / rho;
}

// Moment planes of the gradient features, one thread per cell.
template <class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_ind_moments(const Params<R> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
              R* __restrict__ mrho, R* __restrict__ mux, R* __restrict__ muy) {
  const int x = blockIdx.x * kTX + threadIdx.x, y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long c = x + (long long)p.nx * y;
  const int k = flag[c];
  const LatTab<R>& L = p.lat[k];
  const S* f = k ? f1 : f0;
  const size_t base = (size_t)(y + p.G) * p.pitch + (x + kOX);
  R m[3];
  switch (L.n) {
    case 3: cell_ru<3, S, R>(p, L, f, base, m); break;
    case 4: cell_ru<4, S, R>(p, L, f, base, m); break;
    default: cell_ru<5, S, R>(p, L, f, base, m); break;
  }
  mrho[c] = m[0];
  mux[c] = m[1];
  muy[c] = m[2];
}

__device__ __forceinline__ uint32_t pack2(__half lo, __half hi) {
  const __half2 h = __halves2half2(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ uint32_t pack2f(float lo, float hi) {
  return pack2(__float2half_rn(lo), __float2half_rn(hi));
}

// D += A (16 x 16, row-major, FP16) * B (16 x 8, column-major, FP16), FP32.
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// B fragment of n-tile nt, k-rows k0 .. k0 + 15, of a row-major K x N weight
// matrix W: lane (g, t) holds W[k0 + 2t .. + 1][8 nt + g] and W[k0 + 2t + 8 .. + 9][8 nt + g].
__device__ __forceinline__ void bfrag(const __half* W, int ncols, int k0, int nt, int g, int t,
                                      uint32_t& b0, uint32_t& b1) {
  const int n = 8 * nt + g;
  b0 = pack2(W[(k0 + 2 * t) * ncols + n], W[(k0 + 2 * t + 1) * ncols + n]);
  b1 = pack2(W[(k0 + 2 * t + 8) * ncols + n], W[(k0 + 2 * t + 9) * ncols + n]);
}

// One pass: each warp takes 32 consecutive cells (two m16 tiles).  Lane l
// computes the features of cell base + l into shared memory (FP16); the warp
// then runs the MLP with the C fragments of one layer reused in registers as
// the A fragments of the next.  Outputs (any may be null): FP32 features
// (nc x 16, cell-major), logits, flags (logit > thr).
template <class S, class R>
__global__ void __launch_bounds__(kIndThreads)
k_indicator(const Params<R> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
            const R* __restrict__ mrho, const R* __restrict__ mux,
            const R* __restrict__ muy, const __half* __restrict__ w1,
            const float* __restrict__ b1, const __half* __restrict__ w2,
            const float* __restrict__ b2, const float* __restrict__ w3, float b3, float thr,
            float* feat_out, float* logit_out, uint8_t* flag_out) {
  __shared__ __half sfeat[kIndThreads / 32][32][kFeat + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const long long nc = (long long)p.nx * p.ny;
  // weights in B-fragment form, held for the whole kernel
  uint32_t B1[4][2], B2[2][4][2];
  const bool have_w = w1 != nullptr;
  if (have_w) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) bfrag(w1, kHid, 0, nt, g, t, B1[nt][0], B1[nt][1]);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) bfrag(w2, kHid, 16 * kk, nt, g, t, B2[kk][nt][0], B2[kk][nt][1]);
  }
  for (long long base = ((long long)blockIdx.x * (kIndThreads / 32) + warp) * 32; base < nc;
       base += (long long)gridDim.x * kIndThreads) {
    const long long c = base + lane;
    float fe[kFeat];
#pragma unroll
    for (int q = 0; q < kFeat; ++q) fe[q] = 0.f;
    if (c < nc) {
      const int x = (int)(c % p.nx), y = (int)(c / p.nx);
      cell_features<S, R>(p, f0, f1, flag[c], x, y, mrho, mux, muy, fe);
      if (feat_out)
#pragma unroll
        for (int q = 0; q < kFeat; ++q) feat_out[c * kFeat + q] = fe[q];
    }
#pragma unroll
    for (int q = 0; q < kFeat; ++q) sfeat[warp][lane][q] = __float2half_rn(fe[q]);
    __syncwarp();
    if (have_w) {
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        uint32_t A[4];
        A[0] = pack2(sfeat[warp][r0][2 * t], sfeat[warp][r0][2 * t + 1]);
        A[1] = pack2(sfeat[warp][r1][2 * t], sfeat[warp][r1][2 * t + 1]);
        A[2] = pack2(sfeat[warp][r0][2 * t + 8], sfeat[warp][r0][2 * t + 9]);
        A[3] = pack2(sfeat[warp][r1][2 * t + 8], sfeat[warp][r1][2 * t + 9]);
        // layer 1: 16 -> 32, ReLU
        float H1[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float ba = b1[8 * nt + 2 * t], bb = b1[8 * nt + 2 * t + 1];
          H1[nt][0] = ba; H1[nt][1] = bb; H1[nt][2] = ba; H1[nt][3] = bb;
          mma16816(H1[nt], A, B1[nt][0], B1[nt][1]);
#pragma unroll
          for (int q = 0; q < 4; ++q) H1[nt][q] = fmaxf(H1[nt][q], 0.f);
        }
        // layer 2: 32 -> 32, ReLU; the C fragments of layer 1 are A fragments
        float H2[4][4];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float ba = b2[8 * nt + 2 * t], bb = b2[8 * nt + 2 * t + 1];
          H2[nt][0] = ba; H2[nt][1] = bb; H2[nt][2] = ba; H2[nt][3] = bb;
        }
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          uint32_t A2[4];
          A2[0] = pack2f(H1[2 * kk][0], H1[2 * kk][1]);
          A2[1] = pack2f(H1[2 * kk][2], H1[2 * kk][3]);
          A2[2] = pack2f(H1[2 * kk + 1][0], H1[2 * kk + 1][1]);
          A2[3] = pack2f(H1[2 * kk + 1][2], H1[2 * kk + 1][3]);
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) mma16816(H2[nt], A2, B2[kk][nt][0], B2[kk][nt][1]);
        }
        // output: 32 -> 1, reduced over the four lanes of a row group
        float o0 = 0.f, o1 = 0.f;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const float wa = w3[8 * nt + 2 * t], wb = w3[8 * nt + 2 * t + 1];
          o0 += fmaxf(H2[nt][0], 0.f) * wa + fmaxf(H2[nt][1], 0.f) * wb;
          o1 += fmaxf(H2[nt][2], 0.f) * wa + fmaxf(H2[nt][3], 0.f) * wb;
        }
        o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
        o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
        o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
        o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
        if (t == 0) {
          const long long ca = base + r0, cb = base + r1;
          if (ca < nc) {
            if (logit_out) logit_out[ca] = o0 + b3;
            if (flag_out) flag_out[ca] = (o0 + b3) > thr ? 1 : 0;
          }
          if (cb < nc) {
            if (logit_out) logit_out[cb] = o1 + b3;
            if (flag_out) flag_out[cb] = (o1 + b3) > thr ? 1 : 0;
          }
        }
      }
    }
    __syncwarp();  // sfeat is rewritten next pass
  }
}

}  // namespace

template <class S, class R>
cudaError_t launch_indicator(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                             R* mrho, R* mux, R* muy, const IndicatorDev& w, float thr,
                             float* feat_out, float* logit_out, uint8_t* flag_out,
                             cudaStream_t st) {
  const dim3 tg((p.nx + kTX - 1) / kTX, (p.ny + kTY - 1) / kTY);
  k_ind_moments<S, R><<<tg, dim3(kTX, kTY), 0, st>>>(p, f0, f1, flag, mrho, mux, muy);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long nc = (long long)p.nx * p.ny;
  long long blocks = (nc + kIndThreads - 1) / kIndThreads;
  const long long cap = (long long)p.nsm * 16;
  if (blocks > cap) blocks = cap;
  k_indicator<S, R><<<(unsigned)blocks, kIndThreads, 0, st>>>(
      p, f0, f1, flag, mrho, mux, muy, w.w1, w.b1, w.w2, w.b2, w.w3, w.b3, thr, feat_out,
      logit_out, flag_out);
  return cudaGetLastError();
}

#define SLBM_IND_INST(S, R)                                                                  \
  template cudaError_t launch_indicator<S, R>(const Params<R>&, const S*, const S*,          \
                                              const uint8_t*, R*, R*, R*, const IndicatorDev&, \
                                              float, float*, float*, uint8_t*, cudaStream_t);
SLBM_IND_INST(float, float)
SLBM_IND_INST(double, double)
SLBM_IND_INST(__half, float)
#undef SLBM_IND_INST

}  // namespace slbm
