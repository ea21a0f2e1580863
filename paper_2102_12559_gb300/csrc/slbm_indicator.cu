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
// one tile of 32 x 16 cells per block pass; 8 warps, each two rows of 32
constexpr int kIndTX = 32, kIndTY = 16;
constexpr int kIndWarps = 8, kIndThreads = 32 * kIndWarps;
constexpr int kHaloX = kIndTX + 2, kHaloY = kIndTY + 2;

__constant__ float c_scale[kFeat] = {10.f,  3.f,   3.f,   10.f,  100.f, 100.f, 100.f, 100.f,
                                     100.f, 100.f, 100.f, 100.f, 100.f, 100.f, 100.f, 3.f};

__device__ __forceinline__ int clampwrap(int v, int n, int periodic) {
  if (v < 0) return periodic ? v + n : 0;
  if (v >= n) return periodic ? v - n : n - 1;
  return v;
}

// Raw moments of one cell's stored deviations v_i = f_i - W_i on its own
// lattice (N nodes per axis), M_ab = sum_i c_ix^a c_iy^b v_i, in one pass over
// the populations by row sums r_a(iy) = sum_ix c_ix^a v_i:
//   M[0..2] = M_00, M_10, M_01;  with FULL also
//   M[3..9] = M_20, M_11, M_02, M_30, M_21, M_12, M_03.
template <int N, bool FULL, class S, class R>
__device__ __forceinline__ void raw_moments(const Params<R>& p, const LatTab<R>& L, const S* f,
                                            size_t base, R* M) {
#pragma unroll
  for (int k = 0; k < (FULL ? 10 : 3); ++k) M[k] = R(0);
#pragma unroll
  for (int iy = 0; iy < N; ++iy) {
    R r0 = R(0), r1 = R(0), r2 = R(0), r3 = R(0);
#pragma unroll
    for (int ix = 0; ix < N; ++ix) {
      const R v = from_s<R>(f[(size_t)(ix + N * iy) * p.plane + base], L.sc[ix + N * iy]);
      const R cx = L.c[ix];
      r0 += v;
      r1 += cx * v;
      if (FULL) {
        r2 += cx * cx * v;
        r3 += cx * cx * cx * v;
      }
    }
    const R cy = L.c[iy];
    M[0] += r0;
    M[1] += r1;
    M[2] += cy * r0;
    if (FULL) {
      M[3] += r2;
      M[4] += cy * r1;
      M[5] += cy * cy * r0;
      M[6] += r3;
      M[7] += cy * r2;
      M[8] += cy * cy * r1;
      M[9] += cy * cy * cy * r0;
    }
  }
}

// Features 0-8 and 15 from the raw moments (FULL set) of a cell on a lattice
// of N nodes per axis.  The moments of f^L - W follow from the product form
// f^L = rho phi_x phi_y: with H_a(u) = sum_j c_j^a phi_j(u) = mu_a + d_a(u),
// mu = (1, 0, 1, 0) the moments of the weights (T_L = 1),
//   sum_i c_ix^a c_iy^b (f^L - W)_i = dr mu_a mu_b
//                                   + rho (mu_a d_b(u_y) + d_a(u_x) mu_b + d_a(u_x) d_b(u_y)),
// where d_1 = u, d_2 = u^2 (moment conditions, a < N) and d_3 = u^3 + 3 u for
// N >= 4; on three nodes {0, +-a} c^3 = a^2 c, so d_3 = a^2 u.  The
// non-equilibrium stress and energy flux are M_ab minus these.
template <int N, class R>
__device__ __forceinline__ void moment_features(const LatTab<R>& L, const R* M, float* out) {
  const R dr = M[0], rho = R(1) + dr, inv = R(1) / rho;
  const R ux = M[1] * inv, uy = M[2] * inv;
  const R ux2 = ux * ux, uy2 = uy * uy;
  const R a2 = L.c[N - 1] * L.c[N - 1];
  const R d3x = N >= 4 ? ux * (ux2 + R(3)) : a2 * ux;
  const R d3y = N >= 4 ? uy * (uy2 + R(3)) : a2 * uy;
  const R pxx = M[3] - (dr + rho * ux2);
  const R pxy = M[4] - rho * ux * uy;
  const R pyy = M[5] - (dr + rho * uy2);
  const R qx = R(0.5) * ((M[6] - rho * d3x) + (M[8] - rho * ux * (R(1) + uy2)));
  const R qy = R(0.5) * ((M[7] - rho * uy * (R(1) + ux2)) + (M[9] - rho * d3y));
  const R T = ((R(2) + M[3] + M[5]) * inv - ux2 - uy2) * R(0.5);
  out[0] = (float)dr;
  out[1] = (float)ux;
  out[2] = (float)uy;
  out[3] = (float)(T - R(1));
  out[4] = (float)pxx;
  out[5] = (float)pxy;
  out[6] = (float)pyy;
  out[7] = (float)qx;
  out[8] = (float)qy;
  out[15] = (float)sqrt(ux2 + uy2);
}

// Moments of cell (x, y) (FULL or the first three) from its own lattice; a
// gap cell (no fluid) gets zeros: rho 1, at rest.
template <int NL, int NH, bool FULL, class S, class R>
__device__ __forceinline__ int cell_moments(const Params<R>& p, const S* f0, const S* f1,
                                            const uint8_t* flag, int x, int y, R* M) {
  const int k = flag[x + (long long)p.nx * y];
  const size_t base = (size_t)(y + p.G) * p.pitch + (x + kOX);
  if (k == kFlagGap) {
#pragma unroll
    for (int q = 0; q < (FULL ? 10 : 3); ++q) M[q] = R(0);
  } else if (k) {
    raw_moments<NH, FULL, S, R>(p, p.lat[1], f1, base, M);
  } else {
    raw_moments<NL, FULL, S, R>(p, p.lat[0], f0, base, M);
  }
  return k;
}

__device__ __forceinline__ uint32_t pack2(__half lo, __half hi) {
  const __half2 h = __halves2half2(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&h);
}

// {relu(lo), relu(hi)} rounded to FP16 and packed (lo in the low half) by one
// conversion; the same bits as rounding max(v, 0).
__device__ __forceinline__ uint32_t pack2_relu(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// D += A (16 x 16, row-major, FP16) * B (16 x 8, column-major, FP16), FP32.
__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// D = A * B + C with C = {c0, c1, c0, c1}: a bias per output column pair.
__device__ __forceinline__ void mma16816_bias(float* d, const uint32_t* a, uint32_t b0,
                                              uint32_t b1, float c0, float c1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
      "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%10, %11, %10, %11};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1));
}

// B fragment of n-tile nt, k-rows k0 .. k0 + 15, of a row-major K x N weight
// matrix W: lane (g, t) holds W[k0 + 2t .. + 1][8 nt + g] and W[k0 + 2t + 8 .. + 9][8 nt + g].
__device__ __forceinline__ void bfrag(const __half* W, int ncols, int k0, int nt, int g, int t,
                                      uint32_t& b0, uint32_t& b1) {
  const int n = 8 * nt + g;
  b0 = pack2(W[(k0 + 2 * t) * ncols + n], W[(k0 + 2 * t + 1) * ncols + n]);
  b1 = pack2(W[(k0 + 2 * t + 8) * ncols + n], W[(k0 + 2 * t + 9) * ncols + n]);
}

// One tile per block pass.  First the moments of the tile's cells (the full
// set, kept in registers: each warp owns two rows of 32) and of the one-cell
// ring around it (periodic wrap, else the edge cell repeated; the ring's slots
// spread over the warps), with {dr, u_x, u_y} of every slot in shared memory;
// then per row lane l computes the features of cell x0 + l (gradients from the
// shared moments, a gap neighbour replaced by the cell itself) into shared
// memory (FP16), and the warp runs the MLP with the C fragments of one layer
// reused in registers as the A fragments of the next.  Outputs (any may be
// null): FP32 features (nc x 16, cell-major), logits, flags (logit > thr).
template <int NL, int NH, class S, class R>
__global__ void __launch_bounds__(kIndThreads)
k_indicator(const Params<R> p, const S* f0, const S* f1, const uint8_t* __restrict__ flag,
            const __half* __restrict__ w1, const float* __restrict__ b1,
            const __half* __restrict__ w2, const float* __restrict__ b2,
            const float* __restrict__ w3, float b3, float thr, float* feat_out,
            float* logit_out, uint8_t* flag_out) {
  constexpr int kRing = 2 * kHaloX + 2 * kIndTY;  // 100 slots
  constexpr int kRows = kIndTY / kIndWarps;        // rows per warp
  __shared__ R sm[kHaloY][kHaloX][3];
  __shared__ uint8_t sfl[kHaloY][kHaloX];
  __shared__ __align__(16) __half sfeat[kIndWarps][32][kFeat + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int ntx = (p.nx + kIndTX - 1) / kIndTX, nty = (p.ny + kIndTY - 1) / kIndTY;
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
  for (int tile = blockIdx.x; tile < ntx * nty; tile += gridDim.x) {
    const int x0 = (tile % ntx) * kIndTX, y0 = (tile / ntx) * kIndTY;
    // the ring: slot j on lane j / 8 of warp j % 8; top and bottom rows, then
    // the left and right columns.  A slot beyond the grid's last row or
    // column plus one is read by no cell and is skipped.
    for (int j = lane * kIndWarps + warp; j < kRing; j += 32 * kIndWarps) {
      int hx, hy;
      if (j < 2 * kHaloX) {
        hx = j % kHaloX;
        hy = j < kHaloX ? 0 : kHaloY - 1;
      } else {
        const int i = j - 2 * kHaloX;
        hx = i < kIndTY ? 0 : kHaloX - 1;
        hy = 1 + i % kIndTY;
      }
      const int rx = x0 - 1 + hx, ry = y0 - 1 + hy;
      if (rx > p.nx || ry > p.ny) continue;
      R m[3];
      const int k = cell_moments<NL, NH, false, S, R>(p, f0, f1, flag,
                                                      clampwrap(rx, p.nx, p.periodic_x),
                                                      clampwrap(ry, p.ny, p.periodic_y), m);
      const R inv = R(1) / (R(1) + m[0]);
      sm[hy][hx][0] = m[0];
      sm[hy][hx][1] = m[1] * inv;
      sm[hy][hx][2] = m[2] * inv;
      sfl[hy][hx] = (uint8_t)k;
    }
    // the tile's own slots: the full moments stay in registers (a slot one
    // past the grid's last column or row holds the wrapped or repeated cell)
    R Mi[kRows][10];
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr) {
      const int ly = warp + rr * kIndWarps;
      const int rx = x0 + lane, ry = y0 + ly;
#pragma unroll
      for (int q = 0; q < 10; ++q) Mi[rr][q] = R(0);
      if (rx > p.nx || ry > p.ny) continue;
      const int k = cell_moments<NL, NH, true, S, R>(p, f0, f1, flag,
                                                     clampwrap(rx, p.nx, p.periodic_x),
                                                     clampwrap(ry, p.ny, p.periodic_y), Mi[rr]);
      const R inv = R(1) / (R(1) + Mi[rr][0]);
      sm[ly + 1][lane + 1][0] = Mi[rr][0];
      sm[ly + 1][lane + 1][1] = Mi[rr][1] * inv;
      sm[ly + 1][lane + 1][2] = Mi[rr][2] * inv;
      sfl[ly + 1][lane + 1] = (uint8_t)k;
    }
    __syncthreads();
#pragma unroll
    for (int rr = 0; rr < kRows; ++rr) {
      const int ly = warp + rr * kIndWarps;
      const int x = x0 + lane, y = y0 + ly;
      const bool in = x < p.nx && y < p.ny;
      const long long c = x + (long long)p.nx * y;
      const int hx = lane + 1, hy = ly + 1;
      const int fc = in ? sfl[hy][hx] : (int)kFlagGap;
      float fe[kFeat];
#pragma unroll
      for (int q = 0; q < kFeat; ++q) fe[q] = 0.f;
      if (fc != kFlagGap) {
        if (fc) moment_features<NH, R>(p.lat[1], Mi[rr], fe);
        else moment_features<NL, R>(p.lat[0], Mi[rr], fe);
        // central differences; a gap neighbour (the wall side of a channel)
        // counts as the edge: the cell itself is repeated
        const R* own = sm[hy][hx];
        const R* xm = sfl[hy][hx - 1] == kFlagGap ? own : sm[hy][hx - 1];
        const R* xp = sfl[hy][hx + 1] == kFlagGap ? own : sm[hy][hx + 1];
        const R* ym = sfl[hy - 1][hx] == kFlagGap ? own : sm[hy - 1][hx];
        const R* yp = sfl[hy + 1][hx] == kFlagGap ? own : sm[hy + 1][hx];
        fe[9] = (float)(R(0.5) * (xp[0] - xm[0]));
        fe[10] = (float)(R(0.5) * (yp[0] - ym[0]));
        fe[11] = (float)(R(0.5) * (xp[1] - xm[1]));
        fe[12] = (float)(R(0.5) * (yp[1] - ym[1]));
        fe[13] = (float)(R(0.5) * (xp[2] - xm[2]));
        fe[14] = (float)(R(0.5) * (yp[2] - ym[2]));
#pragma unroll
        for (int q = 0; q < kFeat; ++q) fe[q] *= c_scale[q];
      }
      if (in && feat_out)
#pragma unroll
        for (int q = 0; q < kFeat; ++q) feat_out[c * kFeat + q] = fe[q];
#pragma unroll
      for (int q = 0; q < kFeat; q += 2)  // in pairs: 4-byte shared stores
        *reinterpret_cast<__half2*>(&sfeat[warp][lane][q]) = __floats2half2_rn(fe[q], fe[q + 1]);
      __syncwarp();
      if (have_w) {
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          const int r0 = 16 * mt + g, r1 = r0 + 8;
          uint32_t A[4];
          // pairs of features as 4-byte loads (rows of 18 halves keep them aligned)
          A[0] = *reinterpret_cast<const uint32_t*>(&sfeat[warp][r0][2 * t]);
          A[1] = *reinterpret_cast<const uint32_t*>(&sfeat[warp][r1][2 * t]);
          A[2] = *reinterpret_cast<const uint32_t*>(&sfeat[warp][r0][2 * t + 8]);
          A[3] = *reinterpret_cast<const uint32_t*>(&sfeat[warp][r1][2 * t + 8]);
          // layer 1: 16 -> 32, ReLU
          // (bias pairs as 8-byte loads: the pair index 8 nt + 2 t is even)
          float H1[4][4];
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const float2 bv = *reinterpret_cast<const float2*>(b1 + 8 * nt + 2 * t);
            mma16816_bias(H1[nt], A, B1[nt][0], B1[nt][1], bv.x, bv.y);
          }
          // layer 2: 32 -> 32, ReLU; the C fragments of layer 1, through the
          // ReLU and rounded to FP16, are its A fragments
          float H2[4][4];
#pragma unroll
          for (int kk = 0; kk < 2; ++kk) {
            uint32_t A2[4];
            A2[0] = pack2_relu(H1[2 * kk][0], H1[2 * kk][1]);
            A2[1] = pack2_relu(H1[2 * kk][2], H1[2 * kk][3]);
            A2[2] = pack2_relu(H1[2 * kk + 1][0], H1[2 * kk + 1][1]);
            A2[3] = pack2_relu(H1[2 * kk + 1][2], H1[2 * kk + 1][3]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
              if (kk == 0) {
                const float2 bv = *reinterpret_cast<const float2*>(b2 + 8 * nt + 2 * t);
                mma16816_bias(H2[nt], A2, B2[0][nt][0], B2[0][nt][1], bv.x, bv.y);
              } else {
                mma16816(H2[nt], A2, B2[1][nt][0], B2[1][nt][1]);
              }
            }
          }
          // output: 32 -> 1, reduced over the four lanes of a row group
          float o0 = 0.f, o1 = 0.f;
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            const float2 wv = *reinterpret_cast<const float2*>(w3 + 8 * nt + 2 * t);
            o0 += fmaxf(H2[nt][0], 0.f) * wv.x + fmaxf(H2[nt][1], 0.f) * wv.y;
            o1 += fmaxf(H2[nt][2], 0.f) * wv.x + fmaxf(H2[nt][3], 0.f) * wv.y;
          }
          o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
          o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
          o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
          o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
          if (t == 0 && y < p.ny) {
            // gap cells keep their flag and get logit 0
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = h ? r1 : r0;
              if (x0 + r >= p.nx) continue;
              const long long cr = x0 + r + (long long)p.nx * y;
              const bool gap = sfl[hy][r + 1] == kFlagGap;
              const float o = (h ? o1 : o0) + b3;
              if (logit_out) logit_out[cr] = gap ? 0.f : o;
              if (flag_out) flag_out[cr] = gap ? kFlagGap : (o > thr ? 1 : 0);
            }
          }
        }
      }
      __syncwarp();  // sfeat is rewritten by the warp's next row
    }
    __syncthreads();  // the shared moments are rewritten for the next tile
  }
}

// Refinement buffer of SLBM_CRIT_MLP_REFINE, one axis per launch (0 = x,
// 1 = y): out = 1 where `in` is 1 within r cells along the axis, the scan
// stopping at a gap cell or a bounded side (periodic axes wrap); also where
// keep = 1 (if given); gap cells stay gaps.
__global__ void k_dilate(const uint8_t* __restrict__ in, const uint8_t* __restrict__ keep,
                         uint8_t* __restrict__ out, int nx, int ny, int periodic, int r,
                         int axis) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= (long long)nx * ny) return;
  const int x = (int)(c % nx), y = (int)(c / nx);
  if (in[c] == kFlagGap) {
    out[c] = kFlagGap;
    return;
  }
  int v = in[c] == 1 || (keep && keep[c] == 1);
  const int n = axis ? ny : nx, i0 = axis ? y : x;
  for (int dir = -1; dir <= 1 && !v; dir += 2)
    for (int d = 1; d <= r; ++d) {
      int i = i0 + dir * d;
      if (i < 0 || i >= n) {
        if (!periodic) break;
        i = ((i % n) + n) % n;
      }
      const uint8_t f = in[axis ? x + (long long)nx * i : i + (long long)nx * y];
      if (f == kFlagGap) break;
      if (f == 1) {
        v = 1;
        break;
      }
    }
  out[c] = (uint8_t)v;
}

// Per-cell lattice loss between two buffers of the high-order planes (the
// stored values are deviations f - W, so the weights cancel in a - b and
// rho_a = 1 + sum a); FP64 sums.
template <class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_lattice_loss(const Params<R> p, const S* __restrict__ a, const S* __restrict__ b,
               const uint8_t* __restrict__ flag, double* __restrict__ out) {
  const int x = blockIdx.x * kTX + threadIdx.x, y = blockIdx.y * kTY + threadIdx.y;
  if (x >= p.nx || y >= p.ny) return;
  const long long c = x + (long long)p.nx * y;
  if (flag[c] == kFlagGap) {
    out[c] = 0.0;
    return;
  }
  const size_t base = (size_t)(y + p.G) * p.pitch + (x + kOX);
  const int q = p.lat[1].n * p.lat[1].n;
  double sa = 0.0, d2 = 0.0;
  for (int i = 0; i < q; ++i) {
    const double va = (double)from_s<R>(a[(size_t)i * p.plane + base], p.lat[1].sc[i]);
    const double vb = (double)from_s<R>(b[(size_t)i * p.plane + base], p.lat[1].sc[i]);
    sa += va;
    d2 += (va - vb) * (va - vb);
  }
  out[c] = sqrt(d2) / (1.0 + sa);
}

// ------------------------------------------------------------------ training
//
// Mini-batch Adam on the logistic loss, every step in one thread block (the
// steps are sequential, and a batch of at most 512 rows is a few MFLOP).  Per
// step:
//  F. warp w takes batch rows [w B/8, (w + 1) B/8) in m16 tiles: gathers the
//     rows' features (rounded to FP16) and labels, runs the forward pass with
//     each layer's C fragments reused as the next layer's A fragments, the
//     loss, and back-propagation: dlogit = p - y (the 1/B of the mean is
//     applied to the FP32 gradient, so the FP16 operands stay O(1)),
//     dZ2 = dlogit w3 [Z2 > 0], dH1 = dZ2 W2^T on the tensor cores,
//     dZ1 = dH1 [Z1 > 0].  Bias and output-layer gradients are summed in FP32
//     registers; X, H1, dZ2 and dZ1 go to shared memory transposed (FP16,
//     batch rows contiguous) for
//  G. the weight gradients dW2 = H1^T dZ2 (8 m16n8 tiles, one per warp) and
//     dW1 = X^T dZ1 (4 tiles, each over two halves of the batch), contracted
//     over the batch on the tensor cores;
//  A. Adam on every parameter (FP32 master weights and moments), then the
//     FP16 copies of W1 and W2 for the next step.
constexpr int kTrainWarps = 8;
constexpr int kTrainThreads = 32 * kTrainWarps;
constexpr int kOffB1 = kFeat * kHid, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid;
constexpr int kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid;
static_assert(kOffB3 + 1 == kMlpParams, "parameter layout");
constexpr int kParamPad = (kMlpParams + 3) / 4 * 4;
constexpr int kPartStride = 100;  // per warp: db1 (32), db2 (32), dw3 (32), db3, loss

size_t train_smem_bytes(int batch) {
  const size_t ld = (size_t)batch + 8;
  return sizeof(float) * (3 * kParamPad + kHid * kHid + 2 * kFeat * kHid +
                          kTrainWarps * kPartStride) +
         sizeof(__half) * (kFeat * kHid + kHid * kHid + (kFeat + 3 * kHid) * ld);
}

__device__ __forceinline__ uint32_t lds32(const __half* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// B fragment of the transposed weight W^T (W row-major K x N, here the
// contraction runs over W's columns): lane (g, t) holds W[8 nt + g][k0 + 2t .. + 1]
// and W[8 nt + g][k0 + 2t + 8 .. + 9].
__device__ __forceinline__ void bfrag_t(const __half* W, int ncols, int k0, int nt, int g, int t,
                                        uint32_t& b0, uint32_t& b1) {
  const __half* r = W + (8 * nt + g) * ncols + k0 + 2 * t;
  b0 = lds32(r);
  b1 = lds32(r + 8);
}

__device__ __forceinline__ float softplus(float v) {  // log(1 + e^v), stable
  return fmaxf(v, 0.f) + log1pf(expf(-fabsf(v)));
}

// sum over the 8 lanes of a column group (lanes with the same t)
__device__ __forceinline__ float sum_g(float v) {
  v += __shfl_xor_sync(0xffffffffu, v, 4);
  v += __shfl_xor_sync(0xffffffffu, v, 8);
  v += __shfl_xor_sync(0xffffffffu, v, 16);
  return v;
}

__global__ void __launch_bounds__(kTrainThreads, 1)
k_mlp_train(const float* __restrict__ x, const float* __restrict__ y,
            const int* __restrict__ idx, int steps, int B, float lr, float beta1, float beta2,
            float eps, int t0, float* __restrict__ params, float* __restrict__ adam,
            float* __restrict__ loss_out, float* __restrict__ grad_out) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int ld = B + 8;
  float* sw = reinterpret_cast<float*>(smem);  // master weights
  float* sm = sw + kParamPad;                  // Adam first moments
  float* sv = sm + kParamPad;                  // Adam second moments
  float* sg2 = sv + kParamPad;                 // dW2 (32 x 32)
  float* sg1 = sg2 + kHid * kHid;              // dW1, two batch halves (2 x 16 x 32)
  float* sp = sg1 + 2 * kFeat * kHid;          // per-warp partial sums
  __half* sw1h = reinterpret_cast<__half*>(sp + kTrainWarps * kPartStride);
  __half* sw2h = sw1h + kFeat * kHid;
  __half* sXt = sw2h + kHid * kHid;  // X^T (16 x ld)
  __half* sH1t = sXt + kFeat * ld;   // H1^T (32 x ld)
  __half* sD2t = sH1t + kHid * ld;   // dZ2^T
  __half* sD1t = sD2t + kHid * ld;   // dZ1^T
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int q = tid; q < kMlpParams; q += kTrainThreads) {
    const float w = params[q];
    sw[q] = w;
    sm[q] = adam[q];
    sv[q] = adam[kMlpParams + q];
    if (q < kOffB1) sw1h[q] = __float2half_rn(w);
    else if (q >= kOffW2 && q < kOffB2) sw2h[q - kOffW2] = __float2half_rn(w);
  }
  __syncthreads();
  const int RW = B / kTrainWarps;
  const float invB = 1.f / (float)B;
  for (int step = 0; step < steps; ++step) {
    const int* bidx = idx + (long long)step * B;
    // ---- F: forward and back-propagation over the warp's rows
    uint32_t B1[4][2], B2[2][4][2], BT[2][4][2];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) bfrag(sw1h, kHid, 0, nt, g, t, B1[nt][0], B1[nt][1]);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        bfrag(sw2h, kHid, 16 * kk, nt, g, t, B2[kk][nt][0], B2[kk][nt][1]);
        bfrag_t(sw2h, kHid, 16 * kk, nt, g, t, BT[kk][nt][0], BT[kk][nt][1]);
      }
    float acc_b1[4][2] = {}, acc_b2[4][2] = {}, acc_w3[4][2] = {};
    float acc_b3 = 0.f, acc_loss = 0.f;
    for (int mt = 0; mt < RW / 16; ++mt) {
      const int r0 = warp * RW + 16 * mt + g, r1 = r0 + 8;
      const long long s0 = bidx[r0], s1 = bidx[r1];
      const float2 xa = *reinterpret_cast<const float2*>(x + s0 * kFeat + 2 * t);
      const float2 xb = *reinterpret_cast<const float2*>(x + s1 * kFeat + 2 * t);
      const float2 xc = *reinterpret_cast<const float2*>(x + s0 * kFeat + 2 * t + 8);
      const float2 xd = *reinterpret_cast<const float2*>(x + s1 * kFeat + 2 * t + 8);
      const float y0 = y[s0], y1 = y[s1];
      const __half ha0 = __float2half_rn(xa.x), ha1 = __float2half_rn(xa.y);
      const __half hb0 = __float2half_rn(xb.x), hb1 = __float2half_rn(xb.y);
      const __half hc0 = __float2half_rn(xc.x), hc1 = __float2half_rn(xc.y);
      const __half hd0 = __float2half_rn(xd.x), hd1 = __float2half_rn(xd.y);
      const uint32_t A[4] = {pack2(ha0, ha1), pack2(hb0, hb1), pack2(hc0, hc1), pack2(hd0, hd1)};
      sXt[(2 * t) * ld + r0] = ha0;
      sXt[(2 * t + 1) * ld + r0] = ha1;
      sXt[(2 * t) * ld + r1] = hb0;
      sXt[(2 * t + 1) * ld + r1] = hb1;
      sXt[(2 * t + 8) * ld + r0] = hc0;
      sXt[(2 * t + 9) * ld + r0] = hc1;
      sXt[(2 * t + 8) * ld + r1] = hd0;
      sXt[(2 * t + 9) * ld + r1] = hd1;
      // layer 1
      float z1[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const float ba = sw[kOffB1 + 8 * nt + 2 * t], bb = sw[kOffB1 + 8 * nt + 2 * t + 1];
        z1[nt][0] = ba; z1[nt][1] = bb; z1[nt][2] = ba; z1[nt][3] = bb;
        mma16816(z1[nt], A, B1[nt][0], B1[nt][1]);
      }
      // H1 = relu(Z1) in FP16: layer 2's A fragments, and H1^T for dW2
      __half h1[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
        for (int q = 0; q < 4; ++q) h1[nt][q] = __float2half_rn(fmaxf(z1[nt][q], 0.f));
        const int col = 8 * nt + 2 * t;
        sH1t[col * ld + r0] = h1[nt][0];
        sH1t[(col + 1) * ld + r0] = h1[nt][1];
        sH1t[col * ld + r1] = h1[nt][2];
        sH1t[(col + 1) * ld + r1] = h1[nt][3];
      }
      float z2[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const float ba = sw[kOffB2 + 8 * nt + 2 * t], bb = sw[kOffB2 + 8 * nt + 2 * t + 1];
        z2[nt][0] = ba; z2[nt][1] = bb; z2[nt][2] = ba; z2[nt][3] = bb;
      }
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint32_t A2[4] = {pack2(h1[2 * kk][0], h1[2 * kk][1]),
                                pack2(h1[2 * kk][2], h1[2 * kk][3]),
                                pack2(h1[2 * kk + 1][0], h1[2 * kk + 1][1]),
                                pack2(h1[2 * kk + 1][2], h1[2 * kk + 1][3])};
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma16816(z2[nt], A2, B2[kk][nt][0], B2[kk][nt][1]);
      }
      // output layer (FP32), reduced over the four lanes of a row group
      float o0 = 0.f, o1 = 0.f;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const float wa = sw[kOffW3 + 8 * nt + 2 * t], wb = sw[kOffW3 + 8 * nt + 2 * t + 1];
        o0 += fmaxf(z2[nt][0], 0.f) * wa + fmaxf(z2[nt][1], 0.f) * wb;
        o1 += fmaxf(z2[nt][2], 0.f) * wa + fmaxf(z2[nt][3], 0.f) * wb;
      }
      o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
      o0 += __shfl_xor_sync(0xffffffffu, o0, 2);
      o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
      o1 += __shfl_xor_sync(0xffffffffu, o1, 2);
      const float zl0 = o0 + sw[kOffB3], zl1 = o1 + sw[kOffB3];
      // logistic loss log(1 + exp(-s z)), s = 2y - 1; dloss/dz = sigmoid(z) - y
      const float d0 = 1.f / (1.f + expf(-zl0)) - y0, d1 = 1.f / (1.f + expf(-zl1)) - y1;
      if (t == 0) {  // each row once
        acc_loss += softplus(-(2.f * y0 - 1.f) * zl0) + softplus(-(2.f * y1 - 1.f) * zl1);
        acc_b3 += d0 + d1;
      }
      float dz2[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const float wa = sw[kOffW3 + 8 * nt + 2 * t], wb = sw[kOffW3 + 8 * nt + 2 * t + 1];
        acc_w3[nt][0] += d0 * fmaxf(z2[nt][0], 0.f) + d1 * fmaxf(z2[nt][2], 0.f);
        acc_w3[nt][1] += d0 * fmaxf(z2[nt][1], 0.f) + d1 * fmaxf(z2[nt][3], 0.f);
        dz2[nt][0] = z2[nt][0] > 0.f ? d0 * wa : 0.f;
        dz2[nt][1] = z2[nt][1] > 0.f ? d0 * wb : 0.f;
        dz2[nt][2] = z2[nt][2] > 0.f ? d1 * wa : 0.f;
        dz2[nt][3] = z2[nt][3] > 0.f ? d1 * wb : 0.f;
        acc_b2[nt][0] += dz2[nt][0] + dz2[nt][2];
        acc_b2[nt][1] += dz2[nt][1] + dz2[nt][3];
      }
      __half hd2[4][4];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
#pragma unroll
        for (int q = 0; q < 4; ++q) hd2[nt][q] = __float2half_rn(dz2[nt][q]);
        const int col = 8 * nt + 2 * t;
        sD2t[col * ld + r0] = hd2[nt][0];
        sD2t[(col + 1) * ld + r0] = hd2[nt][1];
        sD2t[col * ld + r1] = hd2[nt][2];
        sD2t[(col + 1) * ld + r1] = hd2[nt][3];
      }
      // dH1 = dZ2 W2^T
      float dh1[4][4] = {};
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint32_t A3[4] = {pack2(hd2[2 * kk][0], hd2[2 * kk][1]),
                                pack2(hd2[2 * kk][2], hd2[2 * kk][3]),
                                pack2(hd2[2 * kk + 1][0], hd2[2 * kk + 1][1]),
                                pack2(hd2[2 * kk + 1][2], hd2[2 * kk + 1][3])};
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma16816(dh1[nt], A3, BT[kk][nt][0], BT[kk][nt][1]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float dz1[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) dz1[q] = z1[nt][q] > 0.f ? dh1[nt][q] : 0.f;
        acc_b1[nt][0] += dz1[0] + dz1[2];
        acc_b1[nt][1] += dz1[1] + dz1[3];
        const int col = 8 * nt + 2 * t;
        sD1t[col * ld + r0] = __float2half_rn(dz1[0]);
        sD1t[(col + 1) * ld + r0] = __float2half_rn(dz1[1]);
        sD1t[col * ld + r1] = __float2half_rn(dz1[2]);
        sD1t[(col + 1) * ld + r1] = __float2half_rn(dz1[3]);
      }
    }
    // the warp's partial sums of the bias and output-layer gradients
    float* pw = sp + warp * kPartStride;
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float v1 = sum_g(acc_b1[nt][j]), v2 = sum_g(acc_b2[nt][j]),
                    v3 = sum_g(acc_w3[nt][j]);
        if (g == 0) {
          pw[8 * nt + 2 * t + j] = v1;
          pw[32 + 8 * nt + 2 * t + j] = v2;
          pw[64 + 8 * nt + 2 * t + j] = v3;
        }
      }
    {
      const float vb = sum_g(acc_b3), vl = sum_g(acc_loss);
      if (lane == 0) {
        pw[96] = vb;
        pw[97] = vl;
      }
    }
    __syncthreads();
    // ---- G: weight gradients, contraction over the batch
    {
      const int mi = warp >> 2, ni = warp & 3;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int k0 = 0; k0 < B; k0 += 16) {
        const __half* h = sH1t + (16 * mi + g) * ld + k0 + 2 * t;
        const uint32_t A[4] = {lds32(h), lds32(h + 8 * ld), lds32(h + 8), lds32(h + 8 * ld + 8)};
        const __half* d = sD2t + (8 * ni + g) * ld + k0 + 2 * t;
        mma16816(acc, A, lds32(d), lds32(d + 8));
      }
      const int i0 = 16 * mi + g, j0 = 8 * ni + 2 * t;
      sg2[i0 * kHid + j0] = acc[0];
      sg2[i0 * kHid + j0 + 1] = acc[1];
      sg2[(i0 + 8) * kHid + j0] = acc[2];
      sg2[(i0 + 8) * kHid + j0 + 1] = acc[3];
      const int hh = warp >> 2;
      float a1[4] = {0.f, 0.f, 0.f, 0.f};
      for (int k0 = hh * (B / 2); k0 < (hh + 1) * (B / 2); k0 += 16) {
        const __half* h = sXt + g * ld + k0 + 2 * t;
        const uint32_t A[4] = {lds32(h), lds32(h + 8 * ld), lds32(h + 8), lds32(h + 8 * ld + 8)};
        const __half* d = sD1t + (8 * ni + g) * ld + k0 + 2 * t;
        mma16816(a1, A, lds32(d), lds32(d + 8));
      }
      float* s1 = sg1 + hh * kFeat * kHid;
      s1[g * kHid + j0] = a1[0];
      s1[g * kHid + j0 + 1] = a1[1];
      s1[(g + 8) * kHid + j0] = a1[2];
      s1[(g + 8) * kHid + j0 + 1] = a1[3];
    }
    __syncthreads();
    // ---- A: Adam (bias corrections of step t0 + step + 1)
    const float bc1 = 1.f - powf(beta1, (float)(t0 + step + 1));
    const float bc2 = 1.f - powf(beta2, (float)(t0 + step + 1));
    for (int q = tid; q < kMlpParams; q += kTrainThreads) {
      float gq = 0.f;
      if (q < kOffB1) {
        gq = sg1[q] + sg1[kFeat * kHid + q];
      } else if (q >= kOffW2 && q < kOffB2) {
        gq = sg2[q - kOffW2];
      } else {
        const int slot = q < kOffW2 ? q - kOffB1
                         : q < kOffW3 ? 32 + q - kOffB2
                         : q < kOffB3 ? 64 + q - kOffW3 : 96;
        for (int w = 0; w < kTrainWarps; ++w) gq += sp[w * kPartStride + slot];
      }
      gq *= invB;
      if (grad_out && step == steps - 1) grad_out[q] = gq;
      const float m = beta1 * sm[q] + (1.f - beta1) * gq;
      const float v = beta2 * sv[q] + (1.f - beta2) * gq * gq;
      sm[q] = m;
      sv[q] = v;
      const float w = sw[q] - lr * (m / bc1) / (sqrtf(v / bc2) + eps);
      sw[q] = w;
      if (q < kOffB1) sw1h[q] = __float2half_rn(w);
      else if (q >= kOffW2 && q < kOffB2) sw2h[q - kOffW2] = __float2half_rn(w);
    }
    if (tid == 0 && loss_out) {
      float l = 0.f;
      for (int w = 0; w < kTrainWarps; ++w) l += sp[w * kPartStride + 97];
      loss_out[step] = l * invB;
    }
    __syncthreads();
  }
  for (int q = tid; q < kMlpParams; q += kTrainThreads) {
    params[q] = sw[q];
    adam[q] = sm[q];
    adam[kMlpParams + q] = sv[q];
  }
}

}  // namespace

template <class S, class R>
cudaError_t launch_indicator(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                             const IndicatorDev& w, float thr, float* feat_out, float* logit_out,
                             uint8_t* flag_out, cudaStream_t st) {
  const long long ntiles = (long long)((p.nx + kIndTX - 1) / kIndTX) * ((p.ny + kIndTY - 1) / kIndTY);
  long long blocks = ntiles;
  const long long cap = (long long)p.nsm * 8;
  if (blocks > cap) blocks = cap;
  const int nl = p.lat[0].n, nh = p.lat[1].n;
#define SLBM_IND_CASE(NL, NH)                                                                 \
  if (nl == NL && nh == NH) {                                                                 \
    k_indicator<NL, NH, S, R><<<(unsigned)blocks, kIndThreads, 0, st>>>(                      \
        p, f0, f1, flag, w.w1, w.b1, w.w2, w.b2, w.w3, w.b3, thr, feat_out, logit_out,         \
        flag_out);                                                                            \
    return cudaGetLastError();                                                                \
  }
  SLBM_IND_CASE(3, 4)
  SLBM_IND_CASE(3, 5)
  SLBM_IND_CASE(4, 5)
#undef SLBM_IND_CASE
  return cudaErrorInvalidValue;
}

template <class S, class R>
cudaError_t launch_lattice_loss(const Params<R>& p, const S* a, const S* b, const uint8_t* flag,
                                double* out, cudaStream_t st) {
  const dim3 tg((p.nx + kTX - 1) / kTX, (p.ny + kTY - 1) / kTY);
  k_lattice_loss<S, R><<<tg, dim3(kTX, kTY), 0, st>>>(p, a, b, flag, out);
  return cudaGetLastError();
}

cudaError_t launch_dilate(const uint8_t* in, const uint8_t* keep, uint8_t* out, int nx, int ny,
                          int periodic, int r, int axis, cudaStream_t st) {
  const long long nc = (long long)nx * ny;
  k_dilate<<<(unsigned)((nc + 255) / 256), 256, 0, st>>>(in, keep, out, nx, ny, periodic, r, axis);
  return cudaGetLastError();
}

cudaError_t launch_mlp_train(const float* x, const float* y, const int* idx, int steps, int batch,
                             float lr, float beta1, float beta2, float eps, int t0, float* params,
                             float* adam, float* loss, float* grad, cudaStream_t st) {
  if (batch < 16 * kTrainWarps || batch > kMlpMaxBatch || batch % (16 * kTrainWarps))
    return cudaErrorInvalidValue;
  const size_t smem = train_smem_bytes(batch);
  cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)train_smem_bytes(kMlpMaxBatch));
  if (e != cudaSuccess) return e;
  k_mlp_train<<<1, kTrainThreads, smem, st>>>(x, y, idx, steps, batch, lr, beta1, beta2, eps, t0,
                                              params, adam, loss, grad);
  return cudaGetLastError();
}

#define SLBM_IND_INST(S, R)                                                                  \
  template cudaError_t launch_indicator<S, R>(const Params<R>&, const S*, const S*,          \
                                              const uint8_t*, const IndicatorDev&, float,     \
                                              float*, float*, uint8_t*, cudaStream_t);        \
  template cudaError_t launch_lattice_loss<S, R>(const Params<R>&, const S*, const S*,       \
                                                 const uint8_t*, double*, cudaStream_t);
SLBM_IND_INST(float, float)
SLBM_IND_INST(double, double)
SLBM_IND_INST(__half, float)
SLBM_IND_INST(fx16, float)
#undef SLBM_IND_INST

}  // namespace slbm
