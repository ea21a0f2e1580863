// slbm_post.cuh -- the post-step kernel: interface conversion (step 2 of
// Sec. III.D) plus the ghost images of boundary cells, templated on the
// lattice pair so every per-cell array lives in registers.
//
// After the stream-collide kernel has written every cell's populations in the
// lattice it was computed in (flag_old), one thread per cell:
//  1. decides from the new flags whether the cell is in the band (a cell of
//     the other lattice within the stencil reach reads it) or flipped;
//  2. converts (lift, Sec. III.B / project, Sec. III.C) so that every node a
//     cell reads next step exists in the reader's lattice -- a flipped node in
//     the band is read as the conversion of its new populations;
//  3. if the cell lies within G of the edge, writes its ghost images: periodic
//     images and OUTFLOW copies (all planes of both lattices), and the INLET
//     equilibrium ghosts, which take the cell's own density.  DIRICHLET
//     ghosts are constant and written once by the setup ghost kernel.
#pragma once

#include "../../include/slbm.h"
#include "slbm_eq.cuh"

namespace slbm {

constexpr int kBandMax = 3;  // largest stencil reach (order 5)

template <int NQ, int NQQ, class R>
struct PostMath {
  // Lifting f_q -> f_Q on deviations: f^L_Q + L (f_q - f^L_q) L^T (moment sums FP64).
  static __device__ __forceinline__ void lift(const Params<R>& p, const R (*sq)[kMaxN],
                                              R (*sQ)[kMaxN]) {
    const LatTab<R>& Lq = p.lat[0];
    double dr = 0.0, mx = 0.0, my = 0.0;
#pragma unroll
    for (int iy = 0; iy < NQ; ++iy)
#pragma unroll
      for (int ix = 0; ix < NQ; ++ix) {
        const double v = (double)sq[iy][ix];
        dr += v;
        mx += (double)Lq.c[ix] * v;
        my += (double)Lq.c[iy] * v;
      }
    const R inv = R(1) / (R)(1.0 + dr);
    const R ux = (R)mx * inv, uy = (R)my * inv;
    R eq[kMaxN][kMaxN], A[kMaxN][kMaxN];
    eq_dev<R>(Lq, NQ, (R)dr, ux, uy, eq);
#pragma unroll
    for (int iy = 0; iy < NQ; ++iy)
#pragma unroll
      for (int ix = 0; ix < NQ; ++ix) eq[iy][ix] = sq[iy][ix] - eq[iy][ix];  // non-equilibrium
    eq_dev<R>(p.lat[1], NQQ, (R)dr, ux, uy, sQ);
#pragma unroll
    for (int ay = 0; ay < NQQ; ++ay)
#pragma unroll
      for (int jx = 0; jx < NQ; ++jx) {
        R t = R(0);
#pragma unroll
        for (int jy = 0; jy < NQ; ++jy) t += p.conv.lift[ay][jy] * eq[jy][jx];
        A[ay][jx] = t;
      }
#pragma unroll
    for (int ay = 0; ay < NQQ; ++ay)
#pragma unroll
      for (int ax = 0; ax < NQQ; ++ax) {
        R t = R(0);
#pragma unroll
        for (int jx = 0; jx < NQ; ++jx) t += p.conv.lift[ax][jx] * A[ay][jx];
        sQ[ay][ax] += t;
      }
  }

  // Projection f_Q -> f_q: P F_Q P^T, P[j][a] = l^q_j(c^Q_a).
  static __device__ __forceinline__ void project(const Params<R>& p, const R (*sQ)[kMaxN],
                                                 R (*sq)[kMaxN]) {
    R A[kMaxN][kMaxN];
#pragma unroll
    for (int jy = 0; jy < NQ; ++jy)
#pragma unroll
      for (int ax = 0; ax < NQQ; ++ax) {
        R t = R(0);
#pragma unroll
        for (int ay = 0; ay < NQQ; ++ay) t += p.conv.proj[jy][ay] * sQ[ay][ax];
        A[jy][ax] = t;
      }
#pragma unroll
    for (int jy = 0; jy < NQ; ++jy)
#pragma unroll
      for (int jx = 0; jx < NQ; ++jx) {
        R t = R(0);
#pragma unroll
        for (int ax = 0; ax < NQQ; ++ax) t += p.conv.proj[jx][ax] * A[jy][ax];
        sq[jy][jx] = t;
      }
  }
};

template <int N, class S, class R>
__device__ __forceinline__ void load_t(const S* f, long long plane, int base, R (*s)[kMaxN]) {
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix) s[iy][ix] = static_cast<R>(f[(size_t)(ix + N * iy) * plane + base]);
}

template <int N, class S, class R>
__device__ __forceinline__ void store_t(S* f, long long plane, int base, const R (*s)[kMaxN]) {
#pragma unroll
  for (int iy = 0; iy < N; ++iy)
#pragma unroll
    for (int ix = 0; ix < N; ++ix) f[(size_t)(ix + N * iy) * plane + base] = static_cast<S>(s[iy][ix]);
}

// Ghost coordinates along one axis that are copies of interior coordinate v
// (periodic images, OUTFLOW extrapolation), v itself first.  Returns count.
__device__ __forceinline__ int copy_images(int v, int n, int G, int periodic, int kind_lo,
                                           int kind_hi, int* out) {
  int c = 0;
  out[c++] = v;
  if (periodic) {
    if (v < G) out[c++] = v + n;
    if (v >= n - G) out[c++] = v - n;
  } else {
    if (v == 0 && kind_lo == SLBM_BC_OUTFLOW)
      for (int g = 1; g <= G; ++g) out[c++] = -g;
    if (v == n - 1 && kind_hi == SLBM_BC_OUTFLOW)
      for (int g = 0; g < G; ++g) out[c++] = n + g;
  }
  return c;
}

template <int NL, int NH, class S, class R>
__device__ void write_eq_t(const Params<R>& p, S* f0, S* f1, int base, R dr, R ux, R uy) {
  R e[kMaxN][kMaxN];
  eq_dev<R>(p.lat[0], NL, dr, ux, uy, e);
  store_t<NL, S, R>(f0, p.plane, base, e);
  eq_dev<R>(p.lat[1], NH, dr, ux, uy, e);
  store_t<NH, S, R>(f1, p.plane, base, e);
}

// Ghost images of boundary cell (x, y) (see the file comment).
template <int NL, int NH, class S, class R>
__device__ void boundary_images(const Params<R>& p, S* f0, S* f1, const BcDev& bc, int x, int y,
                                int flag) {
  const int G = p.G;
  int xs[2 * kBandMax + 2], ys[2 * kBandMax + 2];
  const int nxc = copy_images(x, p.nx, G, p.periodic_x, bc.kind[SLBM_SIDE_XMIN],
                              bc.kind[SLBM_SIDE_XMAX], xs);
  const int nyc = copy_images(y, p.ny, G, p.periodic_y, bc.kind[SLBM_SIDE_YMIN],
                              bc.kind[SLBM_SIDE_YMAX], ys);
  const int src = (y + G) * p.pitch + (x + kOX);
  constexpr int QL = NL * NL, QH = NH * NH;
  if (nxc > 1 || nyc > 1) {
    // all loads first: stores through f0 / f1 may alias later loads for the
    // compiler, which would otherwise serialise one L2 round trip per plane
    S v0[QL], v1[QH];
#pragma unroll
    for (int i = 0; i < QL; ++i) v0[i] = f0[(size_t)i * p.plane + src];
#pragma unroll
    for (int i = 0; i < QH; ++i) v1[i] = f1[(size_t)i * p.plane + src];
    for (int a = 0; a < nyc; ++a)
      for (int b = 0; b < nxc; ++b) {
        if (a == 0 && b == 0) continue;
        const int dst = (ys[a] + G) * p.pitch + (xs[b] + kOX);
#pragma unroll
        for (int i = 0; i < QL; ++i) f0[(size_t)i * p.plane + dst] = v0[i];
#pragma unroll
        for (int i = 0; i < QH; ++i) f1[(size_t)i * p.plane + dst] = v1[i];
      }
  }
  // INLET sides: equilibrium at the prescribed velocity and this cell's density
  const bool inx0 = !p.periodic_x && x == 0 && bc.kind[SLBM_SIDE_XMIN] == SLBM_BC_INLET;
  const bool inx1 = !p.periodic_x && x == p.nx - 1 && bc.kind[SLBM_SIDE_XMAX] == SLBM_BC_INLET;
  const bool iny0 = !p.periodic_y && y == 0 && bc.kind[SLBM_SIDE_YMIN] == SLBM_BC_INLET;
  const bool iny1 = !p.periodic_y && y == p.ny - 1 && bc.kind[SLBM_SIDE_YMAX] == SLBM_BC_INLET;
  if (!(inx0 || inx1 || iny0 || iny1)) return;
  double r = 0.0;
  if (flag) {
#pragma unroll
    for (int i = 0; i < QH; ++i) r += (double)f1[(size_t)i * p.plane + src];
  } else {
#pragma unroll
    for (int i = 0; i < QL; ++i) r += (double)f0[(size_t)i * p.plane + src];
  }
  const R dr = (R)r;
  if (inx0 || inx1) {  // x side: rows = this row and its copy-type y images
    const int side = inx0 ? SLBM_SIDE_XMIN : SLBM_SIDE_XMAX;
    const R ux = (R)bc.ux[side][y], uy = (R)bc.uy[side][y];
    for (int a = 0; a < nyc; ++a)
      for (int g = 1; g <= G; ++g) {
        const int gx = inx0 ? -g : p.nx - 1 + g;
        write_eq_t<NL, NH, S, R>(p, f0, f1, (ys[a] + G) * p.pitch + (gx + kOX), dr, ux, uy);
      }
  }
  if (iny0 || iny1) {  // y side wins at corners: columns = copy images and clamped corners
    const int side = iny0 ? SLBM_SIDE_YMIN : SLBM_SIDE_YMAX;
    const R ux = (R)bc.ux[side][x], uy = (R)bc.uy[side][x];
    int cols[2 * kBandMax + 2];
    int nc = 0;
    cols[nc++] = x;
    if (p.periodic_x) {
      if (x < G) cols[nc++] = x + p.nx;
      if (x >= p.nx - G) cols[nc++] = x - p.nx;
    } else {
      if (x == 0)
        for (int g = 1; g <= G; ++g) cols[nc++] = -g;
      if (x == p.nx - 1)
        for (int g = 0; g < G; ++g) cols[nc++] = p.nx + g;
    }
    for (int b = 0; b < nc; ++b)
      for (int g = 1; g <= G; ++g) {
        const int gy = iny0 ? -g : p.ny - 1 + g;
        write_eq_t<NL, NH, S, R>(p, f0, f1, (gy + G) * p.pitch + (cols[b] + kOX), dr, ux, uy);
      }
  }
}

template <int NL, int NH, class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_post(const Params<R> p, S* f0, S* f1, const uint8_t* __restrict__ flag_old,
       const uint8_t* __restrict__ flag_new, const BcDev bc, int images,
       uint8_t* __restrict__ tile_mask) {
  __shared__ uint8_t sf[kTY + 2 * kBandMax][kTX + 2 * kBandMax];
  const int B = p.band;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  // new flags of the tile and its band-wide halo (outside the grid: a
  // non-periodic side reads as "same as the cell", i.e. never a band reason)
  for (int t = threadIdx.y * kTX + threadIdx.x; t < (kTY + 2 * B) * (kTX + 2 * B);
       t += kTX * kTY) {
    const int ly = t / (kTX + 2 * B), lx = t % (kTX + 2 * B);
    int gx = x0 + lx - B, gy = y0 + ly - B;
    uint8_t v = 2;
    bool ok = true;
    if (gx < 0 || gx >= p.nx) {
      if (p.periodic_x) gx = gx < 0 ? gx + p.nx : gx - p.nx;
      else ok = false;
    }
    if (gy < 0 || gy >= p.ny) {
      if (p.periodic_y) gy = gy < 0 ? gy + p.ny : gy - p.ny;
      else ok = false;
    }
    if (ok) v = flag_new[gx + p.nx * gy];
    sf[ly][lx] = v;
  }
  __syncthreads();
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  const bool in = x < p.nx && y < p.ny;
  const int nw = in ? sf[threadIdx.y + B][threadIdx.x + B] : 2;
  // which lattices the next step's tile holds (read by the stream kernel's
  // producer to choose the planes it stages)
  const int any_lo = __syncthreads_or(nw == 0);
  const int any_hi = __syncthreads_or(nw == 1);
  if (threadIdx.x == 0 && threadIdx.y == 0)
    tile_mask[blockIdx.y * gridDim.x + blockIdx.x] = (uint8_t)(any_lo | (any_hi << 1));
  if (!in) return;
  const int c = x + p.nx * y;
  const int old = flag_old[c];
  bool band = false;
  for (int dy = -B; dy <= B; ++dy)
    for (int dx = -B; dx <= B; ++dx) {
      const int v = sf[threadIdx.y + B + dy][threadIdx.x + B + dx];
      band |= (v != 2) && (v != nw);
    }
  const int base = (y + p.G) * p.pitch + (x + kOX);
  if (old != nw || band) {
    R a[kMaxN][kMaxN], b[kMaxN][kMaxN];
    using M = PostMath<NL, NH, R>;
    if (old == 0) {
      load_t<NL, S, R>(f0, p.plane, base, a);
      M::lift(p, a, b);
      store_t<NH, S, R>(f1, p.plane, base, b);
      if (old != nw && band) {  // now high-order; low-order readers see its projection
        M::project(p, b, a);
        store_t<NL, S, R>(f0, p.plane, base, a);
      }
    } else {
      load_t<NH, S, R>(f1, p.plane, base, b);
      M::project(p, b, a);
      store_t<NL, S, R>(f0, p.plane, base, a);
      if (old != nw && band) {  // now low-order; high-order readers see its lifting
        M::lift(p, a, b);
        store_t<NH, S, R>(f1, p.plane, base, b);
      }
    }
  }
  if (images && (x < p.G || x >= p.nx - p.G || y < p.G || y >= p.ny - p.G))
    boundary_images<NL, NH, S, R>(p, f0, f1, bc, x, y, nw);
}

template <class S, class R>
cudaError_t launch_post_impl(const Params<R>& p, S* f0, S* f1, const uint8_t* flag_old,
                             const uint8_t* flag_new, const BcDev& bc, int images,
                             uint8_t* tile_mask, cudaStream_t st) {
  const dim3 blk(kTX, kTY), grd((p.nx + kTX - 1) / kTX, (p.ny + kTY - 1) / kTY);
  const int nl = p.lat[0].n, nh = p.lat[1].n;
#define SLBM_POST_CASE(NL, NH)                                                              \
  if (nl == NL && nh == NH) {                                                               \
    k_post<NL, NH, S, R>                                                                    \
        <<<grd, blk, 0, st>>>(p, f0, f1, flag_old, flag_new, bc, images, tile_mask);        \
    return cudaGetLastError();                                                              \
  }
  SLBM_POST_CASE(3, 4)
  SLBM_POST_CASE(3, 5)
  SLBM_POST_CASE(4, 5)
#undef SLBM_POST_CASE
  return cudaErrorInvalidValue;
}

}  // namespace slbm
