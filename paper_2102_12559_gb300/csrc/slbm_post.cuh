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
//  3. if the cell lies within G of the edge, writes its ghost images:
//     periodic images and OUTFLOW copies (all planes of both lattices) and the
//     INLET equilibrium ghosts, which take the cell's own density.  DIRICHLET
//     ghosts are constant and written once by the setup ghost kernel.
#pragma once

#include <mutex>

#include "../../include/slbm.h"
#include "slbm_ghost.cuh"

namespace slbm {

template <int NQ, int NQQ, class R>
struct PostMath {
  // Lifting f_q -> f_Q on deviations: f^L_Q + L (f_q - f^L_q) L^T (moment
  // sums in twice the working precision for FP32, see MomentAcc).
  static __device__ __forceinline__ void lift(const Params<R>& p, const R (*sq)[kMaxN],
                                              R (*sQ)[kMaxN]) {
    const LatTab<R>& Lq = p.lat[0];
    MomentAcc<R> ar, ax, ay;
#pragma unroll
    for (int iy = 0; iy < NQ; ++iy)
#pragma unroll
      for (int ix = 0; ix < NQ; ++ix) {
        const R v = sq[iy][ix];
        ar.add(v);
        ax.add_product(Lq.c[ix], v);
        ay.add_product(Lq.c[iy], v);
      }
    const R dr = ar.value();
    const R inv = R(1) / (R(1) + dr);
    const R ux = ax.value() * inv, uy = ay.value() * inv;
    R eq[kMaxN][kMaxN], A[kMaxN][kMaxN];
    eq_dev<R>(Lq, NQ, dr, ux, uy, eq);
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

constexpr int kPostMaxTiles = 1024;  // tiles one persistent post CTA may own

// The work of one tile (tile origin x0, y0): stage the new flags of the tile
// and its band-wide halo, convert band / flipped cells, and in setup calls
// write the tile's lattice mask.  The work word (if `work_word` is given; a
// tile whose word is not work returns false after the first barrier) is
// fetched with the staged flags, so their latencies overlap.
template <int NL, int NH, class S, class R>
__device__ __forceinline__ bool post_tile(const Params<R>& p, S* f0, S* f1,
                                          const uint8_t* __restrict__ flag_old,
                                          const uint8_t* __restrict__ flag_new, const BcDev& bc,
                                          int images, bool setup, uint8_t* mask_out, int x0,
                                          int y0, uint8_t (*sf)[kTX + 2 * kBandMax],
                                          const int* work_word = nullptr) {
  const int B = p.band;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  const bool in = x < p.nx && y < p.ny;
  const int wv = work_word ? *work_word : 4;
  const int old = in ? flag_old[x + p.nx * y] : 2;
  // new flags of the tile and its band-wide halo (outside the grid: a
  // non-periodic side reads as "same as the cell", i.e. never a band reason)
#pragma unroll
  for (int r = 0; r < ((kTY + 2 * kBandMax) * (kTX + 2 * kBandMax) + kTX * kTY - 1) / (kTX * kTY);
       ++r) {
    const int t = threadIdx.y * kTX + threadIdx.x + r * kTX * kTY;
    if (t >= (kTY + 2 * B) * (kTX + 2 * B)) break;
    const int ly = t / (kTX + 2 * B), lx = t % (kTX + 2 * B);
    int gx = x0 + lx - B, gy = y0 + ly - B;
    uint8_t v = 2;
    bool ok = true;
    // periodic images by a full modulo: on a grid narrower than the staged
    // halo one wrap is not enough (those positions are read by no valid cell,
    // but they must stay inside the flag array)
    if (gx < 0 || gx >= p.nx) {
      if (p.periodic_x) gx = ((gx % p.nx) + p.nx) % p.nx;
      else ok = false;
    }
    if (gy < 0 || gy >= p.ny) {
      if (p.periodic_y) gy = ((gy % p.ny) + p.ny) % p.ny;
      else ok = false;
    }
    if (ok) v = flag_new[gx + p.nx * gy];
    sf[ly][lx] = v;
  }
  __syncthreads();
  if (!post_work_word(wv)) {  // all high-order neighbourhood (uniform per CTA)
    __syncthreads();          // sf is reused by the next tile
    return false;
  }
  const int nw = in ? sf[threadIdx.y + B][threadIdx.x + B] : 2;
  if (setup) {  // the lattices the next step's tile holds (read by the stream kernel)
    const int any_lo = __syncthreads_or(nw == 0);
    const int any_hi = __syncthreads_or(nw == 1);
    if (threadIdx.x == 0 && threadIdx.y == 0) *mask_out = (uint8_t)(any_lo | (any_hi << 1));
  }
  // cells that need a conversion, compacted onto the leading threads (the
  // ones computed in the low-order lattice first), so that one or two warps
  // of the tile do the arithmetic: entry = cell | old << 8 | nw << 9 | band << 10
  __shared__ int s_conv[kTX * kTY];
  __shared__ int s_cnt[2][kTY];
  const int tid = threadIdx.y * kTX + threadIdx.x;
  bool conv = false, band = false;
  if (in) {
    for (int dy = -B; dy <= B; ++dy)
      for (int dx = -B; dx <= B; ++dx) {
        const int u = sf[threadIdx.y + B + dy][threadIdx.x + B + dx];
        band |= (u != 2) && (u != nw);
      }
    conv = nw != kFlagGap && old != kFlagGap && (old != nw || band);
  }
  const unsigned b0 = __ballot_sync(0xffffffffu, conv && old == 0);
  const unsigned b1 = __ballot_sync(0xffffffffu, conv && old != 0);
  if (threadIdx.x == 0) {
    s_cnt[0][threadIdx.y] = __popc(b0);
    s_cnt[1][threadIdx.y] = __popc(b1);
  }
  __syncthreads();
  int n0 = 0, n1 = 0, pre0 = 0, pre1 = 0;
#pragma unroll
  for (int w = 0; w < kTY; ++w) {
    const int c0 = s_cnt[0][w], c1 = s_cnt[1][w];
    if (w < (int)threadIdx.y) {
      pre0 += c0;
      pre1 += c1;
    }
    n0 += c0;
    n1 += c1;
  }
  if (conv) {
    const unsigned lt = (1u << threadIdx.x) - 1u;
    const int slot = old == 0 ? pre0 + __popc(b0 & lt) : n0 + pre1 + __popc(b1 & lt);
    s_conv[slot] = tid | (old << 8) | (nw << 9) | ((int)band << 10);
  }
  __syncthreads();
  if (tid < n0 + n1) {
    const int e = s_conv[tid];
    const int cell = e & 255, o = (e >> 8) & 1, nn = (e >> 9) & 1, bd = (e >> 10) & 1;
    const int cx = x0 + (cell & (kTX - 1)), cy = y0 + cell / kTX;
    const int base = (cy + p.G) * p.pitch + (cx + kOX);
    R a[kMaxN][kMaxN], b[kMaxN][kMaxN];
    using M = PostMath<NL, NH, R>;
    if (o == 0) {
      load_t<NL, S, R>(p.lat[0], f0, p.plane, base, a);
      M::lift(p, a, b);
      store_t<NH, S, R>(p.lat[1], f1, p.plane, base, b);
      if (o != nn && bd) {  // now high-order; low-order readers see its projection
        M::project(p, b, a);
        store_t<NL, S, R>(p.lat[0], f0, p.plane, base, a);
      }
    } else {
      load_t<NH, S, R>(p.lat[1], f1, p.plane, base, b);
      M::project(p, b, a);
      store_t<NL, S, R>(p.lat[0], f0, p.plane, base, a);
      if (o != nn && bd) {  // now low-order; high-order readers see its lifting
        M::lift(p, a, b);
        store_t<NH, S, R>(p.lat[1], f1, p.plane, base, b);
      }
    }
  }
  __syncthreads();  // sf is reused by the next tile
  return true;
}

// Persistent post-step kernel: CTA c owns tiles c, c + gridDim.x, ...  After a
// step (mask_in set) a prologue derives every owned tile's work flag from the
// stream kernel's masks -- a flip in the tile, or both lattices in its 3 x 3
// tile neighbourhood (the band radius is below the tile size) -- with all
// mask loads independent; quiet tiles then cost nothing.  Setup calls
// (mask_in null) visit every tile and write its lattice mask.  Ghost rings are
// refreshed afterwards by the halo kernel.
template <int NL, int NH, class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_post(const Params<R> p, S* f0, S* f1, const uint8_t* __restrict__ flag_old,
       const uint8_t* __restrict__ flag_new, const BcDev bc, int images,
       const uint8_t* __restrict__ mask_in, uint8_t* __restrict__ tile_mask, int ntx, int nty) {
  __shared__ uint8_t sf[kTY + 2 * kBandMax][kTX + 2 * kBandMax];
  __shared__ int work[kPostMaxTiles];
  const int ntiles = ntx * nty;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int M = ((int)blockIdx.x < ntiles) ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  for (int m = tid; m < M; m += kTX * kTY) work[m] = mask_in ? 0 : 1;
  __syncthreads();
  if (mask_in) {
    for (int e = tid; e < 9 * M; e += kTX * kTY) {
      const int m = e / 9, q = e % 9;
      const int t = (int)blockIdx.x + m * (int)gridDim.x;
      const int bx = t % ntx, by = t / ntx;
      int tx = bx + q % 3 - 1, ty = by + q / 3 - 1;
      if (tx < 0 || tx >= ntx) tx = p.periodic_x ? (tx < 0 ? tx + ntx : tx - ntx) : bx;
      if (ty < 0 || ty >= nty) ty = p.periodic_y ? (ty < 0 ? ty + nty : ty - nty) : by;
      const int mv = __ldg(mask_in + ty * ntx + tx);
      // bit 0/1: lattices seen; bit 2: this tile flipped
      atomicOr(&work[m], (mv & 3) | (q == 4 ? (mv & 4) : 0));
    }
    __syncthreads();
  }
  for (int m = 0; m < M; ++m) {
    const int t = (int)blockIdx.x + m * (int)gridDim.x;
    const int x0 = (t % ntx) * kTX, y0 = (t / ntx) * kTY;
    const int wv = work[m];
    if (mask_in && !((wv & 4) || (wv & 3) == 3)) continue;  // uniform per CTA
    post_tile<NL, NH, S, R>(p, f0, f1, flag_old, flag_new, bc, images, mask_in == nullptr,
                            tile_mask + t, x0, y0, sf);
  }
}

// Ghost images of the sources in one tile: the n ring cells idx[0..n) whose
// source cell lies in the tile, every plane of both lattices.  Under the
// ghost rule (ghost_source) copy ghosts copy their interior source; INLET
// ghosts are the plane's lattice equilibrium at the source's density (its own
// lattice's populations summed) and the side's velocity; DIFFUSE ghosts are
// diffuse_value; DIRICHLET ghosts are constant and in no list.  Per chunk of
// up to one ghost cell per thread: the cells' source, target and inputs into
// shared memory, then the elements (ghost cell, plane) over the threads, four
// at a time with every load before the stores (the stores may alias the loads
// for the compiler, which would otherwise serialise one L2 round trip per
// element).  Interior values are read through L2 (ld.global.cg): other
// threads of the CTA have just written them.
template <int NL, int NH, class S, class R>
__device__ __forceinline__ void tile_ghosts(const Params<R>& p, S* f0, S* f1,
                                            const uint8_t* __restrict__ flag, const BcDev& bc,
                                            const int* __restrict__ idx, int n) {
  constexpr int q0 = NL * NL, q1 = NH * NH, Q = q0 + q1, T = kTX * kTY, U = 4;
  __shared__ int s_kind[T], s_gb[T], s_sb[T], s_side[T];
  __shared__ R s_dr[T], s_ux[T], s_uy[T];
  const int tid = threadIdx.y * kTX + threadIdx.x;
  for (int c0 = 0; c0 < n; c0 += T) {
    const int m = n - c0 < T ? n - c0 : T;
    if (tid < m) {
      int gx, gy, sx, sy, side = 0, bi = 0;
      const int kind = ghost_cell(p.G, p.nx, p.ny, p.periodic_x, p.periodic_y, bc, idx[c0 + tid],
                                  gx, gy, sx, sy, side, bi);
      const int sb = (sy + p.G) * p.pitch + (sx + kOX);
      s_kind[tid] = kind;
      s_gb[tid] = (gy + p.G) * p.pitch + (gx + kOX);
      s_sb[tid] = sb;
      s_side[tid] = side;
      if (kind == 1 || kind == 3) {
        s_ux[tid] = (R)ghost_ux(bc, side, bi);
        s_uy[tid] = (R)ghost_uy(bc, side, bi);
      }
      if (kind == 1) {  // density deviation of the source from its own lattice
        R dr = R(0);
        if (__ldcg(flag + sx + p.nx * sy)) {
#pragma unroll
          for (int j = 0; j < q1; ++j)
            dr += from_s<R>(ldcg_s(f1 + (size_t)j * p.plane + sb), p.lat[1].sc[j]);
        } else {
#pragma unroll
          for (int j = 0; j < q0; ++j)
            dr += from_s<R>(ldcg_s(f0 + (size_t)j * p.plane + sb), p.lat[0].sc[j]);
        }
        s_dr[tid] = dr;
      }
    }
    __syncthreads();
    for (int e0 = tid; e0 < m * Q; e0 += U * T) {
      S val[U];
      S* dst[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * T;
        dst[u] = nullptr;
        if (e >= m * Q) continue;
        const int plane = e / m, j = e - plane * m;
        const int kind = s_kind[j];
        if (kind == 2) continue;
        const int k = plane < q0 ? 0 : 1;
        const int i = k ? plane - q0 : plane;
        S* f = k ? f1 : f0;
        const size_t off = (size_t)i * p.plane;
        dst[u] = f + off + s_gb[j];
        if (kind == 0) {
          val[u] = ldcg_s(f + off + s_sb[j]);
        } else if (kind == 3) {
          val[u] = to_s<S, R>(
              k ? diffuse_value<NH, S, R>(p.lat[1], f1, p.plane, s_sb[j], s_side[j], s_ux[j],
                                          s_uy[j], i)
                : diffuse_value<NL, S, R>(p.lat[0], f0, p.plane, s_sb[j], s_side[j], s_ux[j],
                                          s_uy[j], i),
              p.lat[k].isc[i]);
        } else {
          val[u] = to_s<S, R>(inlet_value<NL, NH, R>(p, k, i, s_dr[j], s_ux[j], s_uy[j]),
                              p.lat[k].isc[i]);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (dst[u]) *dst[u] = val[u];
    }
    __syncthreads();  // the chunk's shared arrays are reused
  }
}

// Per-step post-step kernel, one CTA (32 x 8 threads) per tile: the choice
// for small grids, whose few tiles each end in one chain of the kernel.
//  1. Interface conversion.  The stream kernel has OR-ed, into one word per
//     tile, the lattices of the tile's 3 x 3 tile neighbourhood and the tile's
//     own flip bit, and listed the candidate tiles (add_work).  CTA b takes
//     items b, b + G, ...; list items whose word is work (both lattices or a
//     flip) are converted (post_tile), so clustered interfaces spread evenly
//     over the GPU.
//  2. Ghost images.  Every ghost element depends on one interior cell (its
//     source), so the CTA that converts a tile writes, after the tile's
//     barrier, the ghosts whose source lies in that tile (per-tile lists
//     gh_start / gh_idx over the ring, built at set-up from the ghost rule);
//     the other border tiles (gh_tiles, items after the list) write theirs at
//     once, their sources being final when the stream kernel ends.  No CTA
//     waits for another.  (A lattice's planes at a cell outside every work
//     tile are read by no cell of that lattice, so their stale copies are
//     never used.)
template <int NL, int NH, class S, class R>
__global__ void __launch_bounds__(kTX * kTY)
k_post_step_block(const Params<R> p, S* f0, S* f1, const uint8_t* __restrict__ flag_old,
            const uint8_t* __restrict__ flag_new, const BcDev bc, const int* __restrict__ work,
            const int* __restrict__ list, const int* __restrict__ nlist, int ntx,
            const int* __restrict__ gh_start, const int* __restrict__ gh_idx,
            const int* __restrict__ gh_tiles, int n_ghtiles) {
  __shared__ uint8_t sf[kTY + 2 * kBandMax][kTX + 2 * kBandMax];
  __shared__ int gb[2];  // ghost list bounds of the list item being converted
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int G = (int)gridDim.x;
  if (blockIdx.x == 0 && tid == 0) ++*p.seed_ctr;  // the next stream launch rounds with a new key
  // the count and this CTA's first list entry are fetched together (each half
  // of the list holds ntiles entries, so the entry is always in bounds)
  const int ntiles = ntx * ((p.ny + kTY - 1) / kTY);
  // every index read from the stream kernel's outputs is checked before it
  // addresses anything: the count against the list's capacity, each entry
  // against the tile count (a tile is listed at most once per step, so a
  // valid list never exceeds either)
  const int nl = min(max(*nlist, 0), ntiles);
  const int t_first = (int)blockIdx.x < ntiles ? list[blockIdx.x] : 0;
  const int total = nl + n_ghtiles;
  for (int r = (int)blockIdx.x; r < total; r += G) {
    if (r < nl) {
      const int t = r == (int)blockIdx.x ? t_first : list[r];
      if (t < 0 || t >= ntiles) continue;  // uniform per CTA: no barrier is skipped by part of it
      // the tile's ghost list bounds are fetched with its work word and flags
      // (through shared memory: published by post_tile's barriers)
      if (tid == 0) {
        gb[0] = gh_start[t];
        gb[1] = gh_start[t + 1];
      }
      // ends with a barrier: the tile's conversions are visible to the CTA
      if (!post_tile<NL, NH, S, R>(p, f0, f1, flag_old, flag_new, bc, 0, false, nullptr,
                                   (t % ntx) * kTX, (t / ntx) * kTY, sf, work + t))
        continue;  // all high-order neighbourhood
    } else {
      const int t = gh_tiles[r - nl];
      if (post_work_word(work[t])) continue;  // written after its conversion
      if (tid == 0) {
        gb[0] = gh_start[t];
        gb[1] = gh_start[t + 1];
      }
      __syncthreads();
    }
    const int g0 = gb[0], n = gb[1] - g0;
    tile_ghosts<NL, NH, S, R>(p, f0, f1, flag_new, bc, gh_idx + g0, n);
    __syncthreads();  // gb is rewritten by the next item
  }
}

// ------------------------------------------------------------- per step
//
// One warp per tile, no block barrier: the per-step post-step kernel for
// large grids gives each warp its own chain of tiles, so an SM keeps many
// independent chains (flag loads, conversions, ghost writes) in flight.

constexpr int kPostWarps = 4;  // warps per CTA of the per-step kernel
// resident CTAs per SM the per-step kernel is compiled for (80 registers;
// FP64, the parity build, keeps its registers)
template <class S>
constexpr int post_blocks() { return sizeof(S) == 8 ? 3 : 6; }

// Diffuse-wall ghost cell of lattice L (N nodes per axis), all Q populations
// by one thread: the same sums as diffuse_value, taken once per cell.
template <int N, class S, class R>
__device__ __forceinline__ void diffuse_cell(const LatTab<R>& L, S* f, long long plane, int sb,
                                             int gb, int side, R uwx, R uwy) {
  const bool axis_y = side >= SLBM_SIDE_YMIN;
  const R nsign = (side == SLBM_SIDE_XMIN || side == SLBM_SIDE_YMIN) ? R(1) : R(-1);
  R dx[N], dy[N];
  dphi<R>(L, N, uwx, dx);
  dphi<R>(L, N, uwy, dy);
  R sv[N * N];
  R s_out = R(0), e_in = R(0), a = R(0);
#pragma unroll
  for (int jy = 0; jy < N; ++jy)
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const int j = jx + N * jy;
      const R cn = (axis_y ? L.c[jy] : L.c[jx]) * nsign;
      const R w = L.w1[jx] * L.w1[jy];
      const R e = L.w1[jx] * dy[jy] + dx[jx] * L.w1[jy] + dx[jx] * dy[jy];
      sv[j] = from_s<R>(ldcg_s(f + (size_t)j * plane + sb), L.sc[j]);
      if (cn < R(0)) s_out -= cn * sv[j];
      if (cn > R(0)) {
        e_in += cn * e;
        a += cn * w;
      }
    }
  const R drw = (s_out - e_in) / (a + e_in);
#pragma unroll
  for (int jy = 0; jy < N; ++jy)
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const int j = jx + N * jy;
      const R cn = (axis_y ? L.c[jy] : L.c[jx]) * nsign;
      const R w = L.w1[jx] * L.w1[jy];
      const R e = L.w1[jx] * dy[jy] + dx[jx] * L.w1[jy] + dx[jx] * dy[jy];
      f[(size_t)j * plane + gb] = to_s<S, R>(cn > R(0) ? drw * (w + e) + e : sv[j], L.isc[j]);
    }
}

// Images of ghost cell g (every plane of both lattices) by one thread, under
// the ghost rule: copies of the source, INLET equilibria (both lattices, in
// product form) at the source's density (summed over its own lattice) and
// the side's velocity, DIFFUSE walls; DIRICHLET ghosts are constant.
// Sources are read through L2 (ld.global.cg): other threads have just
// written them.
template <int NL, int NH, class S, class R>
__device__ __forceinline__ void lane_ghost(const Params<R>& p, S* f0, S* f1,
                                           const uint8_t* __restrict__ flag, const BcDev& bc,
                                           int g) {
  constexpr int q0 = NL * NL, q1 = NH * NH;
  int gx, gy, sx, sy, side = 0, bi = 0;
  const int kind = ghost_cell(p.G, p.nx, p.ny, p.periodic_x, p.periodic_y, bc, g, gx, gy, sx, sy,
                              side, bi);
  if (kind == 2) return;
  const int sb = (sy + p.G) * p.pitch + (sx + kOX);
  const int gb = (gy + p.G) * p.pitch + (gx + kOX);
  if (kind == 0) {
    S v[q1];
#pragma unroll
    for (int i = 0; i < q0; ++i) v[i] = ldcg_s(f0 + (size_t)i * p.plane + sb);
#pragma unroll
    for (int i = 0; i < q0; ++i) f0[(size_t)i * p.plane + gb] = v[i];
#pragma unroll
    for (int i = 0; i < q1; ++i) v[i] = ldcg_s(f1 + (size_t)i * p.plane + sb);
#pragma unroll
    for (int i = 0; i < q1; ++i) f1[(size_t)i * p.plane + gb] = v[i];
  } else if (kind == 3) {
    const R uwx = (R)ghost_ux(bc, side, bi), uwy = (R)ghost_uy(bc, side, bi);
    diffuse_cell<NL, S, R>(p.lat[0], f0, p.plane, sb, gb, side, uwx, uwy);
    diffuse_cell<NH, S, R>(p.lat[1], f1, p.plane, sb, gb, side, uwx, uwy);
  } else {
    R dr = R(0);
    if (__ldcg(flag + sx + p.nx * sy)) {
#pragma unroll
      for (int j = 0; j < q1; ++j)
        dr += from_s<R>(ldcg_s(f1 + (size_t)j * p.plane + sb), p.lat[1].sc[j]);
    } else {
#pragma unroll
      for (int j = 0; j < q0; ++j)
        dr += from_s<R>(ldcg_s(f0 + (size_t)j * p.plane + sb), p.lat[0].sc[j]);
    }
    write_eq_t<NL, NH, S, R>(p, f0, f1, gb, dr, (R)ghost_ux(bc, side, bi),
                             (R)ghost_uy(bc, side, bi));
  }
}

// A staged column (periodic wrap by a full modulo; -1 beyond a bounded side).
__device__ __forceinline__ int stage_col(int c, int n, int periodic) {
  if (c >= 0 && c < n) return c;
  return periodic ? ((c % n) + n) % n : -1;
}

// Interface conversion of one tile (origin x0, y0) by one warp.  Flags of
// the tile's rows and of B rows / columns around it become warp-wide bit
// masks (ballots of each staged row's 32 columns plus the 2B halo columns
// loaded by lanes < 2B); "a cell of lattice v within B columns" is the mask
// OR-ed with itself shifted by 1 .. 2B, and within B rows and columns the OR
// of 2B + 1 such rows.  A cell converts when its lattice changed or a cell of
// the other lattice is within the band radius (the rule of post_tile); the
// cells to convert are compacted over the warp's lanes, lifts first, then
// projections, 32 at a time.
template <int NL, int NH, class S, class R>
__device__ __forceinline__ void warp_convert(const Params<R>& p, S* f0, S* f1,
                                             const uint8_t* __restrict__ flag_old,
                                             const uint8_t* __restrict__ flag_new, int x0,
                                             int y0) {
  constexpr int kRows = kTY + 2 * kBandMax;
  const int lane = threadIdx.x & 31, B = p.band;
  const int cm = stage_col(x0 + lane, p.nx, p.periodic_x);
  const int ch = lane < 2 * B
                     ? stage_col(lane < B ? x0 - B + lane : x0 + kTX + lane - B, p.nx, p.periodic_x)
                     : -1;
  // per staged row, into the warp's shared words: which lanes' windows
  // (columns lane - B .. lane + B) hold lattice 0 / 1 (d[0 / 1][row]); per tile
  // row the new and old lattice masks of the tile's cells (t[0..3][row]:
  // new 0, new 1, old 0, old 1); then per tile row the cells to lift / project,
  // the new lattice and the band mask (c[0..3][row]).  Shared, not registers:
  // the conversions below need the registers.
  __shared__ unsigned s_d[kPostWarps][2][kRows];
  __shared__ unsigned s_t[kPostWarps][4][kTY];
  __shared__ unsigned s_c[kPostWarps][4][kTY];
  const int wq = threadIdx.x >> 5;
  unsigned(*sd)[kRows] = s_d[wq];
  unsigned(*st)[kTY] = s_t[wq];
  unsigned(*sm)[kTY] = s_c[wq];
  const bool xin = x0 + lane < p.nx;
  // every flag this lane stages, loaded before any is used (one memory
  // latency per tile, not one per row): staged row r is grid row
  // y0 - kBandMax + r, whatever the band radius
  int fm[kRows], fh[kRows], fo[kTY];
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const int gy = stage_col(y0 - kBandMax + r, p.ny, p.periodic_y);
    fm[r] = 2;
    fh[r] = 2;
    if (gy >= 0) {
      if (cm >= 0) fm[r] = flag_new[(long long)gy * p.nx + cm];
      if (ch >= 0) fh[r] = flag_new[(long long)gy * p.nx + ch];
    }
  }
#pragma unroll
  for (int i = 0; i < kTY; ++i) {
    const bool in = xin && y0 + i < p.ny;
    fo[i] = in ? flag_old[(long long)(y0 + i) * p.nx + x0 + lane] : 2;
  }
  const unsigned long long lo = (1ull << B) - 1ull;
#pragma unroll
  for (int r = 0; r < kRows; ++r) {
    const unsigned m0 = __ballot_sync(0xffffffffu, fm[r] == 0), m1 = __ballot_sync(0xffffffffu, fm[r] == 1);
    const unsigned h0 = __ballot_sync(0xffffffffu, fh[r] == 0), h1 = __ballot_sync(0xffffffffu, fh[r] == 1);
    const unsigned long long e0 = ((unsigned long long)h0 & lo) | ((unsigned long long)m0 << B) |
                                  ((unsigned long long)(h0 >> B) << (kTX + B));
    const unsigned long long e1 = ((unsigned long long)h1 & lo) | ((unsigned long long)m1 << B) |
                                  ((unsigned long long)(h1 >> B) << (kTX + B));
    unsigned long long a0 = e0, a1 = e1;
    for (int d = 1; d <= 2 * B; ++d) {
      a0 |= e0 >> d;
      a1 |= e1 >> d;
    }
    if (lane == 0) {
      sd[0][r] = (unsigned)a0;
      sd[1][r] = (unsigned)a1;
    }
    const int i = r - kBandMax;  // tile row
    if (i >= 0 && i < kTY) {
      const bool in = xin && y0 + i < p.ny;
      const unsigned t0 = __ballot_sync(0xffffffffu, in && fm[r] == 0);
      const unsigned t1 = __ballot_sync(0xffffffffu, in && fm[r] == 1);
      const unsigned t2 = __ballot_sync(0xffffffffu, in && fo[i] == 0);
      const unsigned t3 = __ballot_sync(0xffffffffu, in && fo[i] == 1);
      if (lane == 0) {
        st[0][i] = t0;
        st[1][i] = t1;
        st[2][i] = t2;
        st[3][i] = t3;
      }
    }
  }
  __syncwarp();
  int nlift = 0, nproj = 0;
  for (int i = 0; i < kTY; ++i) {
    unsigned w0 = 0u, w1 = 0u;  // lattice 0 / 1 within B rows and columns
    for (int d = kBandMax - B; d <= kBandMax + B; ++d) {
      w0 |= sd[0][i + d];
      w1 |= sd[1][i + d];
    }
    const unsigned n0 = st[0][i], n1 = st[1][i], o0 = st[2][i], o1 = st[3][i];
    const unsigned band = (n0 & w1) | (n1 & w0);
    const unsigned flip = (o0 & n1) | (o1 & n0);
    const unsigned conv = (n0 | n1) & (o0 | o1) & (flip | band);
    if (lane == 0) {
      sm[0][i] = conv & o0;
      sm[1][i] = conv & o1;
      sm[2][i] = n1;
      sm[3][i] = band;
    }
    nlift += __popc(conv & o0);
    nproj += __popc(conv & o1);
  }
  __syncwarp();
  using M = PostMath<NL, NH, R>;
  for (int pass = 0; pass < 2; ++pass) {
    const int ntot = pass ? nproj : nlift;
    for (int base = 0; base < ntot; base += 32) {
      const int k = base + lane;
      if (k >= ntot) continue;
      // the k-th cell of the pass: its row by the rows' counts, its column by __fns
      int i = 0, pre = 0;
      for (; i < kTY - 1; ++i) {
        const int c = __popc(sm[pass][i]);
        if (k < pre + c) break;
        pre += c;
      }
      const int col = (int)__fns(sm[pass][i], 0, k - pre + 1);
      const int nw = (int)((sm[2][i] >> col) & 1u), band = (int)((sm[3][i] >> col) & 1u);
      const int base_el = (y0 + i + p.G) * p.pitch + (x0 + col + kOX);
      R a[kMaxN][kMaxN], b[kMaxN][kMaxN];
      if (pass == 0) {  // computed in the low-order lattice
        load_t<NL, S, R>(p.lat[0], f0, p.plane, base_el, a);
        M::lift(p, a, b);
        store_t<NH, S, R>(p.lat[1], f1, p.plane, base_el, b);
        if (nw == 1 && band) {  // now high-order; low-order readers see its projection
          M::project(p, b, a);
          store_t<NL, S, R>(p.lat[0], f0, p.plane, base_el, a);
        }
      } else {
        load_t<NH, S, R>(p.lat[1], f1, p.plane, base_el, b);
        M::project(p, b, a);
        store_t<NL, S, R>(p.lat[0], f0, p.plane, base_el, a);
        if (nw == 0 && band) {  // now low-order; high-order readers see its lifting
          M::lift(p, a, b);
          store_t<NH, S, R>(p.lat[1], f1, p.plane, base_el, b);
        }
      }
    }
  }
  __syncwarp();  // the shared words are rewritten by the warp's next tile
}

// Per-step post-step kernel, one warp per tile (large grids).
//  1. Interface conversion.  The stream kernel has OR-ed, into one word per
//     tile, the lattices of the tile's 3 x 3 tile neighbourhood and the tile's
//     own flip bit, and listed the candidate tiles (add_work).  Each warp takes
//     the next item from a counter; list items whose word is work (both
//     lattices or a flip) are converted by that warp (warp_convert).
//  2. Ghost images.  Every ghost element depends on one interior cell (its
//     source), so the warp that converts a tile then writes the ghosts whose
//     source lies in that tile (per-tile lists gh_start / gh_idx, built at
//     set-up from the ghost rule), one ghost cell per lane; the other border
//     tiles (gh_tiles, items after the list) write theirs at once, their
//     sources being final when the stream kernel ends.  No warp waits for
//     another.  (A lattice's planes at a cell outside every work tile are read
//     by no cell of that lattice, so their stale copies are never used.)
template <int NL, int NH, class S, class R>
__global__ void __launch_bounds__(kPostWarps * 32, post_blocks<S>())
k_post_step_warp(const Params<R> p, S* f0, S* f1, const uint8_t* __restrict__ flag_old,
            const uint8_t* __restrict__ flag_new, const BcDev bc, const int* __restrict__ work,
            const int* __restrict__ list, const int* __restrict__ nlist, int ntx,
            const int* __restrict__ gh_start, const int* __restrict__ gh_idx,
            const int* __restrict__ gh_tiles, int n_ghtiles) {
  const int lane = threadIdx.x & 31;
  if (blockIdx.x == 0 && threadIdx.x == 0) ++*p.seed_ctr;  // the next stream launch rounds with a new key
  // every index read from the stream kernel's outputs is checked before it
  // addresses anything: the count against the list's capacity, each entry
  // against the tile count (a tile is listed at most once per step, so a
  // valid list never exceeds either)
  const int ntiles = ntx * ((p.ny + kTY - 1) / kTY);
  const int nl = min(max(*nlist, 0), ntiles);
  const int total = nl + n_ghtiles;
  // items are taken by lane 0 from the item counter (zeroed by the stream
  // kernel), so tiles of uneven cost even out over the warps; the warp asks
  // for its next item when it starts one, and the counter's answer arrives
  // while the current item is processed
  int r = 0;
  if (lane == 0) r = atomicAdd(p.sched + 2, 1);
  r = __shfl_sync(0xffffffffu, r, 0);
  for (; r < total; r = __shfl_sync(0xffffffffu, r, 0)) {
    const int cur = r;
    if (lane == 0) r = atomicAdd(p.sched + 2, 1);
    int t;
    if (cur < nl) {
      t = list[cur];
      if (t < 0 || t >= ntiles || !post_work_word(work[t])) continue;  // warp-uniform
      warp_convert<NL, NH, S, R>(p, f0, f1, flag_old, flag_new, (t % ntx) * kTX, (t / ntx) * kTY);
      __syncwarp();  // the tile's conversions are visible to the warp's ghost writes
    } else {
      t = gh_tiles[cur - nl];
      if (post_work_word(work[t])) continue;  // written after its conversion
    }
    const int g0 = gh_start[t], g1 = gh_start[t + 1];
    for (int g = g0 + lane; g < g1; g += 32)
      lane_ghost<NL, NH, S, R>(p, f0, f1, flag_new, bc, gh_idx[g]);
  }
}

// Launch cache of the per-step kernel's occupancy, per instantiation and device.
struct PostLaunchCache {
  std::mutex mu;
  int per_sm[64] = {};
};

template <class S, class R>
cudaError_t launch_post_step_impl(const Params<R>& p, S* f0, S* f1, const uint8_t* flag_old,
                                  const uint8_t* flag_new, const BcDev& bc, const int* work,
                                  const int* list, const int* nlist, const GhostTables& gt,
                                  cudaStream_t st) {
  const int ntx = (p.nx + kTX - 1) / kTX;
  const int nl = p.lat[0].n, nh = p.lat[1].n;
  const int nty = (p.ny + kTY - 1) / kTY;
  const long long items = (long long)ntx * nty + gt.ntiles;
  if (!p.post_warp) {
    // one CTA per item; four CTAs fit per SM, and a small grid needs no more
    // CTAs than it can have items (list entries + border tiles), which leaves
    // the GPU to concurrent launches of other handles
    const int grid = (int)(items < 4LL * p.nsm ? items : 4LL * p.nsm);
#define SLBM_POSTSTEP_CASE(NL, NH)                                                          \
  if (nl == NL && nh == NH) {                                                               \
    k_post_step_block<NL, NH, S, R><<<grid > 0 ? grid : 1, dim3(kTX, kTY), 0, st>>>(        \
        p, f0, f1, flag_old, flag_new, bc, work, list, nlist, ntx, gt.start, gt.idx,         \
        gt.tiles, gt.ntiles);                                                               \
    return cudaGetLastError();                                                              \
  }
    SLBM_POSTSTEP_CASE(3, 4)
    SLBM_POSTSTEP_CASE(3, 5)
    SLBM_POSTSTEP_CASE(4, 5)
#undef SLBM_POSTSTEP_CASE
    return cudaErrorInvalidValue;
  }
  // one warp per item: as many warps as fit the GPU at once, and no more than
  // there can be items
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
#define SLBM_POSTSTEP_CASE(NL, NH)                                                          \
  if (nl == NL && nh == NH) {                                                               \
    auto kern = k_post_step_warp<NL, NH, S, R>;                                             \
    static PostLaunchCache cache;                                                           \
    int per_sm = 0;                                                                         \
    {                                                                                       \
      std::lock_guard<std::mutex> lock(cache.mu);                                           \
      if (cache.per_sm[dev] < 1) {                                                          \
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                \
            &cache.per_sm[dev], kern, kPostWarps * 32, 0);                                  \
        if (e != cudaSuccess) return e;                                                     \
      }                                                                                     \
      per_sm = cache.per_sm[dev];                                                           \
    }                                                                                       \
    if (per_sm < 1) return cudaErrorInvalidConfiguration;                                   \
    const long long want = (items + kPostWarps - 1) / kPostWarps;                           \
    const int grid = (int)(want < (long long)per_sm * p.nsm ? want : (long long)per_sm * p.nsm); \
    kern<<<grid > 0 ? grid : 1, kPostWarps * 32, 0, st>>>(p, f0, f1, flag_old, flag_new, bc,  \
                                                          work, list, nlist, ntx, gt.start,  \
                                                          gt.idx, gt.tiles, gt.ntiles);      \
    return cudaGetLastError();                                                              \
  }
  SLBM_POSTSTEP_CASE(3, 4)
  SLBM_POSTSTEP_CASE(3, 5)
  SLBM_POSTSTEP_CASE(4, 5)
#undef SLBM_POSTSTEP_CASE
  return cudaErrorInvalidValue;
}

template <class S, class R>
cudaError_t launch_post_impl(const Params<R>& p, S* f0, S* f1, const uint8_t* flag_old,
                             const uint8_t* flag_new, const BcDev& bc, int images,
                             const uint8_t* mask_in, uint8_t* tile_mask, cudaStream_t st) {
  const int ntx = (p.nx + kTX - 1) / kTX, nty = (p.ny + kTY - 1) / kTY;
  const int ntiles = ntx * nty;
  int grid = p.nsm * 2;  // two resident CTAs per SM at this register count
  if (grid > ntiles) grid = ntiles;
  if ((ntiles + grid - 1) / grid > kPostMaxTiles) grid = (ntiles + kPostMaxTiles - 1) / kPostMaxTiles;
  const dim3 blk(kTX, kTY);
  const int nl = p.lat[0].n, nh = p.lat[1].n;
#define SLBM_POST_CASE(NL, NH)                                                              \
  if (nl == NL && nh == NH) {                                                               \
    k_post<NL, NH, S, R><<<grid, blk, 0, st>>>(p, f0, f1, flag_old, flag_new, bc, images,    \
                                                mask_in, tile_mask, ntx, nty);               \
    return cudaGetLastError();                                                              \
  }
  SLBM_POST_CASE(3, 4)
  SLBM_POST_CASE(3, 5)
  SLBM_POST_CASE(4, 5)
#undef SLBM_POST_CASE
  return cudaErrorInvalidValue;
}

}  // namespace slbm
