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
//      other lattice were converted beforehand by the post-step kernel, so
//      every tap reads the target lattice's own planes.
//   2. rho, rho u (Sec. II.B), the lattice equilibrium in product form
//      f^L_i = rho phi_ix(u_x) phi_iy(u_y), phi = V^-1 h(u) with the Gaussian
//      moments h_m(u) = E[(u + Z)^m] (eq. feqL0 restated for a tensor-product
//      Gauss-Hermite lattice), and BGK: f <- f + omega (f^L - f)
//      (eq. Pond_f_equation with omega_1 = omega_2), all on the stored
//      deviations s_i = f_i - W_i.
//   3. optionally the Mach criterion of Sec. IV.A for the next step's flag.
//
// Work is split into strips of 32 columns by up to four 32 x 8 tiles (fewer
// on small grids, so that every SM gets enough warps).  Every warp works on
// its own: it takes the next strip from a global counter and, for each
// lattice the strip's tiles hold, sweeps the strip's rows top to bottom with
// one lane per column.
//   * A population whose shift has a fractional y part keeps the
//     x-interpolations of the P rows of its stencil in registers and
//     interpolates one new row per output row, so each input row is
//     x-interpolated once per population instead of once per cell that reads
//     it.
//   * Taps are read straight from the population planes through the
//     read-only path: rows start 128-byte aligned (kOX), so a warp's 32
//     columns of a plane row are one cache line and the neighbouring lanes'
//     overlapping taps hit L1; two rows ahead of the sweep, a few lanes
//     prefetch the lines of every plane into L1.
//   * Each row's cells collide in registers and are stored on the lanes
//     whose cell carries the lattice.
// There is no block-wide synchronisation: warps meet only at the strip
// counter and at the per-tile work words of the post-step kernel.
// (Staging the rows through shared memory -- per-warp TMA row rings, or
// block-wide tiles -- was measured slower: the rings cap the resident warps
// and the block-wide tiles pay barriers per tile.)
#pragma once

#include <mutex>

#include "slbm_ghost.cuh"

namespace slbm {

constexpr int kStripTiles = 4;              // tiles per strip at most (strip height 32 rows)
constexpr int kStripWarps = 4;              // warps per CTA
// resident CTAs per SM the kernel is compiled for (FP64, the parity build, keeps
// its registers)
template <class S>
constexpr int strip_blocks() { return sizeof(S) == 8 ? 3 : 4; }
constexpr int kMaxDevices = 64;             // device ordinals the launch caches cover
constexpr int kPrefetchRows = 2;            // rows ahead a sweep prefetches into L1

// ------------------------------------------------------------ the math

// Store conversion of a new population value.  FP32 / FP64: plain.  FP16:
// stochastic rounding of the deviation -- a 13-bit random number r is added
// to the 13 mantissa bits that FP16 drops before truncating, so a value is
// rounded up with probability equal to its distance from the truncated
// neighbour.  r comes from a counter-based generator: one integer hash of the
// cell's index and the step per cell (hash32), then per population one
// multiplicative hash of that key and the population index (pop_random).
// Round-to-nearest errors of a smooth field repeat from cell to cell and step
// to step and add up; these are unbiased and independent, and the
// interpolation averages them away.  Half subnormals (|v| < 2^-14) round to
// nearest.
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

// 13 random bits for population i of the cell with key `key` (the top bits
// of a multiplicative hash of the key and i).
__device__ __forceinline__ uint32_t pop_random(uint32_t key, int i) {
  return ((key ^ ((uint32_t)i * 0x9e3779b9u)) * 0x85ebca6bu) >> 19;
}

template <class S, class R>
__device__ __forceinline__ S to_storage(R v, uint32_t, R) {
  return static_cast<S>(v);
}

template <>
__device__ __forceinline__ __half to_storage<__half, float>(float v, uint32_t r, float) {
  if (!(fabsf(v) >= 6.103515625e-05f) || fabsf(v) >= 65504.0f) return __float2half_rn(v);
  const uint32_t b = __float_as_uint(v);
  return __float2half_rz(__uint_as_float((b + r) & ~0x1fffu));
}

// Fixed point: floor(c + r / 2^13) of the companded value c, saturating at
// +-32767 -- rounded up with probability equal to c's distance from the
// integer below, as above.
template <>
__device__ __forceinline__ fx16 to_storage<fx16, float>(float v, uint32_t r, float isc) {
  const float q = floorf(fx_compand(v, isc) + (float)r * (1.0f / 8192.0f));
  return fx16{(int16_t)__float2int_rz(fminf(fmaxf(q, -32767.f), 32767.f))};
}

// One row of node jx's stencil at plane row pointer `row` (elements a = 0 ..
// P-1 of the stencil), differential form v[r] + sum_{a != r} w[a] (v[a] -
// v[r]), r = (P-1)/2 (see LatTab).
template <int P, class S, class R>
__device__ __forceinline__ R row_interp(const S* __restrict__ row, const R* w) {
  constexpr int r = (P - 1) / 2;
  const R vr = from_s<R>(ldg_s(row + r), R(1));
  R t = vr;
#pragma unroll
  for (int a = 0; a < P; ++a)
    if (a != r) t += w[a] * (from_s<R>(ldg_s(row + a), R(1)) - vr);
  return t;
}

// Value of population I's stencil row at plane row pointer `row`: a single
// tap (integer x shift) or the x-interpolation.  Fixed point: the taps are
// decoded without the plane's scale (q |q|), which multiplies the row's result
// once.
template <int N, bool HI, int P, int I, class S, class R>
__device__ __forceinline__ R tap_row(const LatTab<R>& L, const S* __restrict__ row) {
  constexpr int jx = I % N;
  R v;
  if constexpr (node_snapped(N, HI, jx))
    v = from_s<R>(ldg_s(row), R(1));
  else
    v = row_interp<P, S, R>(row, L.w[jx]);
  if constexpr (is_fx16<S>()) v *= L.sc[I];
  return v;
}

// x offset (first column relative to the cell) of population I's stencil
template <int N, bool HI, int I, class R>
__device__ __forceinline__ int x_off(const LatTab<R>& L) {
  constexpr int jx = I % N;
  if constexpr (node_snapped(N, HI, jx)) return snapped_offset(N, jx);
  else return L.off[jx];
}

// A population is windowed when its y shift is fractional (P stencil rows).
template <int N, bool HI, int I>
__host__ __device__ constexpr bool windowed() { return !node_snapped(N, HI, I / N); }

// Sweep state of one lattice: the y windows of the windowed populations
// (P - 1 kept rows each; entries of the other populations are unused).
template <int N, int P, class R>
struct Windows {
  R v[N * N][P - 1];
};

// Element pointer of plane i at (row r, column of `col`): col points at the
// lane's column in plane 0 of row 0 (ghost offsets included).  Offsets are
// 32-bit: the launcher requires Q * plane < 2^31 elements.
template <class S>
__device__ __forceinline__ const S* plane_row(const S* col, int plane, int pitch, int i, int r) {
  return col + (i * plane + r * pitch);
}

// Input row r of a sweep.  WRAP (strips within the stencil reach of a
// periodic y edge): the row's periodic image inside the grid, so the y ghost
// rows of a periodic axis are never read; otherwise r itself (ghost rows of a
// bounded side hold its boundary states).
template <bool WRAP>
__device__ __forceinline__ int in_row(int r, int ny) {
  if constexpr (WRAP) return r < 0 ? r + ny : (r >= ny ? r - ny : r);
  else return r;
}

template <int N, bool HI, int P, class S, class R, bool WRAP, int I = 0>
__device__ __forceinline__ void prime(const LatTab<R>& L, const S* col, int plane, int pitch,
                                      int ys, int ny, Windows<N, P, R>& W) {
  if constexpr (I < N * N) {
    if constexpr (windowed<N, HI, I>()) {
      const int r0 = ys + L.off[I / N];
      const int xo = x_off<N, HI, I, R>(L);
      if constexpr (WRAP) {
#pragma unroll
        for (int b = 0; b < P - 1; ++b)
          W.v[I][b] = tap_row<N, HI, P, I, S, R>(
              L, plane_row(col, plane, pitch, I, in_row<WRAP>(r0 + b, ny)) + xo);
      } else {
        const S* q = plane_row(col, plane, pitch, I, r0) + xo;
#pragma unroll
        for (int b = 0; b < P - 1; ++b) W.v[I][b] = tap_row<N, HI, P, I, S, R>(L, q + b * pitch);
      }
    }
    prime<N, HI, P, S, R, WRAP, I + 1>(L, col, plane, pitch, ys, ny, W);
  }
}

// Streamed value of every population at output row y (windows advanced).
template <int N, bool HI, int P, class S, class R, bool WRAP, int I = 0>
__device__ __forceinline__ void stream_row(const LatTab<R>& L, const S* col, int plane, int pitch,
                                           int y, int ny, Windows<N, P, R>& W, R* f) {
  if constexpr (I < N * N) {
    constexpr int jy = I / N;
    if constexpr (windowed<N, HI, I>()) {
      constexpr int rr = (P - 1) / 2;
      const S* q = plane_row(col, plane, pitch, I, in_row<WRAP>(y + L.off[jy] + P - 1, ny)) +
                   x_off<N, HI, I, R>(L);
      const R vn = tap_row<N, HI, P, I, S, R>(L, q);
      R v[P];
#pragma unroll
      for (int b = 0; b < P - 1; ++b) v[b] = W.v[I][b];
      v[P - 1] = vn;
      R acc = v[rr];
#pragma unroll
      for (int b = 0; b < P; ++b)
        if (b != rr) acc += L.w[jy][b] * (v[b] - v[rr]);
      f[I] = acc;
#pragma unroll
      for (int b = 0; b < P - 2; ++b) W.v[I][b] = W.v[I][b + 1];
      W.v[I][P - 2] = vn;
    } else {
      const S* q = plane_row(col, plane, pitch, I, in_row<WRAP>(y + snapped_offset(N, jy), ny)) +
                   x_off<N, HI, I, R>(L);
      f[I] = tap_row<N, HI, P, I, S, R>(L, q);
    }
    stream_row<N, HI, P, S, R, WRAP, I + 1>(L, col, plane, pitch, y, ny, W, f);
  }
}

// Collision of one cell of lattice L on its streamed deviations f: rho, u,
// the product-form equilibrium and BGK with rate omega (see slbm_eq.cuh); the
// new values go to `o` (plane stride `plane`) when `store`.
template <int N, class S, class R>
__device__ __forceinline__ void collide(const Params<R>& p, const LatTab<R>& L, R omega, R* f,
                                        S* __restrict__ o, bool store, uint32_t key, R& ux,
                                        R& uy) {
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
  R px[N];
#pragma unroll
  for (int jx = 0; jx < N; ++jx) px[jx] = L.w1[jx] + dx[jx];
#pragma unroll
  for (int jy = 0; jy < N; ++jy) {
    const R py = L.w1[jy] + dy[jy];
    const R ty = dr * py;
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const int i = jx + N * jy;
      // f^L - W = dr px py + w_x dphi_y + dphi_x (w_y + dphi_y)
      const R feq = px[jx] * ty + L.w1[jx] * dy[jy] + dx[jx] * py;
      f[i] += omega * (feq - f[i]);
    }
  }
  if (store) {
    const int pl = (int)p.plane;
#pragma unroll
    for (int i = 0; i < N * N; ++i)
      o[i * pl] = to_storage<S, R>(f[i], pop_random(key, i), L.isc[i]);
  }
}

// Prefetch of input row r of the Q planes for the warp's 32 columns (the
// lines holding columns x0 - G .. x0 + 31 + G): lane l < 2 Q asks for line
// l / Q of plane l % Q, so one or two instructions cover a row.
template <int Q, class S>
__device__ __forceinline__ void prefetch_row(const S* fin, int plane, int pitch, int G, int x0,
                                             int r, int lane) {
  constexpr int kLine = 128 / (int)sizeof(S);  // elements per cache line
#pragma unroll
  for (int l0 = 0; l0 < 2 * Q; l0 += 32) {
    const int l = l0 + lane;
    if (l < 2 * Q) {
      const int i = l % Q, half = l / Q;
      const int c = x0 + kOX - G + half * kLine;  // within the row (an address in the plane)
      const S* a = fin + (i * plane + (r + G) * pitch + (c < pitch ? c : pitch - 1));
      asm volatile("prefetch.global.L1 [%0];" ::"l"(a));
    }
  }
}

// Bit position, in a tile's strip word, of the next-step lattices (2 bits:
// low / high) of its cells within the band radius of side (sx, sy) -- sx, sy
// in {0, 1, 2} = left / whole / right, top / whole / bottom; (1, 1) is not
// used (the tile's own lattices are bits 0-1).
__host__ __device__ constexpr int side_shift(int sx, int sy) { return 8 + 2 * (sx + 3 * sy); }

// One lattice's sweep of a strip: output rows ys .. ye-1 of column x (lane),
// every cell of the lattice streamed, collided and stored; the next flag
// (criterion) written; per tile q of the strip, the OR of the cells' bits
// (bit 0/1: next-step lattice, bit 2: flipped) into tb[q].
template <int N, bool HI, int P, class S, class R, bool WRAP>
__device__ __forceinline__ void sweep(const Params<R>& p, const LatTab<R>& L, int k,
                                      const S* __restrict__ fin, S* __restrict__ fout,
                                      const uint8_t* __restrict__ flag_cur,
                                      uint8_t* __restrict__ flag_nxt, int x, int y0, int ys,
                                      int ye, uint32_t seed, int* tb) {
  const bool xin = x < p.nx;
  const int xl = xin ? x : p.nx - 1;  // loads of lanes past the edge stay in the row
  const S* col = fin + (p.G * p.pitch + xl + kOX);
  const int plane = (int)p.plane;
  // relaxation rate of the lane's column (channels carry their own tau)
  const R om = p.omega_x ? p.omega_x[xl] : p.omega;
  Windows<N, P, R> W;
  prime<N, HI, P, S, R, WRAP>(L, col, plane, p.pitch, ys, p.ny, W);
  int bits = 0, sides = 0;
  const int x0 = x & ~(kTX - 1), lane = threadIdx.x & 31;
  const int rlast = ye + stage_halo(P) - 1;  // last input row the sweep reads
  for (int y = ys; y < ye; ++y) {
    R f[N * N];
    {
      const int r = y + stage_halo(P) + kPrefetchRows;
      if (r <= rlast)
        prefetch_row<N * N, S>(fin, plane, p.pitch, p.G, x0, in_row<WRAP>(r, p.ny), lane);
    }
    stream_row<N, HI, P, S, R, WRAP>(L, col, plane, p.pitch, y, p.ny, W, f);
    const bool act = xin && flag_cur[y * p.nx + x] == k;
    const int ob = (y + p.G) * p.pitch + (x + kOX);
    const uint32_t key = hash32((uint32_t)ob ^ (seed * 0x9e3779b9u));  // FP16 rounding only
    R ux, uy;
    collide<N, S, R>(p, L, om, f, fout + ob, act, key, ux, uy);
    int nf = k;
    if (act) {
      if (p.crit == 1) {
        nf = sqrt(ux * ux + uy * uy) > p.thr ? 1 : 0;
        flag_nxt[y * p.nx + x] = (uint8_t)nf;
      }
      bits |= (1 << nf) | (nf != k ? 4 : 0);
    }
    // the next-step lattices of the row's cells near the tile's sides
    // (warp-uniform): within `band` columns of the left / right side, and, in
    // the first / last `band` rows of the tile, of the top / bottom side
    {
      const unsigned blo = __ballot_sync(0xffffffffu, act && nf == 0);
      const unsigned bhi = __ballot_sync(0xffffffffu, act && nf == 1);
      // the tile's valid columns 0 .. w-1 and rows 0 .. h-1 (a tile at the
      // grid's right / bottom edge may be partial: its facing strips are
      // then its last valid columns / rows, next to the periodic image)
      const int w = min(kTX, p.nx - x0), r = (y - y0) & (kTY - 1);
      const int h = min(kTY, p.ny - (y - r));
      const unsigned all = w >= 32 ? ~0u : (1u << w) - 1u;
      const unsigned lm = (1u << p.band) - 1u;
      const unsigned rm = all & ~(w > p.band ? (1u << (w - p.band)) - 1u : 0u);
      const int row = (blo ? 1 : 0) | (bhi ? 2 : 0);
      const int lf = ((blo & lm) ? 1 : 0) | ((bhi & lm) ? 2 : 0);
      const int rt = ((blo & rm) ? 1 : 0) | ((bhi & rm) ? 2 : 0);
      int e = (lf << side_shift(0, 1)) | (rt << side_shift(2, 1));
      if (r < p.band)
        e |= (lf << side_shift(0, 0)) | (row << side_shift(1, 0)) | (rt << side_shift(2, 0));
      if (r >= h - p.band)
        e |= (lf << side_shift(0, 2)) | (row << side_shift(1, 2)) | (rt << side_shift(2, 2));
      sides |= e;
    }
    // after a tile's last row: its bits, OR-reduced over the warp
    if (((y - y0) & (kTY - 1)) == kTY - 1 || y == ye - 1) {
      const int wb = __reduce_or_sync(0xffffffffu, bits);
      if ((threadIdx.x & 31) == 0) tb[(y - y0) / kTY] |= wb | sides;
      bits = 0;
      sides = 0;
    }
  }
}

// Persistent stream-collide: warps take strips from the global counter
// p.sched[parity] (cleared by the previous launch; this launch clears the
// other one) and sweep them lattice by lattice; then, per tile of the strip,
// write its next-step mask (lattices and flip bit, read by the next launch and
// the post-step kernel) and OR its lattices into the post-step work words of
// its 3 x 3 tile neighbourhood (its flip bit into its own), listing the tiles
// that gain work (add_work, with each returning atomic's result used one tile
// later so the warp does not wait for it).
template <int NL, int NH, int P, class S, class R, bool WRAP>
__global__ void __launch_bounds__(kStripWarps * 32, strip_blocks<S>())
k_stream_collide(const Params<R> p, const S* __restrict__ fin0, const S* __restrict__ fin1,
                 S* __restrict__ fout0, S* __restrict__ fout1,
                 const uint8_t* __restrict__ flag_cur, uint8_t* __restrict__ flag_nxt,
                 const uint8_t* __restrict__ tile_mask_g, uint8_t* __restrict__ mask_next,
                 int ntx, int nty, int stiles, int nstrips) {
  __shared__ int s_tb[kStripWarps][kStripTiles];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ntiles = ntx * nty;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.sched[p.sched_parity ^ 1] = 0;
    p.sched[2] = 0;                    // the post-step kernel's item counter, used after this launch
    p.wcount[p.sched_parity ^ 1] = 0;  // the other work list, likewise
  }
  const uint32_t seed = *p.seed_ctr;  // FP16 rounding key of this step
  int* tb = s_tb[warp];
  // lanes 0-8: a work-word atomic and a list slot whose results are used at
  // the next tile (tile -1: none)
  int pend_t = -1, pend_was = 0, slot_t = -1, slot = 0;
  const int half = p.sched_parity;
  for (;;) {
    int s = 0;
    if (lane == 0) s = atomicAdd(p.sched + p.sched_parity, 1);
    s = __shfl_sync(0xffffffffu, s, 0);
    if (s >= nstrips) break;
    const int sx = s % ntx, ty0 = (s / ntx) * stiles;
    const int nt = nty - ty0 < stiles ? nty - ty0 : stiles;  // tiles in the strip
    const int m = lane < nt ? tile_mask_g[(ty0 + lane) * ntx + sx] : 0;
    const uint32_t has_lo = __ballot_sync(0xffffffffu, m & 1);
    const uint32_t has_hi = __ballot_sync(0xffffffffu, m & 2);
    if (lane < kStripTiles) tb[lane] = 0;
    __syncwarp();
    const int x = sx * kTX + lane, y0 = ty0 * kTY;
    // each lattice over the rows of its first to its last tile in the strip;
    // in the WRAP kernel (handles with wrap_y), a sweep whose input rows
    // (ys - G .. ye - 1 + G) cross the periodic y edge reads their images in
    // the grid
    constexpr int H = stage_halo(P);
    if (has_lo) {
      const int ys = y0 + (__ffs(has_lo) - 1) * kTY;
      const int ye = min(y0 + (32 - __clz(has_lo)) * kTY, p.ny);
      if (WRAP && (ys < H || ye > p.ny - H))
        sweep<NL, false, P, S, R, WRAP>(p, p.lat[0], 0, fin0, fout0, flag_cur, flag_nxt, x, y0,
                                        ys, ye, seed, tb);
      else
        sweep<NL, false, P, S, R, false>(p, p.lat[0], 0, fin0, fout0, flag_cur, flag_nxt, x, y0,
                                         ys, ye, seed, tb);
    }
    if (has_hi) {
      const int ys = y0 + (__ffs(has_hi) - 1) * kTY;
      const int ye = min(y0 + (32 - __clz(has_hi)) * kTY, p.ny);
      if (WRAP && (ys < H || ye > p.ny - H))
        sweep<NH, true, P, S, R, WRAP>(p, p.lat[1], 1, fin1, fout1, flag_cur, flag_nxt, x, y0,
                                       ys, ye, seed, tb);
      else
        sweep<NH, true, P, S, R, false>(p, p.lat[1], 1, fin1, fout1, flag_cur, flag_nxt, x, y0,
                                        ys, ye, seed, tb);
    }
    __syncwarp();
    for (int q = 0; q < nt; ++q) {
      const int t = (ty0 + q) * ntx + sx;
      const int mk = tb[q];
      if (lane == 0) {
        mask_next[t] = (uint8_t)(mk & 7);
        p.work[(size_t)(p.sched_parity ^ 1) * ntiles + t] = 0;  // the next step's half
      }
      if (lane < 9) {
        int ntx_ = sx + lane % 3 - 1, nty_ = ty0 + q + lane / 3 - 1;
        bool in = true;
        if (ntx_ < 0 || ntx_ >= ntx) {
          if (p.periodic_x) ntx_ = ntx_ < 0 ? ntx_ + ntx : ntx_ - ntx;
          else in = false;
        }
        if (nty_ < 0 || nty_ >= nty) {
          if (p.periodic_y) nty_ = nty_ < 0 ? nty_ + nty : nty_ - nty;
          else in = false;
        }
        if (slot_t >= 0) p.wlist[(size_t)half * ntiles + slot] = slot_t;
        slot_t = -1;
        if (pend_t >= 0 && !(pend_was & 6)) {
          slot = atomicAdd(p.wcount + half, 1);
          slot_t = pend_t;
        }
        pend_t = -1;
        // to the neighbour at (dx, dy) = (lane % 3 - 1, lane / 3 - 1): the
        // lattices of this tile's cells within the band radius of the side
        // or corner facing it; to itself, its own lattices and flip bit.  A
        // tile's word then holds both lattices iff one of its cells is within
        // the band radius of a cell of the other lattice.
        const int contrib = lane == 4 ? (mk & 7) : (mk >> side_shift(lane % 3, lane / 3)) & 3;
        if (in && contrib) {
          int* w = p.work + (size_t)half * ntiles + nty_ * ntx + ntx_;
          if (contrib & 6) {
            pend_was = atomicOr(w, contrib);
            pend_t = nty_ * ntx + ntx_;
          } else {
            atomicOr(w, contrib);
          }
        }
      }
    }
    __syncwarp();  // tb is reset by the next strip
  }
  if (lane < 9) {  // the deferred listings of the last tile
    const size_t h = (size_t)half * ntiles;
    if (slot_t >= 0) p.wlist[h + slot] = slot_t;
    if (pend_t >= 0 && !(pend_was & 6)) p.wlist[h + atomicAdd(p.wcount + half, 1)] = pend_t;
  }
}

// Launch cache of one instantiation on one device: the occupancy, queried
// once under a lock.
struct LaunchCache {
  std::mutex mu;
  int per_sm[kMaxDevices] = {};
};

template <class S, class R, bool WRAP>
cudaError_t launch_stream_collide_impl(const Params<R>& p, int P, const S* fin0, const S* fin1,
                                       S* fout0, S* fout1, const uint8_t* flag_cur,
                                       uint8_t* flag_nxt, const uint8_t* tile_mask,
                                       uint8_t* mask_next, cudaStream_t st) {
  const int ntx = (p.nx + kTX - 1) / kTX, nty = (p.ny + kTY - 1) / kTY;
  // strip height: the most tiles (up to four) that still give every SM
  // about 32 strips
  int stiles = kStripTiles;
  while (stiles > 1 && (long long)ntx * ((nty + stiles - 1) / stiles) < 32LL * p.nsm) stiles /= 2;
  const int nstrips = ntx * ((nty + stiles - 1) / stiles);
  const int nl = p.lat[0].n, nh = p.lat[1].n;
  if (p.G < stage_halo(P)) return cudaErrorInvalidValue;  // ghost ring narrower than the stencil
  // 32-bit element offsets within one lattice's planes
  if ((long long)nh * nh * p.plane >= (1LL << 31)) return cudaErrorInvalidValue;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return cudaErrorInvalidDevice;
#define SLBM_SC_CASE(NL, NH, PP)                                                            \
  if (nl == NL && nh == NH && P == PP) {                                                    \
    auto kern = k_stream_collide<NL, NH, PP, S, R, WRAP>;                                   \
    static LaunchCache cache;                                                               \
    int per_sm = 0;                                                                         \
    {                                                                                       \
      std::lock_guard<std::mutex> lock(cache.mu);                                           \
      if (cache.per_sm[dev] < 1) {                                                          \
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                \
            &cache.per_sm[dev], kern, kStripWarps * 32, 0);                                 \
        if (e != cudaSuccess) return e;                                                     \
      }                                                                                     \
      per_sm = cache.per_sm[dev];                                                           \
    }                                                                                       \
    if (per_sm < 1) return cudaErrorInvalidConfiguration;                                   \
    const int want = (nstrips + kStripWarps - 1) / kStripWarps;                             \
    const int grid = want < per_sm * p.nsm ? want : per_sm * p.nsm;                         \
    kern<<<grid, kStripWarps * 32, 0, st>>>(p, fin0, fin1, fout0, fout1, flag_cur, flag_nxt, \
                                            tile_mask, mask_next, ntx, nty, stiles, nstrips); \
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
