// slbm_stream.cuh -- fused stream-collide kernel (sm_103a, TMA-staged).
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
// Work is split into 32 x 8 tiles, one cell per thread; a warp is one 32-cell
// row segment.  A persistent CTA (two per SM) walks its tiles; for each
// lattice a tile holds, one elected thread loads every plane of that lattice
// for the tile and its halo -- a [Q][8 + 2G][40] box -- with a single 3-D TMA
// copy (cp.async.bulk.tensor) into a shared-memory stage, completion signalled
// on an mbarrier, while the previous stage computes.  Threads stream from
// shared memory, where a warp's 32 consecutive taps hit 32 distinct banks.
// Each (tile, lattice) item runs only that lattice's Q-specific code on the
// lanes whose cells carry it, so no warp diverges on Q and a tile of one
// lattice costs one pass.
#pragma once

#include <cuda.h>

#include "slbm_ghost.cuh"

namespace slbm {

// Staged row geometry per storage type: xh halo columns each side (>= G),
// chosen so the TMA box starts 16 bytes aligned (tile x0 + kOX - xh is a
// multiple of 16 / sizeof(S)); txp staged elements per row.
template <class S>
struct StageGeom {
  static constexpr int xh = sizeof(S) == 2 ? 8 : 4;
  static constexpr int txp = kTX + 2 * xh;
  // resident CTAs per SM the kernel is compiled for: FP16 stages are half the
  // size, so three CTAs fit in shared memory (and 80 registers a thread)
  static constexpr int min_blocks = sizeof(S) == 2 ? 3 : 2;
};
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s bound on an mbarrier wait
constexpr int kMaxDevices = 64;                 // device ordinals the launch caches cover

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after ~kWaitCycles without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, uint64_t* bar,
                                            int c0, int c1, int c2) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}

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
__device__ __forceinline__ S to_storage(R v, uint32_t) {
  return static_cast<S>(v);
}

template <>
__device__ __forceinline__ __half to_storage<__half, float>(float v, uint32_t r) {
  if (!(fabsf(v) >= 6.103515625e-05f) || fabsf(v) >= 65504.0f) return __float2half_rn(v);
  const uint32_t b = __float_as_uint(v);
  return __float2half_rz(__uint_as_float((b + r) & ~0x1fffu));
}

// One row of node jx's stencil (differential form v[r] + sum_{a != r}
// w[a] (v[a] - v[r]), r = (P-1)/2, see LatTab).
template <int N, bool HI, int P, class S, class R>
__device__ __forceinline__ R row_interp(const S* row, const LatTab<R>& L, int jx) {
  constexpr int r = (P - 1) / 2;
  const R vr = static_cast<R>(row[r]);
  R t = vr;
#pragma unroll
  for (int a = 0; a < P; ++a)
    if (a != r) t += L.w[jx][a] * (static_cast<R>(row[a]) - vr);
  return t;
}

// Stream + collide one cell of lattice L (N nodes per axis, HI = the
// high-order lattice) from the staged planes (cell at `src`, planes PL
// elements apart, rows StageGeom<S>::txp apart), on deviations s_i = f_i - W_i (streaming
// is affine in the shift; the collision uses the deviation form of the
// product equilibrium, see slbm_eq.cuh).
template <int N, bool HI, int P, class S, class R>
__device__ __forceinline__ void stream_collide_cell(const Params<R>& p, const LatTab<R>& L,
                                                    const S* src, S* __restrict__ fout,
                                                    int obase, uint32_t seed, R& ux, R& uy,
                                                    R& drho) {
  constexpr int kTXP = StageGeom<S>::txp;
  constexpr int PL = (kTY + 2 * stage_halo(P)) * kTXP;
  R f[N * N];
#pragma unroll
  for (int jy = 0; jy < N; ++jy) {
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const S* q = src + (jx + N * jy) * PL;
      constexpr int dummy = 0;
      (void)dummy;
      const int ox = node_snapped(N, HI, jx) ? snapped_offset(N, jx) : L.off[jx];
      const int oy = node_snapped(N, HI, jy) ? snapped_offset(N, jy) : L.off[jy];
      q += ox + oy * kTXP;
      R acc;
      if (node_snapped(N, HI, jy)) {
        acc = node_snapped(N, HI, jx) ? static_cast<R>(q[0]) : row_interp<N, HI, P, S, R>(q, L, jx);
      } else {
        constexpr int rr = (P - 1) / 2;
        R rv[P];
#pragma unroll
        for (int b = 0; b < P; ++b)
          rv[b] = node_snapped(N, HI, jx) ? static_cast<R>(q[b * kTXP])
                                          : row_interp<N, HI, P, S, R>(q + b * kTXP, L, jx);
        acc = rv[rr];
#pragma unroll
        for (int b = 0; b < P; ++b)
          if (b != rr) acc += L.w[jy][b] * (rv[b] - rv[rr]);
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
  drho = dr;
  R dx[N], dy[N];
  dphi<R>(L, N, ux, dx);
  dphi<R>(L, N, uy, dy);
  R px[N];
#pragma unroll
  for (int jx = 0; jx < N; ++jx) px[jx] = L.w1[jx] + dx[jx];
  const uint32_t key = hash32((uint32_t)obase ^ (seed * 0x9e3779b9u));  // FP16 rounding only
#pragma unroll
  for (int jy = 0; jy < N; ++jy) {
    const R py = L.w1[jy] + dy[jy];
    const R ty = dr * py;
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const int i = jx + N * jy;
      // f^L - W = dr px py + w_x dphi_y + dphi_x (w_y + dphi_y)
      const R feq = px[jx] * ty + L.w1[jx] * dy[jy] + dx[jx] * py;
      const size_t idx = (size_t)i * p.plane + obase;
      fout[idx] = to_storage<S, R>(f[i] + p.omega * (feq - f[i]), pop_random(key, i));
    }
  }
}

constexpr int kStages = 2;            // staged work items in flight per CTA

// Work item: tile t (coordinates tx, ty) and lattice k, for every lattice the
// tile's mask holds (bit 0 low-order, bit 1 high-order); t = ntiles ends the
// walk.
struct Item {
  int t, tx, ty, k;
};

// Dynamic tile scheduler of one CTA (run by one thread).  Tiles are taken
// from a global counter, so CTAs that draw expensive tiles (high-order
// lattice, two lattices) take fewer of them: a cluster of high-order tiles
// does not pile up on the CTAs a static stride would give it.  The counter's
// result and the taken tile's mask are fetched one decision ahead, so their
// latencies overlap the computation.
struct TileScheduler {
  int* ctr;
  const uint8_t* mask_g;
  int ntiles, ntx;
  int t_next, m_next;  // next tile to use and its mask (fetched)
  int t_after;         // the one after it (counter value in flight)
  Item cur;            // last decided item
  int cur_mask;

  __device__ __forceinline__ int take() { return atomicAdd(ctr, 1); }
  __device__ __forceinline__ void start() {
    t_next = take();
    m_next = t_next < ntiles ? mask_g[t_next] : 0;
    t_after = take();
    cur.t = -1;
    cur.k = 1;
    cur_mask = 0;
  }
  // The item after the last decided one.
  __device__ __forceinline__ Item decide() {
    if (cur.t >= ntiles) return cur;
    if (cur.t >= 0 && cur.k == 0 && (cur_mask & 2)) {
      cur.k = 1;
      return cur;
    }
    const int t = t_next;
    cur_mask = m_next;
    // fetch the following tile's mask, take the one after
    t_next = t_after < ntiles ? t_after : ntiles;
    m_next = t_next < ntiles ? mask_g[t_next] : 0;
    t_after = t_next < ntiles ? take() : ntiles;
    if (t >= ntiles) {
      cur = Item{ntiles, 0, 0, 0};
      return cur;
    }
    cur = Item{t, t % ntx, t / ntx, (cur_mask & 1) ? 0 : 1};
    return cur;
  }
};

// Position of the k-th (0-based) set bit of b, k < popc(b): a binary search
// on the population counts of halves.
__device__ __forceinline__ int select_bit(uint32_t b, int k) {
  int pos = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1) {
    const int c = __popc(b & ((1u << w) - 1u));
    if (k >= c) {
      k -= c;
      b >>= w;
      pos += w;
    }
  }
  return pos;
}

// Cell of the tile (raster index ty * 32 + tx) that thread `slot` computes
// for an item whose cells of the item's lattice are given by the warps'
// ballots b[0..7]: the slot-th set bit in raster order, or -1.  Threads take
// the item's cells densely, so a lattice that covers a few cells of a tile
// occupies a few warps instead of idling lanes in every warp.
__device__ __forceinline__ int compact_cell(const uint32_t* b, int slot) {
  uint32_t all = 0xffffffffu;
#pragma unroll
  for (int w = 0; w < kTY; ++w) all &= b[w];
  if (all == 0xffffffffu) return slot;  // the lattice covers the whole tile
  int base = 0;
#pragma unroll
  for (int w = 0; w < kTY; ++w) {
    const int c = __popc(b[w]);
    if (slot < base + c) return w * kTX + select_bit(b[w], slot - base);
    base += c;
  }
  return -1;
}

constexpr int kRing = 4;  // decided items visible to every thread: j .. j + 3

// Persistent stream-collide: each CTA walks its items through a kStages-deep
// ring of staged buffers.  Thread 0 decides the items three ahead (dynamic
// scheduler) and keeps kStages TMA copies in flight (the next items' planes
// load while the current item computes); the threads compute the item's
// cells, compacted onto the leading threads, then free the stage.
template <int NL, int NH, int P, class S, class R>
__global__ void __launch_bounds__(kTX * kTY, StageGeom<S>::min_blocks)
k_stream_collide(const Params<R> p, const __grid_constant__ CUtensorMap tm0,
                 const __grid_constant__ CUtensorMap tm1, S* __restrict__ fout0,
                 S* __restrict__ fout1, const uint8_t* __restrict__ flag_cur,
                 uint8_t* __restrict__ flag_nxt, const uint8_t* __restrict__ tile_mask_g,
                 uint8_t* __restrict__ mask_next, int ntx, int ntiles, const BcDev bc,
                 int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ Item ring[kRing];                // decided items, by index & (kRing - 1)
  __shared__ int tile_bits[3];                // next-step mask of the tile being finished
  __shared__ uint32_t ballots[2][kTY];        // cells of the item's lattice, per warp
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
  constexpr int GH = stage_halo(P);
  constexpr int kTXP = StageGeom<S>::txp, kXH = StageGeom<S>::xh;
  constexpr int pl = (kTY + 2 * GH) * kTXP;  // staged elements per plane (rows y0-GH ..)
  constexpr int stage = NH * NH * pl;        // staged elements per stage (larger lattice)
  S* sm = reinterpret_cast<S*>(smem_raw);
  TileScheduler sched;
  auto issue = [&](const Item& q, int s) {
    const int Q = q.k ? NH * NH : NL * NL;
    mbar_expect_tx(&full[s], (uint32_t)(Q * pl * (int)sizeof(S)));
    tma_load_3d(sm + s * stage, q.k ? &tm1 : &tm0, &full[s], q.tx * kTX + kOX - kXH,
                q.ty * kTY + p.G - GH, 0);
  };
  if (tid == 0) {
    // this launch's counter p.sched[parity] was cleared by the previous launch;
    // clear the other one for the next
    if (blockIdx.x == 0) {
      p.sched[p.sched_parity ^ 1] = 0;
      p.wcount[p.sched_parity ^ 1] = 0;  // the other work list, likewise
    }
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
    tile_bits[0] = tile_bits[1] = tile_bits[2] = 0;
    sched = TileScheduler{p.sched + p.sched_parity, tile_mask_g, ntiles, ntx, 0, 0, 0, Item{}, 0};
    sched.start();
    for (int j = 0; j < kRing - 1; ++j) ring[j] = sched.decide();
    for (int s = 0; s < kStages; ++s)
      if (ring[s].t < ntiles) issue(ring[s], s);
  }
  __syncthreads();
  // this thread's raster cell flag for an item (2 outside the grid)
  auto cell_flag = [&](const Item& q) -> int {
    if (q.t >= ntiles) return 2;
    const int xx = q.tx * kTX + tx, yy = q.ty * kTY + ty;
    return (xx < p.nx && yy < p.ny) ? flag_cur[xx + p.nx * yy] : 2;
  };
  {
    const Item it0 = ring[0];
    const uint32_t b = __ballot_sync(0xffffffffu, cell_flag(it0) == it0.k);
    if (tx == 0) ballots[0][ty] = b;
  }
  int fl_next = cell_flag(ring[1]);  // flags are loaded one item ahead
  __syncthreads();
  const uint32_t seed = *p.seed_ctr;  // FP16 rounding key of this step
  int bits = 0;  // cells this thread computed: bit 0/1 = next-step lattice, bit 2 = flipped
  // threads 0-8: a work-word atomic and a list slot whose results are used
  // at the next tile end (tile -1: none)
  int pend_t = -1, pend_was = 0, slot_t = -1, slot = 0;
  for (int j = 0;; ++j) {
    const Item it = ring[j & (kRing - 1)];
    if (it.t >= ntiles) break;
    const Item nx_it = ring[(j + 1) & (kRing - 1)];
    const Item nn_it = ring[(j + 2) & (kRing - 1)];
    if (tid == 0) ring[(j + 3) & (kRing - 1)] = sched.decide();  // published by the barrier
    const int s = j % kStages;
    const int x0 = it.tx * kTX, y0 = it.ty * kTY;
    const int cell = compact_cell(ballots[j & 1], tid);
    // ballot of the next item's cells (published by the barrier below)
    {
      const uint32_t b = __ballot_sync(0xffffffffu, fl_next == nx_it.k);
      if (tx == 0) ballots[(j + 1) & 1][ty] = b;
    }
    if (!mbar_wait(&full[s], (uint32_t)((j / kStages) & 1))) {
      // bounded: record, give the copy one more bounded wait, stop
      if (tid == 0) atomicExch(err, 1);
      mbar_wait(&full[s], (uint32_t)((j / kStages) & 1));
      return;
    }
    fl_next = cell_flag(nn_it);
    if (cell >= 0) {
      const int cx = cell & (kTX - 1), cy = cell / kTX;
      const S* src = sm + s * stage + (cy + GH) * kTXP + (cx + kXH);
      const int x = x0 + cx, y = y0 + cy;
      const int obase = (y + p.G) * p.pitch + (x + kOX);
      R ux, uy, dr;  // dr: density deviation (unused here)
      if (it.k == 0)
        stream_collide_cell<NL, false, P, S, R>(p, p.lat[0], src, fout0, obase, seed, ux, uy, dr);
      else
        stream_collide_cell<NH, true, P, S, R>(p, p.lat[1], src, fout1, obase, seed, ux, uy, dr);
      int nf = it.k;
      if (p.crit == 1) {
        nf = sqrt(ux * ux + uy * uy) > p.thr ? 1 : 0;
        flag_nxt[x + p.nx * y] = (uint8_t)nf;
      }
      bits |= (1 << nf) | (nf != it.k ? 4 : 0);
    }
    // after a tile's last item: the lattices its cells carry next step and
    // whether any flipped (read by the post-step kernel to skip quiet tiles
    // and by the next launch's scheduler), OR-reduced per warp, then through
    // a shared word made visible by the stage-release barrier below
    const bool tile_end = nx_it.t != it.t;
    if (tile_end) {
      const int wbits = __reduce_or_sync(0xffffffffu, bits);
      if (tx == 0 && wbits) atomicOr(&tile_bits[j % 3], wbits);
      bits = 0;
    }
    // the slot the next item accumulates into was last read two items ago
    if (tid == 0) tile_bits[(j + 1) % 3] = 0;
    __syncthreads();  // stage s is free again; tile_bits, ballots and ring complete
    if (tile_end && tid < 9) {
      // the tile's next-step mask, and its contribution to the post-step
      // kernel's work bits of the 3 x 3 tile neighbourhood: the lattices (all
      // nine) and the flip bit (the tile itself); a tile has conversion work
      // iff its word ends with both lattices or a flip, and is then listed
      const int m = tile_bits[j % 3];
      if (tid == 0) mask_next[it.t] = (uint8_t)m;
      int ntx_ = it.tx + tid % 3 - 1, nty_ = it.ty + tid / 3 - 1;
      const int nty = (ntiles + ntx - 1) / ntx;
      bool ok = true;
      if (ntx_ < 0 || ntx_ >= ntx) {
        if (p.periodic_x) ntx_ = ntx_ < 0 ? ntx_ + ntx : ntx_ - ntx;
        else ok = false;
      }
      if (nty_ < 0 || nty_ >= nty) {
        if (p.periodic_y) nty_ = nty_ < 0 ? nty_ + nty : nty_ - nty;
        else ok = false;
      }
      // listing as add_work, with each returning atomic's result used one
      // tile later, so the CTA does not wait for it
      const int half = p.sched_parity;
      if (slot_t >= 0) p.wlist[(size_t)half * ntiles + slot] = slot_t;
      slot_t = -1;
      if (pend_t >= 0 && !(pend_was & 6)) {
        slot = atomicAdd(p.wcount + half, 1);
        slot_t = pend_t;
      }
      pend_t = -1;
      const int contrib = (m & 3) | (tid == 4 ? (m & 4) : 0);
      if (ok && contrib) {
        int* w = p.work + (size_t)half * ntiles + nty_ * ntx + ntx_;
        if (contrib & 6) {
          pend_was = atomicOr(w, contrib);
          pend_t = nty_ * ntx + ntx_;
        } else {
          atomicOr(w, contrib);
        }
      }
      // the other half is the next step's: clear this tile's word there
      if (tid == 0) p.work[(p.sched_parity ^ 1) * ntiles + it.t] = 0;
    }
    if (tid == 0) {
      if (nn_it.t < ntiles) {
        // order the CTA's shared-memory reads of stage s before the async-proxy write
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(nn_it, s);
      }
    }
  }
  if (tid < 9) {  // the deferred listings of the last tile
    const size_t h = (size_t)p.sched_parity * ntiles;
    if (slot_t >= 0) p.wlist[h + slot] = slot_t;
    if (pend_t >= 0 && !(pend_was & 6)) p.wlist[h + atomicAdd(p.wcount + p.sched_parity, 1)] = pend_t;
  }
}

template <class S, class R>
cudaError_t launch_stream_collide_impl(const Params<R>& p, int P, const CUtensorMap* tm0,
                                       const CUtensorMap* tm1, S* fout0, S* fout1,
                                       const uint8_t* flag_cur, uint8_t* flag_nxt,
                                       const uint8_t* tile_mask, uint8_t* mask_next,
                                       const BcDev& bc, int* err, cudaStream_t st) {
  const dim3 blk(kTX, kTY);
  const int ntx = (p.nx + kTX - 1) / kTX, nty = (p.ny + kTY - 1) / kTY;
  const int ntiles = ntx * nty;
  const int nl = p.lat[0].n, nh = p.lat[1].n;
  const size_t smem =
      (size_t)kStages * nh * nh * (kTY + 2 * stage_halo(P)) * StageGeom<S>::txp * sizeof(S);
  if (p.G < stage_halo(P)) return cudaErrorInvalidValue;  // ghost ring narrower than the stage halo
  const int nsm = p.nsm;
  // the dynamic shared-memory attribute and the occupancy are per device:
  // cached per device ordinal (handles of one process may live on several)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return cudaErrorInvalidDevice;
#define SLBM_SC_CASE(NL, NH, PP)                                                            \
  if (nl == NL && nh == NH && P == PP) {                                                    \
    auto kern = k_stream_collide<NL, NH, PP, S, R>;                                         \
    static size_t attr_set[kMaxDevices] = {}; /* largest dynamic size granted so far */     \
    if (smem > attr_set[dev]) {                                                             \
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                           (int)smem);                                      \
      if (e != cudaSuccess) return e;                                                       \
      attr_set[dev] = smem;                                                                 \
    }                                                                                       \
    static size_t occ_smem[kMaxDevices] = {}; /* occupancy queried once per size */         \
    static int occ_per_sm[kMaxDevices] = {};                                                \
    if (occ_smem[dev] != smem) {                                                            \
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_per_sm[dev], kern, \
                                                                    kTX * kTY, smem);       \
      if (e != cudaSuccess) return e;                                                       \
      occ_smem[dev] = smem;                                                                 \
    }                                                                                       \
    const int per_sm = occ_per_sm[dev];                                                     \
    if (per_sm < 1) return cudaErrorInvalidConfiguration;                                   \
    const int grid = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;                         \
    kern<<<grid, blk, smem, st>>>(p, *tm0, *tm1, fout0, fout1, flag_cur, flag_nxt,          \
                                  tile_mask, mask_next, ntx, ntiles, bc, err);              \
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
