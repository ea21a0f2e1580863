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

constexpr int kXH = 4;                           // halo columns each side (>= G, 16-byte aligned)
constexpr int kTXP = kTX + 2 * kXH;              // staged row length (40)
constexpr long long kWaitCycles = 2000000000LL;  // ~1 s bound on an mbarrier wait

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
// elements apart, rows kTXP apart), on deviations s_i = f_i - W_i (streaming
// is affine in the shift; the collision uses the deviation form of the
// product equilibrium, see slbm_eq.cuh).
template <int N, bool HI, int P, class S, class R>
__device__ __forceinline__ void stream_collide_cell(const Params<R>& p, const LatTab<R>& L,
                                                    const S* src, S* __restrict__ fout,
                                                    int obase, R& ux, R& uy, R& drho) {
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
#pragma unroll
  for (int jy = 0; jy < N; ++jy) {
    const R py = L.w1[jy] + dy[jy];
#pragma unroll
    for (int jx = 0; jx < N; ++jx) {
      const int i = jx + N * jy;
      const R px = L.w1[jx] + dx[jx];
      const R feq = dr * px * py + L.w1[jx] * dy[jy] + dx[jx] * L.w1[jy] + dx[jx] * dy[jy];
      fout[(size_t)i * p.plane + obase] = static_cast<S>(f[i] + p.omega * (feq - f[i]));
    }
  }
}

constexpr int kStages = 2;            // staged work items in flight per CTA
constexpr int kMaxTilesPerCta = 4096;  // tile masks a persistent CTA keeps in shared memory

// Work item of a persistent CTA: tile t (this CTA owns t = blockIdx.x,
// blockIdx.x + gridDim.x, ...) and lattice k, for every lattice the tile's
// mask holds (bit 0 low-order, bit 1 high-order).
struct Item {
  int t, k;
};

// `mask` holds the masks of this CTA's tiles by local index (t - blockIdx.x) / gridDim.x.
__device__ __forceinline__ int local_mask(const uint8_t* mask, int t) {
  return mask[(t - (int)blockIdx.x) / (int)gridDim.x];
}

__device__ __forceinline__ Item first_item(const uint8_t* mask, int ntiles) {
  Item it{(int)blockIdx.x, 0};
  if (it.t < ntiles && !(local_mask(mask, it.t) & 1)) it.k = 1;
  return it;
}

__device__ __forceinline__ Item next_item(Item it, const uint8_t* mask, int ntiles) {
  if (it.k == 0 && (local_mask(mask, it.t) & 2)) return Item{it.t, 1};
  it.t += gridDim.x;
  it.k = (it.t < ntiles && !(local_mask(mask, it.t) & 1)) ? 1 : 0;
  return it;
}

// Persistent stream-collide: each CTA walks its items through a kStages-deep
// ring of staged buffers.  One elected thread keeps kStages TMA copies in
// flight (the next items' planes load while the current item computes); all
// threads compute the cells of the item's lattice, then free the stage.
template <int NL, int NH, int P, class S, class R>
__global__ void __launch_bounds__(kTX * kTY, 2)
k_stream_collide(const Params<R> p, const __grid_constant__ CUtensorMap tm0,
                 const __grid_constant__ CUtensorMap tm1, S* __restrict__ fout0,
                 S* __restrict__ fout1, const uint8_t* __restrict__ flag_cur,
                 uint8_t* __restrict__ flag_nxt, const uint8_t* __restrict__ tile_mask_g,
                 uint8_t* __restrict__ mask_next, int ntx, int ntiles, const BcDev bc,
                 int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ uint8_t tmask[kMaxTilesPerCta];  // masks of this CTA's tiles, by local index
  __shared__ int tile_bits[2];                // next-step mask of the tile being finished
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTX + tx;
  for (int m = tid; blockIdx.x + m * gridDim.x < ntiles; m += kTX * kTY)
    tmask[m] = tile_mask_g[blockIdx.x + m * gridDim.x];
  constexpr int GH = stage_halo(P);
  constexpr int pl = (kTY + 2 * GH) * kTXP;  // staged elements per plane (rows y0-GH ..)
  constexpr int stage = NH * NH * pl;        // staged elements per stage (larger lattice)
  S* sm = reinterpret_cast<S*>(smem_raw);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    mbar_fence_init();
    tile_bits[0] = tile_bits[1] = 0;
  }
  __syncthreads();
  const uint8_t* tile_mask = tmask;
  Item pc = first_item(tile_mask, ntiles);  // producer cursor (thread 0 only)
  if (tid == 0)
    for (int s = 0; s < kStages && pc.t < ntiles; ++s) {
      const int Q = pc.k ? NH * NH : NL * NL;
      mbar_expect_tx(&full[s], (uint32_t)(Q * pl * (int)sizeof(S)));
      tma_load_3d(sm + s * stage, pc.k ? &tm1 : &tm0, &full[s], (pc.t % ntx) * kTX + kOX - kXH,
                  (pc.t / ntx) * kTY + p.G - GH, 0);
      pc = next_item(pc, tile_mask, ntiles);
    }
  // this thread's cell flag for an item, loaded one item ahead
  auto cell_flag = [&](const Item& q) -> int {
    if (q.t >= ntiles) return 2;
    const int xx = (q.t % ntx) * kTX + tx, yy = (q.t / ntx) * kTY + ty;
    return (xx < p.nx && yy < p.ny) ? flag_cur[xx + p.nx * yy] : 2;
  };
  int j = 0;
  int bits = 0;  // this thread's cell: bit 0/1 = next-step lattice, bit 2 = flipped
  Item it = first_item(tile_mask, ntiles);
  int fl_next = cell_flag(it);
  for (; it.t < ntiles; ++j) {
    const Item nx_it = next_item(it, tile_mask, ntiles);
    const int fl = fl_next;
    fl_next = cell_flag(nx_it);
    const int s = j % kStages;
    const int x0 = (it.t % ntx) * kTX, y0 = (it.t / ntx) * kTY;
    const int x = x0 + tx, y = y0 + ty;
    if (!mbar_wait(&full[s], (uint32_t)((j / kStages) & 1))) {
      // bounded: record, give the copy one more bounded wait, stop
      if (tid == 0) atomicExch(err, 1);
      mbar_wait(&full[s], (uint32_t)((j / kStages) & 1));
      return;
    }
    if (fl == it.k) {
      const S* cell = sm + s * stage + (ty + GH) * kTXP + (tx + kXH);
      const int obase = (y + p.G) * p.pitch + (x + kOX);
      R ux, uy, dr;  // dr: density deviation (unused here)
      if (it.k == 0)
        stream_collide_cell<NL, false, P, S, R>(p, p.lat[0], cell, fout0, obase, ux, uy, dr);
      else
        stream_collide_cell<NH, true, P, S, R>(p, p.lat[1], cell, fout1, obase, ux, uy, dr);

      int nf = fl;
      if (p.crit == 1) {
        nf = sqrt(ux * ux + uy * uy) > p.thr ? 1 : 0;
        flag_nxt[x + p.nx * y] = (uint8_t)nf;
      }
      bits = (1 << nf) | (nf != fl ? 4 : 0);
    }
    // after a tile's last item: the lattices its cells carry next step and
    // whether any flipped (read by the post-step kernel to skip quiet tiles
    // and by the next launch's producer), OR-reduced per warp, then through
    // a shared word made visible by the stage-release barrier below
    const bool tile_end = nx_it.t != it.t;
    if (tile_end) {
      const int wbits = __reduce_or_sync(0xffffffffu, bits);
      if ((tid & 31) == 0 && wbits) atomicOr(&tile_bits[j & 1], wbits);
      bits = 0;
    }
    __syncthreads();  // stage s is free again; tile_bits complete
    if (tile_end && tid == 0) {
      mask_next[it.t] = (uint8_t)tile_bits[j & 1];
      tile_bits[j & 1] = 0;
    }
    if (tid == 0 && pc.t < ntiles) {
      // order the CTA's shared-memory reads of stage s before the async-proxy write
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const int Q = pc.k ? NH * NH : NL * NL;
      mbar_expect_tx(&full[s], (uint32_t)(Q * pl * (int)sizeof(S)));
      tma_load_3d(sm + s * stage, pc.k ? &tm1 : &tm0, &full[s], (pc.t % ntx) * kTX + kOX - kXH,
                  (pc.t / ntx) * kTY + p.G - GH, 0);
      pc = next_item(pc, tile_mask, ntiles);
    }
    it = nx_it;
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
  const size_t smem = (size_t)kStages * nh * nh * (kTY + 2 * stage_halo(P)) * kTXP * sizeof(S);
  if (p.G < stage_halo(P)) return cudaErrorInvalidValue;  // ghost ring narrower than the stage halo
  const int nsm = p.nsm;
#define SLBM_SC_CASE(NL, NH, PP)                                                            \
  if (nl == NL && nh == NH && P == PP) {                                                    \
    auto kern = k_stream_collide<NL, NH, PP, S, R>;                                         \
    static size_t attr_set = 0; /* largest dynamic size granted so far */                   \
    if (smem > attr_set) {                                                                  \
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                           (int)smem);                                      \
      if (e != cudaSuccess) return e;                                                       \
      attr_set = smem;                                                                      \
    }                                                                                       \
    static size_t occ_smem = 0; /* occupancy is queried once per dynamic size */            \
    static int per_sm = 0;                                                                  \
    if (occ_smem != smem) {                                                                 \
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern,          \
                                                                    kTX * kTY, smem);       \
      if (e != cudaSuccess) return e;                                                       \
      occ_smem = smem;                                                                      \
    }                                                                                       \
    if (per_sm < 1) return cudaErrorInvalidConfiguration;                                   \
    const int grid = ntiles < per_sm * nsm ? ntiles : per_sm * nsm;                         \
    if ((ntiles + grid - 1) / grid > kMaxTilesPerCta) return cudaErrorInvalidValue;         \
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
