// slbm_impl.cuh -- internal declarations of the sm_103a multi-scale
// semi-Lagrangian LBM library: parameter tables passed to every kernel by
// value, the device-memory layout, and the kernel launchers.
//
// Layout in HBM: structure-of-arrays population planes, x fastest.  Every
// plane of lattice k in buffer b holds (ny + 2G) rows of `pitch` elements;
// cell (x, y), x in [-G, nx+G), y in [-G, ny+G), sits at element
// (y + G) * pitch + (x + kOX).  The G-wide ring of ghost cells is refreshed
// after every step (periodic images or boundary states) and read by the
// streaming kernel in place of wrapped indices -- except, on a periodic y
// axis of fewer than kWrapRowsMax rows or with channels (Params::wrap_y),
// the y ghost rows: there the streaming kernel reads the rows' images in the
// grid near its edges, so thin periodic grids (a few rows, where the ghost
// rows hold as many cells as the grid) rewrite no ghost row per step.
//
// Stored values are deviations s_i = f_i - W_i from the rest equilibrium
// (rho = 1, u = 0, whose lattice populations are the weights W_i).  The
// method is affine in that shift (Lagrange weights sum to one, sum W_i = 1,
// sum c_i W_i = 0), and small stored magnitudes keep FP32 rounding small.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

namespace slbm {

constexpr int kMaxN = 5;        // largest 1-D node count (D1Q5)
constexpr int kMaxP = 6;        // largest stencil (order 5)
constexpr int kOX = 32;         // left pad of a row, elements (32-column tiles start on a 128-byte line in FP32)
constexpr int kTX = 32;         // tile width  (one warp per row segment)
constexpr int kTY = 8;          // tile height (8 warps per CTA)

// Stencil shape known at compile time.  With CFL = 1 (Sec. IV) a node's
// shift c_j dt is an exact integer only for the rest node (0) and, on the
// lattice that sets max|c| (the high-order one), the two outer nodes (-+1);
// those are single taps at a fixed offset.  The host checks its tables
// against this at creation.
__host__ __device__ constexpr bool node_snapped(int n, bool hi, int j) {
  return (n % 2 == 1 && j == n / 2) || (hi && (j == 0 || j == n - 1));
}
__host__ __device__ constexpr int snapped_offset(int n, int j) {
  return j == 0 ? 1 : (j == n - 1 ? -1 : 0);  // departure point x - c dt
}
// Ghost / staging halo of a P-point stencil with shifts of at most one cell.
__host__ __device__ constexpr int stage_halo(int P) { return (P + 1) / 2; }

// One lattice of the pair, in the arithmetic type R.
template <class R>
struct LatTab {
  int n;                        // 1-D nodes, Q = n * n
  int off[kMaxN];               // first collocation point of node j, relative to the cell
  int ntap[kMaxN];              // 1 (shift snapped to an integer) or P
  R c[kMaxN];                   // 1-D velocities (T_L = 1, lattice frame)
  R w1[kMaxN];                  // 1-D Gauss-Hermite weights (W_i = w1[ix] w1[iy])
  // Lagrange weights of node j's departure point in differential form: with
  // the reference point r = (P - 1) / 2 the interpolant is
  // v[r] + sum_{a != r} w[a] (v[a] - v[r]) (w[r] stored as 0), which passes
  // constants through exactly even with rounded weights.
  R w[kMaxN][kMaxP];
  R vinv[kMaxN][kMaxN];         // inverse Vandermonde: phi_j(u) = sum_m vinv[j][m] h_m(u)
  // 16-bit companded fixed-point storage (SLBM_FX16): plane i holds
  // q = round(sign(s) sqrt(|s| isc[i])), s = f_i - W_i, read back as
  // sc[i] q |q|; isc = 1 / sc.  Unused by the other storage types.
  R sc[kMaxN * kMaxN];
  R isc[kMaxN * kMaxN];
};

// 16-bit companded fixed-point storage of a deviation s: q with s = sc q |q|
// (sc its plane's scale), so the step between neighbouring values grows like
// sqrt|s| -- fine steps for small deviations, a bounded range for large ones.
struct fx16 {
  int16_t v;
};
template <class S>
__host__ __device__ constexpr bool is_fx16() {
  return std::is_same<S, fx16>::value;
}

// A stored population value in the arithmetic type: plain conversion, or for
// fixed point sc q |q| (q the stored integer, sc the plane's scale).
template <class R, class S>
__device__ __forceinline__ R from_s(S v, R) {
  return static_cast<R>(v);
}
template <class R>
__device__ __forceinline__ R from_s(fx16 v, R sc) {
  const R q = static_cast<R>(v.v);
  return sc * (q * fabs(q));
}

// The companded value sign(v) sqrt(|v| isc) of fixed-point storage, before
// rounding.  The hardware's approximate square root (sqrt.approx.f32, a few
// units in the last of 24 bits) is far finer than the 16-bit rounding that
// follows.
__device__ __forceinline__ float fx_compand(float v, float isc) {
  float r;
  asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(fabsf(v) * isc));
  return copysignf(r, v);
}

// A value to storage, rounded to nearest: plain conversion, or for fixed
// point the companded value rounded, saturating at +-32767.
template <class S, class R>
__device__ __forceinline__ S to_s(R v, R) {
  return static_cast<S>(v);
}
template <>
__device__ __forceinline__ fx16 to_s<fx16, float>(float v, float isc) {
  const float q = fminf(fmaxf(rintf(fx_compand(v, isc)), -32767.f), 32767.f);
  return fx16{(int16_t)__float2int_rn(q)};
}

// Loads through the read-only path (ld.global.nc) and through L2
// (ld.global.cg) of a stored element; fixed point as its raw 16 bits.
template <class S>
__device__ __forceinline__ S ldg_s(const S* a) {
  return __ldg(a);
}
template <>
__device__ __forceinline__ fx16 ldg_s<fx16>(const fx16* a) {
  return fx16{__ldg(reinterpret_cast<const short*>(a))};
}
template <class S>
__device__ __forceinline__ S ldcg_s(const S* a) {
  return __ldcg(a);
}
template <>
__device__ __forceinline__ fx16 ldcg_s<fx16>(const fx16* a) {
  return fx16{__ldcg(reinterpret_cast<const short*>(a))};
}

// Interface conversion tables.
template <class R>
struct ConvTab {
  R lift[kMaxN][kMaxN];         // nQ x nq: non-equilibrium lifting L = VQ^-1[:, :nq] Vq
  R proj[kMaxN][kMaxN];         // nq x nQ: projection P[j][a] = l^q_j(c^Q_a)
};

template <class R>
struct Params {
  int nx, ny;
  int G, pitch, rows;
  long long plane;              // elements per population plane
  int periodic_x, periodic_y;
  int crit;                     // SLBM_CRIT_*
  R thr;                        // Mach threshold
  R omega;
  int band;                     // stencil reach in cells (band radius)
  int nsm;                      // multiprocessors of the handle's device (launch sizing)
  LatTab<R> lat[2];             // 0 = low-order, 1 = high-order
  ConvTab<R> conv;
  uint32_t* seed_ctr;           // step key of the FP16 stochastic rounding (device counter,
                                // advanced by every post-step launch)
  int* sched;                   // two tile counters of the stream kernel's scheduler; sched[2]:
                                // the post-step kernel's item counter (zeroed by the stream kernel)
  int sched_parity;             // the counter (and work-bit half) this step uses
  int* work;                    // 2 x ntiles post-step work bits, accumulated by the stream kernel
  int* wlist;                   // 2 x ntiles: candidate work tiles (see add_work)
  int* wcount;                  // 2 counters: entries of each half of wlist
  double cv;                    // C_v of the two-population co-moving model, else 1
  const R* omega_x;             // per-column omega (channels), else null: omega everywhere
  int wrap_y;                   // 1: periodic y rows are read through their images (no
                                // y ghost rows; see the layout note above)
  int post_warp;                // 1: the per-step post-step kernel runs one warp per tile
                                // (grids of kPostWarpTiles tiles and more), else one CTA per tile
};

constexpr int kPostWarpTiles = 8192;  // tiles from which the warp-per-tile post-step kernel runs

constexpr int kWrapRowsMax = 256;  // periodic y axes shorter than this wrap (wrap_y)

// Flag value of a cell that belongs to no lattice: the gap columns between
// channels (slbm_set_channels), which hold their walls' ghost cells.
constexpr uint8_t kFlagGap = 2;

// A tile has interface-conversion work iff its work word holds both lattices
// (bits 0 and 1, OR-ed from its 3 x 3 tile neighbourhood) or a flip (bit 2).
__device__ __forceinline__ bool post_work_word(int w) { return (w & 4) || (w & 3) == 3; }

// OR `contrib` into the work word of tile t (half `half`).  The first
// contribution that carries the high-order lattice or a flip (bits 1, 2)
// lists t, so the list holds every work tile (each at most once) and also
// tiles whose neighbourhood turns out all high-order, which the post-step
// kernel skips by their final word.  Low-order-only contributions, the common
// case, need no result and use a fire-and-forget atomic.
__device__ __forceinline__ void add_work(int* work, int* wlist, int* wcount, int half, int ntiles,
                                         int t, int contrib) {
  int* w = work + (size_t)half * ntiles + t;
  if (contrib & 6) {
    if (!(atomicOr(w, contrib) & 6))
      wlist[(size_t)half * ntiles + atomicAdd(wcount + half, 1)] = t;
  } else {
    atomicOr(w, contrib);
  }
}

// Co-moving (PonD) frame, Sec. II.C.  Every cell keeps its populations (as
// deviations from W_i) in its own frame lambda = {u_x, u_y, T}, stored in three
// dense nx*ny planes (stride nc).  Grids are periodic; indices wrap.
template <class R>
struct PondLat {
  int n;
  R c[kMaxN];                   // 1-D velocities at T_L = 1
  R w[kMaxN];                   // 1-D weights
  R inv[kMaxN][kMaxN];          // 1 / (c_a - c_m) for a != m (Lagrange basis on the nodes)
  R vinv[kMaxN][kMaxN];         // inverse Vandermonde: phi_a = sum_m vinv[a][m] h_m
};

template <class R>
struct PondParams {
  int nx, ny, G, pitch;
  long long plane;              // population plane stride (elements)
  long long nc;                 // frame plane stride (nx * ny)
  R omega, dt;
  R tol;                        // predictor-corrector tolerance on |du|, |dT|
  int maxit;                    // reconstructions per cell update at most
  int thermal;                  // 1: T from the energy (C_v = D/2); 0: T = T_L
  int twopop;                   // 1: two-population model (g planes, C_v, omega_2)
  R cv, cvm1, omega2;           // C_v, C_v - 1, omega_2 of the two-population model
  // batched quasi-one-dimensional instances (slbm_set_rows): every row is an
  // independent instance, uniform across y, with row_len[y] active cells and
  // fixed end states row_ends[8 y ..] = left {rho, u_x, u_y, T}, right {...}
  int rows;
  const int* row_len;
  const double* row_ends;
  // viscosity law (two-population model): mu = row_visc[2 y] (T / row_visc[2 y + 1])^s_exp,
  // omega_1 from mu = (1/omega_1 - 1/2) rho T dt, omega_2 from Pr = 1 / inv_pr
  int hs;
  const double* row_visc;
  R s_exp, inv_pr;
  int bx, by;                   // thread-block shape of the step kernel (bx * by = 256)
  int nsm;                      // multiprocessors of the device
  int P;                        // collocation points per axis
  R reach;                      // largest departure distance allowed, cells
  PondLat<R> lat[2];
  R proj[kMaxN][kMaxN];         // P[j][A], as ConvTab (frame-independent)
};

// Largest co-moving departure distance, cells.  Interface conversions cover
// the 3 x 3 tile neighbourhood of every tile (tiles are kTY = 8 rows high), so
// a stencil node may lie at most 8 rows away: reach + (P + 1) / 2 <= 8 for
// P <= 6.
constexpr double kPondReach = 5.0;

// Device error word bits.
constexpr int kErrTimeout = 1;  // a bounded wait ran out (the handle fails)
constexpr int kErrNoConv = 2;   // a co-moving predictor-corrector stopped at maxit
constexpr int kErrFrame = 4;    // non-positive / non-finite frame, or departure beyond reach

// Boundary description (device arrays of the prescribed states, may be null).
// Internal walls (channels, slbm_set_channels): nwall extra ghost cells
// beyond the ring, ghost index ring + e for e < nwall, each a diffuse wall
// against an interior source cell in its row: wall[e] = {gx, gy, sx, side},
// with wall velocity (wall_u[2e], wall_u[2e + 1]).  Rows 0 .. ny-1 only: y
// is periodic and a channel handle always wraps it (wrap_y).
struct BcDev {
  int kind[4];                  // per side SLBM_BC_*
  const double* rho[4];
  const double* ux[4];
  const double* uy[4];
  int nwall;
  const int4* wall;
  const double* wall_u;
};

// Co-moving frame launchers (slbm_pond.cu).  lam: three frame planes.
template <class S, class R>
cudaError_t launch_pond_init(const PondParams<R>& p, S* f0, S* f1, S* e0, S* e1, S* lam,
                             const double* rho, const double* ux, const double* uy,
                             const double* T, cudaStream_t st);
// One co-moving step: f planes f0 / f1 (and, two-population model, g planes
// e0 / e1) with frames lam -> g0 / g1 (eo0 / eo1) with frames lam_out.  The g
// planes hold g / T_frame - (C_v - 1) W_i (deviation of the g populations in
// units of the frame temperature); null when the model has one population.
// split: one launch per lattice (when both are in use), each carrying only
// its lattice's code.
template <class S, class R>
cudaError_t launch_pond_step(const PondParams<R>& p, const S* f0, const S* f1, const S* e0,
                             const S* e1, const S* lam, S* g0, S* g1, S* eo0, S* eo1,
                             S* lam_out, const uint8_t* flag, int* err, int split,
                             cudaStream_t st);
// Per 32 x 8 tile: bit 1 / 2 if it holds a cell of lattice 0 / 1 (flag), bit
// 4 if a cell's lattice differs from flag_old (when given).
cudaError_t launch_pond_masks(int nx, int ny, const uint8_t* flag, const uint8_t* flag_old,
                              uint8_t* mask, cudaStream_t st);
// Cell lists of one interface conversion (device): count[0] cells to lift
// (computed in the low-order lattice) in lift[], count[1] to project in proj[],
// each with room for every cell of the grid.
struct ConvLists {
  int* count;
  int* lift;
  int* proj;
};

// Each converted cell's other lattice from its current one (flag): a light
// screening launch lists the cells, then one thread per listed cell converts
// (lifts first, so a warp mostly runs one of the two).  flag_to
// given: only the cells whose lattice flag_to changes (they take the result as
// their new native vector); else mask null: every cell; else the cells of
// tiles whose 3 x 3 tile neighbourhood holds both lattices (batched rows: the
// cells that read the other lattice) and, with near_change, a cell whose
// lattice changed (mask bit 4, see launch_pond_masks).
template <class S, class R>
cudaError_t launch_pond_convert(const PondParams<R>& p, S* f0, S* f1, S* e0, S* e1, const S* lam,
                                const uint8_t* flag, const uint8_t* mask, const uint8_t* flag_to,
                                int near_change, const ConvLists& lists, cudaStream_t st);
template <class S, class R>
cudaError_t launch_pond_frame_io(const PondParams<R>& p, S* lam, double* ux, double* uy,
                                 double* T, int unpack, cudaStream_t st);
// Knudsen refinement criterion on batched rows (Sec. IV.C): new flags to out.
template <class S, class R>
cudaError_t launch_pond_kn(const PondParams<R>& p, const S* f0, const S* f1, const S* e0,
                           const S* e1, const S* lam, const uint8_t* flag, double thr,
                           uint8_t* out, cudaStream_t st);
// Plane i of lattice k's g planes e to / from absolute g = T_frame (s + (C_v - 1) W_i)
// (nc doubles, cell-major within the plane).
template <class S, class R>
cudaError_t launch_pond_gio(const PondParams<R>& p, int k, int i, S* e, const S* lam, double* buf,
                            int unpack, cudaStream_t st);

// Learned refinement indicator (slbm_indicator.cu): MLP 16 -> 32 -> 32 -> 1
// with FP16 weights w1 (16 x 32) and w2 (32 x 32), row-major K x N, FP32 biases
// and output weights.
struct IndicatorDev {
  const __half* w1;             // null: features only
  const float* b1;
  const __half* w2;
  const float* b2;
  const float* w3;
  float b3;
};

// Learned indicator on the current buffer: features and the MLP in one
// launch; features (nc x 16 FP32), logits and flags (logit > thr) to any of
// the non-null outputs.
template <class S, class R>
cudaError_t launch_indicator(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                             const IndicatorDev& w, float thr, float* feat_out, float* logit_out,
                             uint8_t* flag_out, cudaStream_t st);

// Refinement buffer along one axis (0 = x, 1 = y) of radius r: see k_dilate.
cudaError_t launch_dilate(const uint8_t* in, const uint8_t* keep, uint8_t* out, int nx, int ny,
                          int periodic, int r, int axis, cudaStream_t st);

// Per-cell lattice loss || a - b ||_2 / rho_a over the high-order planes of
// two population buffers a, b (same layout as the handle's planes of lattice
// 1); gap cells get 0.  out: nc doubles.
template <class S, class R>
cudaError_t launch_lattice_loss(const Params<R>& p, const S* a, const S* b, const uint8_t* flag,
                                double* out, cudaStream_t st);

// Indicator training (slbm_indicator.cu): `steps` Adam steps of mini-batch
// `batch` in one single-block launch.  Device arrays: x (n x 16 FP32
// features), y (n labels), idx (steps x batch sample indices, validated by the
// caller), params (kMlpParams FP32, in / out), adam (2 x kMlpParams, in / out),
// loss (steps, or null), grad (kMlpParams, the last step's gradient, or null).
constexpr int kMlpParams = 16 * 32 + 32 + 32 * 32 + 32 + 32 + 1;
constexpr int kMlpMaxBatch = 512;
cudaError_t launch_mlp_train(const float* x, const float* y, const int* idx, int steps, int batch,
                             float lr, float beta1, float beta2, float eps, int t0, float* params,
                             float* adam, float* loss, float* grad, cudaStream_t st);

// Launchers (defined in the kernel translation units).  S = storage type,
// R = arithmetic type.  fin0 / fin1 and fout0 / fout1: base of the input and
// output buffers' planes of lattice 0 / 1.  Stream-collide of every cell
// (each in its flag_cur lattice) into the output buffer; with the criterion
// on, the next flags to flag_nxt; the next-step tile masks to mask_next and
// the post-step work words / list (Params::work, wlist, wcount).
template <class S, class R>
cudaError_t launch_stream_collide(const Params<R>& p, int P, const S* fin0, const S* fin1,
                                  S* fout0, S* fout1, const uint8_t* flag_cur,
                                  uint8_t* flag_nxt, const uint8_t* tile_mask,
                                  uint8_t* mask_next, cudaStream_t st);
// The same with rows read through their periodic images near the y edges
// (Params::wrap_y; its own translation units, called by launch_stream_collide).
template <class S, class R>
cudaError_t launch_stream_collide_wrap(const Params<R>& p, int P, const S* fin0, const S* fin1,
                                       S* fout0, S* fout1, const uint8_t* flag_cur,
                                       uint8_t* flag_nxt, const uint8_t* tile_mask,
                                       uint8_t* mask_next, cudaStream_t st);

// Post-step: interface conversion for band / flipped cells (flag_old = the
// lattice each cell was computed in, flag_new = next step's flags) and, if
// `images`, the ghost images of boundary cells.  Tile masks (bit 0: a
// low-order cell, bit 1: a high-order cell, bit 2: a flip): after a step,
// mask_in holds the stream kernel's masks of flag_new and quiet tiles are
// skipped; in setup calls mask_in is null and the masks of flag_new are
// written to tile_mask.
template <class S, class R>
cudaError_t launch_post(const Params<R>& p, S* f0, S* f1, const uint8_t* flag_old,
                        const uint8_t* flag_new, const BcDev& bc, int images,
                        const uint8_t* mask_in, uint8_t* tile_mask, cudaStream_t st);

// Full ghost-ring fill of one buffer (setup paths: every ghost, including the
// constant DIRICHLET states).
template <class S, class R>
cudaError_t launch_ghosts(const Params<R>& p, S* f0, S* f1, const uint8_t* flag,
                          const BcDev& bc, cudaStream_t st);

// Tile masks and post-step work after flags changed between steps (the
// learned indicator): per 32 x 8 tile the lattices of its new flags and
// whether a flag flipped (mask, read by the next stream step), OR-ed into the
// work words of its 3 x 3 tile neighbourhood as the stream kernel does, with
// the work tiles listed (add_work).  Half `half` of work / wlist / wcount is
// used and must be zero on entry.
cudaError_t launch_tile_work(int nx, int ny, int periodic_x, int periodic_y,
                             const uint8_t* flag_old, const uint8_t* flag_new, uint8_t* mask,
                             int* work, int* wlist, int* wcount, int half, cudaStream_t st);

// Per-tile ghost lists: the ring cells (ghost_coords order) idx[start[t] ..
// start[t + 1]) have their source cell (ghost_source) in tile t; tiles[0 ..
// ntiles) are the tiles with at least one.  DIRICHLET ghosts, constant, are
// in no list.
struct GhostTables {
  const int* start;  // ntiles_total + 1
  const int* idx;
  const int* tiles;
  int ntiles;
};

// Source tile of every ghost ring cell under the ghost rule (-1: a constant
// DIRICHLET ghost, or with skip_y a y ghost row), ntx tiles per row: out[0 .. ring) with
// ring = 2 G (nx + 2 G) + 2 G ny.  The host sorts these into GhostTables.
cudaError_t launch_ghost_src(int G, int nx, int ny, int periodic_x, int periodic_y, int skip_y,
                             const BcDev& bc, int* out, cudaStream_t st);

// Per-step post-step kernel: interface conversion of the candidate tiles in
// `list` (*nlist entries, listed by the stream kernel or the tile-work
// kernel) whose final word in `work` (the same half) is work, spread evenly
// over the CTAs, and the ghost images of every tile in `gt`, each written by
// the CTA that owns its source tile (after the tile's conversion, if any).
template <class S, class R>
cudaError_t launch_post_step(const Params<R>& p, S* f0, S* f1, const uint8_t* flag_old,
                             const uint8_t* flag_new, const BcDev& bc, const int* work,
                             const int* list, const int* nlist, const GhostTables& gt,
                             cudaStream_t st);

// Largest |f^L_i - W_i| per plane of both lattices over the equilibria at
// (rho, u) of every cell, as float bits into out[k * 25 + i] (zeroed by the
// caller): the range of the SLBM_FX16 plane scales.
cudaError_t launch_fx_range(const Params<float>& p, const double* rho, const double* ux,
                            const double* uy, unsigned* out, cudaStream_t st);

template <class S, class R>
cudaError_t launch_init_eq(const Params<R>& p, S* f0, S* f1, const double* rho,
                           const double* ux, const double* uy, cudaStream_t st);

template <class S, class R>
cudaError_t launch_moments(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                           double* rho, double* ux, double* uy, double* T, const S* lam,
                           cudaStream_t st, const S* e0 = nullptr, const S* e1 = nullptr);

template <class S, class R>
cudaError_t launch_criterion(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                             uint8_t* flag_new, cudaStream_t st);

template <class S, class R>
cudaError_t launch_audit(const Params<R>& p, const S* f0, const S* f1, const uint8_t* flag,
                         double* partials, int nparts, double* out4, const S* lam,
                         cudaStream_t st, const S* e0 = nullptr, const S* e1 = nullptr);

template <class S, class R>
cudaError_t launch_pack(const Params<R>& p, int k, int i0, int cnt, const S* f, double* out,
                        int unpack, S* fw, const double* in, cudaStream_t st);

int audit_parts(int nx, int ny);

// Host Gauss-Hermite nodes / weights of the n-node 1-D lattice (Table I),
// computed as the roots of He_n (defined with the other host tables).
void host_gauss_hermite(int n, double* c, double* w);

}  // namespace slbm
