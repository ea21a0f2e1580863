// slbm_api.cu -- the C ABI (include/slbm.h): handle, device-memory layout,
// host-side constant tables and the per-step launch sequence.
//
// Host tables are computed here, independently of any other component:
//  - Gauss-Hermite nodes as the roots of the probabilists' Hermite polynomial
//    He_n (bisection + Newton on the three-term recurrence) and the weights
//    w_j = (n-1)! / (n He_{n-1}(c_j)^2); these reproduce Table I.
//  - The inverse Vandermonde matrix as the monomial coefficients of the
//    Lagrange basis on the nodes (its row j gives l_j).
//  - Per 1-D node, the Lagrange stencil of the departure point x - c_j dt
//    (eqs. reconstructionPond / advectionPond), dt = CFL / max|c| with CFL = 1
//    over the pair (Sec. IV).
//  - The lifting and projection matrices of the interface kernel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "../../include/slbm.h"
#include "slbm_impl.cuh"

using namespace slbm;

namespace {

thread_local char g_create_err[256] = "";

// ------------------------------------------------------------ host tables

double hermite_e(int n, double x, double* dprev = nullptr) {
  double hm1 = 0.0, h = 1.0;  // He_{-1} := 0, He_0 = 1
  for (int k = 0; k < n; ++k) {
    const double hn = x * h - k * hm1;
    hm1 = h;
    h = hn;
  }
  if (dprev) *dprev = hm1;    // He_{n-1}(x)
  return h;
}

void gauss_hermite(int n, double* c, double* w) {
  // roots of He_n: sign changes on a fine grid over [-2 sqrt(n) - 1, ...], then
  // bisection to convergence and one Newton polish (He_n' = n He_{n-1})
  const double lim = 2.0 * std::sqrt((double)n) + 1.0;
  const int M = 20000;
  int found = 0;
  double xa = -lim, fa = hermite_e(n, xa);
  for (int s = 1; s <= M && found < n; ++s) {
    const double xb = -lim + 2.0 * lim * s / M, fb = hermite_e(n, xb);
    if (fa == 0.0 || fa * fb < 0.0) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid == lo || mid == hi) break;
        const double fm = hermite_e(n, mid);
        if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
      }
      double r = fa == 0.0 ? xa : 0.5 * (lo + hi);
      double dp;
      const double fr = hermite_e(n, r, &dp);
      if (dp != 0.0) r -= fr / (n * dp);
      c[found++] = r;
    }
    xa = xb;
    fa = fb;
  }
  // exact symmetry about 0
  for (int j = 0; j < n / 2; ++j) {
    const double a = 0.5 * (c[n - 1 - j] - c[j]);
    c[j] = -a;
    c[n - 1 - j] = a;
  }
  if (n % 2) c[n / 2] = 0.0;
  double fact = 1.0;
  for (int k = 2; k < n; ++k) fact *= k;  // (n-1)!
  for (int j = 0; j < n; ++j) {
    double hp;
    hermite_e(n, c[j], &hp);
    w[j] = fact / (n * hp * hp);
  }
}

// Monomial coefficients of the Lagrange basis polynomial l_j on nodes c[0..n).
void lagrange_coeffs(const double* c, int n, int j, double* coef) {
  double poly[kMaxN + 1] = {1.0};
  int deg = 0;
  double den = 1.0;
  for (int r = 0; r < n; ++r) {
    if (r == j) continue;
    double nxt[kMaxN + 1] = {0.0};
    for (int m = 0; m <= deg; ++m) {
      nxt[m + 1] += poly[m];
      nxt[m] -= c[r] * poly[m];
    }
    ++deg;
    for (int m = 0; m <= deg; ++m) poly[m] = nxt[m];
    den *= c[j] - c[r];
  }
  for (int m = 0; m < n; ++m) coef[m] = poly[m] / den;
}

double lagrange_eval(const double* c, int n, int j, double x) {
  double v = 1.0;
  for (int r = 0; r < n; ++r)
    if (r != j) v *= (x - c[r]) / (c[j] - c[r]);
  return v;
}

struct Lattice1D {
  int n;
  double c[kMaxN], w[kMaxN];
  double vinv[kMaxN][kMaxN];
};

Lattice1D make_1d(int n) {
  Lattice1D L{};
  L.n = n;
  gauss_hermite(n, L.c, L.w);
  for (int j = 0; j < n; ++j) lagrange_coeffs(L.c, n, j, L.vinv[j]);
  return L;
}

// Departure-point stencil of one node (shift s = c dt cells) with P points.
void node_stencil(double s, int P, int* off, int* ntap, double* w) {
  const double r = std::nearbyint(s);
  if (std::fabs(s - r) < 1e-12) {  // integer shift: one exact tap
    *off = -(int)r;
    *ntap = 1;
    w[0] = 1.0;
    for (int a = 1; a < kMaxP; ++a) w[a] = 0.0;
    return;
  }
  const double xd = -s;  // departure point relative to the cell
  const int o = (int)std::floor(xd - 0.5 * (P - 1) + 0.5);
  *off = o;
  *ntap = P;
  for (int a = 0; a < kMaxP; ++a) w[a] = 0.0;
  for (int a = 0; a < P; ++a) {
    double v = 1.0;
    for (int q = 0; q < P; ++q)
      if (q != a) v *= (xd - (double)(o + q)) / (double)(a - q);
    w[a] = v;
  }
}

template <class R>
void fill_lat(LatTab<R>& T, const Lattice1D& L, double dt, int P) {
  T.n = L.n;
  for (int j = 0; j < kMaxN; ++j) {
    T.off[j] = 0;
    T.ntap[j] = 1;
    T.c[j] = 0;
    T.w1[j] = 0;
    for (int a = 0; a < kMaxP; ++a) T.w[j][a] = 0;
    for (int m = 0; m < kMaxN; ++m) T.vinv[j][m] = 0;
  }
  for (int j = 0; j < L.n; ++j) {
    double w[kMaxP];
    node_stencil(L.c[j] * dt, P, &T.off[j], &T.ntap[j], w);
    T.c[j] = (R)L.c[j];
    T.w1[j] = (R)L.w[j];
    if (T.ntap[j] > 1) w[(P - 1) / 2] = 0.0;  // differential form (see LatTab)
    for (int a = 0; a < kMaxP; ++a) T.w[j][a] = (R)w[a];
    for (int m = 0; m < L.n; ++m) T.vinv[j][m] = (R)L.vinv[j][m];
  }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int elem_size(int precision) {
  return precision == SLBM_FP64 ? 8 : (precision == SLBM_FP16 || precision == SLBM_FX16 ? 2 : 4);
}

struct Layout {
  int G, pitch, rows;
  long long plane;           // elements per plane, padded
  size_t pops[2][2];         // byte offsets [buffer][lattice]
  size_t flags[2], flag_tmp, tile_mask[2], macro[4], partials, audit_out, err, bc[4][3];
  size_t lam[2];             // co-moving frame planes {u_x, u_y, T} per buffer
  size_t sched;              // two tile counters of the stream kernel's scheduler, then the
                             // post-step kernel's item counter
  size_t seed_ctr;           // FP16 rounding key counter
  size_t gh_start, gh_idx, gh_tiles;  // per-tile ghost lists (GhostTables)
  size_t post_work;          // 2 x ntiles work words (stream kernel -> post-step kernel)
  size_t post_nlist;         // 2 counters: work tiles listed in each half of post_list
  size_t post_list;          // 2 x ntiles: candidate work tiles (stream kernel -> post-step kernel)
  size_t conv_count;         // 2 counters of the co-moving conversion lists (their cell lists
                             // use the macro[2] / macro[3] staging slots, see conv_lists)
  size_t total;
};

bool config_ok(const slbm_grid* g, int lo, int hi, int order, int precision, char* err) {
  if (!g) { snprintf(err, 256, "null grid"); return false; }
  if (lo < SLBM_D2Q9 || hi > SLBM_D2Q25 || lo >= hi) {
    snprintf(err, 256, "lattice pair must satisfy D2Q9 <= lat_lo < lat_hi <= D2Q25");
    return false;
  }
  if (order < 1 || order > 5) { snprintf(err, 256, "interp_order must be in 1..5"); return false; }
  if (precision != SLBM_FP32 && precision != SLBM_FP64 && precision != SLBM_FP16 &&
      precision != SLBM_FX16) {
    snprintf(err, 256, "precision must be SLBM_FP32, SLBM_FP64, SLBM_FP16 or SLBM_FX16");
    return false;
  }
  if (g->nx < 1 || g->ny < 1 || (long long)g->nx * g->ny > (1LL << 30)) {
    snprintf(err, 256, "grid size out of range");
    return false;
  }
  return true;
}

int reach_of(const Lattice1D& L, double dt, int P) {
  int r = 0;
  for (int j = 0; j < L.n; ++j) {
    int off, nt;
    double w[kMaxP];
    node_stencil(L.c[j] * dt, P, &off, &nt, w);
    r = std::max(r, std::max(-off, off + nt - 1));
  }
  return r;
}

double pair_dt(const Lattice1D& a, const Lattice1D& b) {
  double cmax = 0.0;
  for (int j = 0; j < a.n; ++j) cmax = std::max(cmax, std::fabs(a.c[j]));
  for (int j = 0; j < b.n; ++j) cmax = std::max(cmax, std::fabs(b.c[j]));
  return 1.0 / cmax;  // CFL = 1
}

Layout make_layout(const slbm_grid* g, int lo, int hi, int order, int precision) {
  Layout Lo{};
  const Lattice1D a = make_1d(lo), b = make_1d(hi);
  const double dt = pair_dt(a, b);
  const int P = order + 1;
  Lo.G = std::max(1, std::max(reach_of(a, dt, P), reach_of(b, dt, P)));
  Lo.pitch = (int)align_up((size_t)(kOX + g->nx + Lo.G), 32);
  Lo.rows = g->ny + 2 * Lo.G;
  Lo.plane = (long long)align_up((size_t)Lo.pitch * Lo.rows, 64);
  const size_t es = elem_size(precision);
  size_t off = 0;
  const int Q[2] = {lo * lo, hi * hi};
  for (int buf = 0; buf < 2; ++buf)
    for (int k = 0; k < 2; ++k) {
      Lo.pops[buf][k] = off;
      off = align_up(off + (size_t)Q[k] * Lo.plane * es, 256);
    }
  const size_t nc = (size_t)g->nx * g->ny;
  for (int f = 0; f < 2; ++f) { Lo.flags[f] = off; off = align_up(off + nc, 256); }
  Lo.flag_tmp = off; off = align_up(off + nc, 256);
  const size_t ntiles = (size_t)((g->nx + kTX - 1) / kTX) * ((g->ny + kTY - 1) / kTY);
  for (int m = 0; m < 2; ++m) { Lo.tile_mask[m] = off; off = align_up(off + ntiles, 256); }
  for (int m = 0; m < 4; ++m) { Lo.macro[m] = off; off = align_up(off + nc * 8, 256); }
  Lo.partials = off; off = align_up(off + 4 * 1024 * 8, 256);
  Lo.audit_out = off; off = align_up(off + 4 * 8, 256);
  Lo.err = off; off = align_up(off + 16, 256);
  const size_t side = (size_t)std::max(g->nx, g->ny);
  for (int s = 0; s < 4; ++s)
    for (int q = 0; q < 3; ++q) { Lo.bc[s][q] = off; off = align_up(off + side * 8, 256); }
  for (int b = 0; b < 2; ++b) { Lo.lam[b] = off; off = align_up(off + 3 * nc * es, 256); }
  Lo.sched = off; off = align_up(off + 4 * sizeof(int), 256);
  Lo.seed_ctr = off; off = align_up(off + sizeof(uint32_t), 256);
  const size_t ring = 2 * (size_t)Lo.G * (g->nx + 2 * Lo.G) + 2 * (size_t)Lo.G * g->ny;
  Lo.gh_start = off; off = align_up(off + (ntiles + 1) * sizeof(int), 256);
  Lo.gh_idx = off; off = align_up(off + ring * sizeof(int), 256);
  Lo.gh_tiles = off; off = align_up(off + ntiles * sizeof(int), 256);
  Lo.post_work = off; off = align_up(off + 2 * ntiles * sizeof(int), 256);
  Lo.post_nlist = off; off = align_up(off + 2 * sizeof(int), 256);
  Lo.post_list = off; off = align_up(off + 2 * ntiles * sizeof(int), 256);
  Lo.conv_count = off; off = align_up(off + 2 * sizeof(int), 256);
  Lo.total = off;
  return Lo;
}

}  // namespace

void slbm::host_gauss_hermite(int n, double* c, double* w) { gauss_hermite(n, c, w); }

struct slbm_s {
  slbm_grid g;
  int nlo, nhi, P, precision;
  int frame;                     // SLBM_FRAME_*
  double tau;
  Params<float> pf;
  Params<double> pd;
  PondParams<float> qf;          // co-moving frame tables
  PondParams<double> qd;
  double pond_tol;
  int pond_maxit;
  int pond_mixed;                // both lattices present (interface conversions per step)
  // two-population co-moving model (slbm_set_twopop): C_v, tau_2 and the g
  // planes of both buffers and lattices, laid out like the f planes (owned)
  int twopop;
  double cv, tau2;
  char* gbuf;
  // batched quasi-one-dimensional rows (slbm_set_rows) and the viscosity law
  // (slbm_set_viscosity_law): device arrays row_len (ny ints), row_ends
  // (8 ny doubles), row_visc (2 ny doubles) in one owned allocation
  int rows, hs;
  double s_exp, pr;
  char* rowbuf;
  size_t rb_len, rb_ends, rb_visc;
  int pond_bx, pond_by;          // block shape of the co-moving step (slbm_tune)
  int kn_on, kn_interval;        // Knudsen refinement of batched rows (slbm_set_kn_criterion)
  double kn_thr;
  Layout lay;
  cudaStream_t st;
  char* ws;
  bool owns_ws;
  int dev;                       // CUDA device of the workspace
  int nsm;                       // its multiprocessor count
  int cur, fcur;                 // population buffer and flag buffer in use
  int mcur;                      // tile-mask buffer the next stream launch reads
  int crit;
  double thr;
  // channels (slbm_set_channels): per-column gap mask (host), and on the
  // device (owned, one allocation) the internal wall ghosts {gx, gy, sx, side},
  // their velocities, the per-column omega and the ghost index list sized for
  // the ring plus the walls
  int post_kernel;               // per-step post-step kernel: 0 by grid size, 1 warp, 2 block
                                 // (environment SLBM_POST_KERNEL = warp / block at creation)
  int nchan, nwall;
  std::vector<uint8_t> gapcol;
  char* chanbuf;
  size_t cb_wallu, cb_omega, cb_ghidx;
  // learned indicator: weights on the device (owned), evaluation interval
  void* ind_buf;
  IndicatorDev ind;
  int ind_interval;
  double ind_thr;                // logit threshold of SLBM_CRIT_MLP(_REFINE)
  int bc_kind[4];
  long long steps;
  long long sc_launches;         // stream-collide launches (scheduler counter parity)
  int gh_ntiles;                 // tiles with ghost images (GhostTables::ntiles)
  int failed;
  char err[256];
  // tracing: events bracketing the kernels of each profiled step
  int profiling;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used;
  // CUDA graphs of 2 or 16 steps, one per parity state and length (step_pair)
  struct GraphEntry {
    int key;
    cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t cap_st;           // private stream the graphs are captured on
  int graphs_off;                // a capture failed: step with direct launches
  float fx_sc[2][kMaxN * kMaxN];  // SLBM_FX16 plane scales (see include/slbm.h), by lattice

  template <class T> T* at(size_t off) { return reinterpret_cast<T*>(ws + off); }
  void* pops(int buf, int k) { return ws + lay.pops[buf][k]; }
  uint8_t* flags(int f) { return at<uint8_t>(lay.flags[f]); }
  void* lam(int buf) { return ws + lay.lam[buf]; }
  // g planes of buffer buf, lattice k (null without the two-population model)
  void* gp(int buf, int k) {
    if (!twopop) return nullptr;
    const size_t es = precision == SLBM_FP64 ? 8 : 4;
    const size_t q = (size_t)(nlo * nlo + nhi * nhi);
    return gbuf + es * (size_t)lay.plane * ((size_t)buf * q + (k ? (size_t)(nlo * nlo) : 0));
  }
  size_t ncell() const { return (size_t)g.nx * g.ny; }
};

namespace {

int fail(slbm_s* h, int code, const char* what, cudaError_t e = cudaSuccess) {
  if (e != cudaSuccess)
    snprintf(h->err, sizeof(h->err), "%s: %s", what, cudaGetErrorString(e));
  else
    snprintf(h->err, sizeof(h->err), "%s", what);
  if (code == SLBM_ECUDA) h->failed = 1;
  return code;
}

#define SLBM_CK(h, expr, what)                                \
  do {                                                        \
    cudaError_t e_ = (expr);                                  \
    if (e_ != cudaSuccess) return fail((h), SLBM_ECUDA, (what), e_); \
  } while (0)

// Makes the handle's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    else prev = -1;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

#define SLBM_GUARD(h)                                                   \
  if (!(h)) return SLBM_EINVAL;                                         \
  if ((h)->failed) return SLBM_ECUDA;                                   \
  DeviceScope slbm_device_scope_((h)->dev)

bool is_mlp(int kind) { return kind == SLBM_CRIT_MLP || kind == SLBM_CRIT_MLP_REFINE; }

// The stream kernel reads a periodic y axis's rows through their images
// (Params::wrap_y) on thin grids and with channels (whose walls cover rows
// 0 .. ny-1 only); the post-step kernel then refreshes no y ghost row.
int wraps_y(const slbm_s* h) {
  return h->frame == SLBM_FRAME_LATTICE && h->g.periodic_y &&
                 (h->g.ny < kWrapRowsMax || h->nchan > 0)
             ? 1
             : 0;
}

BcDev bc_dev(slbm_s* h) {
  BcDev b{};
  for (int s = 0; s < 4; ++s) {
    b.kind[s] = h->bc_kind[s];
    b.rho[s] = h->at<double>(h->lay.bc[s][0]);
    b.ux[s] = h->at<double>(h->lay.bc[s][1]);
    b.uy[s] = h->at<double>(h->lay.bc[s][2]);
  }
  if (h->nwall) {
    b.nwall = h->nwall;
    b.wall = reinterpret_cast<const int4*>(h->chanbuf);
    b.wall_u = reinterpret_cast<const double*>(h->chanbuf + h->cb_wallu);
  }
  return b;
}

int ntiles_of(const slbm_s* h) {
  return ((h->g.nx + kTX - 1) / kTX) * ((h->g.ny + kTY - 1) / kTY);
}

// Ghost index list: in the workspace (ring cells only), or with channels in
// the channel buffer (ring cells and internal wall ghosts).
int* ghost_idx(slbm_s* h) {
  return h->nwall ? reinterpret_cast<int*>(h->chanbuf + h->cb_ghidx) : h->at<int>(h->lay.gh_idx);
}

GhostTables ghost_tables(slbm_s* h) {
  return GhostTables{h->at<int>(h->lay.gh_start), ghost_idx(h), h->at<int>(h->lay.gh_tiles),
                     h->gh_ntiles};
}

// Per-tile ghost lists of the post-step kernel for the current boundary
// kinds: the source tile of every ring cell from the device's ghost rule,
// sorted here by tile (ring order within a tile).  Synchronous (set-up only).
int build_ghost_tables(slbm_s* h) {
  const int G = h->lay.G, nx = h->g.nx, ny = h->g.ny;
  const size_t ring = 2 * (size_t)G * (nx + 2 * G) + 2 * (size_t)G * ny + (size_t)h->nwall;
  const int nt = ntiles_of(h);
  int* d_idx = ghost_idx(h);
  SLBM_CK(h, launch_ghost_src(G, nx, ny, h->g.periodic_x ? 1 : 0, h->g.periodic_y ? 1 : 0,
                              wraps_y(h), bc_dev(h), d_idx, h->st),
          "ghost source launch");
  std::vector<int> src(ring), start(nt + 1, 0), idx, tiles;
  if (ring)
    SLBM_CK(h, cudaMemcpyAsync(src.data(), d_idx, ring * sizeof(int), cudaMemcpyDeviceToHost, h->st),
            "D2H copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  for (size_t g = 0; g < ring; ++g) {
    if (src[g] >= nt) return fail(h, SLBM_ECUDA, "ghost source outside the grid");
    if (src[g] >= 0) start[src[g] + 1]++;
  }
  for (int t = 0; t < nt; ++t) {
    if (start[t + 1]) tiles.push_back(t);
    start[t + 1] += start[t];
  }
  idx.resize(start[nt]);
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (size_t g = 0; g < ring; ++g)
    if (src[g] >= 0) idx[fill[src[g]]++] = (int)g;
  SLBM_CK(h, cudaMemcpyAsync(h->at<int>(h->lay.gh_start), start.data(), start.size() * sizeof(int),
                             cudaMemcpyHostToDevice, h->st),
          "H2D copy");
  if (!idx.empty())
    SLBM_CK(h, cudaMemcpyAsync(d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice,
                               h->st),
            "H2D copy");
  if (!tiles.empty())
    SLBM_CK(h, cudaMemcpyAsync(h->at<int>(h->lay.gh_tiles), tiles.data(),
                               tiles.size() * sizeof(int), cudaMemcpyHostToDevice, h->st),
            "H2D copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");  // the host vectors are released
  h->gh_ntiles = (int)tiles.size();
  return SLBM_OK;
}

// Storage / arithmetic types of a lattice-frame handle, as a tag.
template <class S_, class R_>
struct Ty {
  using S = S_;
  using R = R_;
};

// f(Ty<S, R>{}, params) for the handle's storage type S and arithmetic type
// R: FP64 -> (double, double), FP16 -> (half, float), FP32 -> (float, float).
template <class F>
auto with_types(slbm_s* h, F&& f) -> decltype(f(Ty<float, float>{}, h->pf)) {
  switch (h->precision) {
    case SLBM_FP64: return f(Ty<double, double>{}, h->pd);
    case SLBM_FP16: return f(Ty<__half, float>{}, h->pf);
    case SLBM_FX16: return f(Ty<fx16, float>{}, h->pf);
    default: return f(Ty<float, float>{}, h->pf);
  }
}

#define SLBM_TYPES(ty)                 \
  using S = typename decltype(ty)::S; \
  using R = typename decltype(ty)::R; \
  (void)sizeof(R)

// Full ghost fill of both buffers (setup paths).  The buffer in use gets its
// exact ghosts; the other one gets the constant DIRICHLET states the step
// never rewrites (its copies are refreshed by the post-step kernel).
cudaError_t ghosts(slbm_s* h, const uint8_t* flag) {
  for (int b = 0; b < 2; ++b) {
    const int buf = b == 0 ? h->cur ^ 1 : h->cur;
    const cudaError_t e = with_types(h, [&](auto ty, const auto& prm) {
      SLBM_TYPES(ty);
      return launch_ghosts<S, R>(prm, (S*)h->pops(buf, 0), (S*)h->pops(buf, 1), flag, bc_dev(h),
                                 h->st);
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Interface conversion of buffer `buf` plus the boundary cells' ghost images.
// Setup calls (mask_in null) also write the tile masks the next step reads.
cudaError_t convert(slbm_s* h, int buf, const uint8_t* fold, const uint8_t* fnew,
                    const uint8_t* mask_in = nullptr) {
  uint8_t* mask = h->at<uint8_t>(h->lay.tile_mask[h->mcur]);
  return with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_post<S, R>(prm, (S*)h->pops(buf, 0), (S*)h->pops(buf, 1), fold, fnew, bc_dev(h),
                             1, mask_in, mask, h->st);
  });
}

// The device error word.  A bounded wait that ran out makes the handle fail;
// the co-moving frame's reports are returned once and cleared.
int check_device_error(slbm_s* h) {
  int v = 0;
  SLBM_CK(h, cudaMemcpyAsync(&v, h->at<int>(h->lay.err), sizeof(int), cudaMemcpyDeviceToHost,
                             h->st),
          "D2H copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  if (v & kErrTimeout) {
    h->failed = 1;
    return fail(h, SLBM_ETIMEOUT, "a bounded device wait ran out");
  }
  if (v) {
    SLBM_CK(h, cudaMemsetAsync(h->at<int>(h->lay.err), 0, sizeof(int), h->st), "memset");
    SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
    if (v & kErrFrame)
      return fail(h, SLBM_ENONFINITE,
                  "co-moving frame: non-positive or non-finite frame, or a departure point "
                  "beyond the reach limit");
    return fail(h, SLBM_ENOCONV, "co-moving frame: predictor-corrector did not converge");
  }
  return SLBM_OK;
}

// Next tracing event (recorded on the handle's stream), or success when off.
cudaError_t mark(slbm_s* h) {
  if (!h->profiling) return cudaSuccess;
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    h->ev_pool.push_back(e);
  }
  return cudaEventRecord(h->ev_pool[h->ev_used++], h->st);
}


// One time step: stream-collide (old flags) -> interface conversion (new
// flags) -> ghost-ring refresh.
// Cell lists of the co-moving conversions: the macro[2] and macro[3] slots
// (nc doubles each, room for nc ints), which otherwise only stage host data
// within one call, every read of it stream-ordered before any conversion the
// call launches.
ConvLists conv_lists(slbm_s* h) {
  return ConvLists{h->at<int>(h->lay.conv_count), h->at<int>(h->lay.macro[2]),
                   h->at<int>(h->lay.macro[3])};
}

int pond_convert_band(slbm_s* h, int buf) {
  if (!h->pond_mixed) return SLBM_OK;
  const uint8_t* mask = h->at<uint8_t>(h->lay.tile_mask[0]);
  cudaError_t e =
      h->precision == SLBM_FP64
          ? launch_pond_convert<double, double>(h->qd, (double*)h->pops(buf, 0),
                                                (double*)h->pops(buf, 1), (double*)h->gp(buf, 0),
                                                (double*)h->gp(buf, 1),
                                                (const double*)h->lam(buf), h->flags(h->fcur),
                                                mask, nullptr, 0, conv_lists(h), h->st)
          : launch_pond_convert<float, float>(h->qf, (float*)h->pops(buf, 0),
                                              (float*)h->pops(buf, 1), (float*)h->gp(buf, 0),
                                              (float*)h->gp(buf, 1), (const float*)h->lam(buf),
                                              h->flags(h->fcur), mask, nullptr, 0, conv_lists(h), h->st);
  SLBM_CK(h, e, "co-moving conversion launch");
  return SLBM_OK;
}

// One co-moving-frame step: predictor-corrector stream-collide, then the
// interface conversions of the new state when both lattices are in use.
// Batched rows with both lattices step in one launch per lattice (each row's
// high-order cells are one run, so warps are whole in either launch); 2-D
// grids keep one launch (scattered high-order regions leave the lattice
// launches' warps partly idle: the 1024 x 512 disc field took 2.93 ms split
// against 1.69 ms).
cudaError_t pond_launch(slbm_s* h, int b, int nb) {
  int* err = h->at<int>(h->lay.err);
  const int split = h->pond_mixed && h->rows ? 1 : 0;
  cudaError_t e;
  if (h->precision == SLBM_FP64)
    e = launch_pond_step<double, double>(
        h->qd, (const double*)h->pops(b, 0), (const double*)h->pops(b, 1),
        (const double*)h->gp(b, 0), (const double*)h->gp(b, 1), (const double*)h->lam(b),
        (double*)h->pops(nb, 0), (double*)h->pops(nb, 1), (double*)h->gp(nb, 0),
        (double*)h->gp(nb, 1), (double*)h->lam(nb), h->flags(h->fcur), err, split,
        h->st);
  else
    e = launch_pond_step<float, float>(
        h->qf, (const float*)h->pops(b, 0), (const float*)h->pops(b, 1),
        (const float*)h->gp(b, 0), (const float*)h->gp(b, 1), (const float*)h->lam(b),
        (float*)h->pops(nb, 0), (float*)h->pops(nb, 1), (float*)h->gp(nb, 0),
        (float*)h->gp(nb, 1), (float*)h->lam(nb), h->flags(h->fcur), err, split,
        h->st);
  return e;
}

int pond_step_once(slbm_s* h) {
  const int b = h->cur, nb = b ^ 1;
  SLBM_CK(h, mark(h), "trace event");
  SLBM_CK(h, pond_launch(h, b, nb), "co-moving step launch");
  SLBM_CK(h, mark(h), "trace event");
  if (int rc = pond_convert_band(h, nb)) return rc;
  SLBM_CK(h, mark(h), "trace event");
  h->cur = nb;
  h->steps++;
  return SLBM_OK;
}

int step_once(slbm_s* h) {
  if (h->frame != SLBM_FRAME_LATTICE) return pond_step_once(h);
  const int b = h->cur, nb = b ^ 1;
  uint8_t* fold = h->flags(h->fcur);
  uint8_t* fnew = h->crit == SLBM_CRIT_MACH ? h->flags(h->fcur ^ 1) : fold;
  cudaError_t e;
  SLBM_CK(h, mark(h), "trace event");
  const uint8_t* mask = h->at<uint8_t>(h->lay.tile_mask[h->mcur]);
  uint8_t* mask_next = h->at<uint8_t>(h->lay.tile_mask[h->mcur ^ 1]);
  h->pf.sched_parity = h->pd.sched_parity = (int)(h->sc_launches & 1);
  h->sc_launches++;
  e = with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_stream_collide<S, R>(prm, h->P, (const S*)h->pops(b, 0),
                                       (const S*)h->pops(b, 1), (S*)h->pops(nb, 0),
                                       (S*)h->pops(nb, 1), fold, fnew, mask, mask_next, h->st);
  });
  SLBM_CK(h, e, "stream_collide launch");
  SLBM_CK(h, mark(h), "trace event");
  const int half = h->pf.sched_parity;
  const size_t nt = (size_t)ntiles_of(h);
  const int* work = h->at<int>(h->lay.post_work) + half * nt;
  const int* list = h->at<int>(h->lay.post_list) + half * nt;
  const int* nlist = h->at<int>(h->lay.post_nlist) + half;
  e = with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_post_step<S, R>(prm, (S*)h->pops(nb, 0), (S*)h->pops(nb, 1), fold, fnew,
                                  bc_dev(h), work, list, nlist, ghost_tables(h), h->st);
  });
  SLBM_CK(h, e, "post-step launch");
  SLBM_CK(h, mark(h), "trace event");
  h->cur = nb;
  h->mcur ^= 1;
  if (h->crit == SLBM_CRIT_MACH) h->fcur ^= 1;
  h->steps++;
  return SLBM_OK;
}

constexpr int kGraphPairs = 8;  // pairs of steps in a long graph

// Knudsen criterion on the current buffer: new flags into the temporary
// plane, the refined cells' other lattice from their current one (their new
// native vector), masks of the new flags (with the tiles whose cells changed
// lattice), then the band conversion (full_band: every cell that reads the
// other lattice; else only those in the 3 x 3 tile neighbourhood of a changed
// cell, the others having been converted after the step, from the same
// native vectors) and the new flags.
int apply_kn(slbm_s* h, bool full_band) {
  uint8_t* tmp = h->at<uint8_t>(h->lay.flag_tmp);
  uint8_t* mask = h->at<uint8_t>(h->lay.tile_mask[0]);
  uint8_t* fl = h->flags(h->fcur);
  const int c = h->cur, near = full_band ? 0 : 1;
  cudaError_t e;
  if (h->precision == SLBM_FP64) {
    double *f0 = (double*)h->pops(c, 0), *f1 = (double*)h->pops(c, 1);
    double *e0 = (double*)h->gp(c, 0), *e1 = (double*)h->gp(c, 1);
    const double* lam = (const double*)h->lam(c);
    e = launch_pond_kn<double, double>(h->qd, f0, f1, e0, e1, lam, fl, h->kn_thr, tmp, h->st);
    SLBM_CK(h, e, "Knudsen criterion launch");
    e = launch_pond_convert<double, double>(h->qd, f0, f1, e0, e1, lam, fl, nullptr, tmp, 0,
                                            conv_lists(h), h->st);
    SLBM_CK(h, e, "co-moving conversion launch");
    SLBM_CK(h, launch_pond_masks(h->g.nx, h->g.ny, tmp, fl, mask, h->st), "mask launch");
    e = launch_pond_convert<double, double>(h->qd, f0, f1, e0, e1, lam, tmp, mask, nullptr, near,
                                            conv_lists(h), h->st);
  } else {
    float *f0 = (float*)h->pops(c, 0), *f1 = (float*)h->pops(c, 1);
    float *e0 = (float*)h->gp(c, 0), *e1 = (float*)h->gp(c, 1);
    const float* lam = (const float*)h->lam(c);
    e = launch_pond_kn<float, float>(h->qf, f0, f1, e0, e1, lam, fl, h->kn_thr, tmp, h->st);
    SLBM_CK(h, e, "Knudsen criterion launch");
    e = launch_pond_convert<float, float>(h->qf, f0, f1, e0, e1, lam, fl, nullptr, tmp, 0,
                                          conv_lists(h), h->st);
    SLBM_CK(h, e, "co-moving conversion launch");
    SLBM_CK(h, launch_pond_masks(h->g.nx, h->g.ny, tmp, fl, mask, h->st), "mask launch");
    e = launch_pond_convert<float, float>(h->qf, f0, f1, e0, e1, lam, tmp, mask, nullptr, near,
                                          conv_lists(h), h->st);
  }
  SLBM_CK(h, e, "co-moving conversion launch");
  SLBM_CK(h, cudaMemcpyAsync(fl, tmp, h->ncell(), cudaMemcpyDeviceToDevice, h->st), "flag copy");
  return SLBM_OK;
}

// The Knudsen criterion after every step (interval 1) is part of the step:
// direct steps apply it after each step_once, and graph replays record it.
bool kn_every_step(const slbm_s* h) { return h->kn_on && h->kn_interval == 1; }

// m pairs of steps as one CUDA graph launch: the kernel launches of 2 m
// step_once calls, captured once per parity state (buffer, flag and mask
// halves, scheduler counter and work-list halves) and length on a private
// stream and replayed on the handle's stream.  (Co-moving steps alternate the
// buffer only.)  After two steps every parity is back where it was, so the
// replay only advances the counters.  Longer graphs cut the host's launches
// for small grids, where one step takes a few microseconds.  With the
// Knudsen criterion every step, each recorded step is followed by the
// criterion's launches.  Returns 1 (and stops trying) if the capture is
// refused, so the caller steps directly.
int step_pair(slbm_s* h, int m) {
  const int key =
      h->cur | h->mcur << 1 | h->fcur << 2 | (int)(h->sc_launches & 1) << 3 | m << 4;
  cudaGraphExec_t exec = nullptr;
  for (const auto& e : h->graphs)
    if (e.key == key) exec = e.exec;
  if (!exec) {
    if (!h->cap_st && cudaStreamCreateWithFlags(&h->cap_st, cudaStreamNonBlocking) != cudaSuccess) {
      h->cap_st = nullptr;
      h->graphs_off = 1;
      return 1;
    }
    // the host state the recorded steps advance
    const int cur = h->cur, mcur = h->mcur, fcur = h->fcur;
    const long long steps = h->steps, scl = h->sc_launches;
    cudaStream_t st = h->st;
    h->st = h->cap_st;
    cudaGraph_t g = nullptr;
    int rc = SLBM_OK;
    cudaError_t e = cudaStreamBeginCapture(h->cap_st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      for (int i = 0; i < 2 * m && rc == SLBM_OK; ++i) {
        rc = step_once(h);
        if (rc == SLBM_OK && kn_every_step(h)) rc = apply_kn(h, false);
      }
      e = cudaStreamEndCapture(h->cap_st, &g);
    }
    h->st = st;
    h->cur = cur;
    h->mcur = mcur;
    h->fcur = fcur;
    h->steps = steps;
    h->sc_launches = scl;
    if (e == cudaSuccess && rc == SLBM_OK && g) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || rc != SLBM_OK || !exec) {
      // nothing recorded has run: clear the refusal and step directly
      cudaGetLastError();
      h->failed = 0;
      h->err[0] = 0;
      h->graphs_off = 1;
      return 1;
    }
    h->graphs.push_back({key, exec});
  }
  SLBM_CK(h, cudaGraphLaunch(exec, h->st), "graph launch");
  h->steps += 2 * m;
  if (h->frame == SLBM_FRAME_LATTICE) h->sc_launches += 2 * m;
  return SLBM_OK;
}

template <class R>
void fill_params(Params<R>& p, const slbm_s* h, const Lattice1D& a, const Lattice1D& b, double dt) {
  std::memset(&p, 0, sizeof(p));
  p.nx = h->g.nx;
  p.ny = h->g.ny;
  p.G = h->lay.G;
  p.pitch = h->lay.pitch;
  p.rows = h->lay.rows;
  p.plane = h->lay.plane;
  p.periodic_x = h->g.periodic_x ? 1 : 0;
  p.periodic_y = h->g.periodic_y ? 1 : 0;
  p.wrap_y = wraps_y(h);
  p.post_warp = h->post_kernel == 1 || (h->post_kernel == 0 && ntiles_of(h) >= kPostWarpTiles);
  p.crit = h->crit;
  p.thr = (R)h->thr;
  p.omega = (R)(1.0 / h->tau);
  p.band = h->lay.G;
  p.nsm = h->nsm;
  p.sched = reinterpret_cast<int*>(h->ws + h->lay.sched);
  p.seed_ctr = reinterpret_cast<uint32_t*>(h->ws + h->lay.seed_ctr);
  p.work = reinterpret_cast<int*>(h->ws + h->lay.post_work);
  p.wlist = reinterpret_cast<int*>(h->ws + h->lay.post_list);
  p.wcount = reinterpret_cast<int*>(h->ws + h->lay.post_nlist);
  p.cv = h->twopop ? h->cv : 1.0;
  // per-column omega of channels, in the arithmetic type of the handle's kernels
  p.omega_x = (h->nchan && sizeof(R) == (h->precision == SLBM_FP64 ? 8u : 4u))
                  ? reinterpret_cast<const R*>(h->chanbuf + h->cb_omega)
                  : nullptr;
  fill_lat(p.lat[0], a, dt, h->P);
  fill_lat(p.lat[1], b, dt, h->P);
  // fixed-point plane scales (1 for the other storage types, unused there)
  for (int k = 0; k < 2; ++k)
    for (int i = 0; i < kMaxN * kMaxN; ++i) {
      const double sc = h->precision == SLBM_FX16 ? (double)h->fx_sc[k][i] : 1.0;
      p.lat[k].sc[i] = (R)sc;
      p.lat[k].isc[i] = (R)(1.0 / sc);
    }
  ConvTab<R>& t = p.conv;
  for (int j = 0; j < kMaxN; ++j)
    for (int m = 0; m < kMaxN; ++m) {
      t.lift[j][m] = R(0);
      t.proj[j][m] = R(0);
    }
  // L[a][j] = sum_{m < nq} VQ^-1[a][m] c_q[j]^m
  for (int aa = 0; aa < b.n; ++aa)
    for (int j = 0; j < a.n; ++j) {
      double s = 0.0, pw = 1.0;
      for (int m = 0; m < a.n; ++m) {
        s += b.vinv[aa][m] * pw;
        pw *= a.c[j];
      }
      t.lift[aa][j] = (R)s;
    }
  // P[j][a] = l^q_j(c^Q_a)
  for (int j = 0; j < a.n; ++j)
    for (int aa = 0; aa < b.n; ++aa) t.proj[j][aa] = (R)lagrange_eval(a.c, a.n, j, b.c[aa]);
}

template <class R>
void fill_pond(PondParams<R>& q, const slbm_s* h, const Params<R>& p, const Lattice1D& a,
               const Lattice1D& b, double dt) {
  std::memset(&q, 0, sizeof(q));
  q.nx = h->g.nx;
  q.ny = h->g.ny;
  q.G = h->lay.G;
  q.pitch = h->lay.pitch;
  q.plane = h->lay.plane;
  q.nc = (long long)h->g.nx * h->g.ny;
  q.omega = (R)(1.0 / h->tau);
  q.dt = (R)dt;
  q.tol = (R)h->pond_tol;
  q.maxit = h->pond_maxit;
  q.thermal = h->frame == SLBM_FRAME_POND ? 1 : 0;
  q.twopop = h->twopop;
  q.cv = (R)(h->twopop ? h->cv : 1.0);
  q.cvm1 = (R)(h->twopop ? h->cv - 1.0 : 0.0);
  q.omega2 = (R)(h->twopop ? 1.0 / h->tau2 : 1.0 / h->tau);
  q.rows = h->rows;
  q.row_len = h->rowbuf ? reinterpret_cast<const int*>(h->rowbuf + h->rb_len) : nullptr;
  q.row_ends = h->rowbuf ? reinterpret_cast<const double*>(h->rowbuf + h->rb_ends) : nullptr;
  q.hs = h->hs;
  q.row_visc = h->rowbuf ? reinterpret_cast<const double*>(h->rowbuf + h->rb_visc) : nullptr;
  q.s_exp = (R)h->s_exp;
  q.inv_pr = (R)(h->hs ? 1.0 / h->pr : 1.0);
  q.bx = h->pond_bx;
  q.by = h->pond_by;
  q.P = h->P;
  q.nsm = h->nsm;
  q.reach = (R)kPondReach;
  for (int k = 0; k < 2; ++k) {
    const Lattice1D& L = k ? b : a;
    PondLat<R>& T = q.lat[k];
    T.n = L.n;
    for (int j = 0; j < L.n; ++j) {
      T.c[j] = (R)L.c[j];
      T.w[j] = (R)L.w[j];
      for (int m = 0; m < L.n; ++m) {
        T.inv[j][m] = m == j ? R(0) : (R)(1.0 / (L.c[j] - L.c[m]));
        T.vinv[j][m] = (R)L.vinv[j][m];
      }
    }
  }
  for (int j = 0; j < kMaxN; ++j)
    for (int m = 0; m < kMaxN; ++m) q.proj[j][m] = p.conv.proj[j][m];
}

// Captured graphs hold kernel arguments by value: drop them whenever the
// parameters or the boundary description change.
void drop_graphs(slbm_s* h) {
  for (auto& e : h->graphs) cudaGraphExecDestroy(e.exec);
  h->graphs.clear();
}

void refresh_params(slbm_s* h) {
  drop_graphs(h);
  const Lattice1D a = make_1d(h->nlo), b = make_1d(h->nhi);
  const double dt = pair_dt(a, b);
  fill_params(h->pf, h, a, b, dt);
  fill_params(h->pd, h, a, b, dt);
  fill_pond(h->qf, h, h->pf, a, b, dt);
  fill_pond(h->qd, h, h->pd, a, b, dt);
}

// Frame planes of the current buffer, or null in the lattice frame.
const void* frame_planes(slbm_s* h) {
  return h->frame != SLBM_FRAME_LATTICE ? h->lam(h->cur) : nullptr;
}

int upload(slbm_s* h, void* dst, const void* src, size_t bytes) {
  SLBM_CK(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->st), "H2D copy");
  return SLBM_OK;
}

template <class S, class R>
int pack_all(slbm_s* h, const Params<R>& prm, int k, double* host, int unpack,
             const double* in_host) {
  const int n = k ? h->nhi : h->nlo, Q = n * n;
  const size_t nc = h->ncell();
  // the four nc-double macro slots stage up to four planes at a time
  for (int i0 = 0; i0 < Q; i0 += 4) {
    const int cnt = std::min(4, Q - i0);
    if (unpack) {
      // macro[0..3] are contiguous nc-double slots; stage cnt planes there
      for (int q = 0; q < cnt; ++q) {
        const int rc = upload(h, h->at<double>(h->lay.macro[q]), in_host + (size_t)(i0 + q) * nc,
                              nc * 8);
        if (rc) return rc;
      }
      for (int q = 0; q < cnt; ++q)
        SLBM_CK(h, (launch_pack<S, R>(prm, k, i0 + q, 1, nullptr, nullptr, 1,
                                      (S*)h->pops(h->cur, k), h->at<double>(h->lay.macro[q]),
                                      h->st)),
                "unpack launch");
    } else {
      for (int q = 0; q < cnt; ++q) {
        SLBM_CK(h, (launch_pack<S, R>(prm, k, i0 + q, 1, (const S*)h->pops(h->cur, k),
                                      h->at<double>(h->lay.macro[q]), 0, nullptr, nullptr, h->st)),
                "pack launch");
        SLBM_CK(h, cudaMemcpyAsync(host + (size_t)(i0 + q) * nc, h->at<double>(h->lay.macro[q]),
                                   nc * 8, cudaMemcpyDeviceToHost, h->st),
                "D2H copy");
      }
    }
    SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  }
  return SLBM_OK;
}

int pack_any(slbm_s* h, int k, double* host, int unpack, const double* in) {
  return with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return pack_all<S, R>(h, prm, k, host, unpack, in);
  });
}

// SLBM_FX16 plane scales from the equilibria staged in macro[0..2] (rho,
// u_x, u_y): per plane of each lattice the range A_i = max(2 max|s_i|, W_i / 4)
// and sc_i = A_i / 32767^2 (the companded integers reach +-32767 at +-A_i).
// Synchronous.
int set_fx_scales(slbm_s* h) {
  constexpr int Q = kMaxN * kMaxN;
  unsigned* d = h->at<unsigned>(h->lay.partials);  // scratch: 2 Q words
  SLBM_CK(h, cudaMemsetAsync(d, 0, 2 * Q * sizeof(unsigned), h->st), "memset");
  SLBM_CK(h, launch_fx_range(h->pf, h->at<double>(h->lay.macro[0]), h->at<double>(h->lay.macro[1]),
                             h->at<double>(h->lay.macro[2]), d, h->st),
          "fixed-point range launch");
  unsigned bits[2 * Q];
  SLBM_CK(h, cudaMemcpyAsync(bits, d, sizeof(bits), cudaMemcpyDeviceToHost, h->st), "D2H copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  const Lattice1D L[2] = {make_1d(h->nlo), make_1d(h->nhi)};
  for (int k = 0; k < 2; ++k)
    for (int i = 0; i < L[k].n * L[k].n; ++i) {
      float m;
      std::memcpy(&m, &bits[k * Q + i], sizeof(m));
      const double W = L[k].w[i % L[k].n] * L[k].w[i / L[k].n];
      h->fx_sc[k][i] = (float)(std::max(2.0 * (double)m, 0.25 * W) / (32767.0 * 32767.0));
    }
  refresh_params(h);
  return SLBM_OK;
}

int init_eq_dev(slbm_s* h, bool with_T = false) {
  cudaError_t e;
  double* r = h->at<double>(h->lay.macro[0]);
  double* u = h->at<double>(h->lay.macro[1]);
  double* v = h->at<double>(h->lay.macro[2]);
  if (h->frame != SLBM_FRAME_LATTICE) {
    const double* T = with_T ? h->at<double>(h->lay.macro[3]) : nullptr;
    e = h->precision == SLBM_FP64
            ? launch_pond_init<double, double>(h->qd, (double*)h->pops(h->cur, 0),
                                               (double*)h->pops(h->cur, 1),
                                               (double*)h->gp(h->cur, 0), (double*)h->gp(h->cur, 1),
                                               (double*)h->lam(h->cur), r, u, v, T, h->st)
            : launch_pond_init<float, float>(h->qf, (float*)h->pops(h->cur, 0),
                                             (float*)h->pops(h->cur, 1), (float*)h->gp(h->cur, 0),
                                             (float*)h->gp(h->cur, 1), (float*)h->lam(h->cur),
                                             r, u, v, T, h->st);
    SLBM_CK(h, e, "init launch");
    return SLBM_OK;
  }
  e = with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_init_eq<S, R>(prm, (S*)h->pops(h->cur, 0), (S*)h->pops(h->cur, 1), r, u, v,
                                h->st);
  });
  SLBM_CK(h, e, "init launch");
  SLBM_CK(h, convert(h, h->cur, h->flags(h->fcur), h->flags(h->fcur)), "post-step launch");
  SLBM_CK(h, ghosts(h, h->flags(h->fcur)), "ghost launch");
  return SLBM_OK;
}

// Every argument check of slbm_create / slbm_create_in, before any CUDA call.
bool create_args_ok(const slbm_grid* g, int lat_lo, int lat_hi, double tau, int interp_order,
                    int frame, int precision) {
  if (!config_ok(g, lat_lo, lat_hi, interp_order, precision, g_create_err)) return false;
  if (!(tau > 0.5) || !std::isfinite(tau)) {
    snprintf(g_create_err, sizeof(g_create_err), "tau must be a finite value > 1/2");
    return false;
  }
  if (frame != SLBM_FRAME_LATTICE && frame != SLBM_FRAME_POND &&
      frame != SLBM_FRAME_POND_ISOTHERMAL) {
    snprintf(g_create_err, sizeof(g_create_err), "unknown frame");
    return false;
  }
  if (frame != SLBM_FRAME_LATTICE && (precision == SLBM_FP16 || precision == SLBM_FX16)) {
    snprintf(g_create_err, sizeof(g_create_err), "the co-moving frame runs in FP32 or FP64");
    return false;
  }
  if (frame != SLBM_FRAME_LATTICE && !(g->periodic_x && g->periodic_y)) {
    snprintf(g_create_err, sizeof(g_create_err), "the co-moving frame needs a periodic grid");
    return false;
  }
  const Layout lay = make_layout(g, lat_lo, lat_hi, interp_order, precision);
  {  // the kernels take the single-tap pattern and the halo as compile-time facts
    const Lattice1D a = make_1d(lat_lo), b = make_1d(lat_hi);
    const double dt = pair_dt(a, b);
    const int P = interp_order + 1;
    bool ok = lay.G == stage_halo(P);
    for (int k = 0; k < 2 && ok; ++k) {
      const Lattice1D& L = k ? b : a;
      for (int j = 0; j < L.n; ++j) {
        int off, nt;
        double w[kMaxP];
        node_stencil(L.c[j] * dt, P, &off, &nt, w);
        const bool snap = node_snapped(L.n, k == 1, j);
        if ((nt == 1) != snap || (snap && off != snapped_offset(L.n, j))) ok = false;
      }
    }
    if (!ok) {
      snprintf(g_create_err, sizeof(g_create_err), "unsupported stencil pattern for this pair");
      return false;
    }
  }
  // in the lattice frame a periodic side's ghost images wrap once (n >= G);
  // a bounded side, and every side of a co-moving grid, needs 2 G + 1
  const bool lat = frame == SLBM_FRAME_LATTICE;
  if (g->nx < (lat && g->periodic_x ? lay.G : 2 * lay.G + 1) ||
      g->ny < (lat && g->periodic_y ? lay.G : 2 * lay.G + 1)) {
    snprintf(g_create_err, sizeof(g_create_err),
             "grid must be at least %d cells per side (%d along a periodic lattice-frame side)",
             2 * lay.G + 1, lay.G);
    return false;
  }
  // lattice frame: interface work is found per 32 x 8 tile from the tiles next
  // to it, so across a periodic side the last (partial) tile must span the
  // stencil reach
  if (frame == SLBM_FRAME_LATTICE &&
      ((g->periodic_x && g->nx % kTX != 0 && g->nx % kTX < lay.G) ||
       (g->periodic_y && g->ny % kTY != 0 && g->ny % kTY < lay.G))) {
    snprintf(g_create_err, sizeof(g_create_err),
             "periodic grid: nx %% %d and ny %% %d must be 0 or at least %d", kTX, kTY, lay.G);
    return false;
  }
  return true;
}

// Evaluate the learned indicator on the current state (features + MLP);
// features / logits / flags to the given device buffers (any may be null).
int run_indicator(slbm_s* h, float* feat, float* logit, uint8_t* flags_out) {
  cudaError_t e = with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_indicator<S, R>(prm, (const S*)h->pops(h->cur, 0), (const S*)h->pops(h->cur, 1),
                                  h->flags(h->fcur), h->ind, (float)h->ind_thr, feat, logit,
                                  flags_out, h->st);
  });
  SLBM_CK(h, e, "indicator launch");
  return SLBM_OK;
}

// New flags from the learned indicator into the second flag plane (unused
// while the plain criterion is off), then the post-step machinery of a
// stream step: tile masks, work words and the work list from the old and new
// flags, and the post-step kernel converts the flipped and band cells of the
// current buffer and refreshes its ghost ring.  The half of the work words and
// list used is the one the next stream launch clears (its words per tile, its
// counter at launch).
int apply_indicator(slbm_s* h) {
  uint8_t* fold = h->flags(h->fcur);
  uint8_t* fnew = h->flags(h->fcur ^ 1);
  if (h->crit == SLBM_CRIT_MLP_REFINE) {
    // the indicator's decisions, widened by the refinement buffer (the cells
    // a disturbance reaches before the next evaluation: one per step at
    // CFL = 1), OR-ed with the current flags
    uint8_t* tmp = h->at<uint8_t>(h->lay.flag_tmp);
    const int r = h->ind_interval;
    if (int rc = run_indicator(h, nullptr, nullptr, fnew)) return rc;
    SLBM_CK(h, launch_dilate(fnew, nullptr, tmp, h->g.nx, h->g.ny, h->g.periodic_x ? 1 : 0, r, 0,
                             h->st),
            "refinement buffer launch");
    SLBM_CK(h, launch_dilate(tmp, fold, fnew, h->g.nx, h->g.ny, h->g.periodic_y ? 1 : 0, r, 1,
                             h->st),
            "refinement buffer launch");
  } else if (int rc = run_indicator(h, nullptr, nullptr, fnew)) {
    return rc;
  }
  const size_t nt = (size_t)ntiles_of(h);
  const int half = (int)((h->sc_launches & 1) ^ 1);
  int* work = h->at<int>(h->lay.post_work);
  int* list = h->at<int>(h->lay.post_list);
  int* nlist = h->at<int>(h->lay.post_nlist);
  SLBM_CK(h, cudaMemsetAsync(work + half * nt, 0, nt * sizeof(int), h->st), "work clear");
  SLBM_CK(h, cudaMemsetAsync(nlist + half, 0, sizeof(int), h->st), "work list clear");
  SLBM_CK(h, launch_tile_work(h->g.nx, h->g.ny, h->g.periodic_x ? 1 : 0, h->g.periodic_y ? 1 : 0,
                              fold, fnew, h->at<uint8_t>(h->lay.tile_mask[h->mcur]), work, list,
                              nlist, half, h->st),
          "tile work launch");
  // the post-step kernel's item counter (zeroed by every stream launch; none
  // ran since the last post-step launch)
  SLBM_CK(h, cudaMemsetAsync(h->at<int>(h->lay.sched) + 2, 0, sizeof(int), h->st),
          "item counter clear");
  cudaError_t e = with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_post_step<S, R>(prm, (S*)h->pops(h->cur, 0), (S*)h->pops(h->cur, 1), fold, fnew,
                                  bc_dev(h), work + half * nt, list + half * nt, nlist + half,
                                  ghost_tables(h), h->st);
  });
  SLBM_CK(h, e, "post-step launch");
  h->fcur ^= 1;
  return SLBM_OK;
}

}  // namespace

extern "C" {

int slbm_workspace_bytes(const slbm_grid* g, int lat_lo, int lat_hi, int interp_order,
                         int precision, size_t* bytes) {
  char err[256];
  if (!bytes || !config_ok(g, lat_lo, lat_hi, interp_order, precision, err)) return SLBM_EINVAL;
  *bytes = make_layout(g, lat_lo, lat_hi, interp_order, precision).total;
  return SLBM_OK;
}

int slbm_create_in(const slbm_grid* g, int lat_lo, int lat_hi, double tau, int interp_order,
                   int frame, int precision, void* cuda_stream, void* workspace,
                   size_t workspace_bytes, slbm_t* out) {
  if (!out) return SLBM_EINVAL;
  *out = nullptr;
  if (!create_args_ok(g, lat_lo, lat_hi, tau, interp_order, frame, precision))
    return SLBM_EINVAL;
  const Layout lay = make_layout(g, lat_lo, lat_hi, interp_order, precision);
  if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < lay.total) {
    snprintf(g_create_err, sizeof(g_create_err),
             "workspace must be 256-byte aligned and hold %zu bytes", lay.total);
    return SLBM_ENOMEM;
  }
  // the handle lives on the device that holds its workspace
  cudaPointerAttributes attr{};
  cudaError_t e = cudaPointerGetAttributes(&attr, workspace);
  if (e != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
    snprintf(g_create_err, sizeof(g_create_err), "workspace is not device memory: %s",
             cudaGetErrorString(e));
    cudaGetLastError();
    return SLBM_EINVAL;
  }
  slbm_s* h = new (std::nothrow) slbm_s();
  if (!h) return SLBM_ENOMEM;
  h->dev = attr.device;
  h->nsm = 1;
  cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev);
  h->g = *g;
  {  // the per-step post-step kernel, by grid size unless the environment says
    const char* pk = std::getenv("SLBM_POST_KERNEL");
    h->post_kernel = pk && !std::strcmp(pk, "warp") ? 1 : (pk && !std::strcmp(pk, "block") ? 2 : 0);
  }
  h->nlo = lat_lo;
  h->nhi = lat_hi;
  h->P = interp_order + 1;
  h->precision = precision;
  h->frame = frame;
  h->pond_tol = precision == SLBM_FP64 ? 1e-12 : 2e-6;
  h->pond_maxit = 20;
  h->tau = tau;
  h->lay = lay;
  h->st = (cudaStream_t)cuda_stream;
  h->ws = (char*)workspace;
  h->owns_ws = false;
  h->thr = 0.3;
  h->ind_interval = 1;
  h->ind_thr = 0.0;
  for (int s = 0; s < 4; ++s) h->bc_kind[s] = SLBM_BC_OUTFLOW;
  {  // fixed-point scales before the first slbm_init_equilibrium: range +-W_i / 4
    const Lattice1D L[2] = {make_1d(lat_lo), make_1d(lat_hi)};
    for (int k = 0; k < 2; ++k)
      for (int i = 0; i < kMaxN * kMaxN; ++i)
        h->fx_sc[k][i] = i < L[k].n * L[k].n
                             ? (float)(0.25 * L[k].w[i % L[k].n] * L[k].w[i / L[k].n] /
                                       (32767.0 * 32767.0))
                             : 1.0f;
  }
  refresh_params(h);
  // zero everything (finite stale values), flags 0, then rest state rho = 1, u = 0
  if (cudaMemsetAsync(h->ws, 0, lay.total, h->st) != cudaSuccess) {
    snprintf(g_create_err, sizeof(g_create_err), "workspace clear failed");
    delete h;
    return SLBM_ECUDA;
  }
  std::vector<double> one(h->ncell(), 1.0), zero(h->ncell(), 0.0);
  int rc = slbm_init_equilibrium(h, one.data(), zero.data(), zero.data(), nullptr);
  if (rc == SLBM_OK) rc = build_ghost_tables(h);
  if (rc == SLBM_OK) rc = slbm_sync(h);
  if (rc != SLBM_OK) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
    delete h;
    return rc;
  }
  *out = h;
  return SLBM_OK;
}

int slbm_create(const slbm_grid* g, int lat_lo, int lat_hi, double tau, int interp_order,
                int frame, int precision, void* cuda_stream, slbm_t* out) {
  if (!out) return SLBM_EINVAL;
  *out = nullptr;
  size_t bytes = 0;
  if (!create_args_ok(g, lat_lo, lat_hi, tau, interp_order, frame, precision))
    return SLBM_EINVAL;
  bytes = make_layout(g, lat_lo, lat_hi, interp_order, precision).total;
  void* ws = nullptr;
  cudaError_t e = cudaMalloc(&ws, bytes);
  if (e != cudaSuccess) {
    snprintf(g_create_err, sizeof(g_create_err), "cudaMalloc(%zu): %s", bytes,
             cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SLBM_ENOMEM : SLBM_ECUDA;
  }
  int rc = slbm_create_in(g, lat_lo, lat_hi, tau, interp_order, frame, precision, cuda_stream, ws,
                          bytes, out);
  if (rc != SLBM_OK) {
    cudaFree(ws);
    return rc;
  }
  (*out)->owns_ws = true;
  return SLBM_OK;
}

int slbm_destroy(slbm_t h) {
  if (!h) return SLBM_EINVAL;
  int rc = SLBM_OK;
  if (cudaStreamSynchronize(h->st) != cudaSuccess) rc = SLBM_ECUDA;
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  drop_graphs(h);
  if (h->cap_st) cudaStreamDestroy(h->cap_st);
  if (h->ind_buf) cudaFree(h->ind_buf);
  if (h->gbuf) cudaFree(h->gbuf);
  if (h->rowbuf) cudaFree(h->rowbuf);
  if (h->chanbuf) cudaFree(h->chanbuf);
  if (h->owns_ws && cudaFree(h->ws) != cudaSuccess) rc = SLBM_ECUDA;
  delete h;
  return rc;
}

int slbm_get_info(slbm_t h, slbm_info_t* info) {
  if (!h || !info) return SLBM_EINVAL;
  const Lattice1D a = make_1d(h->nlo), b = make_1d(h->nhi);
  info->dt = pair_dt(a, b);
  info->omega = 1.0 / h->tau;
  info->q_lo = h->nlo * h->nlo;
  info->q_hi = h->nhi * h->nhi;
  info->halo = h->lay.G;
  info->pitch = h->lay.pitch;
  info->rows = h->lay.rows;
  info->precision = h->precision;
  // lattice frame: stream-collide and post-step; co-moving: the step (one
  // launch per lattice on batched rows using both) and, with both lattices,
  // the conversion's screening and list launches
  info->kernels_per_step =
      h->frame == SLBM_FRAME_LATTICE ? 2 : (h->pond_mixed ? (h->rows ? 4 : 3) : 1);
  info->workspace_bytes = h->lay.total;
  info->steps = h->steps;
  return SLBM_OK;
}

int slbm_init_equilibrium(slbm_t h, const double* rho, const double* ux, const double* uy,
                          const double* T) {
  SLBM_GUARD(h);
  if (!rho || !ux || !uy) return fail(h, SLBM_EINVAL, "rho, ux, uy are required");
  if (T && h->frame != SLBM_FRAME_POND)
    return fail(h, SLBM_EINVAL, "only the thermal co-moving model takes T; pass NULL");
  const size_t b = h->ncell() * 8;
  int rc;
  if (T)
    for (size_t c = 0; c < h->ncell(); ++c)
      if (!(T[c] > 0.0) || !std::isfinite(T[c])) return fail(h, SLBM_EINVAL, "T must be > 0");
  if ((rc = upload(h, h->at<double>(h->lay.macro[0]), rho, b))) return rc;
  if ((rc = upload(h, h->at<double>(h->lay.macro[1]), ux, b))) return rc;
  if ((rc = upload(h, h->at<double>(h->lay.macro[2]), uy, b))) return rc;
  if (T && (rc = upload(h, h->at<double>(h->lay.macro[3]), T, b))) return rc;
  if (h->precision == SLBM_FX16 && (rc = set_fx_scales(h))) return rc;
  if ((rc = init_eq_dev(h, T != nullptr))) return rc;
  // the caller may reuse its arrays on return
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_set_flags(slbm_t h, const uint8_t* flags) {
  SLBM_GUARD(h);
  if (!flags) return fail(h, SLBM_EINVAL, "flags is required");
  std::vector<uint8_t> norm(h->ncell());
  for (size_t c = 0; c < norm.size(); ++c) norm[c] = flags[c] ? 1 : 0;
  if (h->nchan)  // the gap columns between channels stay gaps
    for (size_t c = 0; c < norm.size(); ++c)
      if (h->gapcol[c % h->g.nx]) norm[c] = kFlagGap;
  uint8_t* tmp = h->at<uint8_t>(h->lay.flag_tmp);
  int rc;
  if ((rc = upload(h, tmp, norm.data(), norm.size()))) return rc;
  if (h->frame != SLBM_FRAME_LATTICE) {
    // every cell's other lattice from its current one (flipped cells take it
    // as their new native vector), then the new flags, masks and band
    cudaError_t e =
        h->precision == SLBM_FP64
            ? launch_pond_convert<double, double>(h->qd, (double*)h->pops(h->cur, 0),
                                                  (double*)h->pops(h->cur, 1),
                                                  (double*)h->gp(h->cur, 0),
                                                  (double*)h->gp(h->cur, 1),
                                                  (const double*)h->lam(h->cur),
                                                  h->flags(h->fcur), nullptr, nullptr, 0, conv_lists(h), h->st)
            : launch_pond_convert<float, float>(h->qf, (float*)h->pops(h->cur, 0),
                                                (float*)h->pops(h->cur, 1),
                                                (float*)h->gp(h->cur, 0), (float*)h->gp(h->cur, 1),
                                                (const float*)h->lam(h->cur), h->flags(h->fcur),
                                                nullptr, nullptr, 0, conv_lists(h), h->st);
    SLBM_CK(h, e, "co-moving conversion launch");
    SLBM_CK(h, cudaMemcpyAsync(h->flags(h->fcur), tmp, norm.size(), cudaMemcpyDeviceToDevice,
                               h->st),
            "flag copy");
    SLBM_CK(h, launch_pond_masks(h->g.nx, h->g.ny, h->flags(h->fcur), nullptr,
                                 h->at<uint8_t>(h->lay.tile_mask[0]), h->st),
            "mask launch");
    bool any0 = false, any1 = false;
    for (uint8_t v : norm) (v ? any1 : any0) = true;
    h->pond_mixed = any0 && any1;
    drop_graphs(h);  // the step's kernel set depends on pond_mixed
    if ((rc = pond_convert_band(h, h->cur))) return rc;
    SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
    return SLBM_OK;
  }
  SLBM_CK(h, convert(h, h->cur, h->flags(h->fcur), tmp), "convert launch");
  SLBM_CK(h, cudaMemcpyAsync(h->flags(h->fcur), tmp, norm.size(), cudaMemcpyDeviceToDevice, h->st),
          "flag copy");
  SLBM_CK(h, ghosts(h, h->flags(h->fcur)), "ghost launch");
  // the host vector must stay alive until the copy has consumed it
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_get_flags(slbm_t h, uint8_t* flags) {
  SLBM_GUARD(h);
  if (!flags) return fail(h, SLBM_EINVAL, "flags is required");
  SLBM_CK(h, cudaMemcpyAsync(flags, h->flags(h->fcur), h->ncell(), cudaMemcpyDeviceToHost, h->st),
          "D2H copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_set_criterion(slbm_t h, int kind, double threshold) {
  SLBM_GUARD(h);
  if ((kind != SLBM_CRIT_NONE && kind != SLBM_CRIT_MACH && !is_mlp(kind)) ||
      !std::isfinite(threshold) || (kind == SLBM_CRIT_MACH && !(threshold >= 0.0)))
    return fail(h, SLBM_EINVAL, "criterion kind or threshold invalid");
  if (is_mlp(kind) && !h->ind_buf)
    return fail(h, SLBM_EINVAL, "no indicator weights (slbm_set_indicator); use SLBM_CRIT_MACH");
  if (kind == SLBM_CRIT_MACH && h->nchan)
    return fail(h, SLBM_EINVAL, "channels keep fixed flags or the learned indicator");
  if (kind != SLBM_CRIT_NONE && h->frame != SLBM_FRAME_LATTICE)
    return fail(h, SLBM_EINVAL, "the Mach criterion belongs to the lattice frame");
  // flags live in buffer fcur either way; the other buffer is scratch
  h->crit = kind;
  if (!is_mlp(kind)) h->thr = threshold;
  refresh_params(h);
  if (kind == SLBM_CRIT_MACH) {
    // evaluate the criterion on the current state at once; flips are converted
    uint8_t* tmp = h->at<uint8_t>(h->lay.flag_tmp);
    const cudaError_t e = with_types(h, [&](auto ty, const auto& prm) {
      SLBM_TYPES(ty);
      return launch_criterion<S, R>(prm, (const S*)h->pops(h->cur, 0),
                                    (const S*)h->pops(h->cur, 1), h->flags(h->fcur), tmp, h->st);
    });
    SLBM_CK(h, e, "criterion launch");
    SLBM_CK(h, convert(h, h->cur, h->flags(h->fcur), tmp), "convert launch");
    SLBM_CK(h, cudaMemcpyAsync(h->flags(h->fcur), tmp, h->ncell(), cudaMemcpyDeviceToDevice, h->st),
            "flag copy");
    SLBM_CK(h, ghosts(h, h->flags(h->fcur)), "ghost launch");
  }
  if (is_mlp(kind)) {
    h->ind_thr = threshold;
    return apply_indicator(h);
  }
  return SLBM_OK;
}

int slbm_set_indicator(slbm_t h, const float* w1, const float* b1, const float* w2,
                       const float* b2, const float* w3, float b3, int interval) {
  SLBM_GUARD(h);
  if (!w1 || !b1 || !w2 || !b2 || !w3 || interval < 1 || !std::isfinite(b3))
    return fail(h, SLBM_EINVAL, "indicator weights and interval >= 1 are required");
  if (h->frame != SLBM_FRAME_LATTICE) return fail(h, SLBM_EINVAL, "lattice frame only");
  const size_t nw1 = 16 * 32, nw2 = 32 * 32;
  const size_t bytes = (nw1 + nw2) * sizeof(__half) + (32 + 32 + 32) * sizeof(float);
  if (!h->ind_buf) SLBM_CK(h, cudaMalloc(&h->ind_buf, bytes), "indicator weights cudaMalloc");
  std::vector<__half> hw(nw1 + nw2);
  for (size_t i = 0; i < nw1; ++i) hw[i] = __float2half_rn(w1[i]);
  for (size_t i = 0; i < nw2; ++i) hw[nw1 + i] = __float2half_rn(w2[i]);
  std::vector<float> hf(96);
  for (int i = 0; i < 32; ++i) {
    hf[i] = b1[i];
    hf[32 + i] = b2[i];
    hf[64 + i] = w3[i];
  }
  char* base = (char*)h->ind_buf;
  SLBM_CK(h, cudaMemcpyAsync(base, hw.data(), hw.size() * sizeof(__half), cudaMemcpyHostToDevice,
                             h->st), "H2D copy");
  float* fb = (float*)(base + hw.size() * sizeof(__half));
  SLBM_CK(h, cudaMemcpyAsync(fb, hf.data(), hf.size() * sizeof(float), cudaMemcpyHostToDevice, h->st),
          "H2D copy");
  h->ind = IndicatorDev{(const __half*)base, fb, (const __half*)base + nw1, fb + 32, fb + 64, b3};
  h->ind_interval = interval;
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");  // the host vectors are released
  return SLBM_OK;
}

int slbm_indicator_eval(slbm_t h, float* features, float* logits, uint8_t* flags) {
  SLBM_GUARD(h);
  if (h->frame != SLBM_FRAME_LATTICE) return fail(h, SLBM_EINVAL, "lattice frame only");
  if ((logits || flags) && !h->ind_buf)
    return fail(h, SLBM_EINVAL, "no indicator weights (slbm_set_indicator)");
  const size_t nc = h->ncell();
  float* dfeat = nullptr;
  float* dlog = nullptr;
  uint8_t* dfl = nullptr;
  if (features) SLBM_CK(h, cudaMalloc(&dfeat, nc * 16 * sizeof(float)), "cudaMalloc");
  if (logits && cudaMalloc(&dlog, nc * sizeof(float)) != cudaSuccess) {
    cudaFree(dfeat);
    return fail(h, SLBM_ENOMEM, "cudaMalloc");
  }
  if (flags && cudaMalloc(&dfl, nc) != cudaSuccess) {
    cudaFree(dfeat);
    cudaFree(dlog);
    return fail(h, SLBM_ENOMEM, "cudaMalloc");
  }
  IndicatorDev keep = h->ind;
  if (!h->ind_buf) h->ind = IndicatorDev{nullptr, nullptr, nullptr, nullptr, nullptr, 0.f};
  int rc = run_indicator(h, dfeat, dlog, dfl);
  h->ind = keep;
  if (!rc && features && cudaMemcpyAsync(features, dfeat, nc * 16 * sizeof(float),
                                         cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
    rc = fail(h, SLBM_ECUDA, "D2H copy");
  if (!rc && logits && cudaMemcpyAsync(logits, dlog, nc * sizeof(float), cudaMemcpyDeviceToHost,
                                       h->st) != cudaSuccess)
    rc = fail(h, SLBM_ECUDA, "D2H copy");
  if (!rc && flags && cudaMemcpyAsync(flags, dfl, nc, cudaMemcpyDeviceToHost, h->st) != cudaSuccess)
    rc = fail(h, SLBM_ECUDA, "D2H copy");
  if (!rc && cudaStreamSynchronize(h->st) != cudaSuccess) rc = fail(h, SLBM_ECUDA, "sync");
  cudaFree(dfeat);
  cudaFree(dlog);
  cudaFree(dfl);
  return rc;
}

int slbm_lattice_loss(slbm_t h, double* loss) {
  SLBM_GUARD(h);
  if (!loss) return fail(h, SLBM_EINVAL, "loss is required");
  if (h->frame != SLBM_FRAME_LATTICE) return fail(h, SLBM_EINVAL, "lattice frame only");
  if (h->crit != SLBM_CRIT_NONE)
    return fail(h, SLBM_EINVAL, "the lattice loss needs fixed flags (SLBM_CRIT_NONE)");
  const size_t nc = h->ncell();
  std::vector<uint8_t> fl(nc);
  int rc = slbm_get_flags(h, fl.data());
  if (rc) return rc;
  for (uint8_t v : fl)
    if (v != 1 && v != kFlagGap)
      return fail(h, SLBM_EINVAL, "the lattice loss starts from an all-high-order state");
  const size_t es = (size_t)elem_size(h->precision);
  const size_t bytes = (size_t)(h->nhi * h->nhi) * h->lay.plane * es;
  char* tmp = nullptr;
  if (cudaMalloc(&tmp, 2 * bytes + nc * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return fail(h, SLBM_ENOMEM, "cudaMalloc");
  }
  char* start = tmp;           // f_Q(t), ghost ring included
  char* stepped = tmp + bytes;  // f_Q(t + 1)
  double* dloss = reinterpret_cast<double*>(tmp + 2 * bytes);
  std::vector<uint8_t> lo(nc, 0), hi(nc, 1);
  auto d2d = [&](void* dst, const void* src) {
    return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->st);
  };
  // high-order step; back to the start; projected step; lifting
  rc = d2d(start, h->pops(h->cur, 1)) != cudaSuccess ? fail(h, SLBM_ECUDA, "D2D copy") : SLBM_OK;
  if (!rc) rc = slbm_step(h, 1);
  if (!rc && d2d(stepped, h->pops(h->cur, 1)) != cudaSuccess) rc = fail(h, SLBM_ECUDA, "D2D copy");
  if (!rc && d2d(h->pops(h->cur, 1), start) != cudaSuccess) rc = fail(h, SLBM_ECUDA, "D2D copy");
  if (!rc) rc = slbm_set_flags(h, lo.data());
  if (!rc) rc = slbm_step(h, 1);
  if (!rc) rc = slbm_set_flags(h, hi.data());
  if (!rc) {
    const cudaError_t e = with_types(h, [&](auto ty, const auto& prm) {
      SLBM_TYPES(ty);
      return launch_lattice_loss<S, R>(prm, (const S*)stepped, (const S*)h->pops(h->cur, 1),
                                       h->flags(h->fcur), dloss, h->st);
    });
    if (e != cudaSuccess) rc = fail(h, SLBM_ECUDA, "lattice loss launch", e);
  }
  // the handle continues from the high-order step
  if (!rc && d2d(h->pops(h->cur, 1), stepped) != cudaSuccess) rc = fail(h, SLBM_ECUDA, "D2D copy");
  if (!rc && cudaMemcpyAsync(loss, dloss, nc * sizeof(double), cudaMemcpyDeviceToHost, h->st) !=
                 cudaSuccess)
    rc = fail(h, SLBM_ECUDA, "D2H copy");
  if (!rc && cudaStreamSynchronize(h->st) != cudaSuccess) rc = fail(h, SLBM_ECUDA, "sync");
  if (!rc) h->steps -= 1;  // one step of the state, not two
  cudaFree(tmp);
  return rc;
}

int slbm_mlp_train(const float* x, const float* y, long long n, const int* idx, int steps,
                   int batch, const double hyper[4], int t0, float* params, float* adam,
                   float* loss, float* grad, void* cuda_stream) {
  if (!x || !y || !idx || !params || !adam || !hyper || n < 1 || steps < 0 || t0 < 0 ||
      batch < 128 || batch > kMlpMaxBatch || batch % 128)
    return SLBM_EINVAL;
  const double lr = hyper[0], b1 = hyper[1], b2 = hyper[2], eps = hyper[3];
  if (!(lr > 0.0) || !std::isfinite(lr) || !(b1 >= 0.0 && b1 < 1.0) || !(b2 >= 0.0 && b2 < 1.0) ||
      !(eps > 0.0) || !std::isfinite(eps))
    return SLBM_EINVAL;
  const size_t nidx = (size_t)steps * (size_t)batch;
  for (size_t i = 0; i < nidx; ++i)
    if (idx[i] < 0 || idx[i] >= n) return SLBM_EINVAL;
  for (long long i = 0; i < n; ++i)
    if (!(y[i] == 0.f || y[i] == 1.f)) return SLBM_EINVAL;
  if (steps == 0) return SLBM_OK;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  const size_t bx = (size_t)n * 16 * sizeof(float), by = (size_t)n * sizeof(float);
  const size_t bi = nidx * sizeof(int), bp = kMlpParams * sizeof(float);
  const size_t bl = (size_t)steps * sizeof(float);
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  char* d = nullptr;
  if (cudaMalloc(&d, al(bx) + al(by) + al(bi) + 4 * al(bp) + al(bl)) != cudaSuccess) {
    cudaGetLastError();
    return SLBM_ENOMEM;
  }
  float* dx = reinterpret_cast<float*>(d);
  float* dy = reinterpret_cast<float*>(d + al(bx));
  int* di = reinterpret_cast<int*>(d + al(bx) + al(by));
  float* dp = reinterpret_cast<float*>(d + al(bx) + al(by) + al(bi));
  float* da = dp + al(bp) / sizeof(float);            // 2 x kMlpParams
  float* dg = da + 2 * al(bp) / sizeof(float);
  float* dl = dg + al(bp) / sizeof(float);
  cudaError_t e = cudaMemcpyAsync(dx, x, bx, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, by, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(di, idx, bi, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dp, params, bp, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(da, adam, 2 * bp, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = launch_mlp_train(dx, dy, di, steps, batch, (float)lr, (float)b1, (float)b2, (float)eps, t0,
                         dp, da, loss ? dl : nullptr, grad ? dg : nullptr, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(params, dp, bp, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(adam, da, 2 * bp, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, dl, bl, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, dg, bp, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  return e == cudaSuccess ? SLBM_OK : SLBM_ECUDA;
}

int slbm_set_boundary(slbm_t h, int side, int kind, const double* rho, const double* ux,
                      const double* uy) {
  SLBM_GUARD(h);
  if (side < 0 || side > 3) return fail(h, SLBM_EINVAL, "side out of range");
  if ((side < 2 && h->g.periodic_x) || (side >= 2 && h->g.periodic_y))
    return fail(h, SLBM_EINVAL, "side is periodic");
  if (kind == SLBM_BC_DIRICHLET && (!rho || !ux || !uy))
    return fail(h, SLBM_EINVAL, "DIRICHLET needs rho, ux, uy");
  if ((kind == SLBM_BC_INLET || kind == SLBM_BC_DIFFUSE) && (!ux || !uy))
    return fail(h, SLBM_EINVAL, "INLET and DIFFUSE need ux, uy");
  if (kind != SLBM_BC_OUTFLOW && kind != SLBM_BC_DIRICHLET && kind != SLBM_BC_INLET &&
      kind != SLBM_BC_DIFFUSE)
    return fail(h, SLBM_EINVAL, "unknown boundary kind");
  if (kind == SLBM_BC_DIFFUSE && !(side < 2 ? h->g.periodic_y : h->g.periodic_x))
    return fail(h, SLBM_EINVAL, "a DIFFUSE wall needs the axis along it periodic");
  const size_t len = (size_t)(side < 2 ? h->g.ny : h->g.nx);
  const double* src[3] = {rho, ux, uy};
  for (int q = 0; q < 3; ++q)
    if (src[q]) {
      int rc = upload(h, h->at<double>(h->lay.bc[side][q]), src[q], len * 8);
      if (rc) return rc;
    }
  h->bc_kind[side] = kind;
  drop_graphs(h);
  SLBM_CK(h, ghosts(h, h->flags(h->fcur)), "ghost launch");
  return build_ghost_tables(h);
}


int slbm_set_kn_criterion(slbm_t h, double thr, int interval) {
  SLBM_GUARD(h);
  if (!h->rows || !h->hs || !h->twopop)
    return fail(h, SLBM_EINVAL, "the Knudsen criterion needs batched rows and the viscosity law");
  if (!(thr > 0.0) || interval < 1) return fail(h, SLBM_EINVAL, "need thr > 0 and interval >= 1");
  h->kn_on = 1;
  h->kn_thr = thr;
  h->kn_interval = interval;
  h->pond_mixed = 1;  // flags may change every interval: keep the band conversion on
  drop_graphs(h);
  if (int rc = apply_kn(h, true)) return rc;
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return check_device_error(h);
}

int slbm_step(slbm_t h, int n) {
  SLBM_GUARD(h);
  if (n < 0) return fail(h, SLBM_EINVAL, "n must be >= 0");
  int s = 0;
  while (s < n) {
    // steps up to the next learned-indicator evaluation
    int chunk = n - s;
    if (is_mlp(h->crit)) {
      const int to_eval = h->ind_interval - (int)(h->steps % h->ind_interval);
      if (to_eval < chunk) chunk = to_eval;
    }
    if (h->kn_on && !kn_every_step(h)) {
      const int to_eval = h->kn_interval - (int)(h->steps % h->kn_interval);
      if (to_eval < chunk) chunk = to_eval;
    }
    int done = 0;
    // pairs of steps as graph launches once the kernels have run directly
    // (their one-time attribute and occupancy set-up), unless tracing needs
    // the per-kernel events
    const bool graphs = !h->profiling && !h->graphs_off &&
                        (h->frame == SLBM_FRAME_LATTICE ? h->sc_launches > 0 : h->steps > 0);
    while (graphs && !h->graphs_off && chunk - done >= 2) {
      // 2 kGraphPairs steps per graph while that many remain, then pairs
      const int m = chunk - done >= 2 * kGraphPairs ? kGraphPairs : 1;
      const int rc = step_pair(h, m);
      if (rc == 1) break;
      if (rc) return rc;
      done += 2 * m;
    }
    for (; done < chunk; ++done) {
      int rc = step_once(h);
      if (!rc && kn_every_step(h)) rc = apply_kn(h, false);
      if (rc) return rc;
    }
    s += chunk;
    if (is_mlp(h->crit) && h->steps % h->ind_interval == 0) {
      const int rc = apply_indicator(h);
      if (rc) return rc;
    }
    if (h->kn_on && !kn_every_step(h) && h->steps % h->kn_interval == 0) {
      const int rc = apply_kn(h, false);
      if (rc) return rc;
    }
  }
  return SLBM_OK;
}

int slbm_sync(slbm_t h) {
  SLBM_GUARD(h);
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return check_device_error(h);
}

int slbm_moments_device(slbm_t h, double* rho, double* ux, double* uy, double* T) {
  SLBM_GUARD(h);
  cudaError_t e;
  e = with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_moments<S, R>(prm, (const S*)h->pops(h->cur, 0), (const S*)h->pops(h->cur, 1),
                                h->flags(h->fcur), rho, ux, uy, T, (const S*)frame_planes(h),
                                h->st, (const S*)h->gp(h->cur, 0), (const S*)h->gp(h->cur, 1));
  });
  SLBM_CK(h, e, "moments launch");
  return SLBM_OK;
}

int slbm_moments(slbm_t h, double* rho, double* ux, double* uy, double* T) {
  SLBM_GUARD(h);
  double* d[4];
  for (int m = 0; m < 4; ++m) d[m] = h->at<double>(h->lay.macro[m]);
  int rc = slbm_moments_device(h, rho ? d[0] : nullptr, ux ? d[1] : nullptr, uy ? d[2] : nullptr,
                               T ? d[3] : nullptr);
  if (rc) return rc;
  double* out[4] = {rho, ux, uy, T};
  for (int m = 0; m < 4; ++m)
    if (out[m])
      SLBM_CK(h, cudaMemcpyAsync(out[m], d[m], h->ncell() * 8, cudaMemcpyDeviceToHost, h->st),
              "D2H copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return check_device_error(h);
}

int slbm_audit(slbm_t h, double out[4]) {
  SLBM_GUARD(h);
  if (!out) return fail(h, SLBM_EINVAL, "out is required");
  const int np = audit_parts(h->g.nx, h->g.ny);
  double* part = h->at<double>(h->lay.partials);
  double* res = h->at<double>(h->lay.audit_out);
  cudaError_t e;
  e = with_types(h, [&](auto ty, const auto& prm) {
    SLBM_TYPES(ty);
    return launch_audit<S, R>(prm, (const S*)h->pops(h->cur, 0), (const S*)h->pops(h->cur, 1),
                              h->flags(h->fcur), part, np, res, (const S*)frame_planes(h), h->st,
                              (const S*)h->gp(h->cur, 0), (const S*)h->gp(h->cur, 1));
  });
  SLBM_CK(h, e, "audit launch");
  SLBM_CK(h, cudaMemcpyAsync(out, res, 32, cudaMemcpyDeviceToHost, h->st), "D2H copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  if (int rc = check_device_error(h)) return rc;
  for (int q = 0; q < 4; ++q)
    if (!std::isfinite(out[q])) return fail(h, SLBM_ENONFINITE, "audit: non-finite sum");
  return SLBM_OK;
}

int slbm_get_pops(slbm_t h, int k, double* out) {
  SLBM_GUARD(h);
  if ((k != 0 && k != 1) || !out) return fail(h, SLBM_EINVAL, "lattice index or output invalid");
  return pack_any(h, k, out, 0, nullptr);
}

int slbm_set_pops(slbm_t h, int k, const double* in) {
  SLBM_GUARD(h);
  if ((k != 0 && k != 1) || !in) return fail(h, SLBM_EINVAL, "lattice index or input invalid");
  int rc = pack_any(h, k, nullptr, 1, in);
  if (rc) return rc;
  if (h->frame != SLBM_FRAME_LATTICE) return pond_convert_band(h, h->cur);
  SLBM_CK(h, convert(h, h->cur, h->flags(h->fcur), h->flags(h->fcur)), "post-step launch");
  SLBM_CK(h, ghosts(h, h->flags(h->fcur)), "ghost launch");
  return SLBM_OK;
}

namespace {
struct StateHeader {
  char magic[8];
  int nx, ny, nlo, nhi, precision, pad;
  long long steps;
};
}  // namespace

int slbm_get_state(slbm_t h, void* buf, size_t* bytes) {
  SLBM_GUARD(h);
  if (!bytes) return fail(h, SLBM_EINVAL, "bytes is required");
  const size_t nc = h->ncell();
  const size_t nframe = h->frame != SLBM_FRAME_LATTICE ? 3 * nc * 8 : 0;
  const size_t need =
      sizeof(StateHeader) + nc + nc * 8 * (size_t)(h->nlo * h->nlo + h->nhi * h->nhi) + nframe;
  if (!buf) { *bytes = need; return SLBM_OK; }
  if (*bytes < need) return fail(h, SLBM_EINVAL, "state buffer too small");
  StateHeader hd{};
  std::memcpy(hd.magic, "SLBMST1", 8);
  hd.nx = h->g.nx; hd.ny = h->g.ny; hd.nlo = h->nlo; hd.nhi = h->nhi;
  hd.precision = h->precision; hd.pad = h->frame; hd.steps = h->steps;
  char* p = (char*)buf;
  std::memcpy(p, &hd, sizeof(hd));
  int rc = slbm_get_flags(h, (uint8_t*)(p + sizeof(hd)));
  if (rc) return rc;
  double* pops = (double*)(p + sizeof(hd) + nc);
  if ((rc = slbm_get_pops(h, 0, pops))) return rc;
  if ((rc = slbm_get_pops(h, 1, pops + nc * h->nlo * h->nlo))) return rc;
  if (nframe) {
    double* fr = pops + nc * (size_t)(h->nlo * h->nlo + h->nhi * h->nhi);
    if ((rc = slbm_get_frame(h, fr, fr + nc, fr + 2 * nc))) return rc;
  }
  *bytes = need;
  return SLBM_OK;
}

int slbm_set_state(slbm_t h, const void* buf, size_t bytes) {
  SLBM_GUARD(h);
  const size_t nc = h->ncell();
  const size_t nframe = h->frame != SLBM_FRAME_LATTICE ? 3 * nc * 8 : 0;
  const size_t need =
      sizeof(StateHeader) + nc + nc * 8 * (size_t)(h->nlo * h->nlo + h->nhi * h->nhi) + nframe;
  if (!buf || bytes < need) return fail(h, SLBM_EINVAL, "state buffer too small");
  StateHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  if (std::memcmp(hd.magic, "SLBMST1", 8) || hd.nx != h->g.nx || hd.ny != h->g.ny ||
      hd.nlo != h->nlo || hd.nhi != h->nhi || hd.precision != h->precision ||
      hd.pad != h->frame)
    return fail(h, SLBM_EINVAL, "state does not match this handle");
  const char* p = (const char*)buf;
  int rc;
  if (h->frame != SLBM_FRAME_LATTICE) {
    // flags (with their masks), frames, then populations and band conversions
    std::vector<uint8_t> fl((const uint8_t*)(p + sizeof(hd)), (const uint8_t*)(p + sizeof(hd)) + nc);
    if ((rc = upload(h, h->flags(h->fcur), fl.data(), nc))) return rc;
    SLBM_CK(h, launch_pond_masks(h->g.nx, h->g.ny, h->flags(h->fcur), nullptr,
                                 h->at<uint8_t>(h->lay.tile_mask[0]), h->st),
            "mask launch");
    bool any0 = false, any1 = false;
    for (uint8_t v : fl) (v ? any1 : any0) = true;
    h->pond_mixed = any0 && any1;
    drop_graphs(h);  // the step's kernel set depends on pond_mixed
    const double* fr =
        (const double*)(p + sizeof(hd) + nc) + nc * (size_t)(h->nlo * h->nlo + h->nhi * h->nhi);
    if ((rc = slbm_set_frame(h, fr, fr + nc, fr + 2 * nc))) return rc;
  } else if ((rc = upload(h, h->flags(h->fcur), p + sizeof(hd), nc))) {
    return rc;
  }
  const double* pops = (const double*)(p + sizeof(hd) + nc);
  if ((rc = pack_any(h, 0, nullptr, 1, pops))) return rc;
  if ((rc = pack_any(h, 1, nullptr, 1, pops + nc * h->nlo * h->nlo))) return rc;
  if (h->frame != SLBM_FRAME_LATTICE) {
    if ((rc = pond_convert_band(h, h->cur))) return rc;
  } else {
    // masks from the restored flags; the restored band populations are the
    // conversions of the restored native ones, so recomputing them is exact
    SLBM_CK(h, convert(h, h->cur, h->flags(h->fcur), h->flags(h->fcur)), "post-step launch");
    SLBM_CK(h, ghosts(h, h->flags(h->fcur)), "ghost launch");
  }
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  h->steps = hd.steps;
  return SLBM_OK;
}

namespace {
// The handle's row arrays (allocated on first use, on the handle's device).
int ensure_rowbuf(slbm_t h) {
  if (h->rowbuf) return SLBM_OK;
  const size_t ny = (size_t)h->g.ny;
  h->rb_len = 0;
  h->rb_ends = (ny * sizeof(int) + 255) / 256 * 256;
  h->rb_visc = h->rb_ends + (8 * ny * sizeof(double) + 255) / 256 * 256;
  const size_t bytes = h->rb_visc + 2 * ny * sizeof(double);
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != h->dev) cudaSetDevice(h->dev);
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, bytes);
  if (dev_prev >= 0 && dev_prev != h->dev) cudaSetDevice(dev_prev);
  SLBM_CK(h, e, "row arrays allocation");
  h->rowbuf = (char*)buf;
  SLBM_CK(h, cudaMemsetAsync(h->rowbuf, 0, bytes, h->st), "row arrays clear");
  return SLBM_OK;
}
}  // namespace

int slbm_set_channels(slbm_t h, int n, const int* x0, const int* width, const double* uw_lo,
                      const double* uw_hi, const double* tau) {
  SLBM_GUARD(h);
  if (h->frame != SLBM_FRAME_LATTICE)
    return fail(h, SLBM_EINVAL, "channels belong to the lattice frame");
  if (h->nchan) return fail(h, SLBM_ESTATE, "channels are already set");
  if (h->crit == SLBM_CRIT_MACH)
    return fail(h, SLBM_EINVAL, "channels keep fixed flags or the learned indicator");
  if (!h->g.periodic_y) return fail(h, SLBM_EINVAL, "channels need a periodic y axis");
  if (n < 1 || !x0 || !width || !uw_lo || !uw_hi || !tau)
    return fail(h, SLBM_EINVAL, "n >= 1 and every array are required");
  const int G = h->lay.G, nx = h->g.nx, ny = h->g.ny;
  for (int c = 0; c < n; ++c) {
    const int lo = c ? x0[c - 1] + width[c - 1] + 2 * G : G;
    if (width[c] < 2 * G + 1 || x0[c] < lo || x0[c] + width[c] + G > nx)
      return fail(h, SLBM_EINVAL,
                  "channel c must span x0 .. x0 + width - 1 with width >= 2G + 1, x0 >= G, "
                  "x0 + width + G <= nx, and 2G gap columns before the next channel");
    if (!(tau[c] > 0.5) || !std::isfinite(tau[c]) || !std::isfinite(uw_lo[c]) ||
        !std::isfinite(uw_hi[c]))
      return fail(h, SLBM_EINVAL, "tau must exceed 1/2 and the wall speeds be finite");
  }
  // host tables: gap columns, per-column omega, internal wall ghosts (G
  // columns beside each channel side, every row) and their velocities
  std::vector<uint8_t> gap(nx, 1);
  std::vector<double> om(nx, 1.0 / h->tau);
  std::vector<int> wall;
  std::vector<double> wu;
  for (int c = 0; c < n; ++c) {
    for (int x = x0[c]; x < x0[c] + width[c]; ++x) {
      gap[x] = 0;
      om[x] = 1.0 / tau[c];
    }
    for (int y = 0; y < ny; ++y)
      for (int k = 0; k < G; ++k) {
        wall.insert(wall.end(), {x0[c] - G + k, y, x0[c], SLBM_SIDE_XMIN});
        wu.insert(wu.end(), {0.0, uw_lo[c]});
        wall.insert(wall.end(), {x0[c] + width[c] + k, y, x0[c] + width[c] - 1, SLBM_SIDE_XMAX});
        wu.insert(wu.end(), {0.0, uw_hi[c]});
      }
  }
  const int nwall = (int)(wall.size() / 4);
  const size_t ring = 2 * (size_t)G * (nx + 2 * G) + 2 * (size_t)G * ny;
  const size_t es = h->precision == SLBM_FP64 ? 8 : 4;
  h->cb_wallu = align_up(wall.size() * sizeof(int), 256);
  h->cb_omega = h->cb_wallu + align_up(wu.size() * sizeof(double), 256);
  h->cb_ghidx = h->cb_omega + align_up(nx * es, 256);
  const size_t bytes = h->cb_ghidx + (ring + nwall) * sizeof(int);
  void* buf = nullptr;
  SLBM_CK(h, cudaMalloc(&buf, bytes), "channel arrays allocation");
  h->chanbuf = (char*)buf;
  std::vector<float> omf(om.begin(), om.end());
  int rc;
  if ((rc = upload(h, h->chanbuf, wall.data(), wall.size() * sizeof(int))) ||
      (rc = upload(h, h->chanbuf + h->cb_wallu, wu.data(), wu.size() * sizeof(double))) ||
      (rc = upload(h, h->chanbuf + h->cb_omega,
                   es == 8 ? (const void*)om.data() : (const void*)omf.data(), nx * es)))
    return rc;
  h->gapcol = gap;
  h->nchan = n;
  h->nwall = nwall;
  refresh_params(h);
  if ((rc = build_ghost_tables(h))) return rc;
  // every channel cell starts in the low-order lattice, the gaps as gaps
  std::vector<uint8_t> fl(h->ncell(), 0);
  if ((rc = slbm_set_flags(h, fl.data()))) return rc;
  // the other flag buffer too (the learned indicator writes it)
  for (size_t c = 0; c < fl.size(); ++c) fl[c] = gap[c % nx] ? kFlagGap : 0;
  if ((rc = upload(h, h->flags(h->fcur ^ 1), fl.data(), fl.size()))) return rc;
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_set_rows(slbm_t h, const int* len, const double* ends) {
  SLBM_GUARD(h);
  if (h->frame == SLBM_FRAME_LATTICE) return fail(h, SLBM_EINVAL, "rows need a co-moving frame");
  if (!len || !ends) return fail(h, SLBM_EINVAL, "len and ends are required");
  for (int r = 0; r < h->g.ny; ++r) {
    if (len[r] < h->P || len[r] > h->g.nx) return fail(h, SLBM_EINVAL, "row length out of range");
    for (int side = 0; side < 2; ++side)
      if (!(ends[8 * r + 4 * side] > 0.0) || !(ends[8 * r + 4 * side + 3] > 0.0))
        return fail(h, SLBM_EINVAL, "end states need rho > 0 and T > 0");
  }
  if (int rc = ensure_rowbuf(h)) return rc;
  if (int rc = upload(h, h->rowbuf + h->rb_len, len, (size_t)h->g.ny * sizeof(int))) return rc;
  if (int rc = upload(h, h->rowbuf + h->rb_ends, ends, (size_t)h->g.ny * 8 * sizeof(double)))
    return rc;
  h->rows = 1;
  refresh_params(h);
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_set_viscosity_law(slbm_t h, const double* mu1, const double* T1, double s_exp,
                           double pr) {
  SLBM_GUARD(h);
  if (!h->twopop) return fail(h, SLBM_EINVAL, "the viscosity law needs the two-population model");
  if (!mu1 || !T1 || !(pr > 0.0)) return fail(h, SLBM_EINVAL, "mu1, T1 and pr > 0 are required");
  std::vector<double> v(2 * (size_t)h->g.ny);
  for (int r = 0; r < h->g.ny; ++r) {
    if (!(mu1[r] > 0.0) || !(T1[r] > 0.0)) return fail(h, SLBM_EINVAL, "need mu1 > 0 and T1 > 0");
    v[2 * r] = mu1[r];
    v[2 * r + 1] = T1[r];
  }
  if (int rc = ensure_rowbuf(h)) return rc;
  if (int rc = upload(h, h->rowbuf + h->rb_visc, v.data(), v.size() * sizeof(double))) return rc;
  h->hs = 1;
  h->s_exp = s_exp;
  h->pr = pr;
  refresh_params(h);
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_tune(slbm_t h, int reps, int* bx, int* by) {
  SLBM_GUARD(h);
  if (h->frame == SLBM_FRAME_LATTICE)
    return fail(h, SLBM_EINVAL, "the lattice-frame step has a fixed tile design");
  if (reps < 1) return fail(h, SLBM_EINVAL, "reps must be >= 1");
  static const int shapes[5][2] = {{32, 8}, {64, 4}, {128, 2}, {256, 1}, {16, 16}};
  cudaEvent_t ea, eb;
  SLBM_CK(h, cudaEventCreate(&ea), "event");
  SLBM_CK(h, cudaEventCreate(&eb), "event");
  float best = -1.0f;
  int bi = 0;
  int rc = SLBM_OK;
  for (int c = 0; c < 5 && rc == SLBM_OK; ++c) {
    h->pond_bx = shapes[c][0];
    h->pond_by = shapes[c][1];
    refresh_params(h);
    // the step kernel reads buffer cur and writes the other: repeating it
    // leaves the state as it was
    cudaError_t e = pond_launch(h, h->cur, h->cur ^ 1);
    if (e == cudaSuccess) e = cudaEventRecord(ea, h->st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = pond_launch(h, h->cur, h->cur ^ 1);
    if (e == cudaSuccess) e = cudaEventRecord(eb, h->st);
    if (e == cudaSuccess) e = cudaEventSynchronize(eb);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ea, eb);
    if (e != cudaSuccess) {
      rc = fail(h, SLBM_ECUDA, "tuning launch", e);
      break;
    }
    if (best < 0.0f || ms < best) {
      best = ms;
      bi = c;
    }
  }
  cudaEventDestroy(ea);
  cudaEventDestroy(eb);
  if (rc) return rc;
  h->pond_bx = shapes[bi][0];
  h->pond_by = shapes[bi][1];
  refresh_params(h);
  // the timing launches may have flagged unconverged updates of the scratch buffer
  SLBM_CK(h, cudaMemsetAsync(h->at<int>(h->lay.err), 0, sizeof(int), h->st), "error word clear");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  if (bx) *bx = h->pond_bx;
  if (by) *by = h->pond_by;
  return SLBM_OK;
}

int slbm_set_twopop(slbm_t h, double cv, double tau2) {
  SLBM_GUARD(h);
  if (h->frame != SLBM_FRAME_POND) return fail(h, SLBM_EINVAL, "two populations need the thermal co-moving frame");
  if (!(cv > 0.0) || !(tau2 > 0.5)) return fail(h, SLBM_EINVAL, "need C_v > 0 and tau2 > 1/2");
  if (h->twopop) return fail(h, SLBM_EINVAL, "the two-population model is already set");
  const size_t es = h->precision == SLBM_FP64 ? 8 : 4;
  const size_t bytes =
      2 * es * (size_t)h->lay.plane * (size_t)(h->nlo * h->nlo + h->nhi * h->nhi);
  int dev_prev = -1;
  cudaGetDevice(&dev_prev);
  if (dev_prev != h->dev) cudaSetDevice(h->dev);
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, bytes);
  if (dev_prev >= 0 && dev_prev != h->dev) cudaSetDevice(dev_prev);
  SLBM_CK(h, e, "g planes allocation");
  h->gbuf = (char*)buf;
  SLBM_CK(h, cudaMemsetAsync(h->gbuf, 0, bytes, h->st), "g planes clear");
  h->twopop = 1;
  h->cv = cv;
  h->tau2 = tau2;
  refresh_params(h);
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

namespace {
int gpops_io(slbm_t h, int k, double* out, const double* in) {
  if (!h->twopop) return fail(h, SLBM_EINVAL, "no two-population model on this handle");
  if ((k != 0 && k != 1) || !(out || in)) return fail(h, SLBM_EINVAL, "lattice index or buffer invalid");
  const int n = k ? h->nhi : h->nlo;
  const size_t nc = h->ncell();
  double* stage = h->at<double>(h->lay.macro[0]);
  for (int i = 0; i < n * n; ++i) {
    cudaError_t e;
    if (in) {
      if (int rc = upload(h, stage, in + (size_t)i * nc, nc * 8)) return rc;
    }
    e = h->precision == SLBM_FP64
            ? launch_pond_gio<double, double>(h->qd, k, i, (double*)h->gp(h->cur, k),
                                              (const double*)h->lam(h->cur), stage, in ? 1 : 0,
                                              h->st)
            : launch_pond_gio<float, float>(h->qf, k, i, (float*)h->gp(h->cur, k),
                                            (const float*)h->lam(h->cur), stage, in ? 1 : 0,
                                            h->st);
    SLBM_CK(h, e, "g plane launch");
    if (out)
      SLBM_CK(h, cudaMemcpyAsync(out + (size_t)i * nc, stage, nc * 8, cudaMemcpyDeviceToHost, h->st),
              "D2H copy");
    SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  }
  return SLBM_OK;
}
}  // namespace

int slbm_get_gpops(slbm_t h, int k, double* out) {
  SLBM_GUARD(h);
  return gpops_io(h, k, out, nullptr);
}

int slbm_set_gpops(slbm_t h, int k, const double* in) {
  SLBM_GUARD(h);
  if (int rc = gpops_io(h, k, nullptr, in)) return rc;
  return pond_convert_band(h, h->cur);
}

int slbm_set_pond(slbm_t h, double tol, int max_iter) {
  SLBM_GUARD(h);
  if (h->frame == SLBM_FRAME_LATTICE) return fail(h, SLBM_EINVAL, "lattice-frame handle");
  if (!(tol >= 0.0) || !std::isfinite(tol) || max_iter < 1 || max_iter > 1000)
    return fail(h, SLBM_EINVAL, "tol must be >= 0 and max_iter in 1..1000");
  h->pond_tol = tol;
  h->pond_maxit = max_iter;
  refresh_params(h);
  return SLBM_OK;
}

int slbm_get_frame(slbm_t h, double* ux, double* uy, double* T) {
  SLBM_GUARD(h);
  if (h->frame == SLBM_FRAME_LATTICE) return fail(h, SLBM_EINVAL, "lattice-frame handle");
  if (!ux || !uy || !T) return fail(h, SLBM_EINVAL, "outputs are required");
  double* d[3];
  for (int q = 0; q < 3; ++q) d[q] = h->at<double>(h->lay.macro[q]);
  cudaError_t e =
      h->precision == SLBM_FP64
          ? launch_pond_frame_io<double, double>(h->qd, (double*)h->lam(h->cur), d[0], d[1], d[2],
                                                 0, h->st)
          : launch_pond_frame_io<float, float>(h->qf, (float*)h->lam(h->cur), d[0], d[1], d[2], 0,
                                               h->st);
  SLBM_CK(h, e, "frame pack launch");
  double* out[3] = {ux, uy, T};
  for (int q = 0; q < 3; ++q)
    SLBM_CK(h, cudaMemcpyAsync(out[q], d[q], h->ncell() * 8, cudaMemcpyDeviceToHost, h->st),
            "D2H copy");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_set_frame(slbm_t h, const double* ux, const double* uy, const double* T) {
  SLBM_GUARD(h);
  if (h->frame == SLBM_FRAME_LATTICE) return fail(h, SLBM_EINVAL, "lattice-frame handle");
  if (!ux || !uy || !T) return fail(h, SLBM_EINVAL, "inputs are required");
  const size_t nc = h->ncell();
  for (size_t c = 0; c < nc; ++c) {
    if (!(T[c] > 0.0) || !std::isfinite(T[c]) || !std::isfinite(ux[c]) || !std::isfinite(uy[c]))
      return fail(h, SLBM_EINVAL, "frames must be finite with T > 0");
    if (h->frame == SLBM_FRAME_POND_ISOTHERMAL && T[c] != 1.0)
      return fail(h, SLBM_EINVAL, "the isothermal frame has T = T_L = 1");
  }
  double* d[3];
  for (int q = 0; q < 3; ++q) d[q] = h->at<double>(h->lay.macro[q]);
  const double* in[3] = {ux, uy, T};
  for (int q = 0; q < 3; ++q)
    if (int rc = upload(h, d[q], in[q], nc * 8)) return rc;
  cudaError_t e =
      h->precision == SLBM_FP64
          ? launch_pond_frame_io<double, double>(h->qd, (double*)h->lam(h->cur), d[0], d[1], d[2],
                                                 1, h->st)
          : launch_pond_frame_io<float, float>(h->qf, (float*)h->lam(h->cur), d[0], d[1], d[2], 1,
                                               h->st);
  SLBM_CK(h, e, "frame unpack launch");
  if (int rc = pond_convert_band(h, h->cur)) return rc;
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  return SLBM_OK;
}

int slbm_profile(slbm_t h, int enable) {
  SLBM_GUARD(h);
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  h->profiling = enable ? 1 : 0;
  h->ev_used = 0;
  return SLBM_OK;
}

int slbm_profile_read(slbm_t h, double* ms, long long* steps) {
  SLBM_GUARD(h);
  if (!ms || !steps) return fail(h, SLBM_EINVAL, "outputs are required");
  SLBM_CK(h, cudaStreamSynchronize(h->st), "sync");
  const int per = SLBM_PROFILE_KERNELS + 1;  // events per step
  for (int k = 0; k < SLBM_PROFILE_KERNELS; ++k) ms[k] = 0.0;
  const size_t n = h->ev_used / per;
  for (size_t s = 0; s < n; ++s)
    for (int k = 0; k < SLBM_PROFILE_KERNELS; ++k) {
      float t = 0.f;
      SLBM_CK(h, cudaEventElapsedTime(&t, h->ev_pool[s * per + k], h->ev_pool[s * per + k + 1]),
              "event time");
      ms[k] += t;
    }
  *steps = (long long)n;
  return SLBM_OK;
}

const char* slbm_last_error(slbm_t h) { return h ? h->err : g_create_err; }

}  // extern "C"

static_assert(slbm::kPondReach == SLBM_POND_REACH, "co-moving reach limit mismatch");
