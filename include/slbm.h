/*
 * slbm.h -- C ABI of the GB300 (sm_103a) multi-scale semi-Lagrangian lattice
 * Boltzmann step of Kallikounis, Dorschner & Karlin, "Multi-scale
 * semi-Lagrangian lattice Boltzmann method" (arXiv:2102.12559).
 *
 * One handle = one 2-D grid of nx x ny cells (dx = 1, T_L = 1, R = 1).  Every
 * cell carries a flag choosing the low-order lattice (flag 0) or the
 * high-order lattice (flag 1) of a Gauss-Hermite pair (Table I, eqs. ci/wi).
 * slbm_step() advances the grid: interface conversion of the populations
 * that a cell of the other lattice will read (lifting Sec. III.B / projection
 * Sec. III.C), semi-Lagrangian streaming by tensor-product Lagrange
 * reconstruction at the departure points x - c_i dt (eqs. reconstructionPond,
 * advectionPond; the three steps of Sec. III.D), and BGK collision to the
 * lattice equilibrium f^L (eq. Pond_f_equation with omega_1 = omega_2, eqs.
 * feqL / feqL0).  Optionally the flags follow the Mach refinement criterion of
 * Sec. IV.A after every step.  dt follows CFL = max|c_i| dt / dx = 1 over the
 * pair (Sec. IV); omega = 1 / tau, so the kinematic viscosity is
 * nu = (tau - 1/2) T_L dt (Sec. II.B).
 *
 * Conventions shared by every entry point:
 *  - Host field arrays are nx * ny doubles (or bytes for flags), row-major
 *    with x fastest: element (x, y) at index x + nx * y.
 *  - Population index i = ix + n * iy, with the n 1-D nodes of Table I in
 *    ascending order; a lattice value below is that n (Q = n * n).
 *  - Every call returns SLBM_OK or a negative status.  After a CUDA failure the
 *    handle is sticky-failed: later calls return SLBM_ECUDA.  No call aborts,
 *    throws or prints.  slbm_last_error() gives a message.
 *  - Calls that take host arrays copy them; the caller keeps ownership.  The
 *    handle owns its device memory (or borrows the caller's workspace, see
 *    slbm_create_in) and frees it in slbm_destroy.
 *  - slbm_step() is asynchronous on the handle's stream; calls that return
 *    host data synchronise that stream.
 *
 * The library has no CPU fallback: without a usable CUDA device slbm_create
 * fails with SLBM_ECUDA.
 */
#ifndef SLBM_H
#define SLBM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SLBM_API __attribute__((visibility("default")))
#else
#define SLBM_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct slbm_s *slbm_t;

/* Status codes. */
#define SLBM_OK          0
#define SLBM_EINVAL     -1   /* bad argument: sizes, lattice pair, tau, order, side ... */
#define SLBM_ENOMEM     -2   /* device or host allocation failed / workspace too small */
#define SLBM_ECUDA      -3   /* a CUDA call failed; the handle is now unusable */
#define SLBM_ENONFINITE -4   /* the audit found a non-finite sum, or a co-moving frame
                                became non-positive / non-finite or moved a departure
                                point beyond SLBM_POND_REACH cells (reported once) */
#define SLBM_ENOCONV    -5   /* a co-moving predictor-corrector stopped at max_iter
                                (reported once; the handle stays usable) */
#define SLBM_ETIMEOUT   -6   /* a bounded device wait ran out; the handle is now unusable */
#define SLBM_ESTATE     -7   /* call not valid in the handle's current state */

/* Lattices of Table I, by 1-D node count n: D2Q9 (n=3), D2Q16 (4), D2Q25 (5). */
#define SLBM_D2Q9  3
#define SLBM_D2Q16 4
#define SLBM_D2Q25 5

/* Reference frame of the populations (Sec. II.C).
 *  LATTICE  the fixed lattice frame {u = 0, T = T_L}: the athermal
 *           semi-Lagrangian LBM with the lattice equilibrium f^L (eq. feqL0).
 *  POND     the co-moving frame {u(x, t), T(x, t)} of every cell (eq. comoving):
 *           v_i = sqrt(T) c_i + u (eq. vi), collocation vectors carried between
 *           frames by eq. (fll), the frame found by the predictor-corrector of
 *           eqs. (correctorfieldsrho-u), collision to rho W_i (eq. feqPond).
 *           Thermal single-population model: C_v = D/2 (R = 1, D = 2), so the
 *           g population of eq. (geqPond) vanishes identically and T follows
 *           from the energy; gamma = 2.
 *  POND_ISOTHERMAL  the co-moving frame {u(x, t), T_L}: T held at T_L.
 * The co-moving frames need a periodic grid; the refinement criterion and
 * boundaries belong to the lattice frame. */
#define SLBM_FRAME_LATTICE 0
#define SLBM_FRAME_POND 1
#define SLBM_FRAME_POND_ISOTHERMAL 2

/* Largest departure distance |v_i| dt, in cells, a co-moving step accepts. */
#define SLBM_POND_REACH 5

/* Storage / arithmetic precision of the populations.  Every precision stores
 * deviations s_i = f_i - W_i from the rest state (rho_0 = 1, u = 0). */
#define SLBM_FP32 0          /* float storage, float arithmetic, FP64 conversion moments */
#define SLBM_FP64 1          /* double storage and arithmetic */
#define SLBM_FP16 2          /* half-precision storage of the deviations (half the bytes
                                per cell update), float arithmetic; lattice frame only */
#define SLBM_FX16 3          /* 16-bit companded fixed-point storage of the deviations,
                                one range A_i per population plane: plane i of a lattice
                                holds q = round(32767 sign(s_i) sqrt(|s_i| / A_i)),
                                saturating at +-32767, read back as A_i (q / 32767)^2
                                sign(q), so the step grows like sqrt|s_i|; float
                                arithmetic; lattice frame only.  slbm_init_equilibrium
                                sets A_i = max(2 max|s_i|, W_i / 4) over the initial
                                equilibria (until then W_i / 4); values written later
                                (steps, slbm_set_pops, slbm_set_state) use the ranges in
                                force */

/* Boundary kinds for a non-periodic side (ghost layer contents):
 *  OUTFLOW   zero-order extrapolation: copy of the nearest interior cell;
 *  DIRICHLET lattice equilibrium at a prescribed rho, u ("free stream");
 *  INLET     lattice equilibrium at a prescribed u and the rho of the first
 *            interior cell (fixed velocity, zero pressure gradient, Sec. IV.A);
 *  DIFFUSE   diffuse-reflection wall moving with a prescribed velocity (the
 *            kinetic wall of the Couette flow, Sec. IV.C): populations entering
 *            the fluid are the lattice equilibrium at the wall velocity, scaled
 *            so no net mass crosses the wall against the first interior cell;
 *            the others copy that cell.  The axis along the wall must be
 *            periodic.
 * A non-periodic y side takes precedence over an x side at the corners. */
#define SLBM_BC_OUTFLOW   0
#define SLBM_BC_DIRICHLET 1
#define SLBM_BC_INLET     2
#define SLBM_BC_DIFFUSE   3

/* Sides. */
#define SLBM_SIDE_XMIN 0
#define SLBM_SIDE_XMAX 1
#define SLBM_SIDE_YMIN 2
#define SLBM_SIDE_YMAX 3

/* Refinement criteria (Sec. IV.A). */
#define SLBM_CRIT_NONE 0     /* flags stay as set by slbm_set_flags */
#define SLBM_CRIT_MACH 1     /* after every step: flag = (|u| / c_s > threshold), c_s = 1 */
#define SLBM_CRIT_MLP  2     /* every `interval` steps: flag = (indicator logit > threshold),
                                the learned indicator of slbm_set_indicator */
#define SLBM_CRIT_MLP_REFINE 3  /* as SLBM_CRIT_MLP, refinement only, with a buffer: flag =
                                old flag OR (a cell within `interval` cells along x or y --
                                the distance a disturbance travels between evaluations at
                                CFL = 1 -- has logit > threshold); the buffer stops at bounded
                                sides and channel gaps.  A cell changes lattice at most once:
                                at large tau (weak collisions, high Knudsen number) cells
                                switched back and forth between the lattices every few steps
                                make the hybrid scheme diverge, while an interface that only
                                moves one way is stable */

typedef struct {
    int nx, ny;              /* cells (minimum: see slbm_create) */
    int periodic_x;          /* 1 = periodic along x, 0 = boundary sides XMIN/XMAX */
    int periodic_y;          /* 1 = periodic along y, 0 = boundary sides YMIN/YMAX */
} slbm_grid;

typedef struct {
    double dt;               /* time step, CFL / max|c| over the pair */
    double omega;            /* 1 / tau */
    int q_lo, q_hi;          /* Q of the two lattices */
    int halo;                /* ghost-layer width in cells */
    int pitch;               /* row pitch of a population plane, in elements */
    int rows;                /* rows of a population plane including ghosts */
    int precision;
    int kernels_per_step;    /* kernel launches slbm_step issues per time step */
    size_t workspace_bytes;
    long long steps;         /* time steps taken so far */
} slbm_info_t;

/* Device bytes a handle needs for this configuration (the workspace of
 * slbm_create_in).  Arguments as for slbm_create. */
SLBM_API int slbm_workspace_bytes(const slbm_grid *g, int lat_lo, int lat_hi, int interp_order,
                         int precision, size_t *bytes);

/* Create a handle.  lat_lo < lat_hi are SLBM_D2Q* values; tau > 1/2 is the
 * relaxation time in units of dt (omega = 1/tau, Sec. II.B); interp_order in
 * 1..5 is the Lagrange order (order + 1 collocation points per axis; 3 =
 * the paper's third-order polynomials, Sec. II.C); frame an SLBM_FRAME_*
 * value; precision SLBM_FP32 or SLBM_FP64; cuda_stream is a
 * cudaStream_t (NULL = the legacy default stream).  The handle allocates its
 * own device workspace.  Populations start at rest (rho = 1, u = 0), flags 0,
 * criterion none, every non-periodic side OUTFLOW.  SLBM_EINVAL for bad
 * arguments, among them a grid narrower than 2 G + 1 cells per side (G = the
 * stencil reach; G along a periodic side in the lattice frame) and, in the
 * lattice frame, a periodic axis whose last
 * partial 32 x 8 tile is narrower than G (nx % 32 and ny % 8 must be 0 or at
 * least G). */
SLBM_API int slbm_create(const slbm_grid *g, int lat_lo, int lat_hi, double tau, int interp_order,
                int frame, int precision, void *cuda_stream, slbm_t *out);

/* Same, but the device workspace is the caller's: `workspace` is a device
 * pointer aligned to 256 bytes with at least slbm_workspace_bytes() bytes,
 * which must outlive the handle.  The handle never frees it. */
SLBM_API int slbm_create_in(const slbm_grid *g, int lat_lo, int lat_hi, double tau, int interp_order,
                   int frame, int precision, void *cuda_stream, void *workspace,
                   size_t workspace_bytes, slbm_t *out);

/* Synchronise, release device memory the handle owns, free the handle. */
SLBM_API int slbm_destroy(slbm_t h);

SLBM_API int slbm_get_info(slbm_t h, slbm_info_t *info);

/* Set every cell to the equilibrium of BOTH lattices; flags are kept.
 * Lattice frame: f^L(rho, u) (eq. feqL0), T must be NULL (athermal model).
 * Co-moving frames: rho W_i in the frame {u, T} (eq. feqPond); T (host, > 0)
 * only for SLBM_FRAME_POND, NULL = T_L.  rho, ux, uy: host, nx*ny each. */
SLBM_API int slbm_init_equilibrium(slbm_t h, const double *rho, const double *ux, const double *uy,
                          const double *T);

/* Set the flags (host, nx*ny bytes, 0 = lat_lo, nonzero = lat_hi).  Cells whose
 * flag changes have their populations lifted or projected (Sec. III.B-C). */
SLBM_API int slbm_set_flags(slbm_t h, const uint8_t *flags);
SLBM_API int slbm_get_flags(slbm_t h, uint8_t *flags);

/* Refinement criterion (SLBM_CRIT_*).  SLBM_CRIT_MACH: threshold on the Mach
 * number |u| / c_s, c_s = sqrt(T_L) = 1, applied at once to the current state
 * (flips lifted / projected, asynchronous) and after every step.
 * SLBM_CRIT_MLP / SLBM_CRIT_MLP_REFINE: threshold on the learned indicator's
 * logit (0 = probability 1/2), applied at once and every `interval` steps;
 * needs slbm_set_indicator.
 * Lattice frame only (SLBM_EINVAL otherwise). */
SLBM_API int slbm_set_criterion(slbm_t h, int kind, double threshold);

/* Learned refinement indicator (lattice frame).  Not in the paper, which
 * refines by plain Mach / Knudsen criteria (Sec. IV); the indicator is a small
 * MLP trained to reproduce such a criterion from local moments and their
 * gradients, with the plain criterion as its fallback (SLBM_CRIT_MACH) and
 * the reference its error is measured against.  Per cell, 16 features, each
 * times a fixed scale:
 *   rho - 1 (x10), u_x, u_y (x3), T - 1 (x10, kinetic T), the non-equilibrium
 *   stress sum c_a c_b (f - f^L) for xx, xy, yy (x100), the non-equilibrium
 *   energy flux 1/2 sum c_a |c|^2 (f - f^L) for x, y (x100), the central
 *   differences d/dx, d/dy of rho, u_x, u_y (x100; periodic wrap, else the edge
 *   cell repeated), |u| (x3) -- all from the cell's own lattice.
 * Network: h1 = relu(x W1 + b1) (W1 16 x 32), h2 = relu(h1 W2 + b2) (W2 32 x 32),
 * logit = h2 . w3 + b3; W1, W2 row-major (input index first), stored in FP16,
 * inputs rounded to FP16, accumulation in FP32 (tensor cores).
 * slbm_set_indicator copies the weights (host floats) to device memory it
 * allocates and owns; `interval` >= 1 is the step interval at which
 * SLBM_CRIT_MLP re-evaluates the flags.
 * slbm_indicator_eval: features (nx*ny x 16 floats, cell-major), logits
 * (nx*ny floats) and flags (logit > the criterion threshold, 0 unless set)
 * of the current state to host arrays; any may be NULL (logits / flags need
 * weights).  Synchronises; allocates temporary device memory. */
SLBM_API int slbm_set_indicator(slbm_t h, const float *w1, const float *b1, const float *w2,
                                const float *b2, const float *w3, float b3, int interval);
SLBM_API int slbm_indicator_eval(slbm_t h, float *features, float *logits, uint8_t *flags);

/* Per-cell lattice loss: what the low-order lattice loses in one step, the
 * indicator's training label (Sec. III.B-D).  From a lattice-frame state in
 * which every cell is high-order (flags 1; gap columns between channels
 * allowed) and fixed flags (SLBM_CRIT_NONE), two steps are taken from the same
 * start: a = one step of the all-high-order state, b = the lift (Sec. III.B)
 * of one step of its projection (Sec. III.C, every cell low-order).  Output,
 * per cell (host, nx*ny doubles, x + nx*y):
 *   loss = || a - b ||_2 / rho_a   (norm over the high-order populations),
 * 0 in gap cells.  The handle ends at a, one step advanced (the step counter
 * counts one).  Nothing is lost by a uniform flow at any Mach number, nor by
 * the raw moments m_ab (a, b < n_lo) the low-order lattice carries; the loss
 * holds the non-equilibrium of the higher raw moments (Knudsen layers) and
 * what the low-order lattice's aliased fluxes (c^3 = 3c on D2Q9's nodes) get
 * wrong at high Mach number.  Allocates two population-sized temporaries;
 * synchronises.  SLBM_EINVAL: not lattice frame, a criterion is on, or a
 * non-gap cell is low-order. */
SLBM_API int slbm_lattice_loss(slbm_t h, double *loss);

/* Training of the indicator: mini-batch Adam on the mean logistic loss
 * log(1 + exp(-s z)), s = 2y - 1, of the network above, on the GPU (one
 * thread block runs every step: forward pass, back-propagation and the Adam
 * update).  Not tied to a handle; runs on the current CUDA device.
 *   x: n x 16 features (host floats, row-major, as slbm_indicator_eval
 *      returns them), y: n labels, each 0 or 1;
 *   idx: steps x batch sample indices in [0, n) (host ints, the rows of step s
 *      at idx[s * batch ...]): the mini-batches, drawn by the caller;
 *   batch: 128, 256, 384 or 512;
 *   hyper = {lr, beta1, beta2, eps}: lr > 0, 0 <= beta < 1, eps > 0;
 *   t0: Adam steps already taken (step s uses the bias corrections of
 *      t0 + s + 1);
 *   params: the 1633 parameters W1 (16 x 32 row-major, input index first),
 *      b1 (32), W2 (32 x 32), b2 (32), w3 (32), b3 (1), host floats, in / out;
 *   adam: first then second moments (2 x 1633 host floats, zeros to start),
 *      in / out;
 *   loss: the mean loss of every step's batch before its update (steps
 *      floats, or NULL); grad: the last step's gradient (1633 floats, or NULL).
 * Precision: features, W1, W2, the hidden activations and their gradients
 * rounded to FP16, products accumulated in FP32 on the tensor cores; biases,
 * the output layer, the master weights and Adam in FP32.  cuda_stream: a
 * cudaStream_t, or NULL.  Allocates and frees device memory; synchronises
 * the stream.  SLBM_EINVAL on any invalid argument (checked before any device
 * work), SLBM_ENOMEM, SLBM_ECUDA. */
SLBM_API int slbm_mlp_train(const float *x, const float *y, long long n, const int *idx, int steps,
                            int batch, const double hyper[4], int t0, float *params, float *adam,
                            float *loss, float *grad, void *cuda_stream);

/* Boundary of a non-periodic side.  Arrays run along the side (ny entries
 * for XMIN/XMAX, nx for YMIN/YMAX), host doubles, copied: DIRICHLET needs
 * rho, ux, uy; INLET and DIFFUSE need ux, uy (rho NULL); OUTFLOW needs none. */
SLBM_API int slbm_set_boundary(slbm_t h, int side, int kind, const double *rho, const double *ux,
                      const double *uy);

/* Advance n >= 0 time steps (asynchronous).  Per lattice-frame step: the
 * stream-collide kernel, then the post-step kernel (interface conversions and
 * the ghost ring).  Once the kernels have run directly, runs of 16 (then 2)
 * steps are replayed as CUDA graphs captured on a private stream; n = 1,
 * traced steps and a refused capture launch directly, with bit-identical
 * results.  A learned indicator, or a Knudsen criterion evaluated less often
 * than every step, splits the steps into chunks between its evaluations; a
 * Knudsen criterion every step is recorded in the replays with its step. */
SLBM_API int slbm_step(slbm_t h, int n);
/* The post-step kernel runs one warp per 32 x 8 tile on grids of 8192 tiles
 * and more, one thread block per tile below (a small grid's few tiles each
 * end in one dependent chain, which a block shortens); the environment
 * variable SLBM_POST_KERNEL = "warp" or "block", read by slbm_create, forces
 * one of them (results are the same). */

/* Wait for the handle's stream. */
SLBM_API int slbm_sync(slbm_t h);

/* rho, u and the kinetic temperature T = (sum v^2 f / rho - u^2) / 2 of every
 * cell from its own lattice's populations (Sec. II.B), with the particle
 * velocities v_i of the frame the populations live in.  Host outputs of nx*ny
 * doubles; any pointer may be NULL.  Synchronises; returns a pending
 * SLBM_ENOCONV / SLBM_ENONFINITE report of the co-moving frame. */
SLBM_API int slbm_moments(slbm_t h, double *rho, double *ux, double *uy, double *T);

/* Same into device arrays of nx*ny doubles (asynchronous; NULL skips). */
SLBM_API int slbm_moments_device(slbm_t h, double *rho, double *ux, double *uy, double *T);

/* FP64 global sums over all cells: out = {sum rho, sum rho u_x, sum rho u_y,
 * sum rho E}, rho E = sum v^2/2 f (v_i of each cell's frame).  Returns
 * SLBM_ENONFINITE if any is not finite.  Synchronises. */
SLBM_API int slbm_audit(slbm_t h, double out[4]);

/* Populations of lattice k (0 = lat_lo, 1 = lat_hi) of every cell, host
 * doubles, plane-major: out[i * nx * ny + x + nx * y].  Only cells whose
 * flag is k (plus interface cells) hold meaningful values.  Synchronises. */
SLBM_API int slbm_get_pops(slbm_t h, int k, double *out);

/* Overwrite the populations of lattice k (same layout).  Afterwards the
 * interface cells' other-lattice populations are recomputed from each cell's
 * own lattice (lift / project), as after a step. */
SLBM_API int slbm_set_pops(slbm_t h, int k, const double *in);

/* Snapshot / restore the full state (populations of both lattices, flags,
 * co-moving frames, step count) in a host buffer.  Call with buf = NULL to get
 * the size. */
SLBM_API int slbm_get_state(slbm_t h, void *buf, size_t *bytes);
SLBM_API int slbm_set_state(slbm_t h, const void *buf, size_t bytes);

/* Co-moving frames only (SLBM_EINVAL for a lattice-frame handle).
 *
 * slbm_set_pond: predictor-corrector controls (Sec. II.C): a cell update
 * repeats the reconstruction until the frame it produces differs from the one
 * used by at most tol in every one of u_x, u_y, T, or max_iter (1..1000)
 * reconstructions were made; the last reconstruction's populations and frame
 * are kept.  Defaults: tol 1e-12 (FP64) / 2e-6 (FP32), max_iter 20.
 *
 * slbm_get_frame / slbm_set_frame: the frame {u_x, u_y, T} each cell's
 * populations live in, host nx*ny doubles each (T > 0; T = 1 for the
 * isothermal frame).  Setting frames reinterprets the stored populations; set
 * the frames before slbm_set_pops when writing a state. */
SLBM_API int slbm_set_pond(slbm_t h, double tol, int max_iter);
SLBM_API int slbm_get_frame(slbm_t h, double *ux, double *uy, double *T);
SLBM_API int slbm_set_frame(slbm_t h, const double *ux, const double *uy, const double *T);

/* Two-population co-moving model (Sec. II.B, eqs. Pond_f_equation and
 * Pond_g_equation; SLBM_FRAME_POND handles only, else SLBM_EINVAL).
 *
 * slbm_set_twopop: switch the thermal co-moving model to f and g populations
 * with specific heat C_v = cv > 0 (R = 1, so gamma = (cv + 1) / cv and
 * C_v = 1 with g = 0 is the single-population model) and the second
 * relaxation time tau2 > 1/2 (omega_2 = 1 / tau2 relaxes the quasi-equilibria
 * of eqs. fqeq / gqeq, so the Prandtl number is (tau - 1/2) / (tau2 - 1/2)).
 * Allocates device memory for the g planes of both lattices and buffers
 * (owned by the handle, freed by slbm_destroy); once per handle, before
 * slbm_init_equilibrium, which then sets g = (C_v - 1) T rho W_i (eq. geqPond)
 * in each cell's frame.  T from slbm_moments and the energy of slbm_audit
 * include the g populations.  slbm_get_state / slbm_set_state do not carry
 * the g planes.
 *
 * slbm_get_gpops / slbm_set_gpops: the g populations of lattice k in the
 * frame each cell's populations live in, absolute units, host doubles in the
 * layout of slbm_get_pops (plane-major: g_i of cell c at [i * nx*ny + c]).
 * Writing recomputes the interface cells' other lattice, as slbm_set_pops. */
SLBM_API int slbm_set_twopop(slbm_t h, double cv, double tau2);
SLBM_API int slbm_get_gpops(slbm_t h, int k, double *out);
SLBM_API int slbm_set_gpops(slbm_t h, int k, const double *in);

/* Batched quasi-one-dimensional instances (the shock structure problem of
 * Sec. IV.C; co-moving frames only).
 *
 * slbm_set_rows: every row y of the grid becomes an independent instance,
 * uniform across y (its y interpolation is the identity), with len[y] active
 * cells (interp_order + 1 <= len[y] <= nx; cells beyond are left alone) and
 * fixed end states beyond x < 0 and x >= len[y]: ends[8 y .. 8 y + 3] =
 * {rho, u_x, u_y, T} on the left, ends[8 y + 4 .. 8 y + 7] on the right, each
 * at rest in its own frame (f = rho W_i, g = (C_v - 1) T rho W_i).  Host
 * arrays, copied.  The interface conversions and the step treat each row on
 * its own.  One launch per step advances all rows.
 *
 * slbm_set_viscosity_law: two-population model only.  Per row y the dynamic
 * viscosity mu = mu1[y] (T / T1[y])^s_exp (s_exp = 1/2 for hard spheres) sets
 * omega_1 at every cell update from mu = (1/omega_1 - 1/2) rho T dt at the
 * reconstructed rho and T, and omega_2 from the fixed Prandtl number pr
 * (1/omega_2 - 1/2 = (1/omega_1 - 1/2) / pr).  Host arrays of ny doubles. */
SLBM_API int slbm_set_rows(slbm_t h, const int *len, const double *ends);

/* Batched channels (the micro-Couette problem of Sec. IV.C with many
 * channels advanced together; lattice frame only).
 *
 * slbm_set_channels: the grid becomes n independent channels side by side
 * along x, each bounded by diffuse-reflection walls (as SLBM_BC_DIFFUSE) on
 * its two x sides and periodic along y (the grid's y axis must be periodic,
 * so every channel shares the streamwise period ny).  Channel c holds the
 * columns x0[c] .. x0[c] + width[c] - 1 with width[c] >= 2 G + 1 (G = the
 * stencil reach, slbm_info_t.halo); its wall at the low x side moves along y
 * at uw_lo[c], the one at the high x side at uw_hi[c]; its relaxation time is
 * tau[c] > 1/2 (the handle's tau applies nowhere inside a channel).  x0[0] >= G,
 * x0[c] >= x0[c - 1] + width[c - 1] + 2 G, and x0[n - 1] + width[n - 1] + G <= nx:
 * the G columns beside each channel side hold that wall's ghost cells (the
 * diffuse-wall state against the channel's edge cell of the same row,
 * refreshed after every step by the post-step kernel), and the columns that
 * belong to no channel are gaps: no fluid, never computed, flags reported as
 * 2, moments 0, outside the audit.  Every channel cell starts in the
 * low-order lattice; slbm_set_flags then chooses each cell's lattice (the
 * gaps stay gaps).  The flags stay fixed (SLBM_CRIT_NONE) or follow the
 * learned indicator (SLBM_CRIT_MLP); the Mach criterion is refused.  Host
 * arrays, copied; allocates a device buffer owned by the handle (freed by
 * slbm_destroy); once per handle.  One stream-collide and one post-step
 * launch per step advance every channel.  SLBM_EINVAL for bad arguments,
 * SLBM_ESTATE if channels are already set.  slbm_get_state / slbm_set_state
 * carry populations and flags, not the channel description. */
SLBM_API int slbm_set_channels(slbm_t h, int n, const int *x0, const int *width,
                               const double *uw_lo, const double *uw_hi, const double *tau);

/* Autotuner of the co-moving step kernel (co-moving frames only): times
 * `reps` launches of the step for each thread-block shape of 256 threads
 * (32 x 8, 64 x 4, 128 x 2, 256 x 1, 16 x 16) on the current state -- the
 * kernel reads one buffer and writes the other, so the state is unchanged --
 * and keeps the fastest; its shape to *bx, *by (either may be NULL).
 * Synchronises. */
SLBM_API int slbm_tune(slbm_t h, int reps, int *bx, int *by);
SLBM_API int slbm_set_viscosity_law(slbm_t h, const double *mu1, const double *T1, double s_exp,
                                    double pr);

/* Knudsen refinement criterion of Sec. IV.C on batched rows (needs slbm_set_rows,
 * slbm_set_twopop and slbm_set_viscosity_law): a cell is high-order iff
 * Kn = lambda |d rho / dx| / rho > thr, with central differences (the end
 * states' density beyond the ends) and the local hard-sphere mean free path
 * lambda = 16 / (5 sqrt(2 pi gamma)) mu a / p (mu from the row's law,
 * a = sqrt(gamma T), p = rho T, gamma = (C_v + 1) / C_v).  Applied at once and
 * after every `interval` steps of slbm_step, refinement only (a cell once
 * high-order stays so: Sec. IV.C initialises the shock on the low-order lattice
 * and refines it; cells switched back and forth at the shock's edges make the
 * nearly collisionless hybrid lose positivity); refined cells are lifted as
 * by slbm_set_flags. */
SLBM_API int slbm_set_kn_criterion(slbm_t h, double thr, int interval);

/* Per-kernel timing (tracing).  slbm_profile(h, 1) clears previous records
 * and starts bracketing every kernel slbm_step launches with CUDA events on
 * the handle's stream; slbm_profile(h, 0) stops.  slbm_profile_read()
 * synchronises and returns, per kernel of the step sequence (index 0 =
 * stream-collide, 1 = post-step: interface conversion and, in the lattice
 * frame, the ghost-ring refresh), the summed device milliseconds over the
 * recorded steps, and the number of recorded steps.  ms must hold
 * SLBM_PROFILE_KERNELS doubles. */
#define SLBM_PROFILE_KERNELS 2
SLBM_API int slbm_profile(slbm_t h, int enable);
SLBM_API int slbm_profile_read(slbm_t h, double *ms, long long *steps);

/* FP64 conservation sums of a dense population field without allocating
 * anything (no cudaMalloc, cudaFree or allocating library call).  For callers
 * that cannot allocate device memory: code running inside a CUDA stream
 * capture (an allocation there would break the capture), hard real-time
 * loops that only use memory reserved in advance, and frameworks that own all
 * device memory.  The paper has no counterpart; this is a service entry point.
 *   f:       device, FP32 full populations f_i (not deviations) of lattice
 *            `lattice` (an SLBM_D2Q* value n, Q = n*n), plane-major:
 *            f[i * nx * ny + x + nx * y].
 *   out:     device, 4 doubles: sum rho, sum rho u_x, sum rho u_y, sum rho E
 *            with rho E = sum |c_i|^2 / 2 f_i (the slbm_audit quantities).
 *   cuda_stream: cudaStream_t (NULL = legacy default stream); asynchronous.
 * The reduction's scratch is a static device array in this library of
 * SLBM_NOALLOC_MAX_BLOCKS x 4 doubles (32 KiB), held by every GPU that loads
 * the library until the process exits.  Every call overwrites the entries it
 * uses before reading them; all calls share the array, so calls that overlap
 * on the GPU (different streams or threads without ordering) race.
 * nx * ny must not exceed SLBM_NOALLOC_MAX_CELLS (SLBM_EINVAL otherwise).
 * The first call on a device (with that device current) looks up the
 * array's device address with cudaGetSymbolAddress; make that first call
 * before any stream capture.  A failed lookup is not cached (the next call
 * retries it) and its error is cleared; an error the caller left in the
 * runtime's last-error state is neither reported nor cleared (only this
 * call's own launches are checked).  Returns SLBM_OK, SLBM_EINVAL or
 * SLBM_ECUDA. */
#define SLBM_NOALLOC_MAX_BLOCKS 1024
#define SLBM_NOALLOC_MAX_CELLS (1LL << 30)
SLBM_API int slbm_audit_dense_noalloc(const float *f, int lattice, int nx, int ny, double *out,
                                      void *cuda_stream);

/* Message of the last failure on this handle ("" if none); h may be NULL for
 * the last creation failure of the calling thread. */
SLBM_API const char *slbm_last_error(slbm_t h);

#ifdef __cplusplus
}
#endif

#endif /* SLBM_H */
