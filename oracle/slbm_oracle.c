/*
 * slbm_oracle.c -- plain, slow FP64 CPU oracle of the multi-scale
 * semi-Lagrangian lattice Boltzmann step of Kallikounis, Dorschner & Karlin,
 * "Multi-scale semi-Lagrangian lattice Boltzmann method" (arXiv:2102.12559).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark load this library.  It shares no code,
 * header, table or constant with the CUDA path; it is its independent checker.
 *
 * It runs the method's steps in the paper's order and notation:
 *   - Table I: 1-D Gauss-Hermite abscissae and weights, T_L = 1.
 *   - Eq. (ci), (wi): tensor-product velocity sets D2Q9 / D2Q16 / D2Q25.
 *   - Eq. (vi), (momf), (momfshort): the full Q x Q moment matrix M_lambda of a
 *     frame lambda = {u, T}, with v_i = sqrt(theta) c_i + u, theta = T / T_L.
 *   - Eq. (fll) and the transfer matrix G = M_lambda'^{-1} M_lambda, inverted by
 *     generic Gauss-Jordan elimination (no Kronecker or Lagrange shortcut).
 *   - Eq. (feqPond), (feqL0): co-moving equilibrium rho W_i and the lattice
 *     equilibrium f^L = G_{u,T_L}^{0,T_L} f^eq.
 *   - Sec. III.B / App. C: lifting f_q -> f_Q (keep the q x q moments, fill the
 *     rest from the Q-lattice equilibrium, invert M_Q).
 *   - Sec. III.C / App. C: projection f_Q -> f_q (first q x q moments, invert M_q).
 *   - Eq. (reconstructionPond), (advectionPond) and the three steps of Sec. III.D:
 *     departure point, lattice conversion of every collocation node whose
 *     lattice differs from the target's (memoised, so each node is converted
 *     at most once per step as the paper prescribes), Lagrange reconstruction.
 *   - Eq. (Pond_f_equation) with omega_1 = omega_2: BGK relaxation to the
 *     lattice equilibrium.
 *   - The Mach refinement criterion of Sec. IV.A (threshold on |u| / c_s).
 *   - The co-moving (PonD) frame of Sec. II.C: every node keeps its populations
 *     in its own frame lambda = {u, T}; a cell reconstructs each population at
 *     x - v_i dt with v_i = sqrt(theta) c_i + u of its current frame guess,
 *     after carrying every collocation node's vector into that frame by
 *     eq. (fll); the predictor-corrector of eqs. (correctorfieldsrho-u)
 *     replaces the guess by the reconstructed moments until they agree.
 *     Two variants: thermal (single f population, C_v = D/2 so the g
 *     population of eq. (geqPond) vanishes identically) and isothermal
 *     (T held at T_L).
 *   - The two-population co-moving model of Sec. II.B (orc_set_twopop): f
 *     and g populations (eqs. Pond_f_equation, Pond_g_equation) with C_v
 *     free (gamma = (C_v + 1) / C_v), the equilibria of eqs. (feqPond,
 *     geqPond), the quasi-equilibria of eqs. (fqeq, gqeq) built from the
 *     non-equilibrium third-order tensor and heat flux, relaxation omega_1
 *     towards the equilibria and omega_1 - omega_2 of the quasi-equilibrium
 *     correction; the total energy of eq. (E) with the g populations in the
 *     predictor-corrector of eqs. (correctorfieldsrho-u); g transferred,
 *     reconstructed (eq. reconstructionPondg), lifted and projected as f
 *     (Sec. III.C), its lift completed by g^eq at the node's rho, u, T.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - "third-order Lagrange polynomials": p = order + 1 collocation points per
 *     axis; first node floor(x_dep - (p-1)/2 + 1/2), ties rounding up.
 *   - A per-axis shift within 1e-12 of an integer snaps to it.
 *   - dt = CFL / max|c| over both lattices of the pair (CFL = 1, Sec. IV).
 *   - omega = 1 / tau, so nu = (tau - 1/2) T_L dt.
 *   - The equilibrium that completes a lifted moment vector is the Q-lattice
 *     equilibrium at the cell's own rho, u (and T = T_L for the athermal model)
 *     expressed in the frame the populations live in.
 *   - Boundary ghost nodes hold the boundary state in whichever lattice reads
 *     them: DIRICHLET = equilibrium at a fixed rho, u; INLET = fixed u with rho
 *     copied from the first interior node; OUTFLOW = copy of the nearest
 *     interior node; DIFFUSE = diffuse-reflection wall (populations entering
 *     the fluid at the wall-velocity equilibrium with zero net normal mass
 *     flux against the first interior node, the others copied from it).  A
 *     non-periodic y side takes precedence at corners.
 *   - Co-moving frame: no snapping of departure points; the iteration stops
 *     when max(|du_x|, |du_y|, |dT|) <= tol between the frame used and the
 *     moments it produced, or after maxit reconstructions; the populations
 *     and frame kept are those of the last reconstruction.  Collision relaxes
 *     towards the equilibrium at the reconstructed rho, u, T expressed in
 *     that frame (rho W_i itself once converged, eq. feqPond), so the
 *     collision conserves rho, rho u (and rho E when thermal) exactly.
 *     Lifting in a node's frame completes the moments with the equilibrium
 *     at the node vector's own rho, u, T (T_L when isothermal).
 *   - Two-population model: the quasi-equilibria are formed in the co-moving
 *     frame {u, T} of the reconstructed moments (theta = T, R = T_L = 1) with
 *     the tensors taken from the populations in the frame used, and carried
 *     into that frame by the transfer matrix, like the equilibria.
 *
 * Data layout (private to this file): populations of one cell contiguous,
 * f[k][cell * Q_k + i], cell = x + nx * y, i = ix + n * iy with the 1-D nodes
 * in ascending order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 5
#define ORC_MAXQ 25

typedef struct {
    int n, Q;
    double c[ORC_MAXN], w[ORC_MAXN];      /* 1-D nodes / weights, Table I */
    double cx[ORC_MAXQ], cy[ORC_MAXQ];    /* 2-D velocities, eq. (ci)     */
    double W[ORC_MAXQ];                   /* 2-D weights, eq. (wi)        */
} olat;

/* ---------------------------------------------------------------- Table I */

/* 1-D Gauss-Hermite abscissae and weights with T_L = 1, Table I, nodes in
 * ascending order.  Returns 0, or -1 for an unsupported n. */
int orc_gh1d(int n, double *c, double *w)
{
    if (n == 3) {               /* D1Q3: 0, +-sqrt(3); 2/3, 1/6 */
        double a = sqrt(3.0);
        c[0] = -a;  c[1] = 0.0; c[2] = a;
        w[0] = 1.0 / 6.0; w[1] = 2.0 / 3.0; w[2] = 1.0 / 6.0;
        return 0;
    }
    if (n == 4) {               /* D1Q4: +-sqrt(3 -+ sqrt 6); (3 +- sqrt 6)/12 */
        double s6 = sqrt(6.0);
        double a = sqrt(3.0 - s6), b = sqrt(3.0 + s6);
        c[0] = -b; c[1] = -a; c[2] = a; c[3] = b;
        w[0] = (3.0 - s6) / 12.0; w[1] = (3.0 + s6) / 12.0;
        w[2] = (3.0 + s6) / 12.0; w[3] = (3.0 - s6) / 12.0;
        return 0;
    }
    if (n == 5) {               /* D1Q5: 0, +-sqrt(5 -+ sqrt 10); 8/15, (7 +- 2 sqrt 10)/60 */
        double s10 = sqrt(10.0);
        double a = sqrt(5.0 - s10), b = sqrt(5.0 + s10);
        c[0] = -b; c[1] = -a; c[2] = 0.0; c[3] = a; c[4] = b;
        w[0] = (7.0 - 2.0 * s10) / 60.0; w[1] = (7.0 + 2.0 * s10) / 60.0;
        w[2] = 8.0 / 15.0;
        w[3] = (7.0 + 2.0 * s10) / 60.0; w[4] = (7.0 - 2.0 * s10) / 60.0;
        return 0;
    }
    return -1;
}

static int make_lattice(int n, olat *L)
{
    if (orc_gh1d(n, L->c, L->w)) return -1;
    L->n = n;
    L->Q = n * n;
    for (int iy = 0; iy < n; ++iy)
        for (int ix = 0; ix < n; ++ix) {
            int i = ix + n * iy;
            L->cx[i] = L->c[ix];
            L->cy[i] = L->c[iy];
            L->W[i] = L->w[ix] * L->w[iy];      /* eq. (wi) */
        }
    return 0;
}

/* 2-D tensor-product velocity set, eq. (ci)/(wi).  i = ix + n * iy. */
int orc_lattice(int n, double *cx, double *cy, double *W)
{
    olat L;
    if (make_lattice(n, &L)) return -1;
    memcpy(cx, L.cx, sizeof(double) * L.Q);
    memcpy(cy, L.cy, sizeof(double) * L.Q);
    memcpy(W, L.W, sizeof(double) * L.Q);
    return 0;
}

/* ------------------------------------------------------- linear algebra */

static double ipow(double x, int m)
{
    double r = 1.0;
    for (int k = 0; k < m; ++k) r *= x;
    return r;
}

/* Generic Gauss-Jordan inversion with partial pivoting, N x N row-major.
 * Returns 0, or -1 when a pivot vanishes. */
int orc_invert(int N, const double *A, double *Ainv)
{
    double *a = (double *)malloc(sizeof(double) * N * 2 * N);
    if (!a) return -1;
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < 2 * N; ++c)
            a[r * 2 * N + c] = c < N ? A[r * N + c] : (c - N == r ? 1.0 : 0.0);
    for (int col = 0; col < N; ++col) {
        int piv = col;
        double best = fabs(a[col * 2 * N + col]);
        for (int r = col + 1; r < N; ++r)
            if (fabs(a[r * 2 * N + col]) > best) { best = fabs(a[r * 2 * N + col]); piv = r; }
        if (best == 0.0) { free(a); return -1; }
        if (piv != col)
            for (int c = 0; c < 2 * N; ++c) {
                double t = a[col * 2 * N + c];
                a[col * 2 * N + c] = a[piv * 2 * N + c];
                a[piv * 2 * N + c] = t;
            }
        double d = a[col * 2 * N + col];
        for (int c = 0; c < 2 * N; ++c) a[col * 2 * N + c] /= d;
        for (int r = 0; r < N; ++r) {
            if (r == col) continue;
            double m = a[r * 2 * N + col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * N; ++c) a[r * 2 * N + c] -= m * a[col * 2 * N + c];
        }
    }
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) Ainv[r * N + c] = a[r * 2 * N + N + c];
    free(a);
    return 0;
}

static void matvec(int N, const double *A, const double *x, double *y)
{
    for (int r = 0; r < N; ++r) {
        double s = 0.0;
        for (int c = 0; c < N; ++c) s += A[r * N + c] * x[c];
        y[r] = s;
    }
}

/* ------------------------------------------------ moments and frames */

/* Moment matrix of eq. (momf): row r <-> exponents (a, b) = (r % n, r / n),
 * column i <-> population i; entry (sqrt(theta) c_ix + u_x)^a (sqrt(theta)
 * c_iy + u_y)^b with theta = T / T_L, T_L = 1, R = 1 (eq. theta, vi).
 * lam = {u_x, u_y, T}. */
static void moment_matrix(const olat *L, const double lam[3], double *M)
{
    double st = sqrt(lam[2]);
    for (int r = 0; r < L->Q; ++r) {
        int a = r % L->n, b = r / L->n;
        for (int i = 0; i < L->Q; ++i)
            M[r * L->Q + i] = ipow(st * L->cx[i] + lam[0], a) * ipow(st * L->cy[i] + lam[1], b);
    }
}

int orc_moment_matrix(int n, const double lam[3], double *M)
{
    olat L;
    if (make_lattice(n, &L)) return -1;
    moment_matrix(&L, lam, M);
    return 0;
}

/* G = Mti M_from, with Mti = M_to^{-1} already formed. */
static void transfer_inv(const olat *L, const double from[3], const double *Mti, double *G)
{
    int Q = L->Q;
    double Mf[ORC_MAXQ * ORC_MAXQ];
    moment_matrix(L, from, Mf);
    for (int r = 0; r < Q; ++r)
        for (int c = 0; c < Q; ++c) {
            double s = 0.0;
            for (int k = 0; k < Q; ++k) s += Mti[r * Q + k] * Mf[k * Q + c];
            G[r * Q + c] = s;
        }
}

/* Transfer matrix G_lambda^lambda' = M_lambda'^{-1} M_lambda, eq. (fll). */
static int transfer(const olat *L, const double from[3], const double to[3], double *G)
{
    double Mt[ORC_MAXQ * ORC_MAXQ], Mti[ORC_MAXQ * ORC_MAXQ];
    moment_matrix(L, to, Mt);
    if (orc_invert(L->Q, Mt, Mti)) return -1;
    transfer_inv(L, from, Mti, G);
    return 0;
}

int orc_transfer(int n, const double from[3], const double to[3], double *G)
{
    olat L;
    if (make_lattice(n, &L)) return -1;
    return transfer(&L, from, to, G);
}

/* Co-moving equilibrium f^eq_i = rho W_i, eq. (feqPond), carried into the
 * frame lam by the transfer matrix: G_{u,T}^{lam} f^eq.  With lam = lattice
 * frame {0, T_L} this is f^L of eq. (feqL); with T = T_L it is eq. (feqL0). */
static int feq_in_frame(const olat *L, double rho, double ux, double uy, double T,
                        const double lam[3], double *f)
{
    double G[ORC_MAXQ * ORC_MAXQ], feq[ORC_MAXQ];
    double own[3] = {ux, uy, T};
    for (int i = 0; i < L->Q; ++i) feq[i] = rho * L->W[i];
    if (transfer(L, own, lam, G)) return -1;
    matvec(L->Q, G, feq, f);
    return 0;
}

/* Lattice-frame equilibrium f^L (eq. feqL / feqL0). */
int orc_eq_lattice(int n, double rho, double ux, double uy, double T, double *f)
{
    olat L;
    double lat[3] = {0.0, 0.0, 1.0};
    if (make_lattice(n, &L)) return -1;
    return feq_in_frame(&L, rho, ux, uy, T, lat, f);
}

/* rho, u and the kinetic temperature of a population vector living in frame
 * lam (conservation laws of Sec. II.B; T from sum v^2/2 f = rho u^2/2 + rho T,
 * i.e. C_v = D/2 for the single population, D = 2). */
static void macro(const olat *L, const double lam[3], const double *f,
                  double *rho, double *ux, double *uy, double *T)
{
    double st = sqrt(lam[2]);
    double r = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double vx = st * L->cx[i] + lam[0], vy = st * L->cy[i] + lam[1];
        r += f[i];
        jx += vx * f[i];
        jy += vy * f[i];
        e += (vx * vx + vy * vy) * f[i];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
    *T = (e / r - (*ux) * (*ux) - (*uy) * (*uy)) / 2.0;
}

/* rho, u and T of an (f, g) pair in frame lam, two-population model: the
 * conservation laws of Sec. II.B with rho E = sum v^2/2 f + sum g and
 * eq. (E), rho E = C_v rho T + rho u^2 / 2.  g = NULL: no g population
 * (C_v = D/2 = 1, the single-population thermal model, same as macro). */
static void macro2(const olat *L, const double lam[3], const double *f, const double *g,
                   double cv, double *rho, double *ux, double *uy, double *T)
{
    double st = sqrt(lam[2]);
    double r = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double vx = st * L->cx[i] + lam[0], vy = st * L->cy[i] + lam[1];
        r += f[i];
        jx += vx * f[i];
        jy += vy * f[i];
        e += 0.5 * (vx * vx + vy * vy) * f[i];
        if (g) e += g[i];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
    *T = (e / r - 0.5 * ((*ux) * (*ux) + (*uy) * (*uy))) / (g ? cv : 1.0);
}

/* -------------------------------------------------- lifting / projection */

/* Lifting f_q -> f_Q in frame lam (Sec. III.B, App. C):
 *   m_q = M_q f_q;  M_{q->Q} = m_q (+) M^eq_{Q-q};  f_Q = M_Q^{-1} M_{q->Q}.
 * The completing equilibrium is the Q-lattice equilibrium at the cell's rho,
 * u computed from f_q, and at T = T_fix when T_fix > 0 (athermal model),
 * else at the kinetic T of f_q; it is expressed in frame lam. */
static int lift(const olat *Lq, const olat *LQ, const double lam[3], double T_fix,
                const double *fq, double *fQ)
{
    int nq = Lq->n, nQ = LQ->n, Q = LQ->Q;
    double Mq[ORC_MAXQ * ORC_MAXQ], MQ[ORC_MAXQ * ORC_MAXQ], MQi[ORC_MAXQ * ORC_MAXQ];
    double mq[ORC_MAXQ], feqQ[ORC_MAXQ], Meq[ORC_MAXQ], M[ORC_MAXQ];
    double rho, ux, uy, T;

    moment_matrix(Lq, lam, Mq);
    matvec(Lq->Q, Mq, fq, mq);                   /* m_q = M_q f_q, rows (a + nq b) */
    macro(Lq, lam, fq, &rho, &ux, &uy, &T);
    if (T_fix > 0.0) T = T_fix;
    if (feq_in_frame(LQ, rho, ux, uy, T, lam, feqQ)) return -1;
    moment_matrix(LQ, lam, MQ);
    matvec(Q, MQ, feqQ, Meq);                    /* moments of f^{eq,Q} */
    for (int r = 0; r < Q; ++r) {
        int a = r % nQ, b = r / nQ;
        M[r] = (a < nq && b < nq) ? mq[a + nq * b] : Meq[r];
    }
    if (orc_invert(Q, MQ, MQi)) return -1;
    matvec(Q, MQi, M, fQ);                       /* eq. (liftingF) */
    return 0;
}

/* Lifting of the g populations (Sec. III.C: the mappings apply to g as to
 * f): the q x q moments of g_q kept, the others from g^eq = (C_v - 1) T rho W
 * (eq. geqPond) at the node's rho, u, T (st = {rho, u_x, u_y, T}), expressed
 * in frame lam. */
static int lift_g(const olat *Lq, const olat *LQ, const double lam[3], const double st[4],
                  double cv, const double *gq, double *gQ)
{
    int nq = Lq->n, nQ = LQ->n, Q = LQ->Q;
    double Mq[ORC_MAXQ * ORC_MAXQ], MQ[ORC_MAXQ * ORC_MAXQ], MQi[ORC_MAXQ * ORC_MAXQ];
    double mq[ORC_MAXQ], geqQ[ORC_MAXQ], Meq[ORC_MAXQ], M[ORC_MAXQ];
    moment_matrix(Lq, lam, Mq);
    matvec(Lq->Q, Mq, gq, mq);
    if (feq_in_frame(LQ, st[0], st[1], st[2], st[3], lam, geqQ)) return -1;
    for (int i = 0; i < Q; ++i) geqQ[i] *= (cv - 1.0) * st[3];
    moment_matrix(LQ, lam, MQ);
    matvec(Q, MQ, geqQ, Meq);
    for (int r = 0; r < Q; ++r) {
        int a = r % nQ, b = r / nQ;
        M[r] = (a < nq && b < nq) ? mq[a + nq * b] : Meq[r];
    }
    if (orc_invert(Q, MQ, MQi)) return -1;
    matvec(Q, MQi, M, gQ);
    return 0;
}

/* Projection f_Q -> f_q in frame lam (Sec. III.C, App. C):
 *   m_{Q->q} = the first q x q moments of f_Q;  f_q = M_q^{-1} m_{Q->q}. */
static int project(const olat *LQ, const olat *Lq, const double lam[3],
                   const double *fQ, double *fq)
{
    int nq = Lq->n, q = Lq->Q;
    double st = sqrt(lam[2]);
    double Mq[ORC_MAXQ * ORC_MAXQ], Mqi[ORC_MAXQ * ORC_MAXQ], m[ORC_MAXQ];
    for (int r = 0; r < q; ++r) {
        int a = r % nq, b = r / nq;
        double s = 0.0;
        for (int i = 0; i < LQ->Q; ++i)
            s += ipow(st * LQ->cx[i] + lam[0], a) * ipow(st * LQ->cy[i] + lam[1], b) * fQ[i];
        m[r] = s;
    }
    moment_matrix(Lq, lam, Mq);
    if (orc_invert(q, Mq, Mqi)) return -1;
    matvec(q, Mqi, m, fq);
    return 0;
}

int orc_lift(int nq, int nQ, const double lam[3], double T_fix, const double *fq, double *fQ)
{
    olat Lq, LQ;
    if (nq >= nQ || make_lattice(nq, &Lq) || make_lattice(nQ, &LQ)) return -1;
    return lift(&Lq, &LQ, lam, T_fix, fq, fQ);
}

int orc_project(int nQ, int nq, const double lam[3], const double *fQ, double *fq)
{
    olat Lq, LQ;
    if (nq >= nQ || make_lattice(nq, &Lq) || make_lattice(nQ, &LQ)) return -1;
    return project(&LQ, &Lq, lam, fQ, fq);
}

/* --------------------------------------------------- Lagrange reconstruction */

/* Lagrange interpolation functions a_s of eq. (reconstructionPond) on the p
 * equispaced collocation points x0, x0+1, ..., x0+p-1, evaluated at xd. */
void orc_lagrange(int p, double xd, long x0, double *a)
{
    for (int s = 0; s < p; ++s) {
        double v = 1.0;
        for (int r = 0; r < p; ++r)
            if (r != s) v *= (xd - (double)(x0 + r)) / (double)(s - r);
        a[s] = v;
    }
}

/* First collocation point for p points around the departure point xd. */
long orc_first_node(int p, double xd)
{
    return (long)floor(xd - 0.5 * (p - 1) + 0.5);
}

/* ------------------------------------------------------------ the solver */

enum { ORC_BC_OUTFLOW = 0, ORC_BC_DIRICHLET = 1, ORC_BC_INLET = 2, ORC_BC_DIFFUSE = 3 };

typedef struct {
    int kind;
    double *rho, *ux, *uy;       /* length = side length, or NULL */
} obc;

typedef struct {
    int nx, ny, per_x, per_y;
    olat L[2];                   /* 0 = low-order lattice q, 1 = high-order Q */
    double tau, omega, dt;
    int p;                       /* collocation points per axis */
    int frame;                   /* 0 = lattice frame, 1 = PonD thermal, 2 = PonD isothermal */
    double *lam;                 /* PonD: frame {u_x, u_y, T} of every cell's populations */
    double tol;                  /* predictor-corrector tolerance */
    int maxit;                   /* predictor-corrector reconstructions at most */
    long nonconv;                /* cell updates that stopped at maxit */
    double *mom[2];              /* PonD: per-step memo of node moments M_lambda_s f_s */
    uint8_t *hmom[2];
    double *f[2];                /* f[k][cell * Q_k + i]; meaningful where flag == k */
    uint8_t *flag;
    int crit_kind;               /* 0 = fixed flags, 1 = Mach criterion */
    double crit_thr;
    obc bc[4];                   /* x-, x+, y-, y+ */
    /* per-step memo of node vectors in either lattice, over a padded grid */
    int H, px, py;
    double *memo[2];
    uint8_t *have[2];
    double Minv_lat[2][ORC_MAXQ * ORC_MAXQ];
    long steps;
    /* two-population co-moving model (orc_set_twopop): g populations of
     * eq. (Pond_g_equation) in absolute energy units, same layout as f */
    int twopop;
    double cv, omega2;           /* C_v (R = 1) and omega_2 */
    double *g[2], *gmemo[2], *gmom[2];
    uint8_t *ghave[2], *ghmom[2];
    /* co-moving frame with a non-periodic x axis: fixed end states (rho, u_x,
     * u_y, T) beyond x < 0 (side 0) and x >= nx (side 1), and the moments of
     * their vectors rho W_i (and g^eq) in their own frames, per lattice */
    double ends[2][4];
    double bmom[2][2][ORC_MAXQ], bgmom[2][2][ORC_MAXQ];
    int ends_set;
    /* hard-sphere viscosity law (two-population model): mu = mu1 (T/T1)^s,
     * omega_1 from mu = (1/omega_1 - 1/2) rho T dt, Pr fixed */
    int hs;
    double mu1, T1, s_exp, pr;
    /* Knudsen refinement criterion (Sec. IV.C): every kn_interval steps */
    int kn;
    double kn_thr;
    int kn_interval;
} orc_t;

static long cidx(const orc_t *s, long x, long y) { return x + (long)s->nx * y; }

void orc_destroy(orc_t *s);

orc_t *orc_create(int nx, int ny, int per_x, int per_y, int n_lo, int n_hi,
                  double tau, int order, int frame, double cfl)
{
    if (nx < 1 || ny < 1 || n_lo >= n_hi || tau <= 0.5 || order < 1 || order > 5 ||
        frame < 0 || frame > 2 || (frame != 0 && !per_y))
        return NULL;
    orc_t *s = (orc_t *)calloc(1, sizeof(orc_t));
    if (!s) return NULL;
    s->nx = nx; s->ny = ny; s->per_x = per_x; s->per_y = per_y;
    if (make_lattice(n_lo, &s->L[0]) || make_lattice(n_hi, &s->L[1])) { free(s); return NULL; }
    s->tau = tau;
    s->omega = 1.0 / tau;
    double cmax = 0.0;
    for (int k = 0; k < 2; ++k)
        for (int j = 0; j < s->L[k].n; ++j) cmax = fmax(cmax, fabs(s->L[k].c[j]));
    s->dt = cfl / cmax;                          /* CFL = max|c| dt / dx, Sec. IV */
    s->p = order + 1;
    s->frame = frame;
    long nc = (long)nx * ny;
    for (int k = 0; k < 2; ++k) {
        s->f[k] = (double *)calloc(nc * s->L[k].Q, sizeof(double));
        double lat[3] = {0.0, 0.0, 1.0}, M[ORC_MAXQ * ORC_MAXQ];
        moment_matrix(&s->L[k], lat, M);
        orc_invert(s->L[k].Q, M, s->Minv_lat[k]);
    }
    s->flag = (uint8_t *)calloc(nc, 1);
    s->H = s->p + 2;
    s->px = nx + 2 * s->H;
    s->py = ny + 2 * s->H;
    for (int k = 0; k < 2; ++k) {
        s->memo[k] = (double *)calloc((long)s->px * s->py * s->L[k].Q, sizeof(double));
        s->have[k] = (uint8_t *)calloc((long)s->px * s->py, 1);
    }
    for (int b = 0; b < 4; ++b) s->bc[b].kind = ORC_BC_OUTFLOW;
    s->tol = 1e-12;
    s->maxit = 50;
    int pond_ok = 1;
    if (frame != 0) {
        s->lam = (double *)calloc(3 * nc, sizeof(double));
        for (int k = 0; k < 2; ++k) {
            s->mom[k] = (double *)calloc(nc * s->L[k].Q, sizeof(double));
            s->hmom[k] = (uint8_t *)calloc(nc, 1);
        }
        pond_ok = s->lam && s->mom[0] && s->mom[1] && s->hmom[0] && s->hmom[1];
        for (long c = 0; pond_ok && c < nc; ++c) s->lam[3 * c + 2] = 1.0;
    }
    if (!pond_ok || !s->f[0] || !s->f[1] || !s->flag || !s->memo[0] || !s->memo[1] || !s->have[0] || !s->have[1]) {
        orc_destroy(s);
        return NULL;
    }
    return s;
}

void orc_destroy(orc_t *s)
{
    if (!s) return;
    for (int k = 0; k < 2; ++k) {
        free(s->f[k]); free(s->memo[k]); free(s->have[k]); free(s->mom[k]); free(s->hmom[k]);
        free(s->g[k]); free(s->gmemo[k]); free(s->ghave[k]); free(s->gmom[k]); free(s->ghmom[k]);
    }
    free(s->lam);
    for (int b = 0; b < 4; ++b) { free(s->bc[b].rho); free(s->bc[b].ux); free(s->bc[b].uy); }
    free(s->flag);
    free(s);
}

double orc_dt(const orc_t *s) { return s->dt; }

/* Lattice-frame equilibrium of lattice k, f^L = G_{u,T_L}^{0,T_L} rho W
 * (eq. feqL0); the inverse of the constant lattice-frame moment matrix is
 * formed once at creation (same arithmetic as feq_in_frame). */
static void eq_lat(const orc_t *s, int k, double rho, double ux, double uy, double *f)
{
    const olat *L = &s->L[k];
    double G[ORC_MAXQ * ORC_MAXQ], feq[ORC_MAXQ];
    double own[3] = {ux, uy, 1.0};
    for (int i = 0; i < L->Q; ++i) feq[i] = rho * L->W[i];
    transfer_inv(L, own, s->Minv_lat[k], G);
    matvec(L->Q, G, feq, f);
}

static const double LATTICE_FRAME[3] = {0.0, 0.0, 1.0};

/* Frame the populations of cell c live in: the lattice frame {0, T_L}, or the
 * cell's own co-moving frame in PonD. */
static const double *cell_frame(const orc_t *s, long c)
{
    return s->frame ? s->lam + 3 * c : LATTICE_FRAME;
}

/* Convert the vector of lattice `from` into lattice `to` (lift or project) in
 * the frame lam the vector lives in.  The completing equilibrium of a lift is
 * at T = T_L except in the thermal co-moving model (kinetic T of f_q). */
static void convert(const orc_t *s, int from, int to, const double *lam, const double *src,
                    double *dst)
{
    if (from == to) { memcpy(dst, src, sizeof(double) * s->L[to].Q); return; }
    if (from == 0) lift(&s->L[0], &s->L[1], lam, s->frame == 1 ? -1.0 : 1.0, src, dst);
    else project(&s->L[1], &s->L[0], lam, src, dst);
}

/* rho, u_x, u_y, T of cell c from its native f (and g) in its own frame. */
static void node_state(const orc_t *s, long c, double st[4])
{
    int k = s->flag[c];
    const olat *L = &s->L[k];
    macro2(L, s->lam + 3 * c, s->f[k] + c * L->Q, s->twopop ? s->g[k] + c * L->Q : NULL, s->cv,
           &st[0], &st[1], &st[2], &st[3]);
}

/* Two-population model: cell c's f (which = 0) or g (which = 1) vector in
 * lattice `to`, converted in the cell's frame; a lift completes with the
 * equilibrium at the cell's rho, u, T (T from f and g). */
static int convert2(const orc_t *s, long c, int to, int which, double *dst)
{
    int from = s->flag[c];
    const double *lam = s->lam + 3 * c;
    const double *src = (which ? s->g[from] : s->f[from]) + c * s->L[from].Q;
    if (from == to) { memcpy(dst, src, sizeof(double) * s->L[to].Q); return 0; }
    if (from == 1) return project(&s->L[1], &s->L[0], lam, src, dst);
    double st[4];
    node_state(s, c, st);
    if (!which) return lift(&s->L[0], &s->L[1], lam, st[3], src, dst);
    return lift_g(&s->L[0], &s->L[1], lam, st, s->cv, src, dst);
}

/* Every cell starts at the equilibrium of both lattices (both representations
 * valid), flags 0.  Lattice frame: f^L at (rho, u), T must be NULL (athermal).
 * Co-moving frame: f = rho W_i in the frame {u, T} (eq. feqPond), T = T_L when
 * NULL; the isothermal variant takes T = NULL only. */
int orc_init_equilibrium(orc_t *s, const double *rho, const double *ux, const double *uy,
                         const double *T)
{
    long nc = (long)s->nx * s->ny;
    if (T && s->frame != 1) return -1;
    for (long c = 0; c < nc; ++c)
        for (int k = 0; k < 2; ++k) {
            double *f = s->f[k] + c * s->L[k].Q;
            if (s->frame == 0) {
                eq_lat(s, k, rho[c], ux[c], uy[c], f);
            } else {
                double Tc = T ? T[c] : 1.0;
                for (int i = 0; i < s->L[k].Q; ++i) f[i] = rho[c] * s->L[k].W[i];
                if (s->twopop)                       /* eq. (geqPond) in the cell's frame */
                    for (int i = 0; i < s->L[k].Q; ++i)
                        s->g[k][c * s->L[k].Q + i] = (s->cv - 1.0) * Tc * rho[c] * s->L[k].W[i];
                s->lam[3 * c] = ux[c];
                s->lam[3 * c + 1] = uy[c];
                s->lam[3 * c + 2] = T ? T[c] : 1.0;
            }
        }
    memset(s->flag, 0, nc);
    return 0;
}

/* New flags; a cell whose flag changes has its populations lifted or projected. */
int orc_set_flags(orc_t *s, const uint8_t *fl)
{
    long nc = (long)s->nx * s->ny;
    for (long c = 0; c < nc; ++c) {
        int nf = fl[c] ? 1 : 0;
        if (nf != s->flag[c]) {
            if (s->twopop) {
                convert2(s, c, nf, 0, s->f[nf] + c * s->L[nf].Q);
                convert2(s, c, nf, 1, s->g[nf] + c * s->L[nf].Q);
            } else {
                convert(s, s->flag[c], nf, cell_frame(s, c), s->f[s->flag[c]] + c * s->L[s->flag[c]].Q,
                        s->f[nf] + c * s->L[nf].Q);
            }
            s->flag[c] = (uint8_t)nf;
        }
    }
    return 0;
}

void orc_get_flags(const orc_t *s, uint8_t *fl) { memcpy(fl, s->flag, (size_t)s->nx * s->ny); }

/* Refinement criterion of Sec. IV.A on the current state: high-order iff
 * Ma = |u| / c_s > thr with c_s = sqrt(T_L) = 1 (athermal model); a cell whose
 * flag flips has its populations lifted or projected. */
static void apply_criterion(orc_t *s)
{
    long nc = (long)s->nx * s->ny;
    double lat[3] = {0.0, 0.0, 1.0};
    for (long c = 0; c < nc; ++c) {
        int k = s->flag[c];
        double rho, ux, uy, T;
        macro(&s->L[k], lat, s->f[k] + c * s->L[k].Q, &rho, &ux, &uy, &T);
        int nf = sqrt(ux * ux + uy * uy) > s->crit_thr ? 1 : 0;
        if (nf != k) {
            convert(s, k, nf, LATTICE_FRAME, s->f[k] + c * s->L[k].Q, s->f[nf] + c * s->L[nf].Q);
            s->flag[c] = (uint8_t)nf;
        }
    }
}

/* kind 0: flags stay fixed; kind 1: Mach criterion, applied at once to the
 * current state and after every step from then on. */
int orc_set_criterion(orc_t *s, int kind, double thr)
{
    if (kind != 0 && s->frame != 0) return -1;   /* the Mach criterion is athermal */
    s->crit_kind = kind;
    s->crit_thr = thr;
    if (kind == 1) apply_criterion(s);
    return 0;
}

/* Boundary of a non-periodic side: side 0 = x-, 1 = x+, 2 = y-, 3 = y+.
 * Arrays run along the side (ny entries for x sides, nx for y sides). */
int orc_set_bc(orc_t *s, int side, int kind, const double *rho, const double *ux, const double *uy)
{
    if (side < 0 || side > 3) return -1;
    int len = side < 2 ? s->ny : s->nx;
    obc *b = &s->bc[side];
    free(b->rho); free(b->ux); free(b->uy);
    b->rho = b->ux = b->uy = NULL;
    b->kind = kind;
    if (rho) { b->rho = (double *)malloc(sizeof(double) * len); memcpy(b->rho, rho, sizeof(double) * len); }
    if (ux) { b->ux = (double *)malloc(sizeof(double) * len); memcpy(b->ux, ux, sizeof(double) * len); }
    if (uy) { b->uy = (double *)malloc(sizeof(double) * len); memcpy(b->uy, uy, sizeof(double) * len); }
    return 0;
}

static double cell_rho(const orc_t *s, long c)
{
    int k = s->flag[c];
    double r = 0.0;
    for (int i = 0; i < s->L[k].Q; ++i) r += s->f[k][c * s->L[k].Q + i];
    return r;
}

/* Diffuse-reflection wall ghost (the kinetic wall of the Couette flow of
 * Sec. IV.C; the paper names the condition without giving its formula).
 * The wall's normal is `axis` (0 = x, 1 = y) with the fluid on the side of
 * sign n.  Populations entering the fluid (c.n > 0) are the lattice
 * equilibrium at the wall velocity (eq. feqL0), scaled so that the mass they
 * carry into the fluid equals the mass the first interior node `base` sends
 * into the wall (zero net normal flux); the others copy that node. */
static void diffuse_ghost(const orc_t *s, int k, const double *base, int axis, double n,
                          double uwx, double uwy, double *out)
{
    const olat *L = &s->L[k];
    double feq[ORC_MAXQ];
    eq_lat(s, k, 1.0, uwx, uwy, feq);
    double out_flux = 0.0, in_unit = 0.0;
    for (int i = 0; i < L->Q; ++i) {
        double cn = (axis ? L->cy[i] : L->cx[i]) * n;
        if (cn < 0.0) out_flux -= cn * base[i];
        else if (cn > 0.0) in_unit += cn * feq[i];
    }
    double rho_w = out_flux / in_unit;
    for (int i = 0; i < L->Q; ++i) {
        double cn = (axis ? L->cy[i] : L->cx[i]) * n;
        out[i] = cn > 0.0 ? rho_w * feq[i] : base[i];
    }
}

/* Population vector of node (gx, gy) at the old time level, expressed in
 * lattice k (step 2 of Sec. III.D), with periodic wrap and boundary ghosts. */
static const double *node_vec(orc_t *s, long gx, long gy, int k)
{
    if (s->per_x) gx = ((gx % s->nx) + s->nx) % s->nx;
    if (s->per_y) gy = ((gy % s->ny) + s->ny) % s->ny;
    long mx = gx + s->H, my = gy + s->H;
    long m = mx + (long)s->px * my;
    int Q = s->L[k].Q;
    double *out = s->memo[k] + m * Q;
    if (gx >= 0 && gx < s->nx && gy >= 0 && gy < s->ny) {
        long c = cidx(s, gx, gy);
        if (s->flag[c] == k) return s->f[k] + c * Q;        /* native */
        if (!s->have[k][m]) {
            if (s->twopop)
                convert2(s, c, k, 0, out);
            else
                convert(s, s->flag[c], k, cell_frame(s, c), s->f[s->flag[c]] + c * s->L[s->flag[c]].Q,
                        out);
            s->have[k][m] = 1;
        }
        return out;
    }
    if (s->have[k][m]) return out;
    if (gy < 0 || gy >= s->ny) {                   /* non-periodic y side */
        const obc *b = &s->bc[gy < 0 ? 2 : 3];
        long xi = gx < 0 ? 0 : (gx >= s->nx ? s->nx - 1 : gx);
        long yi = gy < 0 ? 0 : s->ny - 1;
        if (b->kind == ORC_BC_OUTFLOW) {
            memcpy(out, node_vec(s, gx, yi, k), sizeof(double) * Q);
        } else if (b->kind == ORC_BC_DIFFUSE) {
            diffuse_ghost(s, k, node_vec(s, gx, yi, k), 1, gy < 0 ? 1.0 : -1.0, b->ux[xi],
                          b->uy[xi], out);
        } else {
            double rho = b->kind == ORC_BC_INLET ? cell_rho(s, cidx(s, xi, yi)) : b->rho[xi];
            eq_lat(s, k, rho, b->ux[xi], b->uy[xi], out);
        }
    } else {                                       /* non-periodic x side */
        const obc *b = &s->bc[gx < 0 ? 0 : 1];
        long xi = gx < 0 ? 0 : s->nx - 1;
        if (b->kind == ORC_BC_OUTFLOW) {
            memcpy(out, node_vec(s, xi, gy, k), sizeof(double) * Q);
        } else if (b->kind == ORC_BC_DIFFUSE) {
            diffuse_ghost(s, k, node_vec(s, xi, gy, k), 0, gx < 0 ? 1.0 : -1.0, b->ux[gy],
                          b->uy[gy], out);
        } else {
            double rho = b->kind == ORC_BC_INLET ? cell_rho(s, cidx(s, xi, gy)) : b->rho[gy];
            eq_lat(s, k, rho, b->ux[gy], b->uy[gy], out);
        }
    }
    s->have[k][m] = 1;
    return out;
}

static double snap(double v)
{
    double r = nearbyint(v);
    return fabs(v - r) < 1e-12 ? r : v;
}

/* One lattice-frame update of cell (x, y): semi-Lagrangian propagation
 * (Sec. III.D, eq. advectionPond / reconstructionPond) followed by BGK
 * collision to the lattice equilibrium (eq. Pond_f_equation with
 * omega_1 = omega_2, eq. feqL0).  Writes Q_k values to out. */
static void update_cell(orc_t *s, long x, long y, double *out)
{
    int k = s->flag[cidx(s, x, y)];
    const olat *L = &s->L[k];
    int p = s->p;
    double fbar[ORC_MAXQ], ax[8], ay[8];
    for (int i = 0; i < L->Q; ++i) {
        double xd = (double)x - snap(L->cx[i] * s->dt);   /* x_dep = x - v_i dt */
        double yd = (double)y - snap(L->cy[i] * s->dt);
        long x0 = orc_first_node(p, xd), y0 = orc_first_node(p, yd);
        orc_lagrange(p, xd, x0, ax);
        orc_lagrange(p, yd, y0, ay);
        double acc = 0.0;
        for (int t = 0; t < p; ++t)
            for (int u = 0; u < p; ++u)
                acc += ax[u] * ay[t] * node_vec(s, x0 + u, y0 + t, k)[i];
        fbar[i] = acc;
    }
    double rho = 0.0, jx = 0.0, jy = 0.0, feq[ORC_MAXQ];
    for (int i = 0; i < L->Q; ++i) {
        rho += fbar[i];
        jx += L->cx[i] * fbar[i];
        jy += L->cy[i] * fbar[i];
    }
    eq_lat(s, k, rho, jx / rho, jy / rho, feq);
    for (int i = 0; i < L->Q; ++i) out[i] = fbar[i] + s->omega * (feq[i] - fbar[i]);
}

/* Moments M_{lambda_s} f_s (eq. momfshort) of node (gx, gy)'s vector in
 * lattice k, taken in the node's own frame lambda_s; memoised per step.  Only
 * for the co-moving frame, whose grids are periodic. */
static const double *node_moments(orc_t *s, long gx, long gy, int k)
{
    if (!s->per_x && (gx < 0 || gx >= s->nx)) return s->bmom[gx < 0 ? 0 : 1][k];
    gx = ((gx % s->nx) + s->nx) % s->nx;
    gy = ((gy % s->ny) + s->ny) % s->ny;
    long c = cidx(s, gx, gy);
    int Q = s->L[k].Q;
    double *m = s->mom[k] + c * Q;
    if (!s->hmom[k][c]) {
        double M[ORC_MAXQ * ORC_MAXQ];
        moment_matrix(&s->L[k], cell_frame(s, c), M);
        matvec(Q, M, node_vec(s, gx, gy, k), m);
        s->hmom[k][c] = 1;
    }
    return m;
}

/* g vector of node (gx, gy) in lattice k (two-population model; co-moving
 * grids are periodic) and its moments in the node's frame, memoised per step. */
static const double *node_vec_g(orc_t *s, long gx, long gy, int k)
{
    gx = ((gx % s->nx) + s->nx) % s->nx;
    gy = ((gy % s->ny) + s->ny) % s->ny;
    long c = cidx(s, gx, gy);
    int Q = s->L[k].Q;
    if (s->flag[c] == k) return s->g[k] + c * Q;
    double *out = s->gmemo[k] + c * Q;
    if (!s->ghave[k][c]) {
        convert2(s, c, k, 1, out);
        s->ghave[k][c] = 1;
    }
    return out;
}

static const double *node_moments_g(orc_t *s, long gx, long gy, int k)
{
    if (!s->per_x && (gx < 0 || gx >= s->nx)) return s->bgmom[gx < 0 ? 0 : 1][k];
    gx = ((gx % s->nx) + s->nx) % s->nx;
    gy = ((gy % s->ny) + s->ny) % s->ny;
    long c = cidx(s, gx, gy);
    int Q = s->L[k].Q;
    double *m = s->gmom[k] + c * Q;
    if (!s->ghmom[k][c]) {
        double M[ORC_MAXQ * ORC_MAXQ];
        moment_matrix(&s->L[k], cell_frame(s, c), M);
        matvec(Q, M, node_vec_g(s, gx, gy, k), m);
        s->ghmom[k][c] = 1;
    }
    return m;
}

/* Two-population collision (eqs. Pond_f_equation, Pond_g_equation) of the
 * reconstructed fbar, gbar living in frame lam, at their moments rho, u, T:
 * equilibria of eqs. (feqPond, geqPond) and quasi-equilibria of eqs. (fqeq,
 * gqeq) formed in the co-moving frame {u, T} (theta = T with R = T_L = 1) and
 * carried into lam; the tensors Qbar (third-order, of f - f^eq) and qbar (of
 * g - g^eq) are taken with the velocities v_i - u of frame lam. */
static int collide2(const orc_t *s, const olat *L, const double lam[3], double rho, double ux,
                    double uy, double T, const double *fbar, const double *gbar, double *fout,
                    double *gout)
{
    int Q = L->Q;
    double feq[ORC_MAXQ], geq[ORC_MAXQ], df[ORC_MAXQ], dg[ORC_MAXQ], tf[ORC_MAXQ], tg[ORC_MAXQ];
    double G[ORC_MAXQ * ORC_MAXQ], own[3] = {ux, uy, T};
    if (feq_in_frame(L, rho, ux, uy, T, lam, feq)) return -1;
    for (int i = 0; i < Q; ++i) geq[i] = (s->cv - 1.0) * T * feq[i];
    /* Qbar_abc = sum (v-u)_a (v-u)_b (v-u)_c (f - f^eq), qbar_a = sum (v-u)_a (g - g^eq) */
    double st = sqrt(lam[2]);
    double Qb[2][2][2] = {{{0}}}, qb[2] = {0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        double w[2] = {st * L->cx[i] + lam[0] - ux, st * L->cy[i] + lam[1] - uy};
        double nf = fbar[i] - feq[i], ng = gbar[i] - geq[i];
        for (int a = 0; a < 2; ++a) {
            qb[a] += w[a] * ng;
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < 2; ++c) Qb[a][b][c] += w[a] * w[b] * w[c] * nf;
        }
    }
    /* eq. (fqeq): W_i Qbar:(theta^{3/2} c c c - R T theta^{1/2} sym(c (x) 1)) / (6 (RT)^3);
     * eq. (gqeq): W_i theta^{1/2} qbar.c / (R T); in the co-moving frame {u, T} */
    double th = T, RT = T;
    for (int i = 0; i < Q; ++i) {
        double c[2] = {L->cx[i], L->cy[i]};
        double ccc = 0.0, sym = 0.0, qc = 0.0;
        for (int a = 0; a < 2; ++a) {
            qc += qb[a] * c[a];
            for (int b = 0; b < 2; ++b)
                for (int e = 0; e < 2; ++e) {
                    ccc += Qb[a][b][e] * c[a] * c[b] * c[e];
                    /* sym(c (x) 1)_abe = c_a d_be + c_b d_ae + c_e d_ab */
                    sym += Qb[a][b][e] * (c[a] * (b == e) + c[b] * (a == e) + c[e] * (a == b));
                }
        }
        df[i] = L->W[i] * (pow(th, 1.5) * ccc - RT * sqrt(th) * sym) / (6.0 * RT * RT * RT);
        dg[i] = L->W[i] * sqrt(th) * qc / RT;
    }
    if (transfer(L, own, lam, G)) return -1;
    matvec(Q, G, df, tf);                        /* f* - f^eq in frame lam */
    matvec(Q, G, dg, tg);
    double w1 = s->omega, w2 = s->omega2;
    if (s->hs) {  /* mu = (1/omega_1 - 1/2) rho T dt, kappa = C_p mu / Pr (Sec. II.B, IV.C) */
        double mu = s->mu1 * pow(T / s->T1, s->s_exp);
        double tau1 = mu / (rho * T * s->dt) + 0.5;
        w1 = 1.0 / tau1;
        w2 = 1.0 / ((tau1 - 0.5) / s->pr + 0.5);
    }
    for (int i = 0; i < Q; ++i) {
        fout[i] = fbar[i] + w1 * (feq[i] - fbar[i]) + (w1 - w2) * tf[i];
        gout[i] = gbar[i] + w1 * (geq[i] - gbar[i]) + (w1 - w2) * tg[i];
    }
    return 0;
}

/* One co-moving-frame update of cell (x, y), Sec. II.C.
 * Predictor: the cell's frame of the previous step.  Each pass reconstructs
 * every population at its departure point x - v_i dt, v_i = sqrt(theta) c_i + u
 * of the current frame guess lam (eqs. vi, advectionPond), where the
 * collocation vectors are first carried into lam: G_{lambda_s}^{lam} f_s =
 * M_lam^{-1} (M_{lambda_s} f_s) (eqs. fll, reconstructionPond).  The moments
 * of the result (eqs. correctorfieldsrho-u) become the next guess until they
 * agree with it to tol.  Then BGK (eq. Pond_f_equation, omega_1 = omega_2)
 * towards the equilibrium at those moments expressed in lam.  Writes Q values
 * to out and the frame they live in to lam_out. */
static int update_cell_pond(orc_t *s, long x, long y, double *out, double *gout,
                            double *lam_out)
{
    long c = cidx(s, x, y);
    int k = s->flag[c];
    const olat *L = &s->L[k];
    int p = s->p, Q = L->Q;
    double lam[3], nl[3] = {0.0, 0.0, 1.0}, rho = 0.0;
    double fbar[ORC_MAXQ], gbar[ORC_MAXQ], feq[ORC_MAXQ], ax[8], ay[8];
    double Mt[ORC_MAXQ * ORC_MAXQ], Mti[ORC_MAXQ * ORC_MAXQ];
    int converged = 0;
    memcpy(lam, s->lam + 3 * c, sizeof(lam));
    for (int it = 0; it < s->maxit; ++it) {
        moment_matrix(L, lam, Mt);
        if (orc_invert(Q, Mt, Mti)) return -1;
        double st = sqrt(lam[2]);
        for (int i = 0; i < Q; ++i) {
            double xd = (double)x - (st * L->cx[i] + lam[0]) * s->dt;
            double yd = (double)y - (st * L->cy[i] + lam[1]) * s->dt;
            long x0 = orc_first_node(p, xd), y0 = orc_first_node(p, yd);
            orc_lagrange(p, xd, x0, ax);
            orc_lagrange(p, yd, y0, ay);
            double acc = 0.0, gacc = 0.0;
            for (int t = 0; t < p; ++t)
                for (int u = 0; u < p; ++u) {
                    const double *m = node_moments(s, x0 + u, y0 + t, k);
                    double gi = 0.0;                      /* (G_{lambda_s}^{lam} f_s)_i */
                    for (int r = 0; r < Q; ++r) gi += Mti[i * Q + r] * m[r];
                    acc += ax[u] * ay[t] * gi;
                    if (s->twopop) {                      /* eq. (reconstructionPondg) */
                        const double *mg = node_moments_g(s, x0 + u, y0 + t, k);
                        double hi = 0.0;
                        for (int r = 0; r < Q; ++r) hi += Mti[i * Q + r] * mg[r];
                        gacc += ax[u] * ay[t] * hi;
                    }
                }
            fbar[i] = acc;
            gbar[i] = gacc;
        }
        double ux, uy, T;
        macro2(L, lam, fbar, s->twopop ? gbar : NULL, s->cv, &rho, &ux, &uy, &T);
        if (s->frame == 2) T = 1.0;
        nl[0] = ux; nl[1] = uy; nl[2] = T;
        double d = fmax(fabs(ux - lam[0]), fmax(fabs(uy - lam[1]), fabs(T - lam[2])));
        if (d <= s->tol) { converged = 1; break; }
        if (it + 1 < s->maxit) memcpy(lam, nl, sizeof(lam));
    }
    if (!converged) s->nonconv++;
    if (s->twopop) {
        if (collide2(s, L, lam, rho, nl[0], nl[1], nl[2], fbar, gbar, out, gout)) return -1;
    } else {
        if (feq_in_frame(L, rho, nl[0], nl[1], nl[2], lam, feq)) return -1;
        for (int i = 0; i < Q; ++i) out[i] = fbar[i] + s->omega * (feq[i] - fbar[i]);
    }
    memcpy(lam_out, lam, sizeof(lam));
    return 0;
}

static void reset_memo(orc_t *s)
{
    for (int k = 0; k < 2; ++k) {
        memset(s->have[k], 0, (size_t)s->px * s->py);
        if (s->hmom[k]) memset(s->hmom[k], 0, (size_t)s->nx * s->ny);
        if (s->ghave[k]) memset(s->ghave[k], 0, (size_t)s->nx * s->ny);
        if (s->ghmom[k]) memset(s->ghmom[k], 0, (size_t)s->nx * s->ny);
    }
}

/* Knudsen refinement criterion of Sec. IV.C on a quasi-one-dimensional
 * instance: Kn = lambda / L with L = |rho / (d rho / dx)| (central
 * differences, the fixed end states beyond the ends), the local mean free
 * path of hard spheres lambda = 16 / (5 sqrt(2 pi gamma)) mu a / p with
 * mu = mu1 (T / T1)^s, a = sqrt(gamma T), p = rho T, gamma = (C_v + 1) / C_v;
 * high-order iff Kn > thr, flipped cells lifted or projected. */
static void apply_kn(orc_t *s)
{
    long nc = (long)s->nx * s->ny;
    double *rho = (double *)malloc(sizeof(double) * nc), *T = (double *)malloc(sizeof(double) * nc);
    uint8_t *fl = (uint8_t *)malloc(nc);
    if (!rho || !T || !fl) { free(rho); free(T); free(fl); return; }
    for (long c = 0; c < nc; ++c) {
        double st[4];
        node_state(s, c, st);
        rho[c] = st[0];
        T[c] = st[3];
    }
    double gam = (s->cv + 1.0) / s->cv;
    for (long y = 0; y < s->ny; ++y)
        for (long x = 0; x < s->nx; ++x) {
            long c = cidx(s, x, y);
            double rl = x > 0 ? rho[c - 1] : s->ends[0][0];
            double rr = x < s->nx - 1 ? rho[c + 1] : s->ends[1][0];
            double drdx = 0.5 * (rr - rl);
            double mu = s->mu1 * pow(T[c] / s->T1, s->s_exp);
            double lam = 16.0 / (5.0 * sqrt(2.0 * 3.14159265358979323846 * gam)) * mu * sqrt(gam * T[c]) / (rho[c] * T[c]);
            double kn = lam * fabs(drdx) / rho[c];
            fl[c] = (kn > s->kn_thr || s->flag[c]) ? 1 : 0;   /* refinement only */
        }
    orc_set_flags(s, fl);
    free(rho); free(T); free(fl);
}

/* Advance n time steps. */
int orc_step(orc_t *s, int n)
{
    long nc = (long)s->nx * s->ny;
    double *g[2] = {NULL, NULL}, *gg[2] = {NULL, NULL}, *glam = NULL;
    int rc = 0;
    for (int k = 0; k < 2; ++k) {
        g[k] = (double *)malloc(sizeof(double) * nc * s->L[k].Q);
        if (!g[k]) rc = -1;
        if (s->twopop) {                         /* next-step g populations */
            gg[k] = (double *)calloc(nc * s->L[k].Q, sizeof(double));
            if (!gg[k]) rc = -1;
        }
    }
    if (s->frame && !(glam = (double *)malloc(sizeof(double) * 3 * nc))) rc = -1;
    if (s->frame && !s->per_x && !s->ends_set) rc = -1;   /* end states required */
    for (int it = 0; it < n && rc == 0; ++it) {
        reset_memo(s);
        for (long y = 0; y < s->ny && rc == 0; ++y)
            for (long x = 0; x < s->nx; ++x) {
                long c = cidx(s, x, y);
                int k = s->flag[c];
                if (s->frame == 0) {
                    update_cell(s, x, y, g[k] + c * s->L[k].Q);
                } else if (update_cell_pond(s, x, y, g[k] + c * s->L[k].Q,
                                            s->twopop ? gg[k] + c * s->L[k].Q : NULL,
                                            glam + 3 * c)) {
                    rc = -1;
                    break;
                }
            }
        if (rc) break;
        for (int k = 0; k < 2; ++k) {
            double *t = s->f[k]; s->f[k] = g[k]; g[k] = t;
            if (s->twopop) { t = s->g[k]; s->g[k] = gg[k]; gg[k] = t; }
        }
        if (s->frame) { double *t = s->lam; s->lam = glam; glam = t; }
        if (s->crit_kind == 1) apply_criterion(s);   /* flags for the next step */
        if (s->kn && (s->steps + 1) % s->kn_interval == 0) apply_kn(s);
        s->steps++;
    }
    free(g[0]);
    free(g[1]);
    free(gg[0]);
    free(gg[1]);
    free(glam);
    return rc;
}

/* One step's post-collision vectors of a few cells, without changing the
 * state: out[j * 25 + i], i < Q of the cell's lattice (flag[c] tells which);
 * in the co-moving frame lam_out[3 j ..] receives the frame they live in
 * (lam_out may be NULL). */
int orc_step_cells(orc_t *s, int m, const long *cells, double *out, double *lam_out)
{
    reset_memo(s);
    for (int j = 0; j < m; ++j) {
        long c = cells[j];
        if (c < 0 || c >= (long)s->nx * s->ny) return -1;
        if (s->frame == 0) {
            update_cell(s, c % s->nx, c / s->nx, out + (long)j * ORC_MAXQ);
        } else {
            double lam[3], gtmp[ORC_MAXQ];
            if (update_cell_pond(s, c % s->nx, c / s->nx, out + (long)j * ORC_MAXQ, gtmp, lam))
                return -1;
            if (lam_out) memcpy(lam_out + 3 * j, lam, sizeof(lam));
        }
    }
    return 0;
}

/* Predictor-corrector controls of the co-moving frame. */
int orc_set_pond(orc_t *s, double tol, int maxit)
{
    if (!(tol >= 0.0) || maxit < 1) return -1;
    s->tol = tol;
    s->maxit = maxit;
    return 0;
}

long orc_nonconverged(const orc_t *s) { return s->nonconv; }

/* Frames {u_x, u_y, T} of the cells' populations (co-moving frame only). */
int orc_get_frame(const orc_t *s, double *ux, double *uy, double *T)
{
    if (!s->frame) return -1;
    for (long c = 0; c < (long)s->nx * s->ny; ++c) {
        ux[c] = s->lam[3 * c];
        uy[c] = s->lam[3 * c + 1];
        T[c] = s->lam[3 * c + 2];
    }
    return 0;
}

int orc_set_frame(orc_t *s, const double *ux, const double *uy, const double *T)
{
    if (!s->frame) return -1;
    for (long c = 0; c < (long)s->nx * s->ny; ++c) {
        if (!(T[c] > 0.0)) return -1;
        s->lam[3 * c] = ux[c];
        s->lam[3 * c + 1] = uy[c];
        s->lam[3 * c + 2] = T[c];
    }
    return 0;
}

/* rho, u and T of every cell from its native populations (kinetic T, or with
 * the g populations and C_v in the two-population model). */
int orc_moments(const orc_t *s, double *rho, double *ux, double *uy, double *T)
{
    long nc = (long)s->nx * s->ny;
    for (long c = 0; c < nc; ++c) {
        int k = s->flag[c];
        double r, a, b, t;
        macro2(&s->L[k], cell_frame(s, c), s->f[k] + c * s->L[k].Q,
               s->twopop ? s->g[k] + c * s->L[k].Q : NULL, s->cv, &r, &a, &b, &t);
        rho[c] = r; ux[c] = a; uy[c] = b;
        if (T) T[c] = t;
    }
    return 0;
}

/* Global sums rho, rho u_x, rho u_y, rho E with rho E = sum v^2/2 f (+ sum g
 * in the two-population model) and v_i = sqrt(theta) c_i + u of the frame
 * each cell's populations live in. */
int orc_audit(const orc_t *s, double out[4])
{
    long nc = (long)s->nx * s->ny;
    double a[4] = {0, 0, 0, 0};
    for (long c = 0; c < nc; ++c) {
        int k = s->flag[c];
        const olat *L = &s->L[k];
        const double *lam = cell_frame(s, c);
        double st = sqrt(lam[2]);
        for (int i = 0; i < L->Q; ++i) {
            double f = s->f[k][c * L->Q + i];
            double vx = st * L->cx[i] + lam[0], vy = st * L->cy[i] + lam[1];
            a[0] += f;
            a[1] += vx * f;
            a[2] += vy * f;
            a[3] += 0.5 * (vx * vx + vy * vy) * f;
            if (s->twopop) a[3] += s->g[k][c * L->Q + i];
        }
    }
    memcpy(out, a, sizeof(a));
    return 0;
}

/* Populations of lattice k, cell-major: out[cell * Q_k + i]. */
int orc_get_pops(const orc_t *s, int k, double *out)
{
    memcpy(out, s->f[k], sizeof(double) * (size_t)s->nx * s->ny * s->L[k].Q);
    return 0;
}

int orc_set_pops(orc_t *s, int k, const double *in)
{
    memcpy(s->f[k], in, sizeof(double) * (size_t)s->nx * s->ny * s->L[k].Q);
    return 0;
}

/* Switch the thermal co-moving model to the two-population model of
 * Sec. II.B with C_v = cv (gamma = (cv + 1) / cv, R = 1) and omega_2 =
 * 1 / tau2 (Pr = (tau - 1/2) / (tau2 - 1/2)).  Call before
 * orc_init_equilibrium, which then sets g = g^eq of eq. (geqPond). */
int orc_set_twopop(orc_t *s, double cv, double tau2)
{
    if (s->frame != 1 || !(cv > 0.0) || !(tau2 > 0.5) || s->twopop) return -1;
    long nc = (long)s->nx * s->ny;
    for (int k = 0; k < 2; ++k) {
        size_t n = (size_t)nc * s->L[k].Q;
        s->g[k] = (double *)calloc(n, sizeof(double));
        s->gmemo[k] = (double *)calloc(n, sizeof(double));
        s->gmom[k] = (double *)calloc(n, sizeof(double));
        s->ghave[k] = (uint8_t *)calloc(nc, 1);
        s->ghmom[k] = (uint8_t *)calloc(nc, 1);
        if (!s->g[k] || !s->gmemo[k] || !s->gmom[k] || !s->ghave[k] || !s->ghmom[k]) return -1;
    }
    s->twopop = 1;
    s->cv = cv;
    s->omega2 = 1.0 / tau2;
    return 0;
}

int orc_get_gpops(const orc_t *s, int k, double *out)
{
    if (!s->twopop) return -1;
    memcpy(out, s->g[k], sizeof(double) * (size_t)s->nx * s->ny * s->L[k].Q);
    return 0;
}

int orc_set_gpops(orc_t *s, int k, const double *in)
{
    if (!s->twopop) return -1;
    memcpy(s->g[k], in, sizeof(double) * (size_t)s->nx * s->ny * s->L[k].Q);
    return 0;
}

/* Co-moving frame with a non-periodic x axis (the quasi-one-dimensional shock
 * of Sec. IV.C): collocation nodes beyond either end hold the fixed state
 * end[side] = {rho, u_x, u_y, T} at rest in its own frame (f = rho W_i,
 * g = (C_v - 1) T rho W_i, eqs. feqPond, geqPond).  Set the two-population
 * model first when it is used. */
int orc_set_pond_ends(orc_t *s, const double left[4], const double right[4])
{
    if (!s->frame || s->per_x) return -1;
    for (int side = 0; side < 2; ++side) {
        const double *e = side ? right : left;
        if (!(e[0] > 0.0) || !(e[3] > 0.0)) return -1;
        memcpy(s->ends[side], e, sizeof(s->ends[side]));
        double lam[3] = {e[1], e[2], e[3]};
        for (int k = 0; k < 2; ++k) {
            const olat *L = &s->L[k];
            double M[ORC_MAXQ * ORC_MAXQ], v[ORC_MAXQ];
            moment_matrix(L, lam, M);
            for (int i = 0; i < L->Q; ++i) v[i] = e[0] * L->W[i];
            matvec(L->Q, M, v, s->bmom[side][k]);
            for (int i = 0; i < L->Q; ++i) v[i] *= s->twopop ? (s->cv - 1.0) * e[3] : 0.0;
            matvec(L->Q, M, v, s->bgmom[side][k]);
        }
    }
    s->ends_set = 1;
    return 0;
}

/* Hard-sphere-like viscosity law of the shock case (Sec. IV.C): mu = mu1 (T /
 * T1)^s_exp, relaxation omega_1 from mu = (1/omega_1 - 1/2) rho T dt and
 * omega_2 from a fixed Prandtl number pr = C_p mu / kappa, per cell update,
 * at the reconstructed rho and T.  Two-population model only. */
int orc_set_viscosity_law(orc_t *s, double mu1, double T1, double s_exp, double pr)
{
    if (!s->twopop || !(mu1 > 0.0) || !(T1 > 0.0) || !(pr > 0.0)) return -1;
    s->hs = 1;
    s->mu1 = mu1;
    s->T1 = T1;
    s->s_exp = s_exp;
    s->pr = pr;
    return 0;
}

/* Knudsen refinement criterion (apply_kn) every `interval` steps, and at once;
 * needs the viscosity law and fixed end states.  Refinement only (Sec. IV.C:
 * the shock is initialised on the low-order lattice and refined): a cell with
 * Kn > thr becomes high-order and stays so.  A criterion that also coarsens
 * switches cells at the shock's edges back and forth, and in this nearly
 * collisionless regime (tau ~ 110 upstream) the hybrid then loses positivity
 * within 20 steps at Mach 1.6. */
int orc_set_kn_criterion(orc_t *s, double thr, int interval)
{
    if (!s->hs || !s->ends_set || interval < 1 || !(thr > 0.0)) return -1;
    s->kn = 1;
    s->kn_thr = thr;
    s->kn_interval = interval;
    apply_kn(s);
    return 0;
}
