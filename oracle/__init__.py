"""FP64 CPU oracle of the multi-scale semi-Lagrangian LBM step (arXiv:2102.12559).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA path in ``paper_2102_12559_gb300``; neither imports the other.

The arithmetic lives in ``slbm_oracle.c`` (plain C, double precision, one
function per step of the paper).  This module only marshals numpy arrays into
that library through ctypes.  Every function names the passage it follows.

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
facts the paper or mathematics fixes (Table I quadrature exactness, the
printed equilibrium moments of Eqs. QxxxL/RxxL/QxxxPonD/RxxPond, the Fig. 1
deviation, project(lift(f)) = f, lift of an equilibrium, Lagrange exactness
on polynomials, conservation, uniform-flow invariance).  None is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "slbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

# Frames: lattice frame, co-moving (PonD) thermal with C_v = D/2, co-moving
# isothermal (T = T_L).
FRAME_LATTICE = 0
FRAME_POND = 1
FRAME_POND_ISOTHERMAL = 2

# Boundary kinds (same meaning as the solver library's, numbered independently).
BC_OUTFLOW = 0
BC_DIRICHLET = 1
BC_INLET = 2
BC_DIFFUSE = 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction, so the
    x86 and Arm builds round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.c_double
        p = ctypes.c_void_p
        i = ctypes.c_int
        L = _lib
        L.orc_gh1d.argtypes = [i, p, p]
        L.orc_lattice.argtypes = [i, p, p, p]
        L.orc_moment_matrix.argtypes = [i, p, p]
        L.orc_invert.argtypes = [i, p, p]
        L.orc_transfer.argtypes = [i, p, p, p]
        L.orc_eq_lattice.argtypes = [i, d, d, d, d, p]
        L.orc_lift.argtypes = [i, i, p, d, p, p]
        L.orc_project.argtypes = [i, i, p, p, p]
        L.orc_lagrange.argtypes = [i, d, ctypes.c_long, p]
        L.orc_lagrange.restype = None
        L.orc_first_node.argtypes = [i, d]
        L.orc_first_node.restype = ctypes.c_long
        L.orc_create.argtypes = [i, i, i, i, i, i, d, i, i, d]
        L.orc_create.restype = p
        L.orc_destroy.argtypes = [p]
        L.orc_destroy.restype = None
        L.orc_dt.argtypes = [p]
        L.orc_dt.restype = d
        L.orc_init_equilibrium.argtypes = [p, p, p, p, p]
        L.orc_set_pond.argtypes = [p, d, i]
        L.orc_nonconverged.argtypes = [p]
        L.orc_nonconverged.restype = ctypes.c_long
        L.orc_get_frame.argtypes = [p, p, p, p]
        L.orc_set_frame.argtypes = [p, p, p, p]
        L.orc_set_flags.argtypes = [p, p]
        L.orc_get_flags.argtypes = [p, p]
        L.orc_get_flags.restype = None
        L.orc_set_criterion.argtypes = [p, i, d]
        L.orc_set_bc.argtypes = [p, i, i, p, p, p]
        L.orc_step.argtypes = [p, i]
        L.orc_step_cells.argtypes = [p, i, p, p, p]
        L.orc_moments.argtypes = [p, p, p, p, p]
        L.orc_audit.argtypes = [p, p]
        L.orc_get_pops.argtypes = [p, i, p]
        L.orc_set_pops.argtypes = [p, i, p]
        L.orc_set_twopop.argtypes = [p, d, d]
        L.orc_set_pond_ends.argtypes = [p, p, p]
        L.orc_set_viscosity_law.argtypes = [p, d, d, d, d]
        L.orc_set_kn_criterion.argtypes = [p, d, i]
        L.orc_get_gpops.argtypes = [p, i, p]
        L.orc_set_gpops.argtypes = [p, i, p]
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed ({rc})")


# ------------------------------------------------------------ building blocks

def gh1d(n: int):
    """Table I: 1-D Gauss-Hermite nodes (ascending) and weights, T_L = 1."""
    c = np.zeros(n)
    w = np.zeros(n)
    _check(lib().orc_gh1d(n, _ptr(c), _ptr(w)), "gh1d")
    return c, w


def lattice(n: int):
    """Eq. (ci)/(wi): D2Q(n^2) velocities and weights, i = ix + n*iy."""
    Q = n * n
    cx, cy, W = np.zeros(Q), np.zeros(Q), np.zeros(Q)
    _check(lib().orc_lattice(n, _ptr(cx), _ptr(cy), _ptr(W)), "lattice")
    return cx, cy, W


def moment_matrix(n: int, ux: float, uy: float, T: float) -> np.ndarray:
    """Eq. (momf): rows (a, b) = (r % n, r // n), columns populations."""
    M = np.zeros((n * n, n * n))
    lam = _f64([ux, uy, T])
    _check(lib().orc_moment_matrix(n, _ptr(lam), _ptr(M)), "moment_matrix")
    return M


def invert(A) -> np.ndarray:
    A = _f64(A)
    out = np.zeros_like(A)
    _check(lib().orc_invert(A.shape[0], _ptr(A), _ptr(out)), "invert")
    return out


def transfer(n: int, frm, to) -> np.ndarray:
    """Transfer matrix G_lambda^lambda' = M_lambda'^-1 M_lambda, eq. (fll)."""
    G = np.zeros((n * n, n * n))
    a, b = _f64(frm), _f64(to)
    _check(lib().orc_transfer(n, _ptr(a), _ptr(b), _ptr(G)), "transfer")
    return G


def eq_lattice(n: int, rho: float, ux: float, uy: float, T: float = 1.0) -> np.ndarray:
    """Lattice-frame equilibrium f^L = G_{u,T}^{0,T_L} rho W, eqs. (feqL)/(feqL0)."""
    f = np.zeros(n * n)
    _check(lib().orc_eq_lattice(n, rho, ux, uy, T, _ptr(f)), "eq_lattice")
    return f


def lift(nq: int, nQ: int, fq, frame=(0.0, 0.0, 1.0), T_fix: float = 1.0) -> np.ndarray:
    """Lifting f_q -> f_Q, Sec. III.B / App. C (T_fix <= 0: kinetic T of f_q)."""
    fq = _f64(fq)
    out = np.zeros(nQ * nQ)
    lam = _f64(frame)
    _check(lib().orc_lift(nq, nQ, _ptr(lam), T_fix, _ptr(fq), _ptr(out)), "lift")
    return out


def project(nQ: int, nq: int, fQ, frame=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Projection f_Q -> f_q, Sec. III.C / App. C."""
    fQ = _f64(fQ)
    out = np.zeros(nq * nq)
    lam = _f64(frame)
    _check(lib().orc_project(nQ, nq, _ptr(lam), _ptr(fQ), _ptr(out)), "project")
    return out


def lagrange(p: int, xd: float, x0: int) -> np.ndarray:
    """Interpolation functions a_s of eq. (reconstructionPond) on x0..x0+p-1."""
    a = np.zeros(p)
    lib().orc_lagrange(p, xd, x0, _ptr(a))
    return a


def first_node(p: int, xd: float) -> int:
    return int(lib().orc_first_node(p, xd))


# ---------------------------------------------------------------- the solver

class Oracle:
    """Whole-grid oracle state: nx x ny cells, low/high lattices n_lo < n_hi
    (3 = D2Q9, 4 = D2Q16, 5 = D2Q25), relaxation time tau (omega = 1/tau),
    Lagrange order (points = order + 1), frame (FRAME_LATTICE, or one of the
    co-moving frames of Sec. II.C, which need a periodic grid)."""

    def __init__(self, nx, ny, n_lo=3, n_hi=5, tau=0.6, order=3, periodic=(True, True),
                 frame=0, cfl=1.0):
        self.nx, self.ny = nx, ny
        self.frame = frame
        self.periodic = (bool(periodic[0]), bool(periodic[1]))
        self.n = (n_lo, n_hi)
        self.Q = (n_lo * n_lo, n_hi * n_hi)
        h = lib().orc_create(nx, ny, int(periodic[0]), int(periodic[1]), n_lo, n_hi,
                             float(tau), order, frame, float(cfl))
        if not h:
            raise ValueError("oracle: invalid configuration")
        self._h = ctypes.c_void_p(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    @property
    def dt(self) -> float:
        return lib().orc_dt(self._h)

    def init_equilibrium(self, rho, ux, uy, T=None):
        """Lattice frame: f^L(rho, u) (T must be None).  Co-moving frame:
        rho W_i in the frame {u, T} (T = T_L when None), eq. (feqPond)."""
        r, a, b = _f64(rho).ravel(), _f64(ux).ravel(), _f64(uy).ravel()
        t = None if T is None else _f64(np.broadcast_to(T, r.reshape(self.ny, self.nx).shape)).ravel()
        _check(lib().orc_init_equilibrium(self._h, _ptr(r), _ptr(a), _ptr(b),
                                          None if t is None else _ptr(t)), "init")

    def set_twopop(self, cv: float, tau2: float):
        """Two-population co-moving model of Sec. II.B (thermal co-moving
        frame only; before init_equilibrium): C_v = cv, omega_2 = 1 / tau2."""
        _check(lib().orc_set_twopop(self._h, float(cv), float(tau2)), "set_twopop")

    def set_pond_ends(self, left, right):
        """Co-moving frame on a non-periodic x axis: fixed states {rho, u_x,
        u_y, T} beyond the left and right ends (set twopop first)."""
        a, b = _f64(left), _f64(right)
        _check(lib().orc_set_pond_ends(self._h, _ptr(a), _ptr(b)), "set_pond_ends")

    def set_viscosity_law(self, mu1: float, T1: float, s_exp: float, pr: float):
        """mu = mu1 (T / T1)^s_exp and fixed Pr (two-population model)."""
        _check(lib().orc_set_viscosity_law(self._h, float(mu1), float(T1), float(s_exp),
                                           float(pr)), "set_viscosity_law")

    def set_kn_criterion(self, thr: float, interval: int):
        """Knudsen refinement (Sec. IV.C) at once and every `interval` steps."""
        _check(lib().orc_set_kn_criterion(self._h, float(thr), int(interval)), "set_kn_criterion")

    def get_gpops(self, k: int) -> np.ndarray:
        """g populations of lattice k, shape (ny, nx, Q_k), absolute units."""
        out = np.zeros(self.nx * self.ny * self.Q[k])
        _check(lib().orc_get_gpops(self._h, k, _ptr(out)), "get_gpops")
        return out.reshape(self.ny, self.nx, self.Q[k])

    def set_gpops(self, k: int, g):
        g = _f64(g).ravel()
        assert g.size == self.nx * self.ny * self.Q[k]
        _check(lib().orc_set_gpops(self._h, k, _ptr(g)), "set_gpops")

    def set_pond(self, tol: float, maxit: int):
        """Predictor-corrector tolerance and iteration cap (co-moving frame)."""
        _check(lib().orc_set_pond(self._h, tol, maxit), "set_pond")

    def nonconverged(self) -> int:
        """Cell updates whose predictor-corrector stopped at the cap."""
        return int(lib().orc_nonconverged(self._h))

    def get_frame(self):
        """Frames (u_x, u_y, T) the cells' populations live in, each (ny, nx)."""
        n = self.nx * self.ny
        a, b, t = np.zeros(n), np.zeros(n), np.zeros(n)
        _check(lib().orc_get_frame(self._h, _ptr(a), _ptr(b), _ptr(t)), "get_frame")
        shp = (self.ny, self.nx)
        return a.reshape(shp), b.reshape(shp), t.reshape(shp)

    def set_frame(self, ux, uy, T):
        a, b, t = (_f64(np.broadcast_to(v, (self.ny, self.nx))).ravel() for v in (ux, uy, T))
        _check(lib().orc_set_frame(self._h, _ptr(a), _ptr(b), _ptr(t)), "set_frame")

    def set_flags(self, flags):
        f = np.ascontiguousarray(flags, dtype=np.uint8).ravel()
        _check(lib().orc_set_flags(self._h, _ptr(f)), "set_flags")

    def get_flags(self) -> np.ndarray:
        f = np.zeros(self.nx * self.ny, dtype=np.uint8)
        lib().orc_get_flags(self._h, _ptr(f))
        return f.reshape(self.ny, self.nx)

    def set_criterion(self, kind: int, thr: float):
        _check(lib().orc_set_criterion(self._h, kind, thr), "set_criterion")

    def set_bc(self, side: int, kind: int, rho=None, ux=None, uy=None):
        arrs = [None if a is None else _f64(a) for a in (rho, ux, uy)]
        ptrs = [None if a is None else _ptr(a) for a in arrs]
        _check(lib().orc_set_bc(self._h, side, kind, *ptrs), "set_bc")

    def step(self, n: int = 1):
        _check(lib().orc_step(self._h, n), "step")

    def step_cells(self, cells, with_frame: bool = False):
        """One step's post-collision vectors of the given cells (x + nx*y),
        without advancing the state: shape (m, 25), the first Q of the cell's
        lattice valid.  with_frame (co-moving frame): also the (m, 3) frames
        {u_x, u_y, T} the vectors live in."""
        c = np.ascontiguousarray(cells, dtype=np.int64)
        out = np.zeros((len(c), 25))
        lam = np.zeros((len(c), 3))
        _check(lib().orc_step_cells(self._h, len(c), _ptr(c), _ptr(out),
                                    _ptr(lam) if with_frame else None), "step_cells")
        return (out, lam) if with_frame else out

    def moments(self):
        n = self.nx * self.ny
        r, a, b, t = (np.zeros(n) for _ in range(4))
        _check(lib().orc_moments(self._h, _ptr(r), _ptr(a), _ptr(b), _ptr(t)), "moments")
        shp = (self.ny, self.nx)
        return r.reshape(shp), a.reshape(shp), b.reshape(shp), t.reshape(shp)

    def audit(self) -> np.ndarray:
        out = np.zeros(4)
        _check(lib().orc_audit(self._h, _ptr(out)), "audit")
        return out

    def get_pops(self, k: int) -> np.ndarray:
        """Populations of lattice k (0 low, 1 high), shape (ny, nx, Q_k)."""
        out = np.zeros(self.nx * self.ny * self.Q[k])
        _check(lib().orc_get_pops(self._h, k, _ptr(out)), "get_pops")
        return out.reshape(self.ny, self.nx, self.Q[k])

    def set_pops(self, k: int, f):
        f = _f64(f).ravel()
        assert f.size == self.nx * self.ny * self.Q[k]
        _check(lib().orc_set_pops(self._h, k, _ptr(f)), "set_pops")
