"""Thin ctypes binding of ``libslbm.so`` (the C ABI in ``include/slbm.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  The functions keep the C names (``slbm_create``,
``slbm_step`` ...) and take numpy arrays for host buffers; ``Solver`` wraps a
handle whose device workspace and stream come from PyTorch.

There is no CPU fallback: loading fails loudly when the library has not been
built or no CUDA device is present.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

# ---- constants mirrored from include/slbm.h
SLBM_OK, SLBM_EINVAL, SLBM_ENOMEM, SLBM_ECUDA = 0, -1, -2, -3
SLBM_ENONFINITE, SLBM_ENOCONV, SLBM_ETIMEOUT, SLBM_ESTATE = -4, -5, -6, -7
SLBM_D2Q9, SLBM_D2Q16, SLBM_D2Q25 = 3, 4, 5
SLBM_FRAME_LATTICE, SLBM_FRAME_POND, SLBM_FRAME_POND_ISOTHERMAL = 0, 1, 2
SLBM_POND_REACH = 5
SLBM_FP32, SLBM_FP64, SLBM_FP16, SLBM_FX16 = 0, 1, 2, 3
SLBM_BC_OUTFLOW, SLBM_BC_DIRICHLET, SLBM_BC_INLET, SLBM_BC_DIFFUSE = 0, 1, 2, 3
SLBM_SIDE_XMIN, SLBM_SIDE_XMAX, SLBM_SIDE_YMIN, SLBM_SIDE_YMAX = 0, 1, 2, 3
SLBM_CRIT_NONE, SLBM_CRIT_MACH, SLBM_CRIT_MLP, SLBM_CRIT_MLP_REFINE = 0, 1, 2, 3

EXPORTS = [
    "slbm_workspace_bytes", "slbm_create", "slbm_create_in", "slbm_destroy", "slbm_get_info",
    "slbm_init_equilibrium", "slbm_set_flags", "slbm_get_flags", "slbm_set_criterion",
    "slbm_set_boundary", "slbm_step", "slbm_sync", "slbm_moments", "slbm_moments_device",
    "slbm_audit", "slbm_get_pops", "slbm_set_pops", "slbm_get_state", "slbm_set_state",
    "slbm_profile", "slbm_profile_read", "slbm_audit_dense_noalloc", "slbm_last_error",
    "slbm_set_pond", "slbm_get_frame", "slbm_set_frame",
    "slbm_set_indicator", "slbm_indicator_eval", "slbm_lattice_loss", "slbm_mlp_train",
    "slbm_set_twopop", "slbm_get_gpops", "slbm_set_gpops", "slbm_set_rows",
    "slbm_set_viscosity_law", "slbm_tune", "slbm_set_kn_criterion", "slbm_set_channels",
]
SLBM_PROFILE_KERNELS = 2
KERNEL_NAMES = ("stream_collide", "post_step")


class slbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int)]


class slbm_info_t(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("omega", ctypes.c_double),
                ("q_lo", ctypes.c_int), ("q_hi", ctypes.c_int), ("halo", ctypes.c_int),
                ("pitch", ctypes.c_int), ("rows", ctypes.c_int), ("precision", ctypes.c_int),
                ("kernels_per_step", ctypes.c_int), ("workspace_bytes", ctypes.c_size_t),
                ("steps", ctypes.c_longlong)]


class SlbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"slbm error {code}: {msg}")
        self.code = code


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libslbm.so (building it first if allowed and missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {_build.LIB} is missing: run __graft_entry__.build()")
        _build.build()
    L = ctypes.CDLL(_build.LIB)
    p, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    L.slbm_workspace_bytes.argtypes = [P(slbm_grid), i, i, i, i, P(ctypes.c_size_t)]
    L.slbm_create.argtypes = [P(slbm_grid), i, i, d, i, i, i, p, P(p)]
    L.slbm_create_in.argtypes = [P(slbm_grid), i, i, d, i, i, i, p, p, ctypes.c_size_t, P(p)]
    L.slbm_destroy.argtypes = [p]
    L.slbm_get_info.argtypes = [p, P(slbm_info_t)]
    L.slbm_init_equilibrium.argtypes = [p, p, p, p, p]
    L.slbm_set_flags.argtypes = [p, p]
    L.slbm_get_flags.argtypes = [p, p]
    L.slbm_set_criterion.argtypes = [p, i, d]
    L.slbm_set_boundary.argtypes = [p, i, i, p, p, p]
    L.slbm_step.argtypes = [p, i]
    L.slbm_sync.argtypes = [p]
    L.slbm_moments.argtypes = [p, p, p, p, p]
    L.slbm_moments_device.argtypes = [p, p, p, p, p]
    L.slbm_audit.argtypes = [p, p]
    L.slbm_get_pops.argtypes = [p, i, p]
    L.slbm_set_pops.argtypes = [p, i, p]
    L.slbm_get_state.argtypes = [p, p, P(ctypes.c_size_t)]
    L.slbm_set_state.argtypes = [p, p, ctypes.c_size_t]
    L.slbm_profile.argtypes = [p, i]
    L.slbm_profile_read.argtypes = [p, p, P(ctypes.c_longlong)]
    L.slbm_audit_dense_noalloc.argtypes = [p, i, i, i, p, p]
    L.slbm_last_error.argtypes = [p]
    L.slbm_set_pond.argtypes = [p, d, i]
    L.slbm_set_twopop.argtypes = [p, d, d]
    L.slbm_get_gpops.argtypes = [p, i, p]
    L.slbm_set_gpops.argtypes = [p, i, p]
    L.slbm_set_rows.argtypes = [p, p, p]
    L.slbm_set_viscosity_law.argtypes = [p, p, p, d, d]
    L.slbm_tune.argtypes = [p, i, p, p]
    L.slbm_set_kn_criterion.argtypes = [p, d, i]
    L.slbm_set_channels.argtypes = [p, i, p, p, p, p, p]
    L.slbm_get_frame.argtypes = [p, p, p, p]
    L.slbm_set_frame.argtypes = [p, p, p, p]
    L.slbm_set_indicator.argtypes = [p, p, p, p, p, p, ctypes.c_float, i]
    L.slbm_indicator_eval.argtypes = [p, p, p, p]
    L.slbm_lattice_loss.argtypes = [p, p]
    L.slbm_mlp_train.argtypes = [p, p, ctypes.c_longlong, p, i, i, p, i, p, p, p, p, p]
    L.slbm_last_error.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name != "slbm_last_error":
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, h=None):
    if rc != SLBM_OK:
        msg = load().slbm_last_error(h)
        raise SlbmError(rc, msg.decode() if msg else "")


def _f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    if a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


# ---------------------------------------------------------------- C names

def slbm_workspace_bytes(nx, ny, periodic_x, periodic_y, lat_lo, lat_hi, interp_order, precision):
    g = slbm_grid(nx, ny, int(periodic_x), int(periodic_y))
    out = ctypes.c_size_t(0)
    _check(load().slbm_workspace_bytes(ctypes.byref(g), lat_lo, lat_hi, interp_order, precision,
                                       ctypes.byref(out)))
    return out.value


def slbm_create(nx, ny, periodic_x, periodic_y, lat_lo, lat_hi, tau, interp_order=3,
                frame=SLBM_FRAME_LATTICE, precision=SLBM_FP32, stream=0):
    g = slbm_grid(nx, ny, int(periodic_x), int(periodic_y))
    h = ctypes.c_void_p()
    _check(load().slbm_create(ctypes.byref(g), lat_lo, lat_hi, float(tau), interp_order, frame,
                              precision, ctypes.c_void_p(stream), ctypes.byref(h)))
    return h


def slbm_create_in(nx, ny, periodic_x, periodic_y, lat_lo, lat_hi, tau, interp_order, frame,
                   precision, stream, workspace_ptr, workspace_bytes):
    g = slbm_grid(nx, ny, int(periodic_x), int(periodic_y))
    h = ctypes.c_void_p()
    _check(load().slbm_create_in(ctypes.byref(g), lat_lo, lat_hi, float(tau), interp_order, frame,
                                 precision, ctypes.c_void_p(stream), ctypes.c_void_p(workspace_ptr),
                                 workspace_bytes, ctypes.byref(h)))
    return h


def slbm_destroy(h):
    _check(load().slbm_destroy(h))


def slbm_get_info(h) -> slbm_info_t:
    info = slbm_info_t()
    _check(load().slbm_get_info(h, ctypes.byref(info)), h)
    return info


def slbm_init_equilibrium(h, n, rho, ux, uy, T=None):
    r, a, b = _f64(rho, n), _f64(ux, n), _f64(uy, n)
    t = None if T is None else _f64(T, n)
    _check(load().slbm_init_equilibrium(h, _ptr(r), _ptr(a), _ptr(b),
                                        None if t is None else _ptr(t)), h)


def slbm_set_indicator(h, w1, b1, w2, b2, w3, b3, interval=10):
    """MLP weights (16x32, 32, 32x32, 32, 32, scalar), host floats."""
    a = [np.ascontiguousarray(v, dtype=np.float32).ravel() for v in (w1, b1, w2, b2, w3)]
    assert [x.size for x in a] == [512, 32, 1024, 32, 32]
    _check(load().slbm_set_indicator(h, *(_ptr(x) for x in a), float(b3), int(interval)), h)


def slbm_indicator_eval(h, n, features=True, logits=False, flags=False):
    fe = np.zeros((n, 16), np.float32) if features else None
    lo = np.zeros(n, np.float32) if logits else None
    fl = np.zeros(n, np.uint8) if flags else None
    _check(load().slbm_indicator_eval(h, *(None if v is None else _ptr(v) for v in (fe, lo, fl))), h)
    return fe, lo, fl


def slbm_lattice_loss(h, n):
    out = np.zeros(n, np.float64)
    _check(load().slbm_lattice_loss(h, _ptr(out)), h)
    return out


MLP_PARAMS = 16 * 32 + 32 + 32 * 32 + 32 + 32 + 1


def slbm_mlp_train(x, y, idx, hyper, t0, params, adam, want_loss=True, want_grad=False,
                   stream=0):
    """GPU training steps (see include/slbm.h).  x (n, 16), y (n,), idx
    (steps, batch) int; params (1633,) and adam (2, 1633) float32 arrays are
    updated in place.  Returns (per-step losses, last gradient)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32).ravel()
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    if x.ndim != 2 or x.shape[1] != 16 or y.size != x.shape[0] or idx.ndim != 2:
        raise ValueError("x (n, 16), y (n,), idx (steps, batch)")
    if params.dtype != np.float32 or params.size != MLP_PARAMS or not params.flags.c_contiguous:
        raise ValueError("params: contiguous float32, 1633 values")
    if adam.dtype != np.float32 or adam.size != 2 * MLP_PARAMS or not adam.flags.c_contiguous:
        raise ValueError("adam: contiguous float32, 2 x 1633 values")
    steps, batch = idx.shape
    hp = _f64(hyper, 4)
    loss = np.zeros(steps, np.float32) if want_loss else None
    grad = np.zeros(MLP_PARAMS, np.float32) if want_grad else None
    _check(load().slbm_mlp_train(_ptr(x), _ptr(y), x.shape[0], _ptr(idx), steps, batch, _ptr(hp),
                                 int(t0), _ptr(params), _ptr(adam), _ptr(loss), _ptr(grad),
                                 ctypes.c_void_p(stream)))
    return loss, grad


def slbm_set_pond(h, tol, max_iter):
    _check(load().slbm_set_pond(h, float(tol), int(max_iter)), h)


def slbm_set_twopop(h, cv, tau2):
    _check(load().slbm_set_twopop(h, float(cv), float(tau2)), h)


def slbm_set_rows(h, ny, lens, ends):
    a = np.ascontiguousarray(np.asarray(lens, dtype=np.int32).ravel())
    b = _f64(ends, 8 * ny)
    if a.size != ny:
        raise ValueError("one length per row")
    _check(load().slbm_set_rows(h, _ptr(a), _ptr(b)), h)


def slbm_set_channels(h, x0, width, uw_lo, uw_hi, tau):
    n = len(x0)
    a = np.ascontiguousarray(np.asarray(x0, dtype=np.int32).ravel())
    b = np.ascontiguousarray(np.asarray(width, dtype=np.int32).ravel())
    c, d, e = _f64(uw_lo, n), _f64(uw_hi, n), _f64(tau, n)
    if b.size != n:
        raise ValueError("one width per channel")
    _check(load().slbm_set_channels(h, n, _ptr(a), _ptr(b), _ptr(c), _ptr(d), _ptr(e)), h)


def slbm_set_viscosity_law(h, ny, mu1, T1, s_exp, pr):
    a, b = _f64(mu1, ny), _f64(T1, ny)
    _check(load().slbm_set_viscosity_law(h, _ptr(a), _ptr(b), float(s_exp), float(pr)), h)


def slbm_tune(h, reps):
    bx, by = ctypes.c_int(0), ctypes.c_int(0)
    _check(load().slbm_tune(h, int(reps), ctypes.byref(bx), ctypes.byref(by)), h)
    return bx.value, by.value


def slbm_get_gpops(h, k, Q, n):
    out = np.zeros(Q * n)
    _check(load().slbm_get_gpops(h, k, _ptr(out)), h)
    return out


def slbm_set_gpops(h, k, Q, n, pops):
    a = _f64(pops, Q * n)
    _check(load().slbm_set_gpops(h, k, _ptr(a)), h)


def slbm_get_frame(h, n):
    out = [np.zeros(n) for _ in range(3)]
    _check(load().slbm_get_frame(h, *(_ptr(a) for a in out)), h)
    return out


def slbm_set_frame(h, n, ux, uy, T):
    a, b, t = _f64(ux, n), _f64(uy, n), _f64(T, n)
    _check(load().slbm_set_frame(h, _ptr(a), _ptr(b), _ptr(t)), h)


def slbm_set_flags(h, n, flags):
    f = np.ascontiguousarray(flags, dtype=np.uint8).ravel()
    assert f.size == n
    _check(load().slbm_set_flags(h, _ptr(f)), h)


def slbm_get_flags(h, n):
    f = np.zeros(n, dtype=np.uint8)
    _check(load().slbm_get_flags(h, _ptr(f)), h)
    return f


def slbm_set_criterion(h, kind, threshold):
    _check(load().slbm_set_criterion(h, kind, float(threshold)), h)


def slbm_set_boundary(h, side, kind, length, rho=None, ux=None, uy=None):
    arrs = [None if a is None else _f64(a, length) for a in (rho, ux, uy)]
    _check(load().slbm_set_boundary(h, side, kind, *[_ptr(a) for a in arrs]), h)


def slbm_step(h, n=1):
    _check(load().slbm_step(h, int(n)), h)


def slbm_sync(h):
    _check(load().slbm_sync(h), h)


def slbm_moments(h, n, rho=None, ux=None, uy=None, T=None):
    """Host moments; pass preallocated float64 arrays (e.g. pinned) or None
    to allocate."""
    outs = [np.zeros(n) if a is None else a for a in (rho, ux, uy, T)]
    _check(load().slbm_moments(h, *[_ptr(a) for a in outs]), h)
    return outs


def slbm_moments_device(h, rho_ptr=0, ux_ptr=0, uy_ptr=0, T_ptr=0):
    ptrs = [ctypes.c_void_p(p) if p else None for p in (rho_ptr, ux_ptr, uy_ptr, T_ptr)]
    _check(load().slbm_moments_device(h, *ptrs), h)


def slbm_audit(h):
    out = np.zeros(4)
    _check(load().slbm_audit(h, _ptr(out)), h)
    return out


def slbm_get_pops(h, k, Q, n):
    out = np.zeros(Q * n)
    _check(load().slbm_get_pops(h, k, _ptr(out)), h)
    return out


def slbm_set_pops(h, k, Q, n, pops):
    a = _f64(pops, Q * n)
    _check(load().slbm_set_pops(h, k, _ptr(a)), h)


def slbm_get_state(h) -> bytes:
    size = ctypes.c_size_t(0)
    _check(load().slbm_get_state(h, None, ctypes.byref(size)), h)
    buf = ctypes.create_string_buffer(size.value)
    _check(load().slbm_get_state(h, buf, ctypes.byref(size)), h)
    return buf.raw


def slbm_set_state(h, state: bytes):
    buf = ctypes.create_string_buffer(state, len(state))
    _check(load().slbm_set_state(h, buf, len(state)), h)


def slbm_profile(h, enable):
    _check(load().slbm_profile(h, int(bool(enable))), h)


def slbm_profile_read(h):
    """(per-kernel summed device ms over the profiled steps, steps)."""
    ms = np.zeros(SLBM_PROFILE_KERNELS)
    n = ctypes.c_longlong(0)
    _check(load().slbm_profile_read(h, _ptr(ms), ctypes.byref(n)), h)
    return ms, n.value


def slbm_audit_dense_noalloc(f_ptr, lattice, nx, ny, out_ptr, stream=0):
    """Allocation-free FP64 audit of a dense FP32 population field (device
    pointers; see include/slbm.h)."""
    _check(load().slbm_audit_dense_noalloc(ctypes.c_void_p(f_ptr), lattice, nx, ny,
                                           ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream)))


def slbm_last_error(h=None) -> str:
    m = load().slbm_last_error(h)
    return m.decode() if m else ""


# ------------------------------------------------------------ convenience

class Solver:
    """One handle on the current CUDA device.  The device workspace is a torch
    uint8 tensor (PyTorch's allocator) and kernels run on torch's current
    stream, so the library composes with torch code.  Host arrays are
    (ny, nx) numpy arrays, x fastest."""

    def __init__(self, nx, ny, lat_lo=SLBM_D2Q9, lat_hi=SLBM_D2Q25, tau=0.6, interp_order=3,
                 periodic=(True, True), precision=SLBM_FP32, stream=None, torch_workspace=True,
                 frame=SLBM_FRAME_LATTICE):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("slbm.Solver needs a CUDA device (no CPU fallback)")
        self.nx, self.ny = nx, ny
        self.n = nx * ny
        self.lat = (lat_lo, lat_hi)
        self.Q = (lat_lo * lat_lo, lat_hi * lat_hi)
        self.precision = precision
        self.frame = frame
        st = torch.cuda.current_stream() if stream is None else stream
        self.stream = st
        self._ws = None
        if torch_workspace:
            nbytes = slbm_workspace_bytes(nx, ny, periodic[0], periodic[1], lat_lo, lat_hi,
                                          interp_order, precision)
            self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
            ptr = (self._ws.data_ptr() + 255) // 256 * 256
            self.h = slbm_create_in(nx, ny, periodic[0], periodic[1], lat_lo, lat_hi, tau,
                                    interp_order, frame, precision, st.cuda_stream,
                                    ptr, nbytes)
        else:
            self.h = slbm_create(nx, ny, periodic[0], periodic[1], lat_lo, lat_hi, tau,
                                 interp_order, frame, precision, st.cuda_stream)

    def close(self):
        if getattr(self, "h", None) is not None:
            slbm_destroy(self.h)
            self.h = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self) -> slbm_info_t:
        return slbm_get_info(self.h)

    @property
    def dt(self) -> float:
        return self.info.dt

    def init_equilibrium(self, rho, ux, uy, T=None):
        if T is not None:
            T = np.broadcast_to(np.asarray(T, dtype=np.float64), (self.ny, self.nx))
        slbm_init_equilibrium(self.h, self.n, rho, ux, uy, T)

    def set_pond(self, tol, max_iter):
        slbm_set_pond(self.h, tol, max_iter)

    def set_twopop(self, cv, tau2):
        """Two-population co-moving model (before init_equilibrium)."""
        slbm_set_twopop(self.h, cv, tau2)

    def set_rows(self, lens, ends):
        """Rows as independent quasi-1-D instances: lengths (ny) and end
        states (ny, 2, 4) = left / right {rho, u_x, u_y, T}."""
        slbm_set_rows(self.h, self.ny, lens, np.asarray(ends, dtype=np.float64).reshape(-1))

    def set_channels(self, x0, width, uw_lo, uw_hi, tau):
        """Independent channels side by side along x (diffuse walls on their x
        sides moving along y, periodic y, own tau each; see slbm.h)."""
        slbm_set_channels(self.h, x0, width, uw_lo, uw_hi, tau)

    def set_viscosity_law(self, mu1, T1, s_exp=0.5, pr=2.0 / 3.0):
        slbm_set_viscosity_law(self.h, self.ny, np.broadcast_to(mu1, (self.ny,)),
                               np.broadcast_to(T1, (self.ny,)), s_exp, pr)

    def set_kn_criterion(self, thr=0.02, interval=10):
        """Knudsen refinement of batched rows, at once and every `interval` steps."""
        _check(load().slbm_set_kn_criterion(self.h, float(thr), int(interval)), self.h)

    def tune(self, reps=5):
        """Pick the fastest block shape of the co-moving step; returns it."""
        return slbm_tune(self.h, reps)

    def get_gpops(self, k):
        """g populations of lattice k as (ny, nx, Q_k), absolute units."""
        Q = self.Q[k]
        a = slbm_get_gpops(self.h, k, Q, self.n).reshape(Q, self.ny, self.nx)
        return np.moveaxis(a, 0, -1)

    def set_gpops(self, k, pops):
        Q = self.Q[k]
        a = np.moveaxis(np.asarray(pops, dtype=np.float64).reshape(self.ny, self.nx, Q), -1, 0)
        slbm_set_gpops(self.h, k, Q, self.n, np.ascontiguousarray(a))

    def set_indicator(self, weights, interval=10):
        """weights: dict w1 (16x32), b1 (32), w2 (32x32), b2 (32), w3 (32), b3."""
        slbm_set_indicator(self.h, weights["w1"], weights["b1"], weights["w2"], weights["b2"],
                           weights["w3"], weights["b3"], interval)

    def lattice_loss(self):
        """(ny, nx) per-cell lattice loss of one step; the state advances one
        high-order step (see include/slbm.h)."""
        return slbm_lattice_loss(self.h, self.n).reshape(self.ny, self.nx)

    def indicator_eval(self, features=True, logits=False, flags=False):
        """(features (ny, nx, 16), logits (ny, nx), flags (ny, nx)); unrequested are None."""
        fe, lo, fl = slbm_indicator_eval(self.h, self.n, features, logits, flags)
        s = (self.ny, self.nx)
        return (None if fe is None else fe.reshape(self.ny, self.nx, 16),
                None if lo is None else lo.reshape(s), None if fl is None else fl.reshape(s))

    def get_frame(self):
        s = (self.ny, self.nx)
        return tuple(a.reshape(s) for a in slbm_get_frame(self.h, self.n))

    def set_frame(self, ux, uy, T):
        b = lambda v: np.broadcast_to(np.asarray(v, dtype=np.float64), (self.ny, self.nx))
        slbm_set_frame(self.h, self.n, b(ux), b(uy), b(T))

    def set_flags(self, flags):
        slbm_set_flags(self.h, self.n, flags)

    def get_flags(self):
        return slbm_get_flags(self.h, self.n).reshape(self.ny, self.nx)

    def set_criterion(self, kind, thr=0.3):
        slbm_set_criterion(self.h, kind, thr)

    def set_boundary(self, side, kind, rho=None, ux=None, uy=None):
        length = self.ny if side < 2 else self.nx
        slbm_set_boundary(self.h, side, kind, length, rho, ux, uy)

    def step(self, n=1):
        slbm_step(self.h, n)

    def sync(self):
        slbm_sync(self.h)

    def moments(self):
        r, u, v, T = slbm_moments(self.h, self.n)
        s = (self.ny, self.nx)
        return r.reshape(s), u.reshape(s), v.reshape(s), T.reshape(s)

    def audit(self):
        return slbm_audit(self.h)

    def get_pops(self, k):
        """Populations of lattice k as (ny, nx, Q_k) (the oracle's order)."""
        Q = self.Q[k]
        a = slbm_get_pops(self.h, k, Q, self.n).reshape(Q, self.ny, self.nx)
        return np.moveaxis(a, 0, -1)

    def set_pops(self, k, pops):
        Q = self.Q[k]
        a = np.moveaxis(np.asarray(pops, dtype=np.float64).reshape(self.ny, self.nx, Q), -1, 0)
        slbm_set_pops(self.h, k, Q, self.n, np.ascontiguousarray(a))

    def profile(self, enable=True):
        slbm_profile(self.h, enable)

    def profile_read(self):
        return slbm_profile_read(self.h)

    def get_state(self) -> bytes:
        return slbm_get_state(self.h)

    def set_state(self, s: bytes):
        slbm_set_state(self.h, s)
