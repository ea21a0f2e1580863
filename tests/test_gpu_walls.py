"""GPU parity of the diffuse-reflection wall (SLBM_BC_DIFFUSE) against the FP64
oracle: a channel periodic along x with walls at y = 0 and y = ny - 1.

Tolerances as for the other boundaries: FP64 differs from the oracle only in
rounding order (1e-13 on single-step populations, 1e-12 relative L2 on the
moments after 300 steps); FP32 1e-5 relative L2 after 300 steps.
"""
import numpy as np
import pytest

import oracle as O
from paper_2102_12559_gb300 import workloads as WL
from paper_2102_12559_gb300 import slbm

pytestmark = pytest.mark.gpu

FP32, FP64 = slbm.SLBM_FP32, slbm.SLBM_FP64


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def walls(obj, nx, uw_lo, uw_hi, gpu):
    kind = slbm.SLBM_BC_DIFFUSE if gpu else O.BC_DIFFUSE
    lo, hi = (slbm.SLBM_SIDE_YMIN, slbm.SLBM_SIDE_YMAX) if gpu else (2, 3)
    fn = obj.set_boundary if gpu else obj.set_bc
    fn(lo, kind, None, np.full(nx, uw_lo), np.zeros(nx))
    fn(hi, kind, None, np.full(nx, uw_hi), np.zeros(nx))


def pair(nx, ny, lo, hi, tau, precision, fields, flags, uw):
    g = slbm.Solver(nx, ny, lo, hi, tau=tau, periodic=(True, False), precision=precision)
    o = O.Oracle(nx, ny, lo, hi, tau=tau, periodic=(True, False))
    for obj, gpu in ((g, True), (o, False)):
        obj.init_equilibrium(*fields)
        obj.set_flags(flags)
        walls(obj, nx, -uw, uw, gpu)
    return g, o


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-13), (FP32, 2e-6)])
def test_flow_moving_with_the_walls_stays_uniform(precision, tol):
    nx, ny = 40, 24
    g = slbm.Solver(nx, ny, 3, 5, tau=0.7, periodic=(True, False), precision=precision)
    g.init_equilibrium(*WL.uniform(nx, ny, 1.0, 0.08, 0.0))
    fl = np.zeros((ny, nx), np.uint8)
    fl[:5] = 1
    g.set_flags(fl)
    walls(g, nx, 0.08, 0.08, True)
    g.step(10)
    r, u, v, _ = g.moments()
    assert abs(r - 1).max() < tol and abs(u - 0.08).max() < tol and abs(v).max() < tol


@pytest.mark.parametrize("lo,hi", [(3, 4), (3, 5), (4, 5)])
def test_one_step_fp64(lo, hi):
    nx, ny = 37, 21
    fields = WL.perturbed(nx, ny, seed=12, amp_rho=0.04, amp_u=0.1)
    fl = np.zeros((ny, nx), np.uint8)
    fl[:3] = 1
    fl[-4:] = 1
    g, o = pair(nx, ny, lo, hi, 0.65, FP64, fields, fl, 0.07)
    g.step(2)
    o.step(2)
    for k in (0, 1):
        m = fl == k
        np.testing.assert_allclose(g.get_pops(k)[m], o.get_pops(k)[m], rtol=0, atol=1e-13)


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-12), (FP32, 1e-5)])
def test_couette_300_steps(precision, tol):
    """Shear-driven Couette flow, the high-order lattice in the wall layers."""
    nx, ny = 8, 32
    fl = np.zeros((ny, nx), np.uint8)
    fl[:4] = 1
    fl[-4:] = 1
    g, o = pair(nx, ny, 3, 4, 0.9, precision, WL.uniform(nx, ny), fl, 0.05)
    g.step(300)
    o.step(300)
    mg, mo = g.moments(), o.moments()
    assert rel_l2(mg[0], mo[0]) < tol
    assert rel_l2(np.stack(mg[1:3]), np.stack(mo[1:3])) < tol
    ag, ao = g.audit(), o.audit()
    assert abs(ag[0] / ao[0] - 1) < tol


def test_diffuse_wall_needs_periodic_axis_along_it():
    g = slbm.Solver(32, 32, 3, 5, tau=0.6, periodic=(False, False))
    with pytest.raises(slbm.SlbmError):
        g.set_boundary(slbm.SLBM_SIDE_YMIN, slbm.SLBM_BC_DIFFUSE, None, np.zeros(32), np.zeros(32))
