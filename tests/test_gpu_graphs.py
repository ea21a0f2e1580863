"""slbm_step replays pairs of lattice-frame steps as CUDA graphs once the
kernels have run directly; single steps (n = 1) and traced steps always
launch directly.  The two paths launch the same kernels with the same
arguments, so their results agree bit for bit: checked on the jet
(boundaries, Mach criterion flipping cells every step) in FP32 and FP16
(whose stochastic rounding key is a device counter), across a boundary
change (which drops the captured graphs), and with the learned indicator
(graph chunks between its evaluations)."""
import numpy as np
import pytest

from paper_2102_12559_gb300 import slbm
from paper_2102_12559_gb300 import workloads as WL

pytestmark = pytest.mark.gpu


def jet_solver(precision, nx=256, ny=128):
    J = WL.free_jet(nx, ny, slot=16, ma_jet=0.5, ma_co=0.05)
    g = slbm.Solver(nx, ny, 3, 5, tau=0.55, periodic=(False, False), precision=precision)
    g.init_equilibrium(J["rho"], J["ux"], J["uy"])
    g.set_boundary(slbm.SLBM_SIDE_XMIN, slbm.SLBM_BC_INLET, None, J["in_ux"], J["in_uy"])
    g.set_boundary(slbm.SLBM_SIDE_XMAX, slbm.SLBM_BC_OUTFLOW)
    for side in (slbm.SLBM_SIDE_YMIN, slbm.SLBM_SIDE_YMAX):
        g.set_boundary(side, slbm.SLBM_BC_DIRICHLET, np.full(nx, J["fs_rho"]),
                       np.full(nx, J["fs_ux"]), np.full(nx, J["fs_uy"]))
    g.set_criterion(slbm.SLBM_CRIT_MACH, 0.3)
    return g, J


def state(g):
    return [g.get_pops(0), g.get_pops(1), g.get_flags()]


def assert_same(a, b):
    for x, y in zip(state(a), state(b)):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", [slbm.SLBM_FP32, slbm.SLBM_FP16])
def test_graph_steps_equal_direct_steps(precision):
    a, J = jet_solver(precision)
    b, _ = jet_solver(precision)
    for _ in range(41):
        a.step(1)                                  # direct launches only
    b.step(1)
    b.step(40)                                     # 20 graph replays
    assert_same(a, b)
    # a boundary change drops the graphs; both go on from the same state
    u2 = 1.1 * J["in_ux"]
    for g in (a, b):
        g.set_boundary(slbm.SLBM_SIDE_XMIN, slbm.SLBM_BC_INLET, None, u2, J["in_uy"])
    for _ in range(13):
        a.step(1)
    b.step(13)                                     # 6 replays and one direct step
    assert_same(a, b)
    a.close()
    b.close()


def test_graph_steps_with_learned_indicator():
    w = {"w1": np.zeros((16, 32)), "b1": np.zeros(32), "w2": np.eye(32), "b2": np.zeros(32),
         "w3": np.zeros(32), "b3": -0.9}
    w["w1"][15, 0] = 1.0                           # logit = 3|u| - 0.9: the Mach criterion
    w["w3"][0] = 1.0
    a, _ = jet_solver(slbm.SLBM_FP32)
    b, _ = jet_solver(slbm.SLBM_FP32)
    for g in (a, b):
        g.set_indicator(w, interval=7)
        g.set_criterion(slbm.SLBM_CRIT_MLP, 0.0)
    for _ in range(30):
        a.step(1)
    b.step(1)
    b.step(29)                                     # chunks of 6 / 7 steps between evaluations
    assert_same(a, b)
    assert b.get_flags().sum() > 0
    a.close()
    b.close()
