"""GPU parity of batched quasi-one-dimensional co-moving instances (the shock
structure setting of Sec. IV.C): every row of the grid an independent
instance with its own length and fixed end states, two-population model with
the hard-sphere viscosity law, D2Q16 with D2Q25 inside the shock.  Each row
is compared with an oracle run of that instance alone (len x 1 grid, periodic
y, fixed ends).  Inputs: Rankine-Hugoniot end states joined by a tanh ramp,
short instances (40-64 cells) with a mean free path of 4 cells so the
relaxation times stay moderate; Mach 1.3-3.

Tolerances: FP64 1e-11 relative L2 on rho, u_x, T per row after 4 steps
(only rounding order and the frame of the quasi-equilibria differ); FP32
1e-5; u_y, zero in exact arithmetic, below the same fraction of max |u_x|."""
import numpy as np
import pytest

import oracle as O
from paper_2102_12559_gb300 import workloads as WL
from paper_2102_12559_gb300 import slbm

pytestmark = pytest.mark.gpu

CV, PR = 1.5, 2.0 / 3.0


def instances():
    b = WL.shock_batch(6, seed=5, mach_range=(1.3, 3.0), len_range=(40, 64), cells_per_mfp=4.0)
    return b


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def flags_of(inst, nx, w=8):
    L = inst["len"]
    x = np.arange(nx)
    return ((np.abs(x - 0.5 * L) < w) & (x < L)).astype(np.uint8)


@pytest.mark.parametrize("precision,tol", [(slbm.SLBM_FP64, 1e-11), (slbm.SLBM_FP32, 1e-5)])
def test_rows_match_single_instance_oracle(precision, tol):
    b = instances()
    nx, ny, steps = 64, len(b), 4
    g = slbm.Solver(nx, ny, 4, 5, tau=0.7, precision=precision, frame=slbm.SLBM_FRAME_POND)
    g.set_twopop(CV, 0.8)
    prof = [WL.shock_profile(i, nx) for i in b]
    rho = np.stack([p[0] for p in prof]); ux = np.stack([p[1] for p in prof])
    T = np.stack([p[2] for p in prof])
    g.init_equilibrium(rho, ux, np.zeros_like(rho), T)
    ends = np.array([[(i["left"][0], i["left"][1], 0.0, i["left"][2]),
                      (i["right"][0], i["right"][1], 0.0, i["right"][2])] for i in b])
    g.set_rows([i["len"] for i in b], ends)
    g.set_viscosity_law([i["mu1"] for i in b], [i["T1"] for i in b], 0.5, PR)
    g.set_flags(np.stack([flags_of(i, nx) for i in b]))
    g.step(steps)
    gm = g.moments()
    for r, inst in enumerate(b):
        L = inst["len"]
        o = O.Oracle(L, 1, 4, 5, tau=0.7, frame=O.FRAME_POND, periodic=(False, True))
        o.set_twopop(CV, 0.8)
        o.set_pond_ends(ends[r, 0], ends[r, 1])
        o.set_viscosity_law(inst["mu1"], inst["T1"], 0.5, PR)
        o.init_equilibrium(rho[r:r + 1, :L], ux[r:r + 1, :L], np.zeros((1, L)), T[r:r + 1, :L])
        o.set_flags(flags_of(inst, nx)[None, :L])
        o.step(steps)
        om = o.moments()
        for q in (0, 1, 3):                                # rho, u_x, T
            assert rel_l2(gm[q][r, :L], om[q][0]) < tol, (r, q, rel_l2(gm[q][r, :L], om[q][0]))
        # u_y stays zero up to rounding on both sides
        assert np.abs(gm[2][r, :L]).max() < tol * np.abs(om[1]).max()


def test_rows_rules():
    g = slbm.Solver(64, 8, 4, 5, tau=0.7, frame=slbm.SLBM_FRAME_POND)
    ends = np.ones((8, 2, 4))
    with pytest.raises(slbm.SlbmError):
        g.set_rows([64, 64, 2, 64, 64, 64, 64, 64], ends)  # shorter than the stencil
    with pytest.raises(slbm.SlbmError):
        g.set_viscosity_law(1.0, 1.0)                      # needs the two-population model
    h = slbm.Solver(64, 8, 4, 5, tau=0.7)
    with pytest.raises(slbm.SlbmError):
        h.set_rows([64] * 8, np.ones((8, 2, 4)))          # lattice frame


def batch_solver(b, nx, precision=slbm.SLBM_FP32):
    g = slbm.Solver(nx, len(b), 4, 5, tau=0.7, precision=precision, frame=slbm.SLBM_FRAME_POND)
    g.set_twopop(CV, 0.8)
    prof = [WL.shock_profile(i, nx) for i in b]
    rho = np.stack([p[0] for p in prof]); ux = np.stack([p[1] for p in prof])
    T = np.stack([p[2] for p in prof])
    g.init_equilibrium(rho, ux, np.zeros_like(rho), T)
    ends = np.array([[(i["left"][0], i["left"][1], 0.0, i["left"][2]),
                      (i["right"][0], i["right"][1], 0.0, i["right"][2])] for i in b])
    g.set_rows([i["len"] for i in b], ends)
    g.set_viscosity_law([i["mu1"] for i in b], [i["T1"] for i in b], 0.5, PR)
    g.set_flags(np.stack([flags_of(i, nx) for i in b]))
    return g


def test_tuner_keeps_the_state_and_the_results():
    """The autotuner picks a block shape without changing the state, and the
    step gives bit-identical results with any shape; graph replays of pairs
    of co-moving steps equal direct steps bit for bit."""
    b = instances()
    a, c = batch_solver(b, 64), batch_solver(b, 64)
    m0 = a.moments()
    bx, by = a.tune(3)
    assert bx * by == 256
    for x, y in zip(m0, a.moments()):
        np.testing.assert_array_equal(x, y)
    for _ in range(9):
        c.step(1)                                         # default shape, direct launches
    a.step(1)
    a.step(8)                                             # tuned shape, 4 graph replays
    for x, y in zip(a.moments(), c.moments()):
        np.testing.assert_array_equal(x, y)
    for k in (0, 1):
        np.testing.assert_array_equal(a.get_gpops(k), c.get_gpops(k))


@pytest.mark.parametrize("precision,tol", [(slbm.SLBM_FP64, 1e-11), (slbm.SLBM_FP32, 1e-5)])
@pytest.mark.parametrize("interval", [2, 1])
def test_knudsen_refinement_matches_oracle(precision, tol, interval):
    """Knudsen criterion (Kn > 0.02, every 2 steps, or every step -- then
    recorded in the graph replays of the second call) on the batch against
    the oracle's criterion on each instance: identical flags, moments within
    the tolerance after 6 steps."""
    b = instances()
    nx, steps = 64, 6
    g = batch_solver(b, nx, precision)
    g.set_flags(np.zeros((len(b), nx), np.uint8))
    g.set_kn_criterion(0.02, interval)
    g.step(1)
    g.step(steps - 1)
    gm, gf = g.moments(), g.get_flags()
    assert gf.sum() > 0
    for r, inst in enumerate(b):
        L = inst["len"]
        rho, ux, T = WL.shock_profile(inst, nx)
        o = O.Oracle(L, 1, 4, 5, tau=0.7, frame=O.FRAME_POND, periodic=(False, True))
        o.set_twopop(CV, 0.8)
        o.set_pond_ends((inst["left"][0], inst["left"][1], 0.0, inst["left"][2]),
                        (inst["right"][0], inst["right"][1], 0.0, inst["right"][2]))
        o.set_viscosity_law(inst["mu1"], inst["T1"], 0.5, PR)
        o.init_equilibrium(rho[None, :L], ux[None, :L], np.zeros((1, L)), T[None, :L])
        o.set_kn_criterion(0.02, interval)
        o.step(steps)
        np.testing.assert_array_equal(gf[r, :L], o.get_flags()[0])
        om = o.moments()
        for q in (0, 1, 3):
            assert rel_l2(gm[q][r, :L], om[q][0]) < tol


def test_knudsen_every_step_graph_replays_equal_direct_steps():
    """With the criterion every step, slbm_step records it in its graph
    replays: a batch stepped one step per call (direct launches) and one
    stepped in one call (replays of step + criterion) agree bit for bit."""
    b = instances()
    nx = 64
    a = batch_solver(b, nx, slbm.SLBM_FP32)
    c = batch_solver(b, nx, slbm.SLBM_FP32)
    for g in (a, c):
        g.set_flags(np.zeros((len(b), nx), np.uint8))
        g.set_kn_criterion(0.02, 1)
    for _ in range(9):
        a.step(1)
    c.step(1)
    c.step(8)
    for k in (0, 1):
        np.testing.assert_array_equal(a.get_pops(k), c.get_pops(k))
    np.testing.assert_array_equal(a.get_flags(), c.get_flags())
    assert c.get_flags().sum() > 0
