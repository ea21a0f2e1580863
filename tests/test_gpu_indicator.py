"""GPU checks of the learned refinement indicator.

Parity: the GPU features against the oracle's restatement (FP64 run: 1e-6 on
the scaled features, which the API returns as FP32; FP32 run: 1e-4), and the tensor-core MLP against the
reference forward pass with the same FP16 roundings (FP64 run, random
weights: 1e-3 on the logits, the gap being FP32 against exact accumulation).
Function: an indicator trained on an all-high-order run (labels: the plain
Mach criterion) agrees with the plain criterion on held-out states, also
when it sets the flags of a running simulation (SLBM_CRIT_MLP)."""
import numpy as np
import pytest

import oracle as O
from oracle import indicator as OI
from paper_2102_12559_gb300 import indicator as IND
from paper_2102_12559_gb300 import workloads as WL
from paper_2102_12559_gb300 import slbm

pytestmark = pytest.mark.gpu

FP32, FP64 = slbm.SLBM_FP32, slbm.SLBM_FP64


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def state_pair(precision, periodic):
    nx, ny = 37, 29
    fields = WL.perturbed(nx, ny, seed=21, amp_rho=0.05, amp_u=0.3)
    fl = WL.random_flags(nx, ny, seed=4, blobs=2, rmin=3, rmax=6)
    g = slbm.Solver(nx, ny, 3, 5, tau=0.62, periodic=periodic, precision=precision)
    o = O.Oracle(nx, ny, 3, 5, tau=0.62, periodic=periodic)
    for s in (g, o):
        s.init_equilibrium(*fields)
        s.set_flags(fl)
        s.step(2)
    return g, o


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-6), (FP32, 1e-4)])
@pytest.mark.parametrize("periodic", [(True, True), (False, False)])
def test_features_match_oracle(precision, tol, periodic):
    g, o = state_pair(precision, periodic)
    fg = g.indicator_eval()[0]
    fo = OI.features(o)
    assert np.abs(fg - fo).max() < tol, np.abs(fg - fo).max(axis=(0, 1))


def random_weights(seed):
    rng = np.random.default_rng(seed)
    return {"w1": rng.normal(0, 0.4, (16, 32)), "b1": rng.normal(0, 0.1, 32),
            "w2": rng.normal(0, 0.25, (32, 32)), "b2": rng.normal(0, 0.1, 32),
            "w3": rng.normal(0, 0.3, 32), "b3": 0.05}


def test_logits_match_reference_forward():
    g, o = state_pair(FP64, (True, True))
    w = random_weights(9)
    g.set_indicator(w)
    _, lg, flg = g.indicator_eval(features=False, logits=True, flags=True)
    lo = OI.forward_fp16(w, OI.features(o).reshape(-1, 16)).reshape(lg.shape)
    assert np.abs(lg - lo).max() < 1e-3
    sure = np.abs(lo) > 1e-2
    np.testing.assert_array_equal(flg[sure], (lo > 0)[sure])


def training_data(seed, N=192, steps=20):
    """All-high-order (D2Q25) random-vortex run: features and the plain Mach
    criterion's labels."""
    r, u, v = WL.random_vortex_field(N, 48, seed=seed, rmin=6.0, rmax=24.0, umax=0.8)
    g = slbm.Solver(N, N, 3, 5, tau=0.6)
    g.init_equilibrium(r, u, v)
    g.set_flags(np.ones((N, N), np.uint8))
    g.step(steps)
    fe = g.indicator_eval()[0].reshape(-1, 16)
    _, mu, mv, _ = g.moments()
    lab = (np.hypot(mu, mv) > 0.3).ravel().astype(float)
    return fe.astype(np.float64), lab


@pytest.fixture(scope="module")
def trained():
    x, y = training_data(seed=11)
    return IND.train(x, y, epochs=100, batch=512, seed=0, balance=False)


def test_trained_indicator_agrees_with_plain_criterion(trained):
    x, y = training_data(seed=12)                 # held-out field
    assert IND.agreement(trained, x, y) > 0.99
    N = 192
    r, u, v = WL.random_vortex_field(N, 48, seed=12, rmin=6.0, rmax=24.0, umax=0.8)
    g = slbm.Solver(N, N, 3, 5, tau=0.6)
    g.init_equilibrium(r, u, v)
    g.set_flags(np.ones((N, N), np.uint8))
    g.step(20)
    g.set_indicator(trained)
    flags = g.indicator_eval(features=False, flags=True)[2]
    _, mu, mv, _ = g.moments()
    assert np.mean(flags == (np.hypot(mu, mv) > 0.3)) > 0.99


def test_mlp_criterion_sets_flags_during_a_run(trained):
    nx, ny = 256, 128
    J = WL.free_jet(nx, ny, slot=16, ma_jet=0.5, ma_co=0.05)
    g = slbm.Solver(nx, ny, 3, 5, tau=0.55, periodic=(False, False))
    g.init_equilibrium(J["rho"], J["ux"], J["uy"])
    g.set_boundary(slbm.SLBM_SIDE_XMIN, slbm.SLBM_BC_INLET, None, J["in_ux"], J["in_uy"])
    g.set_boundary(slbm.SLBM_SIDE_XMAX, slbm.SLBM_BC_OUTFLOW)
    for side in (slbm.SLBM_SIDE_YMIN, slbm.SLBM_SIDE_YMAX):
        g.set_boundary(side, slbm.SLBM_BC_DIRICHLET, np.full(nx, J["fs_rho"]),
                       np.full(nx, J["fs_ux"]), np.full(nx, J["fs_uy"]))
    g.set_indicator(trained, interval=5)
    g.set_criterion(slbm.SLBM_CRIT_MLP, 0.0)
    g.step(50)                                    # flags re-evaluated at steps 5, 10, ..., 50
    flags = g.get_flags()
    _, mu, mv, _ = g.moments()
    plain = np.hypot(mu, mv) > 0.3
    assert flags.sum() > 0
    assert np.mean(flags == plain) > 0.99
    r, _, _, _ = g.moments()
    assert np.all(np.isfinite(r))


def test_mlp_criterion_needs_weights():
    g = slbm.Solver(32, 32, 3, 5, tau=0.6)
    with pytest.raises(slbm.SlbmError):
        g.set_criterion(slbm.SLBM_CRIT_MLP, 0.0)


@pytest.mark.parametrize("case,crit", [("periodic", slbm.SLBM_CRIT_MLP),
                                       ("walled_high_tau", slbm.SLBM_CRIT_MLP),
                                       ("periodic", slbm.SLBM_CRIT_MLP_REFINE)])
def test_mlp_flips_match_oracle_replay(case, crit):
    """Flags set by the learned indicator during a run (every 5 steps, random
    weights so that cells flip both ways) convert the populations as the
    oracle does when it is given the same flags at the same steps: FP64
    moments within 1e-11 after 40 steps.  Refinement only: no flag ever goes
    back from 1 to 0."""
    if case == "periodic":
        nx, ny, tau, periodic = 45, 37, 0.7, (True, True)
        fields = WL.perturbed(nx, ny, seed=23, amp_rho=0.04, amp_u=0.3)
    else:
        nx, ny, tau, periodic = 40, 8, 20.0, (False, True)
        fields = WL.perturbed(nx, ny, seed=24, amp_rho=0.02, amp_u=0.1)
    g = slbm.Solver(nx, ny, 3, 5, tau=tau, periodic=periodic, precision=FP64)
    o = O.Oracle(nx, ny, 3, 5, tau=tau, order=3, periodic=periodic)
    if not periodic[0]:
        for side, uw in ((0, -0.1), (1, 0.1)):
            g.set_boundary(side, slbm.SLBM_BC_DIFFUSE, None, np.zeros(ny), np.full(ny, uw))
            o.set_bc(side, O.BC_DIFFUSE, None, np.zeros(ny), np.full(ny, uw))
    g.init_equilibrium(*fields)
    o.init_equilibrium(*fields)
    # refinement only: a short interval (buffer) and the threshold at the
    # initial logits' 90th percentile, so the flagged region starts small
    every = 5 if crit == slbm.SLBM_CRIT_MLP else 2
    g.set_indicator(random_weights(9), interval=every)
    thr = 0.0
    if crit == slbm.SLBM_CRIT_MLP_REFINE:
        thr = float(np.quantile(g.indicator_eval(features=False, logits=True)[1], 0.9))
    g.set_criterion(crit, thr)
    fl = g.get_flags()
    o.set_flags(fl)
    flips = 0
    for _ in range(40 // every):
        g.step(every)
        o.step(every)
        nf = g.get_flags()
        flips += int((nf != fl).sum())
        if crit == slbm.SLBM_CRIT_MLP_REFINE:
            assert (nf >= fl).all()
        fl = nf
        o.set_flags(fl)
    assert fl.mean() > 0.1 and flips > 5, (fl.mean(), flips)
    if crit == slbm.SLBM_CRIT_MLP:
        assert fl.mean() < 0.9
    mg, mo = g.moments(), o.moments()
    for q in range(3):
        assert rel_l2(mg[q], mo[q]) < 1e-11, (q, rel_l2(mg[q], mo[q]))
    g.close()


def density_weights():
    """logit = 10 relu(relu(10 (rho - 1))) - 2.5: positive iff rho - 1 > 0.025."""
    w = {"w1": np.zeros((16, 32)), "b1": np.zeros(32), "w2": np.zeros((32, 32)),
         "b2": np.zeros(32), "w3": np.zeros(32), "b3": -2.5}
    w["w1"][0, 0] = 1.0
    w["w2"][0, 0] = 1.0
    w["w3"][0] = 10.0
    return w


def test_refine_buffer_square_and_channel_gaps():
    """SLBM_CRIT_MLP_REFINE widens the indicator's decisions by `interval`
    cells along x and y (a square around an isolated cell on a periodic
    grid), never across a channel gap, and keeps what was flagged before."""
    nx, ny, r = 40, 30, 3
    rho = np.ones((ny, nx))
    rho[10, 38] = 1.05                           # next to the periodic x edge
    g = slbm.Solver(nx, ny, 3, 5, tau=0.7, precision=FP64)
    g.init_equilibrium(rho, np.zeros((ny, nx)), np.zeros((ny, nx)))
    g.set_indicator(density_weights(), interval=r)
    g.set_criterion(slbm.SLBM_CRIT_MLP_REFINE, 0.0)
    want = np.zeros((ny, nx), np.uint8)
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            want[(10 + dy) % ny, (38 + dx) % nx] = 1
    np.testing.assert_array_equal(g.get_flags(), want)
    g.step(2 * r)
    assert (g.get_flags() >= want).all()
    g.close()

    widths, G = [20, 24], 2
    x0, nxc = WL.channel_layout(widths, G)
    rho = np.ones((8, nxc))
    rho[:, x0[0] + 17:x0[0] + 20] = 1.05         # against channel 0's right wall
    c = slbm.Solver(nxc, 8, 3, 5, tau=0.7, periodic=(False, True), precision=FP64)
    c.init_equilibrium(rho, np.zeros((8, nxc)), np.zeros((8, nxc)))
    c.set_channels(x0, widths, [0.0, 0.0], [0.0, 0.0], [0.7, 0.9])
    c.set_indicator(density_weights(), interval=r)
    c.set_criterion(slbm.SLBM_CRIT_MLP_REFINE, 0.0)
    fl = c.get_flags()
    want = np.zeros((8, nxc), np.uint8)
    gap = np.ones(nxc, bool)
    for k, w in enumerate(widths):
        gap[x0[k]:x0[k] + w] = False
    want[:, gap] = 2
    want[:, x0[0] + 17 - r:x0[0] + 20] = 1
    np.testing.assert_array_equal(fl, want)
    c.close()
