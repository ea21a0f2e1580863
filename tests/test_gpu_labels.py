"""GPU checks of the indicator's labels (slbm_lattice_loss) and of its
training kernel (slbm_mlp_train).

Lattice loss: element-wise parity with the oracle's composition of its own
step, lift and projection (oracle/labels.py, pinned by closed forms), FP64
at 1e-9 of the field's largest loss and FP32 at 1e-4 (the loss is a
difference of O(1e-3) between two population vectors that carry FP32 rounding
of about 1e-8), on periodic and walled grids with ragged tiles and on batched
channels; the state after the call is the high-order step's.

Training: the gradient of one step against a numpy restatement with the
kernel's FP16 roundings (1e-3 of each block's largest entry: FP32 against
FP64 accumulation order) and against the exact FP64 gradient (5e-2: the FP16
operands); then a whole run against the FP64 host trainer on the same
mini-batches: the final loss within 10 % and the decisions within 2 points.
"""
import numpy as np
import pytest

import oracle as O
from oracle import labels as OL
from paper_2102_12559_gb300 import indicator as IND
from paper_2102_12559_gb300 import slbm
from paper_2102_12559_gb300 import workloads as WL

pytestmark = pytest.mark.gpu

FP32, FP64 = slbm.SLBM_FP32, slbm.SLBM_FP64


def vortex_pair(precision, periodic, nx=45, ny=37, steps=3):
    fields = WL.perturbed(nx, ny, seed=31, amp_rho=0.04, amp_u=0.5)
    g = slbm.Solver(nx, ny, 3, 5, tau=0.63, periodic=periodic, precision=precision)
    o = O.Oracle(nx, ny, 3, 5, tau=0.63, order=3, periodic=periodic)
    ones = np.ones((ny, nx), np.uint8)
    if not periodic[0]:  # diffuse walls moving along y
        for side, uw in ((0, -0.05), (1, 0.08)):
            o.set_bc(side, O.BC_DIFFUSE, None, np.zeros(ny), np.full(ny, uw))
            g.set_boundary(side, slbm.SLBM_BC_DIFFUSE, None, np.zeros(ny), np.full(ny, uw))
    for s in (g, o):
        s.init_equilibrium(*fields)
        s.set_flags(ones)
        s.step(steps)
    return g, o


@pytest.mark.parametrize("precision,tol", [(FP64, 1e-9), (FP32, 1e-4)])
@pytest.mark.parametrize("periodic", [(True, True), (False, True)])
def test_lattice_loss_matches_oracle(precision, tol, periodic):
    g, o = vortex_pair(precision, periodic)
    lg = g.lattice_loss()
    lo = OL.lattice_loss(o)
    scale = lo.max()
    assert scale > 1e-3
    assert np.abs(lg - lo).max() < tol * scale, np.abs(lg - lo).max() / scale
    # the handle continues from the high-order step, counted once
    assert g.info.steps == 4
    mg, mo = g.moments(), o.moments()
    mtol = 1e-11 if precision == FP64 else 1e-5
    for a, b in zip(mg[:3], mo[:3]):
        assert np.abs(a - b).max() < mtol
    g.close()


def test_lattice_loss_channels():
    widths, taus = [12, 17, 9, 21], [0.6, 3.0, 0.8, 12.0]
    uws = [(-0.1, 0.1), (0.05, 0.1), (0.0, -0.08), (-0.1, 0.1)]
    ny, G = 8, 2
    x0, nx = WL.channel_layout(widths, G)
    g = slbm.Solver(nx, ny, 3, 5, tau=0.6, periodic=(False, True), precision=FP64)
    g.init_equilibrium(*WL.uniform(nx, ny))
    g.set_channels(x0, widths, [u[0] for u in uws], [u[1] for u in uws], taus)
    g.set_flags(np.ones((ny, nx), np.uint8))
    g.step(30)
    lg = g.lattice_loss()
    for c, w in enumerate(widths):
        o = O.Oracle(w, ny, 3, 5, tau=taus[c], order=3, periodic=(False, True))
        o.set_bc(0, O.BC_DIFFUSE, None, np.zeros(ny), np.full(ny, uws[c][0]))
        o.set_bc(1, O.BC_DIFFUSE, None, np.zeros(ny), np.full(ny, uws[c][1]))
        o.init_equilibrium(*WL.uniform(w, ny))
        o.set_flags(np.ones((ny, w), np.uint8))
        o.step(30)
        lo = OL.lattice_loss(o)
        part = lg[:, x0[c]:x0[c] + w]
        assert np.abs(part - lo).max() < 1e-9 * lo.max(), c
    gap = np.ones(nx, bool)
    for c, w in enumerate(widths):
        gap[x0[c]:x0[c] + w] = False
    assert (lg[:, gap] == 0).all()
    g.close()


def test_lattice_loss_refuses():
    g = slbm.Solver(40, 24, 3, 5, tau=0.6)
    g.init_equilibrium(*WL.uniform(40, 24))
    with pytest.raises(slbm.SlbmError):  # low-order cells
        g.lattice_loss()
    g.set_flags(np.ones((24, 40), np.uint8))
    g.set_criterion(slbm.SLBM_CRIT_MACH, 0.3)
    with pytest.raises(slbm.SlbmError):  # criterion on
        g.lattice_loss()
    g.close()


def labelled_set(n=128, steps=10, seed=5):
    """Features and lattice-loss labels of an all-D2Q25 random-vortex run."""
    g = slbm.Solver(n, n, 3, 5, tau=0.6)
    g.init_equilibrium(*WL.random_vortex_field(n, 3, seed=seed, rmin=8, rmax=20, umax=0.9))
    g.set_flags(np.ones((n, n), np.uint8))
    g.step(steps)
    x = g.indicator_eval()[0].reshape(-1, 16).astype(np.float64)
    loss = g.lattice_loss().ravel()
    g.close()
    return x, IND.labels(loss)


def fp16_gradient(w, x, y):
    """The kernel's gradient: FP16 operands, exact (FP64) accumulation."""
    h = lambda a: np.asarray(a, np.float16).astype(np.float64)
    B = len(y)
    x16, w1, w2 = h(x), h(w["w1"]), h(w["w2"])
    z1 = x16 @ w1 + w["b1"]
    h1 = h(np.maximum(z1, 0))
    z2 = h1 @ w2 + w["b2"]
    h2 = np.maximum(z2, 0)
    z = h2 @ w["w3"] + w["b3"]
    d = 1 / (1 + np.exp(-z)) - y
    dz2 = np.outer(d, w["w3"]) * (z2 > 0)
    dz1 = (h(dz2) @ w2.T) * (z1 > 0)
    loss = np.mean(np.logaddexp(0, -(2 * y - 1) * z))
    return loss, {"w1": x16.T @ h(dz1) / B, "b1": dz1.sum(0) / B, "w2": h1.T @ h(dz2) / B,
                  "b2": dz2.sum(0) / B, "w3": h2.T @ d / B, "b3": d.sum() / B}


def test_gradient_matches_host():
    x, y = labelled_set()
    assert 0.02 < y.mean() < 0.5
    w = IND.init_weights(2)
    w["b1"] = np.random.default_rng(3).normal(0, 0.1, 32)
    idx = IND.draw_batches(y, 1, 512, seed=4)[:1]
    params = IND.pack(w).astype(np.float32)
    adam = np.zeros((2, slbm.MLP_PARAMS), np.float32)
    wf = IND.unpack(params.astype(np.float64))  # the weights the kernel starts from
    loss, grad = slbm.slbm_mlp_train(x, y, idx, (1e-3, *IND.ADAM), 0, params, adam,
                                     want_grad=True)
    gk = IND.unpack(grad.astype(np.float64))
    l16, g16 = fp16_gradient(wf, x[idx[0]], y[idx[0]])
    l64, g64 = IND.loss_and_grad(wf, x[idx[0]], y[idx[0]])
    assert abs(loss[0] - l16) < 1e-4 * l16
    assert abs(loss[0] - l64) < 2e-3 * l64
    for k in IND.KEYS:
        a, b, c = np.asarray(gk[k]), np.asarray(g16[k]), np.asarray(g64[k])
        s = np.abs(c).max()
        assert np.abs(a - b).max() < 1e-3 * s, (k, np.abs(a - b).max() / s)
        assert np.abs(a - c).max() < 5e-2 * s, (k, np.abs(a - c).max() / s)
    # one Adam step from zero moments moves each parameter by lr m^/(sqrt(v^) + eps)
    step = 1e-3 * grad / (np.abs(grad) + 1e-8)
    assert np.abs(params - (IND.pack(wf) - step)).max() < 1e-6


def test_gpu_training_reaches_host_loss():
    x, y = labelled_set()
    idx = IND.draw_batches(y, 12, 512, seed=0, balance=True)
    wh, lh, _ = IND.train_steps(IND.init_weights(0), x, y, idx, lr=3e-3)
    wg, lg = IND.train_gpu(x, y, idx=idx, lr=3e-3, seed=0)
    # same start, same batches: the first steps' losses agree closely
    assert np.abs(lg[:5] - lh[:5]).max() < 3e-3 * lh[0]

    def full_loss(w):
        z = IND.forward(w, x)[0]
        return float(np.mean(np.logaddexp(0, -(2 * y - 1) * z)))

    def balanced(w):
        hit = IND.forward(w, x)[0] > 0
        pos = y > 0.5
        return 0.5 * (hit[pos].mean() + (~hit[~pos]).mean())

    fh, fg = full_loss(wh), full_loss(wg)
    assert fg < 1.1 * fh + 0.005, (fg, fh)
    assert abs(IND.agreement(wg, x, y) - IND.agreement(wh, x, y)) < 0.02
    assert abs(balanced(wg) - balanced(wh)) < 0.02
    assert balanced(wg) > 0.85, balanced(wg)
