"""CPU pins of the learned indicator's host parts: the hand-written training
(gradients against finite differences, a separable problem learned) and the
reference features and forward pass of ``oracle.indicator`` (closed forms:
an equilibrium state has no non-equilibrium stress or flux and T = T_L, a
linear field has exact central differences, hand-set weights give a known
logit)."""
import numpy as np
import pytest

import oracle as O
from oracle import indicator as OI
from paper_2102_12559_gb300 import indicator as IND
from paper_2102_12559_gb300 import workloads as WL


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(3)
    w = IND.init_weights(5)
    x = rng.normal(size=(40, 16))
    y = (rng.random(40) > 0.5).astype(float)
    _, g = IND.loss_and_grad(w, x, y)
    eps = 1e-6
    for key in ("w1", "b1", "w2", "b2", "w3"):
        flat = w[key].ravel()
        for idx in rng.choice(flat.size, 5, replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp, _ = IND.loss_and_grad(w, x, y)
            flat[idx] = old - eps
            lm, _ = IND.loss_and_grad(w, x, y)
            flat[idx] = old
            assert abs((lp - lm) / (2 * eps) - g[key].ravel()[idx]) < 1e-6
    w0 = w["b3"]
    w["b3"] = w0 + eps
    lp, _ = IND.loss_and_grad(w, x, y)
    w["b3"] = w0 - eps
    lm, _ = IND.loss_and_grad(w, x, y)
    w["b3"] = w0
    assert abs((lp - lm) / (2 * eps) - g["b3"]) < 1e-6


def test_training_learns_a_threshold():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4000, 16))
    y = (np.abs(x[:, 15]) > 1.0).astype(float)      # a threshold on one feature
    w = IND.train(x, y, epochs=30, batch=256, seed=2)
    assert IND.agreement(w, x, y) > 0.97


def test_equilibrium_state_features():
    nx, ny = 12, 10
    o = O.Oracle(nx, ny, 3, 5, tau=0.7)
    o.init_equilibrium(*WL.uniform(nx, ny, 1.1, 0.2, -0.1))
    fl = np.zeros((ny, nx), np.uint8)
    fl[2:6, 3:8] = 1
    o.set_flags(fl)
    f = OI.features(o) / OI.SCALE
    assert np.allclose(f[..., 0], 0.1) and np.allclose(f[..., 1], 0.2) and np.allclose(f[..., 2], -0.1)
    assert np.abs(f[..., 3]).max() < 1e-13          # T = T_L for the lattice equilibrium
    assert np.abs(f[..., 4:15]).max() < 1e-13       # no non-equilibrium part, no gradients
    assert np.allclose(f[..., 15], np.hypot(0.2, 0.1))


def test_linear_field_gradients():
    nx, ny = 9, 7
    o = O.Oracle(nx, ny, 3, 5, tau=0.7, periodic=(False, False))
    x = np.arange(nx)[None, :].repeat(ny, 0).astype(float)
    y = np.arange(ny)[:, None].repeat(nx, 1).astype(float)
    o.init_equilibrium(1 + 0.01 * x, 0.02 * y, -0.03 * x)
    f = OI.features(o) / OI.SCALE
    inner = (slice(1, -1), slice(1, -1))
    assert np.allclose(f[..., 9][inner], 0.01) and np.allclose(f[..., 10][inner], 0.0)
    assert np.allclose(f[..., 11][inner], 0.0) and np.allclose(f[..., 12][inner], 0.02)
    assert np.allclose(f[..., 13][inner], -0.03) and np.allclose(f[..., 14][inner], 0.0)
    # edges repeat the edge cell: one-sided half difference
    assert np.allclose(f[..., 9][:, 0], 0.005)


def test_forward_with_hand_set_weights():
    w = {"w1": np.zeros((16, 32)), "b1": np.zeros(32), "w2": np.eye(32), "b2": np.zeros(32),
         "w3": np.zeros(32), "b3": -0.5}
    w["w1"][15, 0] = 1.0
    w["w3"][0] = 2.0
    x = np.zeros((3, 16))
    x[:, 15] = [0.25, 1.0, -1.0]
    np.testing.assert_allclose(OI.forward_fp16(w, x), [0.0, 1.5, -0.5], atol=1e-6)
    np.testing.assert_allclose(IND.forward(w, x)[0], [0.0, 1.5, -0.5], atol=1e-12)


def test_nonequilibrium_features_closed_form():
    """Perturbations that leave rho and u unchanged: a symmetric one along an
    axis adds exactly a normal stress 2 c^2 eps and kinetic T 2 c^2 eps / (2 rho),
    an antisymmetric one (corners against the axis pair) exactly a heat flux
    1/2 * 4 c^3 eps along that axis (D2Q9, c = sqrt(3))."""
    nx, ny = 8, 6
    rho0, u0, v0 = 1.1, 0.2, -0.1
    o = O.Oracle(nx, ny, 3, 5, tau=0.7)
    o.init_equilibrium(*WL.uniform(nx, ny, rho0, u0, v0))
    o.set_flags(np.zeros((ny, nx), np.uint8))
    cx, cy, _ = O.lattice(3)
    c = cx.max()
    idx = lambda a, b: int(np.flatnonzero((np.sign(cx) == a) & (np.sign(cy) == b))[0])
    e1, e2 = 1e-3, 2e-3
    dx = np.zeros(9)
    dx[[idx(1, 0), idx(-1, 0)]] += e1
    dx[idx(0, 0)] -= 2 * e1
    dx[[idx(1, 1), idx(1, -1)]] += e2
    dx[[idx(-1, 1), idx(-1, -1)]] -= e2
    dx[idx(1, 0)] -= 2 * e2
    dx[idx(-1, 0)] += 2 * e2
    dy = np.zeros(9)                                 # the same with the axes swapped
    for i in range(9):
        dy[idx(int(np.sign(cy[i])), int(np.sign(cx[i])))] = dx[i]
    f = o.get_pops(0)
    f[:, : nx // 2] += dx
    f[:, nx // 2:] += dy
    o.set_pops(0, f)
    F = OI.features(o) / OI.SCALE
    L, R = F[:, : nx // 2], F[:, nx // 2:]
    np.testing.assert_allclose(F[..., 0], rho0 - 1, atol=1e-13)
    np.testing.assert_allclose(F[..., 1], u0, atol=1e-13)
    np.testing.assert_allclose(F[..., 2], v0, atol=1e-13)
    np.testing.assert_allclose(F[..., 3], c * c * e1 / rho0, atol=1e-13)
    np.testing.assert_allclose(L[..., 4], 2 * c * c * e1, atol=1e-13)
    np.testing.assert_allclose(R[..., 6], 2 * c * c * e1, atol=1e-13)
    np.testing.assert_allclose(L[..., 7], 2 * c ** 3 * e2, atol=1e-13)
    np.testing.assert_allclose(R[..., 8], 2 * c ** 3 * e2, atol=1e-13)
    for part, zero in ((L, (5, 6, 8)), (R, (4, 5, 7))):
        assert np.abs(part[..., list(zero)]).max() < 1e-13
    assert np.abs(F[..., 9:15]).max() < 1e-13
