"""Pins of the oracle's co-moving (PonD) frame step, Sec. II.C.

No worked example is printed for it, so the step is pinned to what the
mathematics fixes:
- a uniform state at rest in its own frame (rho W_i, eq. feqPond) is a fixed
  point, for any u and T, with mixed lattices too;
- discrete Galilean invariance: a boost U with U dt = one cell maps the run
  onto itself shifted by one cell per step, frames shifted by U, because every
  departure point, collocation stencil and transfer matrix of eqs. (vi),
  (fll), (reconstructionPond) depends on velocities only through differences;
- the thermal single-population model (C_v = D/2, g = 0) carries sound at
  sqrt(gamma T) with gamma = C_p / C_v = 2, the isothermal one at sqrt(T_L);
- the frame a cell keeps is the converged one: the moments of its
  populations in that frame equal it to the predictor-corrector tolerance
  (eqs. correctorfieldsrho-u), while a single pass without correction does
  not converge.
"""
import numpy as np
import pytest

import oracle as O


def smooth_field(nx, ny):
    x, y = np.meshgrid(np.arange(nx), np.arange(ny))
    ux = 0.05 * np.sin(2 * np.pi * y / ny + 0.3) + 0.03 * np.cos(2 * np.pi * x / nx)
    uy = 0.04 * np.sin(2 * np.pi * x / nx + 1.0)
    rho = 1 + 0.02 * np.cos(2 * np.pi * (x / nx + y / ny))
    T = 1 + 0.05 * np.sin(2 * np.pi * x / nx)
    return rho, ux, uy, T


@pytest.mark.parametrize("frame", [O.FRAME_POND, O.FRAME_POND_ISOTHERMAL])
def test_uniform_state_in_its_own_frame_is_steady(frame):
    nx, ny = 16, 12
    o = O.Oracle(nx, ny, 3, 5, tau=0.7, frame=frame)
    r = np.ones((ny, nx))
    T = 1.3 if frame == O.FRAME_POND else None
    o.init_equilibrium(r, 0.7 * r, -0.4 * r, T)
    fl = np.zeros((ny, nx), np.uint8)
    fl[3:8, 4:9] = 1
    o.set_flags(fl)
    f0, f1 = o.get_pops(0).copy(), o.get_pops(1).copy()
    o.step(3)
    assert np.abs(o.get_pops(0) - f0)[fl == 0].max() < 1e-13
    assert np.abs(o.get_pops(1) - f1)[fl == 1].max() < 1e-13
    ux, uy, t = o.get_frame()
    assert np.abs(ux - 0.7).max() < 1e-13 and np.abs(uy + 0.4).max() < 1e-13
    assert np.abs(t - (1.3 if T else 1.0)).max() < 1e-13
    assert o.nonconverged() == 0


@pytest.mark.parametrize("frame", [O.FRAME_POND, O.FRAME_POND_ISOTHERMAL])
@pytest.mark.parametrize("lo,hi,k", [(3, 4, 0), (3, 5, 1), (4, 5, 1)])
def test_galilean_boost_by_one_cell_per_step(frame, lo, hi, k):
    nx, ny, steps = 24, 16, 3
    rho, ux, uy, T = smooth_field(nx, ny)
    runs = []
    for U in (0.0, 1.0):
        o = O.Oracle(nx, ny, lo, hi, tau=0.7, frame=frame)
        o.init_equilibrium(rho, ux + U / o.dt, uy, T if frame == O.FRAME_POND else None)
        if k:
            o.set_flags(np.ones((ny, nx), np.uint8))
        o.step(steps)
        runs.append(o)
    a, b = runs
    fa = np.roll(a.get_pops(k), steps, axis=1)
    np.testing.assert_allclose(b.get_pops(k), fa, rtol=0, atol=5e-12)
    la = [np.roll(v, steps, axis=1) for v in a.get_frame()]
    lb = b.get_frame()
    np.testing.assert_allclose(lb[0], la[0] + 1.0 / a.dt, rtol=0, atol=1e-11)
    np.testing.assert_allclose(lb[1], la[1], rtol=0, atol=1e-11)
    np.testing.assert_allclose(lb[2], la[2], rtol=0, atol=1e-11)


def test_galilean_boost_with_interfaces_one_step():
    """Mixed lattices: after one step the boosted run equals the plain run one
    cell upstream wherever the target lattice is the same at x and x - 1."""
    nx, ny = 24, 16
    rho, ux, uy, T = smooth_field(nx, ny)
    fl = np.zeros((ny, nx), np.uint8)
    fl[4:11, 7:15] = 1
    runs = []
    for U in (0.0, 1.0):
        o = O.Oracle(nx, ny, 3, 5, tau=0.7, frame=O.FRAME_POND)
        o.init_equilibrium(rho, ux + U / o.dt, uy, T)
        o.set_flags(fl)
        o.step(1)
        runs.append(o)
    a, b = runs
    same = fl == np.roll(fl, 1, axis=1)
    for k in (0, 1):
        sel = same & (fl == k)
        fa = np.roll(a.get_pops(k), 1, axis=1)
        assert np.abs(b.get_pops(k) - fa)[sel].max() < 5e-12
    assert (~same).sum() > 0


def sound_speed(frame, lo, hi, flag):
    nx, ny, A = 32, 2, 1e-3
    x = np.arange(nx)[None, :].repeat(ny, 0)
    k = 2 * np.pi / nx
    rho = 1 + A * np.cos(k * x)
    z = np.zeros_like(rho)
    T = rho.copy() if frame == O.FRAME_POND else None   # adiabatic for gamma = 2
    o = O.Oracle(nx, ny, lo, hi, tau=0.51, frame=frame)
    o.init_equilibrium(rho, z, z, T)
    if flag:
        o.set_flags(np.ones((ny, nx), np.uint8))
    c_guess = np.sqrt(2.0) if frame == O.FRAME_POND else 1.0
    ts, ys = [], []
    for n in range(int(1.1 * nx / c_guess / o.dt)):
        r = o.moments()[0]
        ts.append(n * o.dt)
        ys.append(np.sum((r[0] - 1) * np.cos(k * np.arange(nx))) * 2 / nx)
        o.step(1)
    from scipy.optimize import curve_fit
    f = lambda t, a, g, w: a * np.exp(-g * t) * np.cos(w * t)
    p, _ = curve_fit(f, np.array(ts), np.array(ys), p0=[A, 0.0, k * c_guess])
    return p[2] / k


@pytest.mark.parametrize("frame,lo,hi,flag,c", [
    (O.FRAME_POND, 3, 5, 0, np.sqrt(2.0)),
    (O.FRAME_POND, 3, 5, 1, np.sqrt(2.0)),
    (O.FRAME_POND, 3, 4, 0, np.sqrt(2.0)),
    (O.FRAME_POND_ISOTHERMAL, 3, 5, 0, 1.0),
    (O.FRAME_POND_ISOTHERMAL, 4, 5, 1, 1.0),
])
def test_sound_speed(frame, lo, hi, flag, c):
    assert abs(sound_speed(frame, lo, hi, flag) / c - 1) < 2e-3


@pytest.mark.parametrize("frame", [O.FRAME_POND, O.FRAME_POND_ISOTHERMAL])
def test_kept_frame_is_the_converged_one(frame):
    nx, ny = 20, 14
    rho, ux, uy, T = smooth_field(nx, ny)
    ux = ux * 6
    o = O.Oracle(nx, ny, 3, 5, tau=0.6, frame=frame)
    o.init_equilibrium(rho, ux, uy, T if frame == O.FRAME_POND else None)
    fl = np.zeros((ny, nx), np.uint8)
    fl[2:9, 3:12] = 1
    o.set_flags(fl)
    o.set_pond(1e-13, 50)
    o.step(2)
    assert o.nonconverged() == 0
    r, mu, mv, mt = o.moments()
    a, b, t = o.get_frame()
    assert np.abs(mu - a).max() < 1e-11 and np.abs(mv - b).max() < 1e-11
    if frame == O.FRAME_POND:
        assert np.abs(mt - t).max() < 1e-11
    # a single pass keeps the predictor frame, which is not the moments' frame
    o1 = O.Oracle(nx, ny, 3, 5, tau=0.6, frame=frame)
    o1.init_equilibrium(rho, ux, uy, T if frame == O.FRAME_POND else None)
    o1.set_flags(fl)
    o1.set_pond(1e-13, 1)
    o1.step(1)
    assert o1.nonconverged() > 0


def test_co_moving_frame_restrictions():
    with pytest.raises(ValueError):
        O.Oracle(16, 16, 3, 5, frame=O.FRAME_POND, periodic=(True, False))
    o = O.Oracle(16, 16, 3, 5, frame=O.FRAME_POND_ISOTHERMAL)
    one = np.ones((16, 16))
    with pytest.raises(RuntimeError):
        o.init_equilibrium(one, 0 * one, 0 * one, one)      # isothermal takes no T
    with pytest.raises(RuntimeError):
        o.set_criterion(1, 0.3)
    lat = O.Oracle(16, 16, 3, 5)
    with pytest.raises(RuntimeError):
        lat.get_frame()


@pytest.mark.parametrize("frame", [O.FRAME_POND, O.FRAME_POND_ISOTHERMAL])
def test_same_state_stored_in_scattered_frames(frame):
    """One uniform state written in a different frame at every node (eq. fll).
    A step must carry every collocation vector into the target frame before
    interpolating; it then returns rho W_i in the state's own frame."""
    nx, ny = 14, 12
    rng = np.random.default_rng(7)
    u0, v0 = 0.3, -0.2
    T0 = 1.2 if frame == O.FRAME_POND else 1.0
    o = O.Oracle(nx, ny, 3, 5, tau=0.7, frame=frame)
    fl = np.zeros((ny, nx), np.uint8)
    fl[3:9, 2:8] = 1
    lam = np.stack([u0 + rng.uniform(-0.2, 0.2, (ny, nx)),
                    v0 + rng.uniform(-0.2, 0.2, (ny, nx)),
                    T0 * (1 + (rng.uniform(-0.2, 0.2, (ny, nx)) if frame == O.FRAME_POND
                               else np.zeros((ny, nx))))],
                   axis=-1)
    one = np.ones((ny, nx))
    o.init_equilibrium(one, u0 * one, v0 * one, T0 * one if frame == O.FRAME_POND else None)
    o.set_flags(fl)
    o.set_frame(lam[..., 0], lam[..., 1], lam[..., 2])
    pops = []
    for k, n in enumerate((3, 5)):
        W = O.lattice(n)[2]
        f = np.zeros((ny, nx, n * n))
        for y in range(ny):
            for x in range(nx):
                f[y, x] = O.transfer(n, (u0, v0, T0), lam[y, x]) @ W
        o.set_pops(k, f)
        pops.append(W)
    o.step(1)
    a, b, t = o.get_frame()
    assert np.abs(a - u0).max() < 1e-11 and np.abs(b - v0).max() < 1e-11
    assert np.abs(t - T0).max() < 1e-11
    for k in (0, 1):
        assert np.abs(o.get_pops(k) - pops[k])[fl == k].max() < 1e-11
