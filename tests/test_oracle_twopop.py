"""Pins of the oracle's two-population co-moving model (Sec. II.B, eqs.
Pond_f_equation / Pond_g_equation, feqPond / geqPond, fqeq / gqeq).

No worked example is printed for it; the pins are what the model's
definitions fix:
- with C_v = D/2 = 1, omega_2 = omega_1 and g = 0 it is the single-population
  thermal model, step for step;
- a uniform state at rest in its own frame (f = rho W_i, g = (C_v - 1) T rho
  W_i) is a fixed point, mixed lattices too;
- in a uniform state the step is the collision alone, so a non-equilibrium
  part that is a pure third-order Hermite term of f, or a first-order term of
  g (the heat flux), relaxes by 1 - omega_2 per step, while a second-order
  term of f (stress) or of g relaxes by 1 - omega_1: the quasi-equilibria
  carry exactly the non-equilibrium third moment of f and first moment of g;
- sound travels at sqrt(gamma T), gamma = (C_v + 1) / C_v;
- an entropy wave (T perturbed at constant pressure) decays with the thermal
  diffusivity kappa / (rho C_p) = (1/omega_2 - 1/2) T dt and a shear wave with
  the kinematic viscosity (1/omega_1 - 1/2) T dt, so Pr = C_p mu / kappa
  follows from the two relaxation times;
- discrete Galilean invariance (a boost of one cell per step).
"""
import numpy as np
import pytest

import oracle as O
from paper_2102_12559_gb300 import workloads as WL


def state(o):
    fl = o.get_flags()
    out = []
    for k in (0, 1):
        m = (fl == k)[..., None]
        out.append(np.where(m, o.get_pops(k), 0.0))
        if o_twopop(o):
            out.append(np.where(m, o.get_gpops(k), 0.0))
    return out


def o_twopop(o):
    return getattr(o, "_twopop", False)


def make(nx, ny, lo, hi, tau, cv=None, tau2=None):
    o = O.Oracle(nx, ny, lo, hi, tau=tau, frame=O.FRAME_POND)
    if cv is not None:
        o.set_twopop(cv, tau2)
        o._twopop = True
    return o


def test_reduces_to_the_single_population_model():
    nx, ny = 16, 8
    r, u, v = WL.perturbed(nx, ny, seed=3, amp_rho=0.05, amp_u=0.2, U=(0.3, 0.1))
    T = WL.perturbed_T(nx, ny, seed=4, amp=0.05)
    fl = np.zeros((ny, nx), np.uint8)
    fl[2:6, 4:9] = 1
    runs = []
    for two in (False, True):
        o = make(nx, ny, 4, 5, 0.7, *((1.0, 0.7) if two else (None, None)))
        o.init_equilibrium(r, u, v, T)
        o.set_flags(fl)
        o.step(3)
        runs.append(o)
    a, b = runs
    for k in (0, 1):
        m = (fl == k)[..., None]
        assert np.abs(np.where(m, a.get_pops(k) - b.get_pops(k), 0)).max() < 1e-13
        assert np.abs(np.where(m, b.get_gpops(k), 0)).max() < 1e-13      # g stays 0
    np.testing.assert_allclose(a.audit(), b.audit(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("lo,hi", [(3, 5), (4, 5)])
def test_uniform_state_in_its_own_frame_is_steady(lo, hi):
    nx, ny = 12, 8
    o = make(nx, ny, lo, hi, 0.7, 1.5, 0.9)
    one = np.ones((ny, nx))
    o.init_equilibrium(1.2 * one, 0.4 * one, -0.2 * one, 1.3 * one)
    fl = np.zeros((ny, nx), np.uint8)
    fl[2:6, 3:8] = 1
    o.set_flags(fl)
    before = state(o)
    o.step(3)
    for x, y in zip(before, state(o)):
        assert np.abs(x - y).max() < 1e-13
    ux, uy, t = o.get_frame()
    assert np.abs(ux - 0.4).max() < 1e-13 and np.abs(uy + 0.2).max() < 1e-13
    assert np.abs(t - 1.3).max() < 1e-13
    # g^eq of eq. (geqPond): (C_v - 1) T rho W_i
    W = O.lattice(lo)[2]
    g0 = o.get_gpops(0)[fl == 0]
    np.testing.assert_allclose(g0, np.broadcast_to(0.5 * 1.3 * 1.2 * W, g0.shape), rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", [4, 5])
def test_quasi_equilibria_set_the_relaxation_rates(n):
    """Uniform state in frame u = (0.3, -0.2), T = 1.2 with one Hermite
    non-equilibrium term at a time; one step multiplies it by 1 - omega_2
    (third order of f, first order of g) or 1 - omega_1 (second order)."""
    nx, ny, tau, tau2, cv = 4, 4, 0.7, 1.1, 1.5
    w1, w2 = 1 / tau, 1 / tau2
    cx, cy, W = O.lattice(n)
    one = np.ones((ny, nx))
    rho, T = 1.1, 1.2
    cases = [
        ("f", W * (cx ** 3 - 3 * cx), 1 - w2),          # He3_xxx
        ("f", W * (cx ** 2 * cy - cy), 1 - w2),         # He3_xxy
        ("f", W * cx * cy, 1 - w1),                     # He2_xy
        ("f", W * (cx ** 2 - cy ** 2), 1 - w1),         # normal stress
        ("g", W * cy, 1 - w2),                          # heat flux of g
        ("g", W * (cx ** 2 - 1), 1 - w1),
    ]
    for which, d, ratio in cases:
        k = 0 if n == 4 else 1                      # D2Q16 / D2Q25 of the pair (4, 5)
        o = make(nx, ny, 4, 5, tau, cv, tau2)
        o.init_equilibrium(rho * one, 0.3 * one, -0.2 * one, T * one)
        if k:
            o.set_flags(np.ones((ny, nx), np.uint8))
        eps = 1e-3
        f = o.get_pops(k)
        g = o.get_gpops(k)
        feq, geq = f.copy(), g.copy()
        if which == "f":
            o.set_pops(k, f + eps * d)
        else:
            o.set_gpops(k, g + eps * T * d)
        o.step(1)
        got = (o.get_pops(k) - feq) if which == "f" else (o.get_gpops(k) - geq)
        want = ratio * eps * (d if which == "f" else T * d)
        np.testing.assert_allclose(got, np.broadcast_to(want, got.shape), rtol=0, atol=1e-13)
        other = (o.get_gpops(k) - geq) if which == "f" else (o.get_pops(k) - feq)
        assert np.abs(other).max() < 1e-13


def decay(kind, tau, tau2, cv=1.5, n=4, nx=32, steps=240):
    """Fourier amplitude of T (entropy wave at constant pressure) or of u_y
    (shear wave) against time; returns the fitted decay rate / k^2."""
    ny, A = 2, 1e-3
    x = np.arange(nx)[None, :].repeat(ny, 0)
    kk = 2 * np.pi / nx
    z = np.zeros((ny, nx))
    if kind == "entropy":
        T = 1 + A * np.cos(kk * x)
        rho, uy = 1.0 / T, z
    else:
        T, rho, uy = 1 + z, 1 + z, A * np.cos(kk * x)
    o = make(nx, ny, n, 5, tau, cv, tau2)
    o.init_equilibrium(rho, z, uy, T)
    ts, ys = [], []
    for s in range(steps):
        m = o.moments()
        sig = m[3][0] - 1 if kind == "entropy" else m[2][0]
        ts.append(s * o.dt)
        ys.append(np.sum(sig * np.cos(kk * np.arange(nx))) * 2 / nx)
        o.step(1)
    ts, ys = np.array(ts), np.array(ys)
    lam = -np.polyfit(ts[20:], np.log(np.abs(ys[20:])), 1)[0]
    return lam / kk ** 2, o.dt


def test_thermal_diffusivity_and_prandtl_number():
    tau, tau2 = 0.8, 1.3
    alpha, dt = decay("entropy", tau, tau2)
    nu, _ = decay("shear", tau, tau2)
    assert abs(alpha / ((tau2 - 0.5) * dt) - 1) < 0.03
    assert abs(nu / ((tau - 0.5) * dt) - 1) < 0.03
    cv = 1.5
    pr = (cv + 1) * nu / ((cv + 1) * alpha)                 # C_p mu / kappa with rho = T = 1
    assert abs(pr / ((tau - 0.5) / (tau2 - 0.5)) - 1) < 0.05


@pytest.mark.parametrize("cv", [1.5, 2.5])
def test_sound_speed_gamma(cv):
    gamma = (cv + 1) / cv
    nx, ny, A = 32, 2, 1e-3
    x = np.arange(nx)[None, :].repeat(ny, 0)
    kk = 2 * np.pi / nx
    rho = 1 + A * np.cos(kk * x)
    T = 1 + (gamma - 1) * A * np.cos(kk * x)                # adiabatic
    z = np.zeros_like(rho)
    o = make(nx, ny, 4, 5, 0.51, cv, 0.51)
    o.init_equilibrium(rho, z, z, T)
    c_guess = np.sqrt(gamma)
    ts, ys = [], []
    for s in range(int(1.1 * nx / c_guess / o.dt)):
        r = o.moments()[0]
        ts.append(s * o.dt)
        ys.append(np.sum((r[0] - 1) * np.cos(kk * np.arange(nx))) * 2 / nx)
        o.step(1)
    from scipy.optimize import curve_fit
    f = lambda t, a, g, w: a * np.exp(-g * t) * np.cos(w * t)
    p, _ = curve_fit(f, np.array(ts), np.array(ys), p0=[A, 0.0, kk * c_guess])
    assert abs(p[2] / kk / c_guess - 1) < 2e-3


def test_galilean_boost_by_one_cell_per_step():
    nx, ny, steps = 16, 8, 2
    xg, yg = np.meshgrid(np.arange(nx), np.arange(ny))
    ux = 0.05 * np.sin(2 * np.pi * yg / ny + 0.3)
    uy = 0.04 * np.sin(2 * np.pi * xg / nx + 1.0)
    rho = 1 + 0.02 * np.cos(2 * np.pi * (xg / nx + yg / ny))
    T = 1 + 0.05 * np.sin(2 * np.pi * xg / nx)
    runs = []
    for U in (0.0, 1.0):
        o = make(nx, ny, 4, 5, 0.7, 1.5, 0.9)
        o.init_equilibrium(rho, ux + U / o.dt, uy, T)
        o.step(steps)
        runs.append(o)
    a, b = runs
    for get in (lambda o: o.get_pops(0), lambda o: o.get_gpops(0)):
        np.testing.assert_allclose(get(b), np.roll(get(a), steps, axis=1), rtol=0, atol=5e-12)


@pytest.mark.parametrize("lo,hi", [(3, 5), (4, 5)])
def test_fixed_ends_hold_a_matching_uniform_state(lo, hi):
    """Non-periodic x with end states equal to the interior's uniform state
    (moving, hot): the state is a fixed point, interfaces included."""
    nx, ny = 20, 1
    st = (1.2, 0.8, -0.1, 1.3)
    o = O.Oracle(nx, ny, lo, hi, tau=0.7, frame=O.FRAME_POND, periodic=(False, True))
    o.set_twopop(1.5, 0.9)
    o.set_pond_ends(st, st)
    one = np.ones((ny, nx))
    o.init_equilibrium(st[0] * one, st[1] * one, st[2] * one, st[3] * one)
    fl = np.zeros((ny, nx), np.uint8)
    fl[:, 6:12] = 1
    o.set_flags(fl)
    o._twopop = True
    before = state(o)
    o.step(3)
    for x, y in zip(before, state(o)):
        assert np.abs(x - y).max() < 1e-13


def test_viscosity_law_sets_the_relaxation_rate():
    """mu = mu1 (T/T1)^s: in a uniform non-equilibrium state the stress term
    decays by 1 - omega_1 with omega_1 from mu = (1/omega_1 - 1/2) rho T dt,
    the heat-flux term by 1 - omega_2 with Pr = 2/3."""
    nx, ny = 4, 4
    rho, T, mu1, T1, s, pr = 1.3, 1.7, 0.8, 1.0, 0.5, 2.0 / 3.0
    cx, cy, W = O.lattice(4)
    one = np.ones((ny, nx))
    for d, kind in ((W * cx * cy, 1), (W * (cx ** 3 - 3 * cx), 2)):
        o = make(nx, ny, 4, 5, 0.7, 1.5, 0.9)
        o.set_viscosity_law(mu1, T1, s, pr)
        o.init_equilibrium(rho * one, 0.2 * one, 0.1 * one, T * one)
        f = o.get_pops(0)
        o.set_pops(0, f + 1e-3 * d)
        o.step(1)
        tau1 = mu1 * (T / T1) ** s / (rho * T * o.dt) + 0.5
        w = 1 / tau1 if kind == 1 else 1 / ((tau1 - 0.5) / pr + 0.5)
        np.testing.assert_allclose(o.get_pops(0) - f, np.broadcast_to((1 - w) * 1e-3 * d, f.shape),
                                   rtol=0, atol=1e-13)


def test_rankine_hugoniot_states():
    """The shock inputs: textbook jumps at Ma = 2, gamma = 5/3, and equal
    mass, momentum and energy fluxes on both sides (R = 1, C_v = 3/2)."""
    (r1, u1, t1), (r2, u2, t2) = WL.rankine_hugoniot(2.0)
    assert abs(r2 / r1 - 16 / 7) < 1e-12 and abs(t2 / t1 - 2.078125) < 1e-12
    cv = 1.5
    for a, b in ((r1 * u1, r2 * u2),
                 (r1 * u1 ** 2 + r1 * t1, r2 * u2 ** 2 + r2 * t2),
                 (u1 * (r1 * (cv * t1 + u1 ** 2 / 2) + r1 * t1), u2 * (r2 * (cv * t2 + u2 ** 2 / 2) + r2 * t2))):
        assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("L,refined", [(2000.0, True), (3000.0, False)])
def test_knudsen_criterion_against_the_mean_free_path(L, refined):
    """An instance built with an upstream mean free path of 50 cells
    (mu_1 from lambda_1, as the shock inputs do) and a density slope 1/L
    at rho = 1, T = T_1 has Kn = 50 / L there: refined at Kn = 0.025 > 0.02,
    not at 0.0167; a uniform state is never refined."""
    nx = 201
    inst = WL.shock_batch(1, seed=1, mach_range=(1.5, 1.5), len_range=(nx, nx))[0]
    x = np.arange(nx)[None, :].astype(float)
    rho = 1 + (x - 100) / L
    o = O.Oracle(nx, 1, 4, 5, tau=0.7, frame=O.FRAME_POND, periodic=(False, True))
    o.set_twopop(1.5, 0.8)
    o.set_pond_ends((rho[0, 0] - 1 / L, 0.0, 0.0, 1.0), (rho[0, -1] + 1 / L, 0.0, 0.0, 1.0))
    o.set_viscosity_law(inst["mu1"], 1.0, 0.5, 2 / 3)
    o.init_equilibrium(rho, 0 * rho, 0 * rho, 1 + 0 * rho)
    o.set_kn_criterion(0.02, 1)
    assert bool(o.get_flags()[0, 100]) == refined
    u = O.Oracle(nx, 1, 4, 5, tau=0.7, frame=O.FRAME_POND, periodic=(False, True))
    u.set_twopop(1.5, 0.8)
    u.set_pond_ends((1.0, 0.3, 0.0, 1.0), (1.0, 0.3, 0.0, 1.0))
    u.set_viscosity_law(inst["mu1"], 1.0, 0.5, 2 / 3)
    one = np.ones((1, nx))
    u.init_equilibrium(one, 0.3 * one, 0 * one, one)
    u.set_kn_criterion(0.02, 1)
    u.step(2)
    assert u.get_flags().sum() == 0


def test_knudsen_refined_shock_stays_positive():
    """The paper's shock case (Sec. IV.C: Mach 1.6, lambda_1 = 50 cells,
    initialised on D2Q16 and refined to D2Q25 where Kn > 0.02): with the
    criterion refining only, the cells once high-order stay so and rho, T stay
    positive and within 10 % of the Rankine-Hugoniot range for 100 steps.  The
    same run coarsening cells again where Kn drops below the threshold (flags
    recomputed from scratch every step) loses positivity within 40 steps: in
    this nearly collisionless regime (tau ~ 110 upstream) cells switched back
    and forth at the shock's edges are what breaks it.  1024 cells, so that
    the initial ramp (two mean free paths wide) meets the fixed end states
    without a jump that the criterion would refine; at 640 cells the upstream
    end is refined at once and the run loses positivity next to it after 56
    steps."""
    nx, gamma, thr = 1024, 5.0 / 3.0, 0.02
    inst = WL.shock_batch(1, seed=1, mach_range=(1.6, 1.6), len_range=(nx, nx))[0]
    rho, ux, T = (a[None, :] for a in WL.shock_profile(inst, nx, width=100.0))
    (r1, u1, t1), (r2, u2, t2) = inst["left"], inst["right"]

    def make():
        o = O.Oracle(nx, 1, 4, 5, tau=0.7, frame=O.FRAME_POND, periodic=(False, True))
        o.set_twopop(1.5, 0.8)
        o.set_pond_ends((r1, u1, 0.0, t1), (r2, u2, 0.0, t2))
        o.set_viscosity_law(inst["mu1"], inst["T1"], 0.5, 2 / 3)
        o.init_equilibrium(rho, ux, 0 * rho, T)
        return o

    def positive(o):
        r, _, _, TT = o.moments()
        return np.isfinite(r).all() and (r > 0).all() and np.isfinite(TT).all() and (TT > 0).all()

    o = make()
    o.set_kn_criterion(thr, 1)
    prev = o.get_flags()
    assert prev.sum() > 0
    for _ in range(100):
        o.step(1)
        fl = o.get_flags()
        assert (fl >= prev).all()
        prev = fl
        assert positive(o)
    r = o.moments()[0]
    assert r.min() > 0.9 * r1 and r.max() < 1.1 * r2

    def kn_flags(o):
        r, _, _, TT = o.moments()
        r, TT = r[0], TT[0]
        mu = inst["mu1"] * (TT / inst["T1"]) ** 0.5
        lam = 16 / (5 * np.sqrt(2 * np.pi * gamma)) * mu * np.sqrt(gamma * TT) / (r * TT)
        rp = np.concatenate([[r1], r, [r2]])
        return (lam * np.abs(0.5 * (rp[2:] - rp[:-2])) / r > thr).astype(np.uint8)[None, :]

    o = make()
    broke = None
    for s in range(40):
        o.set_flags(kn_flags(o))
        o.step(1)
        if not positive(o):
            broke = s + 1
            break
    assert broke is not None
