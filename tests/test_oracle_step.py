"""Pins of the oracle's reconstruction and full step (Sec. III.D, eqs.
reconstructionPond / advectionPond / Pond_f_equation): Lagrange exactness,
the stencil rule, conservation, uniform-flow invariance, the pure-streaming
limit against an independent reconstruction, the refinement criterion and
the boundary ghosts."""
import math

import numpy as np
import pytest
from scipy.interpolate import BarycentricInterpolator

import oracle as O
from paper_2102_12559_gb300 import workloads as WL


def sp_lagrange(xs, ys):
    """scipy's Lagrange interpolating polynomial through (xs, ys)."""
    return BarycentricInterpolator(np.asarray(xs, float), np.asarray(ys, float))


@pytest.mark.parametrize("p", [2, 3, 4, 5, 6])
def test_lagrange_exact_up_to_degree(p):
    rng = np.random.default_rng(p)
    xd = 0.37
    x0 = O.first_node(p, xd)
    a = O.lagrange(p, xd, x0)
    nodes = x0 + np.arange(p)
    for deg in range(p):
        coef = rng.standard_normal(deg + 1)
        assert abs(np.dot(a, np.polyval(coef, nodes)) - np.polyval(coef, xd)) < 1e-12
    assert abs(np.dot(a, nodes ** p) - xd ** p) > 1e-6   # order is exactly p - 1
    assert abs(a.sum() - 1) < 1e-15


def test_stencil_rule_and_delta():
    """p points start at floor(x_dep - (p-1)/2 + 1/2): cubic -> floor(x)-1;
    odd p centred on the nearest node, ties up.  Integer x_dep -> delta."""
    assert O.first_node(4, 2.3) == 1 and O.first_node(4, -0.2) == -2
    assert O.first_node(3, 2.4) == 1 and O.first_node(3, 2.5) == 2
    a = O.lagrange(4, 3.0, O.first_node(4, 3.0))
    np.testing.assert_array_equal(a, [0.0, 1.0, 0.0, 0.0])


def test_dt_from_cfl():
    """CFL = max|c| dt / dx = 1 over the lattice pair (Sec. IV)."""
    o = O.Oracle(8, 8, 3, 5, tau=0.6)
    assert abs(o.dt - 1 / math.sqrt(5 + math.sqrt(10))) < 1e-15
    o = O.Oracle(8, 8, 3, 4, tau=0.6)
    assert abs(o.dt - 1 / math.sqrt(3 + math.sqrt(6))) < 1e-15


@pytest.mark.parametrize("flags", ["lo", "hi", "mixed"])
def test_uniform_flow_stays_uniform(flags):
    N = 20
    o = O.Oracle(N, N, 3, 5, tau=0.52)
    o.init_equilibrium(*WL.uniform(N, N, 1.2, 0.25, -0.15))
    fl = {"lo": np.zeros((N, N), np.uint8), "hi": np.ones((N, N), np.uint8),
          "mixed": WL.random_flags(N, N, seed=3)}[flags]
    o.set_flags(fl)
    o.step(4)
    r, u, v, _ = o.moments()
    assert abs(r - 1.2).max() < 1e-13 and abs(u - 0.25).max() < 1e-13 and abs(v + 0.15).max() < 1e-13


@pytest.mark.parametrize("n_lo,n_hi,flag", [(3, 5, 0), (3, 5, 1), (3, 4, 1), (4, 5, 0)])
def test_single_lattice_periodic_conservation(n_lo, n_hi, flag):
    """One lattice, periodic, lattice frame: constant shifts and weights summing
    to one conserve sum_x f_i for every i, so mass and momentum are exact."""
    N = 18
    o = O.Oracle(N, N, n_lo, n_hi, tau=0.55)
    o.init_equilibrium(*WL.perturbed(N, N, seed=1))
    o.set_flags(np.full((N, N), flag, np.uint8))
    a0 = o.audit()
    o.step(6)
    a1 = o.audit()
    np.testing.assert_allclose(a1[:3], a0[:3], rtol=0, atol=1e-12 * a0[0])


@pytest.mark.parametrize("n,flag", [(3, 0), (5, 1)])
def test_pure_streaming_matches_independent_reconstruction(n, flag):
    """omega -> 0 (tau huge): one step is pure semi-Lagrangian streaming; each
    f_i(x) must equal the tensor-product Lagrange interpolant of the old f_i at
    x - c_i dt, rebuilt here with scipy's Lagrange polynomial."""
    N = 12
    o = O.Oracle(N, N, 3, 5, tau=1e30)
    o.init_equilibrium(*WL.perturbed(N, N, seed=4, amp_rho=0.1, amp_u=0.2))
    o.set_flags(np.full((N, N), flag, np.uint8))
    k = flag
    f0 = o.get_pops(k)
    o.step(1)
    f1 = o.get_pops(k)
    cx, cy, _ = O.lattice(n)
    dt = o.dt
    for i in range(n * n):
        for (x, y) in [(0, 0), (5, 7), (11, 3)]:
            sx, sy = cx[i] * dt, cy[i] * dt
            sx = round(sx) if abs(sx - round(sx)) < 1e-12 else sx
            sy = round(sy) if abs(sy - round(sy)) < 1e-12 else sy
            xd, yd = x - sx, y - sy
            x0, y0 = math.floor(xd - 1), math.floor(yd - 1)
            xs, ys = np.arange(x0, x0 + 4), np.arange(y0, y0 + 4)
            rows = []
            for yy in ys:
                vals = [f0[yy % N, xx % N, i] for xx in xs]
                rows.append(sp_lagrange(xs - x0, vals)(xd - x0) if sx != round(sx)
                            else vals[int(round(xd)) - x0])
            ref = sp_lagrange(ys - y0, rows)(yd - y0) if sy != round(sy) else rows[int(round(yd)) - y0]
            assert abs(f1[y, x, i] - ref) < 1e-11, (i, x, y)


def test_equilibrium_is_collision_fixed_point_and_cells_conserve():
    """A uniform equilibrium state is a fixed point; on a generic state every
    updated cell's post-collision rho, rho u equal those of its streamed
    populations, i.e. the step conserves what the reconstruction delivers."""
    N = 10
    o = O.Oracle(N, N, 3, 5, tau=0.7)
    o.init_equilibrium(*WL.uniform(N, N, 0.9, -0.1, 0.2))
    before = o.get_pops(0)
    o.step(1)
    np.testing.assert_allclose(o.get_pops(0), before, atol=1e-15)
    # omega = 1 (tau = 1): post-collision populations ARE the equilibrium of
    # the streamed moments, so re-equilibrating them changes nothing.
    o = O.Oracle(N, N, 3, 5, tau=1.0)
    o.init_equilibrium(*WL.perturbed(N, N, seed=2))
    o.step(1)
    f = o.get_pops(0)
    cx, cy, _ = O.lattice(3)
    for (y, x) in [(0, 0), (3, 4), (9, 9)]:
        r = f[y, x].sum(); ux = np.dot(cx, f[y, x]) / r; uy = np.dot(cy, f[y, x]) / r
        np.testing.assert_allclose(f[y, x], O.eq_lattice(3, r, ux, uy), atol=1e-14)


def test_mach_criterion_flips_and_converts():
    """Sec. IV.A criterion: a cell is high-order iff |u| > 0.3 (c_s = 1),
    decided when the criterion is switched on and again after every step; a
    flipped cell's populations are lifted / projected, so its rho and u are
    unchanged by the flip."""
    N = 16
    rho, ux, uy = WL.uniform(N, N, 1.0, 0.0, 0.0)
    x = np.arange(N)
    ux = ux + 0.5 * np.exp(-((x - N / 2) ** 2) / 8.0)[None, :]
    o = O.Oracle(N, N, 3, 5, tau=0.6)
    o.init_equilibrium(rho, ux, uy)
    r0, u0, v0, _ = o.moments()
    o.set_criterion(1, 0.3)
    fl = o.get_flags()
    np.testing.assert_array_equal(fl, (np.sqrt(ux ** 2 + uy ** 2) > 0.3).astype(np.uint8))
    assert 0 < fl.sum() < N * N
    r1, u1, v1, _ = o.moments()
    np.testing.assert_allclose(r1, r0, atol=1e-14)
    np.testing.assert_allclose(u1, u0, atol=1e-14)
    cx, cy, _ = O.lattice(5)
    f = o.get_pops(1)[fl == 1]
    ref = np.array([O.eq_lattice(5, 1.0, a, 0.0) for a in ux[fl == 1]])
    np.testing.assert_allclose(f, ref, atol=1e-14)      # lift of an equilibrium
    o.step(1)
    r, u, v, _ = o.moments()
    np.testing.assert_array_equal(o.get_flags(), (np.sqrt(u ** 2 + v ** 2) > 0.3).astype(np.uint8))


def test_boundary_ghosts_keep_uniform_flow():
    """Dirichlet, inlet and outflow ghosts all reproduce a uniform state, so a
    uniform flow through a jet-like box stays uniform."""
    nx, ny = 16, 12
    U = (0.2, 0.0)
    o = O.Oracle(nx, ny, 3, 5, tau=0.56, periodic=(False, False))
    o.init_equilibrium(*WL.uniform(nx, ny, 1.0, *U))
    o.set_flags(WL.random_flags(nx, ny, seed=9, blobs=2, rmin=2, rmax=4))
    o.set_bc(0, O.BC_INLET, None, np.full(ny, U[0]), np.full(ny, U[1]))
    o.set_bc(1, O.BC_OUTFLOW)
    o.set_bc(2, O.BC_DIRICHLET, np.ones(nx), np.full(nx, U[0]), np.full(nx, U[1]))
    o.set_bc(3, O.BC_DIRICHLET, np.ones(nx), np.full(nx, U[0]), np.full(nx, U[1]))
    o.step(3)
    r, u, v, _ = o.moments()
    assert abs(r - 1).max() < 1e-13 and abs(u - U[0]).max() < 1e-13 and abs(v).max() < 1e-13


def test_inlet_ghost_is_equilibrium_at_interior_density():
    """Inlet: fixed velocity, density copied from the first interior node
    (zero pressure gradient, Sec. IV.A jet).  A density step at the inlet
    column therefore does not leak a velocity jump into the ghost."""
    nx, ny = 10, 6
    rho, ux, uy = WL.uniform(nx, ny, 1.0, 0.1, 0.0)
    rho[:, 0] = 1.05
    o = O.Oracle(nx, ny, 3, 5, tau=1.0, periodic=(False, True))
    o.init_equilibrium(rho, ux, uy)
    o.set_bc(0, O.BC_INLET, None, np.full(ny, 0.1), np.zeros(ny))
    o.set_bc(1, O.BC_OUTFLOW)
    o.step(1)
    r, u, v, _ = o.moments()
    # the column next to the inlet reads ghosts at rho = 1.05, u = 0.1
    assert abs(v[:, 0]).max() < 1e-13
    assert abs(r[:, 0] - 1.05).max() < 0.02


def test_hybrid_vortex_closer_to_d2q25_than_d2q9():
    """Sec. IV.A: the D2Q9/25 hybrid tracks the all-D2Q25 solution more
    closely than all-D2Q9 does (qualitative pin, a 32^2 vortex at Ma 0.6).
    Run at tau = 0.8: near omega = 2 on so coarse a grid the interface
    perturbation (lifting resets the higher non-equilibrium moments) is of the
    same size as the D2Q9 error itself."""
    L = 32
    rho, ux, uy, disc = WL.convected_vortex(L, U0=0.25, eps=0.6, R=3.2, disc_r=9)
    res = {}
    for name, fl in (("q9", np.zeros_like(disc)), ("q25", np.ones_like(disc)), ("hyb", disc)):
        o = O.Oracle(L, L, 3, 5, tau=0.8)
        o.init_equilibrium(rho, ux, uy)
        o.set_flags(fl)
        o.step(30)
        res[name] = o.moments()[0]
    e_h = np.linalg.norm(res["hyb"] - res["q25"])
    e_9 = np.linalg.norm(res["q9"] - res["q25"])
    assert e_h < 0.5 * e_9
