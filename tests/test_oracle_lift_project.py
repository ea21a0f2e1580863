"""Pins of the oracle's lifting and projection (Sec. III.B-C, App. C)."""
import math
import os

import numpy as np
import pytest

import oracle as O

PAIRS = [(3, 4), (3, 5), (4, 5)]


def _rand_pop(n, seed, rho=1.0, u=(0.12, -0.08)):
    rng = np.random.default_rng(seed)
    return O.eq_lattice(n, rho, *u) + 0.01 * rng.standard_normal(n * n)


@pytest.mark.parametrize("nq,nQ", PAIRS)
def test_project_after_lift_is_identity(nq, nQ):
    fq = _rand_pop(nq, 7)
    np.testing.assert_allclose(O.project(nQ, nq, O.lift(nq, nQ, fq)), fq, atol=1e-12)


@pytest.mark.parametrize("nq,nQ", PAIRS)
def test_equilibria_map_to_equilibria(nq, nQ):
    rho, ux, uy = 1.05, 0.25, -0.3
    np.testing.assert_allclose(O.lift(nq, nQ, O.eq_lattice(nq, rho, ux, uy)),
                               O.eq_lattice(nQ, rho, ux, uy), atol=1e-13)
    np.testing.assert_allclose(O.project(nQ, nq, O.eq_lattice(nQ, rho, ux, uy)),
                               O.eq_lattice(nq, rho, ux, uy), atol=1e-13)


@pytest.mark.parametrize("nq,nQ", PAIRS)
def test_lift_keeps_low_moments_fills_rest_from_equilibrium(nq, nQ):
    """M_q = m_q (all q x q moments, non-equilibrium included) and
    M_{Q-q} = moments of the Q equilibrium at the cell's rho, u."""
    fq = _rand_pop(nq, 3)
    fQ = O.lift(nq, nQ, fq)
    cq, dq, _ = O.lattice(nq)
    cQ, dQ, _ = O.lattice(nQ)
    rho = fq.sum(); ux = np.sum(cq * fq) / rho; uy = np.sum(dq * fq) / rho
    feq = O.eq_lattice(nQ, rho, ux, uy)
    for a in range(nQ):
        for b in range(nQ):
            mQ = np.sum(cQ ** a * dQ ** b * fQ)
            ref = np.sum(cq ** a * dq ** b * fq) if (a < nq and b < nq) else np.sum(cQ ** a * dQ ** b * feq)
            assert abs(mQ - ref) < 1e-11 * max(1.0, abs(ref)), (a, b)


@pytest.mark.parametrize("nq,nQ", PAIRS)
def test_projection_keeps_low_moments(nq, nQ):
    fQ = _rand_pop(nQ, 5)
    fq = O.project(nQ, nq, fQ)
    cq, dq, _ = O.lattice(nq)
    cQ, dQ, _ = O.lattice(nQ)
    for a in range(nq):
        for b in range(nq):
            assert abs(np.sum(cq ** a * dq ** b * fq) - np.sum(cQ ** a * dQ ** b * fQ)) < 1e-12


def _golden():
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "appendix_orderings.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = np.array([float(x) for x in v])
    return rows


def test_appendix_c_worked_example():
    """App. C, D2Q9 -> D2Q16 with the paper's velocity orders and moment list:
    M_{9->16} = first 9 moments of f_9 (+) the remaining moments of f^{eq,16};
    f_{9->16} = M_16^{-1} M_{9->16}; f_{16->9} = M_9^{-1} M_{16->9}."""
    g = _golden()
    c = math.sqrt(3)
    c1, c2 = math.sqrt(3 - math.sqrt(6)), math.sqrt(3 + math.sqrt(6))
    ax9, ay9 = c * g["appC_d2q9_cx"], c * g["appC_d2q9_cy"]
    unit = lambda v: np.sign(v) * np.where(np.abs(v) == 1, c1, c2)
    ax16, ay16 = unit(g["appC_d2q16_cx"]), unit(g["appC_d2q16_cy"])
    px, py = g["appC_powx"].astype(int), g["appC_powy"].astype(int)
    M9 = np.array([[ax9[j] ** px[i] * ay9[j] ** py[i] for j in range(9)] for i in range(9)])
    M16 = np.array([[ax16[j] ** px[i] * ay16[j] ** py[i] for j in range(16)] for i in range(16)])

    cx9, cy9, _ = O.lattice(3)
    cx16, cy16, _ = O.lattice(4)
    p9 = [int(np.argmin((cx9 - ax9[j]) ** 2 + (cy9 - ay9[j]) ** 2)) for j in range(9)]
    p16 = [int(np.argmin((cx16 - ax16[j]) ** 2 + (cy16 - ay16[j]) ** 2)) for j in range(16)]

    f9 = _rand_pop(3, 11)          # oracle order
    f9_app = f9[p9]                # paper order
    rho = f9.sum(); ux = np.sum(cx9 * f9) / rho; uy = np.sum(cy9 * f9) / rho
    # f^{eq,16}: lattice equilibrium, moments rho h_a(u_x) h_b(u_y) (Sec. II.C)
    from test_oracle_equilibrium import h
    Mlift = np.concatenate([M9 @ f9_app, [rho * h(px[i], ux) * h(py[i], uy) for i in range(9, 16)]])
    f16_app = np.linalg.solve(M16, Mlift)
    np.testing.assert_allclose(O.lift(3, 4, f9)[p16], f16_app, atol=1e-12)

    f16 = _rand_pop(4, 12)
    f9p_app = np.linalg.solve(M9, (M16 @ f16[p16])[:9])
    np.testing.assert_allclose(O.project(4, 3, f16)[p9], f9p_app, atol=1e-12)


@pytest.mark.parametrize("nq,nQ", PAIRS)
def test_comoving_frame_lift_project(nq, nQ):
    """In a co-moving frame {u, T} the same maps hold: project(lift) = id and
    the co-moving equilibrium rho W lifts to rho W (eq. feqPond)."""
    lam = (0.4, -0.2, 1.3)
    _, _, Wq = O.lattice(nq)
    _, _, WQ = O.lattice(nQ)
    np.testing.assert_allclose(O.lift(nq, nQ, 1.1 * Wq, frame=lam, T_fix=lam[2]), 1.1 * WQ, atol=1e-12)
    np.testing.assert_allclose(O.lift(nq, nQ, 1.1 * Wq, frame=lam, T_fix=0.0), 1.1 * WQ, atol=1e-12)
    fq = 1.1 * Wq + 0.005 * np.random.default_rng(2).standard_normal(nq * nq)
    np.testing.assert_allclose(O.project(nQ, nq, O.lift(nq, nQ, fq, frame=lam, T_fix=0.0), frame=lam),
                               fq, atol=1e-11)
