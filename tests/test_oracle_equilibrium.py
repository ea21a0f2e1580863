"""Pins of the oracle's moment matrices, frame transfer and equilibria
(eqs. momf, fll, feqPond, feqL, feqL0) against the moments the paper prints
(eqs. QxxxPonD, RxxPond, QxxxL, RxxL), Fig. 1's deviation, library inversion
and independent derivations."""
import math
import os

import numpy as np
import pytest

import oracle as O


def h(m, u, T=1.0):
    """Raw Gaussian moment E[(sqrt(T) Z + u)^m]."""
    s = 0.0
    for k in range(0, m + 1, 2):
        s += math.comb(m, k) * u ** (m - k) * float(np.prod(np.arange(k - 1, 0, -2))) * T ** (k // 2)
    return s


@pytest.mark.parametrize("n", [3, 4, 5])
def test_moment_matrix_definition_and_inverse(n):
    lam = (0.13, -0.07, 1.2)
    M = O.moment_matrix(n, *lam)
    cx, cy, _ = O.lattice(n)
    st = math.sqrt(lam[2])
    for r in range(n * n):
        a, b = r % n, r // n
        np.testing.assert_allclose(M[r], (st * cx + lam[0]) ** a * (st * cy + lam[1]) ** b, rtol=1e-15)
    Mi = O.invert(M)
    np.testing.assert_allclose(Mi, np.linalg.inv(M), rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(Mi @ M, np.eye(n * n), atol=1e-11)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_transfer_group_properties(n):
    """G_l^l = I; G_l'^l'' G_l^l' = G_l^l''; moments preserved (eq. fmommatch)."""
    a, b, c = (0.1, 0.2, 1.0), (-0.3, 0.05, 0.8), (0.02, -0.2, 1.3)
    np.testing.assert_allclose(O.transfer(n, a, a), np.eye(n * n), atol=1e-12)
    np.testing.assert_allclose(O.transfer(n, b, c) @ O.transfer(n, a, b), O.transfer(n, a, c),
                               atol=1e-10)
    f = np.random.default_rng(1).uniform(0.0, 0.1, n * n)
    np.testing.assert_allclose(O.moment_matrix(n, *b) @ (O.transfer(n, a, b) @ f),
                               O.moment_matrix(n, *a) @ f, rtol=1e-10, atol=1e-12)


def test_transfer_matches_appendix_b_script():
    """App. B: G = inv(M') M built with the paper's own D2Q9 velocity order and
    moment list (th read as sqrt(theta), unit c = sqrt 3 from Table I)."""
    rows = {}
    for line in open(os.path.join(os.path.dirname(__file__), "golden", "appendix_orderings.txt")):
        if line.strip() and not line.startswith("#"):
            k, *v = line.split()
            rows[k] = np.array([float(x) for x in v])
    c = math.sqrt(3)
    ax, ay = c * rows["appB_d2q9_cx"], c * rows["appB_d2q9_cy"]
    px, py = rows["appB_d2q9_powx"].astype(int), rows["appB_d2q9_powy"].astype(int)

    def Mapp(ux, uy, th):
        return np.array([[(th * ax[j] + ux) ** px[i] * (th * ay[j] + uy) ** py[i] for j in range(9)]
                         for i in range(9)])

    lam, lamp = (0.12, -0.2, 1.1), (0.0, 0.05, 0.9)
    Gapp = np.linalg.inv(Mapp(lamp[0], lamp[1], math.sqrt(lamp[2]))) @ Mapp(lam[0], lam[1], math.sqrt(lam[2]))
    cx, cy, _ = O.lattice(3)
    perm = [int(np.argmin((cx - ax[j]) ** 2 + (cy - ay[j]) ** 2)) for j in range(9)]
    G = O.transfer(3, lam, lamp)
    np.testing.assert_allclose(G[np.ix_(perm, perm)], Gapp, atol=1e-12)


def _phi_solve(n, u, T=1.0):
    """1-D factor of the lattice equilibrium solved independently:
    sum_j c_j^m phi_j = h_m(u) for m < n."""
    c, _ = O.gh1d(n)
    V = np.vander(c, n, increasing=True).T
    return np.linalg.solve(V, [h(m, u, T) for m in range(n)])


@pytest.mark.parametrize("n", [3, 4, 5])
@pytest.mark.parametrize("u", [(0.0, 0.0), (0.1, -0.05), (0.35, 0.2), (-0.6, 0.4)])
def test_lattice_equilibrium_product_form(n, u):
    """Eq. (feqL0) with a tensor-product velocity set factorises into
    rho phi(u_x) phi(u_y), phi solving the 1-D moment conditions."""
    rho = 1.07
    f = O.eq_lattice(n, rho, u[0], u[1])
    ref = rho * np.outer(_phi_solve(n, u[1]), _phi_solve(n, u[0])).ravel()
    np.testing.assert_allclose(f, ref, rtol=1e-11, atol=1e-14)


def test_d2q9_closed_form():
    """D1Q3 factor written out by hand: phi_0 = 1 - (1+u^2)/3,
    phi_(+-) = (1 + u^2 +- sqrt(3) u)/6."""
    ux, uy, rho = 0.21, -0.13, 0.93
    def phi(u):
        s = math.sqrt(3)
        return np.array([(1 + u * u - s * u) / 6, 1 - (1 + u * u) / 3, (1 + u * u + s * u) / 6])
    np.testing.assert_allclose(O.eq_lattice(3, rho, ux, uy), rho * np.outer(phi(uy), phi(ux)).ravel(),
                               rtol=1e-13)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_equilibrium_moments(n):
    """Moments of f^L for a, b < n equal rho h_a(u_x) h_b(u_y): the lattice
    equilibrium matches Maxwell-Boltzmann on every moment the lattice carries."""
    rho, ux, uy = 1.1, 0.27, -0.19
    f = O.eq_lattice(n, rho, ux, uy)
    cx, cy, _ = O.lattice(n)
    for a in range(n):
        for b in range(n):
            assert abs(np.sum(cx ** a * cy ** b * f) - rho * h(a, ux) * h(b, uy)) < 1e-12


def test_printed_third_and_fourth_moments():
    """Eqs. (QxxxL), (RxxL): the D2Q9 lattice equilibrium has Q_xxx = 3 rho T_L u
    and R_xxxx = 3 rho T_L^2 + 3 rho T_L u^2; eqs. (QxxxPonD), (RxxPond): the
    Maxwell values 3 rho T u + rho u^3 and 3 rho T^2 + 6 rho T u^2 + rho u^4,
    which D2Q25 reproduces.  Off-diagonal Q_xyy agree in both (Sec. II.C)."""
    rho, ux, uy = 1.2, 0.31, -0.17
    cx, cy, _ = O.lattice(3)
    f9 = O.eq_lattice(3, rho, ux, uy)
    assert abs(np.sum(cx ** 3 * f9) - 3 * rho * ux) < 1e-13
    assert abs(np.sum(cx ** 4 * f9) - (3 * rho + 3 * rho * ux ** 2)) < 1e-12
    assert abs(np.sum(cx * cy * cy * f9) - (rho * ux + rho * ux * uy * uy)) < 1e-13
    Cx, Cy, _ = O.lattice(5)
    f25 = O.eq_lattice(5, rho, ux, uy)
    assert abs(np.sum(Cx ** 3 * f25) - (3 * rho * ux + rho * ux ** 3)) < 1e-12
    assert abs(np.sum(Cx ** 4 * f25) - (3 * rho + 6 * rho * ux ** 2 + rho * ux ** 4)) < 1e-11


def test_fig1_deviation():
    """Fig. 1: eps = (Q^L_xxx - Q^eq_xxx) / Q^eq_xxx = -Ma^2 / (3 + Ma^2);
    about 3 % at the Ma_thr = 0.3 of Sec. IV.A."""
    cx, _, _ = O.lattice(3)
    for ma in (0.05, 0.1, 0.3, 0.6):
        f = O.eq_lattice(3, 1.0, ma, 0.0)
        eps = (np.sum(cx ** 3 * f) - (3 * ma + ma ** 3)) / (3 * ma + ma ** 3)
        assert abs(eps + ma * ma / (3 + ma * ma)) < 1e-12
    f = O.eq_lattice(3, 1.0, 0.3, 0.0)
    eps = (np.sum(cx ** 3 * f) - (0.9 + 0.027)) / 0.927
    assert round(100 * abs(eps)) == 3


def test_thermal_equilibrium_moments():
    """f^L at T != T_L (eq. feqL) keeps rho, rho u and the kinetic temperature
    on D2Q25 (Maxwell moments up to fourth order)."""
    rho, ux, uy, T = 0.9, 0.2, 0.1, 1.15
    f = O.eq_lattice(5, rho, ux, uy, T)
    cx, cy, _ = O.lattice(5)
    assert abs(f.sum() - rho) < 1e-13
    assert abs(np.sum(cx * f) - rho * ux) < 1e-13
    assert abs(np.sum((cx * cx + cy * cy) * f) - rho * (ux * ux + uy * uy + 2 * T)) < 1e-12
