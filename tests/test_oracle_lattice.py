"""Pins of the oracle's velocity sets (Table I, eqs. ci/wi) against the paper's
printed values and against library Gauss-Hermite quadrature."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1.txt")


def _table1():
    rows = {}
    env = {"sqrt": math.sqrt}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        model, TL, c, w, _ = line.split()
        n = int(model[-1])
        assert float(TL) == 1.0
        wv = eval(w, {"__builtins__": {}}, env)
        if c.startswith("+-"):
            cv = eval(c[2:], {"__builtins__": {}}, env)
            rows.setdefault(n, []).extend([(cv, wv), (-cv, wv)])
        else:
            rows.setdefault(n, []).append((eval(c, {"__builtins__": {}}, env), wv))
    return {n: sorted(v) for n, v in rows.items()}


@pytest.mark.parametrize("n", [3, 4, 5])
def test_table1_printed_values(n):
    """Table I, value by value."""
    ref = _table1()[n]
    c, w = O.gh1d(n)
    assert np.all(np.diff(c) > 0)
    np.testing.assert_allclose(c, [r[0] for r in ref], rtol=0, atol=1e-15)
    np.testing.assert_allclose(w, [r[1] for r in ref], rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_nodes_are_hermite_roots_and_library_quadrature(n):
    """The abscissae are the roots of the probabilists' Hermite polynomial He_n
    and the weights those of numpy's Gauss-HermiteE rule (normalised)."""
    c, w = O.gh1d(n)
    x, wl = np.polynomial.hermite_e.hermegauss(n)
    np.testing.assert_allclose(c, x, atol=1e-14)
    np.testing.assert_allclose(w, wl / math.sqrt(2 * math.pi), atol=1e-14)


def _gauss_moment(m, T=1.0):
    return 0.0 if m % 2 else float(np.prod(np.arange(m - 1, 0, -2))) * T ** (m // 2)


@pytest.mark.parametrize("n", [3, 4, 5])
def test_quadrature_degree(n):
    """GH with n nodes is exact for monomials up to degree 2n-1 and not at 2n."""
    c, w = O.gh1d(n)
    for m in range(2 * n):
        assert abs(np.sum(w * c ** m) - _gauss_moment(m)) < 1e-12, m
    assert abs(np.sum(w * c ** (2 * n)) - _gauss_moment(2 * n)) > 1e-3


@pytest.mark.parametrize("n", [3, 4, 5])
def test_tensor_product_lattice(n):
    """Eq. (ci)/(wi): c_i = (c_ix, c_iy), W_i = w_ix w_iy, i = ix + n iy."""
    c, w = O.gh1d(n)
    cx, cy, W = O.lattice(n)
    for iy in range(n):
        for ix in range(n):
            i = ix + n * iy
            assert cx[i] == c[ix] and cy[i] == c[iy]
            assert abs(W[i] - w[ix] * w[iy]) < 1e-16
    assert abs(W.sum() - 1) < 1e-15
    # isotropic second moment = T_L = 1 and vanishing mixed odd moments
    assert abs(np.sum(W * cx * cx) - 1) < 1e-14
    assert abs(np.sum(W * cx * cy)) < 1e-15
