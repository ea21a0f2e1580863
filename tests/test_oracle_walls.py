"""Pins of the oracle's diffuse-reflection wall (the kinetic wall of the
Couette flow, Sec. IV.C).  The paper names the condition without a formula;
the reading here: populations entering the fluid are the wall-velocity
equilibrium, scaled for zero net normal mass flux against the first interior
node, the rest copy that node.  What fixes it:
- the wall-velocity equilibrium is a fixed point (a uniform flow moving with
  both walls stays uniform, with mixed lattices too);
- zero net normal flux: a closed channel keeps its mass to rounding over
  thousands of steps;
- plane Couette flow between walls at -/+ u_w settles to the antisymmetric,
  linear Navier-Stokes profile in the bulk, with an apparent slip at the
  walls that grows with the relaxation time (the Knudsen number).
"""
import numpy as np
import pytest

import oracle as O
from paper_2102_12559_gb300 import workloads as WL


def channel(nx, ny, lo, hi, tau, uw_lo, uw_hi, flags=None, init_u=0.0):
    o = O.Oracle(nx, ny, lo, hi, tau=tau, periodic=(True, False))
    o.init_equilibrium(*WL.uniform(nx, ny, 1.0, init_u, 0.0))
    if flags is not None:
        o.set_flags(flags)
    o.set_bc(2, O.BC_DIFFUSE, None, np.full(nx, uw_lo), np.zeros(nx))
    o.set_bc(3, O.BC_DIFFUSE, None, np.full(nx, uw_hi), np.zeros(nx))
    return o


@pytest.mark.parametrize("lo,hi", [(3, 4), (3, 5)])
def test_flow_moving_with_the_walls_stays_uniform(lo, hi):
    nx, ny = 12, 14
    fl = np.zeros((ny, nx), np.uint8)
    fl[:4] = 1                       # high-order lattice next to one wall
    o = channel(nx, ny, lo, hi, 0.7, 0.08, 0.08, fl, init_u=0.08)
    o.step(5)
    r, u, v, _ = o.moments()
    assert abs(r - 1).max() < 1e-13 and abs(u - 0.08).max() < 1e-13 and abs(v).max() < 1e-13


def couette(tau, ny=16, uw=0.05, lo=3, hi=4, flags=None):
    nx = 4
    o = channel(nx, ny, lo, hi, tau, -uw, uw, flags)
    m0 = o.audit()[0]
    prev = None
    for _ in range(200):
        o.step(200)
        u = o.moments()[1][:, 0]
        if prev is not None and abs(u - prev).max() < 1e-11:
            break
        prev = u.copy()
    return u, o.audit()[0] / m0 - 1


@pytest.mark.parametrize("tau", [0.65, 0.8, 1.2])
def test_couette_profile_and_mass(tau):
    ny, uw = 16, 0.05
    u, drift = couette(tau, ny, uw)
    assert abs(drift) < 1e-11
    assert abs(u + u[::-1]).max() < 1e-12
    y = np.arange(ny) + 0.5 - ny / 2
    A = np.polyfit(y[3:-3], u[3:-3], 1)
    assert abs(u[3:-3] - np.polyval(A, y[3:-3])).max() < 1e-4 * uw
    # wall speed minus the bulk line at the cell face next to the ghosts: the
    # apparent slip (the scheme's effective wall sits near, not exactly at,
    # that face, so only its size and its growth with tau are pinned)
    slip = uw - A[0] * ny / 2
    assert abs(slip) < 0.1 * uw


def test_slip_grows_with_relaxation_time():
    slips = []
    for tau in (0.65, 0.8, 1.2):
        u, _ = couette(tau)
        y = np.arange(16) + 0.5 - 8
        A = np.polyfit(y[3:-3], u[3:-3], 1)
        slips.append(0.05 - A[0] * 8)
    assert slips[0] < slips[1] < slips[2]
    assert slips[0] < 0.5 * slips[2]


def test_couette_with_high_order_lattice_at_the_walls():
    """The paper's multi-scale Couette arrangement: the high-order lattice in
    the wall layers, the low-order one in the bulk; the profile stays
    antisymmetric and mass is conserved through both interfaces."""
    ny = 16
    fl = np.zeros((ny, 4), np.uint8)
    fl[:3] = 1
    fl[-3:] = 1
    u, drift = couette(0.8, ny, flags=fl)
    assert abs(u + u[::-1]).max() < 1e-12
    assert abs(drift) < 1e-10
    assert np.all(np.diff(u) > 0)
