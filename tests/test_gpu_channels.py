"""Batched channels (slbm_set_channels): many independent micro-Couette
channels side by side in one handle, advanced by one stream-collide and one
post-step launch per step, against one oracle run per channel.

Eight heterogeneous channels: widths 5 .. 33 cells between the walls,
relaxation times 0.52 .. 3, wall speeds of either sign, D2Q9 or D2Q25
channels and one channel with D2Q25 next to its walls and D2Q9 in its middle
(interfaces inside the channel), smooth non-uniform initial fields.  Each
oracle run is the channel alone: width x NY cells, periodic along y (NY 8,
and 4 as in the batched Couette workload, a period shorter than 2 G + 1),
diffuse-reflection walls on its two x sides moving along y.  FP64: every
channel's rho, u within 1e-11 relative L2 of its oracle after 20 steps (only
rounding order differs); FP32 within 1e-5.  The gap columns report flag 2 and
zero moments.
"""
import numpy as np
import pytest

import oracle as O
from paper_2102_12559_gb300 import slbm, workloads as WL

pytestmark = pytest.mark.gpu

NYS = (8, 4)
WIDTHS = [12, 17, 5, 24, 9, 33, 20, 15]
TAUS = [0.6, 1.3, 0.75, 0.52, 3.0, 0.9, 0.55, 2.0]
UW = [(-0.1, 0.1), (0.05, -0.05), (0.0, 0.08), (-0.03, 0.1), (0.1, 0.1), (-0.1, 0.02),
      (0.07, -0.1), (-0.05, 0.05)]
LAT = [0, 1, 0, 1, 0, "walls", 1, 0]   # lattice per channel; "walls": D2Q25 within 4 of a wall


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def _channel_flags(w, lat, NY):
    if lat == "walls":
        f = np.zeros((NY, w), np.uint8)
        f[:, :4] = 1
        f[:, -4:] = 1
        return f
    return np.full((NY, w), lat, np.uint8)


def _setup(NY):
    G = 2
    x0, nx = WL.channel_layout(WIDTHS, G)
    rho = np.ones((NY, nx))
    ux = np.zeros((NY, nx))
    uy = np.zeros((NY, nx))
    flags = np.zeros((NY, nx), np.uint8)
    subs = []
    for c, (w, lat) in enumerate(zip(WIDTHS, LAT)):
        r, u, v = WL.perturbed(w, NY, seed=30 + c, amp_rho=0.02, amp_u=0.05)
        sl = slice(x0[c], x0[c] + w)
        rho[:, sl], ux[:, sl], uy[:, sl] = r, u, v
        fl = _channel_flags(w, lat, NY)
        flags[:, sl] = fl
        subs.append((r, u, v, fl))
    return x0, nx, (rho, ux, uy), flags, subs


def single_channel_runs(NY):
    """Moments of every channel run alone by the oracle (20 steps)."""
    x0, nx, fields, flags, subs = _setup(NY)
    out = []
    for c, (w, (r, u, v, fl)) in enumerate(zip(WIDTHS, subs)):
        o = O.Oracle(w, NY, 3, 5, tau=TAUS[c], order=3, periodic=(False, True))
        o.init_equilibrium(r, u, v)
        o.set_bc(0, O.BC_DIFFUSE, None, np.zeros(NY), np.full(NY, UW[c][0]))
        o.set_bc(1, O.BC_DIFFUSE, None, np.zeros(NY), np.full(NY, UW[c][1]))
        o.set_flags(fl)
        o.step(20)
        out.append(o.moments())
    return NY, out


@pytest.fixture(scope="module", params=NYS)
def oracle_runs(request):
    return single_channel_runs(request.param)


@pytest.mark.parametrize("precision,tol", [(slbm.SLBM_FP64, 1e-11), (slbm.SLBM_FP32, 1e-5)])
def test_channels_match_single_channel_oracle(oracle_runs, precision, tol):
    NY, oracle_runs = oracle_runs
    x0, nx, fields, flags, subs = _setup(NY)
    g = slbm.Solver(nx, NY, 3, 5, tau=0.6, interp_order=3, periodic=(False, True),
                    precision=precision)
    g.init_equilibrium(*fields)
    g.set_channels(x0, WIDTHS, [u[0] for u in UW], [u[1] for u in UW], TAUS)
    g.set_flags(flags)
    g.step(20)
    mom = g.moments()
    got_fl = g.get_flags()
    gap = np.ones(nx, bool)
    for c, w in enumerate(WIDTHS):
        gap[x0[c]:x0[c] + w] = False
        sl = slice(x0[c], x0[c] + w)
        np.testing.assert_array_equal(got_fl[:, sl], subs[c][3])
        ref = oracle_runs[c]
        errs = [rel_l2(mom[q][:, sl], ref[q]) for q in range(3)]
        assert max(errs) < tol, (c, errs)
    assert (got_fl[:, gap] == 2).all()
    for q in range(4):
        assert (mom[q][:, gap] == 0).all()


def test_channels_argument_checks():
    G, NY = 2, 8
    x0, nx = WL.channel_layout([8, 8], G)
    g = slbm.Solver(nx, NY, 3, 5, tau=0.6, periodic=(False, True))
    with pytest.raises(slbm.SlbmError):   # channels overlapping their neighbour's wall columns
        g.set_channels([x0[0], x0[0] + 9], [8, 8], [0, 0], [0, 0], [0.6, 0.6])
    with pytest.raises(slbm.SlbmError):   # too narrow for the stencil
        g.set_channels([x0[0]], [4], [0], [0], [0.6])
    g2 = slbm.Solver(nx, NY, 3, 5, tau=0.6, periodic=(False, False))
    with pytest.raises(slbm.SlbmError):   # y must be periodic
        g2.set_channels(x0, [8, 8], [0, 0], [0, 0], [0.6, 0.6])
