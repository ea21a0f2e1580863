"""GPU parity at the full size of the benchmark's headline workload: the
4096 x 4096 random-vortex field (512 vortices, peak Mach 0.9), D2Q9 / D2Q25,
cubic streaming, tau = 0.6, Mach criterion, in the launch configuration the
benchmark times (FP32, FP16 and fixed-point deviation storage).

The oracle cannot hold this field, but one step of a cell depends only on
the initial state within the stencil reach (2 cells) of it and on the flags
within twice that (interface conversions), so each sampled output is
computed by the oracle on a 26 x 26 periodic window cut from the same
initial field and flags: the window's 14 x 14 centre is more than 6 cells
from the wrapped edges and sees exactly the full field's data.  Windows: 40
at random positions plus 24 centred on interface cells.  Both sides start
from the same flags (the host's Mach decision on the initial field) and
apply the criterion after the step; every sampled cell's populations in the
lattice of its new flag are compared (flipped cells hold the lifting or
projection of the step's result on both sides).

Tolerances: FP32 2e-6 absolute (as the other full-size check); FP16 storage
rounds the stored deviations f_i - W_i (|s| < 0.25 here) to 11 significant
bits at the start and after the step, 2.5e-4 absolute; companded fixed-point storage
rounds them by at most 2 * A / 32767 (A <= 0.5, twice the largest initial
|s|) = 3e-5 at the start and after the step, 8e-5 absolute.
"""
import numpy as np
import pytest

import oracle as O
from paper_2102_12559_gb300 import slbm, workloads as WL

pytestmark = pytest.mark.gpu

N, W, M = 4096, 26, 6


@pytest.fixture(scope="module")
def field():
    rho, ux, uy = WL.random_vortex_field(N, 512, seed=4, rmin=8.0, rmax=64.0, umax=0.9)
    flags = (np.hypot(ux, uy) > 0.3).astype(np.uint8)
    rng = np.random.default_rng(1)
    centres = [tuple(c) for c in rng.integers(0, N, size=(40, 2))]
    edge = np.argwhere(flags != np.roll(flags, 1, axis=1))
    centres += [tuple(edge[i]) for i in rng.choice(len(edge), 24, replace=False)]
    return rho, ux, uy, flags, centres


def _window(a, cy, cx):
    iy = (np.arange(cy - W // 2, cy + W // 2)) % N
    ix = (np.arange(cx - W // 2, cx + W // 2)) % N
    return np.ascontiguousarray(a[np.ix_(iy, ix)]), iy, ix


@pytest.mark.parametrize("precision,tol", [(slbm.SLBM_FP32, 2e-6), (slbm.SLBM_FP16, 2.5e-4),
                                           (slbm.SLBM_FX16, 8e-5)])
def test_vortex4096_one_step_sampled(field, precision, tol):
    rho, ux, uy, flags, centres = field
    g = slbm.Solver(N, N, 3, 5, tau=0.6, interp_order=3, precision=precision)
    g.init_equilibrium(rho, ux, uy)
    g.set_criterion(slbm.SLBM_CRIT_MACH, 0.3)
    g.set_flags(flags)
    g.step(1)
    new = g.get_flags()
    # the GPU's populations at the sampled cells only
    cells = []
    for cy, cx in centres:
        iy = (np.arange(cy - W // 2 + M, cy + W // 2 - M)) % N
        ix = (np.arange(cx - W // 2 + M, cx + W // 2 - M)) % N
        cells.append((iy[:, None] * N + ix[None, :]).ravel())
    idx = np.concatenate(cells)
    got = []
    for k in (0, 1):
        p = g.get_pops(k).reshape(N * N, -1)
        got.append(p[idx].copy())
        del p
    g.close()
    nflip = 0
    off = 0
    for (cy, cx), c in zip(centres, cells):
        r, iy, ix = _window(rho, cy, cx)
        u, _, _ = _window(ux, cy, cx)
        v, _, _ = _window(uy, cy, cx)
        f, _, _ = _window(flags, cy, cx)
        o = O.Oracle(W, W, 3, 5, tau=0.6, order=3, periodic=(True, True))
        o.init_equilibrium(r, u, v)
        o.set_criterion(1, 0.3)
        o.set_flags(f)
        o.step(1)
        on = o.get_flags()[M:W - M, M:W - M].ravel()
        gn = new.ravel()[c]
        # the criterion's decisions agree wherever |u| is clear of the
        # threshold by more than the storage's rounding
        _, ou, ov, _ = o.moments()
        speed = np.hypot(ou, ov)[M:W - M, M:W - M].ravel()
        clear = np.abs(speed - 0.3) > (1e-5 if precision == slbm.SLBM_FP32 else 2e-3)
        np.testing.assert_array_equal(gn[clear], on[clear])
        nflip += int((on != f[M:W - M, M:W - M].ravel()).sum())
        for k in (0, 1):
            ref = o.get_pops(k)[M:W - M, M:W - M].reshape(-1, 9 if k == 0 else 25)
            m = (on == k) & (gn == k)
            np.testing.assert_allclose(got[k][off:off + len(c)][m], ref[m], rtol=0, atol=tol)
        off += len(c)
    assert nflip > 0
