"""FP16 storage of the deviations s_i = f_i - W_i (FP32 arithmetic) against the
FP64 oracle and against the FP32 path.

Tolerances.  Every stored deviation keeps 11 significant bits (a rounding of
up to 2^-11 = 4.9e-4 relative, stochastic in the stream-collide kernel).  In
the 200-step convected vortex the populations' deviations are ~0.02, so each
step perturbs the momentum by ~1e-5 against |u| ~ 0.1: measured relative L2
errors are ~4e-5 on rho and ~6e-4 on u (the jet against FP32: ~5e-5 and
~4e-4).  The bound tested is 1e-4 on rho and 1e-3 on u; the u error is above
the 1e-4 aimed at for the reduced-precision form, a limit of the 11-bit
significand, not of the kernels (FP32 storage of the same path is within
1e-5).
"""
import numpy as np
import pytest

import oracle as O
from paper_2102_12559_gb300 import workloads as WL
from paper_2102_12559_gb300 import slbm

pytestmark = pytest.mark.gpu

FP16, FP32 = slbm.SLBM_FP16, slbm.SLBM_FP32


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def test_info_and_workspace():
    g = slbm.Solver(64, 48, 3, 5, tau=0.6, precision=FP16)
    assert g.info.precision == FP16
    n16 = slbm.slbm_workspace_bytes(64, 48, 1, 1, 3, 5, 3, FP16)
    n32 = slbm.slbm_workspace_bytes(64, 48, 1, 1, 3, 5, 3, FP32)
    assert n16 < n32


def test_uniform_flow_fp16():
    N = 48
    g = slbm.Solver(N, N, 3, 5, tau=0.55, precision=FP16)
    g.init_equilibrium(*WL.uniform(N, N, 1.2, 0.25, -0.15))
    g.set_flags(WL.random_flags(N, N, seed=3))
    g.step(20)
    r, u, v, _ = g.moments()
    assert abs(r - 1.2).max() < 5e-4 and abs(u - 0.25).max() < 5e-4 and abs(v + 0.15).max() < 5e-4


@pytest.fixture(scope="module")
def vortex_oracle():
    L = 64
    rho, ux, uy, disc = WL.convected_vortex(L)
    dt = O.Oracle(8, 8, 3, 5, tau=0.6).dt
    tau = 1e-3 / dt + 0.5
    o = O.Oracle(L, L, 3, 5, tau=tau, order=3)
    o.init_equilibrium(rho, ux, uy)
    o.set_flags(disc)
    o.step(200)
    return dict(fields=(rho, ux, uy), disc=disc, tau=tau, mom=o.moments())


def test_convected_vortex_200_steps_fp16(vortex_oracle):
    L = 64
    g = slbm.Solver(L, L, 3, 5, tau=vortex_oracle["tau"], interp_order=3, precision=FP16)
    g.init_equilibrium(*vortex_oracle["fields"])
    g.set_flags(vortex_oracle["disc"])
    g.step(200)
    mom, ref = g.moments(), vortex_oracle["mom"]
    er = rel_l2(mom[0], ref[0])
    eu = rel_l2(np.stack(mom[1:3]), np.stack(ref[1:3]))
    print(f"FP16 vortex: rel L2 rho {er:.2e}, u {eu:.2e}")
    assert er < 1e-4 and eu < 1e-3


@pytest.mark.xfail(strict=True, reason="the reduced-precision target of 1e-4 relative L2 on u "
                   "is not met by 11-bit storage of f_i - W_i: measured 6e-4 on this vortex")
def test_convected_vortex_fp16_meets_1e4_on_u(vortex_oracle):
    """The 1e-4 relative L2 aimed at for the reduced-precision form, on u.
    Kept as an expected failure so the gap stays visible: the stored
    deviations (~0.02 here, the Mach 0.1 advection) carry 11 significant
    bits, whose rounding alone moves u by ~1e-4 relative per step."""
    L = 64
    g = slbm.Solver(L, L, 3, 5, tau=vortex_oracle["tau"], interp_order=3, precision=FP16)
    g.init_equilibrium(*vortex_oracle["fields"])
    g.set_flags(vortex_oracle["disc"])
    g.step(200)
    mom, ref = g.moments(), vortex_oracle["mom"]
    assert rel_l2(np.stack(mom[1:3]), np.stack(ref[1:3])) < 1e-4


@pytest.mark.parametrize("n_lo,n_hi", [(3, 4), (3, 5), (4, 5)])
def test_one_step_fp16_close_to_oracle(n_lo, n_hi):
    nx, ny = 37, 29
    fields = WL.perturbed(nx, ny, seed=4, amp_rho=0.05, amp_u=0.2)
    fl = WL.random_flags(nx, ny, seed=2, blobs=3, rmin=3, rmax=7)
    g = slbm.Solver(nx, ny, n_lo, n_hi, tau=0.57, precision=FP16)
    o = O.Oracle(nx, ny, n_lo, n_hi, tau=0.57)
    for s in (g, o):
        s.init_equilibrium(*fields)
        s.set_flags(fl)
        s.step(1)
    for k in (0, 1):
        m = fl == k
        # |f - W| <= ~0.2 here: half an FP16 ulp of the stored deviation
        np.testing.assert_allclose(g.get_pops(k)[m], o.get_pops(k)[m], rtol=0, atol=2e-4)


def test_jet_fp16_tracks_fp32():
    """The free jet (inlet / outflow / free-stream boundaries, Mach criterion),
    100 steps: FP16 storage against the FP32 path."""
    nx, ny = 256, 128
    J = WL.free_jet(nx, ny, slot=16, ma_jet=0.5, ma_co=0.05)
    out = []
    for prec in (FP32, FP16):
        g = slbm.Solver(nx, ny, 3, 5, tau=0.55, periodic=(False, False), precision=prec)
        g.init_equilibrium(J["rho"], J["ux"], J["uy"])
        g.set_boundary(slbm.SLBM_SIDE_XMIN, slbm.SLBM_BC_INLET, None, J["in_ux"], J["in_uy"])
        g.set_boundary(slbm.SLBM_SIDE_XMAX, slbm.SLBM_BC_OUTFLOW)
        for side in (slbm.SLBM_SIDE_YMIN, slbm.SLBM_SIDE_YMAX):
            g.set_boundary(side, slbm.SLBM_BC_DIRICHLET, np.full(nx, J["fs_rho"]),
                           np.full(nx, J["fs_ux"]), np.full(nx, J["fs_uy"]))
        g.set_criterion(slbm.SLBM_CRIT_MACH, 0.3)
        g.step(100)
        out.append(g.moments())
    er = rel_l2(out[1][0], out[0][0])
    eu = rel_l2(np.stack(out[1][1:3]), np.stack(out[0][1:3]))
    print(f"FP16 jet vs FP32: rel L2 rho {er:.2e}, u {eu:.2e}")
    assert er < 1e-4 and eu < 1e-3


def test_co_moving_frame_rejects_fp16():
    with pytest.raises(slbm.SlbmError):
        slbm.Solver(32, 32, 3, 5, tau=0.6, precision=FP16, frame=slbm.SLBM_FRAME_POND)
