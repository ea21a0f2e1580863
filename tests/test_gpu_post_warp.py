"""The warp-per-tile post-step kernel on small grids.

`slbm_step` runs the post-step kernel one warp per 32 x 8 tile on grids of
8192 tiles and more, one thread block per tile below; the parity tests of
the small grids therefore exercise the block version, and the 4096^2 field
(`test_gpu_vortex4096.py`) the warp version with periodic sides only.  Here
SLBM_POST_KERNEL=warp makes every handle created in the test use the warp
version, and the oracle parity tests of interfaces under the Mach criterion,
inlet / outflow / Dirichlet sides on a ragged grid, the free jet, diffuse
walls, batched channels (gap columns and internal walls), narrow periodic
grids and indicator-driven flips run again with it, at their own tolerances.
"""
import pytest

import test_gpu_channels as TC
import test_gpu_indicator as TI
import test_gpu_parity as TP
import test_gpu_walls as TW
from paper_2102_12559_gb300 import slbm

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def warp_post_kernel(monkeypatch):
    monkeypatch.setenv("SLBM_POST_KERNEL", "warp")


def test_mach_criterion():
    TP.test_mach_criterion_fp64()


def test_free_jet_boundaries():
    TP.test_free_jet_boundaries_fp64()


@pytest.mark.parametrize("periodic,kinds", [
    ((False, False), ("outflow", "inlet", "dirichlet", "outflow")),
    ((True, False), (None, None, "inlet", "outflow")),
])
def test_mixed_boundaries_ragged(periodic, kinds):
    TP.test_mixed_boundaries_ragged_fp64(periodic, kinds)


@pytest.mark.parametrize("nx,ny", [(10, 4), (40, 2)])
def test_narrow_periodic_grids(nx, ny):
    TP.test_narrow_periodic_grids_fp64(nx, ny)


@pytest.mark.parametrize("lo,hi", [(3, 4), (3, 5), (4, 5)])
def test_walls_one_step(lo, hi):
    TW.test_one_step_fp64(lo, hi)


def test_couette_300_steps():
    TW.test_couette_300_steps(slbm.SLBM_FP64, 1e-12)


def test_channels():
    TC.test_channels_match_single_channel_oracle(TC.single_channel_runs(4), slbm.SLBM_FP64, 1e-11)


@pytest.mark.parametrize("case,crit", [("periodic", slbm.SLBM_CRIT_MLP),
                                       ("walled_high_tau", slbm.SLBM_CRIT_MLP)])
def test_indicator_flips(case, crit):
    TI.test_mlp_flips_match_oracle_replay(case, crit)

