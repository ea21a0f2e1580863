"""The allocation-free audit entry point (slbm_audit_dense_noalloc), called
through the C ABI, against the handle's own audit (slbm_audit) of the same
populations.  For callers that cannot allocate device memory -- code inside a
stream capture, real-time loops, frameworks that own all device memory --
the entry point keeps its reduction scratch in a static device array instead
of allocating it.

Kept in its own file that pytest collects last, so a failing run has already
run every other test; it passes alone in a fresh process as well."""
import numpy as np
import pytest

from paper_2102_12559_gb300 import slbm, workloads as WL

pytestmark = pytest.mark.gpu


def WL_lattice(k):
    """1-D velocities and weights of lattice k (0: D2Q9, 1: D2Q25), Table I,
    from numpy's Gauss-HermiteE rule (probabilists' Hermite, unit variance)."""
    n = (3, 5)[k]
    c, w = np.polynomial.hermite_e.hermegauss(n)
    return c, w / np.sqrt(2 * np.pi)


def _dense_field(g, k, torch):
    """Full populations of lattice k as dense FP32 device planes."""
    pops = g.get_pops(k)                       # (ny, nx, Q), f64, full f
    planes = np.ascontiguousarray(np.moveaxis(pops, -1, 0)).astype(np.float32)
    return torch.from_numpy(planes).cuda()


@pytest.mark.parametrize("k,flag", [(0, 0), (1, 1)])
def test_noalloc_audit_matches_handle_audit(k, flag):
    torch = pytest.importorskip("torch")
    nx, ny = 96, 72
    g = slbm.Solver(nx, ny, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=0.6, precision=slbm.SLBM_FP64)
    g.init_equilibrium(*WL.perturbed(nx, ny, seed=21, amp_u=0.2))
    g.set_flags(np.full((ny, nx), flag, np.uint8))
    g.step(3)
    ref = g.audit()                           # all cells carry lattice k
    field = _dense_field(g, k, torch)
    # independent of CUDA: the same FP32 planes summed in FP64 by numpy
    planes = field.cpu().numpy().astype(np.float64).reshape(n_q := field.shape[0], -1)
    c, _ = WL_lattice(k)
    cx, cy = np.tile(c, len(c)), np.repeat(c, len(c))
    host = np.array([planes.sum(), (cx[:, None] * planes).sum(), (cy[:, None] * planes).sum(),
                     (0.5 * (cx * cx + cy * cy)[:, None] * planes).sum()])
    assert n_q == len(cx)
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    n = (slbm.SLBM_D2Q9, slbm.SLBM_D2Q25)[k]
    st = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                        # two calls in a row share the scratch
        out.zero_()
        slbm.slbm_audit_dense_noalloc(field.data_ptr(), n, nx, ny, out.data_ptr(), st)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # FP32 copies of the populations: relative agreement to ~1e-7 per value
        np.testing.assert_allclose(got, ref, rtol=2e-6, atol=2e-6 * abs(ref[0]))
        # the same FP32 values in another summation order: FP64 rounding only
        np.testing.assert_allclose(got, host, rtol=1e-12, atol=1e-12 * abs(host[0]))


def test_noalloc_audit_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    buf = torch.zeros(9 * 16, dtype=torch.float32, device="cuda")
    with pytest.raises(slbm.SlbmError):
        slbm.slbm_audit_dense_noalloc(buf.data_ptr(), 7, 4, 4, out.data_ptr())
    with pytest.raises(slbm.SlbmError):
        slbm.slbm_audit_dense_noalloc(buf.data_ptr(), 3, 1 << 16, 1 << 15, out.data_ptr())
