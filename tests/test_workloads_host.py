"""Host logic of the seeded workload generators and the benchmark's unit
mappings (no GPU): the Couette channel batch and its relaxation times, and the
roofline traffic's lookup in the committed ncu summary."""
import math

import numpy as np

import bench
from paper_2102_12559_gb300 import workloads as WL


def test_couette_batch_seeded_and_in_range():
    a = WL.couette_batch(count=128, seed=3)
    b = WL.couette_batch(count=128, seed=3)
    assert a == b and len(a) == 128
    assert a != WL.couette_batch(count=128, seed=4)
    hs = np.array([c["H"] for c in a])
    kn = np.array([c["kn"] for c in a])
    assert hs.min() >= 64 and hs.max() <= 512
    assert kn.min() >= 0.01 and kn.max() <= 1.0
    # log-uniform: log Kn spreads over the whole decade pair, centred near log 0.1
    assert abs(np.log(kn).mean() - math.log(0.1)) < 0.4
    assert np.log(kn).min() < math.log(0.02) and np.log(kn).max() > math.log(0.5)
    assert all(c["uw_lo"] == -0.1 and c["uw_hi"] == 0.1 for c in a)


def test_couette_tau_matches_the_mean_free_path():
    """tau = nu / dt + 1/2 with the BGK gas's mean free path
    lambda = (mu / p) sqrt(pi R T / 2) = Kn H at rho = 1, p = rho c_s^2,
    c_s = R T = 1."""
    dt = 1.0 / math.sqrt(5.0 + math.sqrt(10.0))
    for kn, h in ((0.01, 64), (0.3, 200), (1.0, 512)):
        tau = bench.couette_tau(kn, h, dt)
        nu = (tau - 0.5) * dt
        lam = nu * math.sqrt(math.pi / 2.0)
        assert abs(lam - kn * h) < 1e-9 * kn * h
    assert bench.couette_tau(0.02, 100, dt) > bench.couette_tau(0.01, 100, dt) > 0.5


def test_profile_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic is read from the committed ncu summary only
    while the stream kernel's source hash matches the one recorded there."""
    h = bench.kernel_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / bench.PROFILE_SUMMARY).write_text(
        f"- kernel_source_hash: `{h}`\n- dram_bytes_per_launch: `123456`\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: h)
    assert bench.read_traffic(h) == 123456.0
    assert bench.read_traffic("0" * 16) is None
    (prof / bench.PROFILE_SUMMARY).write_text("- kernel_source_hash: `x`\n")
    assert bench.read_traffic(h) is None

