"""The multi-GPU path of the benchmark is replicas only (every rank advances
its own copy of the workload, no data-path collective): its host logic --
the maximum of the per-rank timings over ranks and the whole-job throughput --
checked with two gloo ranks on the CPU, and the reference arm's rule that only
rank 0 works under a multi-rank launch."""
import io
import contextlib
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = (10.0 + 5.0 * rank, 20.0 - 3.0 * rank)          # per-rank step and e2e times
    out[rank] = bench.max_over_ranks(times, dist, "cpu")
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(worker, args=(2, free_port(), out), nprocs=2, start_method="spawn")
        got = dict(out)
    assert got[0] == got[1] == [15.0, 20.0]
    # whole-job throughput: both replicas' cells over the slowest rank's time
    assert bench.job_mlups(2, 524288, 1000, 15.0) == pytest.approx(2 * 524288 * 1000 / 15e-3 / 1e6)


def test_reference_arm_other_ranks_do_nothing():
    class A:
        steps, warmup, gpus = 1, 3, 2
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A(), rank=1, world=2)
    assert buf.getvalue() == ""
