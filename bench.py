#!/usr/bin/env python
"""Throughput of the multi-scale semi-Lagrangian LBM step on GB300.

Headline workload (default): the large random-vortex field -- 4096 x 4096
periodic cells, 512 Gaussian vortices with random centres, radii 8-64 cells
and signs, rescaled to a peak Mach number of 0.9 (seed 4), rho = 1, D2Q9 /
D2Q25 pair, cubic Lagrange streaming, tau = 0.6.  One bench step = one time
step of the whole path (fused stream-collide with the refinement criterion,
interface conversion, ghost refresh) through the C ABI.

  value            the plain FP32 form: FP32 populations, Mach > 0.3 criterion
                   after every step.
  reduced arm      FP16 storage of the deviations f_i - W_i (FP32 arithmetic),
                   the learned indicator re-flagging every 10 steps, the FP64
                   conservation audit every 1000 steps; timed over one
                   such period, its closing audit included.
  parity           every arm run 200 steps from the same initial state and
                   compared (relative L2 of rho and u) with the FP64 build of
                   the same library, itself at parity with the FP64 oracle.

Timing: W untimed warm-up steps, then K back-to-back steps bracketed by CUDA
events on the solver's stream.  The populations (1.2 GB read and written per
step in FP32) are larger than the 129 MB L2, so L2 is not flushed.
Per-kernel device times come from the library's own event tracing in a
separate pass.

Launch: ``python bench.py`` (1 GPU) or under torchrun with --gpus N: every
rank advances its own replica of the workload (the path is not sharded
across GPUs), value = cell updates of all ranks / max-over-ranks time.
``--impl reference`` times the FP64 CPU oracle on the same workload's cells
instead.  ``--workload`` selects a secondary study (one JSON line each).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "multi-scale SL-LBM MLUPS & % HBM roofline vs plain FP32, at \u22641e-4 rel L2"
UNIT = "MLUPS"
THR = 0.3
# the large random-vortex field
VN, VCOUNT, VSEED, VRMIN, VRMAX, VUMAX, VTAU = 4096, 512, 4, 8.0, 64.0, 0.9, 0.6
VORTEX = (f"large random-vortex field {VN}x{VN} periodic, {VCOUNT} Gaussian vortices (radii "
          f"{VRMIN:g}-{VRMAX:g} cells, random signs, peak Mach {VUMAX}, seed {VSEED}), D2Q9/D2Q25, "
          f"cubic SL streaming, tau {VTAU}")
# oracle sample: crops of the large field
CPU_N = 512
PARITY_STEPS = 200
# the combined reduced arm runs its FP64 audit every AUDIT_EVERY steps; it is
# timed over one such period (the audit at its end inside the timed region)
AUDIT_EVERY = 1000
E2E_STEPS = 10000  # the large field's horizon
# the free jet (secondary study)
NX, NY, SLOT, MA_JET, MA_CO, RE = 1024, 512, 32, 0.5, 0.05, 1000.0
JET = ("free jet 1024x512, FP32, D2Q9/D2Q25, cubic SL streaming, Mach>0.3 criterion "
       "every step, inlet/outflow/free-stream boundaries")
FALLBACK_HBM_GBS = 6800.0
KERNEL_FILES = ["slbm_stream.cuh", "slbm_ghost.cuh", "slbm_impl.cuh", "slbm_eq.cuh", "slbm_stream_f32.cu"]
PROFILE_SUMMARY = "stream_collide_vortex4096.md"
def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_FILES:
        with open(os.path.join(ROOT, "paper_2102_12559_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def jet_tau(dt: float) -> float:
    nu = MA_JET * SLOT / RE
    return nu / dt + 0.5


def couette_tau(kn: float, h: int, dt: float) -> float:
    """Relaxation time of a Couette channel of height h cells at Knudsen
    number kn: mean free path lambda = kn h cells, kinematic viscosity
    nu = lambda c_s sqrt(2 / pi) (the BGK gas's lambda = (mu / p) sqrt(pi R T / 2)
    with c_s = 1), tau = nu / dt + 1/2."""
    nu = kn * h * np.sqrt(2.0 / np.pi)
    return nu / dt + 0.5


def setup_jet(solver, slbm, J):
    solver.set_boundary(slbm.SLBM_SIDE_XMIN, slbm.SLBM_BC_INLET, None, J["in_ux"], J["in_uy"])
    solver.set_boundary(slbm.SLBM_SIDE_XMAX, slbm.SLBM_BC_OUTFLOW)
    for side in (slbm.SLBM_SIDE_YMIN, slbm.SLBM_SIDE_YMAX):
        solver.set_boundary(side, slbm.SLBM_BC_DIRICHLET, np.full(NX, J["fs_rho"]),
                            np.full(NX, J["fs_ux"]), np.full(NX, J["fs_uy"]))


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBps", "hbm_copy_gbs"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def read_traffic(khash: str):
    """DRAM bytes per stream-collide launch from the committed ncu summary,
    valid only if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", PROFILE_SUMMARY)
    try:
        txt = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_source_hash") != khash:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling while the GPU is loaded."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.uuid = uuid

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(values, dist, device):
    """The per-rank timings reduced to their maximum over ranks (every rank
    gets the result); dist None: a single process."""
    import torch
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def job_mlups(world: int, ncell: int, steps: int, ms: float) -> float:
    """Whole-job throughput of `world` replicas, each advancing `ncell` cells
    `steps` times in `ms` milliseconds (the slowest rank's time)."""
    return world * ncell * steps / (ms * 1e-3) / 1e6


def time_steps(solver, stream, steps, warmup, audit_every=0):
    """Mean device milliseconds of one step over `steps` back-to-back steps
    (with `audit_every`, the FP64 audit after every that many steps and at the
    end, inside the timed region)."""
    import torch
    solver.step(warmup)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    if audit_every:
        done = 0
        while done < steps:
            k = min(audit_every, steps - done)
            solver.step(k)
            solver.audit()
            done += k
    else:
        solver.step(steps)
    b.record(stream)
    torch.cuda.synchronize()
    solver.sync()
    return a.elapsed_time(b) / steps


def profiled(g, steps):
    """Per-kernel device milliseconds (summed) and step count over `steps`
    traced steps (separate from the timed ones)."""
    g.profile(True)
    g.step(steps)
    out = g.profile_read()
    g.profile(False)
    return out


# ------------------------------------------------------------------ oracle timing
# (module-level so that spawned worker processes can import them)

_ORC = {}


def _oracle_crop(fields, n: int, k: int):
    """The k-th n x n crop (along the diagonal) of the large field."""
    o = (k * n) % VN
    return [np.ascontiguousarray(f[o:o + n, o:o + n]) for f in fields]


def _oracle_setup(crop):
    """An n x n crop of the large field in the FP64 oracle, taken as
    periodic, Mach criterion on (the crop's flags are set at once)."""
    import oracle as O
    rho, ux, uy = crop
    n = rho.shape[0]
    o = O.Oracle(n, n, 3, 5, tau=VTAU, order=3, periodic=(True, True))
    o.init_equilibrium(rho, ux, uy)
    o.set_criterion(1, THR)
    return o


def _oracle_steps(job):
    """Worker: `steps` full oracle steps of its crop; (cells, seconds)."""
    crop, steps = job
    o = _oracle_setup(crop)
    t = time.perf_counter()
    o.step(steps)
    return crop[0].size * steps, time.perf_counter() - t


def _oracle_pool_init(crops, sample: int):
    import multiprocessing as _mp
    ident = _mp.current_process()._identity
    k = (ident[0] - 1) if ident else 0
    crop = crops[k % len(crops)]
    _ORC["o"] = _oracle_setup(crop)
    _ORC["cells"] = np.random.default_rng(k).choice(crop[0].size, sample, replace=False)


def _oracle_sample_step(_):
    """Worker: one step's update of the worker's fixed cell sample; seconds."""
    t = time.perf_counter()
    _ORC["o"].step_cells(_ORC["cells"])
    return time.perf_counter() - t


def vortex_fields():
    from paper_2102_12559_gb300 import workloads as WL
    return WL.random_vortex_field(VN, VCOUNT, seed=VSEED, rmin=VRMIN, rmax=VRMAX, umax=VUMAX)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(fields):
    """The FP64 oracle as it stands, on the host cores: full time steps of
    512 x 512 crops of the large field (taken as periodic), one process
    alone, then one process per host core at once (each on its own crop),
    processes started with spawn."""
    ctx = mp.get_context("spawn")
    cores = host_cores()
    steps1, stepsn = 2, 1
    with ctx.Pool(1) as pool:
        cells, el = pool.map(_oracle_steps, [(_oracle_crop(fields, CPU_N, 0), steps1)])[0]
    one = cells / el / 1e6
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_steps, [(_oracle_crop(fields, CPU_N, i), stepsn)
                                       for i in range(cores)], chunksize=1)
    alln = sum(c / e for c, e in res) / 1e6
    return {"value": alln, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full FP64 time steps of {CPU_N}x{CPU_N} crops of the same field (taken as "
                      f"periodic, Mach criterion): {cores} processes at once, {stepsn} step each on "
                      f"its own crop (sum of their rates); one process alone: {one:.4f} MLUPS over "
                      f"{steps1} steps",
            "single_core": {"value": one, "unit": UNIT, "cores": 1}}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle on the host cores, every step a
    bounded sample of the workload -- one process per host core, each updating
    a fixed random sample of 1024 cells of its own 512 x 512 crop of the large
    field (the step's post-collision vectors, state not advanced)."""
    if rank != 0:
        return
    cores = host_cores()
    sample = 1024
    fields = vortex_fields()
    crops = [_oracle_crop(fields, CPU_N, i) for i in range(cores)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_oracle_pool_init, initargs=(crops, sample)) as pool:
        for _ in range(args.warmup):
            pool.map(_oracle_sample_step, range(cores), chunksize=1)
        t = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_sample_step, range(cores), chunksize=1)
        el = time.perf_counter() - t
    value = cores * sample * args.steps / el / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": VORTEX, "nx": VN, "ny": VN},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"per step, {cores} processes each update {sample} random cells "
                                   f"of their own {CPU_N}x{CPU_N} crop of the field "
                                   "(one step's update of each), FP64"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def rel_l2(a, b) -> float:
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def mom_gap(a, b) -> dict:
    """Relative L2 gaps of rho, u (the vector field) and its components."""
    return {"rho": rel_l2(a[0], b[0]), "u": rel_l2(np.stack(a[1:3]), np.stack(b[1:3])),
            "ux": rel_l2(a[1], b[1]), "uy": rel_l2(a[2], b[2])}


KN_HI = 0.1  # plain rule of the Couette batch: channels above it run D2Q25
WALL_BAND = 8  # cells of D2Q25 next to each wall in the fixed wall-layer arm
COUETTE_NY = 4  # streamwise period of the Couette channels, cells


def couette_solver(slbm, WL, batch, mode, weights=None, stream=None):
    """The batched Couette channels in one handle: side by side along x
    (wall-normal), streamwise y periodic with COUETTE_NY cells, 2 G gap
    columns, each channel its own tau.  mode: "plain" (D2Q25 in the channels
    with Kn > KN_HI, fixed), "walls" (D2Q25 within WALL_BAND cells of every
    wall, D2Q9 inside, the paper's layout), "all" (D2Q25 everywhere) or "mlp" (the
    learned indicator refines the flags every 10 steps, from D2Q9 at rest:
    SLBM_CRIT_MLP_REFINE, a cell once high-order stays so)."""
    G, ny = 2, COUETTE_NY
    widths = [ch["H"] for ch in batch]
    x0, nx = WL.channel_layout(widths, G)
    probe = slbm.Solver(8, 8, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=0.6)
    dt = probe.dt
    probe.close()
    taus = [couette_tau(ch["kn"], ch["H"], dt) for ch in batch]
    g = slbm.Solver(nx, ny, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=0.6, periodic=(False, True),
                    stream=stream)
    g.init_equilibrium(*WL.uniform(nx, ny))
    g.set_channels(x0, widths, [ch["uw_lo"] for ch in batch], [ch["uw_hi"] for ch in batch],
                   taus)
    fl = np.zeros((ny, nx), np.uint8)
    for c, ch in enumerate(batch):
        if mode == "all" or (mode == "plain" and ch["kn"] > KN_HI):
            fl[:, x0[c]:x0[c] + widths[c]] = 1
        if mode == "walls":
            fl[:, x0[c]:x0[c] + WALL_BAND] = 1
            fl[:, x0[c] + widths[c] - WALL_BAND:x0[c] + widths[c]] = 1
    g.set_flags(fl)
    if mode == "mlp":  # refinement only: at tau up to ~170 cells must not switch back
        g.set_indicator(weights, interval=10)
        g.set_criterion(slbm.SLBM_CRIT_MLP_REFINE, 0.0)
    return g, x0, widths


def plain_couette_flags(batch, x0, widths, shape):
    fl = np.zeros(shape, np.uint8)
    for c, ch in enumerate(batch):
        if ch["kn"] > KN_HI:
            fl[:, x0[c]:x0[c] + widths[c]] = 1
    return fl


def train_indicator(slbm, WL, stream):
    """Indicator weights trained on the GPU (slbm_mlp_train) from states of
    all-D2Q25 runs labelled by the method's own lattice loss (what D2Q9 loses
    in one step, above the indicator's threshold): a 384^2 random-vortex field
    of the benchmark's generator (12 vortices, seed 5) after 20 steps, and a
    batch of 32 Couette channels (seed 11, a different draw than the
    benchmark's) after 300, 1500 and 6000 steps.  Returns the weights and a
    report of the training set and fit."""
    from paper_2102_12559_gb300 import indicator as IND
    xs, ys = [], []
    n_tr = 384
    t = slbm.Solver(n_tr, n_tr, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=VTAU, stream=stream)
    t.init_equilibrium(*WL.random_vortex_field(n_tr, 12, seed=5, rmin=VRMIN, rmax=VRMAX, umax=VUMAX))
    t.set_flags(np.ones((n_tr, n_tr), np.uint8))
    t.step(20)
    xs.append(t.indicator_eval()[0].reshape(-1, 16))
    ys.append(IND.labels(t.lattice_loss()).ravel())
    t.close()
    tb = WL.couette_batch(count=32, seed=11)
    c, x0, widths = couette_solver(slbm, WL, tb, "all", stream=stream)
    inside = np.zeros(c.nx, bool)
    for k, w in enumerate(widths):
        inside[x0[k]:x0[k] + w] = True
    done = 0
    for at in (300, 1500, 6000):
        c.step(at - done)
        done = at
        fe = c.indicator_eval()[0][:, inside].reshape(-1, 16)
        lab = IND.labels(c.lattice_loss()[:, inside]).ravel()
        done += 1
        xs.append(fe)
        ys.append(lab)
    c.close()
    x = np.concatenate(xs).astype(np.float64)
    y = np.concatenate(ys)
    w, losses = IND.train_gpu(x, y, epochs=20, batch=512, lr=3e-3, seed=0, balance=True)
    hit = IND.forward(w, x)[0] > 0
    pos = y > 0.5
    report = {"samples": int(len(y)), "positive_fraction": float(y.mean()),
              "gpu_steps": int(len(losses)), "first_loss": float(losses[0]),
              "last_loss": float(np.mean(losses[-50:])),
              "train_agreement": float(np.mean(hit == pos)),
              "train_balanced_accuracy": float(0.5 * (hit[pos].mean() + (~hit[~pos]).mean())),
              "labels": f"lattice loss > {IND.LOSS_THRESHOLD} on all-D2Q25 states",
              "trainer": "slbm_mlp_train (one-block Adam kernel, FP16 operands, FP32 accumulation)"}
    return w, report


def decision_gaps(a, b, c, mask=None):
    """Disagreement rates between three 0 / 1 flag fields (over `mask`)."""
    m = np.ones(a.shape, bool) if mask is None else mask
    a, b, c = a[m] > 0, b[m] > 0, c[m] > 0
    return float(np.mean(a != b)), float(np.mean(a != c)), float(np.mean(b != c))


def indicator_check_vortex(slbm, fields, weights, stream):
    """The learned indicator's decisions on the benchmark field: an all-D2Q25
    FP32 run of PARITY_STEPS steps, then per cell the indicator's flag, the
    plain Mach criterion and the method's label (lattice loss above the
    threshold) on that state."""
    from paper_2102_12559_gb300 import indicator as IND
    g = slbm.Solver(VN, VN, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=VTAU, stream=stream)
    g.init_equilibrium(*fields)
    g.set_flags(np.ones((VN, VN), np.uint8))
    g.step(PARITY_STEPS)
    g.set_indicator(weights, interval=10)
    _, _, ind = g.indicator_eval(features=False, flags=True)
    _, mu, mv, _ = g.moments()
    mach = np.hypot(mu, mv) > THR
    lab = IND.labels(g.lattice_loss()) > 0.5
    g.close()
    d_im, d_il, d_ml = decision_gaps(ind, mach, lab)
    return {"state": f"all-D2Q25 FP32 run, {PARITY_STEPS} steps",
            "indicator_vs_plain_mach": d_im, "indicator_vs_lattice_loss_label": d_il,
            "plain_mach_vs_lattice_loss_label": d_ml,
            "fraction_flagged": {"indicator": float(ind.mean()), "plain_mach": float(mach.mean()),
                                 "label": float(lab.mean())}}


def vortex_arm(slbm, stream, fields, precision, weights=None):
    """A solver on the large field: Mach criterion every step, or (weights)
    the learned indicator every 10 steps."""
    g = slbm.Solver(VN, VN, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=VTAU, interp_order=3,
                    precision=precision, stream=stream)
    g.init_equilibrium(*fields)
    if weights is not None:
        g.set_indicator(weights, interval=10)
        g.set_criterion(slbm.SLBM_CRIT_MLP, 0.0)
    else:
        g.set_criterion(slbm.SLBM_CRIT_MACH, THR)
    return g


def headline(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    fields = vortex_fields()
    # the oracle's processes start before the first GPU call
    cpu = cpu_baseline(fields) if (world == 1 and not args.no_cpu_baseline) else None

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2102_12559_gb300 import slbm, workloads as WL
    stream = torch.cuda.current_stream(dev)
    ncell = VN * VN
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)

    # ---- the plain FP32 form: K back-to-back steps after W warm-up steps
    g = vortex_arm(slbm, stream, fields, slbm.SLBM_FP32)
    g.step(args.warmup)
    torch.cuda.synchronize(dev)
    flags_before = g.get_flags()
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    g.step(args.steps)
    b.record(stream)
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    total_ms = a.elapsed_time(b)
    g.sync()
    flags_after = g.get_flags()
    kern, ksteps = profiled(g, min(args.steps, 50))
    kern_ms = [k / max(ksteps, 1) for k in kern]
    kps = g.info.kernels_per_step
    g.close()

    # ---- end to end through the C ABI with pinned host buffers: the H2D of
    # rho and u, the criterion, E steps and the D2H of rho and u
    pin = [torch.from_numpy(np.ascontiguousarray(f, dtype=np.float64).ravel()).pin_memory()
           for f in fields]
    outs = [torch.empty(ncell, dtype=torch.float64).pin_memory() for _ in range(4)]
    g = slbm.Solver(VN, VN, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=VTAU, interp_order=3,
                    precision=slbm.SLBM_FP32, stream=stream)
    torch.cuda.synchronize(dev)
    e2e_steps = args.e2e_steps
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    slbm.slbm_init_equilibrium(g.h, ncell, pin[0].numpy(), pin[1].numpy(), pin[2].numpy())
    slbm.slbm_set_criterion(g.h, slbm.SLBM_CRIT_MACH, THR)
    slbm.slbm_step(g.h, e2e_steps)
    slbm.slbm_moments(g.h, ncell, *[o.numpy() for o in outs])
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    e2e_ms = ev0.elapsed_time(ev1)
    g.close()
    h2d, d2h = ncell * 3 * 8, ncell * 4 * 8

    total_ms, e2e_ms = max_over_ranks((total_ms, e2e_ms), dist, dev)
    if rank != 0:
        dist.barrier()
        dist.destroy_process_group()
        return

    # ---- reduced-precision arms (rank 0): FP16 and fixed-point storage
    # alone, and FP16 with the learned indicator every 10 steps and the FP64
    # audit every 1000
    weights, ind_train = train_indicator(slbm, WL, stream)
    ind_vortex = indicator_check_vortex(slbm, fields, weights, stream)
    arms = {}
    for name, prec, learned in (("fp16", slbm.SLBM_FP16, False), ("fx16", slbm.SLBM_FX16, False),
                                ("fp16+indicator+audit", slbm.SLBM_FP16, True)):
        r = vortex_arm(slbm, stream, fields, prec, weights if learned else None)
        r.step(args.warmup)
        if learned:
            ms = time_steps(r, stream, AUDIT_EVERY, 0, audit_every=AUDIT_EVERY)
        else:
            ms = time_steps(r, stream, args.steps, 0)
        kr, kst = profiled(r, min(args.steps, 50))
        arms[name] = {"ms": ms, "kern": [k / max(kst, 1) for k in kr]}
        r.close()
    # the plain FP32 form over the same window as the combined arm (the field's
    # high-order fraction, and with it the step's cost, changes over the
    # window), for that arm's speed-up
    r = vortex_arm(slbm, stream, fields, slbm.SLBM_FP32)
    r.step(args.warmup)
    fp32_audit_ms = time_steps(r, stream, AUDIT_EVERY, 0)
    r.close()

    # ---- parity: every arm PARITY_STEPS steps from the initial state against
    # the FP64 build of the library
    moms = {}
    for name, prec, learned in (("fp64", slbm.SLBM_FP64, False), ("fp32", slbm.SLBM_FP32, False),
                                ("fp16", slbm.SLBM_FP16, False), ("fx16", slbm.SLBM_FX16, False),
                                ("fp16+indicator+audit", slbm.SLBM_FP16, True)):
        r = vortex_arm(slbm, stream, fields, prec, weights if learned else None)
        if learned:
            r.step(PARITY_STEPS)
            r.audit()
        else:
            r.step(PARITY_STEPS)
        fl = r.get_flags()
        moms[name] = (r.moments(), fl)
        r.close()
    ref, ref_fl = moms["fp64"]
    # the refinement-independent reference: D2Q25 everywhere, FP64
    r = slbm.Solver(VN, VN, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=VTAU, interp_order=3,
                    precision=slbm.SLBM_FP64, stream=stream)
    r.init_equilibrium(*fields)
    r.set_flags(np.ones((VN, VN), np.uint8))
    r.step(PARITY_STEPS)
    ref_hi = r.moments()
    r.close()

    def arm_line(name, ms, kern, fp32_ms=None):
        m, fl = moms[name]
        return {"value": ncell / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                "speedup_vs_fp32": (fp32_ms if fp32_ms else total_ms / args.steps) / ms,
                "kernels_ms_per_step": dict(zip(slbm.KERNEL_NAMES, kern)),
                "rel_l2_vs_fp64_at_200_steps": mom_gap(m[:3], ref[:3]),
                "rel_l2_vs_fp32_at_200_steps": mom_gap(m[:3], moms["fp32"][0][:3]),
                "rel_l2_vs_all_d2q25_fp64_at_200_steps": mom_gap(m[:3], ref_hi[:3]),
                "flags_agree_with_fp64_run": float(np.mean(fl == ref_fl)),
                "high_order_fraction_at_200_steps": float(fl.mean())}

    value = job_mlups(world, ncell, args.steps, total_ms)
    e2e_value = job_mlups(world, ncell, e2e_steps, e2e_ms)
    nhi = 0.5 * (int(flags_before.sum()) + int(flags_after.sum()))
    # algorithmic bytes of one stream-collide launch (FP32): read + write Q
    # populations per cell, read the flag, write the next flag
    bytes_sc = ncell * (8 * 9 + 2) + nhi * 8 * (25 - 9)
    sc_ms = kern_ms[0]
    achieved = bytes_sc / (sc_ms * 1e-3) / 1e9
    peak, peak_src = read_peaks()
    khash = kernel_hash()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": VORTEX, "nx": VN, "ny": VN, "lattices": "D2Q9/D2Q25",
                   "interp_order": 3, "tau": VTAU, "criterion": f"Mach>{THR} after every step",
                   "high_order_fraction": nhi / ncell,
                   "l2": "not flushed: the populations (1.2 GB read and written per step) are "
                         "larger than L2",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": read_traffic(khash),
                     "kernel": "stream_collide", "algorithmic_bytes_per_launch": bytes_sc,
                     "launch_ms": sc_ms, "peak_source": peak_src, "kernel_source_hash": khash},
        "kernels_ms_per_step": dict(zip(slbm.KERNEL_NAMES, kern_ms)),
        "reduced_precision_arm": dict(
            arm_line("fp16+indicator+audit", arms["fp16+indicator+audit"]["ms"],
                     arms["fp16+indicator+audit"]["kern"], fp32_ms=fp32_audit_ms),
            fp32_ms_per_step_same_window=fp32_audit_ms,
            form="FP16 storage of f_i - W_i with FP32 arithmetic, learned indicator every 10 steps, "
                 f"FP64 audit every {AUDIT_EVERY} steps",
            steps_timed=AUDIT_EVERY,
            timed="one audit period: the indicator evaluations and the closing FP64 audit inside "
                  "the timed region; speed-up against the plain FP32 form timed over the same "
                  "steps"),
        "fp16_storage_arm": dict(arm_line("fp16", arms["fp16"]["ms"], arms["fp16"]["kern"]),
                                 form="FP16 storage of f_i - W_i, Mach criterion every step"),
        "fx16_storage_arm": dict(arm_line("fx16", arms["fx16"]["ms"], arms["fx16"]["kern"]),
                                 form="16-bit fixed-point storage of f_i - W_i (one scale per "
                                      "plane), Mach criterion every step"),
        "indicator": {"training": ind_train, "on_this_field": ind_vortex},
        "fp32_parity": {"rel_l2_vs_fp64_at_200_steps": mom_gap(moms["fp32"][0][:3], ref[:3]),
                        "rel_l2_vs_all_d2q25_fp64_at_200_steps": mom_gap(moms["fp32"][0][:3],
                                                                          ref_hi[:3]),
                        "fp64_mach_run_vs_all_d2q25_fp64": mom_gap(ref[:3], ref_hi[:3]),
                        "flags_agree_with_fp64_run": float(np.mean(moms["fp32"][1] == ref_fl)),
                        "reference": "FP64 build of the library (at 1e-11 parity with the FP64 "
                                     "oracle), Mach criterion every step, 200 steps"},
        "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
                "path": "slbm_init_equilibrium (pinned host rho, u) + slbm_set_criterion + "
                        "slbm_step + slbm_moments (pinned host rho, u, T), FP32"},
        "gpu_launches": args.steps * kps,
        "clocks": clk,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_study(args):
    """Secondary measurements, one JSON line each (not the headline line).

    vortex-fp32: the headline's plain FP32 form alone, on an N x N field of the
      same generator and vortex density (--size N).

    jet: the free jet 1024 x 512 (FP32, inlet / outflow / free stream, Mach
      criterion every step), cold-L2 and back-to-back step times.

    strip: the efficiency study of Sec. IV.C -- N x N periodic grids, all-D2Q9,
      all-D2Q25 and a hybrid whose left 10 % of columns are D2Q25; reports
      t_Q25 / t_Q9 and t_Q25 / t_hyb next to the paper's 2.9 and 2.43.
    pond: the co-moving (PonD) frame step, thermal, 1024 x 512 periodic,
      FP32, D2Q9 with a D2Q25 disc, a smooth seeded field around a Mach 1.5
      mean flow at T = 1.
    shock: the batched shock structure problem of Sec. IV.C -- 256 independent
      quasi-1-D instances (Mach 1.2-4.0, 1024-8192 cells, Rankine-Hugoniot
      states, lambda_1 = 50 cells) advanced together, two-population
      co-moving model with the hard-sphere viscosity law; block shape from
      the autotuner; D2Q16 refined to D2Q25 where Kn > 0.02 (refinement only,
      every step), against D2Q25 everywhere.
    couette: the batched high-Knudsen Couette channels -- 128 independent
      channels (H x 4, H 64-512, Kn 0.01-1 log-uniform, diffuse walls moving
      at -0.1 / +0.1), side by side in one grid of one handle, in three arms:
      the plain rule (D2Q25 in channels with Kn > 0.1), the learned indicator
      (trained on the GPU from lattice-loss labels) and all-D2Q25 (reference).
    """
    import torch
    from paper_2102_12559_gb300 import slbm, workloads as WL
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    if args.workload == "vortex-fp32":
        # the headline's plain FP32 form alone on an N x N field of the same
        # generator and vortex density (N = --size): W + K back-to-back steps
        # and the per-kernel split (used for profiler captures)
        n = args.size
        count = max(1, VCOUNT * n * n // (VN * VN))
        fields = WL.random_vortex_field(n, count, seed=VSEED, rmin=VRMIN, rmax=VRMAX, umax=VUMAX)
        g = slbm.Solver(n, n, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=VTAU, interp_order=3,
                        precision=slbm.SLBM_FP32, stream=stream)
        g.init_equilibrium(*fields)
        g.set_criterion(slbm.SLBM_CRIT_MACH, THR)
        ms = time_steps(g, stream, args.steps, args.warmup)
        kern, ksteps = profiled(g, min(args.steps, 50))
        nhi = int(g.get_flags().sum())
        sc_ms = kern[0] / max(ksteps, 1)
        bytes_sc = n * n * (8 * 9 + 2) + nhi * 8 * (25 - 9)
        print(json.dumps({
            "study": "plain FP32 form of the random-vortex field", "n": n, "vortices": count,
            "steps": args.steps, "ms_per_step": ms, "mlups": n * n / (ms * 1e-3) / 1e6,
            "high_order_fraction": nhi / (n * n),
            "kernels_ms_per_step": {k: kern[i] / max(ksteps, 1)
                                    for i, k in enumerate(slbm.KERNEL_NAMES)},
            "stream_collide_gbs": bytes_sc / (sc_ms * 1e-3) / 1e9}), flush=True)
        g.close()
        return
    if args.workload == "indicator":
        # the learned indicator on the headline's field (FP16 storage): its
        # GPU training, then steps with the indicator re-flagging every 10
        # steps against the same steps with the flags held fixed; the
        # difference is the evaluations' cost (features, network, conversions)
        n = args.size
        count = max(1, VCOUNT * n * n // (VN * VN))
        fields = WL.random_vortex_field(n, count, seed=VSEED, rmin=VRMIN, rmax=VRMAX, umax=VUMAX)
        t0 = time.time()
        weights, rep = train_indicator(slbm, WL, stream)
        train_s = time.time() - t0
        out = {}
        for mode in ("indicator", "fixed"):
            g = slbm.Solver(n, n, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=VTAU, interp_order=3,
                            precision=slbm.SLBM_FP16, stream=stream)
            g.init_equilibrium(*fields)
            g.set_indicator(weights, interval=10)
            g.set_criterion(slbm.SLBM_CRIT_MLP, 0.0)
            if mode == "fixed":
                g.set_criterion(slbm.SLBM_CRIT_NONE, 0.0)
            out[mode] = time_steps(g, stream, args.steps, args.warmup)
            if mode == "indicator":
                # one evaluation alone (features, network, new flags and their
                # conversions), back to back on the evolved state
                import torch
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 10
                torch.cuda.synchronize()
                a.record(stream)
                for _ in range(reps):
                    g.set_criterion(slbm.SLBM_CRIT_MLP, 0.0)
                b.record(stream)
                torch.cuda.synchronize()
                out["evaluation"] = a.elapsed_time(b) / reps
            g.close()
        print(json.dumps({
            "study": "learned indicator on the random-vortex field (FP16 storage)", "n": n,
            "steps": args.steps, "ms_per_step_with_indicator": out["indicator"],
            "ms_per_step_fixed_flags": out["fixed"],
            "ms_per_evaluation": out["evaluation"],
            "step_time_difference_per_evaluation_ms": (out["indicator"] - out["fixed"]) * 10,
            "training_wall_s": train_s, "training": rep}), flush=True)
        return
    if args.workload == "jet":
        # the free jet 1024 x 512 (FP32, Mach criterion every step): per-step
        # times with a 256 MiB L2 flush before each step
        J = WL.free_jet(NX, NY, slot=SLOT, ma_jet=MA_JET, ma_co=MA_CO)
        probe = slbm.Solver(8, 8, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=0.6)
        tau = jet_tau(probe.dt)
        probe.close()
        g = slbm.Solver(NX, NY, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=tau, interp_order=3,
                        periodic=(False, False), precision=slbm.SLBM_FP32, stream=stream)
        g.init_equilibrium(J["rho"], J["ux"], J["uy"])
        setup_jet(g, slbm, J)
        g.set_criterion(slbm.SLBM_CRIT_MACH, THR)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        for _ in range(args.warmup):
            flush.zero_()
            g.step(1)
        torch.cuda.synchronize()
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            g.step(1)
            e.record(stream)
            evs.append((s, e))
        torch.cuda.synchronize()
        ms = sum(s.elapsed_time(e) for s, e in evs) / args.steps
        g.profile(True)
        for _ in range(min(args.steps, 200)):
            flush.zero_()
            g.step(1)
        kern_ms, kern_steps = g.profile_read()
        g.profile(False)
        nhi = int(g.get_flags().sum())
        btb = time_steps(g, stream, args.steps, 10)
        print(json.dumps({
            "study": "free jet", "workload": JET, "tau": tau, "steps": args.steps,
            "ms_per_step_cold_l2": ms, "mlups_cold_l2": NX * NY / (ms * 1e-3) / 1e6,
            "ms_per_step_back_to_back": btb, "mlups_back_to_back": NX * NY / (btb * 1e-3) / 1e6,
            "high_order_fraction": nhi / (NX * NY),
            "kernels_ms_per_step": {n: float(kern_ms[i] / max(kern_steps, 1))
                                    for i, n in enumerate(slbm.KERNEL_NAMES)}}), flush=True)
        g.close()
        return
    if args.workload == "strip":
        for N in (128, 256, 512, 1024, 2048, 4096):
            steps = max(20, min(2000, int(4e8 / (N * N))))
            t, kms = {}, {}
            for name in ("q9", "q25", "hyb"):
                g = slbm.Solver(N, N, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=0.6, stream=stream)
                g.init_equilibrium(*WL.perturbed(N, N, seed=1, amp_rho=0.02, amp_u=0.05))
                fl = {"q9": np.zeros((N, N), np.uint8), "q25": np.ones((N, N), np.uint8),
                      "hyb": WL.strip_flags(N, 0.1)}[name]
                g.set_flags(fl)
                t[name] = time_steps(g, stream, steps, 10)
                kern, ksteps = profiled(g, min(steps, 100))
                kms[name] = {n: kern[i] / max(ksteps, 1) for i, n in enumerate(slbm.KERNEL_NAMES)}
                g.close()
            print(json.dumps({
                "study": "strip efficiency (Sec. IV.C)", "N": N, "steps": steps,
                "ms_per_step": t, "mlups": {k: N * N / (v * 1e-3) / 1e6 for k, v in t.items()},
                "kernels_ms_per_step": kms,
                "t_q25_over_t_q9": t["q25"] / t["q9"], "t_q25_over_t_hyb": t["q25"] / t["hyb"],
                "paper": {"t_q25_over_t_q9": 2.9, "t_q25_over_t_hyb_max": 2.43},
                "l2": "not flushed (back-to-back steps)"}), flush=True)
        return
    if args.workload == "shock":
        # batched shock structures (Sec. IV.C): 256 quasi-1-D instances in one
        # grid (every step advances all of them at once), upstream Mach 1.2-4.0,
        # two-population co-moving model, initial ramp 2 mean free paths wide;
        # the paper's scheme: D2Q16 refined to D2Q25 where Kn > 0.02
        # (refinement only, every --kn-interval steps), against D2Q25 everywhere
        b = WL.shock_batch(256, seed=2, mach_range=(1.2, 4.0))
        nx, ny = max(i["len"] for i in b), len(b)
        active = sum(i["len"] for i in b)
        lam1 = 50.0
        ends = np.array([[(i["left"][0], i["left"][1], 0.0, i["left"][2]),
                          (i["right"][0], i["right"][1], 0.0, i["right"][2])] for i in b])
        prof = [WL.shock_profile(i, nx, width=2 * lam1) for i in b]
        rho = np.stack([q[0] for q in prof]); ux = np.stack([q[1] for q in prof])
        T = np.stack([q[2] for q in prof])
        res = {}
        for name, kn in (("D2Q16 refined to D2Q25 where Kn > 0.02", True),
                         ("D2Q25 everywhere", False)):
            g = slbm.Solver(nx, ny, slbm.SLBM_D2Q16, slbm.SLBM_D2Q25, tau=0.7, stream=stream,
                            frame=slbm.SLBM_FRAME_POND)
            g.set_twopop(1.5, 0.8)
            g.init_equilibrium(rho, ux, np.zeros_like(rho), T)
            g.set_rows([i["len"] for i in b], ends)
            g.set_viscosity_law([i["mu1"] for i in b], [i["T1"] for i in b], 0.5, 2.0 / 3.0)
            if kn:
                g.set_kn_criterion(0.02, args.kn_interval)
            else:
                g.set_flags(np.ones((ny, nx), np.uint8))
            g.set_pond(1e-5, 30)          # FP32 predictor-corrector tolerance at T up to ~6
            shape = g.tune(3)
            # D2Q25 everywhere leaves the representable range above Mach ~2.5
            # after 59-149 steps: it is timed over the first 40
            steps = min(args.steps, 60 if kn else 40)
            nonconv = 0

            def settle():  # a predictor-corrector at its cap is reported, the state stays valid
                nonlocal nonconv
                try:
                    g.sync()
                except slbm.SlbmError as e:
                    if e.code != slbm.SLBM_ENOCONV:
                        raise
                    nonconv += 1

            g.step(args.warmup)
            settle()
            a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(g.stream)
            g.step(steps)
            b2.record(g.stream)
            torch.cuda.synchronize()
            settle()
            ms = a.elapsed_time(b2) / steps
            g.profile(True)
            g.step(min(steps, 10))
            settle()
            kern, ksteps = g.profile_read()
            g.profile(False)
            res[name] = ms
            line = {
                "study": "batched shock structure (Sec. IV.C)", "lattices": name,
                "workload": f"{ny} instances, lengths {min(i['len'] for i in b)}-{nx}, "
                            f"Mach 1.2-4.0, lambda_1 = 50 cells, two-population PonD "
                            f"(C_v = 3/2, Pr = 2/3, hard-sphere viscosity), FP32",
                "kn_interval": args.kn_interval if kn else None,
                "active_cells": active, "block_shape": shape, "steps": steps, "ms_per_step": ms,
                "mlups": active / (ms * 1e-3) / 1e6,
                "kernels_ms_per_step": {n: kern[i] / max(ksteps, 1)
                                        for i, n in enumerate(("co_moving_step", "conversion"))},
                "predictor_corrector_cap_reports": nonconv}
            if kn:  # the hybrid on to 300 steps in all: positivity and overshoot
                done = args.warmup + steps + min(steps, 10)
                lost_at = None
                while done < 300 and lost_at is None:
                    g.step(10)
                    done += 10
                    try:
                        g.sync()
                    except slbm.SlbmError as e:
                        if e.code == slbm.SLBM_ENOCONV:
                            nonconv += 1
                        elif e.code == slbm.SLBM_ENONFINITE:
                            lost_at = done  # a frame left the representable range
                        else:
                            raise
                r, _, _, tt = None, None, None, None
                for _ in range(3):  # pending reports come first
                    try:
                        r, _, _, tt = g.moments()
                        break
                    except slbm.SlbmError as e:
                        if e.code not in (slbm.SLBM_ENOCONV, slbm.SLBM_ENONFINITE):
                            raise
                fl_now = g.get_flags()
                ok_rows = [k for k, i in enumerate(b)
                           if np.isfinite(r[k, :i["len"]]).all() and (r[k, :i["len"]] > 0).all()
                           and (tt[k, :i["len"]] > 0).all()]
                lost = sorted(set(range(len(b))) - set(ok_rows))
                over = [float(r[k, :b[k]["len"]].max() / b[k]["right"][0] - 1) for k in ok_rows]
                hi = sum(int(fl_now[k, :i["len"]].sum()) for k, i in enumerate(b))
                line.update({
                    "predictor_corrector_cap_reports": nonconv,
                    "continued_to_step": done, "frame_left_range_at_step": lost_at,
                    "instances_lost": [{"mach": round(b[k]["mach"], 3), "len": b[k]["len"]}
                                       for k in lost],
                    "high_order_fraction": hi / active,
                    "max_density_overshoot_vs_rankine_hugoniot_kept_instances": max(over),
                    "median_density_overshoot": float(np.median(over))})
            print(json.dumps(line), flush=True)
            g.close()
        hyb = [k for k in res if k.startswith("D2Q16")][0]
        print(json.dumps({"study": "batched shock structure (Sec. IV.C)",
                          "t_all_d2q25_over_t_hybrid": res["D2Q25 everywhere"] / res[hyb]}),
              flush=True)
        return
    if args.workload == "couette":
        from paper_2102_12559_gb300 import indicator as IND
        batch = WL.couette_batch(count=128, seed=3)
        weights, ind_train = train_indicator(slbm, WL, stream)
        arms, states = {}, {}
        for mode in ("plain", "walls", "mlp", "all"):
            g, x0, widths = couette_solver(slbm, WL, batch, mode, weights, stream=stream)
            ny, nx = COUETTE_NY, g.nx
            g.step(args.warmup)
            torch.cuda.synchronize()
            st = g.stream
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            g.step(args.steps)
            b.record(st)
            torch.cuda.synchronize()
            sec = a.elapsed_time(b) * 1e-3
            kr, kst = profiled(g, min(args.steps, 200))
            cells = sum(ny * w for w in widths)
            m = g.moments()
            fl = g.get_flags()
            arms[mode] = {"ms_per_step": sec / args.steps * 1e3,
                          "mlups": cells * args.steps / sec / 1e6,
                          "kernels_ms_per_step": dict(zip(slbm.KERNEL_NAMES,
                                                          [k / max(kst, 1) for k in kr]))}
            extra = {}
            if mode == "all":  # the method's labels and the indicator's view of this state
                g.set_indicator(weights, interval=10)
                extra["ind"] = g.indicator_eval(features=False, flags=True)[2]
                extra["lab"] = IND.labels(g.lattice_loss()) > 0.5
            states[mode] = (m, fl, extra)
            g.close()
        inside = np.zeros((COUETTE_NY, nx), bool)
        wall = np.zeros((COUETTE_NY, nx), bool)
        kn_col = np.zeros(nx)
        for c, w in enumerate(widths):
            inside[:, x0[c]:x0[c] + w] = True
            wall[:, x0[c]:x0[c] + 4] = wall[:, x0[c] + w - 4:x0[c] + w] = True
            kn_col[x0[c]:x0[c] + w] = batch[c]["kn"]
        kn = np.broadcast_to(kn_col, (COUETTE_NY, nx))
        ref = states["all"][0]
        u_ref = np.stack(ref[1:3])[:, inside]
        plain_fl = plain_couette_flags(batch, x0, widths, (COUETTE_NY, nx))
        ind_fl = states["mlp"][1]
        lab, ind_all = states["all"][2]["lab"], states["all"][2]["ind"]
        u_all = np.stack(ref[1:3])
        for mode in ("plain", "walls", "mlp"):
            u = np.stack(states[mode][0][1:3])[:, inside]
            arms[mode]["rel_l2_u_vs_all_d2q25"] = float(np.linalg.norm(u - u_ref) /
                                                        np.linalg.norm(u_ref))
            arms[mode]["high_order_fraction"] = float((states[mode][1][inside] == 1).mean())
            ua = np.stack(states[mode][0][1:3])
            per = {}
            for lo, hi in ((0.01, 0.03), (0.03, 0.1), (0.1, 0.3), (0.3, 1.0)):
                sel = inside & (kn > lo) & (kn <= hi)
                per[f"Kn {lo}-{hi}"] = float(np.linalg.norm(ua[:, sel] - u_all[:, sel]) /
                                             np.linalg.norm(u_all[:, sel]))
            arms[mode]["rel_l2_u_by_knudsen_band"] = per
        d_ip, d_il, d_pl = decision_gaps(ind_fl, plain_fl, lab, inside)
        bands = {}
        for lo, hi in ((0.01, 0.03), (0.03, 0.1), (0.1, 0.3), (0.3, 1.0)):
            sel = inside & (kn > lo) & (kn <= hi)
            bands[f"Kn {lo}-{hi}"] = {
                "indicator_near_walls": float((ind_fl[sel & wall] == 1).mean()),
                "indicator_centre": float((ind_fl[sel & ~wall] == 1).mean()),
                "label_near_walls": float(lab[sel & wall].mean()),
                "label_centre": float(lab[sel & ~wall].mean())}
        print(json.dumps({
            "study": "batched Couette channels (Sec. IV.C) with the learned indicator",
            "workload": f"{len(batch)} channels H x {COUETTE_NY}, H {min(widths)}-{max(widths)}, "
                        "Kn 0.01-1 log-uniform, diffuse walls at -0.1 / +0.1, FP32, one "
                        f"{nx} x {COUETTE_NY} grid (channels along x, 2 G gap columns)",
            "cells": int(inside.sum()), "steps": args.steps,
            "timing": "CUDA events on the handle's stream",
            "arms": arms,
            "arm_forms": {"plain": f"D2Q25 in the channels with Kn > {KN_HI} (fixed)",
                          "walls": f"D2Q25 within {WALL_BAND} cells of every wall, D2Q9 "
                                   "inside (fixed, the paper's Sec. IV.C layout)",
                          "mlp": "learned indicator every 10 steps, refinement only "
                                 "(SLBM_CRIT_MLP_REFINE), from D2Q9 at rest",
                          "all": "D2Q25 everywhere (the accuracy reference)"},
            "indicator_decisions_at_end": {
                "indicator_vs_plain_rule": d_ip, "indicator_vs_lattice_loss_label": d_il,
                "plain_rule_vs_lattice_loss_label": d_pl,
                "indicator_on_all_d2q25_state_vs_label":
                    decision_gaps(ind_all, lab, plain_fl, inside)[0],
                "by_knudsen_band": bands},
            "indicator_training": ind_train,
            "finite": all(np.isfinite(v).all() for v in ref[:3])}), flush=True)
        return
    if args.workload == "pond":
        nx, ny = 1024, 512
        rho, ux, uy = WL.perturbed(nx, ny, seed=7, amp_rho=0.05, amp_u=0.2, U=(1.5 * np.sqrt(2.0), 0.0))
        T = WL.perturbed_T(nx, ny, seed=8, amp=0.05)
        disc = WL.random_flags(nx, ny, seed=3, blobs=4, rmin=24, rmax=48)
        for name, fl in (("D2Q9", np.zeros((ny, nx), np.uint8)), ("D2Q9+D2Q25 discs", disc),
                         ("D2Q25", np.ones((ny, nx), np.uint8))):
            g = slbm.Solver(nx, ny, slbm.SLBM_D2Q9, slbm.SLBM_D2Q25, tau=0.6, stream=stream,
                            frame=slbm.SLBM_FRAME_POND)
            g.init_equilibrium(rho, ux, uy, T)
            g.set_flags(fl)
            ms = time_steps(g, stream, args.steps, args.warmup)
            kern, ksteps = profiled(g, min(args.steps, 20))
            print(json.dumps({
                "study": "co-moving frame (PonD) step", "workload": f"thermal PonD {nx}x{ny} {name}",
                "mean_flow_mach": 1.5, "high_order_fraction": float(fl.mean()),
                "steps": args.steps, "ms_per_step": ms, "mlups": nx * ny / (ms * 1e-3) / 1e6,
                "kernels_ms_per_step": {n: kern[i] / max(ksteps, 1)
                                        for i, n in enumerate(slbm.KERNEL_NAMES[:2])}}),
                  flush=True)
            g.close()
        return


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="slbm", choices=["slbm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--size", type=int, default=VN, help="grid side of the vortex-fp32 study")
    ap.add_argument("--kn-interval", type=int, default=1,
                    help="steps between Knudsen criterion evaluations in the shock study")
    ap.add_argument("--e2e-steps", type=int, default=E2E_STEPS,
                    help="steps of the end-to-end measurement (default: the field's horizon)")
    ap.add_argument("--workload", default="vortex4096",
                    choices=["vortex4096", "vortex-fp32", "indicator", "jet", "strip", "pond", "shock",
                             "couette"],
                    help="vortex4096: the headline line; the others: secondary studies")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.workload != "vortex4096":
        run_study(args)
        return
    headline(args)


if __name__ == "__main__":
    main()
