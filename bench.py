#!/usr/bin/env python3
"""Benchmark: observed entries per second per PSGLD sweep on GB300.

A step is one sweep: B part-steps (Algorithm 1 iterations) that together
visit every observed entry once, plus the FP64 posterior accumulation.  The
default workload is the largest single-GPU configuration: sparse Gaussian
matrix factorisation, I = 480000, J = 18000, 10^8 observed entries with
Zipf(1.2) row degrees, K = 100, B = 64 (synthetic data, seeded), FP32, with
the BF16-gathered-factor arm beside it at the same posterior RMSE.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Our arm: value = N_obs * ranks / (max over ranks of the mean sweep time),
each sweep timed with CUDA events on the launching stream, with L2 flushed
(256 MB written) before every timed sweep.  The roofline's part-step time is
the timed sweep divided by B (it includes 1/B of the sweep's posterior
accumulation); the split between the gradient and the update kernel comes
from a separate, untimed pass with events around every launch.  Ranks (torchrun, one per GPU) run
independent replica chains: the sampler needs no collective.  Extra keys:
roofline of the part-step kernel, the oracle's CPU baseline, an end-to-end
job through the C ABI from pinned host buffers, SM clocks during the run.

Reference arm (--impl reference): the FP64 CPU oracle, as it stands, on the
host cores, on the same workload; each step is a bounded sample of
part-steps (for the 10^8-entry workload, of its first 4 x 4 blocks as a
B = 4 problem: the same blocks, so the same work per entry).  Under
torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "observed entries/s per PSGLD sweep"
UNIT = "entries/s"
L2_FLUSH_BYTES = 256 << 20
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1700.0

WORKLOADS = {
    "sparse_gauss_70000x10000_nnz10M_K50_B32": dict(
        I=70000, J=10000, nnz=10_000_000, K=50, B=32, p=0.0, phi=1.0, prior="gaussian",
        sigma=1.0, K_true=20, zipf_row=1.1, zipf_col=1.1, eps=2e-5, init_scale=0.3,
        job_sweeps=500),
    "sparse_gauss_480000x18000_nnz100M_K100_B64": dict(
        I=480000, J=18000, nnz=100_000_000, K=100, B=64, p=0.0, phi=1.0, prior="gaussian",
        sigma=1.0, K_true=20, zipf_row=1.2, zipf_col=None, eps=5e-6, init_scale=0.25,
        job_sweeps=200, bf16_compare=True),
    # the large sparse workload's recipe at 3 * 10^7 entries: W (192 MB)
    # still beyond L2, about 4 GB on the device -- the size of an ncu
    # capture of its kernels
    "sparse_gauss_480000x18000_nnz30M_K100_B64": dict(
        I=480000, J=18000, nnz=30_000_000, K=100, B=64, p=0.0, phi=1.0, prior="gaussian",
        sigma=1.0, K_true=20, zipf_row=1.2, zipf_col=None, eps=5e-6, init_scale=0.25,
        job_sweeps=200),
    "dense_poisson_256x256_K8_B4": dict(
        I=256, J=256, nnz=256 * 256, K=8, B=4, p=1.0, phi=1.0, prior="exponential",
        lam=1.0, K_true=8, eps=1e-4, init_scale=1.0, job_sweeps=1000, dense=True),
    # the standing chain's 2048 x 2048, K = 256 blocks at a size that an ncu
    # capture handles (B = 2: 64 items of the same size)
    "dense_poisson_4096x4096_K256_B2_bf16": dict(
        I=4096, J=4096, nnz=4096 * 4096, K=256, B=2, p=1.0, phi=1.0, prior="exponential",
        lam=1.0, K_true=16, eps=2e-5, init_scale=0.25, job_sweeps=200, dense=True,
        device_gen=True, dense_path=2, dense_v_bf16=1),
    # the standing chain's blocks (2048 x 2048, K = 256) in several waves of
    # items (12 blocks: 192 rows items, 144 columns items) at a size that an
    # ncu capture of the chain kernel handles (about 4 GB on the device)
    "dense_poisson_24576x24576_K256_B12_bf16": dict(
        I=24576, J=24576, nnz=24576 * 24576, K=256, B=12, p=1.0, phi=1.0, prior="exponential",
        lam=1.0, K_true=16, eps=2e-5, init_scale=0.25, job_sweeps=200, dense=True,
        device_gen=True, dense_path=2, dense_v_bf16=1),
    # the standing dense chain: tensor-core block chain, BF16 operands and V
    "dense_poisson_32768x32768_K256_B16_bf16": dict(
        I=32768, J=32768, nnz=32768 * 32768, K=256, B=16, p=1.0, phi=1.0, prior="exponential",
        lam=1.0, K_true=16, eps=2e-5, init_scale=0.25, job_sweeps=200, dense=True,
        device_gen=True, dense_path=2, dense_v_bf16=1),
}
# the serving configuration: Poisson arrivals of dense non-negative jobs
# (I in {257, 513, 1025}, J log-uniform on [500, 20000], p in {1, 1.5},
# K in {16, 64}, B = 8, 20 sweeps each) beside the standing chain, whose
# persistent kernel is held to 120 of the 152 SMs (the jobs' kernels find
# SMs free while it runs) and whose items each form their own mu: with E
# shared the standing chain runs 27 % faster in the mix but the jobs wait
# longer (library loop p50 / p99 94 / 128 ms against 74 / 107 ms)
WORKLOADS["serving_poisson200_mixed_jobs_with_standing_chain"] = dict(
    serving=True, rate=200.0, duration=3.0, sweeps=20, burn_in=10, B=8, eps=1e-4,
    budget_bytes=64 << 30, standing="dense_poisson_32768x32768_K256_B16_bf16", standing_sms=120,
    standing_share_e=0, I=0, J=0, K=0, p=1.0)
# many small dense chains sharing launches: 256 independent chains, each
# I = 513 x J ~ Uniform[200, 5000], V = |W* H*| * Gamma(2, rate 2) noise with
# K* = 16, model K = 32, Tweedie p = 1 and 2 alternating, B = 8
WORKLOADS["batched_dense_nmf_256chains_513xJ200-5000_K32_B8_bf16"] = dict(
    batched=True, chains=256, I=513, J_lo=200, J_hi=5000, K=32, K_true=16, B=8, p_mix=(1.0, 2.0),
    phi=1.0, prior="exponential", lam=1.0, eps=1e-4, init_scale=0.5, job_sweeps=40,
    dense_path=2, p=1.0)
# the same recipe with 64 chains on the single-pass kernel: the size of that
# kernel's full ncu capture (340 MB of V, a few seconds of replay)
WORKLOADS["batched_dense_nmf_64chains_513xJ200-5000_K32_B8_bf16"] = dict(
    WORKLOADS["batched_dense_nmf_256chains_513xJ200-5000_K32_B8_bf16"], chains=64, dense_path=1)
DEFAULT_WORKLOAD = "sparse_gauss_480000x18000_nnz100M_K100_B64"


# ---------------------------------------------------------------------------
# multi-rank plumbing (replicas; used only for the barrier and the max)
# ---------------------------------------------------------------------------

def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def reduce_max(x: float, world: int, device=None) -> float:
    """Max of a scalar over ranks (identity for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def aggregate(ms_per_step_local: float, units_per_step_local: float, world: int, device=None):
    """Whole-job throughput: units of all ranks / slowest rank's step time."""
    ms = reduce_max(ms_per_step_local, world, device)
    return ms, units_per_step_local * world / (ms / 1e3)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

CLOCK_FIELDS = ["timestamp", "clocks.sm", "clocks.max.sm", "power.draw",
                "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
                "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]


class ClockSampler:
    """nvidia-smi sampling every 100 ms in the background."""

    def __init__(self, gpu_id: str):
        self.samples = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", gpu_id, "--query-gpu=" + ",".join(CLOCK_FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, t0: float, t1: float):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        win = [s for (t, s) in self.samples if t0 <= t <= t1]
        where = "timed"
        if not win:   # the timed region was shorter than the sampling period
            win = [s for (t, s) in self.samples if t0 - 1.0 <= t <= t1 + 1.0]
            where = "timed +-1s"
        if not win:
            win = [s for (_, s) in self.samples]
            where = "run"

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(s[1]) for s in win if len(s) >= 8 and num(s[1]) is not None]
        mx = [num(s[2]) for s in win if len(s) >= 8 and num(s[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in win if len(s) >= 8
                          for k in range(4) if s[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(win), "window": where}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_inputs(wl: dict, seed: int, device):
    """Observed entries (i, j, v) -- or, for the tensor-core workloads, the
    dense V as one device tensor with i = j = None -- and initial factors."""
    import torch

    from paper_1506_01418_gb300 import datagen
    if wl.get("device_gen"):
        V = datagen.dense_poisson_device(wl["I"], wl["J"], wl["K_true"], seed, device)
        i = j = None
        v = V
    elif wl.get("dense"):
        V, _, _ = datagen.dense_poisson(wl["I"], wl["J"], wl["K_true"], seed)
        i, j, v = datagen.dense_to_coo(V)
        i, j, v = (torch.from_numpy(x).to(device) for x in (i, j, v))
    else:
        i, j, v = datagen.sparse_ratings(wl["I"], wl["J"], wl["nnz"], wl["K_true"], seed,
                                         zipf_row=wl["zipf_row"], zipf_col=wl["zipf_col"],
                                         device=device)
    nonneg = wl["prior"] == "exponential"
    W0, H0 = datagen.init_factors(wl["I"], wl["J"], wl["K"], seed, scale=wl["init_scale"],
                                  nonneg=nonneg)
    return i, j, v, W0, H0


def tensor_path(wl: dict) -> bool:
    return bool(wl.get("dense_path"))


def set_data(chain, wl, i, j, v):
    if tensor_path(wl):
        chain.set_data_dense(v)
    else:
        chain.set_data_coo(i, j, v)


def dense_part_sizes(wl: dict):
    """Entries of each part of a dense V (every entry observed)."""
    I, J, B = wl["I"], wl["J"], wl["B"]
    rows = [(r + 1) * I // B - r * I // B for r in range(B)]
    cols = [(c + 1) * J // B - c * J // B for c in range(B)]
    return [sum(rows[b] * cols[(b + s) % B] for b in range(B)) for s in range(B)]


def new_chain(wl: dict, seed: int, **opts):
    from paper_1506_01418_gb300 import psgld as P
    kind = P.PSGLD_PRIOR_EXPONENTIAL if wl["prior"] == "exponential" else P.PSGLD_PRIOR_GAUSSIAN
    if tensor_path(wl):
        opts = {"dense_path": wl["dense_path"], "dense_v_bf16": wl.get("dense_v_bf16", 0), **opts}
    return P.PSGLD(wl["I"], wl["J"], wl["K"], wl["B"], wl["p"], wl["phi"], prior_kind=kind,
                   lambda_w=wl.get("lam", 1.0), lambda_h=wl.get("lam", 1.0),
                   sigma_w=wl.get("sigma", 1.0), sigma_h=wl.get("sigma", 1.0), seed=seed,
                   eps=wl["eps"], **opts)


def part_step_bytes(wl: dict, part_sizes) -> float:
    """Algorithmic HBM bytes of one part-step, averaged over the B parts:
    each observed entry of the part once (int32 index + fp32 value, 8 n_Pi),
    one int32 row offset per row and block (4 (I + B)), every factor element
    read and written once in fp32 (8 (I + J) K), and the column-gradient
    scratch G_H zeroed and read once (8 J K)."""
    I, J, K, B = wl["I"], wl["J"], wl["K"], wl["B"]
    mean_n = sum(part_sizes) / len(part_sizes)
    return 8.0 * mean_n + 4.0 * (I + B) + 8.0 * (I + J) * K + 8.0 * J * K


def part_step_flops(wl: dict) -> float:
    """Algorithmic FLOPs of one dense part-step: three contractions of
    2 (IJ/B) K each (mu = W_b H_b, E H_b^T, E^T W_b over the part's blocks).
    The two-sided kernel computes mu twice; that is not counted."""
    return 6.0 * wl["I"] * wl["J"] / wl["B"] * wl["K"]


def read_peaks():
    """(HBM GB/s, BF16 TFLOP/s sustained, source)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, "fallback"


def kernel_traffic(workload: str):
    """DRAM bytes per launch of the roofline's kernel from the committed ncu
    summary, only if the kernel sources are unchanged since the counters were
    taken (the record holds the sha256 of each source it depends on)."""
    path = os.path.join(ROOT, "profiles", "part_step_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d.get(workload)
        if not e:
            return None
        for name, h in e["sources_sha256"].items():
            src = os.path.join(ROOT, "paper_1506_01418_gb300", "csrc", name)
            if hashlib.sha256(open(src, "rb").read()).hexdigest() != h:
                return None
        return float(e["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        return None


def host_cores() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except AttributeError:
        n = os.cpu_count() or 1
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env and env.isdigit() else n


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------

def oracle_setup(wl, i, j, v, W0, H0, seed):
    import numpy as np

    import oracle
    kind = oracle.PRIOR_EXPONENTIAL if wl["prior"] == "exponential" else oracle.PRIOR_GAUSSIAN
    m = oracle.Oracle(wl["I"], wl["J"], wl["K"], wl["B"], wl["p"], wl["phi"], prior_kind=kind,
                      lambda_w=wl.get("lam", 1.0), lambda_h=wl.get("lam", 1.0),
                      sigma_w=wl.get("sigma", 1.0), sigma_h=wl.get("sigma", 1.0))
    m.set_options(seed=seed, eps=wl["eps"])
    m.set_data(np.asarray(i), np.asarray(j), np.asarray(v, dtype=np.float64))
    m.set_factors(W0, H0)
    return m


def oracle_rate(m, wl, t0: int, n_steps: int):
    """Run n_steps oracle part-steps from iteration t0; entries covered / s."""
    ent = 0
    start = time.perf_counter()
    for t in range(t0, t0 + n_steps):
        m.part_step(t)
        ent += m.part_size(t)
    dt = time.perf_counter() - start
    return ent / dt, ent, dt


# above this many entries the oracle runs on a sample of the workload: its
# first SAMPLE_PIECES x SAMPLE_PIECES blocks as a B = SAMPLE_PIECES problem
# (the same blocks, with their entries and factor rows, so the same work per
# entry); loading all 10^8 entries into the oracle would take minutes
SAMPLE_ABOVE_NNZ = 20_000_000
SAMPLE_PIECES = 4


def oracle_sample(wl, i, j, v, W0, H0):
    """(workload, i, j, v, W0, H0, description) the oracle runs on: the whole
    workload, or for the largest ones its first SAMPLE_PIECES^2 blocks."""
    import numpy as np
    if len(v) <= SAMPLE_ABOVE_NNZ:
        return wl, i, j, v, W0, H0, "the workload"
    B, R = wl["B"], SAMPLE_PIECES
    I1, J1 = (R * wl["I"]) // B, (R * wl["J"]) // B
    keep = (np.asarray(i) < I1) & (np.asarray(j) < J1)
    sub = dict(wl, I=I1, J=J1, B=R, nnz=int(keep.sum()))
    what = (f"its first {R} x {R} blocks ({I1} x {J1}, {int(keep.sum())} entries) "
            f"as a B = {R} problem")
    return sub, np.asarray(i)[keep], np.asarray(j)[keep], np.asarray(v)[keep], W0[:I1], H0[:, :J1], what


def cpu_baseline(wl, i, j, v, W0, H0, seed, budget_s: float):
    """The oracle on the host cores (OpenMP over the blocks of a part), then
    single-threaded on a quarter of the budget; both give identical results."""
    import oracle
    wl, i, j, v, W0, H0, what = oracle_sample(wl, i, j, v, W0, H0)
    m = oracle_setup(wl, i, j, v, W0, H0, seed)
    cores = oracle.set_threads(0)
    _, _, dt1 = oracle_rate(m, wl, 1, 1)          # calibration (untimed)
    n = max(1, min(wl["B"] * 200, int(budget_s / max(dt1, 1e-6))))
    rate, ent, dt = oracle_rate(m, wl, 2, n)
    oracle.set_threads(1)
    _, _, dt1s = oracle_rate(m, wl, 2 + n, 1)
    n1 = max(1, min(wl["B"] * 50, int(budget_s / 4 / max(dt1s, 1e-6))))
    rate1, ent1, dts = oracle_rate(m, wl, 3 + n, n1)
    oracle.set_threads(cores)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} part-steps ({ent} observed entries, {dt:.1f} s) of {what}, "
                      f"same data, FP64, OpenMP over the blocks of each part",
            "single_thread": {"value": rate1, "unit": UNIT, "cores": 1,
                              "sample": f"{n1} part-steps ({ent1} entries, {dts:.1f} s)"}}


def cpu_baseline_block(wl, V, W0, H0, seed, budget_s: float):
    """For dense V too large for the oracle's host arrays: the oracle on one
    block of the workload (row piece 0 x column piece 0, its V, W and H rows)
    as a B = 1 problem -- a part-step of it is one block of a part-step of the
    workload -- timed for about budget_s, entries per second."""
    import numpy as np
    B = wl["B"]
    r1, c1 = wl["I"] // B, wl["J"] // B
    blk = dict(wl, I=r1, J=c1, B=1)
    Vb = V[:r1, :c1].float().cpu().numpy()
    ii, jj = np.meshgrid(np.arange(r1, dtype=np.int32), np.arange(c1, dtype=np.int32), indexing="ij")
    m = oracle_setup(blk, ii.ravel(), jj.ravel(), Vb.ravel().astype(np.float64),
                     W0[:r1].astype(np.float64), H0[:, :c1].astype(np.float64), seed)
    n, ent, secs, t = 0, 0, 0.0, 1
    while secs < budget_s and n < 100:
        _, e, dt = oracle_rate(m, blk, t, 1)
        ent += e
        secs += dt
        n += 1
        t += 1
    return {"value": ent / secs, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "sample": f"{n} part-steps of one {r1} x {c1} block of the workload (a B = 1 "
                      f"problem, {ent} entries, {secs:.1f} s), FP64, single block so one core "
                      f"does the work"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def run_ours(args, wl_name, wl):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1506_01418_gb300 import psgld as P

    seed = 1000 + rank
    i, j, v, W0, H0 = make_inputs(wl, seed, dev)
    torch.cuda.empty_cache()   # drop the generator's temporaries
    N = int(v.numel())
    chain = new_chain(wl, seed, use_graphs=1, profile=0)
    set_data(chain, wl, i, j, v)
    chain.set_factors(torch.from_numpy(W0).to(dev), torch.from_numpy(H0.T.copy()).to(dev))
    if wl.get("dense"):
        part_sizes = dense_part_sizes(wl)
    else:
        part_sizes = [P.psgld_part_layout(chain.ctx, s, wl["I"])[0][-1] for s in range(wl["B"])]
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = str(dev.index or 0)
    sampler = ClockSampler(uuid)

    for _ in range(args.warmup):
        chain.sweep(1)
    torch.cuda.synchronize(dev)
    barrier(world)
    torch.cuda.synchronize(dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    w0 = time.time()
    for s in range(args.steps):
        flush.zero_()
        starts[s].record(stream)
        chain.sweep(1)
        ends[s].record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    torch.cuda.synchronize(dev)
    w1 = time.time()
    # Kernel durations come from a separate pass with CUDA events around each
    # launch (event records inside the sweep graph cost about 12 us per
    # part-step, so they stay out of the timed sweeps above).
    chain.set_options(profile=1)
    g_ms, u_ms, k_n = 0.0, 0.0, 0
    for s in range(max(3, min(args.steps, 20))):
        flush.zero_()
        chain.sweep(1)
        g, u, n = chain.profile_read_split()
        if s > 0:   # the first profiled sweep captures a new graph
            g_ms += g
            u_ms += u
            k_n += n
    sweep_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    ms_local = sum(sweep_ms) / len(sweep_ms)
    ms, value = aggregate(ms_local, N, world, dev)
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(w0, w1)
    rmse = chain.rmse()

    hbm_peak, tc_peak, peak_src = read_peaks()
    grad_ms = g_ms / max(k_n, 1)
    upd_ms = u_ms / max(k_n, 1)
    kern_ms = grad_ms + upd_ms
    if tensor_path(wl):
        flops = part_step_flops(wl)
        achieved = flops / (grad_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": achieved / tc_peak, "traffic": kernel_traffic(wl_name),
                    "kernel": "two_sided::chain_kernel", "kernel_ms": grad_ms,
                    "algorithmic_flops_per_launch": flops,
                    "update_kernel_ms": upd_ms, "part_step_ms": kern_ms,
                    "peak_source": f"{peak_src} sustained cuBLAS BF16 GEMM (kernel timed "
                                   f"inside a long sweep)"}
    else:
        # the part-step's time from the timed sweeps themselves (sweep / B,
        # which also holds 1/B of the posterior accumulation), so that it
        # never exceeds the sweep it belongs to; the profiled pass only
        # gives the split between the two kernels
        bytes_launch = part_step_bytes(wl, part_sizes)
        part_ms = ms_local / wl["B"]
        achieved = bytes_launch / (part_ms / 1e3) / 1e9
        share = grad_ms / max(kern_ms, 1e-12)
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": kernel_traffic(wl_name),
                    "kernel": "part_step (gradient kernel + update kernel)", "kernel_ms": part_ms,
                    "kernel_ms_source": "timed sweeps / B",
                    "grad_share": share, "update_share": 1.0 - share,
                    "profiled_grad_kernel_ms": grad_ms, "profiled_update_kernel_ms": upd_ms,
                    "algorithmic_bytes_per_launch": bytes_launch,
                    "bytes_formula": "8 n_Pi + 4 (I + B) + 8 (I + J) K + 8 J K",
                    "peak_source": f"{peak_src} HBM copy bandwidth"}

    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16" if tensor_path(wl) else "f32", "data": "synthetic",
        "config": {"workload": wl_name, "I": wl["I"], "J": wl["J"], "nnz": N, "K": wl["K"],
                   "B": wl["B"], "tweedie_p": wl["p"], "phi": wl["phi"], "prior": wl["prior"],
                   "eps": wl["eps"], "step": "one sweep = B part-steps + FP64 posterior sums",
                   "path": ("tensor-core block chain, BF16 operands" +
                            (" and V" if wl.get("dense_v_bf16") else "") + ", FP32 accumulate"
                            if tensor_path(wl) else "FP32 gather path"),
                   "l2": "256 MB buffer written before every timed sweep",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        # per sweep: B x (gradient + update) + 2 accumulate + advance t + set t
        # per part-step: the chain kernel and the update (tensor-core path),
        # or each side's gradient and update on two streams (sparse path);
        # per sweep four more (posterior sums of W and H, the t counter)
        "gpu_launches": args.steps * ((2 if tensor_path(wl) else 4) * wl["B"] + 4),
        "clocks": clocks,
        "rmse_after": rmse,
    }

    if tensor_path(wl) and args.compare_sweeps > 0:
        chain.close()
        torch.cuda.empty_cache()
        result["precision_compare"] = compare_precision(wl, seed, dev, v, W0, H0, args.compare_sweeps)
    elif wl.get("bf16_compare") and args.compare_sweeps > 0:
        chain.close()
        torch.cuda.empty_cache()
        result["precision_compare"] = compare_sparse_precision(wl, seed, dev, i, j, v, W0, H0,
                                                               args.compare_sweeps)
    if not args.no_e2e:
        result["e2e"] = e2e_job(wl, seed, dev, i, j, v, W0, H0)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import numpy as np
        if i is None:
            result["cpu_baseline"] = cpu_baseline_block(wl, v, W0, H0, seed, args.cpu_budget)
        else:
            hi, hj, hv = (x.cpu().numpy() for x in (i, j, v))
            result["cpu_baseline"] = cpu_baseline(wl, hi, hj, hv.astype(np.float64),
                                                  W0.astype(np.float64), H0.astype(np.float64),
                                                  seed, args.cpu_budget)
    chain.close()
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def compare_precision(wl, seed, dev, V, W0, H0, sweeps: int):
    """BF16 tensor-core path vs the FP32 gather path on the same dense V,
    initial factors, Philox key and number of sweeps: observed entries/s per
    sweep (CUDA events around the sweeps) and the posterior-mean
    reconstruction RMSE over the second half of the sweeps, for both."""
    import torch
    out = {"sweeps": sweeps, "burn_in_sweeps": sweeps // 2}
    N = int(V.numel())
    for name, opts in (("bf16_tensor_core", {}), ("fp32_gather", {"dense_path": 0, "dense_v_bf16": 0})):
        ch = new_chain(wl, seed, use_graphs=1, burn_in_sweeps=sweeps // 2, **opts)
        ch.set_data_dense(V)
        ch.set_factors(torch.from_numpy(W0).to(dev), torch.from_numpy(H0.T.copy()).to(dev))
        stream = torch.cuda.current_stream(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        ch.sweep(sweeps)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        out[name] = {"value": N * sweeps / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms / sweeps,
                     "posterior_mean_rmse": ch.rmse(True)}
        ch.close()
        torch.cuda.empty_cache()
    r16 = out["bf16_tensor_core"]["posterior_mean_rmse"]
    r32 = out["fp32_gather"]["posterior_mean_rmse"]
    out["rmse_rel_diff"] = abs(r16 - r32) / r32
    out["speedup"] = out["bf16_tensor_core"]["value"] / out["fp32_gather"]["value"]
    return out


def compare_sparse_precision(wl, seed, dev, i, j, v, W0, H0, sweeps: int):
    """The FP32 sparse path vs BF16-gathered factors (gather_bf16) on the same
    entries, initial factors, Philox key and number of sweeps: observed
    entries/s per sweep and the posterior-mean reconstruction RMSE over the
    second half of the sweeps."""
    import torch
    out = {"sweeps": sweeps, "burn_in_sweeps": sweeps // 2}
    N = int(v.numel())
    for name, opts in (("fp32_gather", {}), ("bf16_gather", {"gather_bf16": 1})):
        ch = new_chain(wl, seed, use_graphs=1, burn_in_sweeps=sweeps // 2, **opts)
        ch.set_data_coo(i, j, v)
        ch.set_factors(torch.from_numpy(W0).to(dev), torch.from_numpy(H0.T.copy()).to(dev))
        stream = torch.cuda.current_stream(dev)
        ch.sweep(1)                      # graph capture outside the timed region
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        ch.sweep(sweeps)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        out[name] = {"value": N * sweeps / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms / sweeps,
                     "posterior_mean_rmse": ch.rmse(True)}
        ch.close()
        torch.cuda.empty_cache()
    r16 = out["bf16_gather"]["posterior_mean_rmse"]
    r32 = out["fp32_gather"]["posterior_mean_rmse"]
    out["rmse_rel_diff"] = abs(r16 - r32) / r32
    out["speedup"] = out["bf16_gather"]["value"] / out["fp32_gather"]["value"]
    out["note"] = ("each chain runs one untimed sweep (its graph capture) before the timed ones; "
                   "posterior means over the sweeps after burn_in_sweeps")
    return out


def e2e_job(wl, seed, dev, i, j, v, W0, H0):
    """One sampling job through the C ABI from pinned host buffers: entries
    and initial factors in, job_sweeps sweeps, posterior means and variances
    and the log-likelihood out.  value = entries x sweeps / wall time."""
    import numpy as np
    import torch
    dense_in = i is None
    if dense_in:
        hv = v.cpu().pin_memory()
    else:
        hi = i.cpu().pin_memory()
        hj = j.cpu().pin_memory()
        hv = v.cpu().pin_memory()
    hW = torch.from_numpy(W0).pin_memory()
    hHt = torch.from_numpy(H0.T.copy()).pin_memory()
    S = wl["job_sweeps"]
    I, J, K = wl["I"], wl["J"], wl["K"]
    Wm = np.zeros((I, K)); Wv = np.zeros((I, K)); Hm = np.zeros((J, K)); Hv = np.zeros((J, K))
    chain = new_chain(wl, seed, use_graphs=1, burn_in_sweeps=S // 2)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    if dense_in:
        chain.set_data_dense(hv)
    else:
        chain.set_data_coo(hi, hj, hv)
    chain.set_factors(hW, hHt)
    chain.sweep(S)
    from paper_1506_01418_gb300 import psgld as P
    P.psgld_posterior_mean(chain.ctx, Wm, Wv, Hm, Hv)
    # the log-likelihood over a dense V is an FP64 product W H over every
    # entry (0.57 s at 32768^2 on this GPU's FP64 rate): the dense jobs read
    # back their posterior means only
    ll = chain.log_lik() if not dense_in else None
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    chain.close()
    N = int(v.numel())
    h2d = (4 if dense_in else 12) * N + 4 * (I + J) * K
    d2h = 8 * 4 * (I + J) * K + (0 if dense_in else 8)
    return {"value": N * S / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / S,
            "d2h_bytes_per_step": d2h / S, "job_sweeps": S, "job_s": dt,
            "log_lik": ll,
            "api": ("psgld_set_data_dense" if dense_in else "psgld_set_data_coo") +
                   "/set_factors (pinned host) + psgld_sweep + psgld_posterior_mean" +
                   ("" if dense_in else " + psgld_log_lik")}


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------

def batched_specs(wl: dict, seed: int):
    """Per chain of the batched workload: (J, tweedie p, data seed, init seed)."""
    import numpy as np
    rng = np.random.Generator(np.random.Philox(seed))
    Js = rng.integers(wl["J_lo"], wl["J_hi"] + 1, size=wl["chains"])
    ps = wl["p_mix"]
    return [(int(Js[c]), float(ps[c % len(ps)]), seed + 17 * c, seed + 17 * c + 1)
            for c in range(wl["chains"])]


def batched_chain_wl(wl: dict, J: int, p: float) -> dict:
    return dict(wl, J=J, p=p, nnz=wl["I"] * J, batched=False)


def batched_make(wl, specs, dev, host=False, **opts):
    """The chains of the batched workload with their data and initial factors
    (device tensors, or pinned host tensors when host=True: the copies then run
    inside set_data_dense / set_factors)."""
    import torch

    from paper_1506_01418_gb300 import datagen
    chains = []
    for (J, p, ds, iseed) in specs:
        cwl = batched_chain_wl(wl, J, p)
        V = datagen.dense_gamma_device(wl["I"], J, wl["K_true"], ds, dev)
        W0, H0 = datagen.init_factors(wl["I"], J, wl["K"], iseed, scale=wl["init_scale"], nonneg=True)
        W0, Ht0 = torch.from_numpy(W0), torch.from_numpy(H0.T.copy())
        ch = new_chain(cwl, iseed, use_graphs=1, **opts)
        if host:
            V = V.cpu().pin_memory()
            W0, Ht0 = W0.pin_memory(), Ht0.pin_memory()
        else:
            W0, Ht0 = W0.to(dev), Ht0.to(dev)
        chains.append((ch, V, W0, Ht0))
    return chains


def batched_bytes_flops(wl, specs):
    """Algorithmic HBM bytes and FLOPs of one batched gradient launch (one
    part of every chain), averaged over the parts: V of the part once (FP32),
    the part's W rows and H columns read and its G rows written once (FP32);
    three contractions of 2 (I J / B) K each."""
    I, K, B = wl["I"], wl["K"], wl["B"]
    ent = sum(I * J for J, _, _, _ in specs) / B
    fac = sum(8.0 * K * (I + J) for J, _, _, _ in specs)
    return 4.0 * ent + fac, 6.0 * ent * K


def run_batched(args, wl_name, wl):
    """Many small dense chains whose part-steps share launches
    (psgld_batch_sweep); a step is one sweep of every chain."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1506_01418_gb300 import psgld as P

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    seed = 1000
    specs = batched_specs(wl, seed)
    made = batched_make(wl, specs, dev, profile=1)
    chains = [m[0] for m in made]
    for ch, V, W0, Ht0 in made:
        ch.set_data_dense(V)
        ch.set_factors(W0, Ht0)
    del made
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    N = sum(wl["I"] * J for J, _, _, _ in specs)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = "0"
    sampler = ClockSampler(uuid)
    chains[0].set_options(profile=0)
    for _ in range(args.warmup):
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    # the result-neutral launch knobs, tuned on ordinary sweeps of the chains
    from paper_1506_01418_gb300 import autotune
    tuning = autotune.tune_batch(chains)
    # the same sweeps without captured graphs (direct launches), for the record
    chains[0].set_options(use_graphs=0)
    a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(3):
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)
    b0.record(stream)
    torch.cuda.synchronize(dev)
    ms_direct = a0.elapsed_time(b0) / 3
    chains[0].set_options(use_graphs=1)
    for _ in range(2):
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)     # the graphs captured again
    torch.cuda.synchronize(dev)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    w0 = time.time()
    for s in range(args.steps):
        flush.zero_()
        starts[s].record(stream)
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)
        ends[s].record(stream)
    torch.cuda.synchronize(dev)
    w1 = time.time()
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / args.steps
    # kernel durations: events around each part's launches, separate pass
    chains[0].set_options(profile=1)
    g_ms = u_ms = 0.0
    k_n = 0
    for s in range(max(3, min(args.steps, 10))):
        flush.zero_()
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)
        g, u, n = chains[0].profile_read_split()
        g_ms += g
        u_ms += u
        k_n += n
    chains[0].set_options(profile=0)
    # the same chains swept one by one (each its own captured-graph sweep)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n_alone = 3
    a.record(stream)
    for _ in range(n_alone):
        for ch in chains:
            ch.sweep(1, stream.cuda_stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms_alone = a.elapsed_time(b) / n_alone
    time.sleep(0.25)
    sampler.stop()
    clocks = sampler.summary(w0, w1)
    for ch in chains:
        ch.close()
    torch.cuda.empty_cache()
    other = batched_other_kernel(wl, specs, dev, stream, flush, args.steps)

    hbm_peak, tc_peak, peak_src = read_peaks()
    grad_ms = g_ms / max(k_n, 1)
    upd_ms = u_ms / max(k_n, 1)
    bytes_launch, flops_launch = batched_bytes_flops(wl, specs)
    two = wl.get("dense_path", 1) == 2
    achieved = bytes_launch / (grad_ms / 1e3) / 1e9
    tflops = flops_launch / (grad_ms / 1e3) / 1e12
    result = {
        "metric": METRIC, "value": N / (ms / 1e3), "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": wl_name, "chains": wl["chains"], "I": wl["I"],
                   "J": f"Uniform[{wl['J_lo']}, {wl['J_hi']}] per chain", "entries": N,
                   "K": wl["K"], "K_true": wl["K_true"], "B": wl["B"], "tweedie_p": list(wl["p_mix"]),
                   "prior": wl["prior"], "eps": wl["eps"],
                   "step": "one sweep of every chain: per part one tensor-core gradient launch "
                           "per kernel variant (" + ("one persistent launch per Tweedie power"
                           if two else "one per K class") + ") and one update launch over all "
                           "chains, then the FP64 posterior sums",
                   "path": "psgld_batch_sweep, " + ("two-sided" if two else "single-pass") +
                           " tensor-core block chain, BF16 operands, FP32 accumulate, FP32 V",
                   "l2": "V of all chains (1.4 GB) exceeds L2; 256 MB buffer also written before "
                         "every timed sweep"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": kernel_traffic(wl_name),
                     "kernel": ("two_sided::chain_batch_kernel (per part: one launch per power)"
                                if two else "dense_grad_batch_kernel"), "kernel_ms": grad_ms,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "algorithmic_flops_per_launch": flops_launch, "tensor_tflops": tflops,
                     "tensor_frac_of_sustained": tflops / tc_peak,
                     "update_kernel_ms": upd_ms, "part_step_ms": grad_ms + upd_ms,
                     "peak_source": f"{peak_src} HBM copy bandwidth"},
        # per call (one sweep): set t, then one replayed graph of B x
        # (gradient launches + update), accumulate, advance t; the two-sided
        # kernel runs one launch per power, the single-pass one per K class
        "gpu_launches": args.steps * ((len(set(wl["p_mix"])) if two else 1) * wl["B"] + wl["B"] + 3),
        "clocks": clocks,
        "autotune": tuning,
        "graphs": {"ms_per_sweep_captured": ms, "ms_per_sweep_direct_launches": ms_direct,
                   "how": "each batched sweep one replayed CUDA graph (timed region) vs the "
                          "same sweeps launched directly (3 sweeps, L2 not flushed)"},
        "unbatched": {"value": N / (ms_alone / 1e3), "unit": UNIT, "ms_per_sweep": ms_alone,
                      "how": "the same chains, each swept alone (its own captured-graph sweep), "
                             "back to back on one stream"},
        "other_kernel": other,
    }
    if args.compare_sweeps > 0:
        result["precision_compare"] = batched_precision(wl, specs[:16], dev, args.compare_sweeps)
    if not args.no_e2e:
        result["e2e"] = batched_e2e(wl, specs, dev)
    if not args.no_cpu_baseline:
        result["cpu_baseline"] = batched_cpu_baseline(wl, specs[0], args.cpu_budget)
    print(json.dumps(result), flush=True)


def batched_other_kernel(wl, specs, dev, stream, flush, steps: int):
    """The same chains and batched sweeps on the other tensor-core kernel
    (two-sided if the workload runs single-pass, and the reverse): entries/s
    of the timed sweeps."""
    import torch

    from paper_1506_01418_gb300 import psgld as P
    dp = 2 if wl.get("dense_path", 1) != 2 else 3
    # the single-pass kernel reads V in FP32
    made = batched_make(wl, specs, dev, dense_path=dp, dense_v_bf16=wl.get("dense_v_bf16", 0) if dp == 2 else 0)
    chains = [m[0] for m in made]
    for ch, V, W0, Ht0 in made:
        ch.set_data_dense(V)
        ch.set_factors(W0, Ht0)
    del made
    torch.cuda.synchronize(dev)
    for _ in range(3):
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)
    torch.cuda.synchronize(dev)
    n = max(3, min(steps, 10))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    for s in range(n):
        flush.zero_()
        starts[s].record(stream)
        P.psgld_batch_sweep(chains, 1, stream.cuda_stream)
        ends[s].record(stream)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / n
    for ch in chains:
        ch.close()
    torch.cuda.empty_cache()
    N = sum(wl["I"] * J for J, _, _, _ in specs)
    return {"kernel": "two_sided (one persistent launch per part and power)" if dp == 2 else "single_pass",
            "value": N / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms, "sweeps": n}


def batched_precision(wl, specs, dev, sweeps: int):
    """BF16 tensor-core batched sweeps (as configured; the two-sided kernel
    with V kept in BF16; the single-pass kernel with GEMM1 in E4M3 with
    per-tile scales) vs the FP32 gather path (each chain alone) on the same
    chains, data, initial factors and Philox keys: entries/s and the
    posterior-mean reconstruction RMSE (mean over the chains)."""
    import torch

    from paper_1506_01418_gb300 import psgld as P
    out = {"chains": len(specs), "sweeps": sweeps, "burn_in_sweeps": sweeps // 2}
    N = sum(wl["I"] * J for J, _, _, _ in specs)
    stream = torch.cuda.current_stream(dev)
    for name, opts in (("bf16_tensor_core_batched", {}),
                       ("bf16_tensor_core_bf16_v_batched", {"dense_path": 2, "dense_v_bf16": 1}),
                       ("e4m3_gemm1_batched", {"dense_fp8": 1, "dense_path": 3}),
                       ("fp32_gather", {"dense_path": 0})):
        made = batched_make(wl, specs, dev, burn_in_sweeps=sweeps // 2, **opts)
        for ch, V, W0, Ht0 in made:
            ch.set_data_dense(V)
            ch.set_factors(W0, Ht0)
        chains = [m[0] for m in made]
        del made
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        a.record(stream)
        if name == "fp32_gather":
            for ch in chains:
                ch.sweep(sweeps, stream.cuda_stream)
        else:
            P.psgld_batch_sweep(chains, sweeps, stream.cuda_stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ms = a.elapsed_time(b)
        r = [ch.rmse(True) for ch in chains]
        out[name] = {"value": N * sweeps / (ms / 1e3), "unit": UNIT, "ms_per_sweep": ms / sweeps,
                     "posterior_mean_rmse_mean": sum(r) / len(r), "rmse": r}
        for ch in chains:
            ch.close()
        torch.cuda.empty_cache()
    r16 = out["bf16_tensor_core_batched"].pop("rmse")
    r16v = out["bf16_tensor_core_bf16_v_batched"].pop("rmse")
    r8 = out["e4m3_gemm1_batched"].pop("rmse")
    r32 = out["fp32_gather"].pop("rmse")
    out["rmse_rel_diff_max"] = max(abs(x - y) / y for x, y in zip(r16, r32))
    out["e4m3_rmse_rel_diff_max"] = max(abs(x - y) / y for x, y in zip(r8, r32))
    out["bf16_v_rmse_rel_diff_max"] = max(abs(x - y) / y for x, y in zip(r16v, r32))
    out["speedup"] = out["bf16_tensor_core_batched"]["value"] / out["fp32_gather"]["value"]
    return out


def batched_e2e(wl, specs, dev):
    """The whole batch as one job through the C ABI from pinned host buffers:
    every chain's V and initial factors in, job_sweeps batched sweeps,
    every chain's posterior means and variances out."""
    import numpy as np
    import torch

    from paper_1506_01418_gb300 import psgld as P
    S = wl["job_sweeps"]
    # many contexts set up back to back: their memory comes from PyTorch's
    # caching allocator (psgld_set_allocator), so that freeing a context's
    # staging buffer does not wait for the whole device
    P.use_torch_allocator(dev.index if dev.index is not None else 0)
    try:
        made = batched_make(wl, specs, dev, host=True, burn_in_sweeps=S // 2)
        chains = [m[0] for m in made]
        I, K = wl["I"], wl["K"]
        outs = [tuple(np.zeros((n, K)) for n in (I, I, J, J)) for J, _, _, _ in specs]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for ch, V, W0, Ht0 in made:
            ch.set_data_dense(V)
            ch.set_factors(W0, Ht0)
        P.psgld_batch_sweep(chains, S)
        for ch, o in zip(chains, outs):
            P.psgld_posterior_mean(ch.ctx, *o)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        for ch in chains:
            ch.close()
    finally:
        P.psgld_set_allocator(None)
    N = sum(I * J for J, _, _, _ in specs)
    h2d = 4 * N + sum(4 * (I + J) * K for J, _, _, _ in specs)
    d2h = sum(8 * 4 * (I + J) * K for J, _, _, _ in specs)
    return {"value": N * S / dt, "unit": UNIT, "h2d_bytes_per_step": h2d / S,
            "d2h_bytes_per_step": d2h / S, "job_sweeps": S, "job_s": dt,
            "api": "psgld_set_allocator (PyTorch's caching allocator) + psgld_set_data_dense/"
                   "set_factors (pinned host) per chain + psgld_batch_sweep + psgld_posterior_mean "
                   "per chain"}


def batched_cpu_baseline(wl, spec, budget_s: float):
    """The oracle on the first chain of the batch (OpenMP over a part's blocks)."""
    import numpy as np

    import oracle
    from paper_1506_01418_gb300 import datagen
    J, p, ds, iseed = spec
    cwl = batched_chain_wl(wl, J, p)
    V, _, _ = datagen.dense_gamma(wl["I"], J, wl["K_true"], ds)
    i, j, v = datagen.dense_to_coo(V)
    W0, H0 = datagen.init_factors(wl["I"], J, wl["K"], iseed, scale=wl["init_scale"], nonneg=True)
    out = cpu_baseline(cwl, i, j, v.astype(np.float64), W0.astype(np.float64),
                       H0.astype(np.float64), iseed, budget_s)
    out["sample"] = f"chain 0 of the batch ({wl['I']} x {J}, p = {p}): " + out["sample"]
    return out


def serve_trace(wl, executor, dev, uuid):
    """Replay the workload's Poisson trace through the server on `executor`
    (after a warm-up trace of one job per size class); returns the trace's
    measurements."""
    import numpy as np
    import torch

    from paper_1506_01418_gb300 import serving
    factory = serving.mixed_job_factory(wl["sweeps"], wl["burn_in"], wl["B"], wl["eps"])
    warm = []
    for k, (I, K, p) in enumerate([(I, K, p) for I in (257, 513, 1025) for K in (16, 64) for p in (1.0, 1.5)]):
        j = factory(10_000 + k, 0.0, np.random.Generator(np.random.Philox(k)))
        j.I, j.K, j.p, j.J = I, K, p, 800
        warm.append(j)
    wsrv = serving.Server(executor, wl["budget_bytes"])
    try:
        wsrv.run(warm, idle_sleep=0)
    finally:
        wsrv.close()
    jobs = serving.poisson_trace(wl["rate"], wl["duration"], seed=2024, job_factory=factory)
    srv = serving.Server(executor, wl["budget_bytes"])
    standing = None
    if wl.get("standing"):
        sw = WORKLOADS[wl["standing"]]
        standing = serving.Job(job_id=-1, I=sw["I"], J=sw["J"], K=sw["K"], B=sw["B"], p=sw["p"],
                               sweeps=None, burn_in=0, seed=7, eps=sw["eps"], init_scale=sw["init_scale"],
                               dense_path=sw["dense_path"], dense_v_bf16=sw["dense_v_bf16"],
                               max_sms=wl.get("standing_sms", 0),
                               dense_share_e=wl.get("standing_share_e", -1))
        srv.submit(standing)
        srv.poll(0.0)
        torch.cuda.synchronize(dev)
    sampler = ClockSampler(uuid)
    ticks0 = getattr(executor, "ticks", 0)
    w0 = time.time()
    st0 = srv.active[-1][1]["sweeps_queued"] if standing is not None else 0
    try:
        wall = srv.run(jobs, idle_sleep=0)
        st_sweeps = (srv.active[-1][1]["sweeps_queued"] - st0) if standing is not None else 0
        w1 = time.time()
        srv.stop_standing()
    finally:
        srv.close()
    torch.cuda.synchronize(dev)
    time.sleep(0.25)
    sampler.stop()
    job_entries = sum(j.I * j.J * j.sweeps for j in jobs)
    st_entries = (standing.I * standing.J * st_sweeps) if standing is not None else 0
    return {"jobs": jobs, "wall": wall, "job_entries": job_entries, "st_entries": st_entries,
            "st_sweeps": st_sweeps, "standing": standing, "peak_used": srv.peak_used,
            "clocks": sampler.summary(w0, w1), "warm": len(warm),
            "ticks": getattr(executor, "ticks", 0) - ticks0}


def serve_trace_native(wl, dev, uuid):
    """The same trace through the library's native serving loop
    (psgld_server_*): the Python thread only replays arrivals (generating
    each job's data on the GPU and submitting it) and keeps the standing
    chain's sweep queued; admission, batching and read-back run in the
    library's worker thread.  Latency = arrival to read-back."""
    import numpy as np
    import torch

    from paper_1506_01418_gb300 import psgld as P
    from paper_1506_01418_gb300 import serving
    factory = serving.mixed_job_factory(wl["sweeps"], wl["burn_in"], wl["B"], wl["eps"])
    ex = serving.GpuExecutor(dev.index)          # data generation and the standing chain
    srv = P.NativeServer(wl["budget_bytes"])

    def submit(job):
        V, W0, Ht0 = ex._data(job)
        torch.cuda.current_stream(dev).synchronize()     # the job's inputs, not the device
        return srv.submit(job.I, job.J, job.K, job.B, job.p, job.phi, V, W0, Ht0, job.sweeps,
                          lambda_w=job.lam, lambda_h=job.lam, seed=job.seed, eps=job.eps,
                          burn_in_sweeps=job.burn_in, dense_path=job.dense_path)

    # warm-up: one job of each size class
    for k, (I, K, p) in enumerate([(I, K, p) for I in (257, 513, 1025) for K in (16, 64) for p in (1.0, 1.5)]):
        j = factory(10_000 + k, 0.0, np.random.Generator(np.random.Philox(k)))
        j.I, j.K, j.p, j.J = I, K, p, 800
        submit(j)
    srv.wait_idle(600.0)
    srv.poll()
    jobs = serving.poisson_trace(wl["rate"], wl["duration"], seed=2024, job_factory=factory)
    standing, hst, st0 = None, None, 0
    if wl.get("standing"):
        sw = WORKLOADS[wl["standing"]]
        standing = serving.Job(job_id=-1, I=sw["I"], J=sw["J"], K=sw["K"], B=sw["B"], p=sw["p"],
                               sweeps=None, burn_in=0, seed=7, eps=sw["eps"], init_scale=sw["init_scale"],
                               dense_path=sw["dense_path"], dense_v_bf16=sw["dense_v_bf16"],
                               max_sms=wl.get("standing_sms", 0),
                               dense_share_e=wl.get("standing_share_e", -1))
        hst = ex.start(standing)
        torch.cuda.synchronize(dev)
        st0 = hst["sweeps_queued"]
    sampler = ClockSampler(uuid)
    pending = list(jobs)
    by_id = {}
    n_done = 0
    w0 = time.time()
    t0 = time.perf_counter()
    while n_done < len(jobs):
        now = time.perf_counter() - t0
        while pending and pending[0].arrival <= now:
            job = pending.pop(0)
            job.admitted = time.perf_counter() - t0           # submitted
            by_id[submit(job)] = job
        if hst is not None:
            ex.step_standing(standing, hst)
        for jid, lat in srv.poll():
            job = by_id.pop(jid)
            job.finished = job.admitted + lat
            n_done += 1
        if now > 600.0:
            raise TimeoutError("native serving trace did not finish")
        time.sleep(0)
    wall = time.perf_counter() - t0
    st_sweeps = (hst["sweeps_queued"] - st0) if hst is not None else 0
    w1 = time.time()
    if hst is not None:
        ex.finish(standing, hst)
    stats = srv.stats()
    srv.close()
    torch.cuda.synchronize(dev)
    time.sleep(0.25)
    sampler.stop()
    job_entries = sum(j.I * j.J * j.sweeps for j in jobs)
    st_entries = standing.I * standing.J * st_sweeps if standing is not None else 0
    return {"jobs": jobs, "wall": wall, "job_entries": job_entries, "st_entries": st_entries,
            "st_sweeps": st_sweeps, "stats": stats, "clocks": sampler.summary(w0, w1)}


def run_serving(args, wl_name, wl):
    """The serving loop on one GPU: a Poisson trace of jobs replayed in real
    time through the library's native serving loop (psgld_server_*:
    memory-budget admission and continuous batching, every admitted job's
    part-steps in the batch's shared launches, on the library's worker
    threads); value = observed entries x sweeps of every job and of the
    standing chain / wall time of the trace; latency = arrival to read-back.
    The same trace with the Python batching executor and with one stream and
    context per job (no shared launches) is reported beside it."""
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_1506_01418_gb300 import serving
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = "0"
    r = serve_trace_native(wl, dev, uuid)
    jobs, wall = r["jobs"], r["wall"]
    value = (r["job_entries"] + r["st_entries"]) / wall
    lat = serving.latency_summary(jobs)
    h2d = sum(4 * (j.I + j.J) * j.K for j in jobs)
    d2h = sum(8 * (j.I + j.J) * j.K * 2 for j in jobs)
    st = r["stats"]
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(jobs),
        "warmup": 12, "ms_per_step": wall * 1e3 / max(1, len(jobs)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": wl_name, "arrival_rate_per_s": wl["rate"], "trace_s": wl["duration"],
                   "jobs": len(jobs), "sweeps_per_job": wl["sweeps"], "B": wl["B"],
                   "hbm_budget_bytes": wl["budget_bytes"], "standing_chain": wl.get("standing"),
                   "standing_chain_sms": wl.get("standing_sms", 0) or "all",
                   "step": "one job of the trace (value counts every job's and the standing "
                           "chain's entries x sweeps over the trace's wall time)",
                   "path": "the library's serving loop (psgld_server_*): admission by the "
                           "jobs' estimated device memory, continuous batching with every admitted "
                           "job's part-steps in shared tensor-core launches (psgld_batch_sweep, one "
                           "sweep per call, one queued at a time), set-up and read-back on a second "
                           "thread, stream-ordered memory pool; the standing chain on its own "
                           "stream, its persistent kernel on 120 SMs"},
        "latency": lat,
        "job_entries_per_s": r["job_entries"] / wall,
        "standing_chain": ({"sweeps": r["st_sweeps"], "entries_per_s": r["st_entries"] / wall}
                           if r["st_sweeps"] else None),
        "batch": {"sweeps": st["sweeps"], "jobs_per_sweep_mean": st["jobs_per_sweep"]},
        "peak_budget_used_bytes": st["peak_bytes"],
        "roofline": None,
        # per batch sweep: set t, B x (gradient launches per kernel variant
        # (about two) + update), accumulate, advance t; standing chain: 2B + 3
        # per sweep
        "gpu_launches": st["sweeps"] * (3 * wl["B"] + 3) + r["st_sweeps"] * (2 * 16 + 3),
        "clocks": r["clocks"],
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": h2d / max(1, len(jobs)),
                "d2h_bytes_per_step": d2h / max(1, len(jobs)),
                "note": "the serving loop is the end-to-end path: each job's initial factors go "
                        "host to device and its posterior means device to host inside the trace"},
    }
    torch.cuda.empty_cache()
    if not args.no_serving_compare:
        for name, mk, how in (
                ("python_batching", lambda: serving.BatchedGpuExecutor(0),
                 "the same trace through serving.Server with BatchedGpuExecutor: the same shared "
                 "launches driven from a Python loop (set-up and teardown on worker threads)"),
                ("per_job_streams", lambda: serving.GpuExecutor(0),
                 "the same trace, one stream and context per job with all its sweeps enqueued "
                 "at admission (no shared launches)")):
            ex = mk()
            r2 = serve_trace(wl, ex, dev, uuid)
            if hasattr(ex, "shutdown"):
                ex.shutdown()
            del ex
            torch.cuda.empty_cache()
            result[name] = {
                "value": (r2["job_entries"] + r2["st_entries"]) / r2["wall"], "unit": UNIT,
                "job_entries_per_s": r2["job_entries"] / r2["wall"],
                "standing_entries_per_s": r2["st_entries"] / r2["wall"],
                "latency": serving.latency_summary(r2["jobs"]), "clocks": r2["clocks"], "how": how}
    print(json.dumps(result), flush=True)


def run_reference(args, wl_name, wl):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    import torch

    import oracle
    oracle.build()
    seed = 1000
    dev = torch.device("cuda", 0) if torch.cuda.is_available() else torch.device("cpu")
    what = "the workload"
    if wl.get("batched"):
        # chains are independent: the oracle on the batch's first chain
        from paper_1506_01418_gb300 import datagen
        J0, p0, ds, iseed = batched_specs(wl, seed)[0]
        N = sum(wl["I"] * J for J, _, _, _ in batched_specs(wl, seed))
        run_wl = batched_chain_wl(wl, J0, p0)
        V0, _, _ = datagen.dense_gamma(wl["I"], J0, wl["K_true"], ds)
        i, j, v = datagen.dense_to_coo(V0)
        W0, H0 = datagen.init_factors(wl["I"], J0, wl["K"], iseed, scale=wl["init_scale"], nonneg=True)
        i, j, v = (torch.from_numpy(x) for x in (i, j, v))
        what = f"chain 0 of the batch ({wl['I']} x {J0}, p = {p0})"
    else:
        i, j, v, W0, H0 = make_inputs(wl, seed, dev)
        N = int(v.numel())
        run_wl = wl
    if i is None:
        # dense V beyond the oracle's host arrays: one block as a B = 1 problem
        B = wl["B"]
        r1, c1 = wl["I"] // B, wl["J"] // B
        run_wl = dict(wl, I=r1, J=c1, B=1)
        Vb = v[:r1, :c1].float().cpu().numpy()
        hi, hj = (x.ravel() for x in np.meshgrid(np.arange(r1, dtype=np.int32),
                                                 np.arange(c1, dtype=np.int32), indexing="ij"))
        hv = Vb.ravel()
        W0, H0 = W0[:r1], H0[:, :c1]
        what = f"one {r1} x {c1} block of the workload as a B = 1 problem"
    else:
        hi, hj, hv = (x.cpu().numpy() for x in (i, j, v))
        if what == "the workload":
            run_wl, hi, hj, hv, W0, H0, what = oracle_sample(run_wl, hi, hj, hv, W0, H0)
    m = oracle_setup(run_wl, hi, hj, hv.astype(np.float64), W0.astype(np.float64),
                     H0.astype(np.float64), seed)
    wl = run_wl
    _, _, dt1 = oracle_rate(m, wl, 1, 1)
    budget = args.reference_budget / max(1, args.steps + args.warmup)
    per_step = max(1, min(wl["B"], int(budget / max(dt1, 1e-6))))
    t = 2
    for _ in range(args.warmup):
        oracle_rate(m, wl, t, per_step)
        t += per_step
    ent, secs = 0, 0.0
    for _ in range(args.steps):
        _, e, dt = oracle_rate(m, wl, t, per_step)
        ent += e
        secs += dt
        t += per_step
    rate = ent / secs
    ms = secs / args.steps * 1e3 * (N / max(ent / args.steps, 1))   # per full sweep
    sample = (f"each step {per_step} part-steps of {what} "
              f"({ent // args.steps} observed entries), FP64 oracle, OpenMP over blocks")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl_name, "I": WORKLOADS[wl_name]["I"],
                   "J": WORKLOADS[wl_name].get("J") or "per chain", "nnz": N, "K": wl["K"], "B": WORKLOADS[wl_name]["B"], "tweedie_p": wl["p"],
                   "phi": wl["phi"], "prior": wl["prior"], "eps": wl["eps"],
                   "step": "bounded sample of part-steps, rate per entry"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--compare-sweeps", type=int, default=20,
                    help="tensor-core workloads: sweeps of the BF16 vs FP32 comparison (0 = off)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving-compare", action="store_true",
                    help="serving workload: skip the per-job-streams replay of the trace")
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="seconds of oracle work for the cpu_baseline sample")
    ap.add_argument("--reference-budget", type=float, default=120.0,
                    help="seconds of oracle work for the whole reference arm")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        ap.error("--warmup must be >= 3")
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        if wl.get("serving"):
            print(json.dumps({"impl": "reference", "unavailable": "the serving workload has no "
                              "oracle counterpart (the oracle is a CPU chain, not a server)"}))
            return
        run_reference(args, args.workload, wl)
    elif wl.get("serving") or wl.get("batched"):
        # one GPU's loop / batch; under torchrun only rank 0 runs it
        if dist_env()[0] != 0:
            return
        if wl.get("serving"):
            run_serving(args, args.workload, wl)
        else:
            run_batched(args, args.workload, wl)
    else:
        run_ours(args, args.workload, wl)


if __name__ == "__main__":
    main()
