"""Host-side logic of bench.py on the CPU: the max-over-ranks reduction with
two gloo ranks, the algorithmic byte count, the clock summary and the
kernel-traffic guard."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, value = bench.aggregate(ms_per_step_local=1.0 + rank, units_per_step_local=1000.0,
                                world=world)
    bench.barrier(world)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_aggregate_takes_slowest_rank_and_sums_units():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        ms, value = out[r]
        assert ms == 2.0                      # slowest rank
        assert value == pytest.approx(2 * 1000.0 / 2e-3)


def test_single_rank_aggregate_is_identity():
    ms, value = bench.aggregate(4.0, 500.0, 1)
    assert ms == 4.0 and value == pytest.approx(500.0 / 4e-3)


def test_part_step_bytes():
    wl = dict(I=100, J=50, K=10, B=4)
    # 8 bytes per entry + 4 per row offset + factors read and written in fp32
    # + the column-gradient scratch zeroed and read (8 J K)
    assert bench.part_step_bytes(wl, [10, 20, 30, 40]) == \
        8 * 25 + 4 * 104 + 8 * 150 * 10 + 8 * 50 * 10


def test_oracle_sample_keeps_the_first_blocks():
    """Above SAMPLE_ABOVE_NNZ entries the oracle runs on the first R x R
    blocks (rows and columns of the first R pieces) as a B = R problem."""
    import numpy as np
    wl = dict(I=64, J=32, K=3, B=16, nnz=0)
    g = np.random.default_rng(0)
    cells = g.choice(64 * 32, size=900, replace=False)
    i, j = (cells // 32).astype(np.int32), (cells % 32).astype(np.int32)
    v = g.uniform(1, 5, size=900).astype(np.float32)
    W0, H0 = g.uniform(size=(64, 3)), g.uniform(size=(3, 32))
    same = bench.oracle_sample(wl, i, j, v, W0, H0)
    assert same[0] is wl and same[6] == "the workload"
    old = bench.SAMPLE_ABOVE_NNZ
    try:
        bench.SAMPLE_ABOVE_NNZ = 100
        sub, si, sj, sv, sW, sH, what = bench.oracle_sample(wl, i, j, v, W0, H0)
    finally:
        bench.SAMPLE_ABOVE_NNZ = old
    R = bench.SAMPLE_PIECES
    assert (sub["I"], sub["J"], sub["B"]) == (R * 64 // 16, R * 32 // 16, R)
    keep = (i < sub["I"]) & (j < sub["J"])
    assert np.array_equal(si, i[keep]) and np.array_equal(sv, v[keep]) and sub["nnz"] == keep.sum()
    assert sW.shape == (sub["I"], 3) and sH.shape == (3, sub["J"])
    # each block of the sample is a block of the workload: same piece sizes
    assert sub["I"] // sub["B"] == wl["I"] // wl["B"] and sub["J"] // sub["B"] == wl["J"] // wl["B"]


def test_clock_summary_window_and_reasons():
    cs = bench.ClockSampler.__new__(bench.ClockSampler)
    cs.samples = [
        (10.0, ["t", "1500", "2070", "900", "Not Active", "Not Active", "Not Active", "Active"]),
        (11.0, ["t", "1900", "2070", "950", "Not Active", "Not Active", "Not Active",
                "Not Active"]),
        (12.0, ["t", "1950", "2070", "960", "Not Active", "Not Active", "Not Active",
                "Not Active"]),
        (30.0, ["t", "800", "2070", "100", "Active", "Not Active", "Not Active", "Not Active"]),
    ]
    s = cs.summary(10.5, 12.5)
    assert s["sm_mhz"] == 1925.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == []
    assert s["window"] == "timed"
    s = cs.summary(9.5, 30.5)
    assert s["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_kernel_traffic_requires_unchanged_source(tmp_path, monkeypatch):
    """The recorded DRAM traffic is reported only while every source it was
    measured on is unchanged (sha256 of each file in the record)."""
    import hashlib
    import shutil
    wl = bench.DEFAULT_WORKLOAD
    t = bench.kernel_traffic(wl)
    path = os.path.join(ROOT, "profiles", "part_step_traffic.json")
    if not os.path.exists(path):
        assert t is None
        return
    rec = json.load(open(path)).get(wl)
    if rec is None:
        assert t is None
        return
    same = all(hashlib.sha256(open(os.path.join(ROOT, "paper_1506_01418_gb300", "csrc", f), "rb")
                              .read()).hexdigest() == h for f, h in rec["sources_sha256"].items())
    assert t == (rec["dram_bytes_per_launch"] if same else None)
    # a copy of the tree with one recorded source changed reports nothing
    fake = tmp_path / "root"
    (fake / "profiles").mkdir(parents=True)
    (fake / "paper_1506_01418_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(path, fake / "profiles" / "part_step_traffic.json")
    for f in rec["sources_sha256"]:
        shutil.copy(os.path.join(ROOT, "paper_1506_01418_gb300", "csrc", f),
                    fake / "paper_1506_01418_gb300" / "csrc" / f)
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.kernel_traffic(wl) == t
    victim = fake / "paper_1506_01418_gb300" / "csrc" / next(iter(rec["sources_sha256"]))
    victim.write_bytes(victim.read_bytes() + b"\n// changed\n")
    assert bench.kernel_traffic(wl) is None
