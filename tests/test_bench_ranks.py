"""Host logic of bench.py's multi-process (replica) path, on CPU with gloo, world size 2: the job
time is the maximum over ranks, the job value aggregates every rank's layer, and the reference
arm prints from rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, device="cpu")
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    world = 2
    times = [0.125, 0.5]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), times, out), nprocs=world, join=True)
        assert out[0] == out[1] == max(times)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(0.25, 1) == 0.25


def test_job_value_counts_every_rank():
    assert bench.job_value(4096, 1, 0.5) == 4096 ** 3 / 0.5
    assert bench.job_value(4096, 4, 0.5) == 4 * 4096 ** 3 / 0.5


def test_reference_arm_prints_on_rank_zero_only():
    args = bench.parse(["--impl", "reference", "--n", "64", "--steps", "1", "--warmup", "0"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, rank=1, world=2)
    assert buf.getvalue() == ""


def test_reference_arm_line_keeps_the_contract():
    """The reference arm (the oracle on the host cores) prints one JSON line with the fields the
    measurement contract names: the same metric, unit and direction as the GPU arm, and a
    cpu_baseline / e2e pair describing its own run."""
    import json
    args = bench.parse(["--impl", "reference", "--n", "64", "--steps", "1", "--warmup", "3"])
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args, rank=0, world=1)
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["unit"] == "ring-MAC/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["metric"].startswith("secure Z_2^64 ring-MAC/s")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("secure GEMM 64x64x64")


def test_both_arms_report_the_same_config():
    assert bench.layer_config(8192, 8192, 8192, 13, "tc", 1) == bench.layer_config(8192, 8192, 8192, 13, "tc", 1)
    args = bench.parse(["--impl", "reference", "--n", "64", "--steps", "1", "--warmup", "0"])
    import contextlib, io, json
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args, rank=0, world=1)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["config"] == bench.layer_config(64, 64, 64, 13, "tc", 1)
