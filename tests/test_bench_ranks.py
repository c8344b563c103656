"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Under torchrun every rank runs an independent replica of the whole setup.
The job's time is the slowest rank's, and the job delivers one setup per
rank in that time. The reference arm runs on rank 0 only, and the other
ranks exit without work or output.
"""
import argparse
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [1500.0, 2250.0][rank]
        ms = bench.reduce_max_over_ranks(ms_local, dist, device="cpu")
        value = bench.whole_job_seconds_per_setup(ms, world)
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


def test_timing_is_the_slowest_rank_and_value_counts_every_replica():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 2250.0
        assert value == pytest.approx(2250.0 / 1000.0 / world)


def test_single_process_reduction_is_the_identity():
    assert bench.reduce_max_over_ranks(123.5) == 123.5
    assert bench.whole_job_seconds_per_setup(6500.0, 1) == pytest.approx(6.5)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    def fail(*a, **k):
        raise AssertionError("a rank other than 0 ran the oracle")

    monkeypatch.setattr(bench, "cpu_sample", fail)
    args = argparse.Namespace(steps=1, warmup=3)
    cfg = bench.CONFIGS[bench.DEFAULT_CONFIG]
    assert bench.run_reference(args, cfg, bench.DEFAULT_CONFIG, -0.4, "test", rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(capsys, monkeypatch):
    calls = []

    def fake_sample(cfg, m0, coarse_eo=1):
        calls.append(m0)
        return 1.0, 40.0 + len(calls), 16, "fake sample"

    monkeypatch.setattr(bench, "cpu_sample", fake_sample)
    monkeypatch.delenv("OMP_NUM_THREADS", raising=False)  # restored after the test
    args = argparse.Namespace(steps=2, warmup=3, coarse_eo=1)
    cfg = bench.CONFIGS[bench.DEFAULT_CONFIG]
    bench.run_reference(args, cfg, bench.DEFAULT_CONFIG, -0.4, "test", rank=0, world=2)
    import json

    line = json.loads(capsys.readouterr().out.strip())
    assert len(calls) == 5  # warm-up samples are run but not timed
    assert line["impl"] == "reference"
    assert line["value"] == pytest.approx((44.0 + 45.0) / 2)
    assert line["e2e"] == {"value": line["value"], "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert line["cpu_baseline"]["cores"] == 16 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["higher_is_better"] is False and line["n_gpus"] == 2


def test_reference_arm_on_rank_zero_uses_every_host_core(capsys, monkeypatch):
    """torchrun sets OMP_NUM_THREADS=1 for each rank; in the reference arm only
    rank 0 works, so it lifts that limit before the oracle library loads."""
    seen = []

    def fake_sample(cfg, m0, coarse_eo=1):
        seen.append(os.environ.get("OMP_NUM_THREADS"))
        return 1.0, 1.0, int(seen[-1]), "fake sample"

    monkeypatch.setenv("OMP_NUM_THREADS", "1")
    monkeypatch.setattr(bench, "cpu_sample", fake_sample)
    args = argparse.Namespace(steps=1, warmup=0, coarse_eo=1)
    cfg = bench.CONFIGS[bench.DEFAULT_CONFIG]
    bench.run_reference(args, cfg, bench.DEFAULT_CONFIG, -0.4, "test", rank=0, world=2)
    capsys.readouterr()
    assert seen == [str(os.cpu_count() or 1)]
