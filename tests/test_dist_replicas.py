"""Multi-rank logic of bench.py on CPU (gloo, world size 2): every rank runs an independent
replica, the job's time is the slowest rank's, throughput counts all ranks' points, and the
reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import bench
        t = bench.slowest(1.0 + rank, torch.device("cpu"), ws)   # rank r took 1 + r seconds
        out[rank] = (t, bench.job_rate(1000, 10, ws, t))
    finally:
        dist.destroy_process_group()


def test_slowest_rank_and_job_rate_gloo():
    ws, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        t, rate = out[r]
        assert t == 2.0                             # the slowest rank
        assert rate == pytest.approx(1000 * 10 * ws / 2.0)


def test_single_rank_is_identity():
    import bench
    assert bench.slowest(3.5, None, 1) == 3.5
    assert bench.job_rate(8, 2, 1, 4.0) == 4.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    from synth import WORKLOADS
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 3})()
    assert bench.run_reference(args, WORKLOADS["sphere8m_p6_d7"]) == 0
    assert capsys.readouterr().out == ""            # no work, no line on the other ranks
