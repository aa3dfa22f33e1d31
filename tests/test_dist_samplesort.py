"""Step (1) of the distributed setup with real processes (gloo on CPU): the sample sort of the
points by their coarse (local-root) Morton keys.  Pinned by what fixes it independently: the
buckets concatenated in rank order are the stable global sort by leaf key (the single-process
tree's permutation), no local root is split between ranks, and the buckets' deviation from N / P
shrinks as the sample size b grows (Section 2.3: the splitters' spread falls like 1 / sqrt(b))."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

DEPTH, D_GLOBAL = 5, 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _points(kind, n):
    from synth import cube_points, sphere_points
    if kind == "cube":
        return cube_points(n).astype(np.float64), ((0.0, 0.0, 0.0), 1.0)
    return sphere_points(n).astype(np.float64), ((-1.0, -1.0, -1.0), 2.0)


def _worker(rank, ws, port, kind, n, bs, seeds, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from oracle import samplesort
        x, dom = _points(kind, n)
        lo, hi = rank * n // ws, (rank + 1) * n // ws          # this rank's slice of the input
        res = {}
        for b in bs:
            for seed in seeds:
                idx, keys, _, spl = samplesort.samplesort(x[lo:hi], np.arange(lo, hi), DEPTH, D_GLOBAL, *dom, b, seed)
                res[(b, seed)] = (idx, keys)
        out[rank] = res
    finally:
        dist.destroy_process_group()


def _run(ws, kind, n, bs, seeds, monkeypatch):
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.setenv(var, "1")
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(ws, _free_port(), kind, n, bs, seeds, out), nprocs=ws, join=True)
    return {r: out[r] for r in range(ws)}


@pytest.mark.parametrize("ws,kind", [(2, "cube"), (4, "sphere")])
def test_buckets_are_the_global_stable_sort(ws, kind, monkeypatch):
    from oracle import tree as otree
    n = 20_000
    res = _run(ws, kind, n, [64], [0], monkeypatch)
    x, dom = _points(kind, n)
    tr = otree.build_tree(x, DEPTH, *dom)
    idx = np.concatenate([res[r][(64, 0)][0] for r in range(ws)])
    keys = np.concatenate([res[r][(64, 0)][1] for r in range(ws)])
    np.testing.assert_array_equal(idx, tr.perm)
    np.testing.assert_array_equal(keys, tr.keys[tr.perm])
    roots = [set((res[r][(64, 0)][1] >> np.uint64(3 * (DEPTH - D_GLOBAL))).tolist()) for r in range(ws)]
    for a in range(ws):
        for c in range(a + 1, ws):
            assert not roots[a] & roots[c]                     # no local root split between ranks


def test_balance_improves_with_the_sample_size(monkeypatch):
    ws, n = 4, 40_000
    bs, seeds = [8, 512], [0, 1, 2, 3, 4]
    res = _run(ws, "cube", n, bs, seeds, monkeypatch)
    dev = {}
    for b in bs:
        dev[b] = np.mean([max(abs(len(res[r][(b, s)][0]) - n / ws) for r in range(ws)) / (n / ws) for s in seeds])
    assert dev[512] < dev[8] / 2.5, dev
    assert dev[512] < 0.05, dev


def _worker_uneven(rank, ws, port, n, b, out):
    # rank 0 holds 10 points, fewer than the b samples it is asked for: it sends all of them
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from oracle import samplesort
        x, dom = _points("cube", n)
        cuts = [0, 10] + [10 + (n - 10) * k // (ws - 1) for k in range(2, ws)] + [n]
        lo, hi = cuts[rank], cuts[rank + 1]
        idx, keys, _, _ = samplesort.samplesort(x[lo:hi], np.arange(lo, hi), DEPTH, D_GLOBAL, *dom, b, 0)
        out[rank] = (idx, keys)
    finally:
        dist.destroy_process_group()


def test_rank_with_fewer_points_than_samples(monkeypatch):
    from oracle import tree as otree
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.setenv(var, "1")
    ws, n, b = 4, 40_000, 512
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker_uneven, args=(ws, _free_port(), n, b, out), nprocs=ws, join=True)
    x, dom = _points("cube", n)
    tr = otree.build_tree(x, DEPTH, *dom)
    np.testing.assert_array_equal(np.concatenate([out[r][0] for r in range(ws)]), tr.perm)
    # splitters at the quantiles of the samples actually drawn keep the buckets near n / ws
    sizes = [len(out[r][0]) for r in range(ws)]
    assert max(abs(s - n / ws) for s in sizes) / (n / ws) < 0.15, sizes
