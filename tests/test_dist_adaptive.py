"""The distributed scheme over an adaptive tree with real processes (gloo on CPU, world sizes 2
and 4; Section 2.3: uniform global levels, adaptive local trees): the ghosts of every rank's local
essential tree requested from their owners (points and densities for U and X, upward densities
for V and W), the gather of the local roots' u at rank 0, the global pass there, the scatter of
d, and the local downward stage with XLI, WLI and ULI.  The assembled field must equal the
single-process adaptive kiFMM to the order of floating-point sums."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

N, P_ORDER, CAPACITY, DEPTH, D_GLOBAL = 3000, 4, 24, 6, 2
DOMAIN = ((0.0, 0.0, 0.0), 1.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs():
    from synth import charges, mixed_points
    return mixed_points(N).astype(np.float64), charges(N, "u11").astype(np.float64)


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from oracle import distributed
        x, q = _inputs()
        pos, pot, grd, rk = distributed.run_adaptive(x, q, P_ORDER, CAPACITY, DEPTH, *DOMAIN, D_GLOBAL)
        out[rank] = (pos, pot, grd, len(rk["ghost_s"]), len(rk["ghost_u"]))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 4])
def test_distributed_adaptive_equals_single_process(ws, monkeypatch):
    from oracle import adaptive as ad
    # one thread per rank: the ranks' many small sums would otherwise oversubscribe the cores
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.setenv(var, "1")
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(ws, _free_port(), out), nprocs=ws, join=True)
    x, q = _inputs()
    tr = ad.build_tree(x, CAPACITY, DEPTH, *DOMAIN, min_level=D_GLOBAL)
    n = len(x)
    phi_s, grad_s = np.full(n, np.nan), np.full((n, 3), np.nan)
    for r in range(ws):
        pos, pot, grd, _, _ = out[r]
        phi_s[pos], grad_s[pos] = pot, grd
    assert not np.isnan(phi_s).any()                       # every point has exactly one owner
    phi, grad = np.empty(n), np.empty((n, 3))
    phi[tr.perm], grad[tr.perm] = phi_s, grad_s
    ref, gref, _, il = ad.evaluate(x, q, P_ORDER, CAPACITY, DEPTH, *DOMAIN, min_level=D_GLOBAL)
    assert sum(len(m) for m in il.w.values()) > 0
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-12
    assert np.linalg.norm(grad - gref) / np.linalg.norm(gref) < 1e-12
    assert all(out[r][3] > 0 and out[r][4] > 0 for r in range(ws))   # every rank exchanged ghosts


def _worker_one_root(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from oracle import distributed
        x, q = _inputs_one_root()
        pos, pot, grd, _ = distributed.run_adaptive(x, q, P_ORDER, CAPACITY, DEPTH, *DOMAIN, D_GLOBAL)
        out[rank] = (pos, pot, grd)
    finally:
        dist.destroy_process_group()


def _inputs_one_root():
    # every point inside one level-2 box: a single occupied local root for two ranks
    from synth import charges, cube_points
    n = 800
    return 0.26 + 0.23 * cube_points(n, seed=7).astype(np.float64), charges(n, "u11").astype(np.float64)


def test_distributed_adaptive_rank_without_local_roots(monkeypatch):
    from oracle import adaptive as ad
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        monkeypatch.setenv(var, "1")
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker_one_root, args=(2, _free_port(), out), nprocs=2, join=True)
    x, q = _inputs_one_root()
    assert min(len(out[r][0]) for r in range(2)) == 0       # one rank owns nothing
    tr = ad.build_tree(x, CAPACITY, DEPTH, *DOMAIN, min_level=D_GLOBAL)
    n = len(x)
    phi_s, grad_s = np.full(n, np.nan), np.full((n, 3), np.nan)
    for r in range(2):
        pos, pot, grd = out[r]
        phi_s[pos], grad_s[pos] = pot, grd
    assert not np.isnan(phi_s).any()
    phi, grad = np.empty(n), np.empty((n, 3))
    phi[tr.perm], grad[tr.perm] = phi_s, grad_s
    ref, gref, _, _ = ad.evaluate(x, q, P_ORDER, CAPACITY, DEPTH, *DOMAIN, min_level=D_GLOBAL)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-12
    assert np.linalg.norm(grad - gref) / np.linalg.norm(gref) < 1e-12
