"""The distributed scheme of Section 3 with real processes (gloo on CPU, world sizes 2 and 4):
query packets, existence answers, neighbour exchanges of u vectors and ghost points, the gather
of the local roots' u at rank 0, the global pass there and the scatter of d, in FP64 with the
oracle's arithmetic.  The assembled field must equal the single-process kiFMM (to the order of
floating-point sums), and every rank's ghosts and neighbourhoods, found through the messages,
must equal the partition oracle's."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

CASES = {"cube": ("cube", 12_000, 4, 4, 2, ((0, 0, 0), 1.0)), "sphere": ("sphere", 16_000, 4, 5, 3, ((-1, -1, -1), 2.0))}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs(case):
    from synth import cube_points, sphere_points, charges
    kind, n, p, depth, dg, dom = CASES[case]
    x = cube_points(n) if kind == "cube" else sphere_points(n)
    return x.astype(np.float64), charges(n, "u11").astype(np.float64), p, depth, dg, dom


def _worker(rank, ws, port, case, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from oracle import distributed
        x, q, p, depth, dg, dom = _inputs(case)
        pos, pot, grd, facts, _ = distributed.run(x, q, p, depth, *dom, dg)
        out[rank] = (pos, pot, grd, {"nb_u": facts["nb_u"], "nb_v": facts["nb_v"],
                                     "ghost_u": facts["ghost_u"], "ghost_v": facts["ghost_v"]})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 4])
@pytest.mark.parametrize("case", ["cube", "sphere"])
def test_distributed_scheme_equals_single_process(case, ws, monkeypatch):
    from oracle import kifmm, partition as opart, tree as otree
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):   # one thread per rank
        monkeypatch.setenv(var, "1")
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_worker, args=(ws, _free_port(), case, out), nprocs=ws, join=True)
    x, q, p, depth, dg, dom = _inputs(case)
    tr = otree.build_tree(x, depth, *dom)
    n = len(x)
    phi_s, grad_s = np.full(n, np.nan), np.full((n, 3), np.nan)
    for r in range(ws):
        pos, pot, grd, _ = out[r]
        phi_s[pos], grad_s[pos] = pot, grd
    assert not np.isnan(phi_s).any()                       # every point has exactly one owner
    phi, grad = np.empty(n), np.empty((n, 3))
    phi[tr.perm], grad[tr.perm] = phi_s, grad_s
    ref = kifmm.evaluate(x, q, p, depth, *dom)
    assert np.linalg.norm(phi - ref.phi) / np.linalg.norm(ref.phi) < 1e-12
    assert np.linalg.norm(grad - ref.grad) / np.linalg.norm(ref.grad) < 1e-12
    part = opart.partition(tr, dg, ws)
    for r in range(ws):
        facts, rk = out[r][3], part["ranks"][r]
        assert facts["nb_u"] == rk["nb_u"] and facts["nb_v"] == rk["nb_v"]
        assert np.array_equal(facts["ghost_u"], rk["ghost_u"])
        for level in range(dg + 1, depth + 1):
            assert np.array_equal(facts["ghost_v"][level], rk["ghost_v"][level])
