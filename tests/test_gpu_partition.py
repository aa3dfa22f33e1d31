"""Partitioned evaluation on virtual ranks (Section 3) through the C ABI.

Every output of the partitioned evaluation is computed by the same kernels from the same values
in the same order as by fmm_evaluate, so in FP64 (and in FP32) the two must agree bit for bit;
the setup's lists (layout, own boxes, ghosts, neighbourhoods, query sizes) must equal the
partition oracle's, which restates Box comm-setup and Eq. 3 from their definitions.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from oracle import partition as opart, tree as otree
from synth import cube_points, sphere_points, charges
from gpu_helpers import make_fmm

pytestmark = pytest.mark.gpu
CUBE = ((0, 0, 0), 1.0)
BALL = ((-1, -1, -1), 2.0)
CASES = [("cube", 60_000, 4, 4, 2, 1), ("cube", 60_000, 4, 4, 2, 7), ("cube", 60_000, 4, 4, 2, 64),
         ("sphere", 80_000, 5, 5, 2, 19), ("sphere", 80_000, 5, 5, 3, 37), ("sphere", 80_000, 6, 5, 4, 300)]


def _inputs(kind, n):
    x = cube_points(n) if kind == "cube" else sphere_points(n)
    q = charges(n, "u11" if kind == "cube" else "u01")
    return x, q, (CUBE if kind == "cube" else BALL)


@pytest.mark.parametrize("kind,n,p,depth,dg,P", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_partition_equals_unpartitioned(kind, n, p, depth, dg, P, precision):
    x, q, dom = _inputs(kind, n)
    f = make_fmm(x, p, depth, precision, dom)
    dt = torch.float64 if precision == "fp64" else torch.float32
    qd = torch.from_numpy(q).to("cuda", dt)
    phi, grad = f.evaluate(qd)
    f.partition_setup(dg, P)
    phi_p, grad_p = f.partition_evaluate(qd)
    torch.cuda.synchronize()
    assert torch.equal(phi, phi_p)
    assert torch.equal(grad, grad_p)
    # new densities: the U exchange carries them
    q2 = torch.from_numpy(charges(n, "normal", seed=5)).to("cuda", dt)
    a, ga = f.evaluate(q2)
    b, gb = f.partition_evaluate(q2)
    assert torch.equal(a, b) and torch.equal(ga, gb)


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x6"])
def test_partition_tensor_modes(precision):
    x, q, dom = _inputs("sphere", 80_000)
    f = make_fmm(x, 6, 5, precision, dom)
    qd = torch.from_numpy(q).cuda()
    phi, grad = f.evaluate(qd)
    f.partition_setup(3, 23)
    phi_p, grad_p = f.partition_evaluate(qd)
    torch.cuda.synchronize()
    # the tensor-core stencil's tiles differ between the two; its products of absent rows are zero
    assert torch.equal(phi, phi_p), float((phi - phi_p).abs().max() / phi.abs().max())
    assert torch.equal(grad, grad_p)


def test_partition_yukawa_and_gradient_only():
    x, q, dom = _inputs("sphere", 60_000)
    f = make_fmm(x, 5, 5, "fp64", dom, kernel="yukawa", kappa=3.0)
    qd = torch.from_numpy(q).to("cuda", torch.float64)
    phi, grad = f.evaluate(qd)
    f.partition_setup(2, 11)
    phi_p, grad_p = f.partition_evaluate(qd)
    _, g_only = f.partition_evaluate(qd, potential=False)
    torch.cuda.synchronize()
    assert torch.equal(phi, phi_p) and torch.equal(grad, grad_p) and torch.equal(grad, g_only)


@pytest.mark.parametrize("kind,n,p,depth,dg,P", [CASES[1], CASES[3], CASES[4], CASES[5]])
def test_setup_lists_match_oracle(kind, n, p, depth, dg, P):
    x, _, dom = _inputs(kind, n)
    f = make_fmm(x, p, depth, "fp32", dom)
    f.partition_setup(dg, P)
    tr = otree.build_tree(x.astype(np.float64), depth, *dom)
    ref = opart.partition(tr, dg, P)
    keys, owner = f.partition_layout()
    assert np.array_equal(keys.astype(np.uint64), tr.level_keys[dg])
    assert np.array_equal(owner, ref["owner"])
    total_boxes = np.zeros(depth + 1, np.int64)
    for r in range(P):
        rk = ref["ranks"][r]
        info = f.partition_info(r)
        assert info["first_root"] == ref["first_root"][r]
        assert info["n_local_roots"] == ref["first_root"][r + 1] - ref["first_root"][r]
        assert (info["first_point"], info["n_points"]) == rk["points"]
        for level in range(dg, depth + 1):
            own = f.partition_export(r, level, pkg.PARTITION_OWN)
            assert np.array_equal(own, rk["own"][level])
            total_boxes[level] += len(own)
        for level in range(dg + 1, depth + 1):
            gv = f.partition_export(r, level, pkg.PARTITION_GHOST_V)
            assert np.array_equal(gv, rk["ghost_v"][level]), (r, level)
            assert info["n_ghost_v"][level] == len(gv)
        gu = f.partition_export(r, 0, pkg.PARTITION_GHOST_U)
        assert np.array_equal(gu, rk["ghost_u"])
        assert list(f.partition_export(r, 0, pkg.PARTITION_NEIGHBOURS_U)) == rk["nb_u"]
        assert list(f.partition_export(r, 0, pkg.PARTITION_NEIGHBOURS_V)) == rk["nb_v"]
        assert info["n_query_u"] == rk["n_query_u"] and info["n_query_v"] == rk["n_query_v"]
        assert info["n_ghost_points"] == rk["n_ghost_points"]
        # exchange volumes: densities of the ghost points; the gathered u rows are the paper's
        # u vectors padded to 16 entries
        assert info["bytes_u"] == 4 * rk["n_ghost_points"]
        ns = 6 * (p - 1) ** 2 + 2
        nsp = (ns + 15) // 16 * 16
        assert info["bytes_gather"] == opart.message_bytes(info["n_local_roots"], p, 32) * nsp // ns
    for level in range(dg, depth + 1):
        assert total_boxes[level] == len(tr.level_keys[level])


def test_partition_host_buffers_and_timings():
    x, q, dom = _inputs("cube", 60_000)
    f = make_fmm(x, 4, 4, "fp32", dom)
    phi_h = np.zeros(len(x), np.float32)
    grad_h = np.zeros((len(x), 3), np.float32)
    f.partition_setup(2, 9)
    f.partition_evaluate_into(np.ascontiguousarray(q), phi_h, grad_h)
    phi, grad = f.evaluate(torch.from_numpy(q).cuda())
    assert np.array_equal(phi.cpu().numpy(), phi_h) and np.array_equal(grad.cpu().numpy(), grad_h)
    t = f.partition_timings()
    assert set(t) == set(pkg.PARTITION_PHASES)
    assert all(v >= 0 for v in t.values())
    assert t["total"] >= max(v for k, v in t.items() if k != "total")


def test_partition_errors():
    x, q, dom = _inputs("cube", 20_000)
    L = pkg.lib()
    f = make_fmm(x, 4, 4, "fp32", dom)
    qd = torch.from_numpy(q).cuda()
    phi = torch.empty(len(x), device="cuda")
    vp = ctypes.c_void_p
    # before the setup
    assert L.fmm_partition_evaluate(f._ctx, vp(qd.data_ptr()), vp(phi.data_ptr()), None) == 4
    info = pkg.RankInfo()
    assert L.fmm_partition_info(f._ctx, 0, ctypes.byref(info)) == 4
    # ranges
    for dg, P in ((1, 2), (4, 2), (2, 0), (2, 65)):
        assert L.fmm_partition_setup(f._ctx, dg, P) == 1, (dg, P)
    f.partition_setup(2, 4)
    assert L.fmm_partition_info(f._ctx, 4, ctypes.byref(info)) == 1
    cnt = ctypes.c_int64()
    assert L.fmm_partition_export(f._ctx, 0, 1, pkg.PARTITION_OWN, None, ctypes.addressof(cnt)) == 1
    assert L.fmm_partition_export(f._ctx, 0, 3, 9, None, ctypes.addressof(cnt)) == 1
    assert L.fmm_partition_evaluate(f._ctx, vp(qd.data_ptr()), None, None) == 1
    # a new tree drops the partition
    f.build_tree(torch.from_numpy(x).cuda())
    assert L.fmm_partition_evaluate(f._ctx, vp(qd.data_ptr()), vp(phi.data_ptr()), None) == 4
    # no tree / no operators
    g = pkg.FMM(p=4, depth=4, domain=dom)
    assert L.fmm_partition_setup(g._ctx, 2, 2) == 4
    g.build_tree(torch.from_numpy(x).cuda())
    assert L.fmm_partition_setup(g._ctx, 2, 2) == 4
    # the context stays usable
    p2, _ = f.evaluate(qd)
    torch.cuda.synchronize()
    assert torch.isfinite(p2).all()
