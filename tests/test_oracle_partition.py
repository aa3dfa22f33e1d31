"""Pins of the partition oracle (Section 3, Box comm-setup) against the paper's definitions:
Eq. 3 against the existence answers to the query packets, the layout's invariants, the bound of
26 neighbours (exact for an interior rank of a full tree with one local root per rank), and the
message-size formula of Section 4 (no GPU)."""
import numpy as np
import pytest

from oracle import partition as opart, tree as otree
from synth import cube_points, sphere_points


def _tree(kind, n, depth):
    x = cube_points(n) if kind == "cube" else sphere_points(n)
    dom = ((0, 0, 0), 1.0) if kind == "cube" else ((-1, -1, -1), 2.0)
    return otree.build_tree(x.astype(np.float64), depth, *dom)


@pytest.mark.parametrize("kind,n,depth,dg,P", [("cube", 20_000, 4, 2, 7), ("sphere", 30_000, 5, 3, 13),
                                               ("sphere", 30_000, 5, 2, 40), ("cube", 20_000, 4, 3, 1)])
def test_eq3_equals_existence_answers(kind, n, depth, dg, P):
    tr = _tree(kind, n, depth)
    part = opart.partition(tr, dg, P)
    for rk in part["ranks"]:
        for level in range(dg + 1, depth + 1):
            assert np.array_equal(rk["ghost_v"][level], rk["ghost_v_eq3"][level])
        assert np.array_equal(rk["ghost_u"], rk["ghost_u_eq3"])
        # every answer was asked; every neighbour owns what it answered or was asked
        assert rk["n_query_v"] >= sum(len(v) for v in rk["ghost_v"].values())
        assert rk["n_query_u"] >= len(rk["ghost_u"])
    if P == 1:
        rk = part["ranks"][0]
        assert rk["nb_u"] == [] and rk["nb_v"] == [] and len(rk["ghost_u"]) == 0


@pytest.mark.parametrize("P", [1, 2, 5, 16, 56])
def test_layout_invariants(P):
    tr = _tree("sphere", 40_000, 5)
    first, owner = opart.layout(tr, 2, P)
    n_roots = len(tr.level_keys[2])
    assert first[0] == 0 and first[-1] == n_roots and np.all(np.diff(first) >= 1)
    assert np.array_equal(owner, np.repeat(np.arange(P), np.diff(first)))
    part = opart.partition(tr, 2, P)
    counts = [rk["points"][1] for rk in part["ranks"]]
    assert sum(counts) == 40_000
    # contiguous points in sorted order
    starts = [rk["points"][0] for rk in part["ranks"]]
    assert starts == list(np.cumsum([0] + counts[:-1]))
    # balance: no rank exceeds its share by more than one root's points
    leaf_root = tr.leaf_keys >> np.uint64(3 * 3)
    root_pts = np.bincount(np.searchsorted(tr.level_keys[2], leaf_root), weights=np.diff(tr.leaf_offsets))
    assert max(counts) <= np.ceil(40_000 / P) + root_pts.max()
    for level in range(2, 6):
        assert sum(len(rk["own"][level]) for rk in part["ranks"]) == len(tr.level_keys[level])


def test_interior_rank_has_26_neighbours():
    # full tree: depth 4, every leaf non-empty; one local root per rank at d_global = 2 (64 ranks)
    tr = _tree("cube", 200_000, 4)
    assert len(tr.leaf_keys) == 8 ** 4
    part = opart.partition(tr, 2, 64)
    roots = otree.demorton(tr.level_keys[2], 2)
    for r, rk in enumerate(part["ranks"]):
        a = roots[r]
        interior = bool(((a >= 1) & (a <= 2)).all())
        # a root's neighbours: the adjacent roots inside the domain
        n_adj = int(np.prod([3 - (a[k] in (0, 3)) for k in range(3)])) - 1
        assert len(rk["nb_u"]) == n_adj and len(rk["nb_v"]) == n_adj
        if interior:
            assert n_adj == 26
        assert len(rk["nb_u"]) <= 26 and len(rk["nb_v"]) <= 26


def test_message_size_formula():
    # Section 4: each u or d vector has 6(p-1)^2 + 2 entries; p = 3 in single precision is
    # 26 values, 104 bytes per local root
    assert opart.message_bytes(1, 3, 32) == 104
    assert opart.message_bytes(1000, 3, 64) == 208_000
    assert opart.message_bytes(7, 6, 32) == 7 * 152 * 4
