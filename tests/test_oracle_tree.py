"""Pins of the oracle tree (Section 2.1, Table 1): keys by brute-force containment search,
lists straight from their definitions, stencil counts, pre-order of sorted Morton keys."""
import itertools
import json
import os

import numpy as np
import pytest

from oracle import tree as otree
from oracle.kifmm import n_surface, surface_grid
from synth import cube_points, sphere_points


def test_keys_by_bruteforce_containment():
    depth = 3
    x = cube_points(3000).astype(np.float64)
    tr = otree.build_tree(x, depth, (0, 0, 0), 1.0)
    # every box of level 3 by explicit nested refinement of the unit cube; a point belongs to
    # the box whose half-open interval holds it (the clamp puts x == 1 in the last box)
    n = 2 ** depth
    w = 1.0 / n
    found = np.full(len(x), -1)
    for key in range(8 ** depth):
        # descend from the root: at each level the three key bits pick the octant
        lo = np.zeros(3)
        for level in range(depth):
            trip = (key >> (3 * (depth - 1 - level))) & 7
            lo = lo + np.array([(trip >> 2) & 1, (trip >> 1) & 1, trip & 1]) * (0.5 ** (level + 1))
        inside = np.all((x >= lo) & (x < lo + w), axis=1)
        found[inside] = key
    assert np.all(found >= 0)
    np.testing.assert_array_equal(tr.keys.astype(np.int64), found)


def test_morton_roundtrip_and_bit_order():
    a = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [5, 3, 6]])
    k = otree.morton(a, 3)
    assert list(k[:3]) == [4, 2, 1]   # x bit is the most significant of each triple
    np.testing.assert_array_equal(otree.demorton(k, 3), a)


def test_sorted_keys_are_preorder():
    depth = 3
    x = sphere_points(4000).astype(np.float64)
    tr = otree.build_tree(x, depth, (-1, -1, -1), 2.0)
    present = set(tr.leaf_keys.tolist())
    # depth-first, children in octant order 0..7: the leaves met in pre-order
    order = []

    def dfs(level, key):
        if level == depth:
            if key in present:
                order.append(key)
            return
        for c in range(8):
            dfs(level + 1, key * 8 + c)

    dfs(0, 0)
    assert order == tr.leaf_keys.tolist()
    assert np.all(np.diff(tr.leaf_keys.astype(np.int64)) > 0)
    # stable sort: equal keys keep the input order
    for b in range(len(tr.leaf_keys)):
        seg = tr.perm[tr.leaf_offsets[b]:tr.leaf_offsets[b + 1]]
        assert np.all(np.diff(seg) > 0)


@pytest.mark.parametrize("dist", ["cube", "sphere"])
@pytest.mark.parametrize("depth", [2, 3])
def test_lists_match_definitions(dist, depth):
    x = (cube_points(1500) if dist == "cube" else sphere_points(1500)).astype(np.float64)
    tr = otree.build_tree(x, depth)
    uo, ui = otree.u_lists(tr)
    bo, bi = otree.u_lists_bruteforce(tr)
    np.testing.assert_array_equal(uo, bo)
    np.testing.assert_array_equal(ui, bi)
    for level in range(2, depth + 1):
        vo, vi, vt = otree.v_lists(tr, level)
        bo, bi, bt = otree.v_lists_bruteforce(tr, level)
        np.testing.assert_array_equal(vo, bo)
        np.testing.assert_array_equal(vi, bi)
        np.testing.assert_array_equal(vt, bt)


def test_stencil_counts_full_tree():
    # one point per leaf at the leaf centres: every box exists
    depth = 4
    n = 2 ** depth
    g = (np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) + 0.5) / n
    tr = otree.build_tree(g, depth, (0, 0, 0), 1.0)
    uo, _ = otree.u_lists(tr)
    a = tr.level_anchors[depth]
    interior = np.all((a > 0) & (a < n - 1), axis=1)
    assert np.all(np.diff(uo)[interior] == 27)
    for level in (3, 4):
        vo, _, _ = otree.v_lists(tr, level)
        a = tr.level_anchors[level]
        m = 2 ** level
        inner = np.all((a >= 2) & (a < m - 2), axis=1) & np.all((a >> 1 >= 1) & (a >> 1 < m // 2 - 1), axis=1)
        assert inner.any()
        assert np.all(np.diff(vo)[inner] == 189)
        assert np.diff(vo).max() == 189


def test_transfer_vectors():
    tv = otree.transfer_vectors()
    assert len(tv) == 316
    full = set(itertools.product(range(-3, 4), repeat=3))
    inner = set(itertools.product(range(-1, 2), repeat=3))
    assert set(map(tuple, tv)) == full - inner
    np.testing.assert_array_equal(otree.transfer_index(tv), np.arange(316))
    # per child octant, exactly 189 transfer vectors have adjacent parents
    for c in range(8):
        a = np.array([[8 + ((c >> 2) & 1), 8 + ((c >> 1) & 1), 8 + (c & 1)]])
        ok = (np.abs(((a + tv) >> 1) - (a >> 1)) <= 1).all(axis=1)
        assert ok.sum() == 189


def test_surface_size_formula_and_golden():
    for p in range(2, 11):
        assert len(surface_grid(p)) == n_surface(p) == p ** 3 - (p - 2) ** 3 == 6 * (p - 1) ** 2 + 2
    with open(os.path.join(os.path.dirname(__file__), "golden", "surface_sizes.json")) as f:
        gold = json.load(f)
    for case in gold["cases"]:
        assert n_surface(case["p"]) == case["n_s"]
        assert 4 * n_surface(case["p"]) == case["bytes_fp32"]
    # every surface point lies on the boundary of [-1,1]^3
    s = surface_grid(6)
    assert np.all(np.isclose(np.abs(s).max(axis=1), 1.0))
    assert len(np.unique(s, axis=0)) == len(s)


def test_domain_default_and_clamp():
    x = np.array([[0.0, 0.0, 0.0], [1.0, 0.5, 0.25]])
    o, side = otree.domain_from_points(x)
    assert np.all(o == 0.0) and side == 1.0 * (1 + 2.0 ** -20)
    a = otree.anchors(np.array([[1.0, 1.0, 1.0]]), 3, (0, 0, 0), 1.0)
    assert np.all(a == 7)
