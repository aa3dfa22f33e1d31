"""GPU octree (Morton keys, stable sort, leaves, levels, U and V lists) bit-exact against the
oracle tree of Section 2.1 / Table 1."""
import numpy as np
import pytest
import torch

from oracle import tree as otree
from synth import WORKLOADS, cube_points, sphere_points, sample_indices
from gpu_helpers import make_fmm

pytestmark = pytest.mark.gpu


def _check_tree(x, depth, domain, full_lists=True, sample=None):
    import paper_2604_19243_gb300 as pkg
    f = pkg.FMM(p=3, depth=depth, domain=domain)
    f.build_tree(torch.from_numpy(x).cuda())
    got = f.export_tree()
    info = f.info()
    o = otree.build_tree(x.astype(np.float64), depth, *(domain if domain else (None, None)))
    assert info["side"] == o.side and np.array_equal(info["origin"], o.origin)
    np.testing.assert_array_equal(got["perm"], o.perm)
    np.testing.assert_array_equal(got["leaf_keys"], o.leaf_keys)
    np.testing.assert_array_equal(got["leaf_offsets"], o.leaf_offsets)
    assert info["n_boxes"] == [len(k) for k in o.level_keys]
    if full_lists:
        uo, ui = otree.u_lists(o)
        np.testing.assert_array_equal(got["u_offsets"], uo)
        np.testing.assert_array_equal(got["u_idx"], ui)
    else:
        uo, ui = otree.u_lists(o, sample)
        for k, b in enumerate(sample):
            np.testing.assert_array_equal(got["u_idx"][got["u_offsets"][b]:got["u_offsets"][b + 1]],
                                          ui[uo[k]:uo[k + 1]])
    for level in range(depth + 1):
        lv = f.export_level(level, lists=level >= 2)
        np.testing.assert_array_equal(lv["keys"], o.level_keys[level])
        if level < 2:
            continue
        if full_lists:
            vo, vi, vt = otree.v_lists(o, level)
            np.testing.assert_array_equal(lv["v_offsets"], vo)
            np.testing.assert_array_equal(lv["v_idx"], vi)
            np.testing.assert_array_equal(lv["v_tvec"], vt)
        else:
            boxes = np.unique(np.minimum(sample, len(o.level_keys[level]) - 1))
            vo, vi, vt = otree.v_lists(o, level, boxes)
            for k, b in enumerate(boxes):
                s = slice(lv["v_offsets"][b], lv["v_offsets"][b + 1])
                np.testing.assert_array_equal(lv["v_idx"][s], vi[vo[k]:vo[k + 1]])
                np.testing.assert_array_equal(lv["v_tvec"][s], vt[vo[k]:vo[k + 1]])
    f.close()


@pytest.mark.parametrize("dist", ["cube", "sphere"])
@pytest.mark.parametrize("depth", [0, 1, 2, 3, 5, 6, 8])
def test_tree_small(dist, depth):
    # depths 6 and 8: the levels of the 8.39M sphere below its leaves' parents and of the 33.5M
    # cube, with every list compared in full
    n = 30_000
    x = cube_points(n) if dist == "cube" else sphere_points(n)
    domain = ((0, 0, 0), 1.0) if dist == "cube" else ((-1, -1, -1), 2.0)
    _check_tree(x, depth, domain)


@pytest.mark.parametrize("depth", [2, 4])
def test_tree_default_domain_and_ragged(depth):
    # odd N, a duplicated point, points on the domain's upper faces
    x = sphere_points(12_345).copy()
    x[100] = x[7]
    x[200] = x.max(axis=0)
    _check_tree(x, depth, None)


def test_tree_explicit_domain_clamps_boundary():
    x = cube_points(5000)
    x[:10] = 1.0           # exactly on the far faces -> last box
    x[10:20] = 0.0
    _check_tree(x, 3, ((0, 0, 0), 1.0))


@pytest.mark.slow
@pytest.mark.parametrize("name", ["cube1m_p6_d5", "sphere8m_p6_d7", "cube33m_p8_d8"])
def test_tree_full_size_sampled(name):
    w = WORKLOADS[name]
    x = w.points()
    o_leaves = {"sphere8m_p6_d7": 40_000, "cube1m_p6_d5": 30_000, "cube33m_p8_d8": 14_000_000}[name]
    sample = sample_indices(o_leaves, 200)
    _check_tree(x, w.depth, (w.origin, w.side), full_lists=False, sample=sample)
