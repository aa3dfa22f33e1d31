"""Adaptive tree and its U, V, W and X lists built on the device (Section 2.1, Table 1), bit-exact
against the oracle's adaptive tree: the state of every box (not kept, leaf, refined), its point
count, and every list member by member in row order."""
import numpy as np
import pytest
import torch

from oracle import adaptive as ad
from synth import mixed_points, sphere_points

pytestmark = pytest.mark.gpu

UNIT = ((0.0, 0.0, 0.0), 1.0)
SPHERE = ((-1.0, -1.0, -1.0), 2.0)


def _enc(level, key):
    return (np.asarray(level, np.int64) << 40) | np.asarray(key, np.int64)


def _check(x, capacity, depth, domain):
    import paper_2604_19243_gb300 as pkg
    f = pkg.FMM(p=3, depth=depth, domain=domain)
    f.build_tree(torch.from_numpy(np.ascontiguousarray(x)).cuda())
    f.adaptive_setup(capacity)
    # rows of the device tables -> (level, key)
    keys = [f.export_level(l, lists=False)["keys"].astype(np.int64) for l in range(depth + 1)]
    row_enc = np.concatenate([_enc(l, k) for l, k in enumerate(keys)])
    rows = len(row_enc)
    info = f.adaptive_info()
    assert info["n_rows"] == rows and info["capacity"] == capacity

    o = ad.build_tree(x.astype(np.float64), capacity, depth, *domain)
    il = ad.interaction_lists(o)
    lv, ix = o.boxes()
    o_enc = _enc(lv, np.concatenate(o.level_keys).astype(np.int64))
    o_leaf = np.concatenate(o.level_leaf)
    pos = np.searchsorted(row_enc, o_enc)                 # oracle box -> device row
    assert np.array_equal(row_enc[pos], o_enc)

    # states and point counts
    want = np.zeros(rows, np.int64)
    want[pos] = np.where(o_leaf, 1, 2)
    got_state = f.adaptive_export(pkg.ADAPTIVE_STATE)
    np.testing.assert_array_equal(got_state, want)
    assert info["n_leaves"] == [int(l.sum()) for l in o.level_leaf]
    assert info["n_refined"] == [int((~l).sum()) for l in o.level_leaf]
    got_count = f.adaptive_export(pkg.ADAPTIVE_COUNT)
    np.testing.assert_array_equal(got_count[pos], np.concatenate([np.diff(r, axis=1)[:, 0] for r in o.level_ranges]))

    # lists, member by member (device rows sorted ascending = (level, key) ascending)
    for kind, lists in ((pkg.ADAPTIVE_U, il.u), (pkg.ADAPTIVE_V, il.v), (pkg.ADAPTIVE_W, il.w),
                        (pkg.ADAPTIVE_X, il.x)):
        off, idx = f.adaptive_export(kind)
        assert off[0] == 0 and off[-1] == len(idx)
        want_len = np.zeros(rows, np.int64)
        want_rows = {}
        for b, members in lists.items():
            want_len[pos[b]] = len(members)
            want_rows[int(pos[b])] = pos[np.asarray(members, np.int64)]
        np.testing.assert_array_equal(np.diff(off), want_len, err_msg=f"list kind {kind}: lengths")
        for r, m in want_rows.items():
            np.testing.assert_array_equal(idx[off[r]:off[r + 1]], m, err_msg=f"list kind {kind}, row {r}")
        assert info["n_entries"][kind - pkg.ADAPTIVE_U] == len(idx)
    return info


@pytest.mark.parametrize("case", ["mixed", "sphere", "capped", "uniform", "single_leaf", "deep"])
def test_adaptive_tree_and_lists_match_oracle(case):
    if case == "mixed":
        info = _check(mixed_points(3000), 32, 6, UNIT)
        assert info["n_entries"][2] > 0 and info["n_entries"][3] > 0
    elif case == "sphere":
        _check(sphere_points(1500), 20, 5, SPHERE)
    elif case == "capped":        # depth 3 caps refinement: leaves of level 3 hold more than q
        _check(mixed_points(2000), 16, 3, UNIT)
    elif case == "uniform":       # capacity 0 refines every non-empty box: the uniform tree
        info = _check(mixed_points(1500), 0, 3, UNIT)
        assert info["n_entries"][2] == 0 and info["n_entries"][3] == 0
    elif case == "single_leaf":   # capacity >= n: the root is the only leaf
        info = _check(mixed_points(500), 500, 4, UNIT)
        assert info["n_leaves"][0] == 1 and info["n_entries"] == [1, 0, 0, 0]
    else:                         # a tight cluster refined to depth 9
        info = _check(mixed_points(20000, radius=0.02), 8, 9, UNIT)
        assert info["n_leaves"][9] > 0 and info["n_entries"][2] > 0


def test_adaptive_state_errors():
    import paper_2604_19243_gb300 as pkg
    f = pkg.FMM(p=3, depth=3, domain=UNIT)
    with pytest.raises(pkg.FmmError) as e:
        f.adaptive_setup(8)                 # no tree yet
    assert e.value.status == 4
    f.build_tree(torch.from_numpy(mixed_points(400)).cuda())
    with pytest.raises(pkg.FmmError) as e:
        f.adaptive_info()
    assert e.value.status == 4
    with pytest.raises(pkg.FmmError) as e:
        f.adaptive_setup(-1)
    assert e.value.status == 1
    f.adaptive_setup(8)
    with pytest.raises(pkg.FmmError) as e:
        f.adaptive_export(9)
    assert e.value.status == 1
    f.build_tree(torch.from_numpy(mixed_points(300)).cuda())   # a new tree discards the adaptive one
    with pytest.raises(pkg.FmmError) as e:
        f.adaptive_info()
    assert e.value.status == 4
