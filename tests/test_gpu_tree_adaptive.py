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


# ---- evaluation over the adaptive tree (Algorithm 1 with XLI and WLI) ----

def _adaptive_fmm(x, p, depth, precision, domain, capacity):
    from gpu_helpers import make_fmm
    f = make_fmm(x, p, depth, precision, domain)
    f.adaptive_setup(capacity)
    return f


def _dev(a, precision):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64 if precision == "fp64" else torch.float32)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("case", ["mixed", "sphere", "deep"])
def test_adaptive_evaluate_matches_oracle(case, precision):
    import paper_2604_19243_gb300 as pkg
    from gpu_helpers import rel
    from oracle import direct
    from synth import charges
    if case == "mixed":
        n, cap, depth, dom, x = 4000, 32, 6, UNIT, mixed_points(4000)
        qv = charges(n, "u11")
    elif case == "deep":   # a tight cluster in a uniform cloud: leaves from level 2 to level 8
        n, cap, depth, dom, x = 12000, 32, 8, UNIT, mixed_points(12000, radius=0.02)
        qv = charges(n, "u11")
    else:
        n, cap, depth, dom, x = 3000, 24, 5, SPHERE, sphere_points(3000)
        qv = charges(n, "u01")
    p = 6
    f = _adaptive_fmm(x, p, depth, precision, dom, cap)
    x64, q64 = x.astype(np.float64), qv.astype(np.float64)
    qd = _dev(qv, precision)
    # near part: the ULI over the adaptive U lists, to rounding
    phi_n, grad_n = f.adaptive_evaluate(qd, parts=pkg.PART_NEAR)
    o_phi_n, o_grad_n, _, il = ad.evaluate(x64, q64, p, cap, depth, *dom, lists=("U",))
    tol_near = 1e-12 if precision == "fp64" else 2e-6
    assert rel(phi_n.cpu().numpy(), o_phi_n) < tol_near
    assert rel(grad_n.cpu().numpy(), o_grad_n) < tol_near
    # the whole field against the FP64 adaptive oracle at the same p
    phi, grad = f.adaptive_evaluate(qd)
    o_phi, o_grad, _, _ = ad.evaluate(x64, q64, p, cap, depth, *dom)
    assert sum(len(m) for m in il.w.values()) > 0 and il.x
    e_phi, e_grad = rel(phi.cpu().numpy(), o_phi), rel(grad.cpu().numpy(), o_grad)
    assert e_phi < 1e-5 and e_grad < 1e-4, (e_phi, e_grad)
    if precision == "fp64":   # the oracle's steps in its order: rounding and the M2L compression only
        assert e_phi < 1e-8 and e_grad < 1e-8, (e_phi, e_grad)
    # and against the direct sum
    d_phi, d_grad = direct.direct_self(x64, q64)
    assert rel(phi.cpu().numpy(), d_phi) < 2e-5 and rel(grad.cpu().numpy(), d_grad) < 1e-4
    # gradient only: the same gradients
    none, grad_only = f.adaptive_evaluate(qd, potential=False)
    assert none is None and torch.equal(grad_only, grad)


def test_adaptive_evaluate_on_the_fully_refined_tree_is_the_uniform_evaluation():
    from gpu_helpers import rel
    from synth import charges
    x, qv = mixed_points(3000), charges(3000, "u11")
    f = _adaptive_fmm(x, 6, 4, "fp64", UNIT, 0)
    qd = _dev(qv, "fp64")
    phi_a, grad_a = f.adaptive_evaluate(qd)
    phi_u, grad_u = f.evaluate(qd)
    assert rel(phi_a.cpu().numpy(), phi_u.cpu().numpy()) < 1e-13
    assert rel(grad_a.cpu().numpy(), grad_u.cpu().numpy()) < 1e-13


def test_adaptive_evaluate_refusals():
    import paper_2604_19243_gb300 as pkg
    from gpu_helpers import make_fmm
    from synth import charges
    x, qv = mixed_points(1000), charges(1000, "u11")
    f = make_fmm(x, 4, 4, "fp32", UNIT)
    with pytest.raises(pkg.FmmError) as e:
        f.adaptive_evaluate(_dev(qv, "fp32"))             # no adaptive tree yet
    assert e.value.status == 4
    f.adaptive_setup(16)
    with pytest.raises(pkg.FmmError) as e:
        f.adaptive_evaluate(_dev(qv, "fp32"), parts=0)
    assert e.value.status == 1
    g = make_fmm(x, 4, 4, "fp16x3", UNIT)
    g.adaptive_setup(16)
    with pytest.raises(pkg.FmmError) as e:
        g.adaptive_evaluate(_dev(qv, "fp32"))
    assert e.value.status == 6
