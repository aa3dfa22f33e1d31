"""Pins of the adaptive-tree oracle (Section 2.1: adaptive refinement and the U, V, W, X lists;
Algorithm 1: the XLI and WLI branches).

What fixes each piece, independently of the code under test:
  * the tree: a recursive subdivision written here from the refinement rule gives the same boxes
    and leaves; capacity and containment hold box by box;
  * the lists: every ordered pair of leaves (target, source) is accounted for exactly once by U,
    by V between an ancestor of each, by W from an ancestor of the source or by X into an
    ancestor of the target (the partition of the field sum the lists exist for); the geometry of
    each list (levels, adjacency, separation) holds member by member;
  * special cases: a fully refined tree is the uniform tree (lists and field equal the uniform
    oracle's); a single leaf is the direct sum;
  * the field: error against the FP64 direct sum falls with p and is below 5e-6 at p = 6 on a
    strongly non-uniform cloud; leaving out W or X (a planted mistake) breaks it.
"""
import numpy as np
import pytest

from oracle import adaptive as ad, direct, kifmm, tree as otree
from synth import charges, mixed_points, sphere_points

DOMAIN = ((0.0, 0.0, 0.0), 1.0)


def _mixed(n=3000):
    return mixed_points(n).astype(np.float64), charges(n, "u11").astype(np.float64)


@pytest.fixture(scope="module")
def ops6():
    return kifmm.build_operators(6, 1.0, 6)


def _recursive(anchors, depth, q):
    """Boxes and leaves of the refinement rule, by recursion from the root."""
    boxes, leaves = set(), set()

    def rec(level, anc, idx):
        boxes.add((level, anc))
        if len(idx) <= q or level == depth:
            leaves.add((level, anc))
            return
        sub = anchors[idx] >> (depth - level - 1)
        for c in range(8):
            child = (2 * anc[0] + ((c >> 2) & 1), 2 * anc[1] + ((c >> 1) & 1), 2 * anc[2] + (c & 1))
            keep = idx[(sub == np.array(child)).all(axis=1)]
            if len(keep):
                rec(level + 1, child, keep)

    rec(0, (0, 0, 0), np.arange(len(anchors)))
    return boxes, leaves


@pytest.mark.parametrize("case", ["mixed", "sphere", "capped"])
def test_tree_matches_recursive_refinement(case):
    if case == "sphere":
        x, q, depth, dom = sphere_points(1500).astype(np.float64), 20, 5, ((-1.0, -1.0, -1.0), 2.0)
    else:
        x, q, depth, dom = _mixed(2000)[0], 16, (3 if case == "capped" else 6), DOMAIN
    tr = ad.build_tree(x, q, depth, *dom)
    anchors = otree.anchors(x, depth, *dom)
    boxes, leaves = _recursive(anchors, depth, q)
    got = {(l, tuple(int(v) for v in a)) for l in range(depth + 1) for a in tr.level_anchors[l]}
    got_leaves = {(l, tuple(int(v) for v in a)) for l in range(depth + 1)
                  for a in tr.level_anchors[l][tr.level_leaf[l]]}
    assert got == boxes
    assert got_leaves == leaves
    # capacity: only leaves of level D may exceed q; every other box holds more than q
    for l in range(depth + 1):
        cnt = np.diff(tr.level_ranges[l], axis=1)[:, 0]
        assert (cnt > 0).all()
        if l < depth:
            assert (cnt[tr.level_leaf[l]] <= q).all()
        assert (cnt[~tr.level_leaf[l]] > q).all()
    if case == "capped":
        assert (np.diff(tr.level_ranges[depth], axis=1) > q).any()
    # leaves partition the sorted points, and each point lies in its leaf's cube
    lv, ix = tr.leaves()
    rng = np.array([tr.level_ranges[l][i] for l, i in zip(lv, ix)])
    assert rng[0, 0] == 0 and rng[-1, 1] == len(x) and (rng[1:, 0] == rng[:-1, 1]).all()
    sa = anchors[tr.perm]
    for (l, i), (b, e) in zip(zip(lv, ix), rng):
        assert ((sa[b:e] >> (depth - l)) == tr.level_anchors[l][i]).all()


def _leaf_ranges(tr):
    """Pre-order position of every leaf, and for every box the range of its descendant leaves."""
    lv, ix = tr.boxes()
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    leaf_lv, leaf_ix = tr.leaves()
    leaf_id = base[leaf_lv] + leaf_ix
    begins = np.array([tr.level_ranges[l][i, 0] for l, i in zip(leaf_lv, leaf_ix)])
    pos = {int(b): k for k, b in enumerate(leaf_id)}
    span = {}
    for b, (l, i) in enumerate(zip(lv, ix)):
        lo, hi = tr.level_ranges[l][i]
        span[b] = (int(np.searchsorted(begins, lo)), int(np.searchsorted(begins, hi)))
    return pos, span, len(leaf_id)


def _cover(tr, il):
    """How often each ordered pair of leaves (target, source) is accounted for by the lists."""
    pos, span, n = _leaf_ranges(tr)
    cover = np.zeros((n, n), np.int64)
    for t, members in il.u.items():
        for s in members:
            cover[pos[t], pos[int(s)]] += 1
    for b, members in il.v.items():
        for a in members:
            (b0, b1), (a0, a1) = span[b], span[int(a)]
            cover[b0:b1, a0:a1] += 1
    for t, members in il.w.items():
        for a in members:
            a0, a1 = span[int(a)]
            cover[pos[t], a0:a1] += 1
    for b, members in il.x.items():
        for s in members:
            b0, b1 = span[b]
            cover[b0:b1, pos[int(s)]] += 1
    return cover


@pytest.mark.parametrize("case", ["mixed", "sphere"])
def test_lists_account_for_every_leaf_pair_once(case):
    if case == "sphere":
        x, q, depth, dom = sphere_points(1500).astype(np.float64), 20, 5, ((-1.0, -1.0, -1.0), 2.0)
    else:
        x, q, depth, dom = _mixed(2000)[0], 16, 6, DOMAIN
    tr = ad.build_tree(x, q, depth, *dom)
    il = ad.interaction_lists(tr)
    cover = _cover(tr, il)
    assert (cover == 1).all(), np.argwhere(cover != 1)[:5]
    assert sum(len(m) for m in il.w.values()) > 0        # the adaptive branches are exercised
    assert sum(len(m) for m in il.x.values()) > 0


@pytest.mark.parametrize("mistake", ["w_without_parent_condition", "v_with_adjacent_box", "u_missing_coarser_leaf"])
def test_pair_coverage_catches_planted_list_mistakes(mistake):
    """Plausible slips in the list definitions, planted in the oracle's lists: each breaks the
    exact coverage of the leaf pairs."""
    tr = ad.build_tree(_mixed(2000)[0], 16, 6, *DOMAIN)
    il = ad.interaction_lists(tr)
    lv, ix = tr.boxes()
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    anc = np.concatenate(tr.level_anchors)
    par = np.full(len(lv), -1)
    for l in range(1, tr.depth + 1):
        par[base[l]:base[l + 1]] = base[l - 1] + tr.parent(l)
    if mistake == "w_without_parent_condition":      # a W member's child joins the list too
        t, a = next((t, a) for t, m in il.w.items() for a in m if (par == a).any())
        child = int(np.nonzero(par == a)[0][0])
        il.w[t] = np.sort(np.append(il.w[t], child))
        il.x.setdefault(child, np.zeros(0, np.int64))
        il.x[child] = np.sort(np.append(il.x[child], t))
    elif mistake == "v_with_adjacent_box":           # a colleague (adjacent, same level) enters V
        b, c = next((b, c) for b in il.v for c in np.nonzero((lv == lv[b]) & (np.abs(anc - anc[b]).max(axis=1) == 1))[0])
        il.v[b] = np.sort(np.append(il.v[b], c))
    else:                                            # a coarser adjacent leaf drops out of U
        t, s_ = next((t, s_) for t, m in il.u.items() for s_ in m if lv[s_] < lv[t])
        il.u[t] = il.u[t][il.u[t] != s_]
    assert not (_cover(tr, il) == 1).all()


def test_list_geometry():
    x, q = _mixed(2000)[0], 16
    depth = 6
    tr = ad.build_tree(x, q, depth, *DOMAIN)
    il = ad.interaction_lists(tr)
    lv, ix = tr.boxes()
    anc = np.concatenate(tr.level_anchors)
    leaf = np.concatenate(tr.level_leaf)
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    par = np.full(len(lv), -1)
    for l in range(1, depth + 1):
        par[base[l]:base[l + 1]] = base[l - 1] + tr.parent(l)
    unit = lambda b: 1 << (depth - lv[b])
    lo = lambda b: anc[b] * unit(b)
    hi = lambda b: (anc[b] + 1) * unit(b)
    gap = lambda a, b: np.maximum(np.maximum(lo(a) - hi(b), lo(b) - hi(a)), 0).max()
    for t, members in il.u.items():
        assert leaf[t] and t in members
        for s in members:
            assert leaf[s] and gap(t, s) == 0
    for b, members in il.v.items():
        for a in members:
            assert lv[a] == lv[b] and np.abs(anc[a] - anc[b]).max() > 1
            assert np.abs(anc[par[a]] - anc[par[b]]).max() <= 1
    for t, members in il.w.items():
        for a in members:
            assert lv[a] > lv[t] and gap(a, t) >= unit(a) and gap(par[a], t) == 0
            up = anc[a] >> (lv[a] - lv[t])                 # the colleague it descends from
            assert np.abs(up - anc[t]).max() == 1
    pairs_w = {(int(t), int(a)) for t, m in il.w.items() for a in m}
    pairs_x = {(int(s), int(b)) for b, m in il.x.items() for s in m}
    assert pairs_w == pairs_x


def test_fully_refined_tree_is_the_uniform_tree():
    depth, p = 3, 4
    x, qv = _mixed(1500)
    tr = ad.build_tree(x, 0, depth, *DOMAIN)
    ut = otree.build_tree(x, depth, *DOMAIN)
    for l in range(depth + 1):
        assert np.array_equal(tr.level_keys[l], ut.level_keys[l])
        assert tr.level_leaf[l].all() == (l == depth)
    il = ad.interaction_lists(tr)
    assert not any(len(m) for m in il.w.values()) and not il.x
    base = sum(len(tr.level_keys[l]) for l in range(depth))
    uoff, uidx = otree.u_lists(ut)
    for i in range(len(ut.leaf_keys)):
        assert np.array_equal(il.u[base + i] - base, uidx[uoff[i]:uoff[i + 1]])
    phi, g, _, _ = ad.evaluate(x, qv, p, 0, depth, *DOMAIN)
    ref = kifmm.evaluate(x, qv, p, depth, *DOMAIN)
    assert np.linalg.norm(phi - ref.phi) / np.linalg.norm(ref.phi) < 1e-12
    assert np.linalg.norm(g - ref.grad) / np.linalg.norm(ref.grad) < 1e-12


def test_single_leaf_is_the_direct_sum():
    x, qv = _mixed(800)
    phi, g, tr, _ = ad.evaluate(x, qv, 4, len(x), 5, *DOMAIN)
    assert len(tr.level_keys) == 6 and tr.level_leaf[0].all() and sum(map(len, tr.level_keys[1:])) == 0
    ref, gref = direct.direct_numpy(x, x, qv)
    assert np.abs(phi - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.abs(g - gref).max() <= 1e-13 * np.abs(gref).max()


def test_error_falls_with_p(ops6):
    x, qv = _mixed()
    ref, gref = direct.direct_self(x, qv)
    errs = []
    for p in (3, 4, 6):
        phi, g, _, il = ad.evaluate(x, qv, p, 32, 6, *DOMAIN, ops=ops6 if p == 6 else None)
        errs.append((np.linalg.norm(phi - ref) / np.linalg.norm(ref),
                     np.linalg.norm(g - gref) / np.linalg.norm(gref)))
    assert sum(len(m) for m in il.w.values()) > 1000
    assert errs[0][0] > errs[1][0] > errs[2][0] and errs[0][1] > errs[1][1] > errs[2][1]
    assert errs[2][0] < 5e-6 and errs[2][1] < 5e-6


@pytest.mark.parametrize("drop", ["W", "X"])
def test_dropping_an_adaptive_list_is_caught(drop, ops6):
    x, qv = _mixed()
    ref, _ = direct.direct_self(x, qv, gradient=False)
    lists = tuple(c for c in "UVWX" if c != drop)
    phi, _, _, _ = ad.evaluate(x, qv, 6, 32, 6, *DOMAIN, gradient=False, ops=ops6, lists=lists)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) > 1e-2


def test_linear_in_the_charges(ops6):
    x, q1 = _mixed(2000)
    q2 = charges(2000, "normal", seed=7).astype(np.float64)
    f = lambda q: ad.evaluate(x, q, 6, 24, 6, *DOMAIN, gradient=False, ops=ops6)[0]
    a, b = 0.75, -1.5
    lhs, rhs = f(a * q1 + b * q2), a * f(q1) + b * f(q2)
    # exact in exact arithmetic; FP64 rounding is amplified by the pseudo-inverses' condition
    # number (up to ~1e7 at p = 6), so the bound is 1e-10 rather than a few ulps
    assert np.abs(lhs - rhs).max() <= 1e-10 * np.abs(rhs).max()


def test_modified_helmholtz_kernel():
    x, qv = _mixed(2000)
    kappa = 3.0
    ref, gref = direct.direct_self(x, qv, kappa=kappa)
    phi, g, _, _ = ad.evaluate(x, qv, 6, 24, 6, *DOMAIN, kappa=kappa)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-5
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 1e-5


def test_helmholtz_kernel():
    """Complex densities and operators through the same adaptive steps (wavenumber 2)."""
    x = _mixed(2000)[0]
    rng = np.random.default_rng(11)
    qc = rng.uniform(-1, 1, 2000) + 1j * rng.uniform(-1, 1, 2000)
    ref, gref = direct.direct_self(x, qc, wavenumber=2.0)
    phi, g, _, il = ad.evaluate(x, qc, 6, 24, 6, *DOMAIN, wavenumber=2.0)
    assert np.iscomplexobj(phi) and sum(len(m) for m in il.w.values()) > 0
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-5
    assert np.linalg.norm(g - gref) / np.linalg.norm(gref) < 1e-5
