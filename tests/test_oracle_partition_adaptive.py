"""Pins of the local essential trees of an adaptive tree split at d_global (Section 2.3: the
global levels are uniform, the local trees adaptive).  What the paper states about them is
checked member by member: the ghost data that the U, V, W and X lists of a box beta below
d_global need lie within, or overlap, the children of the colleagues of beta's parent; they come
from local trees rooted at boxes adjacent to beta's local root, so each local root talks to at
most 26 others; and every list member is either owned or a ghost."""
import numpy as np
import pytest

from oracle import adaptive as ad, partition as opart
from synth import mixed_points, sphere_points


def _case(name):
    if name == "mixed":
        return mixed_points(3000).astype(np.float64), 24, 6, ((0.0, 0.0, 0.0), 1.0), 2, 8
    return sphere_points(2500).astype(np.float64), 16, 6, ((-1.0, -1.0, -1.0), 2.0), 3, 24


@pytest.mark.parametrize("name", ["mixed", "sphere"])
def test_adaptive_local_essential_trees(name):
    x, q, depth, dom, dg, P = _case(name)
    tr = ad.build_tree(x, q, depth, *dom, min_level=dg)
    il = ad.interaction_lists(tr)
    let = opart.adaptive_let(tr, il, dg, P)
    lv, _ = tr.boxes()
    anc = np.concatenate(tr.level_anchors)
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    par = np.full(len(lv), -1)
    for l in range(1, depth + 1):
        par[base[l]:base[l + 1]] = base[l - 1] + tr.parent(l)
    root, owner = let["root"], let["box_owner"]
    root_anc = tr.level_anchors[dg]
    unit = lambda b: 1 << (depth - lv[b])
    n_s = n_u = 0
    for r, rk in enumerate(let["ranks"]):
        own = set(rk["own"].tolist())
        ghosts = set(rk["ghost_s"].tolist()) | set(rk["ghost_u"].tolist())
        for b in rk["own"]:
            if lv[b] == dg:     # a local root: its V list is the global stage's, and it has no X list
                assert not il.x.get(int(b), [])
                for a in [*il.u.get(int(b), []), *il.w.get(int(b), [])]:
                    assert int(a) in own or int(a) in ghosts
                continue
            P_ = par[b]
            # the children of the colleagues of P(b) (and of P(b) itself): a block of 3 x 3 x 3 boxes
            # of P(b)'s size, in units of the deepest level
            lo = (anc[P_] - 1) * unit(P_)
            hi = (anc[P_] + 2) * unit(P_)
            members = [*il.u.get(int(b), []), *il.v.get(int(b), []), *il.w.get(int(b), []), *il.x.get(int(b), [])]
            for a in members:
                a = int(a)
                assert a in own or a in ghosts                      # every member is owned or a ghost
                a_lo, a_hi = anc[a] * unit(a), (anc[a] + 1) * unit(a)
                assert ((a_lo < hi) & (lo < a_hi)).all(), (b, a)    # within or overlapping the block
                if owner[a] != r:                                   # from an adjacent local root
                    assert np.abs(root_anc[root[a]] - root_anc[root[b]]).max() <= 1
        n_s += len(rk["ghost_s"])
        n_u += len(rk["ghost_u"])
        # each local root talks to the owners of at most its 26 adjacent roots
        for rt in np.nonzero(let["owner"] == r)[0]:
            adj = np.nonzero(np.abs(root_anc - root_anc[rt]).max(axis=1) == 1)[0]
            assert len(adj) <= 26
        allowed = set(let["owner"][np.nonzero((np.abs(root_anc[:, None, :] - root_anc[None, let["owner"] == r, :])
                                                .max(axis=2) <= 1).any(axis=1))[0]].tolist()) - {r}
        assert set(rk["neighbours"]) <= allowed
    assert n_s > 0 and n_u > 0
    # the adaptive lists cross ranks: W members are u ghosts and X members s ghosts somewhere
    cross_w = sum(owner[a] != owner[b] for b, m in il.w.items() if lv[b] >= dg for a in m)
    cross_x = sum(owner[a] != owner[b] for b, m in il.x.items() if lv[b] > dg for a in m)
    assert cross_w > 0 and cross_x > 0


def test_forced_global_levels():
    x, q, depth, dom, dg, _ = _case("mixed")
    tr = ad.build_tree(x, 10 ** 9, depth, *dom, min_level=dg)    # capacity above N: leaves exactly at d_global
    assert all(not tr.level_leaf[l].any() for l in range(dg))
    assert tr.level_leaf[dg].all() and sum(len(k) for k in tr.level_keys[dg + 1:]) == 0
    with pytest.raises(AssertionError):
        opart.adaptive_let(ad.build_tree(x, 10 ** 9, depth, *dom), ad.interaction_lists(ad.build_tree(x, 10 ** 9, depth, *dom)), dg, 4)
