"""Partition of the uniform tree over P ranks (Section 3, Box comm-setup), written from its
definitions.  Test infrastructure only: the CUDA path never imports it.

What it computes, for a tree split at depth d_global (its level-d_global boxes are the local
roots) and P ranks:
  * the layout (step 2): the owner rank of every local root;
  * the local essential tree of every rank (Eq. 3) in its local part: the union, over the rank's
    boxes below d_global (its leaves L_r and their ancestors inside the local trees), of their
    interaction lists (U for the leaves, V at every level); the members it does not own are its
    ghosts.  Levels 0..d_global belong to the global stage;
  * the query packets (steps 3-4): every position of an interaction list (U: the 26 neighbours of
    an own leaf; V: the children of the parent's colleagues that are not adjacent to the box) that
    lies in the domain, inside the local root of another rank, whether or not a box exists there;
  * the neighbourhoods (step 5): the ranks a rank's U and V packets address;
  * the existence answers (step 6): the queried positions that hold a box.

`adaptive_let` gives the same split for an adaptive tree (Section 2.3: the global levels are
uniform, the local trees adaptive), with the U, V, W and X lists of oracle.adaptive.

Readings where the paper is silent or leaves a choice:
  * layout: contiguous runs of local roots in Morton order, balanced by point counts: rank r
    starts at the first root i whose preceding roots hold at least ceil(r N / P) points, kept at
    least one root past rank r - 1's start and leaving one root for every later rank.  The paper
    balances by sampled sort splitters; this rule is exact and deterministic.
  * the query of a position counts once per rank (a position several own boxes need is asked
    once).
"""
from __future__ import annotations

import math

import numpy as np

from . import tree as otree


def layout(tr, d_global, n_ranks):
    """(first_root[P + 1], owner[n_roots]) of the local roots at d_global."""
    d = tr.depth
    roots = tr.level_keys[d_global]
    leaf_root = tr.leaf_keys >> np.uint64(3 * (d - d_global))
    counts = np.diff(tr.leaf_offsets)
    pts = np.zeros(len(roots), np.int64)
    np.add.at(pts, np.searchsorted(roots, leaf_root), counts)
    return layout_from_counts(pts, n_ranks)


def layout_from_counts(pts, n_ranks):
    """The layout rule over local roots holding pts[i] points each (Morton order)."""
    prefix = np.concatenate([[0], np.cumsum(pts)])
    n = int(prefix[-1])
    first = [0]
    for r in range(1, n_ranks):
        target = math.ceil(n * r / n_ranks)
        i = int(np.searchsorted(prefix, target, side="left"))
        i = max(i, first[-1] + 1)
        i = min(i, len(pts) - (n_ranks - r))
        first.append(i)
    first.append(len(pts))
    owner = np.zeros(len(pts), np.int64)
    for r in range(n_ranks):
        owner[first[r]:first[r + 1]] = r
    return np.asarray(first, np.int64), owner


def adaptive_let(tr, il, d_global, n_ranks):
    """Local essential trees of an adaptive tree split at d_global (every box above d_global
    refined, so the local roots are the boxes of level d_global): per rank, its own boxes and the
    ghosts its U, V, W and X lists name.  U and X members carry source points and densities (s
    ghosts); V and W members carry upward densities (u ghosts).  Boxes are global ids of
    `AdaptiveTree.boxes()`; `tr` and `il` come from oracle.adaptive."""
    lv, ix = tr.boxes()
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    keys = np.concatenate(tr.level_keys)
    assert all(not tr.level_leaf[l].any() for l in range(d_global)), "levels above d_global must be refined"
    counts = np.diff(tr.level_ranges[d_global], axis=1)[:, 0]
    first, owner = layout_from_counts(counts, n_ranks)
    root = np.full(len(lv), -1, np.int64)          # local root (index at d_global) of every box
    deep = lv >= d_global
    root[deep] = np.searchsorted(tr.level_keys[d_global],
                                 keys[deep] >> (np.uint64(3) * (lv[deep] - d_global).astype(np.uint64)))
    box_owner = np.where(deep, owner[np.maximum(root, 0)], -1)
    out = {"first_root": first, "owner": owner, "root": root, "box_owner": box_owner, "ranks": []}
    for r in range(n_ranks):
        # own: the rank's local roots and everything below them.  The leaves' U and W lists are
        # local work at every level; V and X below d_global (the V lists of level d_global belong
        # to the global stage, and a local root has no X list: X members are coarser than it)
        own = np.nonzero((box_owner == r) & (lv >= d_global))[0]
        need_s, need_u = set(), set()
        for b in own:
            need_s.update(il.u.get(int(b), []))
            need_u.update(il.w.get(int(b), []))
            if lv[b] > d_global:
                need_s.update(il.x.get(int(b), []))
                need_u.update(il.v.get(int(b), []))
        ghost_s = np.array(sorted(a for a in need_s if box_owner[a] != r), np.int64)
        ghost_u = np.array(sorted(a for a in need_u if box_owner[a] != r), np.int64)
        nb = sorted(set(box_owner[ghost_s].tolist()) | set(box_owner[ghost_u].tolist()))
        out["ranks"].append({"own": own, "ghost_s": ghost_s, "ghost_u": ghost_u, "neighbours": nb})
    return out


def message_bytes(n_roots, p, bits):
    """Bytes of the u (or d) vectors of n_roots local roots at expansion order p and precision
    `bits` (Section 4, global portion): n_P (6 (p - 1)^2 + 2) b / 8."""
    return n_roots * (6 * (p - 1) ** 2 + 2) * bits // 8


def _owner_of(tr, d_global, owner, keys, level):
    """Owner rank of the local root containing each key at `level`, -1 where no root exists."""
    roots = tr.level_keys[d_global]
    rk = keys >> np.uint64(3 * (level - d_global))
    pos = np.minimum(np.searchsorted(roots, rk), len(roots) - 1)
    return np.where(roots[pos] == rk, owner[pos], -1)


def _v_candidates(anc):
    """Positions of the V list of boxes with anchors `anc`: the children of the colleagues of
    the parent (and of the parent itself) that are not adjacent to the box; (n, 216) anchors
    with a validity mask (adjacent ones masked out)."""
    pa = anc >> 1
    cand = []
    for px in (-1, 0, 1):
        for py in (-1, 0, 1):
            for pz in (-1, 0, 1):
                for c in range(8):
                    off = np.array([(c >> 2) & 1, (c >> 1) & 1, c & 1])
                    cand.append(2 * (pa + np.array([px, py, pz])) + off)
    cand = np.stack(cand, axis=1)                            # (n, 216, 3)
    far = np.abs(cand - anc[:, None, :]).max(axis=2) > 1
    return cand, far


def _u_candidates(anc):
    cand = [anc + np.array([dx, dy, dz]) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)
            if dx or dy or dz]
    return np.stack(cand, axis=1), np.ones((len(anc), 26), bool)


def _queries(tr, d_global, owner, r, level, anc, cand_fn):
    """Unique queried keys of rank r at `level` and their owners."""
    cand, ok = cand_fn(anc)
    m = 2 ** level
    ok = ok & ((cand >= 0) & (cand < m)).all(axis=2)
    c = cand[ok]
    if len(c) == 0:
        return np.zeros(0, np.uint64), np.zeros(0, np.int64)
    keys = np.unique(otree.morton(c, level))
    own = _owner_of(tr, d_global, owner, keys, level)
    sel = (own >= 0) & (own != r)
    return keys[sel], own[sel]


def partition(tr, d_global, n_ranks):
    """Per rank: own keys per level, ghosts (V per level, U), query sizes, neighbourhoods."""
    d = tr.depth
    first, owner = layout(tr, d_global, n_ranks)
    out = {"first_root": first, "owner": owner, "ranks": []}
    level_owner = {l: _owner_of(tr, d_global, owner, tr.level_keys[l], l) for l in range(d_global, d + 1)}
    for r in range(n_ranks):
        rk = {"own": {}, "ghost_v": {}, "ghost_v_eq3": {}, "n_query_v": 0, "nb_v": set(), "nb_u": set()}
        for level in range(d_global, d + 1):
            rk["own"][level] = tr.level_keys[level][level_owner[level] == r]
        for level in range(d_global + 1, d + 1):
            boxes = np.nonzero(level_owner[level] == r)[0]
            # existence answers to the V packets
            qk, qo = _queries(tr, d_global, owner, r, level, tr.level_anchors[level][boxes], _v_candidates)
            rk["n_query_v"] += len(qk)
            rk["nb_v"].update(qo.tolist())
            exists = np.isin(qk, tr.level_keys[level])
            rk["ghost_v"][level] = np.sort(qk[exists])
            # Eq. 3: the members of the own boxes' V lists not owned by r
            _, idx, _ = otree.v_lists(tr, level, boxes)
            members = np.unique(idx)
            rk["ghost_v_eq3"][level] = tr.level_keys[level][members[level_owner[level][members] != r]]
        leaves = np.nonzero(level_owner[d] == r)[0]
        qk, qo = _queries(tr, d_global, owner, r, d, tr.level_anchors[d][leaves], _u_candidates)
        rk["n_query_u"] = len(qk)
        rk["nb_u"].update(qo.tolist())
        rk["ghost_u"] = np.sort(qk[np.isin(qk, tr.level_keys[d])])
        _, idx = otree.u_lists(tr, leaves)
        members = np.unique(idx)
        rk["ghost_u_eq3"] = tr.level_keys[d][members[level_owner[d][members] != r]]
        rk["nb_u"] = sorted(rk["nb_u"])
        rk["nb_v"] = sorted(rk["nb_v"])
        lo, hi = tr.leaf_offsets[leaves[0]], tr.leaf_offsets[leaves[-1] + 1]
        rk["points"] = (int(lo), int(hi - lo))
        rk["n_ghost_points"] = int(sum(np.diff(tr.leaf_offsets)[np.searchsorted(tr.leaf_keys, rk["ghost_u"])]))
        out["ranks"].append(rk)
    return out
