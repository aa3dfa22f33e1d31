"""Adaptive octree and the adaptive branches of Algorithm 1 (XLI, WLI) in FP64 (the oracle; test
infrastructure only: the CUDA path never imports it).  Its pins are in
tests/test_oracle_adaptive.py.

Definitions followed (Section 2.1 and Algorithm 1 of the paper):
  * adaptive refinement: a box is refined while it holds more than q points, so no leaf holds more
    than q; only non-empty boxes exist;
  * U(b) of a leaf b: every leaf adjacent to b (sharing a vertex, edge or face), at any level,
    and b itself;
  * V(b): the boxes at b's level whose parents are colleagues of b's parent and that are not
    adjacent to b (unchanged from the uniform tree);
  * W(b) of a leaf b: descendants of colleagues of b that are not adjacent to b;
  * X(b): the boxes a whose W list holds b;
  * XLI (step 2b): the sources of every a in X(b) enter b's downward check potentials directly,
    dc_b += K(dc_b, y_a) s_a (the operator Q of Table 1);
  * WLI (step 3a): the upward equivalent densities of every a in W(b) are evaluated at b's targets,
    f_b += K(x_b, ue_a) u_a (the operator R of Table 1);
  * the remaining steps are those of the uniform tree, run over the boxes of every level: S2U at the
    leaves (of any level), U2U at the other boxes, VLI and D2D at every box of level >= 2, D2T
    and ULI at the leaves.

Readings where the paper is silent:
  * W list: Section 2.1 asks for descendants of colleagues that are not adjacent to b; the
    published method it follows (the kiFMM of Ying, Biros and Zorin) keeps only the largest such
    boxes, those whose parent is adjacent to b.  Without that condition a box and its descendants
    would both carry the same sources; the condition is taken;
  * refinement stops at a maximum depth D (leaves at level D may hold more than q points);
  * a leaf at level 0 or 1 has no downward densities (no box at those levels has a V list);
  * keys, anchors and the bounding cube follow the uniform oracle at depth D, so a box at level l
    holds the points whose depth-D key shifted right by 3 (D - l) equals its key.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import direct, kifmm, tree as otree


@dataclasses.dataclass
class AdaptiveTree:
    depth: int                # D: the deepest level a box may have
    capacity: int             # q: a box of level < D with more points than this is refined
    origin: np.ndarray        # (3,) FP64
    side: float
    perm: np.ndarray          # (N,) int64: sorted position s holds input point perm[s]
    level_keys: list          # per level: sorted uint64 keys of the boxes of the tree
    level_anchors: list       # per level: (n_l, 3) int64
    level_ranges: list        # per level: (n_l, 2) int64 [begin, end) into the sorted points
    level_leaf: list          # per level: (n_l,) bool

    def halfwidth(self, level):
        return self.side / 2.0 ** (level + 1)

    def centres(self, level, boxes=None):
        a = self.level_anchors[level] if boxes is None else self.level_anchors[level][boxes]
        w = self.side / 2.0 ** level
        return self.origin[None, :] + (a.astype(np.float64) + 0.5) * w

    def parent(self, level):
        """Index (into level-1 boxes) of the parent of every box at `level`."""
        return np.searchsorted(self.level_keys[level - 1], self.level_keys[level] >> np.uint64(3))

    def boxes(self):
        """Flat table of every box: (level, index in its level), levels ascending."""
        lv = np.concatenate([np.full(len(k), l, np.int64) for l, k in enumerate(self.level_keys)])
        ix = np.concatenate([np.arange(len(k), dtype=np.int64) for k in self.level_keys])
        return lv, ix

    def leaves(self):
        """(level, index) of every leaf, in pre-order (ascending first point)."""
        lv, ix = self.boxes()
        leaf = np.concatenate(self.level_leaf)
        lv, ix = lv[leaf], ix[leaf]
        begin = np.array([self.level_ranges[l][i, 0] for l, i in zip(lv, ix)], np.int64)
        order = np.argsort(begin, kind="stable")
        return lv[order], ix[order]


def build_tree(points, capacity, depth, origin=None, side=None, min_level=0):
    """Refine the bounding cube while a box holds more than `capacity` points, down to `depth`.
    Boxes above `min_level` are refined whatever they hold (the uniform global levels of the
    distributed scheme, Section 2.3)."""
    if origin is None or side is None:
        origin, side = otree.domain_from_points(points)
    origin = np.asarray(origin, dtype=np.float64).reshape(3)
    side = float(side)
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    if len(x) == 0:
        raise ValueError("the adaptive tree needs at least one point")
    keys = otree.morton(otree.anchors(x, depth, origin, side), depth)
    perm = np.argsort(keys, kind="stable")
    sk = keys[perm]
    active = np.ones(len(sk), bool)          # points whose box at the current level is in the tree
    lk, la, lr, ll = [], [], [], []
    for level in range(depth + 1):
        pk = sk >> np.uint64(3 * (depth - level))
        kl = np.unique(pk[active])
        begin = np.searchsorted(pk, kl, side="left")
        end = np.searchsorted(pk, kl, side="right")
        leaf = ((end - begin <= capacity) & (level >= min_level)) | (level == depth)
        for b, e in zip(begin[leaf], end[leaf]):
            active[b:e] = False
        lk.append(kl)
        la.append(otree.demorton(kl, level))
        lr.append(np.stack([begin, end], axis=1).astype(np.int64))
        ll.append(leaf)
    return AdaptiveTree(depth, int(capacity), origin, side, perm.astype(np.int64), lk, la, lr, ll)


def _touch(lo1, hi1, lo2, hi2):
    """Closed cubes intersect (they share at least a vertex), broadcast over rows."""
    return ((lo1 <= hi2) & (lo2 <= hi1)).all(axis=-1)


@dataclasses.dataclass
class Lists:
    """Interaction lists.  Boxes are global ids into the flat table `AdaptiveTree.boxes()`."""
    u: dict      # leaf id -> sorted array of leaf ids
    v: dict      # box id -> sorted array of box ids (same level)
    w: dict      # leaf id -> sorted array of box ids
    x: dict      # box id -> sorted array of leaf ids


def interaction_lists(tr):
    """U, V, W and X lists straight from their definitions (brute force over all boxes)."""
    lv, ix = tr.boxes()
    anc = np.concatenate(tr.level_anchors)
    s = (1 << (tr.depth - lv))[:, None]
    lo, hi = anc * s, (anc + 1) * s
    leaf = np.concatenate(tr.level_leaf)
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    par = np.full(len(lv), -1, np.int64)
    for level in range(1, tr.depth + 1):
        par[base[level]:base[level + 1]] = base[level - 1] + tr.parent(level)
    keys = np.concatenate(tr.level_keys)
    leaves = np.nonzero(leaf)[0]
    u, v, w = {}, {}, {}
    for b in range(len(lv)):
        same = np.nonzero(lv == lv[b])[0]
        cheb = np.abs(anc[same] - anc[b]).max(axis=1)
        if lv[b] >= 2:
            pcheb = np.abs((anc[same] >> 1) - (anc[b] >> 1)).max(axis=1)
            v[b] = np.sort(same[(pcheb <= 1) & (cheb > 1)])
        if not leaf[b]:
            continue
        u[b] = np.sort(leaves[_touch(lo[leaves], hi[leaves], lo[b], hi[b])])
        # W: deeper boxes whose ancestor at b's level is a colleague of b, not adjacent to b,
        # with a parent adjacent to b.
        deeper = np.nonzero(lv > lv[b])[0]
        shift = (np.uint64(3) * (lv[deeper] - lv[b]).astype(np.uint64))
        up = otree.demorton(keys[deeper] >> shift, int(lv[b]))
        colleague = np.abs(up - anc[b]).max(axis=1) == 1
        keep = colleague & ~_touch(lo[deeper], hi[deeper], lo[b], hi[b])
        keep &= _touch(lo[par[deeper]], hi[par[deeper]], lo[b], hi[b])
        w[b] = np.sort(deeper[keep])
    x = {}
    for b, members in w.items():
        for a in members:
            x.setdefault(int(a), []).append(b)
    x = {a: np.sort(np.asarray(m, np.int64)) for a, m in x.items()}
    return Lists(u, v, w, x)


def _surfaces(tr, level, boxes, p, alpha):
    c = tr.centres(level, boxes)
    return (c[:, None, :] + alpha * tr.halfwidth(level) * kifmm.surface_grid(p)[None, :, :]).reshape(-1, 3)


def evaluate(points, charges, p, capacity, depth, origin=None, side=None, gradient=True,
             pinv_rtol=kifmm.DEFAULT_PINV_RTOL, ops=None, kappa=0.0, wavenumber=0.0,
             lists=("U", "V", "W", "X"), min_level=0):
    """FP64 adaptive kiFMM field at every point (input order): Algorithm 1 with its adaptive
    branches.  `lists` selects which interaction lists contribute (all four by default);
    `min_level` as in build_tree."""
    xs_in = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    tr = build_tree(xs_in, capacity, depth, origin, side, min_level)
    il = interaction_lists(tr)
    if ops is None:
        ops = kifmm.build_operators(p, tr.side, depth, pinv_rtol, kappa=kappa, wavenumber=wavenumber)
    kappa, wavenumber, dt = ops.kappa, ops.wavenumber, ops.dtype
    ns = kifmm.n_surface(p)
    n = len(xs_in)
    xs = xs_in[tr.perm]
    qs = np.asarray(charges, dtype=dt).reshape(-1)[tr.perm]
    lv, ix = tr.boxes()
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    sums = lambda *a, **k: direct.grouped_sum(*a, kappa=kappa, wavenumber=wavenumber, **k)

    # Upward pass (step 1): S2U at the leaves, U2U at the other boxes, levels D .. 2.
    u = {level: np.zeros((len(tr.level_keys[level]), ns), dt) for level in range(2, depth + 1)}
    for level in range(depth, 1, -1):
        leaf = tr.level_leaf[level]
        q_uc = np.zeros((len(leaf), ns), dt)
        lb = np.nonzero(leaf)[0]
        if len(lb):
            chk = _surfaces(tr, level, lb, p, kifmm.ALPHA_OUTER)
            q, _ = sums(np.arange(len(lb) + 1) * ns, chk, np.arange(len(lb) + 1),
                        tr.level_ranges[level][lb], xs, qs, gradient=False)
            q_uc[lb] = q.reshape(len(lb), ns)
        if level < depth:
            par = tr.parent(level + 1)
            oct_ = (tr.level_keys[level + 1] & np.uint64(7)).astype(np.int64)
            for c in range(8):
                sel = oct_ == c
                np.add.at(q_uc, par[sel], u[level + 1][sel] @ ops.m2m[(level, c)].T)
        u[level] = q_uc @ ops.uc2e[level].T

    # Downward pass (step 2): VLI, XLI and D2D into the check potentials of every box of level >= 2.
    dvec = {}
    for level in range(2, depth + 1):
        nb = len(tr.level_keys[level])
        q_dc = np.zeros((nb, ns), dt)
        if "V" in lists:
            ids = np.arange(nb) + base[level]
            members = [il.v[int(b)] for b in ids]
            rows = np.repeat(np.arange(nb), [len(m) for m in members])
            if len(rows):
                idx = np.concatenate(members) - base[level]
                anc = tr.level_anchors[level]
                tvec = otree.transfer_index(anc[idx] - anc[rows])
                assert (tvec >= 0).all()
                for t in np.unique(tvec):
                    sel = tvec == t
                    q_dc[rows[sel]] += u[level][idx[sel]] @ ops.m2l[(level, int(t))].T
        if "X" in lists:
            tb = [b for b in range(nb) if int(base[level] + b) in il.x]
            if tb:
                members = [il.x[int(base[level] + b)] for b in tb]
                r_off = np.concatenate([[0], np.cumsum([len(m) for m in members])])
                src = np.concatenate(members)
                ranges = np.stack([tr.level_ranges[lv[a]][ix[a]] for a in src])
                q, _ = sums(np.arange(len(tb) + 1) * ns, _surfaces(tr, level, np.asarray(tb), p, kifmm.ALPHA_INNER),
                            r_off, ranges, xs, qs, gradient=False)
                q_dc[tb] += q.reshape(len(tb), ns)
        if level >= 3:
            par = tr.parent(level)
            oct_ = (tr.level_keys[level] & np.uint64(7)).astype(np.int64)
            for c in range(8):
                sel = oct_ == c
                q_dc[sel] += dvec[level - 1][par[sel]] @ ops.l2l[(level, c)].T
        dvec[level] = q_dc @ ops.dc2e[level].T

    # Leaf evaluation (step 3): D2T, WLI and ULI at every leaf's targets.
    leaf_lv, leaf_ix = tr.leaves()
    leaf_id = base[leaf_lv] + leaf_ix
    t_off = np.append([tr.level_ranges[l][i, 0] for l, i in zip(leaf_lv, leaf_ix)], n).astype(np.int64)
    pot = np.zeros(n, dt)
    grd = np.zeros((n, 3), dt) if gradient else None
    # D2T: every leaf of level >= 2 against its own downward equivalent surface.
    deep = leaf_lv >= 2
    if deep.any():
        de = np.concatenate([_surfaces(tr, l, np.array([i]), p, kifmm.ALPHA_OUTER)
                             for l, i in zip(leaf_lv[deep], leaf_ix[deep])])
        dens = np.concatenate([dvec[l][i] for l, i in zip(leaf_lv[deep], leaf_ix[deep])])
        k = np.arange(int(deep.sum()))
        ranges = np.stack([k * ns, (k + 1) * ns], axis=1)
        r_off = np.concatenate([[0], np.cumsum(deep)])
        sums(t_off, xs, r_off, ranges, de, dens, gradient, pot, grd)
    # WLI: upward equivalent surfaces of every box of level >= 2 as one source array.
    if "W" in lists:
        ue = np.concatenate([_surfaces(tr, level, np.arange(len(tr.level_keys[level])), p, kifmm.ALPHA_INNER)
                             for level in range(2, depth + 1)]) if depth >= 2 else np.zeros((0, 3))
        uden = np.concatenate([u[level].reshape(-1) for level in range(2, depth + 1)]) if depth >= 2 \
            else np.zeros(0, dt)
        members = [il.w[int(b)] for b in leaf_id]
        r_off = np.concatenate([[0], np.cumsum([len(m) for m in members])])
        if r_off[-1]:
            src = np.concatenate(members) - base[2]
            assert (src >= 0).all()            # W members lie at level 2 or deeper
            ranges = np.stack([src * ns, (src + 1) * ns], axis=1)
            sums(t_off, xs, r_off, ranges, ue, uden, gradient, pot, grd)
    # ULI: every adjacent leaf's points (the pair at distance zero is skipped).
    if "U" in lists:
        members = [il.u[int(b)] for b in leaf_id]
        r_off = np.concatenate([[0], np.cumsum([len(m) for m in members])])
        src = np.concatenate(members)
        ranges = np.stack([tr.level_ranges[lv[a]][ix[a]] for a in src])
        sums(t_off, xs, r_off, ranges, xs, qs, gradient, pot, grd)

    phi = np.empty(n, dt)
    phi[tr.perm] = pot
    grad = None
    if gradient:
        grad = np.empty((n, 3), dt)
        grad[tr.perm] = grd
    return phi, grad, tr, il
