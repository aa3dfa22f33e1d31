"""Uniform octree of the oracle: domain, Morton keys, stable sort, leaves, levels, U and V lists.

Definitions followed (Section 2.1 and Table 1 of the paper):
  * the bounding cube is refined uniformly to depth d; level 0 is the root, level d the leaves;
  * boxes are identified by Morton keys, three bits per level, and sorted keys are a pre-order
    traversal of the tree;
  * colleagues C(b) are the boxes adjacent to b at the same level (they share a vertex, edge
    or face);
  * U(b) of a leaf b is its colleagues plus b itself;
  * V(b) holds the boxes at b's level whose parents are colleagues of b's parent and that are
    not adjacent to b.
Only non-empty boxes exist; lists hold non-empty boxes only.

Readings where the paper is silent:
  * domain: origin = per-axis minimum, side = largest extent * (1 + 2^-20) unless the caller
    gives the cube explicitly;
  * anchor of a point: a = min(max(floor((x - origin) * scale), 0), 2^d - 1) with
    scale = 2^d / side, each FP64 operation rounded separately (no fused multiply-add), on
    the exact FP64 value of the FP32 coordinate;
  * Morton interleave puts the x bit first (most significant) in every triple;
  * sort ties keep input order (stable); lists are sorted ascending by Morton key;
  * transfer vector t of a V pair (target b, source a) is the index of a - b (in box units)
    among the 316 vectors of [-3,3]^3 without [-1,1]^3, enumerated with x slowest, z fastest.
"""
from __future__ import annotations

import dataclasses

import numpy as np


def domain_from_points(points):
    """Default bounding cube: (origin[3], side) in FP64."""
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    lo = x.min(axis=0)
    ext = float((x.max(axis=0) - lo).max())
    side = ext * (1.0 + 2.0 ** -20) if ext > 0.0 else 1.0
    return lo, side


def anchors(points, depth, origin, side):
    """Integer box coordinates of each point at the leaf level, int64 (N, 3)."""
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    o = np.asarray(origin, dtype=np.float64).reshape(1, 3)
    scale = np.float64(2.0 ** depth) / np.float64(side)
    t = (x - o) * scale
    a = np.floor(t)
    a = np.clip(a, 0, 2 ** depth - 1)
    return a.astype(np.int64)


def morton(anc, level):
    """Interleave per-axis box coordinates (level bits each) into Morton keys, uint64."""
    a = np.asarray(anc, dtype=np.int64).reshape(-1, 3)
    key = np.zeros(len(a), dtype=np.uint64)
    for b in range(level):
        for axis in range(3):
            bit = ((a[:, axis] >> b) & 1).astype(np.uint64)
            key |= bit << np.uint64(3 * b + (2 - axis))
    return key


def demorton(keys, level):
    """Inverse of `morton`: keys -> int64 (n, 3) box coordinates."""
    k = np.asarray(keys, dtype=np.uint64).reshape(-1)
    a = np.zeros((len(k), 3), dtype=np.int64)
    for b in range(level):
        for axis in range(3):
            bit = ((k >> np.uint64(3 * b + (2 - axis))) & np.uint64(1)).astype(np.int64)
            a[:, axis] |= bit << b
    return a


def transfer_vectors():
    """The 316 M2L transfer vectors [-3,3]^3 minus [-1,1]^3, x slowest, z fastest."""
    out = [(i, j, k) for i in range(-3, 4) for j in range(-3, 4) for k in range(-3, 4)
           if max(abs(i), abs(j), abs(k)) > 1]
    return np.array(out, dtype=np.int64)


def transfer_index(delta):
    """Index in `transfer_vectors()` of each row of delta (int64 (n,3)); -1 if not a transfer."""
    d = np.asarray(delta, dtype=np.int64).reshape(-1, 3)
    table = -np.ones(343, dtype=np.int64)
    tv = transfer_vectors()
    table[(tv[:, 0] + 3) * 49 + (tv[:, 1] + 3) * 7 + (tv[:, 2] + 3)] = np.arange(len(tv))
    ok = (np.abs(d) <= 3).all(axis=1)
    idx = np.where(ok, (d[:, 0] + 3) * 49 + (d[:, 1] + 3) * 7 + (d[:, 2] + 3), 0)
    return np.where(ok, table[idx], -1)


@dataclasses.dataclass
class Tree:
    depth: int
    origin: np.ndarray        # (3,) FP64
    side: float
    keys: np.ndarray          # (N,) uint64 leaf key of each point, input order
    perm: np.ndarray          # (N,) int64: sorted position s holds input point perm[s]
    leaf_offsets: np.ndarray  # (n_leaf+1,) int64 into the sorted points
    level_keys: list          # level_keys[l]: sorted unique uint64 keys of non-empty boxes
    level_anchors: list       # level_anchors[l]: (n_l, 3) int64

    @property
    def leaf_keys(self):
        return self.level_keys[self.depth]

    def halfwidth(self, level):
        return self.side / 2.0 ** (level + 1)

    def centres(self, level, boxes=None):
        """Box centres at `level` (FP64 (n,3)), for all boxes or the given indices."""
        a = self.level_anchors[level] if boxes is None else self.level_anchors[level][boxes]
        w = self.side / 2.0 ** level
        return self.origin[None, :] + (a.astype(np.float64) + 0.5) * w

    def find(self, level, anc):
        """Index of the non-empty box with the given anchors at `level`, or -1."""
        anc = np.asarray(anc, dtype=np.int64).reshape(-1, 3)
        n = 2 ** level
        inside = ((anc >= 0) & (anc < n)).all(axis=1)
        k = morton(np.where(inside[:, None], anc, 0), level)
        keys = self.level_keys[level]
        pos = np.searchsorted(keys, k)
        pos_c = np.minimum(pos, len(keys) - 1)
        hit = inside & (keys[pos_c] == k)
        return np.where(hit, pos_c, -1)

    def parent(self, level):
        """Index (into level-1 boxes) of the parent of every box at `level`."""
        return np.searchsorted(self.level_keys[level - 1], self.level_keys[level] >> np.uint64(3))

    def children(self, level):
        """(n_level, 8) indices into level+1 boxes of each child octant, -1 if empty."""
        a = self.level_anchors[level]
        out = np.empty((len(a), 8), dtype=np.int64)
        for c in range(8):
            off = np.array([(c >> 2) & 1, (c >> 1) & 1, c & 1], dtype=np.int64)
            out[:, c] = self.find(level + 1, 2 * a + off[None, :])
        return out


def build_tree(points, depth, origin=None, side=None):
    """Keys, stable sort and the per-level box sets (steps of Section 2.1)."""
    if origin is None or side is None:
        origin, side = domain_from_points(points)
    origin = np.asarray(origin, dtype=np.float64).reshape(3)
    side = float(side)
    anc = anchors(points, depth, origin, side)
    keys = morton(anc, depth)
    perm = np.argsort(keys, kind="stable")
    sk = keys[perm]
    uniq, first = np.unique(sk, return_index=True)
    leaf_offsets = np.append(first, len(sk)).astype(np.int64)
    level_keys = [None] * (depth + 1)
    level_keys[depth] = uniq
    for level in range(depth - 1, -1, -1):
        level_keys[level] = np.unique(level_keys[level + 1] >> np.uint64(3))
    level_anchors = [demorton(k, level) for level, k in enumerate(level_keys)]
    return Tree(depth, origin, side, keys, perm.astype(np.int64), leaf_offsets,
                level_keys, level_anchors)


def _csr(rows):
    off = np.zeros(len(rows) + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(r) for r in rows])
    idx = np.concatenate(rows).astype(np.int64) if rows else np.zeros(0, np.int64)
    return off, idx


def u_lists(tree, leaves=None):
    """U list of each leaf (all leaves or the given ones): CSR (offsets, idx), idx ascending."""
    d = tree.depth
    boxes = np.arange(len(tree.leaf_keys)) if leaves is None else np.asarray(leaves)
    a = tree.level_anchors[d][boxes]
    cand = []
    for dx in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dz in (-1, 0, 1):
                cand.append(tree.find(d, a + np.array([dx, dy, dz])))
    cand = np.stack(cand, axis=1)                       # (n, 27)
    cand = np.where(cand < 0, np.iinfo(np.int64).max, cand)
    cand.sort(axis=1)                                   # indices ascend with Morton key
    rows = [r[r != np.iinfo(np.int64).max] for r in cand]
    return _csr(rows)


def v_lists(tree, level, boxes=None):
    """V list of each box at `level` >= 2: CSR (offsets, idx, tvec), idx ascending."""
    assert level >= 2
    boxes = np.arange(len(tree.level_keys[level])) if boxes is None else np.asarray(boxes)
    a = tree.level_anchors[level][boxes]
    tv = transfer_vectors()
    big = np.iinfo(np.int64).max
    idx = np.full((len(a), len(tv)), big, dtype=np.int64)
    for t, delta in enumerate(tv):
        src = a + delta[None, :]
        par_ok = (np.abs((src >> 1) - (a >> 1)) <= 1).all(axis=1)
        hit = tree.find(level, src)
        idx[:, t] = np.where(par_ok & (hit >= 0), hit, big)
    order = np.argsort(idx, axis=1, kind="stable")
    idx_sorted = np.take_along_axis(idx, order, axis=1)
    rows, trows = [], []
    for r in range(len(a)):
        keep = idx_sorted[r] != big
        rows.append(idx_sorted[r][keep])
        trows.append(order[r][keep])
    off, flat = _csr(rows)
    tflat = np.concatenate(trows).astype(np.int64) if trows else np.zeros(0, np.int64)
    return off, flat, tflat


def u_lists_bruteforce(tree):
    """U lists straight from the definition, O(n_leaf^2): adjacent-or-self non-empty leaves."""
    a = tree.level_anchors[tree.depth]
    rows = []
    for i in range(len(a)):
        cheb = np.abs(a - a[i]).max(axis=1)
        rows.append(np.nonzero(cheb <= 1)[0])
    return _csr(rows)


def v_lists_bruteforce(tree, level):
    """V lists from the definition: children of the parent's colleagues, not adjacent."""
    a = tree.level_anchors[level]
    pa = tree.level_anchors[level - 1]
    par = tree.parent(level)
    rows, trows = [], []
    for i in range(len(a)):
        colleagues = np.nonzero(np.abs(pa - pa[par[i]]).max(axis=1) == 1)[0]
        cand = np.nonzero(np.isin(par, colleagues))[0]
        cand = cand[np.abs(a[cand] - a[i]).max(axis=1) > 1]
        cand = np.sort(cand)
        rows.append(cand)
        trows.append(transfer_index(a[cand] - a[i]))
    off, flat = _csr(rows)
    return off, flat, (np.concatenate(trows).astype(np.int64) if trows else np.zeros(0, np.int64))
