"""The distributed scheme of Section 3 run by real processes over torch.distributed (gloo, CPU),
with the oracle's FP64 kiFMM arithmetic.  Test infrastructure only: the CUDA path never imports
it; the GPU library runs the same scheme on virtual ranks sharing one device.

Every process is one rank and calls `run` with the same inputs.

Setup (Box comm-setup):
  (1) tree: every rank builds the global tree from the same points (the distributed sort of
      step 1 is a startup cost outside the paper's runtime and is not reproduced);
  (2) layout: `oracle.partition.layout`;
  (3, 4) query packets: the interaction-list positions of the rank's boxes below d_global that
      lie in another rank's subdomain (`oracle.partition`'s candidates), sent point-to-point to
      their owners;
  (5) neighbourhoods: the ranks addressed by the packets;
  (6) existence answers from the owners; the U ghost leaves' coordinates and densities follow.
Runtime (Box comm-runtime):
  local stage: S2U and U2U up to the local roots on the rank's own boxes; the V ghosts' u vectors
      from their owners (point-to-point);
  global stage: the local roots' u gathered at rank 0 (a gather of variable counts), U2U, VLI and
      D2D over levels 2..d_global there, the local roots' d scattered back;
  local downward stage: VLI, D2D, D2T and ULI of the rank's boxes below d_global.
The result equals the single-process kiFMM up to the order of floating-point sums.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import direct, kifmm, partition as opart, tree as otree


# ---- messages ---------------------------------------------------------------------------------
def _exchange(send, dtype):
    """Neighbourhood exchange: send[dest] is a 1-D array for rank dest (absent or empty: nothing).
    Returns recv[src] for every rank that sent something.  Counts are all-gathered first."""
    P, me = dist.get_world_size(), dist.get_rank()
    counts = torch.zeros(P, dtype=torch.int64)
    for d, a in send.items():
        counts[d] = len(a)
    table = [torch.zeros(P, dtype=torch.int64) for _ in range(P)]
    dist.all_gather(table, counts)
    reqs, recv = [], {}
    tdt = torch.float64 if dtype == np.float64 else torch.int64
    for src in range(P):
        n = int(table[src][me])
        if src != me and n:
            buf = torch.empty(n, dtype=tdt)
            recv[src] = buf
            reqs.append(dist.irecv(buf, src))
    for d, a in send.items():
        if d != me and len(a):
            reqs.append(dist.isend(torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)), d))
    for r in reqs:
        r.wait()
    return {s: b.numpy() for s, b in recv.items()}


def _gatherv(a):
    """Rows of every rank gathered at rank 0 in rank order (counts vary; padded for the collective)."""
    P, me = dist.get_world_size(), dist.get_rank()
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = torch.tensor([a.size], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(P)]
    dist.all_gather(sizes, n)
    m = max(int(s) for s in sizes)
    buf = torch.zeros(m, dtype=torch.float64)
    buf[:a.size] = torch.from_numpy(a.ravel())
    out = [torch.zeros(m, dtype=torch.float64) for _ in range(P)] if me == 0 else None
    dist.gather(buf, out, dst=0)
    if me != 0:
        return None
    return [out[r][:int(sizes[r])].numpy() for r in range(P)]


def _scatterv(parts, n_mine):
    """parts[r] (at rank 0) to every rank r, which expects n_mine values."""
    P, me = dist.get_world_size(), dist.get_rank()
    sizes = torch.zeros(P, dtype=torch.int64)
    if me == 0:
        sizes = torch.tensor([len(p) for p in parts], dtype=torch.int64)
    dist.broadcast(sizes, 0)
    m = int(sizes.max())
    buf = torch.zeros(m, dtype=torch.float64)
    lst = None
    if me == 0:
        lst = []
        for p in parts:
            t = torch.zeros(m, dtype=torch.float64)
            t[:len(p)] = torch.from_numpy(np.asarray(p, dtype=np.float64))
            lst.append(t)
    dist.scatter(buf, lst, src=0)
    assert int(sizes[me]) == n_mine
    return buf[:n_mine].numpy()


# ---- the scheme -------------------------------------------------------------------------------
def run(points, charges, p, depth, origin, side, d_global, pinv_rtol=kifmm.DEFAULT_PINV_RTOL):
    """This rank's part of the distributed evaluation.  Returns (sorted positions of its points,
    their potentials, their gradients, a dict of setup facts for checking)."""
    P, me = dist.get_world_size(), dist.get_rank()
    xs_in = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    q_in = np.asarray(charges, dtype=np.float64).reshape(-1)
    tr = otree.build_tree(xs_in, depth, origin, side)                       # (1)
    xs, qs = xs_in[tr.perm], q_in[tr.perm]
    ops = kifmm.build_operators(p, tr.side, depth, pinv_rtol)
    ns = kifmm.n_surface(p)
    d, dg = depth, d_global
    first, owner = opart.layout(tr, dg, P)                                  # (2)
    own_of = {lvl: opart._owner_of(tr, dg, owner, tr.level_keys[lvl], lvl) for lvl in range(dg, d + 1)}
    mine = {lvl: np.nonzero(own_of[lvl] == me)[0] for lvl in range(dg, d + 1)}
    facts = {"nb_u": set(), "nb_v": set(), "ghost_v": {}, "ghost_u": None}

    # (3)-(6) query packets, existence answers; what every rank must send at runtime
    def ask(level, cand_fn, nb):
        keys, owners = opart._queries(tr, dg, owner, me, level, tr.level_anchors[level][mine[level]], cand_fn)
        nb.update(owners.tolist())
        got = _exchange({o: keys[owners == o].astype(np.int64) for o in np.unique(owners)}, np.int64)
        my_keys = tr.level_keys[level][mine[level]]
        answer = {s: np.asarray(k, np.uint64)[np.isin(np.asarray(k, np.uint64), my_keys)] for s, k in got.items()}
        back = _exchange({s: a.astype(np.int64) for s, a in answer.items()}, np.int64)
        ghosts = np.sort(np.concatenate([np.asarray(v, np.uint64) for v in back.values()])
                         if back else np.zeros(0, np.uint64))
        # what this rank sends each asker at runtime: its boxes, in the asker's order
        sends = {s: np.searchsorted(tr.level_keys[level], a) for s, a in answer.items()}
        return ghosts, sends

    v_sends = {}
    for level in range(dg + 1, d + 1):
        g, v_sends[level] = ask(level, opart._v_candidates, facts["nb_v"])
        facts["ghost_v"][level] = g
    gu, u_sends = ask(d, opart._u_candidates, facts["nb_u"])
    facts["ghost_u"] = gu

    # U ghosts: the points of the answered leaves (coordinates and densities), from their owners
    def leaf_points(leaves):
        rows = [np.arange(tr.leaf_offsets[a], tr.leaf_offsets[a + 1]) for a in leaves]
        return np.concatenate(rows) if rows else np.zeros(0, np.int64)
    got = _exchange({s: np.concatenate([xs[leaf_points(lv)].ravel(), qs[leaf_points(lv)]])
                     for s, lv in u_sends.items()}, np.float64)
    ghost_pts = {}                       # leaf index -> (points, densities), from the owners' data
    for s, buf in got.items():
        # the answers of owner s are the ghosts whose key s owns, in key order
        lv = np.searchsorted(tr.leaf_keys, np.sort(gu[opart._owner_of(tr, dg, owner, gu, d) == s]))
        cnt = np.diff(tr.leaf_offsets)[lv]
        m = int(cnt.sum())
        x, q = buf[:3 * m].reshape(-1, 3), buf[3 * m:]
        off = np.concatenate([[0], np.cumsum(cnt)])
        for i, a in enumerate(lv):
            ghost_pts[int(a)] = (x[off[i]:off[i + 1]], q[off[i]:off[i + 1]])

    # local stage: S2U on the own leaves, U2U up to the local roots
    u = {lvl: np.zeros((len(tr.level_keys[lvl]), ns)) for lvl in range(dg, d + 1)}
    leaves = mine[d]
    chk = kifmm._leaf_surface_points(tr, p, leaves, kifmm.ALPHA_OUTER)
    t_off = np.arange(len(leaves) + 1, dtype=np.int64) * ns
    ranges = np.stack([tr.leaf_offsets[leaves], tr.leaf_offsets[leaves + 1]], axis=1)
    q_uc, _ = direct.grouped_sum(t_off, chk, np.arange(len(leaves) + 1), ranges, xs, qs, gradient=False)
    u[d][leaves] = q_uc.reshape(len(leaves), ns) @ ops.uc2e[d].T
    for level in range(d - 1, dg - 1, -1):
        ch = tr.children(level)[mine[level]]
        q = np.zeros((len(mine[level]), ns))
        for c in range(8):
            has = ch[:, c] >= 0
            q[has] += u[level + 1][ch[has, c]] @ ops.m2m[(level, c)].T
        u[level][mine[level]] = q @ ops.uc2e[level].T
    # V exchange: the owners send the answered boxes' u
    for level in range(dg + 1, d + 1):
        got = _exchange({s: u[level][b].ravel() for s, b in v_sends[level].items()}, np.float64)
        for s, buf in got.items():
            g = facts["ghost_v"][level]
            keys_s = np.sort(g[opart._owner_of(tr, dg, owner, g, level) == s])
            u[level][np.searchsorted(tr.level_keys[level], keys_s)] = buf.reshape(-1, ns)
    # global stage at rank 0: gather the local roots' u, run levels 2..d_global, scatter d
    roots = mine[dg]
    allu = _gatherv(u[dg][roots])
    dvec = {}
    parts = None
    if me == 0:
        ug = {dg: np.concatenate([a.reshape(-1, ns) for a in allu])}
        for level in range(dg - 1, 1, -1):
            ch = tr.children(level)
            q = np.zeros((len(tr.level_keys[level]), ns))
            for c in range(8):
                has = ch[:, c] >= 0
                q[has] += ug[level + 1][ch[has, c]] @ ops.m2m[(level, c)].T
            ug[level] = q @ ops.uc2e[level].T
        dgl = {}
        for level in range(2, dg + 1):
            boxes = np.arange(len(tr.level_keys[level]))
            dgl[level] = _downward_level(tr, ops, level, boxes, ug[level], dgl.get(level - 1), ns)
        parts = [dgl[dg][first[r]:first[r + 1]].ravel() for r in range(P)]
    dvec[dg] = np.zeros((len(tr.level_keys[dg]), ns))
    dvec[dg][roots] = _scatterv(parts, len(roots) * ns).reshape(-1, ns)
    # local downward stage
    for level in range(dg + 1, d + 1):
        dvec[level] = np.zeros((len(tr.level_keys[level]), ns))
        dvec[level][mine[level]] = _downward_level(tr, ops, level, mine[level], u[level], dvec[level - 1], ns)
    # D2T and ULI at the own points
    t_lo, t_hi = tr.leaf_offsets[leaves[0]], tr.leaf_offsets[leaves[-1] + 1]
    tx = xs[t_lo:t_hi]
    grp = (tr.leaf_offsets[np.append(leaves, leaves[-1] + 1)] - t_lo).astype(np.int64)
    pot, grd = np.zeros(len(tx)), np.zeros((len(tx), 3))
    de = kifmm._leaf_surface_points(tr, p, leaves, kifmm.ALPHA_OUTER)
    rng = np.stack([np.arange(len(leaves)) * ns, np.arange(1, len(leaves) + 1) * ns], 1)
    direct.grouped_sum(grp, tx, np.arange(len(leaves) + 1), rng, de, dvec[d][leaves].reshape(-1), True, pot, grd)
    # sources of the ULI: the own points, then the ghost leaves' points
    src_x, src_q, start = [xs[t_lo:t_hi]], [qs[t_lo:t_hi]], {}
    pos = t_hi - t_lo
    for a in sorted(ghost_pts):
        gx, gq = ghost_pts[a]
        start[a] = (pos, pos + len(gq))
        src_x.append(gx), src_q.append(gq)
        pos += len(gq)
    sx, sq = np.concatenate(src_x), np.concatenate(src_q)
    uoff, uidx = otree.u_lists(tr, leaves)
    r_list = []
    for a in uidx:
        if own_of[d][a] == me:
            r_list.append((tr.leaf_offsets[a] - t_lo, tr.leaf_offsets[a + 1] - t_lo))
        else:
            r_list.append(start[int(a)])
    direct.grouped_sum(grp, tx, uoff, np.asarray(r_list, np.int64).reshape(-1, 2), sx, sq, True, pot, grd)
    facts["nb_u"], facts["nb_v"] = sorted(facts["nb_u"]), sorted(facts["nb_v"])
    return np.arange(t_lo, t_hi), pot, grd, facts, tr


def _downward_level(tr, ops, level, boxes, u_level, d_parent, ns):
    """Closed downward densities of `boxes` at `level`: VLI from u_level, plus D2D from the parent
    densities d_parent (full array of level - 1) when level >= 3."""
    q = np.zeros((len(boxes), ns))
    off, idx, tvec = otree.v_lists(tr, level, boxes)
    rows = np.repeat(np.arange(len(boxes)), np.diff(off))
    for t in np.unique(tvec):
        sel = tvec == t
        q[rows[sel]] += u_level[idx[sel]] @ ops.m2l[(level, int(t))].T
    if level >= 3:
        par = tr.parent(level)[boxes]
        oct_ = (tr.level_keys[level][boxes] & np.uint64(7)).astype(np.int64)
        for c in range(8):
            sel = oct_ == c
            q[sel] += d_parent[par[sel]] @ ops.l2l[(level, c)].T
    return q @ ops.dc2e[level].T


# ---- the scheme over an adaptive tree ---------------------------------------------------------
def run_adaptive(points, charges, p, capacity, depth, origin, side, d_global, pinv_rtol=kifmm.DEFAULT_PINV_RTOL):
    """This rank's part of the distributed evaluation over an adaptive tree (Section 2.3: the
    global levels 0..d_global uniform, the local trees below them adaptive), with the lists and
    arithmetic of oracle.adaptive.  Every rank builds the global tree and lists from the same
    points (as `run` does); the ghosts of its local essential tree (oracle.partition.adaptive_let)
    are requested from their owners and arrive as messages: points and densities for the U and X
    members, upward densities for the V and W members.  Returns (sorted positions of its points,
    their potentials, their gradients, the rank's local essential tree)."""
    from . import adaptive as ad
    P, me = dist.get_world_size(), dist.get_rank()
    xs_in = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    q_in = np.asarray(charges, dtype=np.float64).reshape(-1)
    dg = d_global
    tr = ad.build_tree(xs_in, capacity, depth, origin, side, min_level=dg)
    il = ad.interaction_lists(tr)
    let = opart.adaptive_let(tr, il, dg, P)
    rk = let["ranks"][me]
    owner = let["box_owner"]
    lv, ix = tr.boxes()
    base = np.concatenate([[0], np.cumsum([len(k) for k in tr.level_keys])])
    leaf = np.concatenate(tr.level_leaf)
    keys = np.concatenate(tr.level_keys)
    xs, qs = xs_in[tr.perm], q_in[tr.perm]
    ops = kifmm.build_operators(p, tr.side, depth, pinv_rtol)
    ns = kifmm.n_surface(p)
    rng = {int(b): tr.level_ranges[lv[b]][ix[b]] for b in range(len(lv))}
    own = rk["own"]

    def fetch(ghosts, payload, width):
        """Ghost data from their owners: the requests (box ids) go out, each owner answers with
        the payloads in the order asked; returns box id -> payload."""
        req = {int(o): ghosts[owner[ghosts] == o] for o in np.unique(owner[ghosts])}
        asked = _exchange({o: a.astype(np.int64) for o, a in req.items()}, np.int64)
        reply = _exchange({s: np.concatenate([payload(int(b)) for b in ids]) for s, ids in asked.items()}, np.float64)
        out = {}
        for o, ids in req.items():
            buf, k = reply[o], 0
            for b in ids:
                w = width(int(b))
                out[int(b)] = buf[k:k + w]
                k += w
        return out

    # s ghosts (U and X members): their points and densities
    npts = lambda b: int(rng[b][1] - rng[b][0])
    got = fetch(rk["ghost_s"], lambda b: np.concatenate([xs[rng[b][0]:rng[b][1]].ravel(), qs[rng[b][0]:rng[b][1]]]),
                lambda b: 4 * npts(b))
    src = {b: (v[:3 * npts(b)].reshape(-1, 3), v[3 * npts(b):]) for b, v in got.items()}
    for b in own:
        if leaf[b]:
            src[int(b)] = (xs[rng[int(b)][0]:rng[int(b)][1]], qs[rng[int(b)][0]:rng[int(b)][1]])

    def surface(b, alpha):
        level = lv[b]
        c = tr.centres(level, np.array([ix[b]]))[0]
        return kifmm.surface(p, c, tr.halfwidth(level), alpha)

    def sums(targets, sources):
        """Potential (and gradient) at `targets` of the (points, densities) pairs in `sources`."""
        pot, grd = np.zeros(len(targets)), np.zeros((len(targets), 3))
        for sx, sq in sources:
            direct.grouped_sum([0, len(targets)], targets, [0, 1], [[0, len(sq)]], sx, sq, True, pot, grd)
        return pot, grd

    # local upward stage: S2U at the own leaves, U2U at the own refined boxes, down to the local roots
    u = {}
    for level in range(depth, dg - 1, -1):
        for b in own[lv[own] == level]:
            b = int(b)
            if leaf[b]:
                q_uc = sums(surface(b, kifmm.ALPHA_OUTER), [src[b]])[0]
            else:
                q_uc = np.zeros(ns)
                kids = np.nonzero((lv == level + 1) & ((keys >> np.uint64(3)) == keys[b]))[0]
                for c in kids:
                    q_uc += ops.m2m[(level, int(keys[c] & np.uint64(7)))] @ u[int(c)]
            u[b] = ops.uc2e[level] @ q_uc
    # u ghosts (V and W members), from their owners once they have them
    u.update(fetch(rk["ghost_u"], lambda b: u[b], lambda b: ns))

    # global stage at rank 0: the local roots' u gathered, U2U up to level 2, VLI and D2D down to
    # the local roots, their d scattered back
    roots = own[lv[own] == dg]
    allu = _gatherv(np.concatenate([u[int(b)] for b in roots]) if len(roots) else np.zeros(0))
    dvec = {}
    parts = None
    if me == 0:
        ug = {int(base[dg]) + i: v for i, v in enumerate(np.concatenate(allu).reshape(-1, ns))}
        for level in range(dg - 1, 1, -1):
            for b in range(base[level], base[level + 1]):
                q_uc = np.zeros(ns)
                for c in np.nonzero((lv == level + 1) & ((keys >> np.uint64(3)) == keys[b]))[0]:
                    q_uc += ops.m2m[(level, int(keys[c] & np.uint64(7)))] @ ug[int(c)]
                ug[b] = ops.uc2e[level] @ q_uc
        dgl = {}
        for level in range(2, dg + 1):
            for b in range(base[level], base[level + 1]):
                assert len(il.x.get(b, ())) == 0      # no leaf is coarser than d_global
                dgl[b] = ops.dc2e[level] @ _adaptive_check(tr, ops, il, b, lv, keys, base, ug, dgl, None, ns)
        parts = [np.concatenate([dgl[int(base[dg]) + i] for i in range(let["first_root"][r], let["first_root"][r + 1])]
                                + [np.zeros(0)]) for r in range(P)]
    mine = _scatterv(parts, len(roots) * ns).reshape(-1, ns)
    for i, b in enumerate(roots):
        dvec[int(b)] = mine[i]
    # local downward stage: VLI, XLI and D2D into the own boxes below d_global
    for level in range(dg + 1, depth + 1):
        for b in own[lv[own] == level]:
            b = int(b)
            q_dc = _adaptive_check(tr, ops, il, b, lv, keys, base, u, dvec, (src, surface), ns)
            dvec[b] = ops.dc2e[level] @ q_dc
    # leaf evaluation: D2T, WLI and ULI at the own points
    if len(roots) == 0:   # a rank that owns no local root (more ranks than occupied roots)
        return np.zeros(0, np.int64), np.zeros(0), np.zeros((0, 3)), rk
    lo, hi = rng[int(roots[0])][0], rng[int(roots[-1])][1]
    pot, grd = np.zeros(hi - lo), np.zeros((hi - lo, 3))
    for b in own[leaf[own]]:
        b = int(b)
        t0, t1 = rng[b]
        tx = xs[t0:t1]
        terms = [(surface(b, kifmm.ALPHA_OUTER), dvec[b])]
        terms += [(surface(int(a), kifmm.ALPHA_INNER), u[int(a)]) for a in il.w.get(b, [])]
        terms += [src[int(a)] for a in il.u.get(b, [])]
        ph, gr = sums(tx, terms)
        pot[t0 - lo:t1 - lo], grd[t0 - lo:t1 - lo] = ph, gr
    return np.arange(lo, hi), pot, grd, rk


def _adaptive_check(tr, ops, il, b, lv, keys, base, u, dvec, x_sources, ns):
    """Downward check potentials of box b: VLI from the u of its V list, XLI from the points of
    its X list (x_sources = (sources, surface function) below d_global), D2D from its parent's d."""
    level = int(lv[b])
    anc = tr.level_anchors[level]
    q = np.zeros(ns)
    members = np.asarray(il.v.get(b, ()), np.int64)
    if len(members):
        tvec = otree.transfer_index(anc[members - base[level]] - anc[b - base[level]])
        for a, t in zip(members, tvec):
            q += ops.m2l[(level, int(t))] @ u[int(a)]
    if x_sources is not None and len(il.x.get(b, ())):
        src, surface = x_sources
        dc = surface(b, kifmm.ALPHA_INNER)
        for a in il.x[b]:
            sx, sq = src[int(a)]
            direct.grouped_sum([0, len(dc)], dc, [0, 1], [[0, len(sq)]], sx, sq, False, q, None)
    if level >= 3:
        parent = int(base[level - 1]) + int(np.searchsorted(tr.level_keys[level - 1], keys[b] >> np.uint64(3)))
        q += ops.l2l[(level, int(keys[b] & np.uint64(7)))] @ dvec[parent]
    return q
