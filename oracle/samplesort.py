"""Step (1) of the distributed setup (Section 3, Box comm-setup, tree construction; Section 2.3,
distributed sorting and load balancing): a sample sort of the points by their coarse Morton keys
over torch.distributed ranks (gloo, CPU).  Test infrastructure only: the CUDA path never imports
it; on one GPU the whole sort is the library's radix sort.

Every rank holds a slice of the input points.  It computes their Morton keys at the leaf depth d
and at d_global (the local roots' level), draws b of its coarse keys at random, and sends them to
rank 0.  Rank 0 sorts the samples and takes the P - 1 splitters at the P-quantiles of them, which
every rank receives.  A point goes to the bucket (rank) whose splitter range holds its coarse key,
so all points of one local root land on one rank.  The buckets are exchanged all-to-all and every
rank sorts its bucket by (leaf key, input index).  Concatenated in rank order the buckets are the
stable global sort by leaf key.

Readings where the paper is silent:
  * the b samples of a rank are drawn without replacement (all of its keys if it holds fewer);
  * with m samples in all, splitter k (k = 1 .. P - 1) is the sample of 0-based rank floor(k m / P)
    in ascending order (m = P b when every rank holds at least b points; a rank holding fewer sends
    all of its keys, and the quantiles then follow the samples actually drawn), and a key equal to a
    splitter goes to the higher bucket: bucket(key) = number of splitters <= key;
  * ties between equal leaf keys keep the input order (as the single-process sort does).
"""
from __future__ import annotations

import numpy as np
import torch
import torch.distributed as dist

from . import tree as otree
from .distributed import _exchange, _gatherv


def samplesort(points, index, depth, d_global, origin, side, b, seed=0):
    """This rank's bucket after the sort.  points: (n, 3) of this rank's slice, index: their input
    indices.  Returns (input indices, leaf keys, points) of the bucket in sorted order, and the
    splitters."""
    P, me = dist.get_world_size(), dist.get_rank()
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    idx = np.asarray(index, dtype=np.int64)
    leaf = otree.morton(otree.anchors(x, depth, origin, side), depth)
    coarse = leaf >> np.uint64(3 * (depth - d_global))
    # samples at rank 0, splitters back to everyone
    rng = np.random.default_rng(seed * 1000003 + me)
    take = rng.choice(len(coarse), size=min(b, len(coarse)), replace=False) if len(coarse) else np.zeros(0, np.int64)
    gathered = _gatherv(coarse[take].astype(np.float64))
    spl = torch.zeros(max(P - 1, 0), dtype=torch.float64)
    if me == 0:
        samples = np.sort(np.concatenate(gathered))
        for k in range(1, P):
            spl[k - 1] = float(samples[(k * len(samples)) // P]) if len(samples) else 0.0
    if P > 1:
        dist.broadcast(spl, 0)
    splitters = spl.numpy().astype(np.uint64)
    # buckets, all-to-all, local sort
    bucket = np.searchsorted(splitters, coarse, side="right")
    send = {}
    for r in range(P):
        sel = bucket == r
        send[r] = np.concatenate([idx[sel].astype(np.float64), x[sel].ravel()])
    got = _exchange(send, np.float64)
    got[me] = send[me]
    parts_i, parts_x = [], []
    for r in range(P):
        buf = got.get(r, np.zeros(0))
        m = len(buf) // 4
        parts_i.append(buf[:m].astype(np.int64))
        parts_x.append(buf[m:].reshape(-1, 3))
    bi, bx = np.concatenate(parts_i), np.concatenate(parts_x)
    bk = otree.morton(otree.anchors(bx, depth, origin, side), depth)
    order = np.lexsort((bi, bk))
    return bi[order], bk[order], bx[order], splitters
