"""Textbook kernel-independent FMM in FP64 (the oracle; test infrastructure only).

Follows Algorithm 1 of the paper (uniform branches only: S2U, U2U, VLI, D2D, D2T, ULI) with
the operators of the algebraic kiFMM the paper's software uses (Section 2.1): every box
carries equivalent densities on a cube surface, obtained by matching potentials on a check
surface through a pseudo-inverse.

Surface construction (not printed in the paper; the published kiFMM method):
  * a surface of order p around a box with centre c and half-width r is the set of grid points
    c + alpha * r * (2 * idx / (p - 1) - 1), idx in {0..p-1}^3 with at least one index equal to
    0 or p-1, taken in lexicographic order; it has 6(p-1)^2 + 2 points (Section 4, global
    portion);
  * alpha = 1.05 for the upward-equivalent and downward-check surfaces, alpha = 2.95 for the
    upward-check and downward-equivalent surfaces.

Operators (Table 1), all built from the actual box sizes of each level:
  S2U   u_b  = pinv(K(uc_b, ue_b)) K(uc_b, y_b) s_b
  U2U   u_P  = pinv(K(uc_P, ue_P)) sum_c K(uc_P, ue_c) u_c
  VLI   dc_b += sum_{a in V(b)} K(dc_b, ue_a) u_a        (Algorithm 1 prints u_b; read as u_a)
  D2D   dc_b += K(dc_b, de_P) d_P
        d_b  = pinv(K(dc_b, de_b)) dc_b                  (once all contributions are summed)
  D2T   f_i += K(x_i, de_b) d_b
  ULI   f_i += sum_{a in U(b)} sum_{j in a, j != i} K(x_i, y_j) s_j
The VLI sum is evaluated one transfer vector at a time, using that interactions sharing a
transfer vector share one operator (Section 2.2); `m2l="pairwise"` instead builds every
pair's matrix from the two boxes' own coordinates (slow; used to pin the grouped form), and
`m2l="fft"` evaluates each transfer vector's M2L as a lattice convolution by FFT (fft_m2l; it
needs operators built with the lattice radius as `alpha_inner`).
The M2L is not compressed here, so the GPU path's SVD truncation error is inside the budget.

With `kappa` > 0 every K above is the modified Helmholtz (Yukawa) kernel
exp(-kappa r) / (4 pi r), a real kernel admitted by Eq. 1; the steps are unchanged, which is what
makes the method kernel-independent (Section 2.1).  That kernel is not homogeneous, so its
operators of different levels are not rescalings of one another.  With `wavenumber` k > 0 every
K is the Helmholtz kernel exp(i k r) / (4 pi r) (Eq. 1 with F = C): operators, densities and
fields are complex and the pseudo-inverse uses the conjugate transpose; the adjoint is for real
kernels only.

The pseudo-inverse truncates singular values below rtol * sigma_max (the paper is silent on
regularisation).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import direct, tree as otree

INV4PI = 1.0 / (4.0 * np.pi)
ALPHA_INNER = 1.05
ALPHA_OUTER = 2.95
DEFAULT_PINV_RTOL = 1e-7


def n_surface(p):
    """Points on a surface of order p: p^3 - (p-2)^3 = 6(p-1)^2 + 2."""
    return 6 * (p - 1) ** 2 + 2


def surface_grid(p):
    """Unit surface grid in [-1,1]^3, shape (n_surface(p), 3), lexicographic (i, j, k)."""
    if p < 2:
        raise ValueError("expansion order p must be >= 2")
    pts = [(i, j, k) for i in range(p) for j in range(p) for k in range(p)
           if min(i, j, k) == 0 or max(i, j, k) == p - 1]
    return 2.0 * np.array(pts, dtype=np.float64) / (p - 1) - 1.0


def surface(p, centre, halfwidth, alpha):
    return np.asarray(centre, dtype=np.float64).reshape(1, 3) + alpha * halfwidth * surface_grid(p)


def kernel_matrix(x, y, kappa=0.0, wavenumber=0.0):
    """K(x_i, y_j) = exp(-kappa r) / (4 pi r), r = |x_i - y_j| (kappa = 0: Eq. 2 normalised;
    kappa > 0: the modified Helmholtz kernel), or exp(i k r) / (4 pi r) for wavenumber k > 0 (the
    Helmholtz kernel, complex), zero where r = 0."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    y = np.asarray(y, dtype=np.float64).reshape(-1, 3)
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    rs = np.where(r > 0.0, r, 1.0)
    if wavenumber > 0.0:
        return np.where(r > 0.0, INV4PI * np.exp(1j * wavenumber * r) / rs, 0.0)
    return np.where(r > 0.0, INV4PI * np.exp(-kappa * r) / rs, 0.0)


def pinv(a, rtol):
    """Truncated-SVD pseudo-inverse: singular values below rtol * sigma_max are dropped."""
    u, s, vt = np.linalg.svd(a)
    keep = s >= rtol * s[0]
    return (vt[keep].conj().T / s[keep]) @ u[:, keep].conj().T


@dataclasses.dataclass
class Operators:
    """Per-level FP64 operators built from actual box geometry (no homogeneity scaling)."""

    p: int
    uc2e: dict        # level -> pinv(K(uc, ue))
    dc2e: dict        # level -> pinv(K(dc, de))
    m2m: dict         # (parent level, octant) -> K(uc_P, ue_child)
    l2l: dict         # (child level, octant) -> K(dc_child, de_P)
    m2l: dict         # (level, t) -> K(dc_b, ue_{b + t})
    kappa: float = 0.0  # kernel: 0 Laplace, > 0 modified Helmholtz exp(-kappa r) / (4 pi r)
    wavenumber: float = 0.0   # > 0: Helmholtz exp(i k r) / (4 pi r), complex operators and data
    alpha_inner: float = ALPHA_INNER   # radius of the upward-equivalent and downward-check surfaces

    @property
    def dtype(self):
        return np.complex128 if self.wavenumber > 0.0 else np.float64


def child_offset(c):
    """Octant c -> (bx, by, bz), x bit most significant (Morton order)."""
    return np.array([(c >> 2) & 1, (c >> 1) & 1, c & 1], dtype=np.float64)


def build_operators(p, side, depth, rtol=DEFAULT_PINV_RTOL, m2l_levels=None, kappa=0.0, wavenumber=0.0,
                    alpha_inner=ALPHA_INNER):
    """Operators of every level.  `alpha_inner` moves the upward-equivalent and downward-check
    surfaces (1.05 by default; the FFT form of the M2L needs the lattice radius of fft_m2l)."""
    tv = otree.transfer_vectors()
    ops = Operators(p, {}, {}, {}, {}, {}, kappa, wavenumber, alpha_inner)
    km = lambda a, b: kernel_matrix(a, b, kappa, wavenumber)
    zero = np.zeros(3)
    for level in range(0, depth + 1):
        r = side / 2.0 ** (level + 1)
        ops.uc2e[level] = pinv(km(surface(p, zero, r, ALPHA_OUTER),
                                             surface(p, zero, r, alpha_inner)), rtol)
        ops.dc2e[level] = pinv(km(surface(p, zero, r, alpha_inner),
                                             surface(p, zero, r, ALPHA_OUTER)), rtol)
    for level in range(0, depth):
        r_p, r_c = side / 2.0 ** (level + 1), side / 2.0 ** (level + 2)
        for c in range(8):
            cc = (2.0 * child_offset(c) - 1.0) * r_c          # child centre relative to parent
            ops.m2m[(level, c)] = km(surface(p, zero, r_p, ALPHA_OUTER),
                                                surface(p, cc, r_c, alpha_inner))
            ops.l2l[(level + 1, c)] = km(surface(p, cc, r_c, alpha_inner),
                                                    surface(p, zero, r_p, ALPHA_OUTER))
    for level in (range(2, depth + 1) if m2l_levels is None else m2l_levels):
        r = side / 2.0 ** (level + 1)
        tgt = surface(p, zero, r, alpha_inner)
        for t, delta in enumerate(tv):
            ops.m2l[(level, t)] = km(tgt, surface(p, 2.0 * r * delta, r, alpha_inner))
    return ops


@dataclasses.dataclass
class Result:
    phi: np.ndarray               # (N,) or (len(sample),) potentials, input order
    grad: np.ndarray | None       # (N,3) or None
    tree: otree.Tree
    u: dict                       # level -> (n_l, n_s) upward equivalent densities
    need: dict                    # level -> sorted box indices whose d was computed
    d: dict                       # level -> (len(need[level]), n_s) downward densities


def _leaf_surface_points(tr, p, leaves, alpha):
    c = tr.centres(tr.depth, leaves)
    r = tr.halfwidth(tr.depth)
    return (c[:, None, :] + alpha * r * surface_grid(p)[None, :, :]).reshape(-1, 3)


def upward(tr, xs, qs, ops, chunk=65536):
    """S2U at every leaf, then U2U level by level up to level 2 (Algorithm 1, step 1)."""
    p = ops.p
    ns = n_surface(p)
    d = tr.depth
    nl = len(tr.leaf_keys)
    u = {d: np.zeros((nl, ns), ops.dtype)}
    for a in range(0, nl, chunk):
        leaves = np.arange(a, min(a + chunk, nl))
        chk = _leaf_surface_points(tr, p, leaves, ALPHA_OUTER)
        t_off = np.arange(len(leaves) + 1, dtype=np.int64) * ns
        ranges = np.stack([tr.leaf_offsets[leaves], tr.leaf_offsets[leaves + 1]], axis=1)
        q_uc, _ = direct.grouped_sum(t_off, chk, np.arange(len(leaves) + 1), ranges, xs, qs,
                                     gradient=False, kappa=ops.kappa, wavenumber=ops.wavenumber)
        u[d][leaves] = q_uc.reshape(len(leaves), ns) @ ops.uc2e[d].T
    for level in range(d - 1, 1, -1):
        ch = tr.children(level)
        q_uc = np.zeros((len(tr.level_keys[level]), ns), ops.dtype)
        for c in range(8):
            has = ch[:, c] >= 0
            q_uc[has] += u[level + 1][ch[has, c]] @ ops.m2m[(level, c)].T
        u[level] = q_uc @ ops.uc2e[level].T
    return u


def _needed_boxes(tr, leaves):
    """Boxes at every level that are ancestors of (or equal to) the given leaves."""
    need = {tr.depth: np.unique(leaves)}
    for level in range(tr.depth, 0, -1):
        par = tr.parent(level)[need[level]]
        need[level - 1] = np.unique(par)
    return need


def downward(tr, u, ops, leaves, m2l="grouped"):
    """VLI and D2D from level 2 to the leaves, for the given leaves' ancestors only."""
    p = ops.p
    ns = n_surface(p)
    need = _needed_boxes(tr, leaves)
    dvec = {}
    for level in range(2, tr.depth + 1):
        boxes = need[level]
        q_dc = np.zeros((len(boxes), ns), ops.dtype)
        off, idx, tvec = otree.v_lists(tr, level, boxes)
        rows = np.repeat(np.arange(len(boxes)), np.diff(off))
        if m2l == "grouped":
            for t in np.unique(tvec):
                sel = tvec == t
                q_dc[rows[sel]] += u[level][idx[sel]] @ ops.m2l[(level, int(t))].T
        elif m2l == "fft":   # each transfer vector's M2L as a lattice convolution (fft_m2l)
            from . import fft_m2l
            assert ops.alpha_inner == fft_m2l.lattice_alpha(p) and ops.wavenumber == 0.0
            tv = otree.transfer_vectors()
            r = tr.halfwidth(level)
            for t in np.unique(tvec):
                sel = tvec == t
                ghat = fft_m2l.kernel_transform(p, r, tv[int(t)], ops.kappa)
                q_dc[rows[sel]] += fft_m2l.m2l_fft(p, r, tv[int(t)], u[level][idx[sel]], ops.kappa, ghat)
        else:
            r = tr.halfwidth(level)
            ctr = tr.centres(level)
            for k in range(len(idx)):
                b, a = boxes[rows[k]], idx[k]
                kmat = kernel_matrix(surface(p, ctr[b], r, ops.alpha_inner),
                                     surface(p, ctr[a], r, ops.alpha_inner), ops.kappa, ops.wavenumber)
                q_dc[rows[k]] += kmat @ u[level][a]
        if level >= 3:
            par = tr.parent(level)[boxes]
            oct_ = (tr.level_keys[level][boxes] & np.uint64(7)).astype(np.int64)
            prev = dvec[level - 1]
            pos = np.searchsorted(need[level - 1], par)
            for c in range(8):
                sel = oct_ == c
                q_dc[sel] += prev[pos[sel]] @ ops.l2l[(level, c)].T
        dvec[level] = q_dc @ ops.dc2e[level].T
    return need, dvec


def evaluate(points, charges, p, depth, origin=None, side=None, gradient=True,
             pinv_rtol=DEFAULT_PINV_RTOL, sample=None, parts=("near", "far"), m2l="grouped",
             ops=None, kappa=0.0, wavenumber=0.0):
    """FP64 kiFMM field at every point (or at the `sample` indices, input order).  With
    wavenumber > 0 (Helmholtz) the charges, potentials and gradients are complex.

    Returns a Result whose phi/grad follow the input order of the points (or of `sample`).
    `parts` selects the near field (ULI), the far field (VLI/D2D/D2T) or both.
    """
    xs_in = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    tr = otree.build_tree(xs_in, depth, origin, side)
    if ops is None:
        ops = build_operators(p, tr.side, depth, pinv_rtol, kappa=kappa, wavenumber=wavenumber)
    kappa, wavenumber, dt = ops.kappa, ops.wavenumber, ops.dtype
    q_in = np.asarray(charges, dtype=dt).reshape(-1)
    xs = xs_in[tr.perm]
    qs = q_in[tr.perm]
    n = len(xs)
    inv = np.empty(n, dtype=np.int64)
    inv[tr.perm] = np.arange(n)
    if sample is None:
        tpos = np.arange(n)
    else:
        tpos = inv[np.asarray(sample, dtype=np.int64)]              # sorted positions
    leaf_of = np.searchsorted(tr.leaf_offsets, tpos, side="right") - 1
    leaves = np.unique(leaf_of)
    phi_s = np.zeros(n, dt)
    grad_s = np.zeros((n, 3), dt) if gradient else None
    u, dvec, need = {}, {}, {}
    # Target groups: the sampled targets of each leaf, as contiguous sorted positions.
    tsort = np.sort(tpos)
    t_leaf = np.searchsorted(tr.leaf_offsets, tsort, side="right") - 1
    grp_off = np.searchsorted(t_leaf, leaves, side="left")
    grp_off = np.append(grp_off, len(tsort)).astype(np.int64)
    tx = xs[tsort]
    pot = np.zeros(len(tsort), dt)
    grd = np.zeros((len(tsort), 3), dt) if gradient else None
    if "far" in parts and depth >= 2:
        u = upward(tr, xs, qs, ops)
        need, dvec = downward(tr, u, ops, leaves, m2l)
        pos = np.searchsorted(need[depth], leaves)
        de = _leaf_surface_points(tr, p, leaves, ALPHA_OUTER)
        dens = dvec[depth][pos].reshape(-1)
        ns = n_surface(p)
        ranges = np.stack([np.arange(len(leaves)) * ns, np.arange(1, len(leaves) + 1) * ns], 1)
        direct.grouped_sum(grp_off, tx, np.arange(len(leaves) + 1), ranges, de, dens,
                           gradient, pot, grd, kappa=kappa, wavenumber=wavenumber)
    if "near" in parts:
        uoff, uidx = otree.u_lists(tr, leaves)
        ranges = np.stack([tr.leaf_offsets[uidx], tr.leaf_offsets[uidx + 1]], axis=1)
        direct.grouped_sum(grp_off, tx, uoff, ranges, xs, qs, gradient, pot, grd, kappa=kappa,
                           wavenumber=wavenumber)
    phi_s[tsort] = pot
    if gradient:
        grad_s[tsort] = grd
    if sample is None:
        phi = np.empty(n, dt)
        phi[tr.perm] = phi_s
        grad = None
        if gradient:
            grad = np.empty((n, 3), dt)
            grad[tr.perm] = grad_s
    else:
        phi = phi_s[tpos]
        grad = grad_s[tpos] if gradient else None
    return Result(phi, grad, tr, u, need, dvec)


def adjoint(points, g, p, depth, origin=None, side=None, pinv_rtol=DEFAULT_PINV_RTOL,
            parts=("near", "far"), ops=None, kappa=0.0):
    """psi = A^T g for the FP64 kiFMM map A (charges -> potentials), input order.

    The transposed steps run in reverse order of Algorithm 1: D2T^T, the closing pinv^T,
    VLI^T (the V relation is symmetric and K(dc_b, ue_a)^T = K(ue_a, dc_b)), D2D^T to the
    parents, U2U^T to the children and S2U^T back to the points.  ULI is symmetric.
    """
    xs_in = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    g_in = np.asarray(g, dtype=np.float64).reshape(-1)
    tr = otree.build_tree(xs_in, depth, origin, side)
    xs = xs_in[tr.perm]
    gs = g_in[tr.perm]
    n = len(xs)
    if ops is None:
        ops = build_operators(p, tr.side, depth, pinv_rtol, kappa=kappa)
    kappa = ops.kappa
    ns = n_surface(p)
    nl = len(tr.leaf_keys)
    psi = np.zeros(n)
    leaves = np.arange(nl)
    if "far" in parts and depth >= 2:
        # D2T^T: dbar_b = K(de_b, x_b) g_b
        de = _leaf_surface_points(tr, p, leaves, ALPHA_OUTER)
        ranges = np.stack([tr.leaf_offsets[:-1], tr.leaf_offsets[1:]], axis=1)
        dbar, _ = direct.grouped_sum(np.arange(nl + 1) * ns, de, np.arange(nl + 1), ranges,
                                     xs, gs, gradient=False, kappa=kappa)
        dbar = {depth: dbar.reshape(nl, ns)}
        ubar = {lvl: np.zeros((len(tr.level_keys[lvl]), ns)) for lvl in range(2, depth + 1)}
        for level in range(depth, 1, -1):
            qbar = dbar[level] @ ops.dc2e[level]                 # (pinv^T applied to rows)
            off, idx, tvec = otree.v_lists(tr, level)
            rows = np.repeat(np.arange(len(tr.level_keys[level])), np.diff(off))
            for t in np.unique(tvec):
                sel = tvec == t
                np.add.at(ubar[level], idx[sel], qbar[rows[sel]] @ ops.m2l[(level, int(t))])
            if level >= 3:
                par = tr.parent(level)
                oct_ = (tr.level_keys[level] & np.uint64(7)).astype(np.int64)
                acc = np.zeros((len(tr.level_keys[level - 1]), ns))
                for c in range(8):
                    sel = oct_ == c
                    np.add.at(acc, par[sel], qbar[sel] @ ops.l2l[(level, c)])
                dbar[level - 1] = acc
        for level in range(2, depth):
            ch = tr.children(level)
            qbar_uc = ubar[level] @ ops.uc2e[level]
            for c in range(8):
                has = ch[:, c] >= 0
                ubar[level + 1][ch[has, c]] += qbar_uc[has] @ ops.m2m[(level, c)]
        ebar = ubar[depth] @ ops.uc2e[depth]                   # (nl, ns) on the uc surface
        uc = _leaf_surface_points(tr, p, leaves, ALPHA_OUTER)
        ranges = np.stack([np.arange(nl) * ns, np.arange(1, nl + 1) * ns], axis=1)
        direct.grouped_sum(tr.leaf_offsets, xs, np.arange(nl + 1), ranges, uc,
                           ebar.reshape(-1), False, psi, None, kappa=kappa)
    if "near" in parts:
        uoff, uidx = otree.u_lists(tr, leaves)
        ranges = np.stack([tr.leaf_offsets[uidx], tr.leaf_offsets[uidx + 1]], axis=1)
        direct.grouped_sum(tr.leaf_offsets, xs, uoff, ranges, xs, gs, False, psi, None, kappa=kappa)
    out = np.empty(n)
    out[tr.perm] = psi
    return out
