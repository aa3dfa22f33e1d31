"""M2L as a lattice convolution evaluated by FFT, in FP64 (the oracle; test infrastructure only:
the CUDA path never imports it).  Its pins are in tests/test_oracle_fft_m2l.py.

The M2L of the kernel-independent method maps the upward equivalent densities of a source box
(order-p surface grid of radius alpha r around its centre) to check potentials on the target box's
downward check surface (the same grid around the target's centre):
    c_i = sum_j K(x_i, y_j) u_j.
When the grid spacing h = 2 alpha r / (p - 1) divides the box width 2r, every x_i - y_j is a
lattice vector h (i - j - m t), with m = 2r / h and t the transfer vector in box units, so the map
is a discrete convolution with the kernel sampled on the lattice.  Zero-padded to 2p points per
axis, the convolution theorem evaluates it with three-dimensional FFTs: one per source box, one
per target box, and one Hadamard product per (target, source) pair; the kernel's transform is
computed once per transfer vector (the FFT acceleration of the M2L that the paper cites as an
alternative to the BLAS form, Section 2.2).

Readings where the paper is silent:
  * the lattice: alpha = (p - 1) / (p - 2), the smallest radius above the box with
    (p - 1) / alpha an integer (m = p - 2 lattice steps per box width); 1.25 at p = 6.  It needs
    p >= 4: at p = 3 (alpha = 2) the surfaces of boxes two widths apart would touch;
  * densities and potentials live on the p^3 grid; points off the surface hold zero density and
    their potentials are discarded.
"""
from __future__ import annotations

import numpy as np

from . import kifmm


def lattice_alpha(p):
    """Surface radius (in half-widths) whose grid spacing divides the box width: (p-1)/(p-2)."""
    if p < 4:   # p = 3 gives alpha = 2: the surfaces of boxes two widths apart would touch
        raise ValueError("the lattice surface needs p >= 4")
    return (p - 1) / (p - 2)


def surface_mask(p):
    """Boolean p^3 mask of the surface points, in the lexicographic order of surface_grid."""
    i = np.arange(p)
    a, b, c = np.meshgrid(i, i, i, indexing="ij")
    return (np.minimum(np.minimum(a, b), c) == 0) | (np.maximum(np.maximum(a, b), c) == p - 1)


def kernel_transform(p, r, t, kappa=0.0):
    """FFT (size (2p)^3) of the kernel on the lattice differences for transfer vector t (box units)
    between boxes of half-width r, with the lattice surfaces of radius lattice_alpha(p) r."""
    alpha = lattice_alpha(p)
    h = 2.0 * alpha * r / (p - 1)
    m = p - 2
    n = 2 * p
    d = np.arange(n)
    d = np.where(d < p, d, d - n)                      # circular index -> lattice difference
    dx, dy, dz = np.meshgrid(d, d, d, indexing="ij")
    tx, ty, tz = (np.asarray(t, dtype=np.int64) * m)
    vec = h * np.stack([dx - tx, dy - ty, dz - tz], axis=-1)
    rr = np.sqrt((vec ** 2).sum(axis=-1))
    g = np.where(rr > 0, kifmm.INV4PI * np.exp(-kappa * rr) / np.where(rr > 0, rr, 1.0), 0.0)
    g[np.abs(dx) > p - 1] = 0.0                         # differences outside the p^3 grid do not occur
    g[np.abs(dy) > p - 1] = 0.0
    g[np.abs(dz) > p - 1] = 0.0
    return np.fft.rfftn(g)


def m2l_fft(p, r, t, u, kappa=0.0, ghat=None):
    """Check potentials on the target's lattice surface from densities u (n_surface(p) values, or a
    batch (k, n_surface)) on the source's, for transfer vector t: the convolution by FFT."""
    u = np.atleast_2d(np.asarray(u, dtype=np.float64))
    mask = surface_mask(p)
    n = 2 * p
    grid = np.zeros((u.shape[0], n, n, n))
    grid[:, :p, :p, :p][:, mask] = u
    if ghat is None:
        ghat = kernel_transform(p, r, t, kappa)
    c = np.fft.irfftn(np.fft.rfftn(grid, axes=(1, 2, 3)) * ghat[None], s=(n, n, n), axes=(1, 2, 3))
    return c[:, :p, :p, :p][:, mask]


def m2l_dense(p, r, t, u, kappa=0.0):
    """The same map as one dense kernel matrix from the two surfaces' coordinates."""
    alpha = lattice_alpha(p)
    g = kifmm.surface_grid(p)
    tgt = alpha * r * g
    src = 2.0 * r * np.asarray(t, dtype=np.float64) + alpha * r * g
    return np.atleast_2d(u) @ kifmm.kernel_matrix(tgt, src, kappa).T
