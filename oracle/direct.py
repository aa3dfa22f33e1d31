"""FP64 direct evaluation of the field sum (Eq. 1) with the 3D Laplace kernel (Eq. 2).

The kernel is normalised as K(x, y) = 1 / (4 pi |x - y|); with `kappa` > 0 it is the modified
Helmholtz (Yukawa) kernel exp(-kappa |x - y|) / (4 pi |x - y|), and with `wavenumber` k > 0 the Helmholtz
kernel exp(i k |x - y|) / (4 pi |x - y|) with complex densities: the other kernels the
kernel-independent method is run with.  The paper writes 1/|x - y|; the
factor only scales every result, so relative errors are unaffected.  Pairs at distance exactly
zero are skipped (self-interaction and coincident points).

Two independent formulations are kept so that each pins the other:
  * `direct_numpy`: dense NumPy broadcasting in chunks of targets;
  * `grouped_sum` / `direct_c`: the plain C double loop in csrc/oracle_sum.c.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

INV4PI = 1.0 / (4.0 * np.pi)

_lib = None


def _native():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        p = ctypes.c_void_p
        lib.oracle_grouped_sum.argtypes = [ctypes.c_int64, p, p, p, p, p, p, p, p, ctypes.c_double]
        lib.oracle_grouped_sum.restype = None
        lib.oracle_grouped_sum_helm.argtypes = [ctypes.c_int64, p, p, p, p, p, p, p, p, ctypes.c_double]
        lib.oracle_grouped_sum_helm.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """Threads the C helper uses (OpenMP), for reporting the CPU baseline."""
    return int(_native().oracle_num_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def direct_numpy(targets, sources, charges, gradient=True, chunk=2048, kappa=0.0, wavenumber=0.0):
    """phi_i = sum_j K(x_i, y_j) s_j and its gradient, by dense broadcasting (FP64; complex for
    the Helmholtz kernel, wavenumber > 0)."""
    x = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    y = np.asarray(sources, dtype=np.float64).reshape(-1, 3)
    if wavenumber > 0.0:
        return _direct_numpy_helm(x, y, np.asarray(charges, dtype=np.complex128).reshape(-1), gradient, chunk,
                                  wavenumber)
    s = np.asarray(charges, dtype=np.float64).reshape(-1)
    pot = np.zeros(len(x))
    grad = np.zeros((len(x), 3)) if gradient else None
    for a in range(0, len(x), chunk):
        d = x[a:a + chunk, None, :] - y[None, :, :]          # x_i - y_j
        r2 = np.einsum("ijk,ijk->ij", d, d)
        with np.errstate(divide="ignore"):
            rinv = np.where(r2 > 0.0, 1.0 / np.sqrt(np.where(r2 > 0.0, r2, 1.0)), 0.0)
        r = r2 * rinv
        w = rinv * np.exp(-kappa * r) * s[None, :]
        pot[a:a + chunk] = w.sum(axis=1) * INV4PI
        if gradient:
            w3 = w * (1.0 + kappa * r) * rinv * rinv
            grad[a:a + chunk] = -np.einsum("ij,ijk->ik", w3, d) * INV4PI
    return pot, grad


def _direct_numpy_helm(x, y, s, gradient, chunk, k):
    """exp(i k r) / (4 pi r) with complex densities; the gradient of exp(i k r) / r with respect to
    the target is exp(i k r) (i k r - 1) (x - y) / r^3."""
    pot = np.zeros(len(x), np.complex128)
    grad = np.zeros((len(x), 3), np.complex128) if gradient else None
    for a in range(0, len(x), chunk):
        d = x[a:a + chunk, None, :] - y[None, :, :]
        r2 = np.einsum("ijk,ijk->ij", d, d)
        with np.errstate(divide="ignore"):
            rinv = np.where(r2 > 0.0, 1.0 / np.sqrt(np.where(r2 > 0.0, r2, 1.0)), 0.0)
        r = r2 * rinv
        w = rinv * np.exp(1j * k * r) * s[None, :]
        pot[a:a + chunk] = w.sum(axis=1) * INV4PI
        if gradient:
            w3 = w * (1j * k * r - 1.0) * rinv * rinv
            grad[a:a + chunk] = np.einsum("ij,ijk->ik", w3, d) * INV4PI
    return pot, grad


def grouped_sum(t_off, tx, r_off, ranges, sx, sq, gradient=True, pot=None, grad=None, kappa=0.0,
                wavenumber=0.0):
    """Accumulate kernel sums over (target group, source ranges) with the C helper (FP64).

    t_off[g]:t_off[g+1] are the targets of group g; ranges[r_off[g]:r_off[g+1]] are its
    (begin, end) source index ranges.  Returns (pot, grad) accumulated into the given arrays.
    """
    t_off = np.ascontiguousarray(t_off, dtype=np.int64)
    tx = np.ascontiguousarray(tx, dtype=np.float64).reshape(-1, 3)
    r_off = np.ascontiguousarray(r_off, dtype=np.int64)
    ranges = np.ascontiguousarray(ranges, dtype=np.int64).reshape(-1, 2)
    sx = np.ascontiguousarray(sx, dtype=np.float64).reshape(-1, 3)
    n_groups = len(t_off) - 1
    assert len(r_off) == n_groups + 1
    if wavenumber > 0.0:   # complex densities and outputs, interleaved (re, im) for the C helper
        sq = np.ascontiguousarray(sq, dtype=np.complex128).reshape(-1)
        if pot is None:
            pot = np.zeros(len(tx), np.complex128)
        if gradient and grad is None:
            grad = np.zeros((len(tx), 3), np.complex128)
        assert pot.dtype == np.complex128 and pot.flags.c_contiguous
        if gradient:
            assert grad.dtype == np.complex128 and grad.flags.c_contiguous
        _native().oracle_grouped_sum_helm(n_groups, _ptr(t_off), _ptr(tx), _ptr(r_off), _ptr(ranges), _ptr(sx),
                                          _ptr(sq), _ptr(pot), _ptr(grad) if gradient else None, float(wavenumber))
        return pot, (grad if gradient else None)
    sq = np.ascontiguousarray(sq, dtype=np.float64).reshape(-1)
    if pot is None:
        pot = np.zeros(len(tx))
    if gradient and grad is None:
        grad = np.zeros((len(tx), 3))
    assert pot.dtype == np.float64 and pot.flags.c_contiguous
    if gradient:
        assert grad.dtype == np.float64 and grad.flags.c_contiguous
    _native().oracle_grouped_sum(n_groups, _ptr(t_off), _ptr(tx), _ptr(r_off), _ptr(ranges),
                                 _ptr(sx), _ptr(sq), _ptr(pot), _ptr(grad) if gradient else None,
                                 float(kappa))
    return pot, (grad if gradient else None)


def direct_c(targets, sources, charges, gradient=True, kappa=0.0, wavenumber=0.0):
    """Eq. 1 at the given targets from all sources, with the C helper (FP64)."""
    tx = np.asarray(targets, dtype=np.float64).reshape(-1, 3)
    n_s = len(np.asarray(sources).reshape(-1, 3))
    return grouped_sum([0, len(tx)], tx, [0, 1], [[0, n_s]], sources, charges, gradient, kappa=kappa,
                       wavenumber=wavenumber)


def direct_self(points, charges, gradient=True, sample=None, kappa=0.0, wavenumber=0.0):
    """Field at the points themselves (targets = sources), optionally only at `sample` indices."""
    x = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    t = x if sample is None else x[np.asarray(sample)]
    return direct_c(t, x, charges, gradient, kappa=kappa, wavenumber=wavenumber)
