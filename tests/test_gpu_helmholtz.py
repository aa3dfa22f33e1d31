"""GPU kiFMM with the Helmholtz kernel exp(i k r) / (4 pi r) and complex densities (Eq. 1 with
F = C) against the FP64 oracle run with the same kernel.  The contractions act on the real form
[Re v; Im v] of every box vector; the point kernels are complex.

Tolerances as for the real kernels: potentials 1e-5 and gradients 1e-4 relative L2 for FP32 and
the split tensor-core modes, 1e-8 for FP64; the near field alone is exact arithmetic on the same
pairs (FP32 rounding, sincos included: 2e-6).
"""
import ctypes
import functools

import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from oracle import direct, kifmm
from synth import cube_points, sphere_points, charges
from gpu_helpers import PINV_RTOL, SVD_RTOL, rel

pytestmark = pytest.mark.gpu
CUBE = ((0, 0, 0), 1.0)
BALL = ((-1, -1, -1), 2.0)
TOL = {"fp32": (1e-5, 1e-4), "fp64": (1e-8, 1e-8), "fp16x3": (1e-5, 1e-4), "bf16x6": (1e-5, 1e-4)}
# one wavelength across the unit cube; on the ball, 0.6 of a wavelength across the cube of side 2
CASES = {"cube": ("cube", 20_000, 5, 3, 2 * np.pi), "sphere": ("sphere", 40_000, 5, 4, 2.0),
         "cube_p6": ("cube", 20_000, 6, 3, 2 * np.pi)}


def _inputs(case):
    dist, n, p, depth, k = CASES[case]
    x = cube_points(n) if dist == "cube" else sphere_points(n)
    q = charges(n, "u11", seed=1) + 1j * charges(n, "u11", seed=101)
    return x, q, p, depth, k, (CUBE if dist == "cube" else BALL)


def _fmm(x, p, depth, precision, dom, k, **kw):
    f = pkg.FMM(p=p, depth=depth, precision=precision, domain=dom, pinv_rtol=PINV_RTOL, svd_rtol=SVD_RTOL,
                kernel="helmholtz", kappa=k, **kw)
    dt = torch.float64 if precision == "fp64" else torch.float32
    f.build_tree(torch.from_numpy(np.ascontiguousarray(x)).to("cuda", dt))
    f.precompute()
    return f


def _run(f, q, **kw):
    dt = torch.complex128 if f.precision == "fp64" else torch.complex64
    phi, grad = f.evaluate(torch.from_numpy(q).to("cuda", dt), **kw)
    torch.cuda.synchronize()
    return (phi.cpu().numpy().astype(np.complex128) if phi is not None else None,
            grad.cpu().numpy().astype(np.complex128) if grad is not None else None)


@functools.lru_cache(maxsize=None)
def _oracle(case, parts=("near", "far")):
    x, q, p, depth, k, dom = _inputs(case)
    return kifmm.evaluate(x.astype(np.float64), q, p, depth, *dom, pinv_rtol=PINV_RTOL, parts=parts,
                          wavenumber=k)


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16x3", "bf16x6"])
@pytest.mark.parametrize("case", ["cube", "sphere"])
def test_against_oracle(precision, case):
    x, q, p, depth, k, dom = _inputs(case)
    phi, grad = _run(_fmm(x, p, depth, precision, dom, k), q)
    ref = _oracle(case)
    tp, tg = TOL[precision]
    assert rel(phi, ref.phi) < tp, rel(phi, ref.phi)
    assert rel(grad, ref.grad) < tg, rel(grad, ref.grad)


def test_p6_against_oracle_and_direct():
    x, q, p, depth, k, dom = _inputs("cube_p6")
    phi, grad = _run(_fmm(x, p, depth, "fp16x3", dom, k), q)
    ref = _oracle("cube_p6")
    assert rel(phi, ref.phi) < 1e-5 and rel(grad, ref.grad) < 1e-4
    idx = np.arange(0, len(x), 97)
    dp, dg = direct.direct_self(x.astype(np.float64), q, sample=idx, wavenumber=k)
    assert rel(phi[idx], dp) < 1e-5 and rel(grad[idx], dg) < 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_parts_near_and_far(precision):
    x, q, p, depth, k, dom = _inputs("sphere")
    f = _fmm(x, p, depth, precision, dom, k)
    near, gnear = _run(f, q, parts=pkg.PART_NEAR)
    far, gfar = _run(f, q, parts=pkg.PART_FAR)
    rn, rf = _oracle("sphere", ("near",)), _oracle("sphere", ("far",))
    assert rel(near, rn.phi) < (2e-6 if precision == "fp32" else 1e-13)
    assert rel(gnear, rn.grad) < (2e-6 if precision == "fp32" else 1e-13)
    assert rel(far, rf.phi) < TOL[precision][0]
    assert rel(gfar, rf.grad) < TOL[precision][1]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_direct_sum(precision, depth):
    x = cube_points(3000)
    q = charges(3000, "u11") + 1j * charges(3000, "normal", seed=7)
    phi, grad = _run(_fmm(x, 4, depth, precision, CUBE, 2 * np.pi), q)
    dp, dg = direct.direct_self(x.astype(np.float64), q, wavenumber=2 * np.pi)
    tol = 2e-6 if precision == "fp32" else 1e-13
    assert rel(phi, dp) < tol and rel(grad, dg) < tol


def test_complex_linearity_gradient_only_and_host_buffers():
    x, q, p, depth, k, dom = _inputs("cube")
    f = _fmm(x, p, depth, "fp32", dom, k)
    a, ga = _run(f, q.real.astype(np.complex128))
    b, gb = _run(f, q.imag.astype(np.complex128))
    c, gc = _run(f, q)
    # linear up to the FP32 rounding of the three evaluations (a wrong sign or conjugate is O(1))
    assert rel(c, a + 1j * b) < 2e-5 and rel(gc, ga + 1j * gb) < 2e-5
    _, g_only = _run(f, q, potential=False)
    assert np.array_equal(g_only, gc)
    ph = np.zeros(len(x), np.complex64)
    gh = np.zeros((len(x), 3), np.complex64)
    f.evaluate_into(np.ascontiguousarray(q.astype(np.complex64)), ph, gh)
    assert np.array_equal(ph.astype(np.complex128), c) and np.array_equal(gh.astype(np.complex128), gc)


def test_small_wavenumber_is_laplace():
    x, q, p, depth, _, dom = _inputs("cube")
    lap = pkg.FMM(p=p, depth=depth, precision="fp64", domain=dom, pinv_rtol=PINV_RTOL, svd_rtol=SVD_RTOL)
    lap.build_tree(torch.from_numpy(x).to("cuda", torch.float64))
    lap.precompute()
    pl, _ = lap.evaluate(torch.from_numpy(q.real.copy()).cuda())
    ph, _ = _run(_fmm(x, p, depth, "fp64", dom, 1e-6), q.real.astype(np.complex128))
    assert rel(ph.real, pl.cpu().numpy()) < 1e-8


def test_unsupported_and_invalid():
    x, q, p, depth, k, dom = _inputs("cube")
    f = _fmm(x, 4, 3, "fp32", dom, k)
    qd = torch.from_numpy(q).to("cuda", torch.complex64)
    psi = torch.empty_like(qd)
    L = pkg.lib()
    assert L.fmm_adjoint(f._ctx, ctypes.c_void_p(qd.data_ptr()), ctypes.c_void_p(psi.data_ptr()), None) == 6
    assert L.fmm_partition_setup(f._ctx, 2, 2) == 6
    with pytest.raises(pkg.FmmError):
        pkg.FMM(p=4, depth=3, kernel="helmholtz", kappa=1.0)          # no domain
    with pytest.raises(pkg.FmmError):
        pkg.FMM(p=4, depth=3, kernel="helmholtz", kappa=0.0, domain=dom)


def test_leaf_check_values_exported():
    # S2U input: every leaf's complex check values are a plain kernel sum over its own points,
    # exported as [Re | Im] rows of 2 n_surface values
    from oracle import tree as otree
    x, q, _, _, k, dom = _inputs("sphere")
    p, depth = 4, 4
    f = _fmm(x, p, depth, "fp32", dom, k)
    _run(f, q, gradient=False)
    got = f.export_check(depth, "upward")
    tr = otree.build_tree(x.astype(np.float64), depth, *dom)
    ns = kifmm.n_surface(p)
    nl = len(tr.leaf_keys)
    assert got.shape == (nl, 2 * ns)
    chk = kifmm._leaf_surface_points(tr, p, np.arange(nl), kifmm.ALPHA_OUTER)
    want, _ = direct.grouped_sum(np.arange(nl + 1) * ns, chk, np.arange(nl + 1),
                                 np.stack([tr.leaf_offsets[:-1], tr.leaf_offsets[1:]], 1),
                                 x.astype(np.float64)[tr.perm], q[tr.perm], False, wavenumber=k)
    want = want.reshape(nl, ns)
    assert rel(got[:, :ns] + 1j * got[:, ns:], want) < 1e-6
