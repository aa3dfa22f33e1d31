"""The FFT form of the M2L on the GPU (fmm_options.m2l = FMM_M2L_FFT; Section 2.2 names it beside
the BLAS form) against the FP64 oracle run with the same lattice surfaces and its own FFT M2L
(oracle.kifmm.evaluate(..., m2l="fft") with alpha_inner = lattice_alpha(p)).

Tolerances as for the BLAS form: FP32 potentials 1e-5 and gradients 1e-4 relative L2, FP64 1e-8.
Unlike the compressed BLAS form, the FFT form applies the M2L without truncation, so FP64 results
differ from the oracle by rounding and the two pseudo-inverse factorisations only."""
import functools

import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from oracle import direct, fft_m2l, kifmm
from synth import cube_points, sphere_points, charges
from gpu_helpers import PINV_RTOL, make_fmm, rel, run

pytestmark = pytest.mark.gpu
CUBE = ((0, 0, 0), 1.0)
BALL = ((-1, -1, -1), 2.0)
TOL = {"fp32": (1e-5, 1e-4), "fp64": (1e-8, 1e-8)}


def _inputs(dist, n):
    x = cube_points(n) if dist == "cube" else sphere_points(n)
    return x, charges(n, "u11"), (CUBE if dist == "cube" else BALL)


@functools.lru_cache(maxsize=None)
def _oracle_fft(dist, n, p, depth):
    x, q, domain = _inputs(dist, n)
    ops = kifmm.build_operators(p, domain[1], depth, PINV_RTOL, alpha_inner=fft_m2l.lattice_alpha(p))
    return kifmm.evaluate(x.astype(np.float64), q.astype(np.float64), p, depth, *domain, pinv_rtol=PINV_RTOL,
                          ops=ops, m2l="fft")


@pytest.mark.parametrize("dist,n,p,depth", [("cube", 20_000, 6, 3), ("sphere", 40_000, 6, 5),
                                            ("cube", 20_000, 8, 3), ("cube", 12_000, 4, 3)])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_fft_m2l_against_oracle(precision, dist, n, p, depth):
    x, q, domain = _inputs(dist, n)
    f = make_fmm(x, p, depth, precision, domain, m2l="fft")
    phi, grad = run(f, q)
    f.sync()
    f.close()
    ref = _oracle_fft(dist, n, p, depth)
    tp, tg = TOL[precision]
    assert rel(phi, ref.phi) < tp and rel(grad, ref.grad) < tg, (rel(phi, ref.phi), rel(grad, ref.grad))


def test_fft_and_dense_forms_agree_with_the_direct_sum():
    # p = 8 on a depth-4 cube: both forms within their truncation error of the FP64 direct sum
    n, p, depth = 30_000, 8, 4
    x, q = cube_points(n, seed=41), charges(n, "u01", seed=42)
    idx = np.arange(0, n, 97)
    dp, dg = direct.direct_self(x.astype(np.float64), q.astype(np.float64), sample=idx)
    for m2l in ("dense", "fft"):
        f = make_fmm(x, p, depth, "fp32", CUBE, m2l=m2l)
        phi, grad = run(f, q)
        f.close()
        assert rel(phi[idx], dp) < 1e-5 and rel(grad[idx], dg) < 1e-4, (m2l, rel(phi[idx], dp), rel(grad[idx], dg))


def test_fft_form_options():
    with pytest.raises(pkg.FmmError):   # tensor-core precisions take the BLAS form only
        pkg.FMM(p=6, depth=3, precision="fp16x3", m2l="fft")
    with pytest.raises(pkg.FmmError):   # the lattice needs p >= 4
        pkg.FMM(p=3, depth=3, m2l="fft")
    x = torch.from_numpy(cube_points(5000)).cuda()
    f = pkg.FMM(p=4, depth=3, domain=CUBE, m2l="fft")
    f.build_tree(x).precompute()
    with pytest.raises(pkg.FmmError) as e:
        f.adjoint(torch.ones(5000, device="cuda"))
    assert e.value.status == 6   # FMM_EUNSUPPORTED
    f.close()
