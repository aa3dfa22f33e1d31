"""Split-precision tensor-core contractions (tcgen05): BF16x3, BF16x6, TF32x3 and FP16x3 forms of
the surface contractions and of the M2L, against the FP64 oracle and against the FP32 form.
FP16x3 runs every tensor-core contraction (U2U, the M2L compress, stencil and decompress, D2D) on
power-of-two scaled FP16 hi/lo splits (~2^-22 per term); its bar is that of BF16x6.

Tolerances: 1e-5 (potentials) and 1e-4 (gradients) relative L2, the bar stated for the FMM,
for BF16x6 and TF32x3 (22 or more significant bits per operand; measured ~1e-6).  BF16x3 keeps
~16 bits (hi + lo) and drops lo*lo, ~2^-17 relative per product: with positive charges the
far field has no cancellation and BF16x3 stays near 3e-6, but with charges of both signs the
potentials are differences of larger sums and its relative error grows by the cancellation
factor, so for mixed-sign charges its bound is stated as 3e-5 (measured 1.0e-5).
"""
import numpy as np
import pytest
import torch

from oracle import direct, kifmm, tree as otree
from synth import cube_points, sphere_points, charges
from gpu_helpers import PINV_RTOL, make_fmm, rel, run

pytestmark = pytest.mark.gpu
CUBE = ((0, 0, 0), 1.0)
BALL = ((-1, -1, -1), 2.0)
MODES = ["bf16x3", "tf32x3", "bf16x6", "fp16x3"]


def _oracle(x, q, p, depth, domain, **kw):
    return kifmm.evaluate(x.astype(np.float64), q.astype(np.float64), p, depth, *domain,
                          pinv_rtol=PINV_RTOL, **kw)


def test_tensor_smoke_bf16x3():
    # smallest case first: one level of M2L, p=4 (N=64 columns)
    x, q = cube_points(5000), charges(5000, "u11")
    f = make_fmm(x, 4, 2, "bf16x3", CUBE)
    phi, grad = run(f, q)
    f.sync()
    ref = _oracle(x, q, 4, 2, CUBE)
    assert rel(phi, ref.phi) < 1e-5 and rel(grad, ref.grad) < 1e-4


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dist,n,p,depth", [("cube", 60_000, 6, 4), ("sphere", 80_000, 6, 5),
                                            ("cube", 30_000, 8, 3), ("sphere", 40_000, 4, 4)])
def test_tensor_against_oracle(mode, dist, n, p, depth):
    x = cube_points(n) if dist == "cube" else sphere_points(n)
    q = charges(n, "u11" if dist == "cube" else "u01")
    dom = CUBE if dist == "cube" else BALL
    f = make_fmm(x, p, depth, mode, dom)
    phi, grad = run(f, q)
    f.sync()
    ref = _oracle(x, q, p, depth, dom)
    mixed_sign = dist == "cube"
    tol = 3e-5 if (mode == "bf16x3" and mixed_sign) else 1e-5
    assert rel(phi, ref.phi) < tol
    assert rel(grad, ref.grad) < 1e-4


@pytest.mark.parametrize("mode", MODES)
def test_tensor_matches_fp32_contractions(mode):
    # the downward check potentials of every level against the FP32 SIMT form
    x, q = sphere_points(60_000), charges(60_000, "u01")
    p, depth = 6, 5
    a = make_fmm(x, p, depth, "fp32", BALL)
    b = make_fmm(x, p, depth, mode, BALL)
    run(a, q, gradient=False)
    run(b, q, gradient=False)
    b.sync()
    for level in range(2, depth + 1):
        assert rel(b.export_check(level, "upward"), a.export_check(level, "upward")) < 1e-5, level
        assert rel(b.export_check(level, "downward"), a.export_check(level, "downward")) < 1e-5, level


@pytest.mark.parametrize("mode", MODES)
def test_tensor_adjoint_dot_product(mode):
    n = 50_000
    x = cube_points(n)
    q = charges(n, "u11").astype(np.float64)
    g = charges(n, "normal", seed=2).astype(np.float64)
    f = make_fmm(x, 6, 4, mode, CUBE)
    aq = run(f, q, gradient=False)[0]
    psi, _ = f.adjoint(torch.from_numpy(g).float().cuda())
    f.sync()
    atg = psi.cpu().numpy().astype(np.float64)
    tol = 3e-5 if mode == "bf16x3" else 1e-5       # mixed-sign charges (module docstring)
    assert abs(g @ aq - atg @ q) / (np.linalg.norm(g) * np.linalg.norm(aq)) < tol
    ref = kifmm.adjoint(x.astype(np.float64), g, 6, 4, *CUBE, pinv_rtol=PINV_RTOL)
    assert rel(atg, ref) < tol


def test_tensor_sparse_tiles_and_ragged_levels():
    # a thin sheet: most stencil slots of most tiles are empty, classes are ragged
    rng = np.random.default_rng(9)
    x = np.stack([rng.random(30_000), rng.random(30_000), 0.5 + 0.002 * rng.random(30_000)], 1)
    x = x.astype(np.float32)
    q = charges(30_000, "u01")
    f = make_fmm(x, 5, 5, "bf16x3", CUBE)
    phi, grad = run(f, q)
    f.sync()
    ref = _oracle(x, q, 5, 5, CUBE)
    assert rel(phi, ref.phi) < 1e-5 and rel(grad, ref.grad) < 1e-4
