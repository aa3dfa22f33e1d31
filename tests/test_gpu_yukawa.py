"""GPU kiFMM with the modified Helmholtz (Yukawa) kernel exp(-kappa r) / (4 pi r) against the
FP64 oracle run with the same kernel (Eq. 1 with a second real kernel; Section 2.1's steps
unchanged, operators per level because the kernel is not homogeneous).

Tolerances as for Laplace: potentials 1e-5 and gradients 1e-4 relative L2 for FP32 and the
split tensor-core modes, 1e-8 for FP64; the near field alone is exact arithmetic on the same
pairs (FP32 rounding of the screening factor included, 2e-6).
"""
import functools

import numpy as np
import pytest

import paper_2604_19243_gb300 as pkg
from oracle import direct, kifmm
from synth import WORKLOADS, cube_points, sphere_points, charges, sample_indices
from gpu_helpers import PINV_RTOL, make_fmm, rel, run

pytestmark = pytest.mark.gpu
CUBE = ((0, 0, 0), 1.0)
BALL = ((-1, -1, -1), 2.0)
TOL = {"fp32": (1e-5, 1e-4), "fp64": (1e-8, 1e-8), "fp16x3": (1e-5, 1e-4), "bf16x6": (1e-5, 1e-4)}
# kappa r at the leaves from 0.04 to 0.6 and at level 2 from 0.4 to 5: mild to strong screening
CASES = {"cube_k3": ("cube", 30_000, 5, 3, 3.0), "sphere_k3": ("sphere", 50_000, 6, 4, 3.0),
         "sphere_k20": ("sphere", 40_000, 6, 4, 20.0)}


def _inputs(case):
    dist, n, p, depth, kappa = CASES[case]
    x = cube_points(n) if dist == "cube" else sphere_points(n)
    q = charges(n, "u11" if dist == "cube" else "u01")
    return x, q, p, depth, kappa, (CUBE if dist == "cube" else BALL)


@functools.lru_cache(maxsize=None)
def _oracle(case, parts=("near", "far")):
    x, q, p, depth, kappa, dom = _inputs(case)
    return kifmm.evaluate(x.astype(np.float64), q.astype(np.float64), p, depth, *dom,
                          pinv_rtol=PINV_RTOL, parts=parts, kappa=kappa)


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16x3", "bf16x6"])
@pytest.mark.parametrize("case", list(CASES))
def test_against_oracle(precision, case):
    x, q, p, depth, kappa, dom = _inputs(case)
    f = make_fmm(x, p, depth, precision, dom, kernel="yukawa", kappa=kappa)
    phi, grad = run(f, q)
    ref = _oracle(case)
    tp, tg = TOL[precision]
    assert rel(phi, ref.phi) < tp, rel(phi, ref.phi)
    assert rel(grad, ref.grad) < tg, rel(grad, ref.grad)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_parts_near_and_far(precision):
    x, q, p, depth, kappa, dom = _inputs("sphere_k3")
    f = make_fmm(x, p, depth, precision, dom, kernel="yukawa", kappa=kappa)
    near, gnear = run(f, q, parts=pkg.PART_NEAR)
    far, gfar = run(f, q, parts=pkg.PART_FAR)
    rn, rf = _oracle("sphere_k3", ("near",)), _oracle("sphere_k3", ("far",))
    assert rel(near, rn.phi) < (2e-6 if precision == "fp32" else 1e-13)
    assert rel(gnear, rn.grad) < (2e-6 if precision == "fp32" else 1e-13)
    assert rel(far, rf.phi) < TOL[precision][0]
    assert rel(gfar, rf.grad) < TOL[precision][1]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_direct_sum(precision, depth):
    x, q = cube_points(3000), charges(3000, "u11")
    f = make_fmm(x, 4, depth, precision, CUBE, kernel="yukawa", kappa=5.0)
    phi, grad = run(f, q)
    dp, dg = direct.direct_self(x.astype(np.float64), q.astype(np.float64), kappa=5.0)
    tol = 2e-6 if precision == "fp32" else 1e-13
    assert rel(phi, dp) < tol and rel(grad, dg) < tol


@pytest.mark.parametrize("precision", ["fp32", "fp16x3"])
def test_adjoint_against_oracle(precision):
    import torch
    x, _, p, depth, kappa, dom = _inputs("sphere_k3")
    g = charges(len(x), "normal", seed=11)
    f = make_fmm(x, p, depth, precision, dom, kernel="yukawa", kappa=kappa)
    psi, _ = f.adjoint(torch.from_numpy(g).to("cuda", torch.float32))
    ref = kifmm.adjoint(x.astype(np.float64), g.astype(np.float64), p, depth, *dom,
                        pinv_rtol=PINV_RTOL, kappa=kappa)
    assert rel(psi.cpu().numpy(), ref) < 1e-5


def test_screening_changes_the_field():
    # a Yukawa context and a Laplace context on the same points differ by the screening, and
    # kappa -> 0 recovers Laplace within the FP32 bar
    x, q, p, depth, _, dom = _inputs("cube_k3")
    lap, _ = run(make_fmm(x, p, depth, "fp32", dom), q)
    yk, _ = run(make_fmm(x, p, depth, "fp32", dom, kernel="yukawa", kappa=3.0), q)
    tiny, _ = run(make_fmm(x, p, depth, "fp32", dom, kernel="yukawa", kappa=1e-7), q)
    assert rel(yk, lap) > 0.1
    assert rel(tiny, lap) < 1e-5


@pytest.mark.slow
def test_cube1m_against_oracle_sampled():
    # the 1M-point uniform workload (p = 6, depth 5) with kappa = 10 (kappa r = 0.16 at the
    # leaves, 1.25 at level 2), in the benchmark's FP16X3 mode and in FP32, at 64 sampled targets
    w = WORKLOADS["cube1m_p6_d5"]
    x, q = w.points(), w.charges()
    idx = sample_indices(w.n, 64)
    ref = kifmm.evaluate(x.astype(np.float64), q.astype(np.float64), w.p, w.depth, w.origin, w.side,
                         pinv_rtol=PINV_RTOL, sample=idx, kappa=10.0)
    for precision in ("fp16x3", "fp32"):
        f = make_fmm(x, w.p, w.depth, precision, (w.origin, w.side), kernel="yukawa", kappa=10.0)
        phi, grad = run(f, q)
        f.close()
        assert rel(phi[idx], ref.phi) < 1e-5, (precision, rel(phi[idx], ref.phi))
        assert rel(grad[idx], ref.grad) < 1e-4, (precision, rel(grad[idx], ref.grad))
