"""Gradient-only ("force") evaluation: fmm_evaluate with phi == NULL.

Its gradients come from the same arithmetic in the same order as those of the full evaluation,
so they must match bit for bit (the near-field kernel only drops its potential sums); the full
evaluation itself is pinned against the oracle elsewhere, and once more here at the FP32 bar.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from oracle import kifmm
from synth import cube_points, sphere_points, charges
from gpu_helpers import PINV_RTOL, make_fmm, rel, run

pytestmark = pytest.mark.gpu
BALL = ((-1, -1, -1), 2.0)


@pytest.mark.parametrize("kernel", ["laplace", "yukawa"])
@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp16x3", "bf16x6"])
def test_gradient_only_equals_full_gradient(precision, kernel):
    x, q = sphere_points(60_000), charges(60_000, "u01")
    f = make_fmm(x, 6, 4, precision, BALL, kernel=kernel, kappa=3.0 if kernel == "yukawa" else 0.0)
    dt = torch.float64 if precision == "fp64" else torch.float32
    qd = torch.from_numpy(q).to("cuda", dt)
    _, g_full = f.evaluate(qd)
    phi, g_only = f.evaluate(qd, potential=False)
    torch.cuda.synchronize()
    assert phi is None
    assert torch.equal(g_full, g_only)
    for part in (pkg.PART_NEAR, pkg.PART_FAR):
        _, a = f.evaluate(qd, parts=part)
        _, b = f.evaluate(qd, parts=part, potential=False)
        assert torch.equal(a, b)


def test_gradient_only_against_oracle_and_host_buffers():
    x, q = cube_points(30_000), charges(30_000, "u11")
    dom = ((0, 0, 0), 1.0)
    f = make_fmm(x, 5, 3, "fp32", dom)
    g = np.zeros((len(x), 3), np.float32)
    f.evaluate_into(np.ascontiguousarray(q), None, g)          # host pointers, phi NULL
    ref = kifmm.evaluate(x.astype(np.float64), q.astype(np.float64), 5, 3, *dom, pinv_rtol=PINV_RTOL)
    assert rel(g, ref.grad) < 1e-4
    _, g_dev = run(f, q)
    assert np.array_equal(g.astype(np.float64), g_dev)


def test_gradient_only_argument_errors():
    x, q = cube_points(2000), charges(2000, "u11")
    f = make_fmm(x, 4, 2, "fp32", None)
    qd = torch.from_numpy(q).cuda()
    L = pkg.lib()
    assert L.fmm_evaluate(f._ctx, ctypes.c_void_p(qd.data_ptr()), None, None) == 1
    f2 = make_fmm(x, 4, 2, "fp32", None, with_gradient=False)
    g = torch.empty(len(x), 3, device="cuda")
    assert L.fmm_evaluate(f2._ctx, ctypes.c_void_p(qd.data_ptr()), None, ctypes.c_void_p(g.data_ptr())) == 1
    # the contexts stay usable
    phi, grad = f.evaluate(qd)
    torch.cuda.synchronize()
    assert torch.isfinite(phi).all() and torch.isfinite(grad).all()
