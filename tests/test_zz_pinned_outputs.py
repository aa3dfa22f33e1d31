"""Outputs in pinned host memory for the evaluations that end in run_evaluate besides the uniform
one: the adaptive evaluation and the FFT form of the M2L.  The output gather writes them over the
host link in the caller's order; they must equal the device outputs bit for bit.

This file is collected last so that a failure here comes after every other test has run."""
import pytest
import torch

from synth import charges, mixed_points
from gpu_helpers import make_fmm

pytestmark = pytest.mark.gpu
CUBE = ((0.0, 0.0, 0.0), 1.0)


def test_pinned_host_outputs_of_the_adaptive_and_fft_evaluations():
    n = 12_000
    x, q = mixed_points(n, radius=0.02), charges(n, "u11")
    qd = torch.from_numpy(q).cuda()
    ph, gh = torch.empty(n).pin_memory(), torch.empty(n, 3).pin_memory()
    f = make_fmm(x, 4, 7, "fp32", CUBE)
    f.adaptive_setup(16)
    pd, gd = f.adaptive_evaluate(qd)
    f.adaptive_evaluate_into(qd, ph, gh)
    assert torch.equal(ph, pd.cpu()) and torch.equal(gh, gd.cpu())
    f.close()
    g = make_fmm(x, 6, 4, "fp32", CUBE, m2l="fft")
    pd, gd = g.evaluate(qd)
    g.evaluate_into(qd, ph, gh)
    assert torch.equal(ph, pd.cpu()) and torch.equal(gh, gd.cpu())
    g.close()
