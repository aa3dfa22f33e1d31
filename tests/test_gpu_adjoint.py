"""The transposed FMM pass (psi = A^T g) and the autograd wrapper (energy derivatives)."""
import numpy as np
import pytest
import torch

import paper_2604_19243_gb300 as pkg
from oracle import direct, kifmm
from synth import cube_points, sphere_points, charges
from gpu_helpers import PINV_RTOL, make_fmm, rel, run

pytestmark = pytest.mark.gpu
CUBE = ((0, 0, 0), 1.0)


def _adj(f, g):
    dt = torch.float64 if f.precision == "fp64" else torch.float32
    psi, _ = f.adjoint(torch.from_numpy(g).to("cuda", dt))
    torch.cuda.synchronize()
    return psi.cpu().numpy().astype(np.float64)


def test_adjoint_is_explicit_transpose_fp64():
    n = 300
    x = sphere_points(n)
    f = make_fmm(x, 3, 3, "fp64", None)
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(run(f, e, gradient=False)[0])
    a = np.stack(cols, 1)
    g = charges(n, "normal", seed=2).astype(np.float64)
    psi = _adj(f, g)
    np.testing.assert_allclose(psi, a.T @ g, rtol=1e-10, atol=1e-12 * np.abs(psi).max())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_adjoint_matches_oracle_transpose(precision):
    n = 20_000
    x, g = cube_points(n), charges(n, "normal", seed=2)
    f = make_fmm(x, 5, 3, precision, CUBE)
    psi = _adj(f, g.astype(np.float64))
    ref = kifmm.adjoint(x.astype(np.float64), g.astype(np.float64), 5, 3, *CUBE, pinv_rtol=PINV_RTOL)
    assert rel(psi, ref) < (1e-8 if precision == "fp64" else 1e-5)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dot_product_identity(precision):
    n = 50_000
    x = sphere_points(n)
    q = charges(n, "u11").astype(np.float64)
    g = charges(n, "normal", seed=2).astype(np.float64)
    f = make_fmm(x, 6, 4, precision, None)
    aq = run(f, q, gradient=False)[0]
    atg = _adj(f, g)
    lhs, rhs = g @ aq, atg @ q
    scale = np.linalg.norm(g) * np.linalg.norm(aq)
    assert abs(lhs - rhs) / scale < (1e-12 if precision == "fp64" else 2e-6)


def test_autograd_energy_gradients():
    # E = 1/2 q . phi ; dE/dq = (phi + A^T q)/2 ; dE/dx_k = q_k grad phi(x_k) (C-10 reading)
    n = 40_000
    x = cube_points(n)
    qn = charges(n, "normal")
    f = make_fmm(x, 6, 4, "fp32", CUBE)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    qt = torch.from_numpy(qn).cuda().requires_grad_(True)
    e = pkg.fmm_energy(qt, xt, f)
    e.backward()
    dq = qt.grad.cpu().numpy().astype(np.float64)
    dx = xt.grad.cpu().numpy().astype(np.float64)
    q64 = qn.astype(np.float64)
    phi_d, grad_d = direct.direct_self(x.astype(np.float64), q64)
    assert abs(float(e.detach()) - 0.5 * q64 @ phi_d) / abs(0.5 * q64 @ phi_d) < 1e-5
    assert rel(dq, phi_d) < 1e-5                      # the symmetric direct-sum derivative
    assert rel(dx, q64[:, None] * grad_d) < 1e-4
    # central differences of the FP64 direct-sum energy (Richardson): moving x_k changes only
    # the pairs (k, j), so E(x + h e) - E(x - h e) = q_k [Phi_k(x_k + h e) - Phi_k(x_k - h e)]
    # with Phi_k the potential of all the other points
    xs = x.astype(np.float64)
    for k in (11, 2024, 39_000):
        others = np.delete(np.arange(n), k)
        for a in range(3):
            def fd(h):
                t = np.repeat(xs[k:k + 1], 2, axis=0)
                t[0, a] += h
                t[1, a] -= h
                p, _ = direct.direct_c(t, xs[others], q64[others], gradient=False)
                return q64[k] * (p[0] - p[1]) / (2 * h)
            rich = (4 * fd(5e-4) - fd(1e-3)) / 3
            assert dx[k, a] == pytest.approx(rich, rel=2e-3, abs=1e-3 * np.abs(dx).max())


def test_autograd_charges_only():
    n = 10_000
    x, q = cube_points(n), charges(n, "u11")
    f = make_fmm(x, 4, 3, "fp32", CUBE)
    qt = torch.from_numpy(q).cuda().requires_grad_(True)
    phi = pkg.FmmFunction.apply(qt, torch.from_numpy(x).cuda(), f)
    w = torch.from_numpy(charges(n, "normal", seed=4)).cuda()
    (phi * w).sum().backward()
    want = _adj(f, w.cpu().numpy().astype(np.float64))
    assert rel(qt.grad.cpu().numpy(), want) < 1e-6
