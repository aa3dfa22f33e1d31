"""Pins of the oracle's second kernel, the modified Helmholtz (Yukawa) kernel
K(x, y) = exp(-kappa |x - y|) / (4 pi |x - y|), the free-space Green's function of
(Delta - kappa^2): closed forms, the PDE itself, kappa -> 0, two independent direct sums, and
the kernel-independent FMM against the direct sum (no GPU)."""
import numpy as np
import pytest

from oracle import direct, kifmm
from synth import cube_points, charges

KAPPA = 3.0


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("impl", ["numpy", "c"])
def test_two_points_closed_form(impl):
    y = np.array([[0.1, -0.2, 0.3]])
    x = np.array([[0.6, 0.1, -0.1]])
    q = np.array([2.5])
    d = x[0] - y[0]
    r = np.linalg.norm(d)
    f = direct.direct_numpy if impl == "numpy" else direct.direct_c
    phi, grad = f(x, y, q, kappa=KAPPA)
    assert phi[0] == pytest.approx(2.5 * np.exp(-KAPPA * r) / (4 * np.pi * r), rel=1e-14)
    g_exact = -2.5 * (1 + KAPPA * r) * np.exp(-KAPPA * r) * d / (4 * np.pi * r ** 3)
    np.testing.assert_allclose(grad[0], g_exact, rtol=1e-13)


def test_kappa_zero_is_laplace_and_implementations_agree():
    x, q = cube_points(300, seed=5).astype(np.float64), charges(300, "u11", seed=6).astype(np.float64)
    p0, g0 = direct.direct_c(x, x, q)
    pk, gk = direct.direct_c(x, x, q, kappa=0.0)
    assert np.array_equal(p0, pk) and np.array_equal(g0, gk)
    pn, gn = direct.direct_numpy(x, x, q, kappa=KAPPA)
    pc, gc = direct.direct_c(x, x, q, kappa=KAPPA)
    assert rel(pc, pn) < 1e-13 and rel(gc, gn) < 1e-13
    # screening: every pair's contribution shrinks by exp(-kappa r)
    assert np.all(np.abs(pc) <= np.abs(direct.direct_c(x, x, np.abs(q))[0]) + 1e-15)


def test_greens_function_pde():
    # (Delta - kappa^2) G = 0 away from the source, by a central-difference Laplacian
    y, q = np.zeros((1, 3)), np.array([1.0])
    x0 = np.array([0.3, 0.2, -0.25])
    phi = lambda pt: direct.direct_numpy(pt.reshape(1, 3), y, q, gradient=False, kappa=KAPPA)[0][0]
    lap_h = lambda h: sum(phi(x0 + h * e) + phi(x0 - h * e) - 2 * phi(x0) for e in np.eye(3)) / h ** 2
    lap = (4 * lap_h(1e-3) - lap_h(2e-3)) / 3  # Richardson: the O(h^2) term cancels
    assert lap == pytest.approx(KAPPA ** 2 * phi(x0), rel=1e-7)


def test_gradient_is_derivative_of_potential():
    rng = np.random.default_rng(4)
    y, q = rng.random((40, 3)), rng.standard_normal(40)
    x = np.array([[1.7, -0.4, 0.9]])
    _, g = direct.direct_c(x, y, q, kappa=KAPPA)
    h = 1e-5
    for a in range(3):
        e = np.zeros((1, 3))
        e[0, a] = h
        fd = (direct.direct_c(x + e, y, q, False, KAPPA)[0] - direct.direct_c(x - e, y, q, False, KAPPA)[0]) / (2 * h)
        assert g[0, a] == pytest.approx(fd[0], rel=1e-7)


@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_direct_sum(depth):
    x, q = cube_points(1500, seed=1).astype(np.float64), charges(1500, "u11", seed=2).astype(np.float64)
    res = kifmm.evaluate(x, q, 4, depth, (0, 0, 0), 1.0, kappa=KAPPA)
    p, g = direct.direct_self(x, q, kappa=KAPPA)
    assert rel(res.phi, p) < 1e-13 and rel(res.grad, g) < 1e-13


def test_error_decreases_with_order():
    x, q = cube_points(3000, seed=3).astype(np.float64), charges(3000, "u01", seed=4).astype(np.float64)
    p_ref, g_ref = direct.direct_self(x, q, kappa=KAPPA)
    errs = []
    for p in (3, 4, 6):
        res = kifmm.evaluate(x, q, p, 3, (0, 0, 0), 1.0, kappa=KAPPA)
        errs.append(rel(res.phi, p_ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5


def test_level_operators_are_not_rescalings():
    # Laplace operators of two levels differ by the factor 2 (homogeneity); the screened
    # kernel's do not, which is why the GPU path builds them per level for it
    ops_l = kifmm.build_operators(4, 1.0, 3)
    ops_y = kifmm.build_operators(4, 1.0, 3, kappa=KAPPA)
    a, b = ops_l.m2l[(2, 0)], ops_l.m2l[(3, 0)]
    assert rel(b, 2.0 * a) < 1e-12
    a, b = ops_y.m2l[(2, 0)], ops_y.m2l[(3, 0)]
    assert rel(b, 2.0 * a) > 1e-2


def test_adjoint_is_explicit_transpose():
    n = 300
    x = cube_points(n, seed=8).astype(np.float64)
    tr_depth, p = 2, 3
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(kifmm.evaluate(x, e, p, tr_depth, (0, 0, 0), 1.0, gradient=False, kappa=KAPPA).phi)
    a = np.stack(cols, axis=1)
    g = charges(n, "normal", seed=9).astype(np.float64)
    psi = kifmm.adjoint(x, g, p, tr_depth, (0, 0, 0), 1.0, kappa=KAPPA)
    assert rel(psi, a.T @ g) < 1e-12
