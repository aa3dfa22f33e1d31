"""Pins of the oracle's Helmholtz kernel exp(i k |x - y|) / (4 pi |x - y|) with complex
densities (Eq. 1 with F = C): closed forms, the Helmholtz equation, the small-k expansion,
complex linearity, two independent direct sums and the kernel-independent FMM (no GPU)."""
import numpy as np
import pytest

from oracle import direct, kifmm
from synth import cube_points, charges

K = 2.0 * np.pi    # one wavelength across the unit cube


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def cq(n, seed):
    return charges(n, "u11", seed=seed).astype(np.float64) + 1j * charges(n, "u11", seed=seed + 100)


@pytest.mark.parametrize("impl", ["numpy", "c"])
def test_two_points_closed_form(impl):
    y, x = np.array([[0.1, -0.2, 0.3]]), np.array([[0.6, 0.1, -0.1]])
    q = np.array([2.5 - 0.75j])
    d = x[0] - y[0]
    r = np.linalg.norm(d)
    f = direct.direct_numpy if impl == "numpy" else direct.direct_c
    phi, grad = f(x, y, q, wavenumber=K)
    g = np.exp(1j * K * r) / (4 * np.pi * r)
    assert abs(phi[0] - q[0] * g) < 1e-15
    g_exact = q[0] * g * (1j * K * r - 1.0) * d / r ** 2
    np.testing.assert_allclose(grad[0], g_exact, rtol=1e-13)


def test_helmholtz_equation():
    # (Delta + k^2) G = 0 away from the source, by a Richardson-extrapolated difference Laplacian
    y, q, x0 = np.zeros((1, 3)), np.array([1.0 + 0.5j]), np.array([0.3, 0.2, -0.25])
    phi = lambda pt: direct.direct_numpy(pt.reshape(1, 3), y, q, gradient=False, wavenumber=K)[0][0]
    lap_h = lambda h: sum(phi(x0 + h * e) + phi(x0 - h * e) - 2 * phi(x0) for e in np.eye(3)) / h ** 2
    lap = (4 * lap_h(1e-3) - lap_h(2e-3)) / 3
    assert abs(lap + K ** 2 * phi(x0)) < 1e-6 * abs(K ** 2 * phi(x0))


def test_small_wavenumber_expansion():
    # exp(i k r) / r = 1/r + i k - k^2 r / 2 + O(k^3): the real part is Laplace, the imaginary
    # part is k sum_j q_j / (4 pi) for real charges
    x, q = cube_points(400, seed=5).astype(np.float64), charges(400, "u11", seed=6).astype(np.float64)
    k = 1e-5
    ph, gh = direct.direct_c(x, x, q.astype(np.complex128), wavenumber=k)
    pl, gl = direct.direct_c(x, x, q)
    assert rel(ph.real, pl) < 1e-9 and rel(gh.real, gl) < 1e-9
    expect = k * (q.sum() - q) / (4 * np.pi)      # j != i
    assert rel(ph.imag, expect) < 1e-5


def test_complex_linearity_and_implementations_agree():
    x = cube_points(300, seed=7).astype(np.float64)
    q1 = charges(300, "u11", seed=8).astype(np.float64)
    q2 = charges(300, "u11", seed=9).astype(np.float64)
    p1, g1 = direct.direct_c(x, x, q1.astype(np.complex128), wavenumber=K)
    p2, g2 = direct.direct_c(x, x, q2.astype(np.complex128), wavenumber=K)
    p, g = direct.direct_c(x, x, q1 + 1j * q2, wavenumber=K)
    assert rel(p, p1 + 1j * p2) < 1e-14 and rel(g, g1 + 1j * g2) < 1e-14
    pn, gn = direct.direct_numpy(x, x, q1 + 1j * q2, wavenumber=K)
    assert rel(p, pn) < 1e-13 and rel(g, gn) < 1e-13


def test_gradient_is_derivative_of_potential():
    rng = np.random.default_rng(4)
    y, q = rng.random((40, 3)), rng.standard_normal(40) + 1j * rng.standard_normal(40)
    x = np.array([[1.7, -0.4, 0.9]])
    _, g = direct.direct_c(x, y, q, wavenumber=K)
    h = 1e-5
    for a in range(3):
        e = np.zeros((1, 3))
        e[0, a] = h
        fd = (direct.direct_c(x + e, y, q, False, wavenumber=K)[0] -
              direct.direct_c(x - e, y, q, False, wavenumber=K)[0]) / (2 * h)
        assert abs(g[0, a] - fd[0]) < 1e-7 * abs(fd[0])


@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_direct_sum(depth):
    x, q = cube_points(1500, seed=1).astype(np.float64), cq(1500, 2)
    res = kifmm.evaluate(x, q, 4, depth, (0, 0, 0), 1.0, wavenumber=K)
    p, g = direct.direct_self(x, q, wavenumber=K)
    assert rel(res.phi, p) < 1e-13 and rel(res.grad, g) < 1e-13


def test_error_decreases_with_order():
    x, q = cube_points(3000, seed=3).astype(np.float64), cq(3000, 4)
    p_ref, g_ref = direct.direct_self(x, q, wavenumber=K)
    errs = []
    for p in (3, 4, 6):
        res = kifmm.evaluate(x, q, p, 3, (0, 0, 0), 1.0, wavenumber=K)
        errs.append(rel(res.phi, p_ref))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-5, errs
