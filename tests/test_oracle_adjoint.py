"""Pins of the oracle's transposed FMM pass and of the energy derivatives (C-10 reading:
the tree is held fixed, position derivatives come from the kernel gradient)."""
import numpy as np
import pytest

from oracle import direct, kifmm
from synth import cube_points, sphere_points, charges


def _explicit_matrix(x, p, depth, ops):
    n = len(x)
    cols = []
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        cols.append(kifmm.evaluate(x, e, p, depth, gradient=False, ops=ops).phi)
    return np.stack(cols, axis=1)


def test_adjoint_is_explicit_transpose():
    x = sphere_points(160).astype(np.float64)
    p, depth = 3, 3
    tr = kifmm.otree.build_tree(x, depth)
    ops = kifmm.build_operators(p, tr.side, depth)
    a = _explicit_matrix(x, p, depth, ops)
    g = charges(160, "normal", seed=2).astype(np.float64)
    psi = kifmm.adjoint(x, g, p, depth, ops=ops)
    np.testing.assert_allclose(psi, a.T @ g, rtol=1e-11, atol=1e-12 * np.abs(psi).max())
    # the FMM map is not symmetric, but close to the symmetric direct-sum matrix
    asym = np.linalg.norm(a - a.T) / np.linalg.norm(a)
    assert 0 < asym < 1e-2


@pytest.mark.parametrize("dist", ["cube", "sphere"])
def test_dot_product_identity(dist):
    n = 3000
    x = (cube_points(n) if dist == "cube" else sphere_points(n)).astype(np.float64)
    q = charges(n, "u11").astype(np.float64)
    g = charges(n, "normal", seed=2).astype(np.float64)
    aq = kifmm.evaluate(x, q, 5, 3, gradient=False).phi
    atg = kifmm.adjoint(x, g, 5, 3)
    lhs, rhs = g @ aq, atg @ q
    assert abs(lhs - rhs) <= 1e-12 * np.abs(g).sum() * np.abs(aq).max()


def test_energy_charge_derivative_finite_difference():
    # E(q) = 1/2 q . A q is quadratic, so the central difference is exact up to rounding
    n = 800
    x = cube_points(n).astype(np.float64)
    q = charges(n, "normal").astype(np.float64)
    tr = kifmm.otree.build_tree(x, 3)
    ops = kifmm.build_operators(4, tr.side, 3)
    phi = kifmm.evaluate(x, q, 4, 3, gradient=False, ops=ops).phi
    dedq = 0.5 * phi + 0.5 * kifmm.adjoint(x, q, 4, 3, ops=ops)

    def energy(qq):
        return 0.5 * qq @ kifmm.evaluate(x, qq, 4, 3, gradient=False, ops=ops).phi

    h = 1e-3
    for k in (0, 123, 799):
        e = np.zeros(n)
        e[k] = h
        fd = (energy(q + e) - energy(q - e)) / (2 * h)
        assert fd == pytest.approx(dedq[k], rel=1e-8, abs=1e-10)


def test_energy_position_derivative_direct_sum():
    # dE/dx_k = q_k grad phi(x_k) for E = 1/2 q . phi of the direct sum (Richardson FD)
    n = 400
    x = cube_points(n).astype(np.float64)
    q = charges(n, "normal").astype(np.float64)
    _, grad = direct.direct_self(x, q)

    def energy(xx):
        phi, _ = direct.direct_c(xx, xx, q, gradient=False)
        return 0.5 * q @ phi

    def fd(k, axis, h):
        e = np.zeros_like(x)
        e[k, axis] = h
        return (energy(x + e) - energy(x - e)) / (2 * h)

    for k in (3, 77, 250):
        for axis in range(3):
            h = 1e-3
            rich = (4 * fd(k, axis, h / 2) - fd(k, axis, h)) / 3
            assert rich == pytest.approx(q[k] * grad[k, axis], rel=1e-5, abs=1e-7)
