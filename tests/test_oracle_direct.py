"""Pins of the oracle's direct sum (Eq. 1, Laplace kernel of Eq. 2) against closed forms,
invariants and an independent SciPy formulation."""
import json
import os

import numpy as np
import pytest
from scipy.spatial.distance import cdist

from oracle import direct
from synth import cube_points, charges

GOLD = os.path.join(os.path.dirname(__file__), "golden")
FOURPI = 4.0 * np.pi


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


@pytest.mark.parametrize("impl", ["numpy", "c"])
def test_two_points_closed_form(impl):
    g = _gold("direct_closed_forms.json")["two_points"]
    x = np.array(g["x"])
    q = np.array(g["q"])
    f = direct.direct_numpy if impl == "numpy" else direct.direct_c
    phi, grad = f(x, x, q)
    np.testing.assert_allclose(phi * FOURPI, g["phi_times_4pi"], rtol=1e-14)
    np.testing.assert_allclose(grad * FOURPI, g["grad_times_4pi"], rtol=1e-13, atol=1e-16)


@pytest.mark.parametrize("impl", ["numpy", "c"])
def test_cube_corners_closed_form(impl):
    corners = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], float)
    x = np.vstack([corners, np.zeros((1, 3))])
    q = np.array([1.0] * 8 + [0.0])
    f = direct.direct_numpy if impl == "numpy" else direct.direct_c
    phi, grad = f(x, x, q)
    assert phi[8] * FOURPI == pytest.approx(8.0 / np.sqrt(3.0), rel=1e-14)
    corner = 1.5 + 1.5 / np.sqrt(2.0) + 0.5 / np.sqrt(3.0)
    np.testing.assert_allclose(phi[:8] * FOURPI, corner, rtol=1e-14)
    np.testing.assert_allclose(grad[8], 0.0, atol=1e-15)
    # corner gradient points away from the cube (field of positive charges pushes outward):
    # -grad phi is outward, so grad phi . corner < 0
    assert np.all(np.einsum("ij,ij->i", grad[:8], corners) < 0)


def test_self_exclusion_and_coincident():
    phi, grad = direct.direct_c(np.zeros((1, 3)), np.zeros((1, 3)), np.ones(1))
    assert phi[0] == 0.0 and np.all(grad == 0.0)
    x = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3], [1.1, 0.2, 0.3]])
    q = np.array([1.0, 2.0, 3.0])
    phi, _ = direct.direct_c(x, x, q)
    # the coincident pair is skipped: point 0 sees only point 2 at distance 1
    assert phi[0] * FOURPI == pytest.approx(3.0, rel=1e-14)
    assert phi[2] * FOURPI == pytest.approx(3.0, rel=1e-14)


def test_linearity_in_charges():
    x = cube_points(500).astype(np.float64)
    q1 = charges(500, "u11", seed=11).astype(np.float64)
    q2 = charges(500, "normal", seed=12).astype(np.float64)
    a, b = 0.7, -1.3
    p1, g1 = direct.direct_c(x, x, q1)
    p2, g2 = direct.direct_c(x, x, q2)
    p3, g3 = direct.direct_c(x, x, a * q1 + b * q2)
    np.testing.assert_allclose(p3, a * p1 + b * p2, rtol=0, atol=1e-14 * np.abs(p3).max())
    np.testing.assert_allclose(g3, a * g1 + b * g2, rtol=0, atol=1e-14 * np.abs(g3).max())


def test_against_scipy_cdist():
    x = cube_points(700).astype(np.float64)
    y = cube_points(900, seed=5).astype(np.float64)
    q = charges(900, "u11").astype(np.float64)
    r = cdist(x, y)
    ref = (q[None, :] / r).sum(axis=1) / FOURPI
    # gradient from the kernel derivative, written independently with cdist's distances
    diff = x[:, None, :] - y[None, :, :]
    gref = -(q[None, :, None] * diff / r[:, :, None] ** 3).sum(axis=1) / FOURPI
    for f in (direct.direct_c, direct.direct_numpy):
        phi, grad = f(x, y, q)
        np.testing.assert_allclose(phi, ref, rtol=1e-12)
        np.testing.assert_allclose(grad, gref, rtol=1e-10, atol=1e-12 * np.abs(gref).max())


def test_gradient_is_derivative_of_potential():
    rng = np.random.default_rng(7)
    y = rng.random((50, 3))
    q = rng.standard_normal(50)
    x0 = np.array([[1.7, -0.4, 0.9]])
    _, g = direct.direct_c(x0, y, q)
    h = 1e-5
    fd = np.zeros(3)
    for k in range(3):
        e = np.zeros((1, 3)); e[0, k] = h
        fd[k] = (direct.direct_c(x0 + e, y, q)[0][0] - direct.direct_c(x0 - e, y, q)[0][0]) / (2 * h)
    np.testing.assert_allclose(g[0], fd, rtol=1e-7)


def test_grouped_ranges_match_full_sum():
    x = cube_points(300).astype(np.float64)
    q = charges(300, "u01").astype(np.float64)
    full, gfull = direct.direct_c(x, x, q)
    # split the sources into three ranges and the targets into two groups
    pot, grad = direct.grouped_sum([0, 120, 300], x, [0, 3, 6],
                                   [[0, 100], [100, 250], [250, 300]] * 2, x, q)
    np.testing.assert_allclose(pot, full, rtol=1e-13)
    np.testing.assert_allclose(grad, gfull, rtol=1e-12, atol=1e-14)
