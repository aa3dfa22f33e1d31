"""Pins of the oracle kiFMM (Algorithm 1, uniform branches) against the direct sum, closed
forms and exact identities.  Each operator is checked on its own against the field it must
reproduce, so a dropped term, a wrong sign or a transposed operand fails here."""
import numpy as np
import pytest

from oracle import direct, kifmm, tree as otree
from oracle.kifmm import (ALPHA_INNER, ALPHA_OUTER, build_operators, kernel_matrix, n_surface,
                          surface)
from synth import cube_points, sphere_points, charges


def rel(a, b):
    return np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b))


@pytest.mark.parametrize("depth", [0, 1])
def test_shallow_tree_is_direct_sum(depth):
    x = cube_points(1200).astype(np.float64)
    q = charges(1200, "u11").astype(np.float64)
    r = kifmm.evaluate(x, q, 4, depth)
    phi, grad = direct.direct_self(x, q)
    assert rel(r.phi, phi) < 1e-13
    assert rel(r.grad, grad) < 1e-13


def test_error_decreases_with_order():
    x = cube_points(2000).astype(np.float64)
    q = charges(2000, "u01").astype(np.float64)
    phi, grad = direct.direct_self(x, q)
    errs = [rel(kifmm.evaluate(x, q, p, 3, (0, 0, 0), 1.0, gradient=False).phi, phi)
            for p in range(2, 9)]
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-3 and errs[-1] < 1e-7


def test_sphere_p6_accuracy():
    x = sphere_points(4000).astype(np.float64)
    q = charges(4000, "u01").astype(np.float64)
    r = kifmm.evaluate(x, q, 6, 4, (-1, -1, -1), 2.0)
    phi, grad = direct.direct_self(x, q)
    assert rel(r.phi, phi) < 1e-5
    assert rel(r.grad, grad) < 1e-4


def _box_sources(n, centre, r, seed):
    rng = np.random.default_rng(seed)
    return centre + (2 * rng.random((n, 3)) - 1) * r, rng.standard_normal(n)


def _far_points(centre, r, seed, m=64, dist=(3.2, 6.0)):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((m, 3))
    d /= np.abs(d).max(axis=1, keepdims=True)          # on the cube of radius 1
    return centre + d * r * rng.uniform(*dist, (m, 1))


@pytest.mark.parametrize("p", [3, 5, 7])
def test_s2u_reproduces_far_field(p):
    r = 0.125
    c = np.array([0.3, -0.2, 0.5])
    y, s = _box_sources(40, c, r, 1)
    uc2e = kifmm.pinv(kernel_matrix(surface(p, 0 * c, r, ALPHA_OUTER),
                                    surface(p, 0 * c, r, ALPHA_INNER)), 1e-12)
    u = uc2e @ (kernel_matrix(surface(p, c, r, ALPHA_OUTER), y) @ s)
    far = _far_points(c, r, 2)
    err = rel(kernel_matrix(far, surface(p, c, r, ALPHA_INNER)) @ u, kernel_matrix(far, y) @ s)
    assert err < {3: 5e-3, 5: 2e-4, 7: 1e-5}[p]


def test_monopole_far_field():
    p, r = 4, 0.25
    c = np.zeros(3)
    y, s = _box_sources(30, c, r, 3)
    s = np.abs(s)
    ops = kifmm.pinv(kernel_matrix(surface(p, c, r, ALPHA_OUTER), surface(p, c, r, ALPHA_INNER)), 1e-12)
    u = ops @ (kernel_matrix(surface(p, c, r, ALPHA_OUTER), y) @ s)
    assert u.sum() == pytest.approx(s.sum(), rel=1e-3)    # equivalent charge = total charge
    far = np.array([[1000.0, 0.0, 0.0]])
    val = (kernel_matrix(far, surface(p, c, r, ALPHA_INNER)) @ u)[0]
    assert val == pytest.approx(s.sum() / (4 * np.pi * 1000.0), rel=1e-3)


def test_u2u_and_d2d_and_vli_reproduce_fields():
    p, depth, side = 6, 3, 1.0
    ops = build_operators(p, side, depth, 1e-12)
    lvl = 2
    r_p, r_c = side / 2 ** (lvl + 1), side / 2 ** (lvl + 2)
    cP = np.array([0.375, 0.375, 0.625])
    # U2U: children's u (built by S2U of random sources) -> parent's u, checked far away
    ys, ss, u_par_q = [], [], np.zeros(n_surface(p))
    for c in range(8):
        cc = cP + (2 * kifmm.child_offset(c) - 1) * r_c
        y, s = _box_sources(10, cc, r_c, 10 + c)
        uc = ops.uc2e[lvl + 1] @ (kernel_matrix(surface(p, cc, r_c, ALPHA_OUTER), y) @ s)
        u_par_q += ops.m2m[(lvl, c)] @ uc
        ys.append(y); ss.append(s)
    y, s = np.vstack(ys), np.concatenate(ss)
    uP = ops.uc2e[lvl] @ u_par_q
    far = _far_points(cP, r_p, 4)
    assert rel(kernel_matrix(far, surface(p, cP, r_p, ALPHA_INNER)) @ uP,
               kernel_matrix(far, y) @ s) < 1e-5
    # VLI: a well-separated source box's u -> target box's d, checked inside the target box
    tv = otree.transfer_vectors()
    t = 200
    ca = cP + 2 * r_p * tv[t]
    ya, sa = _box_sources(30, ca, r_p, 20)
    ua = ops.uc2e[lvl] @ (kernel_matrix(surface(p, ca, r_p, ALPHA_OUTER), ya) @ sa)
    dP = ops.dc2e[lvl] @ (ops.m2l[(lvl, t)] @ ua)
    inside = cP + (2 * np.random.default_rng(5).random((50, 3)) - 1) * r_p
    want = kernel_matrix(inside, ya) @ sa
    assert rel(kernel_matrix(inside, surface(p, cP, r_p, ALPHA_OUTER)) @ dP, want) < 1e-5
    # D2D: parent's d -> child's d, checked inside the child
    for c in (0, 5):
        cc = cP + (2 * kifmm.child_offset(c) - 1) * r_c
        dc = ops.dc2e[lvl + 1] @ (ops.l2l[(lvl + 1, c)] @ dP)
        pts = cc + (2 * np.random.default_rng(6 + c).random((40, 3)) - 1) * r_c
        assert rel(kernel_matrix(pts, surface(p, cc, r_c, ALPHA_OUTER)) @ dc,
                   kernel_matrix(pts, ya) @ sa) < 1e-5


def test_transfer_operator_transpose_identity():
    ops = build_operators(4, 1.0, 2, m2l_levels=[2])
    tv = otree.transfer_vectors()
    neg = otree.transfer_index(-tv)
    for t in range(316):
        # equal up to the rounding of the coordinate differences
        np.testing.assert_allclose(ops.m2l[(2, int(neg[t]))], ops.m2l[(2, t)].T, rtol=1e-14)


def test_level_homogeneity():
    # K is homogeneous of degree -1: operators at level l are 2^l (or 2^-l) times level 0's
    ops = build_operators(5, 1.0, 4, m2l_levels=[2, 4])
    for level in range(1, 5):
        s = 2.0 ** level
        assert rel(ops.uc2e[level], ops.uc2e[0] / s) < 1e-12
        assert rel(ops.dc2e[level], ops.dc2e[0] / s) < 1e-12
        for c in range(8):
            if level < 4:
                assert rel(ops.m2m[(level, c)], ops.m2m[(0, c)] * s) < 1e-13
            assert rel(ops.l2l[(level, c)], ops.l2l[(1, c)] * s / 2) < 1e-13
    for t in (0, 100, 315):
        assert rel(ops.m2l[(4, t)], ops.m2l[(2, t)] * 4) < 1e-13


def test_grouped_vli_equals_pairwise():
    x = sphere_points(1500).astype(np.float64)
    q = charges(1500, "u01").astype(np.float64)
    sample = np.arange(0, 1500, 37)
    a = kifmm.evaluate(x, q, 3, 3, sample=sample, m2l="grouped")
    b = kifmm.evaluate(x, q, 3, 3, sample=sample, m2l="pairwise")
    assert rel(a.phi, b.phi) < 1e-13
    assert rel(a.grad, b.grad) < 1e-12


def test_sampled_equals_full():
    x = cube_points(3000).astype(np.float64)
    q = charges(3000, "u11").astype(np.float64)
    full = kifmm.evaluate(x, q, 4, 3)
    sample = np.array([5, 17, 2999, 1000, 42])
    part = kifmm.evaluate(x, q, 4, 3, sample=sample)
    np.testing.assert_allclose(part.phi, full.phi[sample], rtol=1e-11)
    np.testing.assert_allclose(part.grad, full.grad[sample], rtol=1e-10)


def test_near_plus_far_is_whole():
    x = cube_points(2000).astype(np.float64)
    q = charges(2000, "u11").astype(np.float64)
    whole = kifmm.evaluate(x, q, 4, 3)
    near = kifmm.evaluate(x, q, 4, 3, parts=("near",))
    far = kifmm.evaluate(x, q, 4, 3, parts=("far",))
    np.testing.assert_allclose(near.phi + far.phi, whole.phi, rtol=1e-12)
