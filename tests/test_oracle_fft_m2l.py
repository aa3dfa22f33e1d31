"""Pins of the FFT form of the M2L (the lattice convolution of the kernel-independent M2L,
Section 2.2's FFT alternative to the BLAS form): it equals the dense kernel matrix from the two
surfaces' coordinates for every transfer vector (the convolution theorem), and the check
potentials it produces from fitted equivalent densities reproduce the sources' exact field, with
an error that falls with p."""
import numpy as np
import pytest

from oracle import fft_m2l, kifmm, tree as otree


@pytest.mark.parametrize("p", [4, 6, 8])
def test_fft_equals_the_dense_matrix(p):
    rng = np.random.default_rng(p)
    r = 0.5 / 8
    tv = otree.transfer_vectors()
    pick = range(len(tv)) if p == 4 else rng.choice(len(tv), 24, replace=False)
    u = rng.standard_normal((3, kifmm.n_surface(p)))
    for k in pick:
        t = tv[k]
        got = fft_m2l.m2l_fft(p, r, t, u)
        want = fft_m2l.m2l_dense(p, r, t, u)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max(), (p, t)


def test_fft_modified_helmholtz_equals_the_dense_matrix():
    rng = np.random.default_rng(1)
    p, r, kappa = 6, 0.1, 3.0
    u = rng.standard_normal(kifmm.n_surface(p))
    for t in ((2, 0, 0), (-3, 1, 2), (3, 3, -3)):
        got = fft_m2l.m2l_fft(p, r, t, u, kappa)
        want = fft_m2l.m2l_dense(p, r, t, u, kappa)
        assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_lattice_radius():
    assert fft_m2l.lattice_alpha(6) == 1.25
    for p in range(4, 11):
        a = fft_m2l.lattice_alpha(p)
        assert 1.0 < a < 2.0 and abs((p - 1) / a - round((p - 1) / a)) < 1e-12
    with pytest.raises(ValueError):
        fft_m2l.lattice_alpha(3)
    assert fft_m2l.surface_mask(6).sum() == kifmm.n_surface(6)


def test_fitted_densities_reproduce_the_far_field():
    """Sources in a box; densities on its lattice surface fitted to their potential on the 2.95
    check surface; the FFT M2L of those densities against the exact potential on the lattice
    surface of a V-list box."""
    rng = np.random.default_rng(3)
    r = 0.5 / 8
    src = (rng.random((100, 3)) * 2 - 1) * r
    q = rng.random(100) - 0.5
    errs = []
    for p in (4, 6, 8):
        a = fft_m2l.lattice_alpha(p)
        g = kifmm.surface_grid(p)
        uc, ue = kifmm.ALPHA_OUTER * r * g, a * r * g
        u = kifmm.pinv(kifmm.kernel_matrix(uc, ue), 1e-12) @ (kifmm.kernel_matrix(uc, src) @ q)
        worst = 0.0
        for t in ((2, 0, 0), (2, 2, 2), (3, -1, 0), (-3, 3, 3)):
            c = fft_m2l.m2l_fft(p, r, t, u)[0]
            exact = kifmm.kernel_matrix(a * r * g, src + 2.0 * r * np.asarray(t, float)) @ q   # source box at 2 r t
            worst = max(worst, np.linalg.norm(c - exact) / np.linalg.norm(exact))
        errs.append(worst)
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 1e-4 and errs[2] < 1e-5


def test_kifmm_with_fft_m2l_equals_the_dense_form():
    """The whole method with every VLI evaluated as lattice convolutions equals the grouped dense
    M2L on the same (lattice) surfaces."""
    from synth import cube_points, charges
    x = cube_points(1500).astype(np.float64)
    q = charges(1500, "u11").astype(np.float64)
    p, depth = 4, 3
    ops = kifmm.build_operators(p, 1.0, depth, alpha_inner=fft_m2l.lattice_alpha(p))
    a = kifmm.evaluate(x, q, p, depth, (0, 0, 0), 1.0, ops=ops, m2l="fft")
    b = kifmm.evaluate(x, q, p, depth, (0, 0, 0), 1.0, ops=ops, m2l="grouped")
    assert np.linalg.norm(a.phi - b.phi) / np.linalg.norm(b.phi) < 1e-10
    assert np.linalg.norm(a.grad - b.grad) / np.linalg.norm(b.grad) < 1e-10


def test_lattice_surfaces_meet_the_accuracy_bar_at_p6():
    from oracle import direct
    from synth import cube_points, charges
    x = cube_points(4000).astype(np.float64)
    q = charges(4000, "u11").astype(np.float64)
    ref, gref = direct.direct_self(x, q)
    ops = kifmm.build_operators(6, 1.0, 4, alpha_inner=fft_m2l.lattice_alpha(6))
    r = kifmm.evaluate(x, q, 6, 4, (0, 0, 0), 1.0, ops=ops)
    assert np.linalg.norm(r.phi - ref) / np.linalg.norm(ref) < 1e-5
    assert np.linalg.norm(r.grad - gref) / np.linalg.norm(gref) < 5e-5
