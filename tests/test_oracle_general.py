"""Pins of the general (non-Hermitian) FEAST oracle against what the
mathematics fixes: the whole-circle quadrature at the center and against the
Hermitian half-circle rule, the filter against the eigendecomposition of a
planted matrix, the end result against planted spectra, the iterates round
by round against subspace iteration on rho(A), one-round exactness on the
full space, and the Hermitian special case."""
import numpy as np
import pytest

from oracle.feast import feast_solve
from oracle.general import (factor_circle, feast_solve_general, filter_apply_general, norm2_estimate_general,
                            rayleigh_ritz_general)
from oracle.quadrature import circle_filter, circle_nodes, contour_nodes, rational_filter
from workloads import planted_general, random_subspace, spectrum_disk, haar_unitary, planted_matrix


@pytest.mark.parametrize("n_c", [2, 5, 8, 16])
def test_circle_rule_is_exact_at_the_center(n_c):
    # rho(c) = sum_k w_k / (r e^{i theta_k}) = sum_k omega_k / 4 over both
    # halves = 2 * 2 / 4 = 1 exactly (up to rounding)
    c, r = 0.3 - 0.7j, 2.5
    z, w = circle_nodes(c, r, n_c)
    assert abs(circle_filter(c, z, w) - 1.0) < 1e-15
    assert np.allclose(np.abs(z - c), r, rtol=0, atol=1e-15)


def test_circle_rule_on_the_real_line_is_the_hermitian_rule():
    # a real center: the lower nodes are the conjugates, so for real lambda
    # the whole-circle filter is sum_j 2 Re(w_j / (z_j - lambda)), the
    # (separately pinned) half-circle rule of the Hermitian case
    z, w = circle_nodes(0.5, 1.5, 8)
    zu, wu = contour_nodes(-1.0, 2.0, 8)
    lam = np.linspace(-3.0, 4.0, 71)
    rho = circle_filter(lam, z, w)
    assert np.max(np.abs(rho - rational_filter(lam, zu, wu))) < 1e-14
    assert np.max(np.abs(rho.imag)) < 1e-15
    assert np.allclose(z[8:], np.conj(z[:8]), rtol=0, atol=0) and np.allclose(w[8:], np.conj(w[:8]), rtol=0, atol=0)


def test_circle_rule_approaches_the_indicator_of_the_disk():
    # (1/2 pi i) \oint dz / (z - lambda) is 1 inside the circle, 0 outside;
    # the Gauss rule converges to it away from the circle
    c, r = 0.1 + 0.2j, 1.0
    inside = c + 0.5 * np.exp(1j * np.linspace(0.0, 2 * np.pi, 13))
    outside = c + 3.0 * np.exp(1j * np.linspace(0.0, 2 * np.pi, 13))
    errs = []
    for n_c in (4, 8, 16):
        z, w = circle_nodes(c, r, n_c)
        errs.append(max(np.max(np.abs(circle_filter(inside, z, w) - 1.0)),
                        np.max(np.abs(circle_filter(outside, z, w)))))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-4


@pytest.mark.parametrize("real", [False, True])
def test_filter_matches_the_eigendecomposition(real):
    # rho(A) X by resolvent solves against V diag(rho(lambda_i)) V^{-1} X
    # with the planted eigenvectors
    n, n_c = 40, 6
    lam = spectrum_disk(3, n, 8, center=0.2, radius=1.0, real_pairs=real)
    A, V = planted_general(lam, 3, cond=5.0, real=real)
    z, w, lus = factor_circle(A, 0.2, 1.0, n_c)
    X = random_subspace(n, 5, 4, complex_=True)
    Y = filter_apply_general(w, lus, X)
    ref = (V * circle_filter(lam, z, w)[None, :]) @ np.linalg.solve(V, X)
    assert np.max(np.abs(Y - ref)) < 1e-11 * np.max(np.abs(ref))


def test_norm_estimate_and_rayleigh_ritz_on_the_full_space():
    n = 30
    lam = spectrum_disk(5, n, 6)
    A, V = planted_general(lam, 5)
    est = norm2_estimate_general(A, iters=400)
    assert abs(est - np.linalg.norm(A, 2)) < 1e-8 * np.linalg.norm(A, 2)
    Q = haar_unitary(n, 9, True)
    ev, X, res = rayleigh_ritz_general(A, Q, est)
    assert np.max(np.abs(np.sort_complex(ev) - np.sort_complex(lam))) < 1e-11 * est
    assert np.max(res) < 1e-13
    assert np.allclose(np.linalg.norm(X, axis=0), 1.0)


@pytest.mark.parametrize("real", [False, True])
def test_solve_finds_the_planted_pairs_inside_the_disk(real):
    n, m_in, m0, n_c = 120, 10, 20, 8
    c, r = (0.3 if real else 0.3 + 0.4j), 1.0
    lam = spectrum_disk(7, n, m_in, center=c, radius=r, gap=0.15, outer=8.0, real_pairs=real)
    A, V = planted_general(lam, 7, cond=8.0, real=real)
    X0 = random_subspace(n, m0, 11, complex_=True)
    out = feast_solve_general(A, c, r, m0, n_c, 1e-11, X0, max_iter=20)
    assert out.status == 0
    want = np.array(sorted(lam[np.abs(lam - c) < r], key=lambda x: (x.real, x.imag)))
    assert out.lam.size == m_in == want.size
    an = np.linalg.norm(A, 2)
    assert np.max(np.abs(out.lam - want)) < 1e-10 * an
    assert np.max(out.res) <= 1e-11
    R = A @ out.X - out.X * out.lam[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) < 2e-11 * an


def test_full_space_converges_in_one_round():
    # m0 = n: the filtered block spans the whole space, so the first
    # Rayleigh-Ritz returns the exact eigenpairs and the exact count
    n = 24
    lam = spectrum_disk(2, n, 5, center=-0.1j, radius=0.8, gap=0.2)
    A, _ = planted_general(lam, 2)
    out = feast_solve_general(A, -0.1j, 0.8, n, 4, 1e-12, random_subspace(n, n, 1, complex_=True), max_iter=3)
    assert out.iterations == 1 and out.lam.size == 5
    want = np.array(sorted(lam[np.abs(lam + 0.1j) < 0.8], key=lambda x: (x.real, x.imag)))
    assert np.max(np.abs(out.lam - want)) < 1e-12 * np.linalg.norm(A, 2)


def test_hermitian_matrix_gives_the_hermitian_solvers_eigenvalues():
    # a Hermitian A on the circle through (lmin, lmax): the same eigenvalues
    # as the Hermitian FEAST, real up to rounding
    n, m0 = 80, 16
    rng = np.random.default_rng(4)
    lam = np.concatenate([rng.uniform(-0.9, 0.9, 7), rng.uniform(1.3, 6.0, 40), rng.uniform(-6.0, -1.3, n - 47)])
    A = planted_matrix(haar_unitary(n, 6, True), lam)
    X0 = random_subspace(n, m0, 3, complex_=True)
    g = feast_solve_general(A, 0.0, 1.0, m0, 8, 1e-11, X0, max_iter=20)
    h = feast_solve(A, -1.0, 1.0, m0, 8, 1e-11, X0, max_iter=20)
    assert g.status == 0 and h.status == 0 and g.lam.size == h.lam.size == 7
    assert np.max(np.abs(g.lam.imag)) < 1e-12
    assert np.max(np.abs(g.lam.real - h.lam)) < 1e-12 * 6.0


@pytest.mark.parametrize("real", [False, True])
def test_iterates_are_subspace_iteration_on_rho(real):
    # FEAST for a general A = V diag(lam) V^{-1} is subspace iteration on
    # rho(A) = V diag(rho(lam)) V^{-1} (Sect. I, the whole circle): round k
    # works on span W_k, W_k = orth(rho(A) W_{k-1}), W_0 = X0, here from the
    # planted eigendecomposition (LAPACK SVD and eig, no LU solve).  Every
    # round's Ritz values in the disk (eigenvalues of W_k^H A W_k) and its
    # maximum residual follow.
    n, m_in, m0, n_c = 120, 10, 14, 8
    c, r = (0.3 if real else 0.3 + 0.4j), 1.0
    lam = spectrum_disk(7, n, m_in, center=c, radius=r, gap=0.15, outer=8.0, real_pairs=real)
    A, V = planted_general(lam, 7, cond=8.0, real=real)
    X0 = random_subspace(n, m0, 11, complex_=True)
    z, w = circle_nodes(c, r, n_c)
    rho = circle_filter(lam, z, w)
    an = np.linalg.norm(A, 2)
    full = feast_solve_general(A, c, r, m0, n_c, 1e-11, X0, max_iter=30, anorm=an)
    assert full.status == 0 and full.iterations >= 3
    Vi = np.linalg.inv(V)
    W = X0.astype(np.complex128)
    prev = None
    for k in range(1, full.iterations + 1):
        W = np.linalg.svd(V @ (rho[:, None] * (Vi @ W)), full_matrices=False)[0]
        mu, Y = np.linalg.eig(W.conj().T @ A @ W)
        X = W @ Y
        X /= np.linalg.norm(X, axis=0)[None, :]
        res = np.linalg.norm(A @ X - X * mu[None, :], axis=0) / an
        ins = np.abs(mu - c) < r
        want = np.array(sorted(mu[ins], key=lambda x: (x.real, x.imag)))
        if k < full.iterations:
            assert abs(full.history[k - 1] - res[ins].max()) <= 1e-6 * res[ins].max() + 1e-15
        if k <= 2:
            out = feast_solve_general(A, c, r, m0, n_c, 1e-11, X0, max_iter=k, anorm=an)
            assert out.lam.size == want.size
            assert np.abs(out.lam - want).max() <= 1e-12 * an
            if prev is not None:
                assert np.abs(prev - want).max() > 1e3 * 1e-12 * an   # the iterates move
            prev = want
