"""Parity of FEAST for a general (non-Hermitian) matrix, CUDA path through
the C ABI, with the oracle: the reduced general eigensolver (Hessenberg + QR
to Schur form) against the eigenvalues of numpy's eig (the oracle's step) and
its own residuals, the whole-circle filter against the oracle's resolvent
solves, and the disk solve against the oracle's solve and the planted
spectrum."""
import numpy as np
import pytest

import paper_1605_08771_gb300 as fg
from gpu_common import cuda, ctx, host  # noqa: F401
from oracle.general import factor_circle, feast_solve_general, filter_apply_general
from workloads import haar_unitary, planted_general, planted_matrix, random_subspace, spectrum_disk

pytestmark = pytest.mark.gpu


def _match(a, b):
    """Largest distance of a greedy nearest pairing of two eigenvalue lists
    (the order of equal-real-part conjugate pairs is not unique)."""
    a, b = list(np.asarray(a)), list(np.asarray(b))
    assert len(a) == len(b)
    d = 0.0
    for x in a:
        j = int(np.argmin(np.abs(np.asarray(b) - x)))
        d = max(d, abs(b[j] - x))
        b.pop(j)
    return d


def _check_eig(H, ev, V, tol):
    hn = np.linalg.norm(H)
    assert _match(ev, np.linalg.eigvals(H)) < tol * hn
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0, rtol=0, atol=1e-12)
    R = H @ V - V * ev[None, :]
    assert np.max(np.linalg.norm(R, axis=0)) < 1e-12 * hn


@pytest.mark.parametrize("k,seed", [(1, 0), (2, 1), (3, 2), (37, 3), (130, 4), (300, 5)])
def test_eig_general_random_matches_oracle(ctx, k, seed):
    rng = np.random.default_rng(seed)
    H = np.asfortranarray(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    ev, V, sweeps = fg.feast_eig_general(ctx, cuda(H))
    _check_eig(H, ev, host(V), 1e-11)
    assert sweeps <= 30 * k


def test_eig_general_special_matrices(ctx):
    rng = np.random.default_rng(7)
    k = 40
    # already triangular: the eigenvalues are the diagonal, no QR sweep
    T = np.triu(rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k)))
    ev, V, sweeps = fg.feast_eig_general(ctx, cuda(T))
    np.testing.assert_allclose(ev, np.diag(T), rtol=0, atol=1e-14 * np.linalg.norm(T))
    assert sweeps == 0
    _check_eig(T, ev, host(V), 1e-13)
    # real with complex-conjugate pairs (a real rotation block structure)
    Hr = rng.standard_normal((k, k)).astype(np.complex128)
    ev, V, _ = fg.feast_eig_general(ctx, cuda(Hr))
    _check_eig(Hr, ev, host(V), 1e-11)
    # companion matrix of a polynomial with known roots
    roots = np.exp(2j * np.pi * np.arange(12) / 12) * (1.0 + 0.05 * np.arange(12))
    C = np.zeros((12, 12), dtype=np.complex128)
    C[1:, :-1] = np.eye(11)
    C[:, -1] = -np.poly(roots)[::-1][:-1]
    ev, V, _ = fg.feast_eig_general(ctx, cuda(C))
    assert _match(ev, roots) < 1e-8
    # a multiple of the identity: every vector is an eigenvector
    ev, V, _ = fg.feast_eig_general(ctx, cuda((2.0 - 1.0j) * np.eye(9)))
    np.testing.assert_allclose(ev, 2.0 - 1.0j, rtol=0, atol=1e-15)


def test_eig_general_rejects_bad_input(ctx):
    H = np.eye(4, dtype=np.complex128)
    H[1, 2] = np.nan
    with pytest.raises(fg.FeastError):
        fg.feast_eig_general(ctx, cuda(H))


@pytest.mark.parametrize("real", [False, True])
def test_filter_general_matches_oracle(ctx, real):
    n, m, n_c = 300, 7, 6
    lam = spectrum_disk(3, n, 20, center=0.2, radius=1.0, real_pairs=real)
    A, _ = planted_general(lam, 3, cond=5.0, real=real)
    X = random_subspace(n, m, 4, complex_=True)
    Y = host(fg.feast_filter_apply_general(ctx, cuda(A), 0.2, 1.0, n_c, cuda(X)))
    _, w, lus = factor_circle(A, 0.2, 1.0, n_c)
    ref = filter_apply_general(w, lus, X)
    # forward error of the solves: kappa(z_k I - A) is up to ~1e3 here
    assert np.max(np.abs(Y - ref)) < 1e-10 * np.max(np.abs(ref))


@pytest.mark.parametrize("real,n", [(False, 400), (True, 300)])
def test_disk_solve_vs_oracle_and_planted(ctx, real, n):
    m_in, m0, n_c = 16, 30, 8
    c = 0.3 if real else 0.3 + 0.4j
    lam = spectrum_disk(7, n, m_in, center=c, radius=1.0, gap=0.15, outer=8.0, real_pairs=real)
    A, _ = planted_general(lam, 7, cond=8.0, real=real)
    X0 = random_subspace(n, m0, 11, complex_=True)
    out = fg.feast_disk_solve(ctx, cuda(A), c, 1.0, m0, n_c, 1e-11, max_iter=20, x0=cuda(X0))
    assert out["status"] == 0
    want = lam[np.abs(lam - c) < 1.0]
    assert out["evals"].size == want.size == m_in
    an = np.linalg.norm(A, 2)
    assert _match(out["evals"], want) < 1e-10 * an
    assert out["res"].max() <= 1e-11
    V = host(out["evecs"])
    R = A @ V - V * out["evals"][None, :]
    assert np.max(np.linalg.norm(R, axis=0)) < 2e-11 * an
    ref = feast_solve_general(A, c, 1.0, m0, n_c, 1e-11, X0, max_iter=20)
    assert ref.status == 0
    assert _match(out["evals"], ref.lam) < 1e-10 * an
    assert abs(out["iterations"] - ref.iterations) <= 1


def test_disk_solve_full_space_one_round(ctx):
    # m0 = n: the filtered block spans the whole space and round 1 returns
    # the exact pairs inside the disk
    n = 48
    lam = spectrum_disk(2, n, 6, center=-0.1j, radius=0.8, gap=0.2)
    A, _ = planted_general(lam, 2)
    out = fg.feast_disk_solve(ctx, cuda(A), -0.1j, 0.8, n, 4, 1e-12, max_iter=3,
                              x0=cuda(random_subspace(n, n, 1, complex_=True)))
    assert out["status"] == 0 and out["iterations"] == 1 and out["evals"].size == 6
    assert _match(out["evals"], lam[np.abs(lam + 0.1j) < 0.8]) < 1e-12 * np.linalg.norm(A, 2)


def test_disk_solve_hermitian_matrix_matches_interval_solve(ctx):
    # (every outside eigenvalue on one side: both solvers' literal checks
    # converge in a few rounds, as on the paper's spectra)
    n, m0 = 200, 24
    rng = np.random.default_rng(4)
    lam = np.concatenate([rng.uniform(-0.9, 0.9, 9), rng.uniform(1.3, 6.0, n - 9)])
    A = planted_matrix(haar_unitary(n, 6, True), lam)
    X0 = random_subspace(n, m0, 3, complex_=True)
    g = fg.feast_disk_solve(ctx, cuda(A), 0.0, 1.0, m0, 8, 1e-11, max_iter=20, x0=cuda(X0))
    h = fg.feast_interval_solve(ctx, cuda(A), -1.0, 1.0, m0, 8, 1e-11, x0=cuda(X0))
    assert g["status"] == 0 and h["status"] == 0 and g["evals"].size == h["evals"].size == 9
    assert np.max(np.abs(g["evals"].imag)) < 1e-11
    np.testing.assert_allclose(np.sort(g["evals"].real), np.sort(lam[np.abs(lam) < 1.0]), rtol=0, atol=1e-11 * 6.0)


def test_disk_solve_empty_disk_and_errors(ctx):
    n = 60
    lam = spectrum_disk(6, n, 0, center=0.0, radius=1.0, gap=0.3)
    A, _ = planted_general(lam, 6)
    X0 = random_subspace(n, 8, 1, complex_=True)
    # no eigenvalue inside: no Ritz value falls inside in two rounds (as in
    # the oracle on the same start), and the solve stops with nothing found
    ref = feast_solve_general(A, 0.0, 1.0, 8, 4, 1e-10, X0, max_iter=10)
    assert ref.status == 0 and ref.lam.size == 0 and ref.iterations == 2
    out = fg.feast_disk_solve(ctx, cuda(A), 0.0, 1.0, 8, 4, 1e-10, max_iter=10, x0=cuda(X0))
    assert out["status"] == 0 and out["evals"].size == 0 and out["iterations"] == 2
    with pytest.raises(fg.FeastError):
        fg.feast_disk_solve(ctx, cuda(A), 0.0, 1.0, n + 1, 4, 1e-10)
    with pytest.raises(fg.FeastError):
        fg.feast_disk_solve(ctx, cuda(A), 0.0, -1.0, 8, 4, 1e-10)
    B = A.copy()
    B[3, 4] = np.inf
    with pytest.raises(fg.FeastError):
        fg.feast_disk_solve(ctx, cuda(B), 0.0, 1.0, 8, 4, 1e-10)
