"""Pins of the oracle's dense kernels against LAPACK (an independent
implementation), reconstruction identities and invariants."""
import numpy as np
import pytest

import oracle.dense as D
from oracle import (cholesky_upper, cholqr, cholqr2, gram_eig_orth, jacobi_eigh,
                    lu_factor, lu_solve, lu_solve_adjoint, lu_unpack, round_robin_pairs)

RNG = np.random.default_rng(1234)


def crandn(*shape):
    return RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)


@pytest.mark.parametrize("n", [1, 2, 7, 31, 64, 65])
def test_lu_reconstructs(n):
    M = crandn(n, n)
    LU, piv = lu_factor(M)
    P, L, U = lu_unpack(LU, piv)
    assert np.linalg.norm(P @ M - L @ U) <= 1e-14 * n * np.linalg.norm(M)
    assert np.all(np.abs(np.tril(LU, -1)) <= 1.0 + 1e-15)  # partial pivoting bound


@pytest.mark.parametrize("n,m", [(1, 1), (5, 3), (40, 7), (64, 65)])
def test_lu_solves_match_lapack(n, m):
    z = 0.3 + 0.05j
    H = crandn(n, n)
    A = 0.5 * (H + H.conj().T)
    M = z * np.eye(n) - A
    B = crandn(n, m)
    LU, piv = lu_factor(M)
    np.testing.assert_allclose(lu_solve(LU, piv, B), np.linalg.solve(M, B), rtol=0,
                               atol=1e-9 * np.abs(np.linalg.solve(M, B)).max())
    # adjoint solve = solve with conj(z) I - A for Hermitian A
    Mb = np.conj(z) * np.eye(n) - A
    ref = np.linalg.solve(Mb, B)
    np.testing.assert_allclose(lu_solve_adjoint(LU, piv, B), ref, rtol=0,
                               atol=1e-9 * np.abs(ref).max())


def test_planted_mistake_in_adjoint_is_caught(monkeypatch):
    # dropping the conjugate of the diagonal in U^H gives the wrong solve
    n = 12
    H = crandn(n, n)
    A = 0.5 * (H + H.conj().T)
    M = (0.1 + 0.4j) * np.eye(n) - A
    B = crandn(n, 2)
    LU, piv = lu_factor(M)
    good = lu_solve_adjoint(LU, piv, B)
    monkeypatch.setattr(D.np, "conj", lambda x: x)
    bad = D.lu_solve_adjoint(LU, piv, B)
    assert np.abs(bad - good).max() > 1e-3


@pytest.mark.parametrize("k", [1, 3, 16, 50])
@pytest.mark.parametrize("cplx", [False, True])
def test_cholesky_matches_lapack(k, cplx):
    X = crandn(3 * k, k) if cplx else RNG.standard_normal((3 * k, k))
    G = X.conj().T @ X
    R = cholesky_upper(G)
    np.testing.assert_allclose(R.conj().T @ R, G, atol=1e-12 * np.abs(G).max())
    Lref = np.linalg.cholesky(G)
    np.testing.assert_allclose(R, Lref.conj().T, atol=1e-11 * np.abs(Lref).max())


def test_cholesky_breakdown_detected():
    X = RNG.standard_normal((20, 4))
    X[:, 3] = X[:, 0]
    with pytest.raises(D.CholeskyBreakdown):
        cholqr(X)


@pytest.mark.parametrize("cplx", [False, True])
def test_cholqr2_orthonormal_and_factorises(cplx):
    n, k = 300, 40
    X = crandn(n, k) if cplx else RNG.standard_normal((n, k))
    X = X @ np.diag(np.logspace(0, -5, k))  # cond ~ 1e5
    Q, R = cholqr2(X)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k)) < 1e-13
    assert np.linalg.norm(Q @ R - X) < 1e-13 * np.linalg.norm(X)
    assert np.allclose(np.tril(R, -1), 0)


def test_round_robin_pairs_cover_each_pair_once():
    for k in [2, 3, 4, 7, 10, 31]:
        seen = set()
        for P, Q in round_robin_pairs(k):
            used = list(P) + list(Q)
            assert len(used) == len(set(used))           # disjoint in a round
            for p, q in zip(P, Q):
                assert p < q < k
                assert (p, q) not in seen
                seen.add((p, q))
        assert len(seen) == k * (k - 1) // 2


@pytest.mark.parametrize("k", [1, 2, 3, 7, 33, 64])
@pytest.mark.parametrize("cplx", [False, True])
def test_jacobi_matches_lapack_and_invariants(k, cplx):
    H = crandn(k, k) if cplx else RNG.standard_normal((k, k))
    H = 0.5 * (H + H.conj().T)
    lam, V, sweeps = jacobi_eigh(H)
    ref = np.linalg.eigvalsh(H)
    scale = max(1.0, np.linalg.norm(H))
    np.testing.assert_allclose(lam, ref, atol=1e-13 * scale)
    assert np.all(np.diff(lam) >= 0)
    assert np.linalg.norm(V.conj().T @ V - np.eye(k)) < 1e-13 * k
    assert np.linalg.norm(H @ V - V * lam) < 1e-13 * scale * k
    assert sweeps < 20


def test_jacobi_degenerate_and_diagonal():
    lam, V, _ = jacobi_eigh(np.eye(5) * 3.0)
    np.testing.assert_allclose(lam, 3.0)
    Q = np.linalg.qr(crandn(6, 6))[0]
    H = Q @ np.diag([1, 1, 1, -2, -2, 5.0]) @ Q.conj().T
    lam, V, _ = jacobi_eigh(H)
    np.testing.assert_allclose(lam, [-2, -2, 1, 1, 1, 5], atol=1e-13)
    assert np.linalg.norm(H @ V - V * lam) < 1e-12


def test_gram_eig_orth_truncates_rank():
    X = RNG.standard_normal((100, 8))
    Xd = np.hstack([X, X @ RNG.standard_normal((8, 4))])   # rank 8 of 12
    U = gram_eig_orth(Xd)
    assert U.shape[1] == 8
    assert np.linalg.norm(U.conj().T @ U - np.eye(8)) < 1e-13
    P = U @ (U.conj().T @ Xd)
    assert np.linalg.norm(P - Xd) < 1e-10 * np.linalg.norm(Xd)


def test_block_qr_orth_keeps_small_but_resolved_directions():
    X = crandn(200, 10)
    tiny = crandn(200, 10) * 1e-9         # far below sqrt(eps) relative
    blocks = [X, X + tiny]
    Q = D.block_qr_orth(blocks)
    assert Q.shape[1] == 20
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(20)) < 1e-12
    for B in blocks:
        assert np.linalg.norm(Q @ (Q.conj().T @ B) - B) < 1e-12 * np.linalg.norm(B)
    # the Gram route of the whole window cannot see those directions
    assert gram_eig_orth(np.hstack(blocks)).shape[1] == 10


def test_lu_pivot_ties_take_the_first_row():
    # reading R11: the pivot is the first row of largest |m_ik|^2; here every
    # candidate of column 0 ties in magnitude (with different phases), so the
    # first step keeps row 0; a real 2 x 2 tie does the same
    M = np.array([[1.0, 2.0, 0.5],
                  [1j, 3.0, 1.0],
                  [-1.0, 1.0, 2.0]], dtype=complex)
    LU, piv = lu_factor(M)
    assert int(piv[0]) == 0
    # after step 1 the column-1 entries of rows 1 and 2 are 3 - 2j and 3: |3 - 2j| > 3
    assert int(piv[1]) == 1
    T = np.array([[2.0, 0.0], [2.0, 1.0]], dtype=complex)   # exact tie in column 0
    LU2, piv2 = lu_factor(T)
    assert int(piv2[0]) == 0
    P, L, U = lu_unpack(LU2, piv2)
    np.testing.assert_allclose(P @ T, L @ U, atol=1e-15)
