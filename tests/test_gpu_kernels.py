"""Kernel-level parity of the CUDA path with the FP64 oracle: shifted LU
(pivots bit-exact in FP64), triangular solves and their adjoints, the filter
of Eq. 3, Jacobi, orthonormalisation and Rayleigh-Ritz.  Sizes span several
32-wide panels and a ragged tail."""
import numpy as np
import pytest

import oracle as O
import paper_1605_08771_gb300 as fg
from gpu_common import cuda, ctx, host, rand_hermitian, rand_mat  # noqa: F401
from workloads import make_problem, random_subspace, spectrum_uniform

pytestmark = pytest.mark.gpu
ZS = np.array([0.3 + 0.5j, -0.7 + 0.2j, 1.1 + 0.05j])
SIZES = [1, 2, 31, 32, 33, 65, 100, 257]


PRECS_ALL = [fg.FEAST_PREC_F64, fg.FEAST_PREC_MIXED, fg.FEAST_PREC_MIXED_SIMT]


@pytest.mark.parametrize("n", SIZES + [520])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", PRECS_ALL)
def test_shifted_lu_matches_oracle(ctx, n, cplx, prec):
    # FEAST_PREC_MIXED runs the two-level LU whose 128-column outer updates
    # use the tensor cores: n = 257 and 520 span several outer blocks and a
    # ragged tail
    A = rand_hermitian(n, cplx, seed=n)
    LU, perm = fg.feast_shifted_lu(ctx, cuda(A), ZS, prec)
    LU, perm = host(LU).astype(np.complex128), host(perm)
    u = 1.2e-16 if prec == fg.FEAST_PREC_F64 else 6e-8
    for e, z in enumerate(ZS):
        M = z * np.eye(n) - A
        L = np.tril(LU[e], -1) + np.eye(n)
        U = np.triu(LU[e])
        err = np.linalg.norm(M[perm[e], :] - L @ U) / np.linalg.norm(M)
        assert err <= 8 * n * u, err
        assert np.all(np.abs(np.tril(LU[e], -1)) <= 1 + 1e-6)
        if prec == fg.FEAST_PREC_F64:
            LUo, pivo = O.lu_factor(M)
            permo = np.arange(n)
            O.dense.apply_row_swaps(permo, pivo)
            assert np.array_equal(perm[e], permo)          # pivots bit-exact
            assert np.abs(LU[e] - LUo).max() <= 1e-12 * max(1.0, np.abs(LUo).max())


@pytest.mark.parametrize("n", [1, 33, 100, 257])
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("prec", PRECS_ALL)
def test_shifted_solve_matches_oracle(ctx, n, cplx, adjoint, prec):
    A = rand_hermitian(n, cplx, seed=7 * n + 1)
    B = rand_mat(n, 5, True, seed=n)
    LU, perm = fg.feast_shifted_lu(ctx, cuda(A), ZS, prec)
    Y = host(fg.feast_shifted_solve(ctx, LU, perm, cuda(B), adjoint=adjoint, prec=prec))
    tol = 1e-11 if prec == fg.FEAST_PREC_F64 else 2e-4
    for e, z in enumerate(ZS):
        LUo, pivo = O.lu_factor(z * np.eye(n) - A)
        ref = (O.lu_solve_adjoint if adjoint else O.lu_solve)(LUo, pivo, B)
        assert np.abs(Y[e] - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("prec,m", [(fg.FEAST_PREC_MIXED, 7), (fg.FEAST_PREC_MIXED, 300),
                                    (fg.FEAST_PREC_MIXED_SIMT, 7)])
def test_shifted_solve_complex_fp32_large_n(ctx, adjoint, prec, m):
    # n = 1100: 17 full 64-row diagonal blocks and a ragged one, each followed
    # by a block update of every remaining row (tensor cores: 128-row output
    # tiles over 9 row tiles, m = 300 over three 128-column tiles, the last
    # ragged); the reference is LAPACK's FP64 solve of each shifted system
    n = 1100
    A = np.asfortranarray(0.1 * rand_hermitian(n, True, seed=5))  # spectrum within about +-5
    B = rand_mat(n, m, True, seed=6)
    LU, perm = fg.feast_shifted_lu(ctx, cuda(A), ZS, prec)
    Y = host(fg.feast_shifted_solve(ctx, LU, perm, cuda(B), adjoint=adjoint, prec=prec))
    for e, z in enumerate(ZS):
        Mz = z * np.eye(n) - A
        ref = np.linalg.solve(Mz.conj().T if adjoint else Mz, B)
        assert np.abs(Y[e] - ref).max() <= 2e-4 * np.abs(ref).max()


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", PRECS_ALL)
@pytest.mark.parametrize("n_c", [3, 8])
def test_filter_matches_oracle_and_closed_form(ctx, cplx, prec, n_c):
    lam, a, b = spectrum_uniform(150, 10, seed=11, bulk=20.0)
    P = make_problem("f", lam, a, b, 12, n_c, seed=11, complex_=cplx)
    X = random_subspace(P.n, 7, seed=2, complex_=cplx)
    Y = host(fg.feast_filter_apply(ctx, cuda(P.A), a, b, n_c, cuda(X),
                                   fg.feast_opts_default(prec=prec, anorm=P.anorm)))
    F = O.factor_shifts(P.A, a, b, n_c)
    ref = O.filter_apply(F, X)
    rho = O.rational_filter(P.lam, F.z, F.w)
    closed = P.Q @ (rho[:, None] * (P.Q.conj().T @ X))
    assert np.abs(Y - ref).max() <= 1e-12 * np.abs(X).max()
    assert np.abs(Y - (closed if cplx else closed.real)).max() <= 1e-12 * np.abs(X).max()


@pytest.mark.parametrize("k", [1, 2, 3, 7, 33, 64, 130])
@pytest.mark.parametrize("cplx", [False, True])
def test_jacobi_matches_lapack(ctx, k, cplx):
    H = rand_hermitian(k, cplx, seed=100 + k)
    ev, V, sweeps = fg.feast_jacobi_eigh(ctx, cuda(H))
    V = host(V)
    scale = max(1.0, np.linalg.norm(H))
    np.testing.assert_allclose(ev, np.linalg.eigvalsh(H), atol=1e-13 * scale)
    evo, Vo, _ = O.jacobi_eigh(H)
    np.testing.assert_allclose(ev, evo, atol=1e-13 * scale)
    assert np.linalg.norm(V.conj().T @ V - np.eye(k)) <= 1e-13 * k
    assert np.linalg.norm(H @ V - V * ev) <= 1e-13 * scale * k
    assert sweeps < 30


@pytest.mark.parametrize("big_group", [False, True])
@pytest.mark.parametrize("cplx", [False, True])
def test_two_phase_eigensolver_cluster_finish(ctx, cplx, big_group, capfd, monkeypatch):
    # Rayleigh-Ritz on an invariant subspace whose eigenvalues come in groups
    # 1e-9 apart: after the first full FP64 sweeps of the two-phase reduced
    # eigensolver only pairs inside the groups exceed the threshold, and each
    # group is finished in shared memory; a group larger than the set limit
    # (64) falls back to full sweeps
    monkeypatch.setenv("FEAST_LOG", "1")
    n, k = 320, 200
    rng = np.random.default_rng(41 + 2 * cplx + big_group)
    lam = rng.uniform(-10.0, 10.0, n)
    start = 0
    for size in [2, 3, 5, 8, 13, 21, 40] + ([70] if big_group else []):
        lam[start:start + size] = lam[start] + 1e-9 * rng.standard_normal(size)
        start += size
    Qp, _ = np.linalg.qr(rand_mat(n, n, cplx, seed=77 + big_group))
    A = (Qp * lam[None, :]) @ Qp.conj().T
    A = np.asfortranarray(0.5 * (A + A.conj().T))
    Rk, _ = np.linalg.qr(rand_mat(k, k, cplx, seed=78 + big_group))
    Q0 = np.asfortranarray(Qp[:, :k] @ Rk)
    anorm = np.abs(lam).max()
    ev, X, res = fg.feast_rayleigh_ritz(ctx, cuda(A), cuda(Q0), anorm)
    X = host(X)
    np.testing.assert_allclose(ev, np.sort(lam[:k]), atol=1e-13 * anorm)
    np.testing.assert_allclose(X.conj().T @ X, np.eye(k), atol=1e-12)
    assert res.max() <= 1e-12
    log = capfd.readouterr().err
    passes = [l for l in log.splitlines() if "FP64 polish" in l and "pass" in l]
    if big_group:
        assert any("full sweep" in l for l in passes), log[-3000:]
    else:
        assert any("full sweep" not in l for l in passes), log[-3000:]


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("method", [0, 1])
def test_orthonormalize(ctx, cplx, method):
    n, k = 300, 40
    X = rand_mat(n, k, cplx, seed=5) @ np.diag(np.logspace(0, -5, k))
    Q, r = fg.feast_orthonormalize(ctx, cuda(X), method)
    Q = host(Q)
    assert r == k
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k)) <= 1e-13
    assert np.linalg.norm(Q @ (Q.conj().T @ X) - X) <= 1e-12 * np.linalg.norm(X)
    Qo, _ = O.cholqr2(X) if method == 0 else (O.gram_eig_orth(X), None)
    # same span
    assert np.linalg.norm(Q @ (Q.conj().T @ Qo) - Qo) <= 1e-11


def test_orthonormalize_rank_deficient_falls_back(ctx):
    X = rand_mat(200, 10, True, seed=9)
    Xd = np.asfortranarray(np.hstack([X, X[:, :4] * 2.0]))
    Q, r = fg.feast_orthonormalize(ctx, cuda(Xd), 0)
    assert r == 10
    Q = host(Q)
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(10)) <= 1e-13


@pytest.mark.parametrize("k", [64, 130, 257])
@pytest.mark.parametrize("cplx", [False, True])
def test_rayleigh_ritz_two_phase_eigensolver(ctx, k, cplx):
    # k >= 64 takes the two-phase reduced eigensolver (FP32 block Jacobi,
    # FP64 orthonormalisation and Jacobi polish); the spectrum has exact
    # triples and pairs 1e-9 apart, so the FP32 phase cannot separate them
    n = 320
    rng = np.random.default_rng(k + 7 * cplx)
    lam = np.sort(rng.uniform(-5.0, 5.0, n))
    lam[10:13] = lam[10]
    lam[40:42] = lam[40] + np.array([0.0, 1e-9])
    lam = np.sort(lam)
    P = make_problem("rr2", lam, -1.0, 1.0, 12, 8, seed=k, complex_=cplx)
    Q0, _ = np.linalg.qr(random_subspace(P.n, k, seed=3, complex_=cplx))
    Q0 = np.asfortranarray(Q0)
    ev, X, res = fg.feast_rayleigh_ritz(ctx, cuda(P.A), cuda(Q0), P.anorm)
    X = host(X)
    rp = O.rayleigh_ritz(P.A, Q0, P.anorm)
    np.testing.assert_allclose(ev, rp.lam, atol=1e-13 * P.anorm)
    np.testing.assert_allclose(res, rp.res, atol=1e-12)
    # Ritz vectors: orthonormal, and each one's residual as small as the oracle's
    np.testing.assert_allclose(X.conj().T @ X, np.eye(k), atol=1e-12)
    R = P.A @ X - X * ev[None, :]
    assert np.linalg.norm(R, axis=0).max() <= np.linalg.norm(P.A @ rp.X - rp.X * rp.lam[None, :], axis=0).max() + 1e-11 * P.anorm


@pytest.mark.parametrize("cplx", [False, True])
def test_rayleigh_ritz_matches_oracle(ctx, cplx):
    lam, a, b = spectrum_uniform(120, 9, seed=4, bulk=8.0)
    P = make_problem("rr", lam, a, b, 12, 8, seed=4, complex_=cplx)
    Q0, _ = np.linalg.qr(random_subspace(P.n, 14, seed=1, complex_=cplx))
    Q0 = np.asfortranarray(Q0)
    ev, X, res = fg.feast_rayleigh_ritz(ctx, cuda(P.A), cuda(Q0), P.anorm)
    X = host(X)
    rp = O.rayleigh_ritz(P.A, Q0, P.anorm)
    np.testing.assert_allclose(ev, rp.lam, atol=1e-13 * P.anorm)
    np.testing.assert_allclose(res, rp.res, atol=1e-13)
    overlap = np.abs(np.sum(X.conj() * rp.X, axis=0))
    np.testing.assert_allclose(overlap, 1.0, atol=1e-9)
