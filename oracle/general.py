"""FEAST for a general (non-Hermitian) matrix, in plain FP64.

Sect. I names the non-Hermitian problem among the extensions the FEAST
framework takes directly; the paper gives no algorithm for it.  The reading
taken here (each step also recorded in the design notes):
  filter        Y = sum_k w_k (z_k I - A)^{-1} X over the 2 n_c nodes of the
                whole circle |z - c| = r (quadrature.circle_nodes): Eq. 3
                without the Hermitian mirror, so both half-circles take
                their own factorisations.  For A diagonalisable,
                rho(A) = V diag(rho(lambda_i)) V^{-1} with rho ~ 1 inside the
                disk and ~ 0 outside.
  Rayleigh-Ritz on an orthonormal basis Q of Y (Cholesky-QR twice, the
                Gram-eigendecomposition route on breakdown): A' = Q^H A Q,
                A' v = lambda v by a general eigensolver (the library routine
                numpy.linalg.eig, a step the Hermitian case takes by
                Jacobi), Ritz vectors x = Q v with unit 2-norm.
  check         max ||A x - lambda x|| / ||A||_2 over the Ritz values inside
                the disk, ||A||_2 from 40 power iterations of A^H A started
                at the normalised all-ones vector; stop when it is <= tol
                (the FEAST Algorithm's step 3), or with nothing found when no
                Ritz value lies inside after two iterations.
  next X        all m0 Ritz vectors (step 2(ii)).
Returned pairs: those inside the disk, ordered by (Re lambda, Im lambda).

Test infrastructure only (see quadrature.py).
"""
from __future__ import annotations

import numpy as np

from .dense import lu_factor, lu_solve
from .feast import FeastResult, orthonormalize
from .quadrature import circle_nodes


def norm2_estimate_general(A, iters=40):
    """||A||_2 by `iters` power iterations of A^H A from ones / sqrt(n)."""
    n = A.shape[0]
    v = np.ones(n, dtype=np.complex128) / np.sqrt(n)
    est = 0.0
    for _ in range(iters):
        w = A.conj().T @ (A @ v)
        nw = float(np.linalg.norm(w))
        if nw == 0.0:
            return 0.0
        est = np.sqrt(nw)
        v = w / nw
    return est


def factor_circle(A, center, radius, n_c):
    """LU factors of z_k I - A for the 2 n_c circle nodes."""
    z, w = circle_nodes(center, radius, n_c)
    n = A.shape[0]
    lus = [lu_factor(zk * np.eye(n) - np.asarray(A, dtype=np.complex128)) for zk in z]
    return z, w, lus


def filter_apply_general(w, lus, X):
    """Y = sum_k w_k (z_k I - A)^{-1} X (Eq. 3 over the whole circle)."""
    X = np.asarray(X, dtype=np.complex128)
    out = np.zeros(X.shape, dtype=np.complex128)
    for wk, (LU, piv) in zip(w, lus):
        out += wk * lu_solve(LU, piv, X)
    return out


def rayleigh_ritz_general(A, Q, anorm):
    """A' = Q^H A Q, its eigenpairs (numpy.linalg.eig), Ritz vectors with unit
    2-norm and relative residual norms."""
    W = A @ Q
    Ar = Q.conj().T @ W
    lam, V = np.linalg.eig(Ar)
    X = Q @ V
    nrm = np.linalg.norm(X, axis=0)
    X = X / nrm[None, :]
    AX = (W @ V) / nrm[None, :]
    res = np.linalg.norm(AX - X * lam[None, :], axis=0) / anorm
    return lam, X, res


def inside_disk(lam, center, radius):
    return np.abs(np.asarray(lam) - center) < radius


def feast_solve_general(A, center, radius, m0, n_c, tol, X0, max_iter=100, anorm=None):
    A = np.asarray(A, dtype=np.complex128)
    if anorm is None or anorm <= 0:
        anorm = norm2_estimate_general(A)
    z, w, lus = factor_circle(A, center, radius, n_c)
    X = np.asarray(X0, dtype=np.complex128).copy()
    hist = []
    lam = res = None
    for it in range(1, max_iter + 1):
        Q, _ = orthonormalize(filter_apply_general(w, lus, X))
        lam, X, res = rayleigh_ritz_general(A, Q, anorm)
        ins = np.where(inside_disk(lam, center, radius))[0]
        r = float(np.max(res[ins])) if ins.size else np.inf
        hist.append(r)
        if (ins.size and r <= tol) or (ins.size == 0 and it >= 2):
            return _result(0, lam, X, res, ins, it, hist)
    ins = np.where(inside_disk(lam, center, radius))[0]
    return _result(1, lam, X, res, ins, max_iter, hist)


def _result(status, lam, X, res, ins, it, hist):
    order = sorted(ins, key=lambda i: (lam[i].real, lam[i].imag))
    return FeastResult(status=status, lam=lam[order], X=X[:, order], res=res[order], iterations=it,
                       filters=it, history=hist)
