"""Dense FP64 building blocks of the FEAST oracle, written as textbook loops.

* complex LU with partial pivoting and the two triangular solve pairs it
  serves: (zI - A)^{-1} X and, for complex Hermitian A, the adjoint
  (conj(z) I - A)^{-1} X = (zI - A)^{-H} X through the same factors.  The paper
  only says "a linear system solver" (Sect. I, after Eq. 3).
* Cholesky factorisation and Cholesky-QR, used to orthonormalise the filtered
  subspace so the reduced problem A'q = lambda B'q (FEAST Algorithm, step 2(i))
  becomes a standard Hermitian problem.
* Gram-matrix eigendecomposition orthogonalisation X'^T X' = V Sigma^2 V^T,
  U = X' V Sigma^{-1} (Sect. II-A, the two equations after "we orthogonalize").
* Two-sided Jacobi eigensolver for the small Hermitian reduced matrix.

Every routine is an unblocked loop in the order the textbook algorithm states;
numpy is used only to vectorise the inner row/column operation of each step.

Test infrastructure only (see quadrature.py).
"""
from __future__ import annotations

import numpy as np

EPS = np.finfo(np.float64).eps


class CholeskyBreakdown(ArithmeticError):
    """Raised when a Gram matrix is not numerically positive definite."""

    def __init__(self, column):
        super().__init__(f"Cholesky breakdown at column {column}")
        self.column = column


class SingularShift(ArithmeticError):
    pass


# --------------------------------------------------------------------------
# LU with partial pivoting (Golub & Van Loan, Algorithm 3.4.1, outer-product form)
# --------------------------------------------------------------------------
def lu_factor(M):
    """P M = L U for a square complex matrix.

    At step k the pivot is the first row i >= k maximising |m_ik|^2 =
    Re(m_ik)^2 + Im(m_ik)^2; rows k and p are swapped across the whole matrix,
    column k below the diagonal is divided by the pivot, and the trailing block
    takes the rank-1 update.  Returns (LU, ipiv) with the unit-lower L below the
    diagonal, U on and above it, and ipiv[k] = the row swapped with row k.
    """
    a = np.array(M, dtype=np.complex128, order="C", copy=True)
    n = a.shape[0]
    ipiv = np.zeros(n, dtype=np.int64)
    for k in range(n):
        col = a[k:, k]
        mag = col.real * col.real + col.imag * col.imag
        p = k + int(np.argmax(mag))
        ipiv[k] = p
        if p != k:
            tmp = a[k, :].copy()
            a[k, :] = a[p, :]
            a[p, :] = tmp
        piv = a[k, k]
        if piv == 0:
            raise SingularShift(f"zero pivot at column {k}")
        a[k + 1:, k] /= piv
        a[k + 1:, k + 1:] -= np.outer(a[k + 1:, k], a[k, k + 1:])
    return a, ipiv


def apply_row_swaps(X, ipiv, reverse=False):
    """Apply the interchange sequence of lu_factor to the rows of X in place
    (P X), or its inverse P^T X with reverse=True."""
    order = range(len(ipiv) - 1, -1, -1) if reverse else range(len(ipiv))
    for k in order:
        p = ipiv[k]
        if p != k:
            tmp = X[k].copy()
            X[k] = X[p]
            X[p] = tmp
    return X


def lu_solve(LU, ipiv, B):
    """Y = (P^T L U)^{-1} B = U^{-1} L^{-1} P B by forward then back
    substitution, one row at a time, all right-hand sides together."""
    x = np.array(B, dtype=np.complex128, copy=True)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    n = LU.shape[0]
    apply_row_swaps(x, ipiv)
    for i in range(1, n):
        x[i] -= LU[i, :i] @ x[:i]
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - LU[i, i + 1:] @ x[i + 1:]) / LU[i, i]
    return x[:, 0] if squeeze else x


def lu_solve_adjoint(LU, ipiv, B):
    """Y = (P^T L U)^{-H} B = P^T L^{-H} U^{-H} B.

    For Hermitian A and M = zI - A this is (conj(z) I - A)^{-1} B, the solve of
    the mirrored lower-half node, through the factors of the upper node.
    U^H is lower triangular (forward substitution with conj(u_ii) on the
    diagonal), L^H is unit upper triangular (back substitution), then the row
    interchanges are undone in reverse order."""
    x = np.array(B, dtype=np.complex128, copy=True)
    squeeze = x.ndim == 1
    if squeeze:
        x = x[:, None]
    n = LU.shape[0]
    for i in range(n):
        x[i] = (x[i] - LU[:i, i].conj() @ x[:i]) / np.conj(LU[i, i])
    for i in range(n - 2, -1, -1):
        x[i] -= LU[i + 1:, i].conj() @ x[i + 1:]
    apply_row_swaps(x, ipiv, reverse=True)
    return x[:, 0] if squeeze else x


def lu_unpack(LU, ipiv):
    """Return (P, L, U) as dense matrices with P M = L U (for tests)."""
    n = LU.shape[0]
    L = np.tril(LU, -1) + np.eye(n)
    U = np.triu(LU)
    perm = np.arange(n)
    apply_row_swaps(perm, ipiv)
    P = np.eye(n)[perm]
    return P, L, U


# --------------------------------------------------------------------------
# Cholesky and Cholesky-QR
# --------------------------------------------------------------------------
def cholesky_upper(G):
    """G = R^H R with R upper triangular, column by column
    (r_jj = sqrt(g_jj - sum_{i<j} |r_ij|^2),
     r_jl = (g_jl - sum_{i<j} conj(r_ij) r_il) / r_jj for l > j)."""
    G = np.asarray(G)
    k = G.shape[0]
    R = np.zeros_like(G, dtype=G.dtype)
    for j in range(k):
        s = np.real(G[j, j]) - np.sum(np.abs(R[:j, j]) ** 2)
        if not np.isfinite(s) or s <= 0.0:
            raise CholeskyBreakdown(j)
        R[j, j] = np.sqrt(s)
        if j + 1 < k:
            R[j, j + 1:] = (G[j, j + 1:] - R[:j, j].conj() @ R[:j, j + 1:]) / R[j, j]
    return R


def solve_right_upper(X, R):
    """Q = X R^{-1} for upper-triangular R: column j of Q is
    (x_j - Q[:, :j] R[:j, j]) / r_jj."""
    n, k = X.shape
    Q = np.zeros((n, k), dtype=np.result_type(X, R))
    for j in range(k):
        Q[:, j] = (X[:, j] - Q[:, :j] @ R[:j, j]) / R[j, j]
    return Q


def cholqr(X):
    """One Cholesky-QR pass: G = X^H X = R^H R, Q = X R^{-1}."""
    G = X.conj().T @ X
    G = 0.5 * (G + G.conj().T)
    R = cholesky_upper(G)
    return solve_right_upper(X, R), R


def cholqr2(X):
    """Cholesky-QR applied twice (the second pass restores the orthogonality
    the first loses in proportion to cond(X)^2).  Returns Q, R with X = Q R."""
    Q1, R1 = cholqr(X)
    Q, R2 = cholqr(Q1)
    return Q, R2 @ R1


# --------------------------------------------------------------------------
# Jacobi eigensolver for a Hermitian matrix
# --------------------------------------------------------------------------
def round_robin_pairs(k):
    """The k-1 rounds of disjoint index pairs of the circle-method tournament
    ordering (every pair p < q appears in exactly one round).  For odd k a
    dummy index k is added and its pairs dropped."""
    kk = k + (k & 1)
    rounds = []
    for r in range(kk - 1):
        ps, qs = [], []
        pairs = [(r % (kk - 1), kk - 1)]
        for i in range(1, kk // 2):
            pairs.append(((r + i) % (kk - 1), (r - i) % (kk - 1)))
        for a, b in pairs:
            p, q = (a, b) if a < b else (b, a)
            if q < k:
                ps.append(p)
                qs.append(q)
        rounds.append((np.array(ps, dtype=np.int64), np.array(qs, dtype=np.int64)))
    return rounds


def jacobi_rotation(app, aqq, apq):
    """Parameters (c, s, e) of the unitary U = [[c, s], [-s e, c e]] that
    diagonalises the Hermitian 2x2 block [[app, apq], [conj(apq), aqq]]:
    e = conj(apq)/|apq| removes the phase, then the real symmetric Jacobi
    rotation with tau = (aqq - app)/(2|apq|), t = sign(tau)/(|tau| +
    sqrt(1 + tau^2)), c = 1/sqrt(1 + t^2), s = t c (Golub & Van Loan,
    Algorithm 8.5.1).  Vectorised over arrays of blocks."""
    g = np.abs(apq)
    safe = np.where(g > 0, g, 1.0)
    e = np.where(g > 0, np.conj(apq) / safe, 1.0)
    tau = (aqq - app) / (2.0 * safe)
    sgn = np.where(tau >= 0, 1.0, -1.0)
    t = sgn / (np.abs(tau) + np.sqrt(1.0 + tau * tau))
    c = 1.0 / np.sqrt(1.0 + t * t)
    s = t * c
    return c, s, e


def jacobi_eigh(H, max_sweeps=60, tol=1e-15):
    """Eigenvalues (ascending) and eigenvectors of a Hermitian matrix by
    two-sided Jacobi with the round-robin parallel ordering (Golub & Van Loan,
    Sect. 8.5.5): each round rotates k/2 disjoint (p, q) planes, each rotation
    computed from its 2x2 diagonal block and applied as A <- U^H A U,
    V <- V U.  A plane is rotated only when |a_pq| > tol * ||H||_F; sweeps stop
    after the first sweep with no rotation.  Returns (lam, V, sweeps)."""
    a = np.array(H, copy=True)
    cplx = np.iscomplexobj(a)
    if not cplx:
        a = a.astype(np.float64)
    k = a.shape[0]
    V = np.eye(k, dtype=a.dtype)
    if k == 1:
        return np.real(np.diag(a)).copy(), V, 0
    thr = tol * np.linalg.norm(a)
    rounds = round_robin_pairs(k)
    sweeps = 0
    for sweep in range(max_sweeps):
        rotated = False
        for P, Q in rounds:
            apq = a[P, Q]
            act = np.abs(apq) > thr
            if not np.any(act):
                continue
            rotated = True
            P, Q, apq = P[act], Q[act], apq[act]
            app = np.real(a[P, P])
            aqq = np.real(a[Q, Q])
            c, s, e = jacobi_rotation(app, aqq, apq)
            if not cplx:
                e = np.real(e)
            # columns: [a_p, a_q] <- [a_p, a_q] U
            cp, cq = a[:, P].copy(), a[:, Q].copy()
            a[:, P] = cp * c - cq * (s * e)
            a[:, Q] = cp * s + cq * (c * e)
            vp, vq = V[:, P].copy(), V[:, Q].copy()
            V[:, P] = vp * c - vq * (s * e)
            V[:, Q] = vp * s + vq * (c * e)
            # rows: [a_p; a_q] <- U^H [a_p; a_q]
            rp, rq = a[P, :].copy(), a[Q, :].copy()
            ec = np.conj(e)
            a[P, :] = c[:, None] * rp - (s * ec)[:, None] * rq
            a[Q, :] = s[:, None] * rp + (c * ec)[:, None] * rq
            a[P, Q] = 0.0
            a[Q, P] = 0.0
            a[P, P] = np.real(a[P, P])
            a[Q, Q] = np.real(a[Q, Q])
        sweeps = sweep + 1
        if not rotated:
            break
    lam = np.real(np.diag(a)).copy()
    order = np.argsort(lam, kind="stable")
    return lam[order], V[:, order], sweeps


# --------------------------------------------------------------------------
# Gram-eigendecomposition orthogonalisation (Sect. II-A)
# --------------------------------------------------------------------------
# Directions with sigma_k^2 < GRAM_TRUNC * sigma_1^2 are dropped: the Gram
# matrix squares the condition number, so below this level the computed
# directions are not resolved in FP64.
GRAM_TRUNC = 1e-12


def gram_eig_orth(X, trunc=GRAM_TRUNC):
    """X'^T X' = V Sigma^2 V^T (Jacobi), sigma descending, U = X' V Sigma^{-1}
    restricted to the numerically resolved directions sigma_k^2 >= trunc *
    sigma_1^2; then one Cholesky-QR pass restores the orthogonality the Gram
    route loses.  Returns U (n x r) with r the retained rank."""
    G = X.conj().T @ X
    G = 0.5 * (G + G.conj().T)
    sig2, V, _ = jacobi_eigh(G)
    order = np.argsort(-sig2, kind="stable")
    sig2, V = sig2[order], V[:, order]
    if sig2[0] <= 0:
        raise CholeskyBreakdown(0)
    keep = sig2 >= trunc * sig2[0]
    U = (X @ V[:, keep]) / np.sqrt(sig2[keep])[None, :]
    U, _ = cholqr(U)
    return U


# Block-QR route: a direction of a new block survives when its component
# orthogonal to the basis so far is at least BLOCK_TRUNC times the block's
# largest column norm (the projection leaves rounding noise of order
# eps * ||B||, so smaller remnants are not resolved).
BLOCK_TRUNC = 1e-13


def block_qr_orth(blocks, trunc=BLOCK_TRUNC):
    """Orthonormal basis of span([B_1 ... B_s]) by block Gram-Schmidt, one
    block at a time: P = B - Q (Q^H B) applied twice (CGS2), the Gram matrix
    P^H P = V S^2 V^H (Jacobi), U = P V_r S_r^{-1} over the directions with
    s_k >= trunc * max_j ||b_j||, U re-projected against Q once more and
    finished with one Cholesky-QR pass, Q <- [Q U].  This is a QR-type
    orthogonalisation of the expanded subspace (Sect. II-A names QR and the
    SVD as the two options) that, unlike the Gram matrix of the whole window,
    keeps directions far below sqrt(eps) relative size."""
    Q = None
    for B in blocks:
        bnorm = float(np.max(np.linalg.norm(B, axis=0))) if B.size else 0.0
        if bnorm == 0.0:
            continue
        P = np.array(B, copy=True)
        if Q is not None:
            for _ in range(2):
                P = P - Q @ (Q.conj().T @ P)
        G = P.conj().T @ P
        G = 0.5 * (G + G.conj().T)
        s2, V, _ = jacobi_eigh(G)
        keep = s2 >= (trunc * bnorm) ** 2
        if not np.any(keep):
            continue
        U = (P @ V[:, keep]) / np.sqrt(s2[keep])[None, :]
        if Q is not None:
            U = U - Q @ (Q.conj().T @ U)
        U, _ = cholqr(U)
        Q = U if Q is None else np.hstack([Q, U])
    if Q is None:
        raise CholeskyBreakdown(0)
    return Q
