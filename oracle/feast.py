"""FEAST, XFEAST and RFEAST as the paper's Appendix states them, in plain FP64.

Steps and where they come from:
  filter        X' = rho(A) X ~ sum_j w_j (z_j I - A)^{-1} X (Eq. 3); for real
                symmetric A and real X the mirrored lower-half nodes contribute
                the complex conjugate, so X' = sum_j 2 Re(w_j Y_j); for complex
                Hermitian A they contribute conj(w_j) (conj(z_j) I - A)^{-1} X.
  Rayleigh-Ritz A' = X'^H A X', B' = X'^H X', A'q = lambda B'q (FEAST step 2(i));
                here X' is first orthonormalised so B' = I.
  Ritz vectors  X_{i+1} = X' Q (step 2(ii)).
  check         r = max ||A x_k - lambda_k x_k|| over the pairs with lambda_k in I
                (step 3), taken relative to ||A||_2.
  XFEAST        window of s filtered blocks, warm-up X_i = rho(A)^i X_0, Gram
                eigendecomposition orthogonalisation, selection of m0 pairs,
                filter of the selected block, oldest block evicted
                (Sect. II-A; XFEAST Algorithm steps 0-5).
  RFEAST        after the filter, s Rayleigh-Ritz passes, each appending the Ritz
                residual block R = A X - X Lambda (Sect. II-B; RFEAST Algorithm).
  selection     all pairs inside I first; if fewer than m0, fill with the
                outside pairs of lowest residual (Sect. II-A, end).
  RFEAST check  the m pairs inside I with lowest residual, m counted at the
                first Rayleigh-Ritz pass of the iteration (Sect. II-B).

Readings where the paper is silent (each also recorded in the design notes):
  * orthonormalisation before Rayleigh-Ritz is Cholesky-QR applied twice,
    falling back to the Gram-eigendecomposition route when the Gram matrix is
    not numerically positive definite;
  * XFEAST keeps the window blocks as the filter returns them (X_0 with unit
    columns, then rho(A)^i X_0 unscaled, as step 0 writes them) and
    orthogonalises the window with a block QR (Sect. II-A allows QR or the SVD;
    the Gram matrix of the whole window cannot resolve directions below
    sqrt(eps), which loses the expansion once the iterates agree to ~1e-6);
  * the RFEAST expansion appends R = A X - X Lambda for every selected pair,
    as step 2(iii) of the RFEAST Algorithm says (expand="all", the default);
    the columns of R are normalised, their (rounding-level) component along
    the current basis is removed twice, and they are orthonormalised before
    the append (same span as [X' R]); the append after the last pass is
    dropped because nothing uses it;
  * option expand="unconverged" (a reading, not the paper's text): only the
    selected pairs whose relative residual is still above tol expand the
    subspace, and the passes end once every selected pair has converged; a
    converged pair's residual is rounding noise, whose normalised direction
    adds spurious Ritz pairs (Sect. II-B reports them) but no information;
  * option response_stop=True (a reading, not the paper's text): on spectra
    with eigenvalues on both sides of I, mixtures of outside eigenvectors give
    Ritz values inside I that never converge (in plain FEAST the m0 - m
    outside directions of the subspace mix) and (with m0 below the number
    of eigenvalues near |rho| = 1/2) also inflate RFEAST's first-pass count.
    All three variants then also stop when every (selected) in-I pair whose
    filter response mu_k = Re(x_k^H rho(A) x_k) exceeds 1/2 has converged;
    mu_k is read off the filter application the next step performs anyway
    (rho > 1/2 exactly inside I for the circle contour, rho < 1/2 outside, so
    a mixture of outside eigenvectors has mu < 1/2); the pairs returned are
    those.  Off by default: the paper's checks (step 3) alone decide;
  * selection ties are broken by ascending eigenvalue; with more than m0 pairs
    inside I the m0 of lowest residual are kept;
  * ||A||_2 is the caller's value when given, else 40 power iterations from the
    normalised all-ones vector.

Test infrastructure only (see quadrature.py).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .dense import (CholeskyBreakdown, block_qr_orth, cholqr2, gram_eig_orth, jacobi_eigh,
                    lu_factor, lu_solve, lu_solve_adjoint)
from .quadrature import contour_nodes

PLAIN, XFEAST, RFEAST = "feast", "xfeast", "rfeast"
EXPAND_ALL, EXPAND_UNCONVERGED = "all", "unconverged"


# --------------------------------------------------------------------------
# filter
# --------------------------------------------------------------------------
@dataclass
class ShiftedFactors:
    """LU factors of z_j I - A for the upper-half nodes (computed once; A and
    z_j do not change between iterations)."""
    z: np.ndarray
    w: np.ndarray
    lus: list
    hermitian_complex: bool


def factor_shifts(A, lmin, lmax, n_c, aspect=1.0):
    z, w = contour_nodes(lmin, lmax, n_c, aspect)
    n = A.shape[0]
    lus = [lu_factor(zj * np.eye(n) - A) for zj in z]
    return ShiftedFactors(z=z, w=w, lus=lus, hermitian_complex=np.iscomplexobj(A))


def filter_apply(F: ShiftedFactors, X):
    """rho(A) X by the quadrature of Eq. 3 over both half-contours."""
    if F.hermitian_complex:
        out = np.zeros(X.shape, dtype=np.complex128)
        for wj, (LU, piv) in zip(F.w, F.lus):
            out += wj * lu_solve(LU, piv, X)
            out += np.conj(wj) * lu_solve_adjoint(LU, piv, X)
        return out
    if np.iscomplexobj(X):
        raise ValueError("real symmetric A takes a real subspace")
    out = np.zeros(X.shape, dtype=np.float64)
    for wj, (LU, piv) in zip(F.w, F.lus):
        out += 2.0 * np.real(wj * lu_solve(LU, piv, X))
    return out


# --------------------------------------------------------------------------
# Rayleigh-Ritz, residuals, selection
# --------------------------------------------------------------------------
def norm_estimate(A, iters=40):
    """||A||_2 estimate: `iters` power iterations from ones/sqrt(n)."""
    n = A.shape[0]
    v = np.ones(n, dtype=A.dtype) / np.sqrt(n)
    est = 0.0
    for _ in range(iters):
        w = A @ v
        est = float(np.linalg.norm(w))
        if est == 0.0:
            return 0.0
        v = w / est
    return est


def orthonormalize(X):
    """Cholesky-QR twice, Gram-eigendecomposition route on breakdown."""
    try:
        Q, _ = cholqr2(X)
        return Q, "cholqr2"
    except CholeskyBreakdown:
        return gram_eig_orth(X), "gram_eig"


@dataclass
class RitzPairs:
    lam: np.ndarray       # k Ritz values, ascending
    X: np.ndarray         # n x k Ritz vectors (unit 2-norm)
    AX: np.ndarray        # A X
    res: np.ndarray       # ||A x_k - lambda_k x_k|| / ||A||_2
    Ar: np.ndarray = None  # the reduced matrix A' = Q^H A Q


def rayleigh_ritz(A, Q, anorm):
    """A' = Q^H A Q for orthonormal Q, A' V = V Lambda (Jacobi), Ritz vectors
    X = Q V with A X = (A Q) V, relative residual norms."""
    W = A @ Q
    Ar = Q.conj().T @ W
    Ar = 0.5 * (Ar + Ar.conj().T)
    lam, V, _ = jacobi_eigh(Ar)
    X = Q @ V
    AX = W @ V
    R = AX - X * lam[None, :]
    res = np.linalg.norm(R, axis=0) / anorm
    return RitzPairs(lam=lam, X=X, AX=AX, res=res, Ar=Ar)


def inside(lam, lmin, lmax):
    return (lam > lmin) & (lam < lmax)


def select_pairs(lam, res, lmin, lmax, m0):
    """Indices of the m0 selected pairs (Sect. II-A): every pair inside I (the
    m0 of lowest residual when more than m0 are inside), filled with outside
    pairs by ascending residual; ties by ascending lambda.  Returned sorted by
    ascending lambda."""
    idx = np.arange(lam.size)
    ins = inside(lam, lmin, lmax)
    key_in = np.lexsort((lam[ins], res[ins]))
    chosen = list(idx[ins][key_in][:m0])
    if len(chosen) < m0:
        outs = ~ins
        key_out = np.lexsort((lam[outs], res[outs]))
        chosen += list(idx[outs][key_out][: m0 - len(chosen)])
    chosen = np.array(sorted(chosen, key=lambda i: (lam[i], i)), dtype=np.int64)
    return chosen


def normalize_columns(X):
    nrm = np.linalg.norm(X, axis=0)
    nrm = np.where(nrm > 0, nrm, 1.0)
    return X / nrm[None, :]


# --------------------------------------------------------------------------
# drivers
# --------------------------------------------------------------------------
@dataclass
class FeastResult:
    status: int                 # 0 converged, 1 max_iter reached
    lam: np.ndarray             # returned eigenvalues (ascending), inside I
    X: np.ndarray               # n x m eigenvectors
    res: np.ndarray             # relative residuals of the returned pairs
    iterations: int             # Rayleigh-Ritz / check rounds
    filters: int                # applications of rho(A) (n_c * m0 solves each)
    history: list = field(default_factory=list)   # max residual per round
    m_expected: int | None = None
    rr_dims: list = field(default_factory=list)   # dimension of every Rayleigh-Ritz pass


def _check(lam, res, sel, lmin, lmax):
    ins = sel[inside(lam[sel], lmin, lmax)]
    r = float(np.max(res[ins])) if ins.size else np.inf
    return ins, r


def feast_solve(A, lmin, lmax, m0, n_c, tol, X0, variant=PLAIN, s=3,
                max_iter=100, aspect=1.0, anorm=None, factors=None,
                expand=EXPAND_ALL, response_stop=False):
    """Eigenpairs of Hermitian A with eigenvalues in the open interval
    (lmin, lmax), by FEAST / XFEAST / RFEAST (Appendix).

    expand: RFEAST residual columns appended at step 2(iii): "all" selected
    pairs (the paper) or only the "unconverged" ones (a reading).
    response_stop: XFEAST/RFEAST also stop on converged non-spurious pairs
    by filter response (a reading; off = the paper's checks only)."""
    if expand not in (EXPAND_ALL, EXPAND_UNCONVERGED):
        raise ValueError(expand)
    A = np.asarray(A)
    if anorm is None or anorm <= 0:
        anorm = norm_estimate(A)
    F = factors or factor_shifts(A, lmin, lmax, n_c, aspect)
    if variant == PLAIN:
        return _feast(A, F, lmin, lmax, m0, tol, X0, max_iter, anorm, response_stop)
    if variant == XFEAST:
        return _xfeast(A, F, lmin, lmax, m0, tol, X0, s, max_iter, anorm, response_stop)
    if variant == RFEAST:
        return _rfeast(A, F, lmin, lmax, m0, tol, X0, s, max_iter, anorm, expand, response_stop)
    raise ValueError(variant)


def _result(status, rp, idx, it, filters, hist, m_expected=None, dims=None):
    order = np.argsort(rp.lam[idx], kind="stable")
    idx = idx[order]
    return FeastResult(status=status, lam=rp.lam[idx].copy(), X=rp.X[:, idx].copy(),
                       res=rp.res[idx].copy(), iterations=it, filters=filters,
                       history=hist, m_expected=m_expected, rr_dims=list(dims or []))


def _feast(A, F, lmin, lmax, m0, tol, X0, max_iter, anorm, response_stop=False):
    X = np.array(X0, copy=True)
    hist, dims = [], []
    rp = None
    pend = None
    for it in range(1, max_iter + 1):
        Xf = filter_apply(F, X)                         # step 1
        if pend is not None:
            keep = _spurious_free(pend, filter_response(X, Xf), tol)
            if keep is not None:
                return _result(0, pend["rp"], pend["sel"][keep], it - 1, it, hist, dims=dims)
            pend = None
        Q, _ = orthonormalize(Xf)                       # B' = I
        dims.append(Q.shape[1])
        rp = rayleigh_ritz(A, Q, anorm)                 # step 2(i)
        X = rp.X                                        # step 2(ii)
        sel = np.arange(rp.lam.size)
        ins, r = _check(rp.lam, rp.res, sel, lmin, lmax)   # step 3
        hist.append(r)
        if ins.size and r <= tol:
            return _result(0, rp, ins, it, it, hist, dims=dims)
        if ins.size == 0 and it >= 2:
            return _result(0, rp, ins, it, it, hist, dims=dims)
        if response_stop:
            in_cols = [c for c in range(rp.lam.size) if lmin < rp.lam[c] < lmax]
            if any(rp.res[c] <= tol for c in in_cols):
                pend = {"in_cols": in_cols, "res": rp.res, "sel": sel, "rp": rp}
    ins, _ = _check(rp.lam, rp.res, np.arange(rp.lam.size), lmin, lmax)
    return _result(1, rp, ins, max_iter, max_iter, hist, dims=dims)


def filter_response(X, Xf):
    """mu_k = Re(x_k^H rho(A) x_k) for unit columns x_k of X, from Xf = rho(A) X:
    the Rayleigh quotient of the filter, rho(lambda) for an eigenvector."""
    return np.real(np.sum(X.conj() * Xf, axis=0))


def _spurious_free(pend, mu, tol):
    """Deferred stopping test of the previous round: its selected pairs inside
    I whose filter response exceeds 1/2 (rho > 1/2 exactly inside I for the
    circle contour) must all have converged; the others are spurious."""
    keep = [k for k in pend["in_cols"] if mu[k] > 0.5]
    if keep and max(pend["res"][k] for k in keep) <= tol:
        return keep
    return None


def _xfeast(A, F, lmin, lmax, m0, tol, X0, s, max_iter, anorm, response_stop):
    # step 0: X' = [X_0, X_1, ..., X_{s-1}] with X_i = rho(A)^i X_0
    blocks = [normalize_columns(np.array(X0, copy=True))]
    filters = 0
    for _ in range(1, s):
        blocks.append(filter_apply(F, blocks[-1]))
        filters += 1
    hist, dims = [], []
    rp = None
    for it in range(1, max_iter + 1):
        Q = block_qr_orth(blocks)                       # step 1
        dims.append(Q.shape[1])
        rp = rayleigh_ritz(A, Q, anorm)                 # step 2(i)
        sel = select_pairs(rp.lam, rp.res, lmin, lmax, m0)   # step 2(ii)
        ins, r = _check(rp.lam, rp.res, sel, lmin, lmax)     # step 3
        hist.append(r)
        if ins.size and r <= tol:
            return _result(0, rp, ins, it, filters, hist, dims=dims)
        if ins.size == 0 and it >= 2:
            return _result(0, rp, ins, it, filters, hist, dims=dims)
        if it == max_iter:
            break
        Xs = rp.X[:, sel]
        Xn = filter_apply(F, Xs)                        # step 4(i)
        filters += 1
        if response_stop:
            pend = {"in_cols": [c for c, i in enumerate(sel) if lmin < rp.lam[i] < lmax],
                    "res": rp.res[sel]}
            keep = _spurious_free(pend, filter_response(Xs, Xn), tol)
            if keep is not None:
                return _result(0, rp, sel[keep], it, filters, hist, dims=dims)
        blocks = blocks[1:] + [Xn]                      # step 4(ii)
    return _result(1, rp, ins, max_iter, filters, hist, dims=dims)


def _rfeast(A, F, lmin, lmax, m0, tol, X0, s, max_iter, anorm, expand, response_stop):
    X = np.array(X0, copy=True)
    hist, dims = [], []
    rp = None
    pend = None
    filters = 0
    for it in range(1, max_iter + 1):
        Xf = filter_apply(F, X)                         # step 1
        filters += 1
        if pend is not None:
            keep = _spurious_free(pend, filter_response(X, Xf), tol)
            if keep is not None:
                prp = pend["rp"]
                return _result(0, prp, pend["sel"][keep], it - 1, filters, hist, pend["m"], dims=dims)
            pend = None
        Q, _ = orthonormalize(Xf)
        m_expected = 0
        for j in range(1, s + 1):                       # step 2
            dims.append(Q.shape[1])
            rp = rayleigh_ritz(A, Q, anorm)             # (i)
            if j == 1:
                m_expected = int(np.sum(inside(rp.lam, lmin, lmax)))
            sel = select_pairs(rp.lam, rp.res, lmin, lmax, m0)   # (ii)
            X = rp.X[:, sel]
            if j < s:                                   # (iii)
                if expand == EXPAND_ALL:
                    act = sel                           # R = A X_{i+1} - X_{i+1} Lambda
                else:
                    # the pairs not yet converged only (a reading)
                    act = sel[rp.res[sel] > tol]
                    if act.size == 0:
                        break
                R = rp.AX[:, act] - rp.X[:, act] * rp.lam[act][None, :]
                Rn = normalize_columns(R)
                for _ in range(2):
                    Rn = Rn - Q @ (Q.conj().T @ Rn)
                U, _ = orthonormalize(Rn)
                Q = np.hstack([Q, U])
        # step 3: the m_expected in-I pairs of lowest residual
        ins = sel[inside(rp.lam[sel], lmin, lmax)]
        ins = ins[np.lexsort((rp.lam[ins], rp.res[ins]))][:m_expected]
        r = float(np.max(rp.res[ins])) if ins.size else np.inf
        hist.append(r)
        if ins.size and r <= tol:
            return _result(0, rp, ins, it, filters, hist, m_expected, dims=dims)
        if ins.size == 0 and it >= 2:
            return _result(0, rp, ins, it, filters, hist, m_expected, dims=dims)
        in_cols = [c for c, i in enumerate(sel) if lmin < rp.lam[i] < lmax]
        if response_stop and any(rp.res[sel[c]] <= tol for c in in_cols):
            pend = {"in_cols": in_cols, "res": rp.res[sel], "sel": sel, "rp": rp, "m": m_expected}
    return _result(1, rp, ins, max_iter, filters, hist, m_expected, dims=dims)


# --------------------------------------------------------------------------
# the generalized problem A x = lambda B x (B Hermitian positive definite)
# --------------------------------------------------------------------------
def feast_solve_generalized(A, B, lmin, lmax, m0, n_c, tol, X0, max_iter=100, aspect=1.0):
    """Plain FEAST for A x = lambda B x as the FEAST Algorithm states it with
    B (Appendix: A' = X'^H A X', B' = X'^H B X'): the filter
    sum_j w_j (z_j B - A)^{-1} B X (both half-contours), the subspace
    B-orthonormalised (Cholesky of X'^H B X', twice) so that B' = I, then the
    standard reduced problem.  Residual: ||A x - lambda B x|| / ((||A|| +
    |lambda| ||B||) ||x||), the backward error of the pencil, with the
    2-norms of A and B from eigvalsh (test infrastructure)."""
    from .dense import cholesky_upper, solve_right_upper
    A = np.asarray(A)
    B = np.asarray(B)
    n = A.shape[0]
    cplx = np.iscomplexobj(A) or np.iscomplexobj(B)
    an = float(np.max(np.abs(np.linalg.eigvalsh(A))))
    bn = float(np.max(np.abs(np.linalg.eigvalsh(B))))
    z, w = contour_nodes(lmin, lmax, n_c, aspect)
    lus = [lu_factor(zj * B - A) for zj in z]

    def filt(X):
        BX = B @ X
        if cplx:
            out = np.zeros(X.shape, dtype=np.complex128)
            for wj, (LU, piv) in zip(w, lus):
                out += wj * lu_solve(LU, piv, BX) + np.conj(wj) * lu_solve_adjoint(LU, piv, BX)
            return out
        out = np.zeros(X.shape)
        for wj, (LU, piv) in zip(w, lus):
            out += 2.0 * np.real(wj * lu_solve(LU, piv, BX))
        return out

    def b_orth(X):
        for _ in range(2):
            G = X.conj().T @ (B @ X)
            R = cholesky_upper(0.5 * (G + G.conj().T))
            X = solve_right_upper(X, R)
        return X

    X = np.array(X0, copy=True)
    hist = []
    for it in range(1, max_iter + 1):
        Q = b_orth(filt(X))
        Ar = Q.conj().T @ (A @ Q)
        lam, V, _ = jacobi_eigh(0.5 * (Ar + Ar.conj().T))
        X = Q @ V
        R = A @ X - (B @ X) * lam[None, :]
        res = np.linalg.norm(R, axis=0) / ((an + np.abs(lam) * bn) * np.linalg.norm(X, axis=0))
        ins = np.where(inside(lam, lmin, lmax))[0]
        r = float(np.max(res[ins])) if ins.size else np.inf
        hist.append(r)
        if (ins.size and r <= tol) or (ins.size == 0 and it >= 2):
            return FeastResult(status=0, lam=lam[ins], X=X[:, ins], res=res[ins], iterations=it, filters=it,
                               history=hist)
    ins = np.where(inside(lam, lmin, lmax))[0]
    return FeastResult(status=1, lam=lam[ins], X=X[:, ins], res=res[ins], iterations=max_iter, filters=max_iter,
                       history=hist)
