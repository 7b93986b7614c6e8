"""Closed forms of FEAST iterates on planted spectra A = Q diag(lam) Q^H,
computed in the planted eigenbasis with LAPACK (SVD, eigh) and the rational
filter's values rho(lam): no linear solve, orthonormalisation or Jacobi of
the oracle or of the CUDA path is involved.  The pair selection (Sect.
II-A) is the oracle's select_pairs, itself pinned by hand-worked cases in
test_oracle_feast.py.  Shared by the oracle pins and the CUDA parity
tests."""
import numpy as np

from oracle.feast import inside, select_pairs


def ritz_in_eigencoordinates(lam, C, anorm):
    """Ritz values (ascending) and relative residual norms of diag(lam) on
    span(C): Rayleigh-Ritz of A on span(Q C)."""
    U = np.linalg.svd(C, full_matrices=False)[0]
    H = U.conj().T @ (lam[:, None] * U)
    mu, V = np.linalg.eigh(0.5 * (H + H.conj().T))
    Y = U @ V
    return mu, np.linalg.norm(lam[:, None] * Y - Y * mu[None, :], axis=0) / anorm


def plain_feast_rounds(lam, C0, rho, anorm, a, b, rounds):
    """Plain FEAST is subspace iteration on rho(A) (Sect. I): round k works on
    span(rho(A)^k X0), here C_k = orth(diag(rho) C_{k-1}).  Per round: the
    Ritz values in (a, b) and their maximum residual."""
    C, out = C0, []
    for _ in range(rounds):
        C = np.linalg.qr(rho[:, None] * C)[0]
        mu, res = ritz_in_eigencoordinates(lam, C, anorm)
        ins = inside(mu, a, b)
        out.append((mu[ins], float(res[ins].max()) if ins.any() else np.inf))
    return out


def xfeast_round(lam, C0, rho, anorm, a, b, m0, s, k=1):
    """Round k = 1 or 2 of XFEAST (Sect. II-A): Rayleigh-Ritz on the Krylov
    window span[D^{k-1} C0, ..., D^{k+s-2} C0], D = diag(rho), then the
    m0-pair selection.  Round 1's window is [X0, rho X0, ..., rho^{s-1} X0]
    itself.  Round 2's is [rho X0, ..., rho^{s-1} X0, rho X_sel] with X_sel
    in round 1's window W, so it lies in rho(A) W, and equals it when it has
    full dimension s m0 (X_sel has components along rho^{s-1} X0 for a
    generic X0).  From round 3 on the window holds selections of two
    different rounds and no such closed form exists.  Returns the selected
    Ritz values in (a, b) (ascending) and their maximum residual."""
    if k not in (1, 2):
        raise ValueError(k)
    blocks = [C0 if k == 1 else rho[:, None] * C0]
    for _ in range(1, s):
        blocks.append(rho[:, None] * blocks[-1])
    mu, res = ritz_in_eigencoordinates(lam, np.hstack(blocks), anorm)
    sel = select_pairs(mu, res, a, b, m0)
    ins = sel[inside(mu[sel], a, b)]
    return np.sort(mu[ins]), float(res[ins].max())


def xfeast_first_round(lam, C0, rho, anorm, a, b, m0, s):
    """The first XFEAST round: xfeast_round with k = 1."""
    return xfeast_round(lam, C0, rho, anorm, a, b, m0, s, 1)


def rfeast_first_round_s2(lam, C0, rho, anorm, a, b, m0):
    """First RFEAST round with s = 2 (Sect. II-B), while no pair has
    converged after the first pass: Rayleigh-Ritz on Y = D C0 fixes the
    expected count m; every pair is selected, so the appended residuals add
    A Y and the second pass works on span[Y, A Y]; step 3 keeps the m
    selected in-I pairs of lowest residual.  Returns (m, their Ritz values
    ascending, their maximum residual, the first pass's smallest residual)."""
    Y = rho[:, None] * C0
    mu1, res1 = ritz_in_eigencoordinates(lam, Y, anorm)
    m = int(np.sum(inside(mu1, a, b)))
    mu, res = ritz_in_eigencoordinates(lam, np.hstack([Y, lam[:, None] * Y]), anorm)
    sel = select_pairs(mu, res, a, b, m0)
    ins = sel[inside(mu[sel], a, b)]
    keep = ins[np.lexsort((mu[ins], res[ins]))][:m]
    return m, np.sort(mu[keep]), float(res[keep].max()), float(res1.min())
