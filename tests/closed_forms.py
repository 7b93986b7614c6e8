"""Closed forms of FEAST iterates on planted spectra A = Q diag(lam) Q^H,
computed in the planted eigenbasis with LAPACK (SVD, eigh) and the rational
filter's values rho(lam): no linear solve, orthonormalisation or Jacobi of
the oracle or of the CUDA path is involved.  Shared by the oracle pins and
the CUDA parity tests."""
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


def xfeast_first_round(lam, C0, rho, anorm, a, b, m0, s):
    """First XFEAST round (Sect. II-A): Rayleigh-Ritz on the window
    [C0, D C0, ..., D^{s-1} C0], D = diag(rho), then the m0-pair selection.
    Returns the selected Ritz values in (a, b) (ascending) and their maximum
    residual."""
    blocks = [C0]
    for _ in range(1, s):
        blocks.append(rho[:, None] * blocks[-1])
    mu, res = ritz_in_eigencoordinates(lam, np.hstack(blocks), anorm)
    sel = select_pairs(mu, res, a, b, m0)
    ins = sel[inside(mu[sel], a, b)]
    return np.sort(mu[ins]), float(res[ins].max())


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
