"""Stochastic-trace Chebyshev moments of the spectral density (for the
learned m0 / node proposer; the paper names spectrum estimation as future
work in Sect. IV).

For a Hermitian A with spectrum inside [c - r, c + r], the scaled operator
B = (A - c I) / r has its spectrum in [-1, 1], and the k-th Chebyshev moment
of the spectral density is

    mu_k = (1/n) tr T_k(B) = (1/n) sum_i T_k(lambda_i'),  lambda_i' = (lambda_i - c)/r,

estimated with probe vectors v (columns of V, E[v v^H] = I) as
mu_k ~ (1/(n nv)) sum_v v^H T_k(B) v, where T_k(B) v follows the three-term
recurrence t_0 = v, t_1 = B v, t_{k+1} = 2 B t_k - t_{k-1}.  The probes are
inputs (the same seeded array for the oracle and the GPU path).

Jackson damping g_k (kernel polynomial method) turns the moments into a
non-negative density estimate; the proposer's features are the damped
moments g_k mu_k.

Test infrastructure only (see quadrature.py).
"""
from __future__ import annotations

import numpy as np


def chebyshev_moments(A, V, c, r, M):
    """mu_0..mu_{M-1} by the three-term recurrence on the probe block V."""
    A = np.asarray(A)
    V = np.asarray(V)
    n, nv = V.shape
    mu = np.zeros(M)
    t_prev = V.astype(np.complex128 if np.iscomplexobj(A) or np.iscomplexobj(V) else np.float64)
    mu[0] = np.real(np.vdot(V, t_prev)) / (n * nv)
    if M == 1:
        return mu
    t = (A @ t_prev - c * t_prev) / r
    mu[1] = np.real(np.vdot(V, t)) / (n * nv)
    for k in range(2, M):
        t_next = 2.0 * (A @ t - c * t) / r - t_prev
        mu[k] = np.real(np.vdot(V, t_next)) / (n * nv)
        t_prev, t = t, t_next
    return mu


def exact_moments(lam, c, r, M):
    """(1/n) sum_i T_k((lambda_i - c)/r) from the eigenvalues, T_k(x) = cos(k arccos x)."""
    x = (np.asarray(lam, dtype=np.float64) - c) / r
    th = np.arccos(np.clip(x, -1.0, 1.0))
    return np.array([np.mean(np.cos(k * th)) for k in range(M)])


def jackson(M):
    """Jackson damping factors g_0..g_{M-1} (Weisse et al., Rev. Mod. Phys. 78, 2006)."""
    k = np.arange(M, dtype=np.float64)
    q = np.pi / (M + 1)
    return ((M - k + 1) * np.cos(q * k) + np.sin(q * k) / np.tan(q)) / (M + 1)


def count_estimate(mu, c, r, a, b, n):
    """n times the damped density integrated over (a, b): with x = (lambda - c)/r
    and theta = arccos x, the integral of T_k(x) / (pi sqrt(1 - x^2)) over
    (x_a, x_b) is (theta_a - theta_b)/pi for k = 0 and
    2 (sin(k theta_a) - sin(k theta_b)) / (k pi) for k >= 1."""
    M = len(mu)
    g = jackson(M)
    ta = np.arccos(np.clip((a - c) / r, -1.0, 1.0))
    tb = np.arccos(np.clip((b - c) / r, -1.0, 1.0))
    s = g[0] * mu[0] * (ta - tb) / np.pi
    for k in range(1, M):
        s += g[k] * mu[k] * 2.0 * (np.sin(k * ta) - np.sin(k * tb)) / (k * np.pi)
    return n * s
