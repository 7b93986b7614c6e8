"""Quadrature of the FEAST contour integral (Sect. I, Eqs. 2-3).

The spectral projector is rho(A) = (1/2 pi i) \\oint_C (zI - A)^{-1} dz over a
closed contour C that encloses the search interval I = (lambda_min,
lambda_max) (Eq. 2), approximated by sum_j w_j (z_j I - A)^{-1} with Gauss
quadrature (Eq. 3).

Readings of the paper taken here (the paper names "Gauss quadrature" but gives
no contour or weight formula):
  * C is an ellipse centred at c = (lambda_min + lambda_max)/2 with horizontal
    semi-axis r = (lambda_max - lambda_min)/2 and vertical semi-axis a*r
    (a = 1, a circle, by default).
  * Gauss-Legendre nodes t_j on [-1, 1] are mapped to the upper half-contour by
    theta_j = (pi/2)(1 - t_j); z_j = c + r cos(theta_j) + i a r sin(theta_j).
  * The weight absorbs dz/(2 pi i) and the pi/2 Jacobian:
    w_j = (omega_j / 4) (a r cos(theta_j) + i r sin(theta_j)).
  * The lower half-contour is the mirror image; its nodes are conj(z_j) with
    weights conj(w_j).  So n_c counts the upper-half nodes, which is also the
    number of shifted factorisations.

Test infrastructure only: this package is imported by tests/, by the
package smoke check and by the CPU-baseline leg of bench.py, never by the
product path.
"""
from __future__ import annotations

import numpy as np


def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1]: nodes ascending, weights.

    Newton's method on the Legendre polynomial P_n, evaluated with the
    three-term recurrence (k+1) P_{k+1}(t) = (2k+1) t P_k(t) - k P_{k-1}(t),
    started from the estimate cos(pi (j - 1/4) / (n + 1/2)).  The weights are
    omega_j = 2 / ((1 - t_j^2) P_n'(t_j)^2) with
    P_n'(t) = n (t P_n(t) - P_{n-1}(t)) / (t^2 - 1).
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    j = np.arange(1, n + 1, dtype=np.float64)
    t = np.cos(np.pi * (j - 0.25) / (n + 0.5))

    def legendre(t):
        p_prev = np.ones_like(t)
        p = t.copy()
        for k in range(1, n):
            p_prev, p = p, ((2 * k + 1) * t * p - k * p_prev) / (k + 1)
        dp = n * (t * p - p_prev) / (t * t - 1.0)
        return p, dp

    for _ in range(100):
        p, dp = legendre(t)
        dt = p / dp
        t = t - dt
        if np.max(np.abs(dt)) < 1e-16:
            break
    p, dp = legendre(t)
    w = 2.0 / ((1.0 - t * t) * dp * dp)
    order = np.argsort(t)
    return t[order], w[order]


def contour_nodes(lmin: float, lmax: float, n_c: int, aspect: float = 1.0):
    """Upper-half-contour nodes z_j and weights w_j (complex arrays, length n_c).

    Ordered by ascending Gauss-Legendre abscissa t_j, i.e. from the node next
    to lambda_min towards the node next to lambda_max.
    """
    if not lmin < lmax:
        raise ValueError("lambda_min must be < lambda_max")
    t, om = gauss_legendre(n_c)
    c = 0.5 * (lmin + lmax)
    r = 0.5 * (lmax - lmin)
    theta = 0.5 * np.pi * (1.0 - t)
    z = c + r * np.cos(theta) + 1j * aspect * r * np.sin(theta)
    w = 0.25 * om * (aspect * r * np.cos(theta) + 1j * r * np.sin(theta))
    return z, w


def rational_filter(lam, z, w):
    """Scalar filter rho(lambda) = sum_j [w_j/(z_j - lambda) + conj(w_j)/(conj(z_j) - lambda)]
    = sum_j 2 Re(w_j / (z_j - lambda)) for real lambda (Eq. 3 applied to a
    1x1 matrix, both half-contours)."""
    lam = np.asarray(lam, dtype=np.float64)
    out = np.zeros(lam.shape, dtype=np.float64)
    for zj, wj in zip(z, w):
        out += 2.0 * np.real(wj / (zj - lam))
    return out
