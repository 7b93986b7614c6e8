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


def legendre_values(t, nmax):
    """P_0..P_{nmax-1} at the points t (rows: degree), three-term recurrence."""
    t = np.asarray(t, dtype=np.float64)
    P = np.zeros((nmax, t.size))
    P[0] = 1.0
    if nmax > 1:
        P[1] = t
    for k in range(1, nmax - 1):
        P[k + 1] = ((2 * k + 1) * t * P[k] - k * P[k - 1]) / (k + 1)
    return P


def offset_nodes(n_c: int, offsets):
    """Abscissae and weights of the interpolatory rule on moved nodes (the
    node placement a proposer may choose instead of Gauss-Legendre):
    t_j' = tanh(atanh(t_j) + delta_j) for the Gauss-Legendre t_j, and weights
    omega' solving sum_j omega'_j P_p(t_j') = integral of P_p over [-1, 1]
    (= 2 for p = 0, else 0), p < n_c: exact for polynomials of degree
    < n_c.  delta = 0 gives the Gauss rule back.  The moved nodes must stay
    strictly increasing."""
    t, om = gauss_legendre(n_c)
    d = np.asarray(offsets, dtype=np.float64)
    if d.size != n_c:
        raise ValueError("one offset per node")
    tp = np.tanh(np.arctanh(t) + d)
    if np.any(np.diff(tp) <= 0) or np.any(np.abs(tp) >= 1):
        raise ValueError("moved nodes must stay strictly increasing inside (-1, 1)")
    rhs = np.zeros(n_c)
    rhs[0] = 2.0
    omp = np.linalg.solve(legendre_values(tp, n_c), rhs)
    return tp, omp


def contour_nodes_offset(lmin: float, lmax: float, n_c: int, offsets, aspect: float = 1.0):
    """contour_nodes with the moved-node interpolatory rule of offset_nodes."""
    if not lmin < lmax:
        raise ValueError("lambda_min must be < lambda_max")
    t, om = offset_nodes(n_c, offsets)
    c = 0.5 * (lmin + lmax)
    r = 0.5 * (lmax - lmin)
    theta = 0.5 * np.pi * (1.0 - t)
    z = c + r * np.cos(theta) + 1j * aspect * r * np.sin(theta)
    w = 0.25 * om * (aspect * r * np.cos(theta) + 1j * r * np.sin(theta))
    return z, w


def circle_nodes(center: complex, radius: float, n_c: int):
    """Nodes and weights of the whole circle |z - center| = radius for a
    general (non-Hermitian) matrix, whose filter takes both half-circles:
    2 n_c nodes.  The first n_c are the upper half-circle nodes of the
    Hermitian rule (theta_j = (pi/2)(1 - t_j), z_j = center + r e^{i theta_j},
    w_j = (omega_j / 4) r e^{i theta_j}); the last n_c their mirror images
    z = center + r e^{-i theta_j}, w = (omega_j / 4) r e^{-i theta_j} (the
    Gauss-Legendre rule on the lower half, theta in (pi, 2 pi), has these
    nodes because the abscissae are symmetric).  With a real center the
    mirror is the complex conjugate."""
    if not radius > 0.0:
        raise ValueError("radius must be positive")
    t, om = gauss_legendre(n_c)
    theta = 0.5 * np.pi * (1.0 - t)
    e_up = np.exp(1j * theta)
    e_lo = np.exp(-1j * theta)
    z = np.concatenate([center + radius * e_up, center + radius * e_lo])
    w = np.concatenate([0.25 * om * radius * e_up, 0.25 * om * radius * e_lo])
    return z, w


def circle_filter(lam, z, w):
    """Scalar filter rho(lambda) = sum_k w_k / (z_k - lambda) of the whole
    circle at complex lambda (Eq. 3 applied to a 1 x 1 matrix)."""
    lam = np.asarray(lam, dtype=np.complex128)
    out = np.zeros(lam.shape, dtype=np.complex128)
    for zk, wk in zip(z, w):
        out += wk / (zk - lam)
    return out
