"""Pins of the oracle's quadrature (Eqs. 2-3) against closed forms and an
independent Gauss-Legendre implementation."""
import json
import os

import numpy as np
import pytest

from oracle import contour_nodes, gauss_legendre, rational_filter
import oracle.quadrature as quad

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_setups.json")


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 13, 16, 24, 32])
def test_gauss_legendre_matches_numpy(n):
    t, w = gauss_legendre(n)
    t_ref, w_ref = np.polynomial.legendre.leggauss(n)
    np.testing.assert_allclose(t, t_ref, atol=2e-15)
    np.testing.assert_allclose(w, w_ref, rtol=0, atol=5e-15)


@pytest.mark.parametrize("n", [1, 3, 8, 16])
def test_gauss_legendre_exact_for_degree_2n_minus_1(n):
    t, w = gauss_legendre(n)
    for p in range(2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * t ** p) - exact) < 1e-14


@pytest.mark.parametrize("n_c", [1, 3, 8, 16])
@pytest.mark.parametrize("lmin,lmax", [(-1.0, 1.0), (0.3, 7.9), (-120.0, -20.0)])
def test_filter_special_values_on_circle(n_c, lmin, lmax):
    # circle + Gauss-Legendre: rho(centre) = sum(omega)/2 = 1 and
    # rho(edge) = sum(omega)/4 = 1/2 exactly (Re[1/(1 - e^{-i theta})] = 1/2)
    z, w = contour_nodes(lmin, lmax, n_c)
    c = 0.5 * (lmin + lmax)
    scale = max(1.0, abs(c) / (0.5 * (lmax - lmin)))
    assert abs(rational_filter(c, z, w) - 1.0) < 1e-14 * scale
    assert abs(rational_filter(lmin, z, w) - 0.5) < 1e-13 * scale
    assert abs(rational_filter(lmax, z, w) - 0.5) < 1e-13 * scale


def test_filter_converges_to_indicator():
    # with many nodes the quadrature approaches the exact contour integral:
    # 1 strictly inside I, 0 outside (Eq. 2)
    z, w = contour_nodes(-1.0, 1.0, 64)
    inside = np.array([-0.9, -0.5, 0.0, 0.3, 0.85])
    outside = np.array([-3.0, -1.2, 1.2, 2.0, 10.0])
    np.testing.assert_allclose(rational_filter(inside, z, w), 1.0, atol=1e-8)
    np.testing.assert_allclose(rational_filter(outside, z, w), 0.0, atol=1e-8)


def test_nodes_lie_on_upper_half_ellipse():
    lmin, lmax, a = -2.0, 6.0, 0.3
    z, w = contour_nodes(lmin, lmax, 8, aspect=a)
    c, r = 2.0, 4.0
    assert np.all(z.imag > 0)
    np.testing.assert_allclose(((z.real - c) / r) ** 2 + (z.imag / (a * r)) ** 2, 1.0, atol=1e-14)
    # weights carry the contour tangent dz/dtheta = -r sin + i a r cos, times
    # omega pi/2 /(2 pi i):  w = omega/4 (a r cos + i r sin)
    th = np.arctan2(z.imag / a, z.real - c)
    t, om = gauss_legendre(8)
    tangent = -r * np.sin(th) + 1j * a * r * np.cos(th)
    np.testing.assert_allclose(w, 0.5 * np.pi * om * tangent / (2j * np.pi), atol=1e-14)


def test_filter_matches_independent_trapezoid_contour_integral():
    # The quadrature sum approximates (1/2 pi i) \oint dz/(z - lambda); an
    # independent 4000-point trapezoid rule on the full circle (exponentially
    # accurate for periodic integrands) gives the exact indicator, and a
    # 64-node Gauss rule must agree with it away from the edges.
    lam = np.array([-0.7, 0.2, 1.6, -2.5])
    th = np.linspace(0, 2 * np.pi, 4000, endpoint=False)
    zc = np.exp(1j * th)
    dz = 1j * np.exp(1j * th) * (2 * np.pi / th.size)
    trap = np.array([np.real(np.sum(dz / (zc - l)) / (2j * np.pi)) for l in lam])
    np.testing.assert_allclose(trap, [1, 1, 0, 0], atol=1e-12)
    z, w = contour_nodes(-1.0, 1.0, 64)
    np.testing.assert_allclose(rational_filter(lam, z, w), trap, atol=1e-6)


def test_planted_mistake_in_weights_is_caught(monkeypatch):
    # A dropped factor of 1/2 in the weights (omega/2 instead of omega/4)
    # must break the rho(centre) = 1 pin.
    orig = quad.contour_nodes

    def wrong(lmin, lmax, n_c, aspect=1.0):
        z, w = orig(lmin, lmax, n_c, aspect)
        return z, 2.0 * w

    monkeypatch.setattr(quad, "contour_nodes", wrong)
    z, w = quad.contour_nodes(-1.0, 1.0, 8)
    assert abs(rational_filter(0.0, z, w) - 1.0) > 0.5


@pytest.mark.parametrize("n_c", [2, 4, 8, 16])
def test_filter_above_half_exactly_inside_the_circle(n_c):
    # the XFEAST/RFEAST filter-response test keeps a pair inside I only if
    # mu = x^H rho(A) x exceeds 1/2; that separates I from its complement
    # because, for the circle, rho(lambda) > 1/2 strictly inside I and < 1/2
    # outside (with rho = 1/2 at the edges): checked on a dense grid, up to
    # 1e-6 of the half-width from each edge
    lmin, lmax = -1.0, 1.0
    z, w = contour_nodes(lmin, lmax, n_c)
    inside = np.linspace(lmin + 1e-6, lmax - 1e-6, 20001)
    outside = np.concatenate([np.linspace(lmax + 1e-6, 60.0, 20001), np.linspace(-60.0, lmin - 1e-6, 20001)])
    assert np.all(rational_filter(inside, z, w) > 0.5)
    assert np.all(rational_filter(outside, z, w) < 0.5)
    # and a mixture of eigenvectors from outside I responds below 1/2
    rng = np.random.default_rng(n_c)
    c = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    c /= np.linalg.norm(c)
    lam_out = rng.choice(outside, 40)
    assert np.sum(np.abs(c) ** 2 * rational_filter(lam_out, z, w)) < 0.5


@pytest.mark.parametrize("m", [50, 100, 200])
def test_rate_of_order_ten_thousand_at_n_c_8_and_m0_one_and_a_half_m(m):
    # Sect. I: FEAST's rate is rho(lambda_i) / rho(lambda_{m0+1}) (the
    # (m0+1)-th largest filter value), and with n_c = 8 and m0 ~ 1.5 m a rate
    # of 10^4 is common.  For a spectrum of uniform density across I and far
    # beyond, the worst in-I eigenvalue (half a spacing from an edge, rho ~
    # 1/2) gets 3-4e3 and the median one ~5e3: order 10^4, and far from what
    # another rule gives (n_c = 2: 6-11; n_c = 16: ~3e7)
    g = json.load(open(GOLDEN))["typical_rate"]
    z, w = contour_nodes(-1.0, 1.0, g["n_c"])
    h = 2.0 / m
    lam = np.arange(-50.0 + h / 2, 50.0, h)
    rho = np.abs(rational_filter(lam, z, w))
    ins = (lam > -1.0) & (lam < 1.0)
    assert ins.sum() == m
    nxt = np.sort(rho)[::-1][int(g["m0_over_m"] * m)]
    lo, hi = g["rate_order"] / 10, g["rate_order"] * 10
    assert lo <= rho[ins].min() / nxt <= hi
    assert lo <= np.median(rho[ins]) / nxt <= hi
