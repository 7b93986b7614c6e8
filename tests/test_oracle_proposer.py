"""Pins of the oracle parts of the learned m0 / node proposer: Chebyshev
moments (exact with a complete probe basis; the stochastic estimate within
its standard error), the kernel-polynomial count estimate, the moved-node
quadrature, and the MLP's gradients and Adam step."""
import numpy as np
import pytest

import oracle as O
from oracle.density import chebyshev_moments, count_estimate, exact_moments, jackson
from oracle.mlp import adam_step, backward, forward, init_params, loss
from oracle.quadrature import contour_nodes_offset, legendre_values, offset_nodes
from workloads import make_problem, spectrum_uniform


@pytest.mark.parametrize("cplx", [False, True])
def test_moments_exact_with_identity_probes(cplx):
    # with V = sqrt(n) I (each probe of squared norm n, like a Gaussian probe
    # in expectation) the trace estimator is the trace: (1/n) sum_i T_k(lambda_i')
    lam, a, b = spectrum_uniform(40, 6, seed=2, bulk=5.0)
    P = make_problem("m", lam, a, b, 8, 8, seed=2, complex_=cplx)
    c, r = 0.3, 1.05 * np.max(np.abs(lam - 0.3))
    mu = chebyshev_moments(P.A, np.sqrt(P.n) * np.eye(P.n), c, r, 48)
    np.testing.assert_allclose(mu, exact_moments(lam, c, r, 48), atol=1e-12)
    assert abs(mu[0] - 1.0) < 1e-14


def test_moments_stochastic_estimate_within_standard_error():
    # Gaussian probes: unbiased, variance of a single probe's estimate of
    # (1/n) tr f(B) is about 2 ||f(B)||_F^2 / n^2 <= 2/n for |T_k| <= 1
    lam, a, b = spectrum_uniform(300, 20, seed=4, bulk=5.0)
    P = make_problem("m", lam, a, b, 30, 8, seed=4)
    rng = np.random.default_rng(7)
    V = rng.standard_normal((P.n, 64))
    r = 1.02 * np.max(np.abs(lam))
    mu = chebyshev_moments(P.A, V, 0.0, r, 32)
    ex = exact_moments(lam, 0.0, r, 32)
    se = np.sqrt(2.0 / P.n / 64)
    assert np.all(np.abs(mu - ex) <= 5 * se)


def test_jackson_damping_and_count_estimate():
    g = jackson(64)
    assert abs(g[0] - 1.0) < 1e-15 and np.all(np.diff(g) < 0) and g[-1] > 0
    # eigenvalue count of an interval from the damped moments: close to the
    # exact count when the interval edges sit in gaps of the spectrum
    lam = np.concatenate([np.linspace(-9, -2, 70), np.linspace(-0.6, 0.6, 25), np.linspace(2, 9, 70)])
    mu = exact_moments(lam, 0.0, 10.0, 256)
    est = count_estimate(mu, 0.0, 10.0, -1.3, 1.3, lam.size)
    assert abs(est - 25) < 1.0
    # the whole spectrum: mu_0 = 1 gives n exactly
    assert abs(count_estimate(mu, 0.0, 10.0, -10.0, 10.0, lam.size) - lam.size) < 1e-9


def test_offset_nodes_zero_is_gauss_and_rule_is_exact():
    for n_c in (3, 8, 12):
        t, w = O.gauss_legendre(n_c)
        tp, wp = offset_nodes(n_c, np.zeros(n_c))
        np.testing.assert_allclose(tp, t, atol=1e-15)
        np.testing.assert_allclose(wp, w, atol=1e-14)
    # moved nodes: interpolatory, so exact for every polynomial of degree < n_c
    n_c = 8
    d = np.array([-0.3, -0.1, 0.05, 0.0, 0.1, -0.05, 0.2, 0.25])
    tp, wp = offset_nodes(n_c, d)
    rng = np.random.default_rng(1)
    coef = rng.standard_normal(n_c)            # a random polynomial of degree n_c - 1
    poly = np.polynomial.Polynomial(coef)
    exact = poly.integ()(1.0) - poly.integ()(-1.0)
    assert abs(np.sum(wp * poly(tp)) - exact) < 1e-13
    # and not for degree n_c (in general)
    P = legendre_values(tp, n_c + 1)[n_c]
    assert abs(np.sum(wp * P)) > 1e-6
    with pytest.raises(ValueError):
        offset_nodes(n_c, np.array([0, 0, 0, 3.0, -3.0, 0, 0, 0]))   # crossing nodes


def test_offset_contour_reduces_to_gauss_and_keeps_filter_values():
    z, w = contour_nodes_offset(-1.0, 1.0, 8, np.zeros(8))
    z0, w0 = O.contour_nodes(-1.0, 1.0, 8)
    np.testing.assert_allclose(z, z0, atol=1e-15)
    np.testing.assert_allclose(w, w0, atol=1e-15)
    # moving the outer nodes towards the edges sharpens the filter just
    # outside I (rho(1.01) drops) at the price of the far rejection
    d = 0.3 * np.array([-1, -0.5, -0.2, 0, 0, 0.2, 0.5, 1.0])
    z1, w1 = contour_nodes_offset(-1.0, 1.0, 8, d)
    r0 = O.rational_filter(np.array([0.0, 1.01, 2.0]), z0, w0)
    r1 = O.rational_filter(np.array([0.0, 1.01, 2.0]), z1, w1)
    assert r1[1] < r0[1] and abs(r1[2]) > abs(r0[2])
    assert abs(r1[0] - 1.0) < 1e-3


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    layers = [(6, 16), (16, 16), (16, 16), (16, 3)]
    ps = init_params(seed=5, layers=layers)
    for i in range(1, len(ps), 2):
        ps[i] = 0.1 * rng.standard_normal(ps[i].shape)   # nonzero biases
    X = rng.standard_normal((7, 6))
    T = rng.standard_normal((7, 3))
    grads = backward(ps, X, T)
    h = 1e-6
    for i in range(len(ps)):
        for _ in range(4):
            idx = tuple(rng.integers(0, s) for s in ps[i].shape)
            old = ps[i][idx]
            ps[i][idx] = old + h
            lp = loss(ps, X, T)
            ps[i][idx] = old - h
            lm = loss(ps, X, T)
            ps[i][idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(grads[i][idx] - fd) <= 1e-6 * max(1.0, abs(fd)), (i, idx, grads[i][idx], fd)


def test_adam_first_step_closed_form():
    # at step 1 the bias-corrected moments are g and g^2, so the update is
    # -lr g / (|g| + eps): a step of size lr per coordinate in the sign of -g
    ps = [np.array([1.0, -2.0, 0.5])]
    g = [np.array([0.3, -4.0, 1e-3])]
    m, v = [np.zeros(3)], [np.zeros(3)]
    adam_step(ps, g, m, v, step=1, lr=0.01, eps=1e-8)
    np.testing.assert_allclose(ps[0], np.array([1.0, -2.0, 0.5]) - 0.01 * g[0] / (np.abs(g[0]) + 1e-8), rtol=1e-14)


def test_mlp_forward_shapes_and_relu():
    ps = init_params(seed=1)
    X = np.random.default_rng(0).standard_normal((5, 64))
    Y, acts = forward(ps, X)
    assert Y.shape == (5, 9) and len(acts) == 5
    assert all(np.all(h >= 0) for h in acts[1:4])
