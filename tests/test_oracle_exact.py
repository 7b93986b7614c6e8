"""Pins of the exact dot product (oracle/exact.py) against rational
arithmetic: TwoProduct is error-free and the dot product is the correctly
rounded exact sum, bit for bit."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import exact


def _rand(rng, k, spread):
    return rng.standard_normal(k) * np.exp2(rng.integers(-spread, spread + 1, k))


@pytest.mark.parametrize("spread", [0, 20, 200])
def test_two_prod_is_error_free(spread):
    rng = np.random.default_rng(spread)
    a, b = _rand(rng, 500, spread), _rand(rng, 500, spread)
    p, e = exact.two_prod(a, b)
    for ai, bi, pi, ei in zip(a, b, p, e):
        assert Fraction(pi) + Fraction(ei) == Fraction(ai) * Fraction(bi)
        assert pi == ai * bi


@pytest.mark.parametrize("k,spread", [(1, 0), (7, 3), (1000, 0), (1000, 30), (300, 300)])
def test_dot_exact_is_correctly_rounded(k, spread):
    rng = np.random.default_rng(k + spread)
    x, y = _rand(rng, k, spread), _rand(rng, k, spread)
    ref = sum((Fraction(a) * Fraction(b) for a, b in zip(x, y)), Fraction(0))
    got = exact.dot_exact(x, y)
    assert Fraction(got) == Fraction(float(ref)) or got == float(ref)


def test_dot_exact_cancellation():
    # a sum whose naive FP64 evaluation loses every digit: exact result 2^-60
    x = np.array([1.0, 2.0 ** -60, -1.0])
    y = np.array([1.0, 1.0, 1.0])
    assert float(np.dot(x, y)) == 0.0
    assert exact.dot_exact(x, y) == 2.0 ** -60
    # products that cancel up to their rounding errors
    a = 1.0 + 2.0 ** -30
    assert exact.dot_exact([a, -1.0], [a, 1.0 + 2.0 ** -29]) == 2.0 ** -60


def test_matmul_entries_matches_fraction_product():
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((6, 40)), rng.standard_normal((40, 5))
    rows, cols = np.array([0, 3, 5, 2]), np.array([4, 0, 2, 2])
    got = exact.matmul_entries(A, B, rows, cols)
    for t, (i, j) in enumerate(zip(rows, cols)):
        ref = sum((Fraction(A[i, k]) * Fraction(B[k, j]) for k in range(40)), Fraction(0))
        assert got[t] == float(ref)
