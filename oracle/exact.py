"""Exact FP64 dot products: the reference for the FP64-accurate products A Y
of the mixed precision's iterative refinement (R = X - (zI - A) Y).

The paper solves in full precision and has no refinement step; the product
these functions define is plain mathematics: sum_k a_k b_k of FP64 numbers,
correctly rounded to FP64.

Method: every product a*b is written exactly as p + e with p = fl(a*b) by
Dekker's TwoProduct (Veltkamp splitting into 26-bit halves, Dekker 1971), and
math.fsum (Shewchuk's exact summation) rounds the sum of all p and e once.
Valid while no product over- or underflows (|a*b| well inside 2^-969 ..
2^996), which holds for every test input.

Test infrastructure like the rest of oracle/.
"""
import math

import numpy as np

_SPLIT = 134217729.0  # 2^27 + 1


def _veltkamp(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    """p, e with p = fl(a b) and p + e == a b exactly (elementwise)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    p = a * b
    ah, al = _veltkamp(a)
    bh, bl = _veltkamp(b)
    e = al * bl - (((p - ah * bh) - al * bh) - ah * bl)
    return p, e


def dot_exact(x, y):
    """sum_k x_k y_k correctly rounded to FP64."""
    p, e = two_prod(np.ravel(x), np.ravel(y))
    return math.fsum(np.concatenate([p, e]).tolist())


def matmul_entries(A, B, rows, cols):
    """Exact (correctly rounded) entries C[rows[t], cols[t]] of C = A B."""
    return np.array([dot_exact(A[i, :], B[:, j]) for i, j in zip(rows, cols)])
