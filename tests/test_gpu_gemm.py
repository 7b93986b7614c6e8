"""Parity of the FP64-accurate GEMM of the mixed precision's refinement
(C = A B, feast_gemm_f64acc) with exact, correctly rounded dot products
(oracle.exact), on sampled entries.

method 0 (bf16 tensor cores, digit splitting) is held to its bound
2^-45 K 2^(e_i + f_j) with 2^e_i > max_k |A_ik|, 2^f_j > max_k |B_kj|; the
expected error is about 2^-48 sqrt(K) 2^(e_i + f_j).  A tensor-core sum that
were not exact would leave errors near 2^-24 of a 128-term digit sum, orders
of magnitude above the bound.  method 1 (double-float) is held to
2^-44 sum_k |A_ik| |B_kj|."""
import numpy as np
import pytest

import oracle as O
import paper_1605_08771_gb300 as fg
from gpu_common import ctx, cuda, host  # noqa: F401

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (2, 3, 5), (130, 97, 33), (129, 191, 128), (300, 200, 1000), (257, 96, 4099)]


def _pow2_above(v):
    e = np.frexp(v)[1]
    return np.where(v > 0, np.ldexp(1.0, e), 0.0)


def _sample(M, N, count, seed):
    rng = np.random.default_rng(seed)
    t = min(count, M * N)
    idx = rng.choice(M * N, size=t, replace=False)
    rows, cols = idx % M, idx // M
    # always include the corners and the ragged edge
    extra_r = np.array([0, M - 1, M - 1, 0])
    extra_c = np.array([0, N - 1, 0, N - 1])
    return np.concatenate([rows, extra_r]), np.concatenate([cols, extra_c])


def _check(A, B, C, method, seed):
    M, K = A.shape
    N = B.shape[1]
    rows, cols = _sample(M, N, 300, seed)
    ref = O.matmul_entries(A, B, rows, cols)
    err = np.abs(C[rows, cols] - ref)
    if method == 0:
        sa = _pow2_above(np.abs(A).max(axis=1))[rows]
        sb = _pow2_above(np.abs(B).max(axis=0))[cols]
        bound = 2.0 ** -45 * K * sa * sb
    else:
        bound = 2.0 ** -44 * np.array([np.abs(A[i, :]) @ np.abs(B[:, j]) for i, j in zip(rows, cols)])
    assert np.all(err <= bound), (err / np.maximum(bound, 1e-300)).max()
    return err


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("method", [0, 1])
def test_gemm_f64acc_gaussian(ctx, M, N, K, method):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = host(fg.feast_gemm_f64acc(ctx, cuda(A), cuda(B), method))
    _check(A, B, C, method, seed=K)


@pytest.mark.parametrize("method", [0, 1])
def test_gemm_f64acc_row_and_column_scales(ctx, method):
    # rows of A and columns of B spread over 2^-40 .. 2^40: each output keeps
    # its own relative accuracy (per-row and per-column exponents)
    rng = np.random.default_rng(11)
    M, N, K = 200, 150, 700
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-40, 41, M))[:, None]
    B = rng.standard_normal((K, N)) * np.exp2(rng.integers(-40, 41, N))[None, :]
    A[3, :] = 0.0                      # an all-zero row
    B[:, 5] = 0.0                      # and column
    C = host(fg.feast_gemm_f64acc(ctx, cuda(A), cuda(B), method))
    _check(A, B, C, method, seed=1)
    assert np.all(C[3, :] == 0.0) and np.all(C[:, 5] == 0.0)


def test_gemm_f64acc_largest_digit_sums(ctx):
    # every element just below a power of two with the same sign: every
    # digit-product sum of a 128-wide chunk reaches its largest value
    # (2^23 for the leading digits), the case the exactness argument bounds
    M, N, K = 128, 96, 4096
    v = 1.0 - 2.0 ** -9
    A = np.full((M, K), v)
    B = np.full((K, N), v)
    B[:, 1] = -v
    C = host(fg.feast_gemm_f64acc(ctx, cuda(A), cuda(B), 0))
    exact = K * v * v                   # exactly representable
    assert np.all(C[:, 0] == exact) and np.all(C[:, 1] == -exact)
    assert np.all(C == np.where(np.arange(N) == 1, -exact, exact)[None, :])


def test_gemm_f64acc_digits_beyond_fp32(ctx):
    # entries that differ from a base matrix only 2^-32 below their leading
    # bit: a product through FP32 (or through bf16/TF32 without the digit
    # split) cannot see the difference; the split resolves it to ~2^-10
    rng = np.random.default_rng(3)
    M, N, K = 160, 100, 512
    base = rng.standard_normal((M, K))
    A = base + base * 2.0 ** -32 * rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    C = host(fg.feast_gemm_f64acc(ctx, cuda(A), cuda(B), 0))
    Cb = host(fg.feast_gemm_f64acc(ctx, cuda(base), cuda(B), 0))
    rows, cols = _sample(M, N, 200, 9)
    d_ref = O.matmul_entries(A, B, rows, cols) - O.matmul_entries(base, B, rows, cols)
    d = C[rows, cols] - Cb[rows, cols]
    sa = _pow2_above(np.abs(A).max(axis=1))[rows]
    sb = _pow2_above(np.abs(B).max(axis=0))[cols]
    assert np.all(np.abs(d - d_ref) <= 2.0 ** -44 * K * sa * sb)
    assert np.median(np.abs(d - d_ref) / np.abs(d_ref)) < 0.01


def _exact_complex(A, B, rows, cols):
    # (Ar + i Ai)(Br + i Bi) entrywise from four exact real dot products
    Ar, Ai, Br, Bi = A.real.copy(), A.imag.copy(), B.real.copy(), B.imag.copy()
    re = np.array([O.dot_exact(np.concatenate([Ar[i], -Ai[i]]), np.concatenate([Br[:, j], Bi[:, j]]))
                   for i, j in zip(rows, cols)])
    im = np.array([O.dot_exact(np.concatenate([Ar[i], Ai[i]]), np.concatenate([Bi[:, j], Br[:, j]]))
                   for i, j in zip(rows, cols)])
    return re + 1j * im


# sizes with several output tiles per persistent CTA (more tiles than SMs)
# and a partial last K chunk (K % 128 != 0)
@pytest.mark.parametrize("M,N,K", [(2000, 900, 900), (700, 300, 8192), (129, 97, 161)])
@pytest.mark.parametrize("transA,transB", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_f64acc_complex_ops(ctx, M, N, K, transA, transB):
    rng = np.random.default_rng(M + N + K + 2 * transA + transB)
    opA = rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))
    opB = rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))
    A = opA.conj().T if transA else opA
    B = opB.conj().T if transB else opB
    C0 = rng.standard_normal((M, N)) + 1j * rng.standard_normal((M, N))
    alpha, beta = -1.0, 0.5
    C = host(fg.feast_gemm_f64acc(ctx, cuda(np.asfortranarray(A)), cuda(np.asfortranarray(B)), 0,
                                  transA=transA, transB=transB, alpha=alpha, beta=beta,
                                  C=cuda(np.asfortranarray(C0))))
    rows, cols = _sample(M, N, 150, 5)
    ref = alpha * _exact_complex(opA, opB, rows, cols) + beta * C0[rows, cols]
    scale = (np.abs(opA).max(axis=1)[rows] * np.abs(opB).max(axis=0)[cols]) * K
    assert np.all(np.abs(C[rows, cols] - ref) <= 2.0 ** -42 * scale + 4e-16 * np.abs(ref))


@pytest.mark.parametrize("transA", [False, True])
def test_gemm_f64acc_real_transposed(ctx, transA):
    rng = np.random.default_rng(21 + transA)
    M, N, K = 1500, 700, 300
    opA = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    A = opA.T.copy() if transA else opA
    C = host(fg.feast_gemm_f64acc(ctx, cuda(np.asfortranarray(A)), cuda(B), 0, transA=transA))
    _check(opA, B, C, 0, seed=3)


def test_gemm_f64acc_rejects_bad_arguments(ctx):
    import torch
    A = torch.zeros((4, 3), dtype=torch.float64, device="cuda:0")
    B = torch.zeros((4, 2), dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        fg.feast_gemm_f64acc(ctx, A, B, 0)
    with pytest.raises(RuntimeError):
        fg.feast_gemm_f64acc(ctx, A, A.T.contiguous(), 2)
    with pytest.raises(RuntimeError):   # the double-float route has no transposes
        fg.feast_gemm_f64acc(ctx, A, B, 1, transA=True)
