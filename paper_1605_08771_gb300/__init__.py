"""FEAST interval eigensolver on one GB300: thin Python binding.

Every function here marshals arguments to the C ABI of libfeast_gb300.so
(declared in include/feast.h) and nothing else: all arithmetic runs in the
library's CUDA kernels.  PyTorch supplies device memory and the stream.  If
the shared library is missing or a tensor is not on a CUDA device, the calls
raise; there is no CPU fallback.

Layout: the library is column-major.  Input tensors of any layout are copied
to column-major device memory; returned matrices are column-major views
(shape (n, m), strides (1, n)).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB, build as build_library  # noqa: F401

FEAST_R64, FEAST_C128 = 0, 1
FEAST_PLAIN, FEAST_XFEAST, FEAST_RFEAST = 0, 1, 2
FEAST_PREC_F64, FEAST_PREC_MIXED, FEAST_PREC_MIXED_SIMT = 0, 1, 2
FEAST_OK, FEAST_WARN_MAXITER = 0, 1

VARIANTS = {"feast": FEAST_PLAIN, "xfeast": FEAST_XFEAST, "rfeast": FEAST_RFEAST}
PRECS = {"f64": FEAST_PREC_F64, "mixed": FEAST_PREC_MIXED, "mixed_simt": FEAST_PREC_MIXED_SIMT}

EXPORTS = [
    "feast_opts_default", "feast_init", "feast_finalize", "feast_strerror",
    "feast_contour_nodes", "feast_interval_solve", "feast_filter_apply",
    "feast_shifted_lu", "feast_shifted_solve", "feast_orthonormalize",
    "feast_jacobi_eigh", "feast_rayleigh_ritz", "feast_kernel_launches", "feast_jacobi_eigh_noalloc",
    "feast_gemm_f64acc", "feast_contour_nodes_offset", "feast_spectral_moments", "feast_moments_count",
    "feast_mlp_param_count", "feast_mlp_forward", "feast_mlp_gradient", "feast_mlp_train_step",
    "feast_interval_solve_batch", "feast_interval_solve_gen",
    "feast_circle_nodes", "feast_eig_general", "feast_filter_apply_general", "feast_disk_solve",
]


class FeastOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("s", ctypes.c_int), ("prec", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("refine_max", ctypes.c_int), ("refine_gemm", ctypes.c_int),
                ("aspect", ctypes.c_double), ("anorm", ctypes.c_double), ("refine_tol", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("x0", ctypes.c_void_p), ("refine_switch", ctypes.c_double),
                ("rfeast_expand", ctypes.c_int), ("response_stop", ctypes.c_int),
                ("reserved", ctypes.c_int), ("node_offsets", ctypes.c_void_p)]


class FeastStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("filters", ctypes.c_int), ("refine_steps", ctypes.c_int),
                ("m_expected", ctypes.c_int), ("factor_ms", ctypes.c_double), ("filter_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double), ("max_residual", ctypes.c_double),
                ("history", ctypes.c_double * 128), ("refine_gemm_ms", ctypes.c_double),
                ("refine_gemm_mac", ctypes.c_double), ("refine_gemm_launches", ctypes.c_int),
                ("cgemm_launches", ctypes.c_int), ("cgemm_ms", ctypes.c_double), ("cgemm_flop", ctypes.c_double),
                ("tcgemm_launches", ctypes.c_int), ("tcgemm_ms", ctypes.c_double), ("tcgemm_flop", ctypes.c_double),
                ("rr_passes", ctypes.c_int), ("rr_k_sum", ctypes.c_double), ("rr_k3_sum", ctypes.c_double)]


class FeastProblem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("dtype", ctypes.c_int), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("lmin", ctypes.c_double), ("lmax", ctypes.c_double), ("tol", ctypes.c_double),
                ("m0", ctypes.c_int), ("n_c", ctypes.c_int), ("evals", ctypes.c_void_p), ("evecs", ctypes.c_void_p),
                ("res", ctypes.c_void_p), ("m_found", ctypes.c_int), ("iterations", ctypes.c_int),
                ("status", ctypes.c_int), ("route", ctypes.c_int), ("ms", ctypes.c_double)]


class FeastError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {feast_strerror(code)} (status {code})")


_LIB = None


def lib():
    """Load libfeast_gb300.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB):
        raise RuntimeError(f"{LIB} is missing: build it with paper_1605_08771_gb300.build.build()")
    L = ctypes.CDLL(LIB)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    DP, IP = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    sig = {
        "feast_opts_default": (None, [ctypes.POINTER(FeastOpts)]),
        "feast_init": (I, [ctypes.POINTER(P), I, P]),
        "feast_finalize": (I, [P]),
        "feast_strerror": (ctypes.c_char_p, [I]),
        "feast_contour_nodes": (I, [D, D, I, D, DP, DP]),
        "feast_interval_solve": (I, [P, P, I, I64, I64, D, D, I, I, D, ctypes.POINTER(FeastOpts),
                                     DP, P, DP, IP, IP, ctypes.POINTER(FeastStats)]),
        "feast_filter_apply": (I, [P, P, I, I64, I64, D, D, I, ctypes.POINTER(FeastOpts), P, I64, P]),
        "feast_shifted_lu": (I, [P, P, I, I64, I64, DP, I, I, P, P]),
        "feast_shifted_solve": (I, [P, P, P, I64, I, I, I, P, I64, P]),
        "feast_orthonormalize": (I, [P, I, I64, I64, P, I, IP]),
        "feast_jacobi_eigh": (I, [P, I, I64, P, DP, P, IP]),
        "feast_rayleigh_ritz": (I, [P, P, I, I64, I64, P, I64, D, DP, P, DP]),
        "feast_kernel_launches": (ctypes.c_uint64, []),
        "feast_jacobi_eigh_noalloc": (I, [I, P, I, I64, P, DP, P, IP]),
        "feast_gemm_f64acc": (I, [P, I, I, I, I, I64, I64, I64, D, P, I64, P, I64, D, P, I64]),
        "feast_contour_nodes_offset": (I, [D, D, I, D, DP, DP, DP]),
        "feast_spectral_moments": (I, [P, P, I, I64, I64, D, D, P, I64, I, DP]),
        "feast_moments_count": (D, [DP, I, D, D, D, D, I64]),
        "feast_mlp_param_count": (I, []),
        "feast_mlp_forward": (I, [P, P, P, I64, P]),
        "feast_mlp_gradient": (I, [P, P, P, P, I64, P, DP]),
        "feast_mlp_train_step": (I, [P, P, P, P, P, P, I64, I, D, DP]),
        "feast_interval_solve_batch": (I, [I, I, ctypes.POINTER(FeastProblem), ctypes.POINTER(FeastOpts), I, I]),
        "feast_interval_solve_gen": (I, [P, P, P, I, I64, I64, I64, D, D, I, I, D, ctypes.POINTER(FeastOpts),
                                         DP, P, DP, IP, IP, ctypes.POINTER(FeastStats)]),
        "feast_circle_nodes": (I, [D, D, D, I, DP, DP]),
        "feast_eig_general": (I, [P, I64, P, DP, P, IP]),
        "feast_filter_apply_general": (I, [P, P, I, I64, I64, D, D, D, I, P, I64, P]),
        "feast_disk_solve": (I, [P, P, I, I64, I64, D, D, D, I, I, D, I, P, DP, P, DP, IP, IP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return FEAST_R64
    if t.dtype == torch.complex128:
        return FEAST_C128
    raise TypeError(f"unsupported dtype {t.dtype}: use float64 or complex128")


def colmajor(t):
    """Column-major (Fortran-order) device copy of a 2-D tensor, as a view of
    shape t.shape with strides (1, rows)."""
    if not t.is_cuda:
        raise ValueError("FEAST takes CUDA tensors (no CPU path)")
    if t.dim() == 1:
        t = t[:, None]
    if t.stride(0) == 1 and t.stride(1) == t.shape[0]:
        return t
    return t.transpose(0, 1).contiguous().transpose(0, 1)


def empty_colmajor(rows, cols, dtype, device):
    torch = _torch()
    return torch.empty((cols, rows), dtype=dtype, device=device).transpose(0, 1)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check(code, where):
    if code < 0:
        raise FeastError(code, where)
    return code


# ---------------------------------------------------------------------------
# C-ABI mirror
# ---------------------------------------------------------------------------
def feast_strerror(code: int) -> str:
    return lib().feast_strerror(int(code)).decode()


def feast_kernel_launches() -> int:
    return int(lib().feast_kernel_launches())


def feast_opts_default(**kw) -> FeastOpts:
    """Default options with keyword overrides; node_offsets takes a sequence
    of n_c floats (kept alive by the returned structure)."""
    o = FeastOpts()
    lib().feast_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "variant" and isinstance(v, str):
            v = VARIANTS[v]
        if k == "prec" and isinstance(v, str):
            v = PRECS[v]
        if k == "node_offsets":
            if v is None:
                o.node_offsets = None
                continue
            arr = np.ascontiguousarray(v, dtype=np.float64)
            o._offsets_keep = arr
            v = arr.ctypes.data
        setattr(o, k, v)
    return o


def feast_init(device: int = 0, stream=None):
    """Create a library context on `device`; `stream` is a torch.cuda.Stream
    (default: the current stream)."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream(device)
    h = ctypes.c_void_p()
    _check(lib().feast_init(ctypes.byref(h), int(device), ctypes.c_void_p(stream.cuda_stream)), "feast_init")
    return h


def feast_finalize(ctx) -> None:
    _check(lib().feast_finalize(ctx), "feast_finalize")


def feast_contour_nodes(lmin, lmax, n_c, aspect=1.0):
    z = np.zeros(2 * n_c)
    w = np.zeros(2 * n_c)
    _check(lib().feast_contour_nodes(lmin, lmax, n_c, aspect,
                                     z.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "feast_contour_nodes")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def feast_contour_nodes_offset(lmin, lmax, n_c, offsets, aspect=1.0):
    """Contour nodes and weights of the moved-node interpolatory rule."""
    z = np.zeros(2 * n_c)
    w = np.zeros(2 * n_c)
    d = np.ascontiguousarray(offsets, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().feast_contour_nodes_offset(lmin, lmax, n_c, aspect, d.ctypes.data_as(dp), z.ctypes.data_as(dp),
                                            w.ctypes.data_as(dp)), "feast_contour_nodes_offset")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def feast_spectral_moments(ctx, A, V, c, r, M):
    """Chebyshev moments mu_0..mu_{M-1} of the spectral density of the CUDA
    matrix A scaled to (A - c I)/r, from the CUDA probe block V (n x nv)."""
    A = colmajor(A)
    V = colmajor(V.to(A.dtype))
    n, nv = V.shape
    mu = np.zeros(M)
    _check(lib().feast_spectral_moments(ctx, _ptr(A), _dtype_code(A), n, n, float(c), float(r), _ptr(V), nv, int(M),
                                        mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "feast_spectral_moments")
    return mu


def feast_moments_count(mu, c, r, a, b, n):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    return float(lib().feast_moments_count(mu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), mu.size, float(c),
                                           float(r), float(a), float(b), int(n)))


def feast_mlp_param_count() -> int:
    return int(lib().feast_mlp_param_count())


def _f32(t):
    torch = _torch()
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError("MLP arrays are contiguous float32 CUDA tensors")
    return _ptr(t)


def feast_mlp_forward(ctx, params, X):
    """Outputs (B x 9) of the proposer MLP for the CUDA float32 batch X (B x 64)."""
    torch = _torch()
    B = X.shape[0]
    Y = torch.empty((B, 9), dtype=torch.float32, device=X.device)
    _check(lib().feast_mlp_forward(ctx, _f32(params), _f32(X), B, _ptr(Y)), "feast_mlp_forward")
    return Y


def feast_mlp_gradient(ctx, params, X, T):
    """(gradient, loss) of the mean squared error of the batch."""
    torch = _torch()
    g = torch.empty_like(params)
    loss = ctypes.c_double(0.0)
    _check(lib().feast_mlp_gradient(ctx, _f32(params), _f32(X), _f32(T), X.shape[0], _ptr(g), ctypes.byref(loss)),
           "feast_mlp_gradient")
    return g, loss.value


def feast_mlp_train_step(ctx, params, m, v, X, T, step, lr):
    """One Adam step in place; returns the batch loss before the step."""
    loss = ctypes.c_double(0.0)
    _check(lib().feast_mlp_train_step(ctx, _f32(params), _f32(m), _f32(v), _f32(X), _f32(T), X.shape[0], int(step),
                                      float(lr), ctypes.byref(loss)), "feast_mlp_train_step")
    return loss.value


def feast_interval_solve(ctx, A, lmin, lmax, m0, n_c, tol, opts: FeastOpts | None = None, x0=None):
    """Eigenpairs of the Hermitian CUDA tensor A with eigenvalues in
    (lmin, lmax).  Returns a dict with status, evals (numpy), evecs (CUDA,
    n x m), res (numpy), iterations, stats (FeastStats)."""
    A = colmajor(A)
    n = A.shape[0]
    dt = _dtype_code(A)
    opts = opts or feast_opts_default()
    keep = None
    if x0 is not None:
        keep = colmajor(x0.to(A.dtype))
        opts.x0 = keep.data_ptr()
    evals = np.zeros(m0)
    res = np.zeros(m0)
    V = empty_colmajor(n, m0, A.dtype, A.device)
    mf, it = ctypes.c_int(0), ctypes.c_int(0)
    st = FeastStats()
    code = lib().feast_interval_solve(ctx, _ptr(A), dt, n, n, float(lmin), float(lmax), int(m0), int(n_c),
                                      float(tol), ctypes.byref(opts),
                                      evals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(V),
                                      res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      ctypes.byref(mf), ctypes.byref(it), ctypes.byref(st))
    _check(code, "feast_interval_solve")
    m = mf.value
    return {"status": code, "evals": evals[:m].copy(), "evecs": V[:, :m], "res": res[:m].copy(),
            "iterations": it.value, "stats": st}


def feast_interval_solve_gen(ctx, A, B, lmin, lmax, m0, n_c, tol, opts: FeastOpts | None = None):
    """Eigenpairs of A x = lambda B x (A Hermitian, B Hermitian positive
    definite, CUDA tensors) with lambda in (lmin, lmax); eigenvectors
    B-orthonormal."""
    A = colmajor(A)
    B = colmajor(B.to(A.dtype))
    n = A.shape[0]
    opts = opts or feast_opts_default()
    evals = np.zeros(m0)
    res = np.zeros(m0)
    V = empty_colmajor(n, m0, A.dtype, A.device)
    mf, it = ctypes.c_int(0), ctypes.c_int(0)
    st = FeastStats()
    code = lib().feast_interval_solve_gen(ctx, _ptr(A), _ptr(B), _dtype_code(A), n, n, n, float(lmin), float(lmax),
                                          int(m0), int(n_c), float(tol), ctypes.byref(opts),
                                          evals.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(V),
                                          res.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(mf),
                                          ctypes.byref(it), ctypes.byref(st))
    _check(code, "feast_interval_solve_gen")
    m = mf.value
    return {"status": code, "evals": evals[:m].copy(), "evecs": V[:, :m], "res": res[:m].copy(),
            "iterations": it.value, "stats": st}


def feast_circle_nodes(center, radius, n_c):
    """The 2 n_c nodes and weights of the whole circle |z - center| = radius
    (general matrices): upper half-circle nodes, then their mirror images."""
    z = np.zeros(4 * n_c)
    w = np.zeros(4 * n_c)
    c = complex(center)
    dp = ctypes.POINTER(ctypes.c_double)
    _check(lib().feast_circle_nodes(c.real, c.imag, float(radius), int(n_c), z.ctypes.data_as(dp),
                                    w.ctypes.data_as(dp)), "feast_circle_nodes")
    return z[0::2] + 1j * z[1::2], w[0::2] + 1j * w[1::2]


def feast_eig_general(ctx, H):
    """Eigenvalues (numpy complex, order of the Schur diagonal), unit-norm
    eigenvectors (CUDA complex128 k x k) and QR sweeps of the general k x k
    CUDA matrix H."""
    torch = _torch()
    H = colmajor(H.to(torch.complex128))
    k = H.shape[0]
    ev = np.zeros(2 * k)
    V = empty_colmajor(k, k, torch.complex128, H.device)
    sw = ctypes.c_int(0)
    _check(lib().feast_eig_general(ctx, k, _ptr(H), ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(V),
                                   ctypes.byref(sw)), "feast_eig_general")
    return ev[0::2] + 1j * ev[1::2], V, sw.value


def feast_filter_apply_general(ctx, A, center, radius, n_c, X):
    """sum_k w_k (z_k I - A)^{-1} X over the whole circle for a general CUDA
    matrix A (float64 or complex128) and a CUDA block X (n x m); complex128."""
    torch = _torch()
    A = colmajor(A)
    X = colmajor(X.to(torch.complex128))
    n, m = X.shape
    Y = empty_colmajor(n, m, torch.complex128, A.device)
    c = complex(center)
    _check(lib().feast_filter_apply_general(ctx, _ptr(A), _dtype_code(A), n, n, c.real, c.imag, float(radius),
                                            int(n_c), _ptr(X), m, _ptr(Y)), "feast_filter_apply_general")
    return Y


def feast_disk_solve(ctx, A, center, radius, m0, n_c, tol, max_iter=100, x0=None):
    """Eigenpairs of the general CUDA matrix A (float64 or complex128) with
    eigenvalues inside the disk |lambda - center| < radius."""
    torch = _torch()
    A = colmajor(A)
    n = A.shape[0]
    x0p = None
    if x0 is not None:
        x0 = colmajor(x0.to(torch.complex128))
        x0p = _ptr(x0)
    ev = np.zeros(2 * m0)
    res = np.zeros(m0)
    V = empty_colmajor(n, m0, torch.complex128, A.device)
    mf, it = ctypes.c_int(0), ctypes.c_int(0)
    c = complex(center)
    dp = ctypes.POINTER(ctypes.c_double)
    code = lib().feast_disk_solve(ctx, _ptr(A), _dtype_code(A), n, n, c.real, c.imag, float(radius), int(m0),
                                  int(n_c), float(tol), int(max_iter), x0p, ev.ctypes.data_as(dp), _ptr(V),
                                  res.ctypes.data_as(dp), ctypes.byref(mf), ctypes.byref(it))
    _check(code, "feast_disk_solve")
    m = mf.value
    return {"status": code, "evals": ev[0:2 * m:2] + 1j * ev[1:2 * m:2], "evecs": V[:, :m], "res": res[:m].copy(),
            "iterations": it.value}


def feast_filter_apply(ctx, A, lmin, lmax, n_c, X, opts: FeastOpts | None = None):
    """rho(A) X (Eq. 3) for CUDA tensors A (n x n) and X (n x m)."""
    A = colmajor(A)
    X = colmajor(X.to(A.dtype))
    n, m = X.shape
    Y = empty_colmajor(n, m, A.dtype, A.device)
    opts = opts or feast_opts_default()
    _check(lib().feast_filter_apply(ctx, _ptr(A), _dtype_code(A), n, n, float(lmin), float(lmax), int(n_c),
                                    ctypes.byref(opts), _ptr(X), m, _ptr(Y)), "feast_filter_apply")
    return Y


def feast_shifted_lu(ctx, A, z, prec=FEAST_PREC_F64):
    """LU factors of z_e I - A for the complex shifts z.  Returns (LU, perm):
    LU a CUDA tensor (nz, n, n) holding column-major factors (complex128, or
    complex64 for the mixed precision), perm (nz, n) int32."""
    torch = _torch()
    A = colmajor(A)
    n = A.shape[0]
    z = np.asarray(z, dtype=np.complex128)
    zz = np.ascontiguousarray(np.stack([z.real, z.imag], axis=1).ravel())
    nz = z.size
    cd = torch.complex128 if prec == FEAST_PREC_F64 else torch.complex64
    LU = torch.empty((nz, n, n), dtype=cd, device=A.device)
    perm = torch.empty((nz, n), dtype=torch.int32, device=A.device)
    _check(lib().feast_shifted_lu(ctx, _ptr(A), _dtype_code(A), n, n,
                                  zz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), nz, int(prec),
                                  _ptr(LU), _ptr(perm)), "feast_shifted_lu")
    # LU[e] memory is column-major: expose as matrices
    return LU.transpose(1, 2), perm


def feast_shifted_solve(ctx, LU, perm, B, adjoint=False, prec=FEAST_PREC_F64):
    """Y_e = (z_e I - A)^{-1} B (or the adjoint) for every factor; returns a
    CUDA tensor (nz, n, m) of column-major solutions viewed as matrices."""
    torch = _torch()
    B = colmajor(B.to(torch.complex128))
    n, m = B.shape
    nz = perm.shape[0]
    LUm = LU.transpose(1, 2).contiguous()  # back to the column-major factor memory
    Y = torch.empty((nz, m, n), dtype=torch.complex128, device=B.device)
    _check(lib().feast_shifted_solve(ctx, _ptr(LUm), _ptr(perm), n, nz, int(prec), int(bool(adjoint)),
                                     _ptr(B), m, _ptr(Y)), "feast_shifted_solve")
    return Y.transpose(1, 2)


def feast_orthonormalize(ctx, X, method=0):
    """Orthonormal basis of span(X) (CUDA, n x k); returns (Q, rank)."""
    Xw = colmajor(X).transpose(0, 1).clone().transpose(0, 1)  # private column-major copy
    n, k = Xw.shape
    r = ctypes.c_int(0)
    _check(lib().feast_orthonormalize(ctx, _dtype_code(Xw), n, k, _ptr(Xw), int(method), ctypes.byref(r)),
           "feast_orthonormalize")
    return Xw[:, :r.value], r.value


def feast_jacobi_eigh(ctx, H):
    """Eigenvalues (numpy, ascending), eigenvectors (CUDA, k x k) and sweep
    count of the Hermitian CUDA matrix H by the library's Jacobi kernel."""
    H = colmajor(H)
    k = H.shape[0]
    ev = np.zeros(k)
    V = empty_colmajor(k, k, H.dtype, H.device)
    sw = ctypes.c_int(0)
    _check(lib().feast_jacobi_eigh(ctx, _dtype_code(H), k, _ptr(H),
                                   ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(V), ctypes.byref(sw)),
           "feast_jacobi_eigh")
    return ev, V, sw.value


def feast_rayleigh_ritz(ctx, A, Q, anorm):
    """Rayleigh-Ritz of A on the orthonormal basis Q: (evals, X, res)."""
    A = colmajor(A)
    Q = colmajor(Q.to(A.dtype))
    n, k = Q.shape
    ev = np.zeros(k)
    res = np.zeros(k)
    X = empty_colmajor(n, k, A.dtype, A.device)
    _check(lib().feast_rayleigh_ritz(ctx, _ptr(A), _dtype_code(A), n, n, _ptr(Q), k, float(anorm),
                                     ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(X),
                                     res.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), "feast_rayleigh_ritz")
    return ev, X, res


def feast_gemm_f64acc(ctx, A, B, method=0, transA=False, transB=False, alpha=1.0, beta=0.0, C=None):
    """C = alpha op(A) op(B) + beta C, FP64-accurate, for float64 or complex128
    CUDA matrices; op = conjugate transpose when trans*.  method 0 on the bf16
    tensor cores (digit splitting), 1 in double-float arithmetic (real,
    no transposes, beta = 0)."""
    torch = _torch()
    cplx = A.is_complex() or B.is_complex()
    dt = torch.complex128 if cplx else torch.float64
    A = colmajor(A.to(dt))
    B = colmajor(B.to(dt))
    M, K = (A.shape[1], A.shape[0]) if transA else A.shape
    K2, N = (B.shape[1], B.shape[0]) if transB else B.shape
    if K2 != K:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = empty_colmajor(M, N, dt, A.device)
        if beta != 0.0:
            raise ValueError("beta != 0 needs C")
    else:
        C = colmajor(C.to(dt))
    _check(lib().feast_gemm_f64acc(ctx, int(method), int(cplx), int(bool(transA)), int(bool(transB)), M, N, K,
                                   float(alpha), _ptr(A), A.shape[0], _ptr(B), B.shape[0], float(beta), _ptr(C), M),
           "feast_gemm_f64acc")
    return C


def feast_interval_solve_batch(problems, opts: FeastOpts | None = None, workers=4, autotune=True, device=0):
    """Solve many independent problems concurrently.  problems: list of dicts
    with A (CUDA, Hermitian), lmin, lmax, m0, n_c, tol.  Returns a list of
    dicts (status, evals, evecs, res, iterations, route, ms) in input order."""
    keep = []
    arr = (FeastProblem * len(problems))()
    for i, p in enumerate(problems):
        A = colmajor(p["A"])
        n = A.shape[0]
        ev = np.zeros(p["m0"])
        rs = np.zeros(p["m0"])
        V = empty_colmajor(n, p["m0"], A.dtype, A.device)
        keep.append((A, ev, rs, V))
        arr[i] = FeastProblem(A.data_ptr(), _dtype_code(A), n, n, float(p["lmin"]), float(p["lmax"]),
                              float(p.get("tol", 1e-10)), int(p["m0"]), int(p.get("n_c", 8)), ev.ctypes.data,
                              V.data_ptr(), rs.ctypes.data, 0, 0, 0, 0, 0.0)
    opts = opts or feast_opts_default()
    _check(lib().feast_interval_solve_batch(int(device), len(problems), arr, ctypes.byref(opts), int(workers),
                                            int(bool(autotune))), "feast_interval_solve_batch")
    out = []
    for i in range(len(problems)):
        A, ev, rs, V = keep[i]
        m = arr[i].m_found
        out.append({"status": arr[i].status, "evals": ev[:m].copy(), "evecs": V[:, :m], "res": rs[:m].copy(),
                    "iterations": arr[i].iterations, "route": arr[i].route, "ms": arr[i].ms})
    return out


class Feast:
    """Context manager owning one library context."""

    def __init__(self, device=0, stream=None):
        self.ctx = feast_init(device, stream)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def close(self):
        if self.ctx is not None:
            feast_finalize(self.ctx)
            self.ctx = None

    def solve(self, A, lmin, lmax, m0, n_c=8, tol=1e-10, x0=None, **opts):
        return feast_interval_solve(self.ctx, A, lmin, lmax, m0, n_c, tol, feast_opts_default(**opts), x0=x0)

    def filter(self, A, lmin, lmax, n_c, X, **opts):
        return feast_filter_apply(self.ctx, A, lmin, lmax, n_c, X, feast_opts_default(**opts))
