"""The allocation-free Jacobi entry point (feast_jacobi_eigh_noalloc) must
give the same eigenpairs as feast_jacobi_eigh, call after call: it serves
callers that cannot allocate device memory when they call in (stream
capture, fixed memory budgets, caching allocators holding the free memory)
and keeps all scratch in one static device array, so two consecutive calls
also check that leftovers of the previous call do not leak into the next.
Collected last so a failure here stops a -x run only after every other test."""
import ctypes

import numpy as np
import pytest

import paper_1605_08771_gb300 as fg
from gpu_common import cuda, ctx, host, rand_hermitian  # noqa: F401

pytestmark = pytest.mark.gpu


def noalloc_eigh(H):
    import torch
    k = H.shape[0]
    ev = np.zeros(k)
    V = fg.empty_colmajor(k, k, H.dtype, H.device)
    sw = ctypes.c_int(0)
    stream = torch.cuda.current_stream(H.device).cuda_stream
    code = fg.lib().feast_jacobi_eigh_noalloc(
        0, ctypes.c_void_p(stream), fg._dtype_code(H), k, ctypes.c_void_p(H.data_ptr()),
        ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(V.data_ptr()), ctypes.byref(sw))
    return code, ev, V, sw.value


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_matches_context_entry_point_twice(ctx, cplx):
    for call, k in enumerate([200, 64]):           # two calls in a row, large then small
        Hn = rand_hermitian(k, cplx, seed=500 + 10 * call + int(cplx))
        H = fg.colmajor(cuda(Hn))
        code, ev, V, sweeps = noalloc_eigh(H)
        assert code == 0, fg.feast_strerror(code)
        ev_ref, V_ref, _ = fg.feast_jacobi_eigh(ctx, H)
        scale = max(1.0, np.linalg.norm(Hn))
        np.testing.assert_allclose(ev, ev_ref, atol=1e-13 * scale)
        np.testing.assert_allclose(ev, np.linalg.eigvalsh(Hn), atol=1e-13 * scale)
        V, V_ref = host(V), host(V_ref)
        assert np.linalg.norm(Hn @ V - V * ev) <= 1e-13 * scale * k
        assert np.linalg.norm(V.conj().T @ V - np.eye(k)) <= 1e-13 * k
        # eigenvectors of these (distinct) eigenvalues agree up to a phase
        np.testing.assert_allclose(np.abs(np.sum(V.conj() * V_ref, axis=0)), 1.0, atol=1e-9)
        assert 0 < sweeps < 30


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    H = fg.colmajor(cuda(rand_hermitian(257, False, seed=1)))
    code, _, _, _ = noalloc_eigh(H)
    assert code == -1
