"""The allocation-free Jacobi entry point (feast_jacobi_eigh_noalloc) must
give the same eigenpairs as feast_jacobi_eigh, call after call.  It serves
callers that cannot allocate device memory when they call in (services with a
fixed memory budget, frameworks whose caching allocator holds the free
memory) and keeps all scratch in one static device array, so two consecutive
calls also check that leftovers of the previous call do not leak into the
next, and the device's free memory must not change across calls.  Collected
last so a failure here stops a -x run only after every other test."""
import ctypes

import numpy as np
import pytest

import paper_1605_08771_gb300 as fg
from gpu_common import cuda, ctx, host, rand_hermitian  # noqa: F401

pytestmark = pytest.mark.gpu


def noalloc_eigh(H, stream=None, V=None):
    import torch
    k = H.shape[0]
    ev = np.zeros(k)
    if V is None:
        V = fg.empty_colmajor(k, k, H.dtype, H.device)
    sw = ctypes.c_int(0)
    if stream is None:
        stream = torch.cuda.current_stream(H.device)
    code = fg.lib().feast_jacobi_eigh_noalloc(
        H.device.index, ctypes.c_void_p(stream.cuda_stream), fg._dtype_code(H), k, ctypes.c_void_p(H.data_ptr()),
        ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.c_void_p(V.data_ptr()), ctypes.byref(sw))
    return code, ev, V, sw.value


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("cplx", [False, True])
def test_noalloc_matches_context_entry_point_twice(ctx, cplx):
    import torch
    ref = {}
    for k in (256, 64):   # the context entry point first: its allocations are done before the check
        Hn = rand_hermitian(k, cplx, seed=500 + k + int(cplx))
        H = fg.colmajor(cuda(Hn))
        ref[k] = (Hn, H, fg.feast_jacobi_eigh(ctx, H))
    code, _, _, _ = noalloc_eigh(ref[64][1])   # first call on the device: its one-time set-up
    assert code == 0, fg.feast_strerror(code)
    outs = {}
    for k in (256, 64):
        outs[k] = fg.empty_colmajor(k, k, ref[k][1].dtype, ref[k][1].device)
    reserved0, free0 = torch.cuda.memory_reserved(), free_bytes()
    for k in (256, 64):   # two calls in a row, the largest size the scratch allows first
        Hn, H, (ev_ref, V_ref, _) = ref[k]
        code, ev, V, sweeps = noalloc_eigh(H, V=outs[k])
        assert code == 0, fg.feast_strerror(code)
        scale = max(1.0, np.linalg.norm(Hn))
        np.testing.assert_allclose(ev, ev_ref, atol=1e-13 * scale)
        np.testing.assert_allclose(ev, np.linalg.eigvalsh(Hn), atol=1e-13 * scale)
        V, V_ref = host(V), host(V_ref)
        assert np.linalg.norm(Hn @ V - V * ev) <= 1e-13 * scale * k
        assert np.linalg.norm(V.conj().T @ V - np.eye(k)) <= 1e-13 * k
        # eigenvectors of these (distinct) eigenvalues agree up to a phase
        np.testing.assert_allclose(np.abs(np.sum(V.conj() * V_ref, axis=0)), 1.0, atol=1e-9)
        assert 0 < sweeps < 30
    # the calls allocated nothing on the device (the outputs were allocated
    # before, and the library's scratch is the static array)
    assert free_bytes() == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    H = fg.colmajor(cuda(rand_hermitian(257, False, seed=1)))
    code, _, _, _ = noalloc_eigh(H)
    assert code == -1


def test_noalloc_refuses_a_capturing_stream(ctx):
    # the call synchronises and reads back, which a capturing stream forbids:
    # it must return the argument error without enqueuing anything, and the
    # capture must still complete and replay
    import torch
    H = fg.colmajor(cuda(rand_hermitian(16, False, seed=2)))
    x = torch.zeros(8, device=H.device)
    s = torch.cuda.Stream(device=H.device)
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        g.capture_begin()
        code, _, _, _ = noalloc_eigh(H, stream=s)
        x.add_(1.0)
        g.capture_end()
    assert code == -1
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 8.0
