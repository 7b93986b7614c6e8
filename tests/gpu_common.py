"""Shared helpers of the GPU parity tests (CUDA path through the C ABI)."""
import numpy as np
import pytest


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a) if np.asarray(a).ndim < 2 else np.asfortranarray(a)).to("cuda:0")


def host(t):
    return t.detach().cpu().numpy()


@pytest.fixture(scope="module")
def ctx():
    import paper_1605_08771_gb300 as fg
    fg.build_library()
    c = fg.feast_init(0)
    yield c
    fg.feast_finalize(c)


def rand_hermitian(n, cplx, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    H = rng.standard_normal((n, n))
    if cplx:
        H = H + 1j * rng.standard_normal((n, n))
    return np.asfortranarray(scale * 0.5 * (H + H.conj().T))


def rand_mat(n, m, cplx, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, m))
    if cplx:
        X = X + 1j * rng.standard_normal((n, m))
    return np.asfortranarray(X)
