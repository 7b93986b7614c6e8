"""Parity of the learned-proposer kernels (CUDA path, C ABI) with the oracle:
stochastic-trace Chebyshev moments (same probes on both sides), the MLP's
forward pass, gradients and Adam step (FP32 kernels against the FP64 numpy
oracle); and the shipped weights against the plain m0 rule on held-out
spectra."""
import numpy as np
import pytest

import paper_1605_08771_gb300 as fg
from gpu_common import cuda, ctx, host  # noqa: F401
from oracle.density import chebyshev_moments, exact_moments
from oracle.mlp import LAYERS, adam_step, backward, forward, init_params, loss
from workloads import make_problem, random_subspace, spectrum_uniform

pytestmark = pytest.mark.gpu


def pack(ps):
    return np.concatenate([p.ravel() for p in ps]).astype(np.float32)


def unpack(flat):
    out, o = [], 0
    for din, dout in LAYERS:
        out.append(flat[o:o + din * dout].reshape(dout, din))
        o += din * dout
        out.append(flat[o:o + dout])
        o += dout
    return out


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("n,nv", [(100, 4), (333, 9)])
def test_moments_match_oracle(ctx, cplx, n, nv):
    lam, a, b = spectrum_uniform(n, 10, seed=n, bulk=6.0)
    P = make_problem("m", lam, a, b, 16, 8, seed=n, complex_=cplx)
    V = random_subspace(n, nv, seed=7, complex_=cplx)
    r = 1.02 * np.max(np.abs(lam - 0.25))
    mu = fg.feast_spectral_moments(ctx, cuda(P.A), cuda(V), 0.25, r, 64)
    ref = chebyshev_moments(P.A, V, 0.25, r, 64)
    np.testing.assert_allclose(mu, ref, atol=1e-12)
    # and a complete probe basis gives the exact (1/n) tr T_k
    mu_i = fg.feast_spectral_moments(ctx, cuda(P.A), cuda(np.sqrt(n) * np.eye(n)), 0.25, r, 32)
    np.testing.assert_allclose(mu_i, exact_moments(lam, 0.25, r, 32), atol=1e-12)


def test_mlp_forward_and_gradient_match_oracle(ctx):
    import torch
    rng = np.random.default_rng(11)
    ps = init_params(seed=3)
    for i in range(1, len(ps), 2):
        ps[i] = 0.05 * rng.standard_normal(ps[i].shape)
    B = 37
    X = rng.standard_normal((B, 64))
    T = rng.standard_normal((B, 9))
    flat = pack(ps)
    p32 = [x.astype(np.float32).astype(np.float64) for x in unpack(flat)]
    dev = "cuda:0"
    P = torch.from_numpy(flat).to(dev)
    Xd = torch.from_numpy(X.astype(np.float32)).to(dev)
    Td = torch.from_numpy(T.astype(np.float32)).to(dev)
    Y = host(fg.feast_mlp_forward(ctx, P, Xd))
    Yo, _ = forward(p32, X.astype(np.float32).astype(np.float64))
    assert np.abs(Y - Yo).max() <= 1e-4 * max(1.0, np.abs(Yo).max())
    g, l = fg.feast_mlp_gradient(ctx, P, Xd, Td)
    go = backward(p32, X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64))
    lo = loss(p32, X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64))
    assert abs(l - lo) <= 1e-5 * max(1.0, lo)
    gh = unpack(host(g).astype(np.float64))
    for a_, b_ in zip(gh, go):
        assert np.abs(a_ - b_).max() <= 1e-4 * max(1e-3, np.abs(b_).max())


def test_adam_step_matches_oracle(ctx):
    # three Adam steps of the kernel against the oracle's update applied to
    # the kernel's own gradient and parameters (the gradients themselves are
    # compared above; here only the update arithmetic is)
    import torch
    rng = np.random.default_rng(2)
    ps = init_params(seed=8)
    B = 16
    X = rng.standard_normal((B, 64)).astype(np.float32)
    T = rng.standard_normal((B, 9)).astype(np.float32)
    dev = "cuda:0"
    P = torch.from_numpy(pack(ps)).to(dev)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    Xd = torch.from_numpy(X).to(dev)
    Td = torch.from_numpy(T).to(dev)
    mo = [np.zeros(P.numel())]
    vo = [np.zeros(P.numel())]
    lr = 1e-3
    for step in (1, 2, 3):
        g, _ = fg.feast_mlp_gradient(ctx, P, Xd, Td)
        ref = [host(P).astype(np.float64)]
        adam_step(ref, [host(g).astype(np.float64)], mo, vo, step, lr=lr)
        fg.feast_mlp_train_step(ctx, P, m, v, Xd, Td, step, lr)
        assert np.abs(host(P) - ref[0]).max() <= 1e-3 * lr





def test_learned_proposer_cuts_mean_iterations_on_held_out_spectra(ctx):
    # the trained proposer (weights shipped with the package) against the
    # plain rule m0 = ceil(1.5 m_hat) with Gauss nodes, on held-out
    # edge-clustered spectra (seeds the training never saw), both with the
    # filter-response stop; the plain rule is the fallback when a proposal
    # does not converge.  The learned rule must need fewer rounds on average
    # and find every planted pair at least as often
    import os
    from paper_1605_08771_gb300 import proposer as PR
    assert os.path.exists(PR.WEIGHTS)
    params = PR.load_params()
    rows = PR.evaluate(ctx, params, range(PR.HELD_OUT_BASE, PR.HELD_OUT_BASE + 16), 2048)
    s = PR.summary(rows)
    assert s["learned"]["mean_iterations"] < s["plain"]["mean_iterations"], s
    assert s["learned"]["converged"] >= s["plain"]["converged"], s
