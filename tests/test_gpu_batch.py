"""Batched solves of independent interval problems (feast_interval_solve_batch,
C ABI): a 4-problem subset of the uneven batched workload, scaled down so the
oracle solves each one, against the FP64 oracle and the planted spectra; the
autotuner's route choice is one of the two mixed routes."""
import numpy as np
import pytest

import oracle as O
import paper_1605_08771_gb300 as fg
from gpu_common import cuda, ctx, host  # noqa: F401
from workloads import make_problem, random_subspace
from workloads.planted import spectrum_config3

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_batch_subset_matches_oracle(ctx, prec):
    probs, planted = [], []
    # four problems of the scaled workload that the oracle solves within the
    # round limit (seed 3's scaled m0 = 6 holds 4 inside plus a cluster of
    # 2 just outside, and converges at about 0.8 per round)
    for seed in (0, 1, 2, 4):
        lam, a, b, m0, n_c = spectrum_config3(seed, scale=0.125)
        P = make_problem("c3", lam, a, b, m0, n_c, seed=seed)
        probs.append({"A": cuda(P.A), "lmin": a, "lmax": b, "m0": m0, "n_c": n_c, "tol": 1e-10})
        planted.append(P)
    # the spectra have eigenvalues on both sides of each interval: plain FEAST
    # with the filter-response stop (R18) on both sides
    opts = fg.feast_opts_default(prec=prec, max_iter=40, response_stop=1)
    out = fg.feast_interval_solve_batch(probs, opts, workers=3, autotune=True)
    for P, p, r in zip(planted, probs, out):
        assert r["status"] == 0
        if prec == "mixed":
            assert r["route"] in (fg.FEAST_PREC_MIXED, fg.FEAST_PREC_MIXED_SIMT)
        assert r["evals"].size == P.inside.size
        err = np.abs(r["evals"] - P.inside)
        assert np.all(err <= 1e-10 * np.abs(P.inside) + 1e-12 * P.anorm)
        assert r["res"].max() <= 1e-10
        X = host(r["evecs"])
        R = P.A @ X - X * r["evals"][None, :]
        assert np.max(np.linalg.norm(R, axis=0)) / P.anorm <= 2e-10
        # the oracle (its own norm estimate, like the library without anorm)
        ref = O.feast_solve(P.A, p["lmin"], p["lmax"], p["m0"], p["n_c"], 1e-10,
                            random_subspace(P.n, p["m0"], seed=1), max_iter=40, response_stop=True)
        assert ref.status == 0
        np.testing.assert_allclose(r["evals"], ref.lam, rtol=1e-10, atol=1e-12 * P.anorm)


def test_batch_argument_errors(ctx):
    with pytest.raises(fg.FeastError):
        fg.feast_interval_solve_batch([{"A": cuda(np.eye(4)), "lmin": -1, "lmax": 1, "m0": 2}],
                                      fg.feast_opts_default(), workers=0)
