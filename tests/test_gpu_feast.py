"""End-to-end parity of feast_interval_solve (CUDA path, C ABI) with the FP64
oracle and with the planted spectra: eigenvalue count exact, eigenvalues to
1e-10 relative, residuals <= 1e-10 relative to ||A||_2, eigenvector spans;
all three variants, both precisions; edge cases."""
import json
import os

import numpy as np
import pytest

import closed_forms as CF
import oracle as O
import paper_1605_08771_gb300 as fg
from gpu_common import cuda, ctx, host  # noqa: F401
from workloads import (make_problem, random_subspace, spectrum_config1, spectrum_config2, spectrum_paper,
                       spectrum_uniform)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_setups.json")

pytestmark = pytest.mark.gpu
VARIANTS = [("feast", O.PLAIN), ("xfeast", O.XFEAST), ("rfeast", O.RFEAST)]


def check_against_planted(out, P, tol=1e-10):
    assert out["evals"].size == P.inside.size
    np.testing.assert_allclose(out["evals"], P.inside, rtol=1e-10, atol=1e-12 * P.anorm)
    assert np.max(out["res"]) <= tol
    X = host(out["evecs"])
    # recompute residuals independently in FP64 on the host
    R = P.A @ X - X * out["evals"][None, :]
    assert np.max(np.linalg.norm(R, axis=0)) / P.anorm <= 2 * tol
    # span: sin(angle) <= ||residual|| / gap (Davis-Kahan), gap = distance from
    # the wanted eigenvalues to the rest of the spectrum
    Qi = P.inside_vectors
    ins = (P.lam > P.lmin) & (P.lam < P.lmax)
    gap = np.min(np.abs(P.lam[ins][:, None] - P.lam[~ins][None, :])) if np.any(~ins) else P.anorm
    bound = max(1e-8, 4.0 * np.sqrt(P.inside.size) * tol * P.anorm / gap)
    assert np.linalg.norm(X - Qi @ (Qi.conj().T @ X), 2) <= bound


@pytest.mark.parametrize("vname,vor", VARIANTS)
@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", ["f64", "mixed", "mixed_simt"])
def test_small_planted_vs_oracle(ctx, vname, vor, cplx, prec):
    lam, a, b = spectrum_uniform(90, 8, seed=3, bulk=10.0)
    P = make_problem("s", lam, a, b, 12, 8, seed=3, complex_=cplx)
    X0 = random_subspace(P.n, P.m0, seed=5, complex_=cplx)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, P.m0, 8, 1e-10,
                                  fg.feast_opts_default(variant=vname, prec=prec, anorm=P.anorm),
                                  x0=cuda(X0))
    assert out["status"] == 0
    check_against_planted(out, P)
    ref = O.feast_solve(P.A, a, b, P.m0, 8, 1e-10, X0, variant=vor, anorm=P.anorm, max_iter=100)
    assert ref.status == 0
    np.testing.assert_allclose(out["evals"], ref.lam, atol=1e-12 * P.anorm)
    assert abs(out["iterations"] - ref.iterations) <= 1


# readings of the expanded variants: the paper's text (every selected
# residual appended, step-3 check alone) and the two named options
READINGS = {"paper": ({}, {}),
            "options": ({"rfeast_expand": 1, "response_stop": 1},
                        {"expand": O.EXPAND_UNCONVERGED, "response_stop": True})}


@pytest.mark.parametrize("vname,vor", VARIANTS)
def test_n500_workload_vs_oracle(ctx, vname, vor):
    # n = 500 real symmetric, 40 eigenvalues in [-1, 1] (5 within 1e-3 of each
    # edge), 460 on both sides of I; n_c = 8, m0 = 60, tol 1e-10, FP64.  On a
    # two-sided spectrum the expanded variants meet spurious in-I pairs
    # (mixtures of eigenvectors from both sides) that the paper's step-3
    # checks alone may never clear, so XFEAST and RFEAST run with the two
    # named options here; the paper's text is checked on its own one-sided
    # spectra below
    gk, ok = READINGS["options"] if vor != O.PLAIN else ({}, {})
    if vor == O.XFEAST:
        gk = {k: v for k, v in gk.items() if k != "rfeast_expand"}
        ok = {k: v for k, v in ok.items() if k != "expand"}
    lam, a, b = spectrum_config1(0)
    P = make_problem("c1", lam, a, b, 60, 8, seed=0)
    X0 = random_subspace(P.n, 60, seed=1)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, 60, 8, 1e-10,
                                  fg.feast_opts_default(variant=vname, anorm=P.anorm, **gk), x0=cuda(X0))
    assert out["status"] == 0
    check_against_planted(out, P)
    ref = O.feast_solve(P.A, a, b, 60, 8, 1e-10, X0, variant=vor, anorm=P.anorm, **ok)
    np.testing.assert_allclose(out["evals"], ref.lam, atol=1e-12 * P.anorm)
    if vor == O.PLAIN:
        # the expanded variants' round counts on a two-sided spectrum vary
        # with rounding (x86 vs Arm oracle runs differ): only plain FEAST's
        # is pinned
        assert abs(out["iterations"] - ref.iterations) <= 1


@pytest.mark.parametrize("kind", ["sparse", "dense"])
@pytest.mark.parametrize("vname,vor", VARIANTS[1:])
def test_paper_spectra_literal_variants_vs_oracle(ctx, kind, vname, vor):
    # the paper's n = 545 "Sparse" and "Dense" spectra (Sect. III; 50
    # eigenvalues in [-1, 1], the other 495 above I), n_c = 8, m0 = 51, with
    # XFEAST and RFEAST exactly as the Appendix states them (every selected
    # residual appended, step-3 checks alone): GPU and oracle converge to the
    # planted pairs in the same number of rounds (+-1; +-2 on Dense), and on
    # Dense the expanded variant needs fewer right-hand sides than FEAST
    g = json.load(open(GOLDEN))["fig1_fig2_matrices"]
    lam, a, b = spectrum_paper(kind, seed=0, n=g["n"], m_in=g["inside"])
    m0 = g["m0_expanded_variants"]
    P = make_problem(kind, lam, a, b, m0, 8, seed=0)
    X0 = random_subspace(P.n, m0, seed=1)
    F = O.factor_shifts(P.A, a, b, 8)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, 1e-10,
                                  fg.feast_opts_default(variant=vname, anorm=P.anorm), x0=cuda(X0))
    ref = O.feast_solve(P.A, a, b, m0, 8, 1e-10, X0, variant=vor, anorm=P.anorm, factors=F)
    assert out["status"] == 0 == ref.status
    check_against_planted(out, P)
    np.testing.assert_allclose(out["evals"], ref.lam, atol=1e-12 * P.anorm)
    assert abs(out["iterations"] - ref.iterations) <= (2 if kind == "dense" else 1)
    if kind == "dense":
        plain = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, 1e-10,
                                        fg.feast_opts_default(anorm=P.anorm), x0=cuda(X0))
        assert out["stats"].filters < plain["stats"].filters


@pytest.mark.parametrize("prec", ["f64", "mixed"])
@pytest.mark.parametrize("reading", ["paper", "options"])
def test_edge_clustered_complex_rfeast(ctx, prec, reading):
    # scaled-down edge-cluster workload: clusters within 1e-4 inside and
    # outside both edges, bulk in [-50, 50]; plain FEAST stalls here
    lam, a, b = spectrum_config2(0, n=640, m_in=16, edge_in=3, edge_out=5, width=1e-4, bulk=50.0)
    P = make_problem("c2s", lam, a, b, 24, 8, seed=0, complex_=True)
    X0 = random_subspace(P.n, 24, seed=1, complex_=True)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, 24, 8, 1e-10,
                                  fg.feast_opts_default(variant="rfeast", prec=prec, anorm=P.anorm,
                                                        **READINGS[reading][0]),
                                  x0=cuda(X0))
    assert out["status"] == 0
    check_against_planted(out, P)
    # the Rayleigh-Ritz passes: at least one and at most s = 3 per round,
    # none larger than s m0 = 72
    st = out["stats"]
    assert out["iterations"] <= st.rr_passes <= 3 * out["iterations"]
    assert st.rr_passes <= st.rr_k_sum <= 72 * st.rr_passes
    assert st.rr_k_sum ** 3 / st.rr_passes ** 2 <= st.rr_k3_sum * (1 + 1e-12)
    assert st.rr_k3_sum <= st.rr_passes * 72.0 ** 3


def test_internal_random_start_and_norm_estimate(ctx):
    lam, a, b = spectrum_uniform(200, 12, seed=8, bulk=15.0)
    P = make_problem("r", lam, a, b, 18, 8, seed=8)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, 18, 8, 1e-10, fg.feast_opts_default(seed=42))
    assert out["status"] == 0
    assert out["evals"].size == 12
    np.testing.assert_allclose(out["evals"], P.inside, rtol=1e-10, atol=1e-12 * P.anorm)


def test_empty_interval(ctx):
    lam = np.concatenate([np.linspace(-10, -2, 30), np.linspace(2, 10, 30)])
    P = make_problem("gap", lam, -1.0, 1.0, 8, 8, seed=4)
    out = fg.feast_interval_solve(ctx, cuda(P.A), -1.0, 1.0, 8, 8, 1e-10, fg.feast_opts_default(anorm=10.0),
                                  x0=cuda(random_subspace(60, 8, seed=1)))
    assert out["status"] == 0 and out["evals"].size == 0


def test_tiny_n(ctx):
    A = np.asfortranarray(np.array([[0.25]]))
    out = fg.feast_interval_solve(ctx, cuda(A), -1.0, 1.0, 1, 4, 1e-12, fg.feast_opts_default(anorm=0.25),
                                  x0=cuda(np.ones((1, 1))))
    assert out["evals"].size == 1 and abs(out["evals"][0] - 0.25) < 1e-15
    A2 = np.asfortranarray(np.diag([0.5, 3.0]))
    out = fg.feast_interval_solve(ctx, cuda(A2), -1.0, 1.0, 2, 8, 1e-12, fg.feast_opts_default(anorm=3.0),
                                  x0=cuda(np.asfortranarray([[1.0, 0.3], [0.2, 1.0]])))
    assert out["evals"].size == 1 and abs(out["evals"][0] - 0.5) < 1e-14


def test_errors(ctx):
    A = np.asfortranarray(np.eye(10))
    with pytest.raises(fg.FeastError) as e:
        fg.feast_interval_solve(ctx, cuda(A), -1.0, 1.0, 11, 8, 1e-10)   # m0 > n
    assert e.value.code == -1
    with pytest.raises(fg.FeastError) as e:
        fg.feast_interval_solve(ctx, cuda(A), 1.0, -1.0, 4, 8, 1e-10)    # empty interval
    assert e.value.code == -1
    B = A.copy()
    B[3, 4] = np.nan
    with pytest.raises(fg.FeastError) as e:
        fg.feast_interval_solve(ctx, cuda(B), -1.0, 1.0, 4, 8, 1e-10)
    assert e.value.code == -2


@pytest.mark.parametrize("vname,vor", VARIANTS)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_invariant_start_converges_in_one_round(ctx, vname, vor, prec):
    # X0 spanning an invariant subspace that holds every eigenvector inside I:
    # one round for every variant, as in the oracle, with RFEAST's expected
    # count exact
    lam, a, b = spectrum_uniform(100, 8, seed=3, bulk=10.0)
    P = make_problem("inv", lam, a, b, 12, 8, seed=3, complex_=True)
    ins = np.where((P.lam > a) & (P.lam < b))[0]
    outs = [i for i in np.argsort(np.abs(P.lam - 0.5 * (a + b))) if i not in set(ins)][:P.m0 - ins.size]
    R, _ = np.linalg.qr(random_subspace(P.m0, P.m0, seed=3, complex_=True))
    X0 = np.asfortranarray(P.Q[:, np.concatenate([ins, outs])] @ R)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, P.m0, 8, 1e-10,
                                  fg.feast_opts_default(variant=vname, prec=prec, anorm=P.anorm), x0=cuda(X0))
    ref = O.feast_solve(P.A, a, b, P.m0, 8, 1e-10, X0, variant=vor, anorm=P.anorm)
    assert out["status"] == 0 and out["iterations"] == 1 == ref.iterations
    check_against_planted(out, P)
    if vname == "rfeast":
        assert out["stats"].m_expected == ins.size == ref.m_expected


@pytest.mark.parametrize("cplx", [False, True])
def test_rfeast_literal_expansion_matches_oracle(ctx, cplx):
    # RFEAST step 2(iii) as the paper states it (every selected pair's
    # residual appended): the Rayleigh-Ritz passes of each round have
    # dimensions m0, 2 m0, 3 m0, like the oracle's, and the result matches it
    lam, a, b = spectrum_uniform(150, 8, seed=3, bulk=10.0)
    P = make_problem("lit", lam, a, b, 12, 8, seed=3, complex_=cplx)
    X0 = random_subspace(P.n, P.m0, seed=5, complex_=cplx)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, P.m0, 8, 1e-10,
                                  fg.feast_opts_default(variant="rfeast", anorm=P.anorm), x0=cuda(X0))
    ref = O.feast_solve(P.A, a, b, P.m0, 8, 1e-10, X0, variant=O.RFEAST, anorm=P.anorm)
    assert out["status"] == 0 == ref.status
    check_against_planted(out, P)
    np.testing.assert_allclose(out["evals"], ref.lam, atol=1e-12 * P.anorm)
    assert abs(out["iterations"] - ref.iterations) <= 1
    st = out["stats"]
    assert st.rr_passes == 3 * out["iterations"]
    assert st.rr_k_sum == 6 * P.m0 * out["iterations"]
    assert ref.rr_dims[:3] == [12, 24, 36]


FULL_SPAN = [(v, s, r) for v in ("xfeast", "rfeast") for s in (2, 3) for r in ("paper", "options")]


@pytest.mark.parametrize("vname,s,reading", FULL_SPAN)
@pytest.mark.parametrize("prec", ["f64", "mixed"])
@pytest.mark.parametrize("cplx", [False, True])
def test_full_span_expansion_converges_in_one_round(ctx, vname, s, reading, prec, cplx):
    # s m0 = n: the expanded subspace of round 1 spans the whole space
    # (block Krylov of rho(A) for XFEAST, of A for RFEAST), so Rayleigh-Ritz
    # is exact and round 1 returns exactly the planted pairs, as in the oracle
    n = 60
    lam, a, b = spectrum_uniform(n, n // 8, seed=1, bulk=2.0)
    m0 = n // s
    P = make_problem("full", lam, a, b, m0, 8, seed=1, complex_=cplx)
    X0 = random_subspace(n, m0, seed=12, complex_=cplx)
    gk = dict(READINGS[reading][0])
    if vname == "xfeast":
        gk.pop("rfeast_expand", None)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, 1e-10,
                                  fg.feast_opts_default(variant=vname, s=s, prec=prec, anorm=P.anorm, max_iter=3,
                                                        **gk), x0=cuda(X0))
    assert out["status"] == 0 and out["iterations"] == 1
    assert out["evals"].size == P.inside.size
    np.testing.assert_allclose(out["evals"], P.inside, atol=1e-12 * P.anorm)
    check_against_planted(out, P)


@pytest.mark.parametrize("cplx", [False, True])
def test_plain_feast_rounds_follow_subspace_iteration(ctx, cplx):
    # plain FEAST on the n = 500 workload (FP64), round by round against
    # subspace iteration on rho(A) in the planted eigenbasis (Sect. I): the
    # round count, the residual history (stats) and, stopped after k rounds
    # (max_iter = k), that round's in-I Ritz values
    lam, a, b = spectrum_config1(0)
    m0, tol = 60, 1e-10
    P = make_problem("c1", lam, a, b, m0, 8, seed=0, complex_=cplx)
    X0 = random_subspace(P.n, m0, seed=1, complex_=cplx)
    z, w = O.contour_nodes(a, b, 8)
    rho = O.rational_filter(P.lam, z, w)
    full = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, tol, fg.feast_opts_default(prec="f64", anorm=P.anorm),
                                   x0=cuda(X0))
    assert full["status"] == 0
    K = full["iterations"]
    closed = CF.plain_feast_rounds(P.lam, P.Q.conj().T @ X0, rho, P.anorm, a, b, K)
    assert [k for k, (_, r) in enumerate(closed, 1) if r <= tol][:1] == [K]
    hist = list(full["stats"].history)[:K]
    for h, (_, r) in zip(hist[:-1], closed[:-1]):
        assert abs(h - r) <= 1e-5 * r
    for k in (1, 2, 3):
        out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, tol,
                                      fg.feast_opts_default(prec="f64", anorm=P.anorm, max_iter=k), x0=cuda(X0))
        assert out["status"] == fg.FEAST_WARN_MAXITER and out["iterations"] == k
        assert out["evals"].size == closed[k - 1][0].size
        np.testing.assert_allclose(out["evals"], closed[k - 1][0], rtol=0, atol=1e-10 * P.anorm)


@pytest.mark.parametrize("vname,s", [("xfeast", 2), ("xfeast", 3), ("rfeast", 2)])
@pytest.mark.parametrize("cplx", [False, True])
def test_first_expanded_round_closed_form(ctx, vname, s, cplx):
    # the first XFEAST round (Rayleigh-Ritz on [X0, rho X0, ..., rho^{s-1}
    # X0], then the m0-pair selection) and the first RFEAST round with s = 2
    # (span[Y, A Y], Y = rho(A) X0, the paper's expansion), s m0 < n, FP64,
    # against their closed forms in the planted eigenbasis
    n, m0 = 120, 14
    lam, a, b = spectrum_uniform(n, 10, seed=1, bulk=3.0)
    P = make_problem("x1", lam, a, b, m0, 8, seed=1, complex_=cplx)
    X0 = random_subspace(n, m0, seed=6, complex_=cplx)
    z, w = O.contour_nodes(a, b, 8)
    rho = O.rational_filter(P.lam, z, w)
    C0 = P.Q.conj().T @ X0
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, 1e-10,
                                  fg.feast_opts_default(variant=vname, s=s, prec="f64", anorm=P.anorm, max_iter=1),
                                  x0=cuda(X0))
    assert out["status"] == fg.FEAST_WARN_MAXITER
    if vname == "xfeast":
        mu, rmax = CF.xfeast_first_round(P.lam, C0, rho, P.anorm, a, b, m0, s)
        atol = 1e-8 * P.anorm       # the s = 3 window's condition number is ~1e7
    else:
        m_exp, mu, rmax, _ = CF.rfeast_first_round_s2(P.lam, C0, rho, P.anorm, a, b, m0)
        assert out["stats"].m_expected == m_exp
        atol = 1e-10 * P.anorm
    assert out["evals"].size == mu.size
    np.testing.assert_allclose(out["evals"], mu, rtol=0, atol=atol)
    assert abs(out["stats"].history[0] - rmax) <= 1e-5 * rmax


@pytest.mark.parametrize("s", [2, 3])
@pytest.mark.parametrize("cplx", [False, True])
def test_second_xfeast_round_closed_form(ctx, s, cplx):
    # round 2 of XFEAST works on rho(A) times the first window,
    # span[rho X0, ..., rho^s X0] (the selected vectors it filters lie in
    # the first window), FP64, against the closed form in the planted
    # eigenbasis; the power basis's condition (~1e7 for s = 2, ~1e12 for
    # s = 3) sets the bounds
    n, m0 = 120, 14
    lam, a, b = spectrum_uniform(n, 10, seed=1, bulk=3.0)
    P = make_problem("x2", lam, a, b, m0, 8, seed=1, complex_=cplx)
    X0 = random_subspace(n, m0, seed=6, complex_=cplx)
    z, w = O.contour_nodes(a, b, 8)
    rho = O.rational_filter(P.lam, z, w)
    mu, rmax = CF.xfeast_round(P.lam, P.Q.conj().T @ X0, rho, P.anorm, a, b, m0, s, 2)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, 1e-10,
                                  fg.feast_opts_default(variant="xfeast", s=s, prec="f64", anorm=P.anorm, max_iter=2),
                                  x0=cuda(X0))
    assert out["status"] == fg.FEAST_WARN_MAXITER and out["iterations"] == 2
    assert out["evals"].size == mu.size
    np.testing.assert_allclose(out["evals"], mu, rtol=0, atol=(1e-9 if s == 2 else 1e-5) * P.anorm)
    assert abs(out["stats"].history[1] - rmax) <= 1e-4 * rmax


@pytest.mark.parametrize("n", [2048, 4096])
def test_full_size_paths_mixed_rfeast_edge_clusters(ctx, n):
    # the mixed path at sizes where the GEMM tile dispatch, the split-K
    # Rayleigh-Ritz reductions, the two-phase eigensolver and the refinement
    # stop all take their large-n branches: the edge-cluster workload scaled
    # to n (clusters within 1e-4 inside and outside both edges, bulk in
    # [-50, 50]), RFEAST s = 3 with the two named readings, as benchmarked
    sc = n / 8192
    m_in, e_in, e_out, m0 = int(200 * sc), int(30 * sc), int(60 * sc), int(300 * sc)
    lam, a, b = spectrum_config2(0, n=n, m_in=m_in, edge_in=e_in, edge_out=e_out)
    P = make_problem("c2n", lam, a, b, m0, 8, seed=0, complex_=True, keep_q=True)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, 1e-10,
                                  fg.feast_opts_default(variant="rfeast", prec="mixed", anorm=P.anorm,
                                                        max_iter=20, rfeast_expand=1, response_stop=1))
    assert out["status"] == 0
    # count exact, |dl| <= 1e-10 |l| + 1e-12 ||A||, residuals (reported and
    # recomputed on the host), span within the Davis-Kahan bound
    check_against_planted(out, P)
    assert out["stats"].refine_steps > 0


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_filter_closed_form_n2048(ctx, prec):
    # rho(A) X = Q diag(rho(lambda)) Q^H X on a planted n = 2048 complex
    # Hermitian A (Eq. 3; rho from the oracle's scalar filter), a few columns
    lam, a, b = spectrum_config2(0, n=2048, m_in=50, edge_in=8, edge_out=15)
    P = make_problem("f2048", lam, a, b, 8, 8, seed=0, complex_=True)
    X = random_subspace(P.n, 6, seed=3, complex_=True)
    Y = host(fg.feast_filter_apply(ctx, cuda(P.A), a, b, 8, cuda(X),
                                   fg.feast_opts_default(prec=prec, anorm=P.anorm)))
    z, w = O.contour_nodes(a, b, 8)
    rho = O.rational_filter(P.lam, z, w)
    ref = P.Q @ (rho[:, None] * (P.Q.conj().T @ X))
    # forward error of the shifted solves: kappa(z_j I - A) ~ 50 / 0.06 times
    # their backward error (FP64 LU, or refinement to 16 eps sqrt(n))
    err = np.abs(Y - ref).max() / np.abs(X).max()
    assert err <= 2e-10, err


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_generalized_problem_vs_oracle(ctx, cplx, prec):
    # A x = lambda B x (planted pencil): the library's Cholesky-reduced solve
    # against the oracle's generalized FEAST with B-inner products (a
    # different algorithm for the same eigenpairs) and the planted values
    from workloads.planted import planted_pencil
    lam, a, b = spectrum_uniform(300, 14, seed=9, bulk=8.0)
    A, B, X = planted_pencil(lam, 9, complex_=cplx)
    out = fg.feast_interval_solve_gen(ctx, cuda(A), cuda(B), a, b, 21, 8, 1e-10,
                                      fg.feast_opts_default(prec=prec))
    assert out["status"] == 0
    ins = (lam > a) & (lam < b)
    assert out["evals"].size == ins.sum()
    np.testing.assert_allclose(out["evals"], lam[ins], rtol=1e-10, atol=1e-12 * np.abs(lam).max())
    V = host(out["evecs"])
    assert np.abs(V.conj().T @ B @ V - np.eye(V.shape[1])).max() < 1e-9
    an = np.abs(lam).max()
    bn = np.abs(np.linalg.eigvalsh(B)).max()
    R = A @ V - (B @ V) * out["evals"][None, :]
    # the library stops on the reduced problem's residual (<= 1e-10); the
    # pencil's backward error is within cond(B) of it
    assert np.max(np.linalg.norm(R, axis=0) / ((an + np.abs(out["evals"]) * bn) * np.linalg.norm(V, axis=0))) < 1e-9
    assert out["res"].max() <= 1e-10
    ref = O.feast.feast_solve_generalized(A, B, a, b, 21, 8, 1e-10, random_subspace(300, 21, seed=2, complex_=cplx))
    assert ref.status == 0
    np.testing.assert_allclose(out["evals"], ref.lam, rtol=1e-10, atol=1e-12 * an)


@pytest.mark.parametrize("prec", ["f64", "mixed"])
def test_plain_feast_response_stop_vs_oracle(ctx, prec):
    # plain FEAST with m0 well above m on a two-sided spectrum: the literal
    # check stalls on spurious in-I pairs; with the filter-response stop the
    # GPU and the oracle return the planted pairs within a few rounds
    from workloads import spectrum_config4
    lam, a, b, meta = spectrum_config4(10000, n=512)
    m = int(np.sum((lam > a) & (lam < b)))
    m0 = int(np.ceil(1.8 * m)) + 4
    P = make_problem("c4", lam, a, b, m0, 8, seed=10000)
    X0 = random_subspace(512, m0, seed=1)
    out = fg.feast_interval_solve(ctx, cuda(P.A), a, b, m0, 8, 1e-10,
                                  fg.feast_opts_default(prec=prec, anorm=P.anorm, max_iter=12, response_stop=1),
                                  x0=cuda(X0))
    ref = O.feast_solve(P.A, a, b, m0, 8, 1e-10, X0, anorm=P.anorm, max_iter=12, response_stop=True)
    assert out["status"] == 0 == ref.status
    assert out["iterations"] <= 4
    check_against_planted(out, P)
    np.testing.assert_allclose(out["evals"], ref.lam, atol=1e-12 * P.anorm)
