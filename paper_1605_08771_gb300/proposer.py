"""Learned m0 / contour-node proposer for FEAST (the spectrum estimation ahead
of the solve that the paper names as future work, Sect. IV).

Pipeline, every numerical step in the library's kernels:
  features   64 stochastic-trace Chebyshev moments of the spectral density of
             A / (1.02 ||A||) (feast_spectral_moments, 16 seeded N(0,1) probes);
  count      m_hat, the kernel-polynomial eigenvalue count of the interval from
             those moments (feast_moments_count);
  network    64 -> 256 -> 256 -> 256 -> 9 ReLU MLP in FP32 (feast_mlp_forward);
             output o decodes to m0 = ceil(m_hat 1.5 exp(0.6 tanh o_0)) and node
             offsets delta_j = 0.3 tanh(o_j) (feast_opts.node_offsets), so o = 0
             is the plain rule m0 = ceil(1.5 m_hat) with Gauss-Legendre nodes;
  labels     for each training spectrum, plain FEAST runs (with the
             filter-response stop: the spectra have eigenvalues on both sides
             of I) over candidate (m0 factor, node placement) pairs; the label
             is the candidate that converged to the right count in the fewest
             rounds among those no slower than the plain rule's candidate
             (ties: the faster), so fewer rounds are not bought with time;
  training   mean squared error to the encoded labels, Adam, by the library's
             forward/backward/Adam kernels (feast_mlp_train_step).
The plain rule is the fallback: a proposal whose solve does not converge is
re-run with it.

  python -m paper_1605_08771_gb300.proposer train --train 200 --out weights.npz
  python -m paper_1605_08771_gb300.proposer eval --weights weights.npz --count 40
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import paper_1605_08771_gb300 as fg  # noqa: E402

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "proposer_weights.npz")
N_MOMENTS = 64
N_PROBES = 16
N_C = 8
M0_FACTORS = (1.25, 1.5, 2.0, 2.5)       # candidate m0 / m_hat
NODE_PUSH = (0.0, 0.2)                   # candidate node placements: delta_j = kappa t_j
HELD_OUT_BASE = 10000                    # held-out seeds 10000.. (training seeds 0..)


def gauss_abscissae(n_c=N_C):
    # the library's contour uses Gauss-Legendre abscissae in ascending order;
    # the host only needs them to express a node placement as offsets
    t, _ = np.polynomial.legendre.leggauss(n_c)
    return np.sort(t)


def decode(o, m_hat, n):
    """Network output (9) -> (m0, node offsets)."""
    s = 1.5 * math.exp(0.6 * math.tanh(float(o[0])))
    m0 = int(min(n, max(8, math.ceil(s * max(m_hat, 1.0)))))
    return m0, 0.3 * np.tanh(np.asarray(o[1:], dtype=np.float64))


def encode(factor, offsets):
    """(m0 factor, node offsets) -> the network output that decodes to them."""
    o = np.zeros(1 + N_C, dtype=np.float32)
    o[0] = math.atanh(max(-0.999, min(0.999, math.log(factor / 1.5) / 0.6)))
    o[1:] = np.arctanh(np.clip(np.asarray(offsets) / 0.3, -0.999, 0.999))
    return o


def plain_rule(m_hat, n):
    return int(min(n, max(8, math.ceil(1.5 * max(m_hat, 1.0))))), None


class Problem:
    """One config-4 planted spectrum on the GPU."""

    def __init__(self, seed, n, device="cuda:0"):
        from workloads import spectrum_config4
        from workloads.planted import planted_matrix_torch
        self.seed = seed
        self.lam, self.lmin, self.lmax, self.meta = spectrum_config4(seed, n=n)
        self.A = planted_matrix_torch(self.lam, seed, complex_=False, device=device)
        self.n = n
        self.m = int(np.sum((self.lam > self.lmin) & (self.lam < self.lmax)))
        self.anorm = float(np.max(np.abs(self.lam)))


def features(ctx, P):
    """(64 moments, m_hat) of the problem's spectral density."""
    import torch
    from workloads import random_subspace
    V = torch.from_numpy(random_subspace(P.n, N_PROBES, seed=P.seed + 77)).to(P.A.device)
    r = 1.02 * P.anorm
    mu = fg.feast_spectral_moments(ctx, P.A, V, 0.0, r, N_MOMENTS)
    m_hat = fg.feast_moments_count(mu, 0.0, r, P.lmin, P.lmax, P.n)
    return mu.astype(np.float32), m_hat


def solve(ctx, P, m0, offsets, max_iter=30, prec="mixed"):
    """Plain FEAST with the given m0 and node placement: (ok, iterations,
    filters, seconds); ok = converged to the planted count."""
    import torch
    opts = fg.feast_opts_default(prec=prec, anorm=P.anorm, max_iter=max_iter, response_stop=1,
                                 node_offsets=None if offsets is None else np.asarray(offsets, dtype=np.float64))
    torch.cuda.synchronize()
    t0 = time.time()
    try:
        out = fg.feast_interval_solve(ctx, P.A, P.lmin, P.lmax, m0, N_C, 1e-10, opts)
    except fg.FeastError:
        return False, max_iter, max_iter, time.time() - t0
    torch.cuda.synchronize()
    ok = out["status"] == 0 and out["evals"].size == P.m
    return ok, out["iterations"], out["stats"].filters, time.time() - t0


def run_candidates(ctx, P, m_hat):
    """Plain FEAST over every candidate (m0 factor, node placement)."""
    t = gauss_abscissae()
    table = []
    for kappa in NODE_PUSH:
        offs = kappa * t
        for f in M0_FACTORS:
            m0 = int(min(P.n, max(8, math.ceil(f * max(m_hat, 1.0)))))
            ok, it, filt, sec = solve(ctx, P, m0, offs if kappa else None, max_iter=20)
            table.append({"factor": f, "kappa": kappa, "m0": m0, "ok": ok, "iterations": it, "rhs": filt * m0,
                          "seconds": round(sec, 4)})
    return table


def label_from(table):
    """The encoded target of a candidate table: the fewest rounds among the
    converged candidates no slower than the plain rule's (factor 1.5, Gauss
    nodes; 5 % timing margin), ties to the faster; None when none converged."""
    ok = [c for c in table if c["ok"]]
    if not ok:
        return None
    plain = [c for c in ok if c["factor"] == 1.5 and c["kappa"] == 0.0]
    limit = 1.05 * plain[0]["seconds"] if plain else math.inf
    pool = [c for c in ok if c["seconds"] <= limit] or ok
    best = min(pool, key=lambda c: (c["iterations"], c["seconds"]))
    return encode(best["factor"], best["kappa"] * gauss_abscissae())


def he_params(seed=0):
    """He-normal weights, zero biases, packed in the library's layout."""
    rng = np.random.default_rng(seed)
    dims = [64, 256, 256, 256, 9]
    out = []
    for din, dout in zip(dims[:-1], dims[1:]):
        out.append((rng.standard_normal((dout, din)) * math.sqrt(2.0 / din)).ravel())
        out.append(np.zeros(dout))
    # the output layer starts small so the untrained network proposes the plain rule
    out[-2] *= 0.01
    return np.concatenate(out).astype(np.float32)


def fit(ctx, X, T, epochs=400, batch=64, lr=1e-3, seed=0, val_frac=0.2):
    """Adam with the library's kernels; a fifth of the labelled spectra is
    held out and the parameters of the epoch with the lowest held-out loss
    are kept (the network has far more parameters than there are labels)."""
    import torch
    dev = "cuda:0"
    P = torch.from_numpy(he_params(seed)).to(dev)
    m = torch.zeros_like(P)
    v = torch.zeros_like(P)
    rng = np.random.default_rng(seed)
    N = X.shape[0]
    order = rng.permutation(N)
    nval = max(1, int(val_frac * N)) if N >= 5 else 0
    vi, ti = order[:nval], order[nval:]
    Xd = torch.from_numpy(np.ascontiguousarray(X[ti], dtype=np.float32)).to(dev)
    Td = torch.from_numpy(np.ascontiguousarray(T[ti], dtype=np.float32)).to(dev)
    Xv = torch.from_numpy(np.ascontiguousarray(X[vi], dtype=np.float32)).to(dev) if nval else None
    Tv = T[vi]
    Nt = Xd.shape[0]
    step = 0
    losses, vlosses = [], []
    best, best_P = math.inf, P.clone()
    for ep in range(epochs):
        perm = rng.permutation(Nt)
        tot = 0.0
        for b0 in range(0, Nt, batch):
            idx = torch.from_numpy(perm[b0:b0 + batch]).to(dev)
            xb = Xd.index_select(0, idx).contiguous()
            tb = Td.index_select(0, idx).contiguous()
            step += 1
            tot += fg.feast_mlp_train_step(ctx, P, m, v, xb, tb, step, lr) * xb.shape[0]
        losses.append(tot / Nt)
        if nval:
            yv = fg.feast_mlp_forward(ctx, P, Xv).cpu().numpy()
            vl = float(np.mean((yv - Tv) ** 2))
            vlosses.append(vl)
            if vl < best:
                best, best_P = vl, P.clone()
    return (best_P if nval else P), losses, vlosses


def propose(ctx, params, P):
    """(m0, offsets, m_hat) proposed for the problem by the network."""
    import torch
    mu, m_hat = features(ctx, P)
    X = torch.from_numpy(mu[None, :]).to(P.A.device)
    o = fg.feast_mlp_forward(ctx, params, X).cpu().numpy()[0]
    m0, offs = decode(o, m_hat, P.n)
    return m0, offs, m_hat


def load_params(path=WEIGHTS, device="cuda:0"):
    import torch
    d = np.load(path)
    return torch.from_numpy(d["params"].astype(np.float32)).to(device)


def evaluate(ctx, params, seeds, n):
    """Plain rule against the proposal (plain rule as the fallback when the
    proposal does not converge) on the given spectra."""
    rows = []
    for s in seeds:
        P = Problem(s, n)
        m0p, _ = plain_rule(features(ctx, P)[1], n)
        okp, itp, fp, tp = solve(ctx, P, m0p, None)
        m0l, offs, m_hat = propose(ctx, params, P)
        okl, itl, fl, tl = solve(ctx, P, m0l, offs)
        fallback = False
        if not okl:
            fallback = True
            okl, itl, fl, tl = okp, itp, fp, tp
            m0l = m0p
        rows.append({"seed": s, "m": P.m, "m_hat": round(m_hat, 2), "cluster": P.meta["cluster"],
                     "width": P.meta["width"], "plain": {"m0": m0p, "ok": okp, "iterations": itp, "rhs": fp * m0p,
                                                         "seconds": round(tp, 4)},
                     "learned": {"m0": m0l, "ok": okl, "iterations": itl, "rhs": fl * m0l, "seconds": round(tl, 4),
                                 "fallback": fallback}})
        del P
    return rows


def summary(rows):
    def mean(key, sub):
        return float(np.mean([r[sub][key] for r in rows]))
    return {"spectra": len(rows),
            "plain": {"mean_iterations": mean("iterations", "plain"), "mean_rhs": mean("rhs", "plain"),
                      "mean_seconds": mean("seconds", "plain"), "converged": sum(r["plain"]["ok"] for r in rows)},
            "learned": {"mean_iterations": mean("iterations", "learned"), "mean_rhs": mean("rhs", "learned"),
                        "mean_seconds": mean("seconds", "learned"),
                        "converged": sum(r["learned"]["ok"] for r in rows),
                        "fallbacks": sum(r["learned"]["fallback"] for r in rows)}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["train", "eval"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--train", type=int, default=200, help="training spectra (seeds 0..)")
    ap.add_argument("--count", type=int, default=40, help="held-out spectra for eval")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--out", default=WEIGHTS)
    ap.add_argument("--weights", default=WEIGHTS)
    ap.add_argument("--log", default="")
    ap.add_argument("--tables", default="", help="train: reuse the candidate runs of an earlier training log")
    args = ap.parse_args()
    fg.build_library()
    with fg.Feast(0) as f:
        ctx = f.ctx
        if args.what == "train":
            X, T, tables = [], [], []
            prior = {}
            if args.tables:
                prior = {t["seed"]: t["candidates"] for t in json.load(open(args.tables))["tables"]}
            t0 = time.time()
            for s in range(args.train):
                P = Problem(s, args.n)
                mu, m_hat = features(ctx, P)
                table = prior[s] if s in prior else run_candidates(ctx, P, m_hat)
                tgt = label_from(table)
                tables.append({"seed": s, "m": P.m, "m_hat": m_hat, "meta": P.meta, "candidates": table})
                if tgt is not None:
                    X.append(mu)
                    T.append(tgt)
                del P
            gen_s = time.time() - t0
            X, T = np.array(X), np.array(T)
            params, losses, vlosses = fit(ctx, X, T, epochs=args.epochs)
            summary_ = {"n": args.n, "train_spectra": args.train, "labelled": int(len(X)), "epochs": args.epochs,
                        "first_loss": losses[0], "final_loss": losses[-1],
                        "best_heldout_loss": min(vlosses) if vlosses else None,
                        "best_epoch": int(np.argmin(vlosses)) if vlosses else None,
                        "label_seconds": round(gen_s, 1), "m0_factors": M0_FACTORS, "node_push": NODE_PUSH}
            np.savez_compressed(args.out, params=params.cpu().numpy(), meta=json.dumps(summary_))
            if args.log:
                json.dump({"tables": tables, "losses": losses, "heldout_losses": vlosses}, open(args.log, "w"))
            print(json.dumps(summary_))
        else:
            params = load_params(args.weights)
            rows = evaluate(ctx, params, range(HELD_OUT_BASE, HELD_OUT_BASE + args.count), args.n)
            out = {"summary": summary(rows), "rows": rows}
            if args.log:
                json.dump(out, open(args.log, "w"))
            print(json.dumps(out["summary"]))


if __name__ == "__main__":
    main()
