#!/usr/bin/env python
"""Benchmark of the FEAST interval eigensolver on one GB300.

Workload (the single-large-problem case): complex Hermitian planted matrix
A = Q diag(lambda) Q^H, n = 8192, Q from the QR factorisation of a seeded
complex Gaussian; 200 eigenvalues in I = [-1, 1] of which 30 lie within 1e-4
inside each edge, 60 lie within 1e-4 outside each edge, the rest uniform in
[-50, 50]; n_c = 8 Gauss nodes, m0 = 300, tol 1e-10.  Plain FEAST stalls on it
(more than m0 eigenvalues have |rho| near 1/2), so it runs RFEAST (s = 3), the
paper's residual-expansion variant, in the mixed precision (complex FP32
factorisations and solves, FP64-accurate refinement and Rayleigh-Ritz), with
two readings of the paper switched on: only unconverged pairs expand the
subspace (rfeast_expand = 1) and the filter-response stop (response_stop = 1);
with the paper's literal checks alone, spurious in-I Ritz pairs of this
two-sided spectrum keep the step-3 check from passing.

A step is one complete feast_interval_solve (factorisations, filters,
Rayleigh-Ritz, checks) with A resident in HBM.  value = eigenpairs found inside
I (all at residual <= 1e-10) / seconds, summed over ranks.  Also reported:
e2e (same call with A in pinned host memory and the results copied back inside
the timed region), the roofline of the dominant kernel of the factorisations and solves, the
filter-apply rate, per-pair errors against the planted spectrum and the FP64
path, the FP64 path on the same input (mixed vs FP64), the n = 500 plain FP64
FEAST workload, the CPU oracle (timed in full on the n = 500 workload and on
this workload scaled to n = 2048, and extrapolated to n = 8192 from a sample
of the same matrix), clocks and the number of kernel launches.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "converged eigenpairs/sec at residual 1e-10; filter-apply TFLOP/s vs peak; mixed vs FP64"
UNIT = "eigenpairs/s"
WORKLOAD = dict(n=8192, m_in=200, edge_in=30, edge_out=60, width=1e-4, bulk=50.0,
                lmin=-1.0, lmax=1.0, m0=300, n_c=8, tol=1e-10, variant="rfeast", s=3, seed=0,
                rfeast_expand=1, response_stop=1, gen="torch_cpu", refine_switch=0.0)
# the n = 500 plain FP64 FEAST workload (real symmetric, 40 of 500 eigenvalues in
# [-1, 1], 5 within 1e-3 of each edge; n_c = 8, m0 = 60)
CONFIG1 = dict(n=500, m0=60, n_c=8, tol=1e-10, lmin=-1.0, lmax=1.0, seed=0)
# eigenvalue gate: |lambda - lambda_planted| <= 1e-10 |lambda| + 1e-12 ||A||
EIG_RTOL, EIG_ATOL_ANORM = 1e-10, 1e-12
NUM_SMS = 152
FP32_LANES_PER_SM = 128
DF32_FP32_OPS_PER_MAC = 12   # TwoProd (2) + TwoSum (6) + 2 cross FMAs + 2 adds
OZ_PAIRS = 21                # digit products p + q <= 5 of six 8-bit digits
# DRAM bytes per flop of cgemm_prefetch_kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum over every launch of the n = 4096 solve, profiles/); each launch is
# a rank-64 (or rank-32) update whose C read-modify-write dominates its traffic, so traffic
# scales with the flops of the launch; None until captured
CGEMM_DRAM_BYTES_PER_FLOP = 171.81e9 / 5.2540e12
CGEMM_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum over the 3151 cgemm_prefetch_kernel "
                        "launches of the n = 4096 solve (171.81 GB, cold-cache replay) / their 5.254e12 flops, "
                        "x flops per launch")
# the same for the tensor-core cg_update_kernel: two single-launch ncu captures of the n = 4096
# filter (profiles/cg_update_kernel_lu_solve_n4096.md), an LU trailing update (M = N = 2688,
# K = 128, 8 nodes: 931.6 MB for 5.92e10 flops) and a rank-256 solve update (M = 3840, N = 150,
# K = 256, 8 nodes: 150.4 MB for 9.44e9 flops); both near 0.0157 B/flop, the C read-modify-write
# plus the operand planes, so traffic is taken in proportion to a launch's flops
TCG_DRAM_BYTES_PER_FLOP = (931.6e6 + 150.4e6) / (5.92e10 + 9.44e9)
TCG_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one LU and one solve cg_update_kernel "
                      "launch (n = 4096 filter, 1082 MB for 6.86e10 flops) x flops per launch")
# the same for the digit-split GEMM: one full-size launch of the n = 8192 solve (the second oz_gemm_kernel
# launch, M = K = 8192, N = 16 x 300: 6.90 GB read + 0.31 GB written for 3.22e11 multiply-adds; one pass,
# profiles/oz_gemm_kernel_filter_n4096.md); a launch's waves of 152 tiles each stream their row and column
# panels, so traffic grows with the launch's multiply-adds
OZ_DRAM_BYTES_PER_MAC = (6.90e9 + 0.31387e9) / (8192.0 * 8192.0 * 4800.0)
OZ_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one full-size oz_gemm_kernel launch "
                     "(M = K = 8192, N = 4800: 7.21 GB for 3.22e11 multiply-adds) x multiply-adds per launch")



def workload_name(w):
    rd = ""
    if w["variant"] == "rfeast" and (w.get("rfeast_expand") or w.get("response_stop")):
        rd = " (readings: unconverged-only expansion, filter-response stop)"
    return (f"complex Hermitian planted n={w['n']}, {w['m_in']} eigenvalues in [-1,1] with "
            f"{w['edge_in']}+{w['edge_in']} within {w['width']:g} inside and {w['edge_out']}+{w['edge_out']} "
            f"within {w['width']:g} outside the edges, bulk in [-{w['bulk']:g},{w['bulk']:g}]; "
            f"n_c={w['n_c']}, m0={w['m0']}, {w['variant'].upper()} s={w['s']}{rd}")


def scaled_workload(n):
    """The benchmark workload scaled to n (counts and m0 in proportion)."""
    w = dict(WORKLOAD)
    scale = n / w["n"]
    w.update(n=n, m_in=max(4, int(w["m_in"] * scale)), edge_in=max(1, int(w["edge_in"] * scale)),
             edge_out=max(1, int(w["edge_out"] * scale)), m0=max(8, int(w["m0"] * scale)))
    return w


def pair_errors(evals, res, planted, anorm):
    """Per-pair pointwise relative eigenvalue errors and relative residuals
    against the planted eigenvalues (None when the counts differ)."""
    if evals.size != planted.size:
        return None
    err = np.abs(evals - planted)
    rel = err / np.maximum(np.abs(planted), 1e-300)
    gate = bool(np.all(err <= EIG_RTOL * np.abs(planted) + EIG_ATOL_ANORM * anorm))
    return {"count": int(evals.size), "gate": gate,
            "eig_rel_err_max": float(rel.max()) if rel.size else 0.0,
            "eig_abs_err_max_rel_anorm": float(err.max() / anorm) if err.size else 0.0,
            "residual_max": float(np.max(res)) if res.size else 0.0,
            "eig_rel_err": [float("%.3g" % v) for v in rel],
            "residual": [float("%.3g" % v) for v in res]}


# ---------------------------------------------------------------------------
# measured peaks
# ---------------------------------------------------------------------------
def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["not sampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample(A_host, w, filters, rr_k_sum, rr_k3_sum, budget_s=30.0, ns_max=2048):
    """Time the FP64 CPU oracle on bounded pieces of the same solve and
    extrapolate to the full solve by operation counts.

    Sample: the oracle's LU of the leading ns x ns block of z_1 I - A, its
    forward/back solve of m_s right-hand sides, one Rayleigh-Ritz of that block
    on an orthonormal ns x m_s basis (W = A Q, A' = Q^H W, Jacobi); ns chosen so
    the sample takes about 10 s.  Extrapolation: LU ~ n^3 (times n_c nodes),
    solves ~ n^2 m (times the solve entries of every filter application),
    Rayleigh-Ritz GEMMs ~ n^2 k and Jacobi ~ k^3 summed over the passes of the
    run (rr_k_sum = sum of k, rr_k3_sum = sum of k^3)."""
    import oracle

    n, m0, nc = w["n"], w["m0"], w["n_c"]
    z, _ = oracle.contour_nodes(w["lmin"], w["lmax"], nc)
    t_start = time.time()
    ns = 512
    while True:
        M = z[0] * np.eye(ns) - A_host[:ns, :ns]
        t0 = time.time()
        LU, piv = oracle.lu_factor(M)
        t_lu = time.time() - t0
        if t_lu > 1.5 or ns >= min(ns_max, A_host.shape[0]) or time.time() - t_start > budget_s / 3:
            break
        ns *= 2
    ms = max(8, int(round(m0 * ns / n)))
    rng = np.random.default_rng(1)
    B = rng.standard_normal((ns, ms)) + 1j * rng.standard_normal((ns, ms))
    t0 = time.time()
    oracle.lu_solve(LU, piv, B)
    t_solve = time.time() - t0
    Qs, _ = np.linalg.qr(B)
    t0 = time.time()
    oracle.rayleigh_ritz(A_host[:ns, :ns], Qs, 50.0)
    t_rr = time.time() - t0
    # split the Rayleigh-Ritz sample into its GEMM (n^2 k) and Jacobi (k^3) parts
    H = Qs.conj().T @ (A_host[:ns, :ns] @ Qs)
    t0 = time.time()
    oracle.jacobi_eigh(0.5 * (H + H.conj().T))
    t_jac = time.time() - t0
    t_gemm = max(t_rr - t_jac, 1e-9)
    entries = 2 * nc
    T = nc * t_lu * (n / ns) ** 3
    T += filters * entries * t_solve * (n / ns) ** 2 * (m0 / ms)
    T += t_gemm * (n / ns) ** 2 * (rr_k_sum / ms) + t_jac * rr_k3_sum / float(ms) ** 3
    sample_s = time.time() - t_start
    return T, ns, ms, sample_s


# ---------------------------------------------------------------------------
def build_problem(w, device):
    from workloads import spectrum_config2
    from workloads.planted import planted_matrix_torch
    lam, a, b = spectrum_config2(w["seed"], n=w["n"], m_in=w["m_in"], edge_in=w["edge_in"],
                                 edge_out=w["edge_out"], width=w["width"], bulk=w["bulk"])
    A = planted_matrix_torch(lam, w["seed"], complex_=True, device=device, gen=w["gen"])
    # A_store: contiguous buffer holding A column-major; A is its transposed view
    A_store = A.transpose(0, 1)
    assert A_store.is_contiguous()
    return A_store, lam


def aggregate_ranks(ms_total, pairs, world, device="cpu"):
    """Whole-job figures over the ranks of one node: the pairs all ranks
    found, over the slowest rank's time (each rank runs its own replica of
    the problem; no data-path collective).  Returns (t_max_ms, pairs_sum)."""
    if world <= 1:
        return float(ms_total), float(pairs)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms_total)], dtype=torch.float64, device=device)
    p = torch.tensor([float(pairs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def tc_peak(peaks):
    """The measured sustained bf16 rate (the kernels run inside a seconds-long
    step) and the dense TF32 roof derived from it (nominal TF32:bf16 1:2)."""
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
    return bf16 / 2.0, bf16


# bf16 multiply-adds per complex multiply-add of the tensor-core complex-FP32
# GEMM: 4 real products x 6 split products of three-part bf16 operands
CG_BF16_PER_CMAC = 24


def factor_solve_roofline(st, ms_step, peaks, peak_kind, sm_max):
    """Roofline of the GEMM updates of the shifted factorisations and solves:
    on the tensor cores (cg_update_kernel) by default, on the FP32 SIMT pipes
    (cgemm_prefetch_kernel) with --prec mixed_simt.  achieved = algorithmic
    flops (8 per complex multiply-add, M N K per launch) / CUDA-event time per
    launch.  Tensor cores: the FP32-exact products cost 24 bf16 multiply-adds
    per complex multiply-add, so the roof of this arithmetic is the measured
    sustained bf16 rate x 8/48; the fraction equals executed bf16 flops over
    the bf16 rate."""
    tf32, bf16 = tc_peak(peaks)
    fp32_simt = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    if st.tcgemm_launches > 0:
        launches, ms, flop = st.tcgemm_launches, st.tcgemm_ms, st.tcgemm_flop
        avg_ms = ms / launches
        achieved = flop / launches / (avg_ms / 1e3) / 1e12
        peak = bf16 * 8.0 / (2.0 * CG_BF16_PER_CMAC)
        traffic = int(TCG_DRAM_BYTES_PER_FLOP * flop / launches) if TCG_DRAM_BYTES_PER_FLOP else None
        return {"kernel": "cg_update_kernel (tcgen05 complex-FP32 GEMM updates of the LU and solves)",
                "bound": "tensor", "achieved": round(achieved, 2), "peak": round(peak, 1), "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": ("MEASURED_PEAKS.json bf16_tflops_sustained (%s, %.1f) x 8/48: 24 bf16 "
                                "multiply-adds per complex-FP32 multiply-add" % (peak_kind, bf16)),
                "flop_def": "8 real flops per complex multiply-add, M N K per launch",
                "executed_bf16_tflops": round(achieved * 2 * CG_BF16_PER_CMAC / 8, 1),
                "frac_of_tf32_roof": round(achieved / tf32, 4),
                "traffic_source": TCG_TRAFFIC_SOURCE,
                "launches_per_step": launches, "avg_launch_ms": round(avg_ms, 4),
                "share_of_step": round(ms / ms_step, 3)}
    cg_launches = max(1, st.cgemm_launches)
    cg_avg_ms = st.cgemm_ms / cg_launches
    cg_flop_per_launch = st.cgemm_flop / cg_launches
    achieved = cg_flop_per_launch / (cg_avg_ms / 1e3) / 1e12 if st.cgemm_ms > 0 else 0.0
    traffic = int(CGEMM_DRAM_BYTES_PER_FLOP * cg_flop_per_launch) if CGEMM_DRAM_BYTES_PER_FLOP else None
    return {"kernel": "cgemm_prefetch_kernel (complex-FP32 GEMM updates of the LU and solves, SIMT)",
            "bound": "alu", "achieved": round(achieved, 3), "peak": round(fp32_simt, 2), "unit": "TFLOP/s",
            "frac": round(achieved / fp32_simt, 4), "traffic": traffic,
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x max SM clock (unit counts)",
            "flop_def": "8 real flops per complex multiply-add, M N K per launch",
            "frac_of_tf32_roof": round(achieved / tf32, 4),
            "traffic_source": CGEMM_TRAFFIC_SOURCE,
            "launches_per_step": st.cgemm_launches, "avg_launch_ms": round(cg_avg_ms, 4),
            "share_of_step": round(st.cgemm_ms / ms_step, 3)}


def host_residuals(A, V, evals, anorm):
    """||A x - lambda x|| / ||A|| of the returned pairs, recomputed in FP64 by
    torch (a check outside the library)."""
    import torch
    if evals.size == 0:
        return np.zeros(0)
    lam = torch.as_tensor(evals, dtype=torch.float64, device=V.device).to(V.dtype)
    R = A @ V - V * lam[None, :]
    return (torch.linalg.vector_norm(R, dim=0) / anorm).cpu().numpy()


def run_config1(fg, ctx, stream, dev, cpu):
    """The n = 500 plain FP64 FEAST workload: time-to-solution on the GPU
    (median of 5 after one warm-up) and, with cpu, the oracle timed in full on
    the same matrix and starting subspace."""
    import torch
    from workloads import make_problem, random_subspace, spectrum_config1
    c = CONFIG1
    lam, a, b = spectrum_config1(c["seed"])
    P = make_problem("c1", lam, a, b, c["m0"], c["n_c"], seed=c["seed"])
    X0 = random_subspace(P.n, c["m0"], seed=1)
    A = torch.from_numpy(P.A).to(f"cuda:{dev}")
    x0 = torch.from_numpy(X0).to(f"cuda:{dev}")
    opts = fg.feast_opts_default(variant="feast", prec="f64", anorm=P.anorm)
    times, out = [], None
    for i in range(6):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fg.feast_interval_solve(ctx, A, a, b, c["m0"], c["n_c"], c["tol"], opts, x0=x0)
        e1.record(stream)
        torch.cuda.synchronize()
        if i > 0:
            times.append(e0.elapsed_time(e1))
    ms = float(np.median(times))
    pe = pair_errors(out["evals"], out["res"], P.inside, P.anorm)
    line = {"workload": "real symmetric planted n=500, 40 eigenvalues in [-1,1] (5 within 1e-3 of each edge), "
                        "460 uniform in [-10,10] outside; n_c=8, m0=60, plain FEAST, FP64",
            "ms_per_solve": round(ms, 2), "value": round(out["evals"].size / (ms / 1e3), 2), "unit": UNIT,
            "iterations": out["iterations"], "correct": bool(out["status"] == 0 and pe is not None and pe["gate"]
                                                             and pe["residual_max"] <= c["tol"]),
            "eig_rel_err_max": pe["eig_rel_err_max"] if pe else None,
            "residual_max": pe["residual_max"] if pe else None}
    if cpu:
        import oracle
        t0 = time.time()
        r = oracle.feast_solve(P.A, a, b, c["m0"], c["n_c"], c["tol"], X0, anorm=P.anorm)
        t = time.time() - t0
        line["oracle"] = {"seconds": round(t, 2), "value": round(r.lam.size / t, 3), "iterations": r.iterations,
                          "timed": "in full (same matrix and X0)"}
        line["speedup_vs_oracle"] = round(t * 1e3 / ms, 1)
    return line


def run_config5(fg, ctx, stream, dev, n=32768):
    """The largest single problem (real symmetric n = 32768, m0 = 1000, 700
    eigenvalues in I, 80 within 1e-5 outside each edge; plain FEAST, mixed
    precision): one timed solve after the matrix is built on the GPU."""
    import torch
    from workloads import spectrum_config5
    from workloads.planted import planted_matrix_torch
    lam, a, b = spectrum_config5(0, n=n, m_in=int(700 * n / 32768), edge_out=int(80 * n / 32768))
    m0 = int(1000 * n / 32768)
    t0 = time.time()
    A = planted_matrix_torch(lam, 0, complex_=False, device=f"cuda:{dev}")
    torch.cuda.synchronize()
    build_s = time.time() - t0
    torch.cuda.empty_cache()
    inside = lam[(lam > a) & (lam < b)]
    anorm = float(np.max(np.abs(lam)))
    opts = fg.feast_opts_default(variant="feast", prec="mixed", anorm=anorm, max_iter=20, response_stop=1)
    # a context of its own: its workspace (about 200 GB at n = 32768) is freed after
    ctx5 = fg.feast_init(dev, stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fg.feast_interval_solve(ctx5, A, a, b, m0, 8, 1e-10, opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    pe = pair_errors(out["evals"], out["res"], inside, anorm)
    hres = host_residuals(A, out["evecs"], out["evals"], anorm)
    st = out["stats"]
    free, total = torch.cuda.mem_get_info()
    res = {"workload": f"real symmetric planted n={n}, {inside.size} eigenvalues in [-1,1], "
                       f"{int(80 * n / 32768)}+{int(80 * n / 32768)} within 1e-5 outside the edges, bulk in [-50,50]; "
                       f"n_c=8, m0={m0}, plain FEAST with the filter-response stop, mixed precision",
           "ms_per_solve": round(ms, 1), "value": round(out["evals"].size / (ms / 1e3), 3), "unit": UNIT,
           "iterations": out["iterations"], "filters": st.filters, "refine_steps": st.refine_steps,
           "factor_ms": round(st.factor_ms, 1), "filter_ms": round(st.filter_ms, 1),
           "tcgemm_tflops": round(st.tcgemm_flop / max(st.tcgemm_ms, 1e-9) / 1e9, 1),
           "correct": bool(out["status"] == 0 and pe is not None and pe["gate"] and pe["residual_max"] <= 1e-10
                           and hres.max() <= 2e-10),
           "eig_rel_err_max": pe["eig_rel_err_max"] if pe else None,
           "residual_max": pe["residual_max"] if pe else None,
           "host_residual_max": float(hres.max()) if hres.size else None,
           "matrix_build_s": round(build_s, 1), "device_free_gb_during": round(free / 1e9, 1)}
    fg.feast_finalize(ctx5)
    del A
    torch.cuda.empty_cache()
    return res


def run_config3(fg, dev, count=64, workers=8):
    """The batched workload: `count` independent real symmetric problems of
    uneven n (512..4096) and m0, mixed precision, plain FEAST: one batch on a
    pool of streams (autotuned route) against the same problems one after
    another on one stream; both timed on the host clock around the call."""
    import torch
    from workloads.planted import planted_matrix_torch, spectrum_config3
    probs, inside = [], []
    for seed in range(count):
        lam, a, b, m0, n_c = spectrum_config3(seed)
        A = planted_matrix_torch(lam, seed, complex_=False, device=f"cuda:{dev}")
        probs.append({"A": A, "lmin": a, "lmax": b, "m0": m0, "n_c": n_c, "tol": 1e-10})
        inside.append(lam[(lam > a) & (lam < b)])
    torch.cuda.synchronize()
    opts = fg.feast_opts_default(prec="mixed", max_iter=40, response_stop=1)
    fg.feast_interval_solve_batch(probs[:2], opts, workers=2, autotune=True)   # warm-up, fills the tuner
    res = {}
    for label, w in (("batched", workers), ("sequential", 1)):
        torch.cuda.synchronize()
        t0 = time.time()
        out = fg.feast_interval_solve_batch(probs, opts, workers=w, autotune=True)
        torch.cuda.synchronize()
        t = time.time() - t0
        ok = sum(int(r["status"] == 0 and r["evals"].size == ins.size and
                     np.all(np.abs(r["evals"] - ins) <= 1e-10 * np.abs(ins) + 1e-12 * np.max(np.abs(ins))))
                 for r, ins in zip(out, inside))
        pairs = sum(r["evals"].size for r in out)
        res[label] = {"workers": w, "seconds": round(t, 3), "value": round(pairs / t, 2), "unit": UNIT,
                      "pairs": pairs, "problems_correct": ok,
                      "routes": {"tensor": sum(r["route"] == fg.FEAST_PREC_MIXED for r in out),
                                 "simt": sum(r["route"] == fg.FEAST_PREC_MIXED_SIMT for r in out)}}
    res["workload"] = (f"{count} real symmetric planted problems, n in 512..4096, 10..170 eigenvalues in each own "
                       "interval with edge clusters, m0 = ceil(1.5 m), n_c in {8, 16}; plain FEAST with the "
                       "filter-response stop, mixed")
    res["speedup"] = round(res["sequential"]["seconds"] / res["batched"]["seconds"], 3)
    del probs
    torch.cuda.empty_cache()
    return res


def oracle_full_scaled(n):
    """The oracle timed in full on the benchmark workload scaled to n (same
    generator and readings), with its own iteration and filter counts."""
    import oracle
    from workloads import make_problem, random_subspace, spectrum_config2
    w = scaled_workload(n)
    lam, a, b = spectrum_config2(w["seed"], n=w["n"], m_in=w["m_in"], edge_in=w["edge_in"],
                                 edge_out=w["edge_out"], width=w["width"], bulk=w["bulk"])
    P = make_problem("c2", lam, a, b, w["m0"], w["n_c"], seed=w["seed"], complex_=True)
    X0 = random_subspace(n, w["m0"], seed=1, complex_=True)
    t0 = time.time()
    r = oracle.feast_solve(P.A, a, b, w["m0"], w["n_c"], w["tol"], X0, variant=oracle.RFEAST, s=w["s"],
                           anorm=P.anorm, max_iter=30,
                           expand=oracle.EXPAND_UNCONVERGED if w["rfeast_expand"] else oracle.EXPAND_ALL,
                           response_stop=bool(w["response_stop"]))
    t = time.time() - t0
    pe = pair_errors(r.lam, r.res, P.inside, P.anorm)
    return {"n": n, "m0": w["m0"], "seconds": round(t, 1), "value": round(r.lam.size / t, 4), "unit": UNIT,
            "iterations": r.iterations, "filters": r.filters, "rr_dims": r.rr_dims, "status": r.status,
            "correct": bool(pe is not None and pe["gate"]), "timed": "in full"}


def run_ours(args, rank, world, dev):
    import torch
    import paper_1605_08771_gb300 as fg

    w = scaled_workload(args.n) if args.n else dict(WORKLOAD)
    w["prec"] = args.prec
    w["variant"] = args.variant
    w["gen"] = args.gen
    w["refine_switch"] = args.refine_switch
    fg.build_library()
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    A_store, lam = build_problem(w, f"cuda:{dev}")
    A = A_store.transpose(0, 1)
    inside = lam[(lam > w["lmin"]) & (lam < w["lmax"])]
    anorm = float(np.max(np.abs(lam)))
    ctx = fg.feast_init(dev, stream)
    rd = dict(rfeast_expand=w["rfeast_expand"], response_stop=w["response_stop"]) if w["variant"] != "feast" else {}
    if w["variant"] == "xfeast":
        rd.pop("rfeast_expand")
    opts = fg.feast_opts_default(variant=w["variant"], s=w["s"], prec=w["prec"], anorm=anorm, max_iter=30,
                                 refine_gemm=args.refine_gemm, refine_switch=w["refine_switch"], **rd)

    def solve(Adev):
        return fg.feast_interval_solve(ctx, Adev, w["lmin"], w["lmax"], w["m0"], w["n_c"], w["tol"], opts)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up
    out = None
    for _ in range(args.warmup):
        out = solve(A)
    barrier()
    # timed region
    launches0 = fg.feast_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    results = []
    with ClockSampler(dev) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            out = solve(A)
            results.append(out)
        ev1.record(stream)
        barrier()
    ms_total = ev0.elapsed_time(ev1)
    launches = fg.feast_kernel_launches() - launches0
    ms_step = ms_total / args.steps
    found = [r["evals"].size for r in results]
    errs = [pair_errors(r["evals"], r["res"], inside, anorm) for r in results]
    ok = all(r["status"] == 0 and e is not None and e["gate"] and e["residual_max"] <= w["tol"]
             for r, e in zip(results, errs))
    t_max, pairs_all = aggregate_ranks(ms_total, sum(found), world, device=f"cuda:{dev}")
    value = pairs_all / (t_max / 1e3)
    st = results[-1]["stats"]
    last = results[-1]
    hres = host_residuals(A, last["evecs"], last["evals"], anorm)
    ok = ok and bool(hres.size == 0 or hres.max() <= 2 * w["tol"])

    # e2e: A in pinned host memory, copied in; results copied out; all timed
    Ah = A_store.cpu().pin_memory()
    e2e_steps = max(1, min(2, args.steps))
    Ad = torch.empty_like(A_store)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_found = 0
    d2h = 0
    for _ in range(e2e_steps):
        Ad.copy_(Ah, non_blocking=True)
        r = solve(Ad.transpose(0, 1))
        V = r["evecs"].cpu()
        e2e_found += r["evals"].size
        d2h = V.numel() * V.element_size() + 2 * r["evals"].nbytes
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    h2d = A.numel() * A.element_size()

    # per-kernel CUDA events on the library's stream (inside the library)
    peaks, peak_kind = measured_peaks()
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    roofline_fs = factor_solve_roofline(st, ms_step, peaks, peak_kind, sm_max)
    tf32_peak, _ = tc_peak(peaks)

    # the refinement GEMM: tensor-core digit-split GEMM by default,
    # double-float SIMT GEMM with --refine-gemm 1
    rg_launches = max(1, st.refine_gemm_launches)
    rg_avg_ms = st.refine_gemm_ms / rg_launches
    rg_mac_per_launch = st.refine_gemm_mac / rg_launches
    rg_secs = rg_avg_ms / 1e3
    if args.refine_gemm == 0:
        # 21 bf16 digit products per FP64 multiply-add: the bf16 tensor flops
        # the method executes, against the measured bf16 peak (sustained: the
        # kernel runs inside a seconds-long step)
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops", 1900.0))
        achieved = OZ_PAIRS * 2.0 * rg_mac_per_launch / rg_secs / 1e12 if rg_secs > 0 else 0.0
        roofline_refine = {"kernel": "oz_gemm_kernel", "bound": "tensor", "achieved": round(achieved, 2),
                           "peak": round(peak, 1), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                           "traffic": int(OZ_DRAM_BYTES_PER_MAC * rg_mac_per_launch),
                           "traffic_source": OZ_TRAFFIC_SOURCE,
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (%s)" % peak_kind,
                           "flop_def": "21 bf16 digit products x 2 x M N K per launch",
                           "fp64_equiv_tflops": round(achieved / OZ_PAIRS, 3)}
    else:
        peak = NUM_SMS * FP32_LANES_PER_SM * sm_max * 1e6 / DF32_FP32_OPS_PER_MAC * 2 / 1e12
        achieved = 2.0 * rg_mac_per_launch / rg_secs / 1e12 if rg_secs > 0 else 0.0
        roofline_refine = {"kernel": "gemm_df32_kernel", "bound": "alu", "achieved": round(achieved, 3),
                           "peak": round(peak, 3), "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                           "traffic": None,
                           "peak_source": ("FP32 lanes x clock / 12 FP32 ops per double-float multiply-add "
                                           "(152 SMs x 128 lanes x max SM clock)")}
    roofline_refine.update({"launches_per_step": st.refine_gemm_launches, "avg_launch_ms": round(rg_avg_ms, 3),
                            "share_of_step": round(st.refine_gemm_ms / ms_step, 3)})
    # `roofline` is the kernel with the larger share of the step; the other
    # tensor-core contraction is reported beside it
    if roofline_refine["share_of_step"] > roofline_fs["share_of_step"]:
        roofline, roofline_other, other_key = roofline_refine, roofline_fs, "roofline_factor_solve_gemm"
    else:
        roofline, roofline_other, other_key = roofline_fs, roofline_refine, "roofline_refine_gemm"

    # filter-apply rate: algorithmic flops of the solves (8 n^2 m per entry,
    # complex MAC = 8 real flops) per filter application, refinement excluded
    n, m0, nc = w["n"], w["m0"], w["n_c"]
    filt_flop = 2 * nc * 8.0 * n * n * m0
    filter_tflops = filt_flop * st.filters / (st.filter_ms / 1e3) / 1e12 if st.filter_ms > 0 else None
    emu_peak = roofline_fs["peak"] if roofline_fs["bound"] == "tensor" else tf32_peak

    pe = errs[-1] or {}
    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": ("c64+bf16x21" if args.refine_gemm == 0 else "c64+df32") if w["prec"] != "f64" else "c128",
            "data": "synthetic planted spectrum (seeded), no dataset",
            "config": {"workload": workload_name(w), "n": n, "m0": m0, "n_c": nc, "variant": w["variant"],
                       "s": w["s"], "prec": w["prec"], "tol": w["tol"],
                       "rfeast_expand": w["rfeast_expand"], "response_stop": w["response_stop"],
                       "refine_switch": w["refine_switch"], "q_gaussian": w["gen"],
                       "l2": "inputs larger than L2 (A is %.2f GB, L2 129 MB)" % (h2d / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "correct": bool(ok),
            "gate": "every step: count exact, |dl| <= 1e-10 |l| + 1e-12 ||A|| per pair, residual <= tol, "
                    "host-recomputed residual <= 2 tol",
            "eigenpairs_per_step": found[-1], "iterations": last["iterations"],
            "filters": st.filters, "refine_steps": st.refine_steps,
            "factor_ms": round(st.factor_ms, 1), "filter_ms": round(st.filter_ms, 1),
            "pairs_vs_planted": pe,
            "host_residual_max": float(hres.max()) if hres.size else None,
            "roofline": roofline, other_key: roofline_other,
            "filter_apply": {"tflops": round(filter_tflops, 3) if filter_tflops else None,
                             "peak": round(emu_peak, 1),
                             "frac": round(filter_tflops / emu_peak, 4) if filter_tflops else None,
                             "frac_of_tf32_roof": round(filter_tflops / tf32_peak, 4) if filter_tflops else None,
                             "flop_per_filter": filt_flop,
                             "note": ("solve flops 8 n^2 m0 per entry, 2 n_c entries, refinement excluded, over "
                                      "the whole filter time (solves, refinement, accumulation); peak: the "
                                      "tensor-core roof of the complex-FP32 solve arithmetic (roofline_factor_solve)")},
            "e2e": {"value": round(e2e_found / e2e_steps / (e2e_ms / 1e3), 4), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 1)},
            "gpu_launches": int(launches), "clocks": clocks, "peak_source": peak_kind}

    # mixed vs FP64 on the same input (one solve, CUDA events), per-pair errors
    if args.fp64 and w["prec"] != "f64":
        o64 = fg.feast_opts_default(variant=w["variant"], s=w["s"], prec="f64", anorm=anorm, max_iter=30, **rd)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r64 = fg.feast_interval_solve(ctx, A, w["lmin"], w["lmax"], m0, nc, w["tol"], o64)
        f1.record(stream)
        barrier()
        t64 = f0.elapsed_time(f1)
        d = rel = None
        if r64["evals"].size == last["evals"].size:
            dd = np.abs(r64["evals"] - last["evals"])
            d = float(dd.max() / anorm)
            rel = dd / np.maximum(np.abs(r64["evals"]), 1e-300)
        line["mixed_vs_fp64"] = {"fp64_ms": round(t64, 1), "mixed_ms": round(ms_step, 1),
                                 "speedup": round(t64 / ms_step, 3),
                                 "fp64_value": round(r64["evals"].size / (t64 / 1e3), 4),
                                 "max_eig_diff_rel_anorm": d, "fp64_iterations": r64["iterations"],
                                 "fp64_pairs": int(r64["evals"].size),
                                 "eig_rel_diff_max": float(rel.max()) if rel is not None and rel.size else None,
                                 "eig_rel_diff": [float("%.3g" % v) for v in rel] if rel is not None else None}

    # the batched uneven workload (opt-in)
    if args.config3:
        line["config3"] = run_config3(fg, dev, count=args.config3)

    # the largest single problem (opt-in: the matrix takes minutes to build)
    if args.config5:
        line["config5"] = run_config5(fg, ctx, stream, dev, n=args.config5)

    # the n = 500 plain FP64 FEAST workload (and its oracle timed in full)
    if args.config1:
        line["config1"] = run_config1(fg, ctx, stream, dev, args.cpu and world == 1)

    # CPU oracle (rank 0, N = 1 only): timed in full on the workload scaled to
    # n = 2048, and extrapolated to this workload from a sample of its matrix
    if args.cpu and world == 1:
        A_host = Ah.numpy().T
        T, ns, ms_, samp = oracle_sample(A_host, w, st.filters, st.rr_k_sum, st.rr_k3_sum)
        full = oracle_full_scaled(args.cpu_full_n) if args.cpu_full_n else None
        line["cpu_baseline"] = {"value": round(inside.size / T, 6), "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle", "extrapolated": True,
                                "sample": (f"extrapolated: oracle LU of the leading {ns}x{ns} block of z_1 I - A "
                                           f"(this matrix), its solve of {ms_} right-hand sides and one {ns}x{ms_} "
                                           f"Rayleigh-Ritz ({samp:.1f} s of CPU work), scaled by operation counts "
                                           f"to the full solve with this run's counts ({st.filters} filters, "
                                           f"{st.rr_passes} Rayleigh-Ritz passes, their dimensions): {T:.0f} s"),
                                "extrapolated_s": round(T, 1),
                                "timed_in_full": [x for x in [full] if x is not None]}
        if "config1" in line and "oracle" in line["config1"]:
            c1 = line["config1"]
            line["cpu_baseline"]["timed_in_full"].insert(0, {"n": 500, "seconds": c1["oracle"]["seconds"],
                                                             "value": c1["oracle"]["value"], "unit": UNIT,
                                                             "iterations": c1["oracle"]["iterations"],
                                                             "workload": "n = 500 plain FP64 FEAST (config1)",
                                                             "timed": "in full"})
    fg.feast_finalize(ctx)
    return line


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle on the host cores, on this
    workload's matrix (same spectrum and Gaussian seed; Q from the host's QR).
    Each step is a bounded sample (the oracle's LU, solve and Rayleigh-Ritz on
    a leading block), extrapolated by operation counts to the full solve with
    the oracle's own counts from a solve it runs in full, once, on the
    workload scaled to n = 1024 (its Rayleigh-Ritz dimensions scaled by n).
    ms_per_step is a step's measured wall time; value is the eigenpairs of
    the full solve over its extrapolated time."""
    if rank != 0:
        return None
    from workloads import spectrum_config2
    from workloads.planted import planted_block_host
    w = scaled_workload(args.n) if args.n else dict(WORKLOAD)
    w["prec"], w["variant"], w["gen"] = args.prec, args.variant, args.gen
    lam, a, b = spectrum_config2(w["seed"], n=w["n"], m_in=w["m_in"], edge_in=w["edge_in"],
                                 edge_out=w["edge_out"], width=w["width"], bulk=w["bulk"])
    t_build = time.time()
    A_host = planted_block_host(lam, w["seed"], min(1024, w["n"]), complex_=True,
                                gen=w["gen"] if w["gen"] != "torch_cuda" else "torch_cpu")
    t_build = time.time() - t_build
    small = oracle_full_scaled(min(1024, w["n"]))
    f = w["n"] / small["n"]
    filters = small["filters"]
    rr_dims = [d * f for d in small["rr_dims"]]
    k_sum, k3_sum = float(sum(rr_dims)), float(sum(k ** 3 for k in rr_dims))
    for _ in range(args.warmup):
        oracle_sample(A_host, w, filters, k_sum, k3_sum, budget_s=6.0, ns_max=1024)
    Ts, samples = [], []
    t0 = time.time()
    for _ in range(args.steps):
        T, ns, ms_, samp = oracle_sample(A_host, w, filters, k_sum, k3_sum, budget_s=6.0, ns_max=1024)
        Ts.append(T)
        samples.append(samp)
    wall = time.time() - t0
    value = w["m_in"] / float(np.mean(Ts))
    return {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * wall / max(args.steps, 1), 1),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic planted spectrum (seeded)",
            "impl": "reference", "extrapolated": True,
            "step": "one bounded sample of the workload (ms_per_step is its measured wall time); value is "
                    "the full solve's eigenpairs over extrapolated_ms_per_solve",
            "extrapolated_ms_per_solve": round(1e3 * float(np.mean(Ts)), 1),
            "sample_ms_per_step": round(1e3 * float(np.mean(samples)), 1),
            "config": {"workload": workload_name(w), "n": w["n"], "m0": w["m0"], "n_c": w["n_c"],
                       "variant": w["variant"], "s": w["s"], "prec": w["prec"], "tol": w["tol"],
                       "rfeast_expand": w["rfeast_expand"], "response_stop": w["response_stop"],
                       "q_gaussian": w["gen"],
                       "l2": "inputs larger than L2 (A is %.2f GB, L2 129 MB)" % (16.0 * w["n"] ** 2 / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": (f"extrapolated: the oracle's LU, solve and Rayleigh-Ritz on the leading "
                                        f"{ns}x{ns} block of this workload's matrix (built on the host in "
                                        f"{t_build:.0f} s), {float(np.mean(samples)):.1f} s per step, scaled by "
                                        f"operation counts to the full solve with the oracle's own counts from its "
                                        f"full solve of the workload scaled to n = {small['n']} ({small['seconds']} s: "
                                        f"{filters} filters, {small['iterations']} iterations, Rayleigh-Ritz "
                                        f"dimensions {small['rr_dims']} x {f:g})"),
                             "timed_in_full": [small]},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=0, help="override n (scaled workload, for quick checks)")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "mixed_simt", "f64"])
    ap.add_argument("--refine-gemm", type=int, default=0, choices=[0, 1],
                    help="refinement products: 0 tensor cores (digit split), 1 double-float SIMT")
    ap.add_argument("--variant", default="rfeast", choices=["feast", "xfeast", "rfeast"])
    ap.add_argument("--no-fp64", dest="fp64", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu", action="store_false")
    ap.add_argument("--no-config1", dest="config1", action="store_false")
    ap.add_argument("--config3", type=int, default=0,
                    help="also run the batched workload with this many problems (64 = full; 0: skip)")
    ap.add_argument("--config5", type=int, default=0,
                    help="also run the largest single problem at this n (32768 = full size; 0: skip)")
    ap.add_argument("--gen", default=WORKLOAD["gen"], choices=["torch_cpu", "torch_cuda", "numpy"],
                    help="generator of the Gaussian whose QR gives Q")
    ap.add_argument("--refine-switch", type=float, default=WORKLOAD["refine_switch"],
                    help="mixed: skip the FP64 refinement of a filter while the previous residual is above this "
                         "and still falling tenfold (0: always refine)")
    ap.add_argument("--cpu-full-n", type=int, default=2048,
                    help="n of the scaled workload the oracle solves in full (0: skip)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
