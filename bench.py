#!/usr/bin/env python
"""Benchmark of the FEAST interval eigensolver on one GB300.

Workload (the single-large-problem case): complex Hermitian planted matrix
A = Q diag(lambda) Q^H, n = 8192, Q from the QR factorisation of a seeded
complex Gaussian; 200 eigenvalues in I = [-1, 1] of which 30 lie within 1e-4
inside each edge, 60 lie within 1e-4 outside each edge, the rest uniform in
[-50, 50]; n_c = 8 Gauss nodes, m0 = 300, tol 1e-10.  Plain FEAST stalls on it
(more than m0 eigenvalues have |rho| near 1/2), so it runs RFEAST (s = 3), the
paper's residual-expansion variant, in the mixed precision (complex FP32
factorisations and solves, FP64-accurate refinement and Rayleigh-Ritz).

A step is one complete feast_interval_solve (factorisations, filters,
Rayleigh-Ritz, checks) with A resident in HBM.  value = eigenpairs found inside
I (all at residual <= 1e-10) / seconds, summed over ranks.  Also reported:
e2e (same call with A in pinned host memory and the results copied back inside
the timed region), the roofline of the dominant kernel (the double-float GEMM),
the filter-apply rate, the FP64 path on the same input (mixed vs FP64), the CPU
oracle on a bounded sample, clocks and the number of kernel launches.

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
                lmin=-1.0, lmax=1.0, m0=300, n_c=8, tol=1e-10, variant="rfeast", s=3, seed=0)
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



def workload_name(w):
    return (f"complex Hermitian planted n={w['n']}, {w['m_in']} eigenvalues in [-1,1] with "
            f"{w['edge_in']}+{w['edge_in']} within {w['width']:g} inside and {w['edge_out']}+{w['edge_out']} "
            f"within {w['width']:g} outside the edges, bulk in [-{w['bulk']:g},{w['bulk']:g}]; "
            f"n_c={w['n_c']}, m0={w['m0']}, {w['variant'].upper()} s={w['s']}")


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
def oracle_sample(A_host, w, filters, rr_k_sum, rr_k3_sum, budget_s=30.0):
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
        if t_lu > 1.5 or ns >= 2048 or time.time() - t_start > budget_s / 3:
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
    A = planted_matrix_torch(lam, w["seed"], complex_=True, device=device)
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


def run_ours(args, rank, world, dev):
    import torch
    import paper_1605_08771_gb300 as fg

    w = dict(WORKLOAD)
    if args.n:
        scale = args.n / w["n"]
        w.update(n=args.n, m_in=max(4, int(w["m_in"] * scale)), edge_in=max(1, int(w["edge_in"] * scale)),
                 edge_out=max(1, int(w["edge_out"] * scale)), m0=max(8, int(w["m0"] * scale)))
    w["prec"] = args.prec
    w["variant"] = args.variant
    fg.build_library()
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    A_store, lam = build_problem(w, f"cuda:{dev}")
    A = A_store.transpose(0, 1)
    inside = lam[(lam > w["lmin"]) & (lam < w["lmax"])]
    anorm = float(np.max(np.abs(lam)))
    ctx = fg.feast_init(dev, stream)
    opts = fg.feast_opts_default(variant=w["variant"], s=w["s"], prec=w["prec"], anorm=anorm, max_iter=30,
                                 refine_gemm=args.refine_gemm)

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
    ok = all(r["status"] == 0 and r["evals"].size == inside.size and np.max(r["res"]) <= w["tol"]
             and np.max(np.abs(r["evals"] - inside)) <= 1e-10 * anorm for r in results)
    t_max, pairs_all = aggregate_ranks(ms_total, sum(found), world, device=f"cuda:{dev}")
    value = pairs_all / (t_max / 1e3)
    st = results[-1]["stats"]

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
    # dominant kernel of the step (launch list of the solve, profiles/): the
    # complex-FP32 SIMT GEMM of the LU trailing and triangular-solve updates
    cg_launches = max(1, st.cgemm_launches)
    cg_avg_ms = st.cgemm_ms / cg_launches
    cg_flop_per_launch = st.cgemm_flop / cg_launches
    fp32_peak = NUM_SMS * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    cg_achieved = cg_flop_per_launch / (cg_avg_ms / 1e3) / 1e12 if st.cgemm_ms > 0 else 0.0
    cg_traffic = None
    if CGEMM_DRAM_BYTES_PER_FLOP is not None:
        cg_traffic = int(CGEMM_DRAM_BYTES_PER_FLOP * cg_flop_per_launch)
    roofline = {"kernel": "cgemm_prefetch_kernel (complex-FP32 SIMT GEMM)", "bound": "alu",
                "achieved": round(cg_achieved, 3), "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                "frac": round(cg_achieved / fp32_peak, 4), "traffic": cg_traffic,
                "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x max SM clock (unit counts; no measured FP32 peak)",
                "flop_def": "8 real flops per complex multiply-add, M N K per launch",
                "traffic_source": CGEMM_TRAFFIC_SOURCE,
                "launches_per_step": st.cgemm_launches, "avg_launch_ms": round(cg_avg_ms, 4),
                "share_of_step": round(st.cgemm_ms / ms_step, 3)}

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
                           "traffic": None,
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

    # filter-apply rate: algorithmic flops of the solves (8 n^2 m per entry,
    # complex MAC = 8 real flops) per filter application
    n, m0, nc = w["n"], w["m0"], w["n_c"]
    filt_flop = 2 * nc * 8.0 * n * n * m0
    filter_tflops = filt_flop * st.filters / (st.filter_ms / 1e3) / 1e12 if st.filter_ms > 0 else None

    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max / args.steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": ("c64+bf16x21" if args.refine_gemm == 0 else "c64+df32") if w["prec"] != "f64" else "c128",
            "data": "synthetic planted spectrum (seeded), no dataset",
            "config": {"workload": workload_name(w), "n": n, "m0": m0, "n_c": nc, "variant": w["variant"],
                       "s": w["s"], "prec": w["prec"], "tol": w["tol"],
                       "l2": "inputs larger than L2 (A is %.2f GB, L2 129 MB)" % (h2d / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "correct": bool(ok), "eigenpairs_per_step": found[-1], "iterations": results[-1]["iterations"],
            "filters": st.filters, "refine_steps": st.refine_steps,
            "factor_ms": round(st.factor_ms, 1), "filter_ms": round(st.filter_ms, 1),
            "roofline": roofline, "roofline_refine_gemm": roofline_refine,
            "filter_apply": {"tflops": round(filter_tflops, 3) if filter_tflops else None,
                             "flop_per_filter": filt_flop,
                             "note": "solve flops 8 n^2 m0 per entry, 2 n_c entries; refinement excluded"},
            "e2e": {"value": round(e2e_found / e2e_steps / (e2e_ms / 1e3), 4), "unit": UNIT,
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 1)},
            "gpu_launches": int(launches), "clocks": clocks, "peak_source": peak_kind}

    # mixed vs FP64 on the same input (one untimed-by-steps solve, CUDA events)
    if args.fp64 and w["prec"] != "f64":
        o64 = fg.feast_opts_default(variant=w["variant"], s=w["s"], prec="f64", anorm=anorm, max_iter=30)
        barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        r64 = fg.feast_interval_solve(ctx, A, w["lmin"], w["lmax"], m0, nc, w["tol"], o64)
        f1.record(stream)
        barrier()
        t64 = f0.elapsed_time(f1)
        d = None
        if r64["evals"].size == results[-1]["evals"].size:
            d = float(np.max(np.abs(r64["evals"] - results[-1]["evals"])) / anorm)
        line["mixed_vs_fp64"] = {"fp64_ms": round(t64, 1), "mixed_ms": round(ms_step, 1),
                                 "speedup": round(t64 / ms_step, 3),
                                 "fp64_value": round(r64["evals"].size / (t64 / 1e3), 4),
                                 "max_eig_diff_rel_anorm": d, "fp64_iterations": r64["iterations"]}

    # CPU oracle on a bounded sample (rank 0, N = 1 only)
    if args.cpu and world == 1:
        A_host = Ah.numpy().T
        T, ns, ms_, samp = oracle_sample(A_host, w, st.filters, st.rr_k_sum, st.rr_k3_sum)
        line["cpu_baseline"] = {"value": round(inside.size / T, 6), "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": (f"oracle LU of the leading {ns}x{ns} block of z_1 I - A, its solve of "
                                           f"{ms_} right-hand sides and one {ns}x{ms_} Rayleigh-Ritz "
                                           f"({samp:.1f} s of CPU work), scaled by operation counts to the full "
                                           f"solve ({st.filters} filters, {st.rr_passes} Rayleigh-Ritz passes with the run's dimensions): "
                                           f"{T:.0f} s extrapolated"),
                                "extrapolated_s": round(T, 1)}
    fg.feast_finalize(ctx)
    return line


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle, timed on the host cores on
    bounded samples of the same workload (each step one sample)."""
    if rank != 0:
        return None
    from workloads import spectrum_config2
    from workloads import haar_unitary  # noqa: F401  (numpy generator for the host matrix)
    w = dict(WORKLOAD)
    if args.n:
        scale = args.n / w["n"]
        w.update(n=args.n, m0=max(8, int(w["m0"] * scale)))
    lam, a, b = spectrum_config2(w["seed"])
    # the sample needs only a leading block of A: build a planted matrix of the
    # sample's largest block size with the same spectrum distribution
    nb = min(2048, w["n"])
    rng = np.random.default_rng(w["seed"])
    G = rng.standard_normal((nb, nb)) + 1j * rng.standard_normal((nb, nb))
    Qm, _ = np.linalg.qr(G)
    lam_b = np.sort(rng.choice(lam, nb, replace=False))
    A_host = (Qm * lam_b) @ Qm.conj().T
    # the solve's own counts on this seeded workload: 2 rounds, 3 filter
    # applications; Rayleigh-Ritz dimensions m0, 2 m0, 3 m0 in the first round,
    # then m0 growing by the 17 of 300 residual columns that have not converged
    filters, iters = 3, 2
    m0, grow = w["m0"], max(1, round(17 * w["m0"] / 300))
    rr_dims = [m0 * (j + 1) for j in range(w["s"])] + [m0 + grow * j for j in range(w["s"])]
    k_sum, k3_sum = float(sum(rr_dims)), float(sum(k ** 3 for k in rr_dims))
    for _ in range(args.warmup):
        oracle_sample(A_host, w, filters, k_sum, k3_sum, budget_s=10.0)
    Ts, samples = [], []
    t0 = time.time()
    for _ in range(args.steps):
        T, ns, ms_, samp = oracle_sample(A_host, w, filters, k_sum, k3_sum, budget_s=10.0)
        Ts.append(T)
        samples.append(samp)
    wall = time.time() - t0
    value = w["m_in"] / float(np.mean(Ts))
    return {"metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * float(np.mean(Ts)), 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic planted spectrum (seeded)",
            "impl": "reference",
            "config": {"workload": workload_name(w), "n": w["n"], "m0": w["m0"], "n_c": w["n_c"],
                       "variant": w["variant"], "s": w["s"], "prec": "f64 (CPU oracle)", "tol": w["tol"]},
            "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": (f"oracle LU/solve/Rayleigh-Ritz on a leading {ns}x{ns} block, "
                                        f"{float(np.mean(samples)):.1f} s per step, extrapolated by operation "
                                        f"counts to the full solve ({filters} filters, {iters} iterations, Rayleigh-Ritz "
                                        f"dimensions {rr_dims})")},
            "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=0, help="override n (scaled workload, for quick checks)")
    ap.add_argument("--prec", default="mixed", choices=["mixed", "mixed_tc", "f64"])
    ap.add_argument("--refine-gemm", type=int, default=0, choices=[0, 1],
                    help="refinement products: 0 tensor cores (digit split), 1 double-float SIMT")
    ap.add_argument("--variant", default="rfeast", choices=["feast", "xfeast", "rfeast"])
    ap.add_argument("--no-fp64", dest="fp64", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu", action="store_false")
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
