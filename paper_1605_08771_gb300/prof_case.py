"""Small, self-contained cases of the library for profiler captures.

  python -m paper_1605_08771_gb300.prof_case --what filter --n 4096 --m 150
      one mixed-precision filter application rho(A) X (shifted LU of the 8
      nodes, complex-FP32 solves, FP64-accurate refinement) on the
      edge-cluster complex Hermitian workload scaled to n;
  python -m paper_1605_08771_gb300.prof_case --what solve --n 2048
      one complete mixed RFEAST solve of that workload.
The inputs come from the seeded planted-spectrum generator; nothing is timed
here (capture with a profiler, or set FEAST_PROFILE=1 for phase times).
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--what", default="filter", choices=["filter", "solve"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--prec", default="mixed")
    ap.add_argument("--refine-gemm", type=int, default=0, help="0 tensor cores (digit split), 1 double-float")
    args = ap.parse_args()
    import torch

    import paper_1605_08771_gb300 as fg
    from workloads import spectrum_config2
    from workloads.planted import planted_matrix_torch

    n = args.n
    sc = n / 8192
    lam, a, b = spectrum_config2(0, n=n, m_in=max(4, int(200 * sc)), edge_in=max(1, int(30 * sc)),
                                 edge_out=max(1, int(60 * sc)))
    A = planted_matrix_torch(lam, 0, True)
    anorm = float(np.max(np.abs(lam)))
    m = args.m or max(8, int(300 * sc))
    fg.build_library()
    with fg.Feast(0) as f:
        if args.what == "filter":
            g = torch.Generator(device="cuda:0")
            g.manual_seed(3)
            X = torch.randn((n, m), generator=g, dtype=torch.complex128, device="cuda:0")
            f.filter(A, a, b, 8, X, prec=args.prec, anorm=anorm, refine_gemm=args.refine_gemm)
        else:
            out = f.solve(A, a, b, m, 8, 1e-10, variant="rfeast", prec=args.prec, anorm=anorm,
                          refine_gemm=args.refine_gemm, rfeast_expand=1, response_stop=1)
            print("status", out["status"], "pairs", out["evals"].size, "iterations", out["iterations"])
            st = out["stats"]
            print("cgemm launches %d flop %.6e ms %.3f; tensor-core cgemm launches %d flop %.6e ms %.3f; "
                  "refine gemm launches %d mac %.6e ms %.3f"
                  % (st.cgemm_launches, st.cgemm_flop, st.cgemm_ms, st.tcgemm_launches, st.tcgemm_flop,
                     st.tcgemm_ms, st.refine_gemm_launches, st.refine_gemm_mac, st.refine_gemm_ms))
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
