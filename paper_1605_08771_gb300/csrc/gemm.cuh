// Batched dense GEMM on CUDA cores for the FP64 and complex-FP32 paths:
//   C_b = alpha * op(A_b) * op(B_b) + beta * C_b,  op in {N, T, C (conjugate transpose)}
// All matrices column-major.  Used for the LU trailing update, the blocked
// triangular-solve updates, the FP64 refinement residual A*Y, and the
// Rayleigh-Ritz / orthonormalisation products.
#pragma once

#include "common.cuh"

namespace feast {

enum Op : int { OP_N = 0, OP_T = 1, OP_C = 2 };

struct GemmArgs {
  int64_t M, N, K;
  const void* A; int64_t lda, strideA; int opA;
  const void* B; int64_t ldb, strideB; int opB;
  void* C; int64_t ldc, strideC;
  c128 alpha, beta;
  int batch;
  // split-K: when ksplit > 1, partial products go to Cpart (ksplit x batch
  // column-major blocks of ldc x N) and gemm_reduce_splitk sums them.
  int ksplit;
  void* Cpart;
};

// Launch C = alpha op(A) op(B) + beta C on `stream`.  TA, TB are the stored
// element types of A and B, TC the type of C (also the accumulation type).
template <typename TA, typename TB, typename TC>
void gemm(const GemmArgs& g, cudaStream_t stream);

// Convenience wrapper for the common unbatched case.
template <typename TA, typename TB, typename TC>
inline void gemm_simple(int64_t M, int64_t N, int64_t K, c128 alpha,
                        const TA* A, int64_t lda, int opA,
                        const TB* B, int64_t ldb, int opB, c128 beta,
                        TC* C, int64_t ldc, cudaStream_t stream,
                        int ksplit = 1, void* Cpart = nullptr) {
  GemmArgs g{};
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.strideA = 0; g.opA = opA;
  g.B = B; g.ldb = ldb; g.strideB = 0; g.opB = opB;
  g.C = C; g.ldc = ldc; g.strideC = 0;
  g.alpha = alpha; g.beta = beta; g.batch = 1;
  g.ksplit = ksplit; g.Cpart = Cpart;
  gemm<TA, TB, TC>(g, stream);
}

inline c128 C1(double re, double im = 0.0) { return c128{re, im}; }

}  // namespace feast

namespace feast {

// FP64-accurate real GEMM on the FP32 pipes ("double-float"):
//   C[(i + j*ldc)*cs + co] = alpha * sum_k A[i,k] B[k,j] + beta * C[...]
// with A and B given as hi/lo float planes (x = hi + lo, |lo| <= 2^-24 |hi|),
// column-major, op N.  Each hi*hi product is made exact with an FMA
// (TwoProd), each addition to the running FP32 sum exact with TwoSum; the
// error terms and the hi*lo cross products go to an FP32 accumulator that is
// flushed into an FP64 accumulator every 32 k-steps.  The error stays within
// 2^-44 of sum |a||b| (the parity tests' bound, K up to 4099), at a small
// fraction of the FP64 cost on sm_103.
// timer_class: the kernel-timer class the launch is recorded under (-1: none).
// ksplit > 1: the reduction is cut into ksplit slices, slice z writing its own
// output block at C + z * czs (to be summed by sum_partials).
void gemm_df32(int64_t M, int64_t N, int64_t K, double alpha,
               const float* Ahi, const float* Alo, int64_t lda,
               const float* Bhi, const float* Blo, int64_t ldb,
               double beta, double* C, int64_t ldc, int cs, int co, cudaStream_t s,
               int timer_class = TIMER_REFINE_GEMM, int ksplit = 1, int64_t czs = 0);

// 3M complex combination: C_re = T1 - T2, C_im = T3 - T1 - T2 where T1 and T3
// already sit in C (re, im) and T2 in a separate real array (n x k, ld n).
void combine_3m(double* C, const double* T2, int64_t n, int64_t k, cudaStream_t s);

// C (M x N, leading dim ldc) = alpha T + beta C.  Real (cplx = false): T is
// M x N with leading dim M.  Complex (C interleaved): T holds the 3M parts
// T1 (real slots) and T3 (imaginary slots) interleaved, T2 real, both with
// leading dim M, and the value is (T1 - T2) + i (T3 - T1 - T2).
void combine_axpby(double* C, int64_t ldc, bool cplx, const double* T, const double* T2, int64_t M, int64_t N,
                   double alpha, double beta, cudaStream_t s);

// hi/lo planes (rows x cols, ld rows) of the transpose of a column-major
// source: plane element (i, j) = src[(j + i*lds)*ss + so] (negated when neg,
// e.g. the imaginary part of a conjugate transpose).
void split_df32_t(const double* src, int64_t rows, int64_t cols, int64_t lds, int ss, int so, bool neg, float* hi,
                  float* lo, cudaStream_t s);

// C (M x N, leading dim ldc; interleaved complex when cplx) = sum of ks
// partial blocks P + z * M * N * (cplx ? 2 : 1), each with leading dim M.
void sum_partials(double* C, int64_t ldc, const double* P, int64_t M, int64_t N, int ks, bool cplx, cudaStream_t s);

// Split FP64 values into hi/lo float planes: src element (i, j) at
// src[(i + j*lds)*ss + so] (so = 2 with ss = 2: the sum Re + Im of a complex
// element); planes are dense rows x cols (ld = rows).
void split_df32(const double* src, int64_t rows, int64_t cols, int64_t lds, int ss, int so,
                float* hi, float* lo, cudaStream_t s);

}  // namespace feast
