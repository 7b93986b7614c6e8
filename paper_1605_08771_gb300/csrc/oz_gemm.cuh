// FP64-accurate real GEMM on the bf16 tensor cores by error-free digit
// splitting (Ozaki scheme), used for the residual products A Y of the
// mixed-precision refinement.
#pragma once

#include "common.cuh"

namespace feast {

constexpr int kOzDigits = 6;      // 8-bit digits per operand element (48 bits)
constexpr int kOzTileM = 128;     // output rows per tile (TMEM lanes)
constexpr int kOzTileN = 96;      // output columns per tile
constexpr int kOzTileK = 32;      // K granularity of the planes

// Padded sizes of an operand of nvec vectors of length K.
inline int64_t oz_kpad(int64_t K) { return cdiv(K, kOzTileK) * kOzTileK; }
inline int64_t oz_vpad(int64_t nvec, bool left) {
  const int64_t t = left ? kOzTileM : kOzTileN;
  return cdiv(nvec, t) * t;
}
// Bytes of one split operand (digit planes + per-vector exponents).
inline size_t oz_operand_bytes(int64_t nvec, int64_t K, bool left) {
  const int64_t vp = oz_vpad(nvec, left);
  return (size_t)kOzDigits * vp * oz_kpad(K) * 2 + ((size_t)vp * 4 + 255) / 256 * 256;
}

// One operand split into digit planes: vector v (a row of the left operand or
// a column of the right one) is x_v = 2^(e_v - 8) sum_p plane_p[v], where
// plane_p holds d_p 2^(-8p) in bf16 with integer digits |d_0| <= 256,
// |d_p| <= 128.  planes: kOzDigits planes of vpad x kpad bf16 (K contiguous),
// exps: vpad ints; both inside one buffer of oz_operand_bytes.
struct OzOperand {
  uint16_t* planes;
  int* exps;
  int64_t nvec, vpad, K, kpad;
};
OzOperand oz_operand(void* buf, int64_t nvec, int64_t K, bool left);

// Split nvec vectors of length K into `op`.  Element k of vector v is taken
// from src at complex/real index (k * se + v * sv) (ss = 1: real doubles,
// ss = 2: interleaved complex), combined per `mode`: 0 re, 1 im, 2 re + im,
// 3 -im, 4 re - im (modes 1-4 need ss = 2).
void oz_split(const double* src, int ss, int mode, int64_t K, int64_t se, int64_t sv, const OzOperand& op,
              cudaStream_t s);
// The same for nm <= 3 modes of the same elements in one pass (modes[t] into
// ops[t]; the operands must have the same shape).
void oz_split_modes(const double* src, int ss, const int* modes, int nm, int64_t K, int64_t se, int64_t sv,
                    const OzOperand* ops, cudaStream_t s);

// C[(i + j ldc) cs + co] = sum_k A(i,k) B(k,j) for i < M, j < N from split
// operands (A: M vectors = rows, B: N vectors = columns, same K).  Error about
// 2^-47 sum_k 2^(eA_i + eB_j) per element.  A timed-out device wait sets
// *status to DEV_BARRIER_TIMEOUT (the output is then undefined).
void oz_gemm(int64_t M, int64_t N, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc, int cs, int co,
             int* status, int num_sms, cudaStream_t s);

// General FP64-accurate product C = alpha op(A) op(B) + beta C (alpha, beta
// real) from column-major A, B, C: real (cplx = false) or interleaved complex
// (three real products, 3M: T1 = Ar Br, T2 = Ai Bi, T3 = (Ar + Ai)(Br + Bi),
// Re = T1 - T2, Im = T3 - T1 - T2).  op(A) is A (transA = false, M x K,
// leading dim lda) or its conjugate transpose (A is K x M); the same for B
// (K x N, or N x K when transB).  Scratch: L[0..2] and R[0..2] of
// oz_operand_bytes(M, K, true) / oz_operand_bytes(N, K, false) bytes (one of
// each for real), T of (cplx ? 2 : 1) M N doubles, T2 of M N doubles
// (complex only).
struct OzScratch {
  void* L[3];
  void* R[3];
  double* T;
  double* T2;
};
void oz_gemm_op(bool cplx, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, bool transA,
                const double* B, int64_t ldb, bool transB, double beta, double* C, int64_t ldc, const OzScratch& w,
                int* status, int num_sms, cudaStream_t s);

}  // namespace feast
