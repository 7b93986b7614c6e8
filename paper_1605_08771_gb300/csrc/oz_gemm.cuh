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

// C[(i + j ldc) cs + co] = sum_k A(i,k) B(k,j) for i < M, j < N from split
// operands (A: M vectors = rows, B: N vectors = columns, same K).  Error about
// 2^-47 sum_k 2^(eA_i + eB_j) per element.  A timed-out device wait sets
// *status to DEV_BARRIER_TIMEOUT (the output is then undefined).
void oz_gemm(int64_t M, int64_t N, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc, int cs, int co,
             int* status, int num_sms, cudaStream_t s);

}  // namespace feast
