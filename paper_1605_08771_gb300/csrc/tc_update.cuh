// Tensor-core (tcgen05, split-TF32) trailing update of the complex-FP32 shifted LU.
#pragma once

#include "common.cuh"

namespace feast {

// Column width of the outer blocks whose trailing update runs on the tensor
// cores (K = 2 * kTcBlock real).
constexpr int kTcBlock = 128;

// A complex-FP32 operand block inside a column-major source (per node at
// base + node * node_stride, leading dim ld).  Element (v, k) -- v the
// output row (left operand) or output column (right operand), k the
// reduction index -- is base[(r0 + v) + (c0 + k) ld] when vec_rows, else
// base[(r0 + k) + (c0 + v) ld]; conjugated when conj_t.
struct TcSrc {
  const c64* base;
  int64_t node_stride, ld, r0, c0;
  bool vec_rows, conj_t;
};

// Scratch bytes of the three TF32 operand planes for updates of up to `rows`
// output rows, `cols` output columns, `nodes` shifts and kb <= kTcBlock.
size_t tc_update_planes_bytes(int64_t rows, int64_t cols, int nodes);

// C[c_r0 + i, c_c0 + j] -= sum_k A(i, k) B(k, j), i < R, j < C, k < kb
// (kb <= kTcBlock), for every node (C at Cm + node * cstride, leading dim
// ldc), on the tensor cores (persistent, at most num_sms CTAs).  `planes` is
// scratch of tc_update_planes_bytes(R, C, nodes) bytes or more; a timed-out
// device wait sets *status to DEV_BARRIER_TIMEOUT.
void tc_block_update(const TcSrc& a, const TcSrc& b, int kb, int64_t R, int64_t C, c64* Cm, int64_t ldc,
                     int64_t cstride, int64_t c_r0, int64_t c_c0, int nodes, void* planes, int* status, int num_sms,
                     cudaStream_t s);

// LU trailing update A22 -= L21 U12 for the block of columns [k0, k0 + kb)
// of every node's factor M (column major, leading dimension ld, node stride
// `stride`); planes of tc_update_planes_bytes(n, n, nodes) bytes.
void tc_trailing_update(c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, int64_t k0, int kb, void* planes,
                        int* status, int num_sms, cudaStream_t s);

}  // namespace feast
