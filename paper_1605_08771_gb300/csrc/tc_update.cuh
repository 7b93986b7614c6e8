// Tensor-core (tcgen05, split-TF32) trailing update of the complex-FP32 shifted LU.
#pragma once

#include "common.cuh"

namespace feast {

// Column width of the outer blocks whose trailing update runs on the tensor
// cores (K = 2 * kTcBlock real).
constexpr int kTcBlock = 128;

// Scratch bytes of the three TF32 operand planes for matrices of order
// up to n, `nodes` shifts and blocks of up to kTcBlock columns.
size_t tc_update_planes_bytes(int64_t n, int nodes);

// A22 -= L21 U12 for the block of columns [k0, k0 + kb) (kb <= kTcBlock) of
// every node's factor M (column major, leading dimension ld, node stride
// `stride`), on the tensor cores (persistent, at most num_sms CTAs).
// `planes` is scratch of tc_update_planes_bytes(n, nodes) bytes; a timed-out
// device wait sets *status to DEV_BARRIER_TIMEOUT.
void tc_trailing_update(c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, int64_t k0, int kb, void* planes,
                        int* status, int num_sms, cudaStream_t s);

}  // namespace feast
