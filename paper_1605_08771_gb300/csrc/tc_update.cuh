// Tensor-core (tcgen05, 3xTF32) trailing update of the complex-FP32 shifted LU.
#pragma once

#include "common.cuh"

namespace feast {

// Scratch bytes of the TF32 head/tail operand planes for matrices of order
// up to n and `nodes` shifts.
size_t tc_update_planes_bytes(int64_t n, int nodes);

// A22 -= L21 U12 for the panel [k0, k0 + jb) of every node's factor M (column
// major, leading dimension ld, node stride `stride`), on the tensor cores.
// `planes` is scratch of tc_update_planes_bytes(n, nodes) bytes; a timed-out
// device wait sets *status to DEV_BARRIER_TIMEOUT.
void tc_trailing_update(c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, int64_t k0, int jb, void* planes,
                        int* status, cudaStream_t s);

}  // namespace feast
