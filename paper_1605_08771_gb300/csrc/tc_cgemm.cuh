// Tensor-core (tcgen05) complex-FP32 block update C -= A B for the shifted
// LU and the triangular solves of the mixed precision, with FP32-exact
// operands: every FP32 value is split into three bf16 parts.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace feast {

constexpr int kCgTileM = 128;   // output rows per tile
constexpr int kCgTileN = 128;   // output columns per tile
constexpr int kCgChunk = 32;    // k per pipeline stage (64 bytes of bf16)
constexpr int kCgPlanes = 6;    // Re hi, mid, lo; Im hi, mid, lo

// Planes of one operand, K-major bf16: element (v, k) of plane p of slab b of
// node e sits at row base_row + e node_rows + b slab_rows + p plane_rows + v,
// column k - b kslab, of a row-major array of `kdim` bf16 per row and
// total_rows rows.  A slab holds kslab consecutive k (a single slab holds all
// of K); v is the output row (left operand) or output column (right operand).
struct CgOperand {
  const uint16_t* planes;
  int64_t total_rows, kdim;
  int64_t node_rows, slab_rows, plane_rows, base_row;
  int kslab;
  int base_x = 0;   // first k column of the operand inside a slab (a multiple of 32)
};

// x = p0 + p1 + p2 exactly: p0 = bf16(x), p1 = bf16(x - p0), p2 = x - p0 - p1
// (both subtractions exact in FP32; 3 x 8 significant bits cover FP32's 24)
__device__ __forceinline__ void cg_split3(float x, uint16_t& p0, uint16_t& p1, uint16_t& p2) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r1 = __fsub_rn(x, __bfloat162float(h));
  const __nv_bfloat16 m = __float2bfloat16_rn(r1);
  const float r2 = __fsub_rn(r1, __bfloat162float(m));
  const __nv_bfloat16 l = __float2bfloat16_rn(r2);
  p0 = __bfloat16_as_ushort(h);
  p1 = __bfloat16_as_ushort(m);
  p2 = __bfloat16_as_ushort(l);
}

// bf16 elements of the planes of `slabs` slabs of vpad x kdim for `nodes`
// nodes.
inline size_t cg_planes_elems(int64_t vpad, int64_t kdim, int64_t slabs, int nodes) {
  return (size_t)nodes * (size_t)slabs * kCgPlanes * (size_t)vpad * (size_t)kdim;
}
inline int64_t cg_vpad(int64_t v) { return cdiv(v, kCgTileM) * kCgTileM; }
inline int64_t cg_kpad(int64_t k) { return cdiv(k, kCgChunk) * kCgChunk; }

// Split complex-FP32 blocks into the six bf16 planes, for `nodes` nodes and
// `slabs` slabs each.  Source element (v, k) of slab b of node e is
//   vec_rows:  src[e node_stride + b slab_src + (r0 + v) + (c0 + k) ld]
//   otherwise: src[e node_stride + b slab_src + (r0 + k) + (c0 + v) ld]
// conjugated when conj_src; v < V, k < min(kslab, K - b kslab).  Out: plane p
// of slab b of node e at out + ((e slabs + b) 6 + p) vpad kdim, row v, column
// k; rows V..vpad and columns past the slab's K are zero.
void cg_split(const c64* src, int64_t node_stride, int64_t slab_src, int64_t ld, int64_t r0, int64_t c0,
              bool vec_rows, bool conj_src, int64_t V, int64_t K, int kslab, int64_t slabs, int64_t vpad,
              int64_t kdim, int nodes, uint16_t* out, cudaStream_t s);

// C_e[i, j] -= sum_k A_e(i, k) B_e(k, j) for i < R, j < N, k < K (the planes
// of at least one operand are zero from K to the next multiple of 32),
// every node e < nodes (C_e = C + e cstride, column major, leading dim ldc),
// on the tensor cores: the 6 x 6 split products of each real product whose
// parts sum to at least 2^-18 of it (hi hi, hi mid, mid hi, hi lo, mid mid,
// lo hi), FP32 accumulation in tensor memory.  A timed-out device wait sets
// *status to DEV_BARRIER_TIMEOUT.
void cg_update(const CgOperand& A, const CgOperand& B, int64_t K, int64_t R, int64_t N, c64* C, int64_t ldc,
               int64_t cstride, int nodes, int* status, int num_sms, cudaStream_t s);

// The operand descriptor of planes written by cg_split with one slab per node.
inline CgOperand cg_operand(const uint16_t* planes, int64_t vpad, int64_t kdim, int nodes, int64_t slabs = 1,
                            int kslab = 0) {
  CgOperand o;
  o.planes = planes;
  o.kdim = kdim;
  o.plane_rows = vpad;
  o.slab_rows = kCgPlanes * vpad;
  o.node_rows = slabs * o.slab_rows;
  o.total_rows = nodes * o.node_rows;
  o.base_row = 0;
  o.kslab = kslab > 0 ? kslab : (int)kdim;
  return o;
}

}  // namespace feast
