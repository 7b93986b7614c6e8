// Shifted complex LU with partial pivoting, batched over the quadrature nodes,
// and the multi-right-hand-side triangular solves that apply (z_j I - A)^{-1}
// and its adjoint.  F is the factor precision: c128 (FP64 path) or c64 (the
// low-precision factor of the mixed path).
#pragma once

#include "common.cuh"
#include "gemm.cuh"
#include "tc_cgemm.cuh"

namespace feast {

constexpr int kPanel = 32;        // panel width = triangular-solve block size
constexpr int kTcBlock = 128;     // outer block of the two-level LU whose trailing update
                                  // runs on the tensor cores
constexpr int kSolveBlock = 64;   // diagonal blocks of the complex-FP32 triangular solves
constexpr int kSolveOuter = 256;  // outer blocks of the tensor-core triangular solves

// Scratch the cooperative panel kernel needs (device pointers, sized by
// panel_work_bytes()).
struct PanelWork {
  unsigned* counters;   // [nodes] monotone barrier counters
  int* status;          // [1] fatal device status (DeviceStatus)
  int* zero_pivot;      // [nodes] first zero-pivot column + 1, or 0
  double* cand_val;     // [nodes][2][pmax]
  int* cand_idx;        // [nodes][2][pmax]
  void* cand_row;       // [nodes][2][pmax][kPanel] of F
  void* diag_row;       // [nodes][2][kPanel] of F
  int* swap_src;        // [nodes][2*kPanel]
  int* swap_dst;        // [nodes][2*kPanel]
  int* swap_cnt;        // [nodes]
  int* blk_src;         // [nodes][2*kTcBlock] block interchange summary (two-level LU)
  int* blk_dst;
  int* blk_cnt;         // [nodes]
  int pmax;
  void* tc_planes;      // complex-FP32 factors: scratch of the tensor-core trailing update
                        // (lu_tc_planes_bytes); null: SIMT trailing updates
};

// Scratch bytes of the tensor-core trailing update of n x n factors.
size_t lu_tc_planes_bytes(int64_t n, int nodes);

// bf16 planes of complex-FP32 factors for the tensor-core block updates of
// the triangular solves: every 64-column block of each factor (normal
// solves: L below and U above the diagonal block), and, for the adjoint
// solves, every 64-row block conjugated; plus scratch for one block row of
// the right-hand sides.
struct SolvePlanes {
  uint16_t* col = nullptr;   // [node][block][6][npad][64]
  uint16_t* row = nullptr;   // the same of the conjugated row blocks (null: no adjoint solves)
  uint16_t* rhs = nullptr;   // [entry][6][mpad][256]
  int64_t npad = 0, nblk = 0, mpad = 0;
};
size_t solve_planes_bytes(int64_t n, int64_t m, int nodes, int entries, bool adjoint);
SolvePlanes solve_planes_carve(void* base, int64_t n, int64_t m, int nodes, int entries, bool adjoint);
// Split the factors M (n x n, leading dim ld, node stride `stride`) into the
// planes (once per factorisation).
void solve_planes_build(const c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, const SolvePlanes& sp,
                        cudaStream_t s);

size_t panel_work_bytes(int nodes, int pmax, size_t elem_bytes);
PanelWork panel_work_carve(void* base, int nodes, int pmax, size_t elem_bytes);

// M_j = z_j I - A for the `nodes` shifts z (device array of c128), A real
// (double) or complex (c128), column-major with leading dimension lda.
template <typename F, typename TA>
void form_shifted(F* M, int64_t n, int64_t ld, int64_t stride, int nodes,
                  const TA* A, int64_t lda, const c128* z, cudaStream_t s);

// In-place P_j M_j = L_j U_j for every node.  ipiv[j*n + k] is the row swapped
// with row k at step k; perm[j*n + i] the original row now at row i.
template <typename F>
void lu_factor_batched(F* M, int64_t n, int64_t ld, int64_t stride, int nodes,
                       int32_t* ipiv, int32_t* perm, const PanelWork& w,
                       int num_sms, cudaStream_t s);

// Y_e <- (P^T L U)^{-1} Y_e  (adjoint = false) or (P^T L U)^{-H} Y_e
// (adjoint = true) for e = 0..nodes-1, Y_e = Y + e*ystride (n x m, ld n).
// The row permutation is applied by permute_in / permute_out.  Complex-FP32
// factors with planes (solve_planes_build; m <= the planes' m) take the block
// updates of the triangular solves on the tensor cores; otherwise SIMT.  Both
// use 64-row diagonal blocks (32 for complex FP64).
template <typename F>
void lu_solve_batched(const F* M, int64_t n, int64_t ld, int64_t stride, int nodes,
                      F* Y, int64_t m, int64_t ystride, bool adjoint, cudaStream_t s,
                      const SolvePlanes* planes = nullptr, int* status = nullptr, int num_sms = 0);

// Y_e = P B_e (normal) or B_e (adjoint) converted to F;  B_e = B + e*bstride is
// n x m with ld ldb (bstride = 0: one right-hand side block for every node).
template <typename F, typename TB>
void permute_in(F* Y, int64_t ystride, const TB* B, int64_t ldb, int64_t bstride, int64_t n, int64_t m,
                const int32_t* perm, int nodes, bool adjoint, cudaStream_t s);

// Out_e = Y_e (normal) or P^T Y_e (adjoint), converted to TO, optionally
// accumulated (Out_e += ...).
template <typename F, typename TO>
void permute_out(TO* Out, int64_t ostride, const F* Y, int64_t ystride, int64_t n, int64_t m,
                 const int32_t* perm, int nodes, bool adjoint, bool accumulate, cudaStream_t s);

// pinv[e n + perm[e n + i]] = i for every node e.
void invert_perm(const int32_t* perm, int32_t* pinv, int64_t n, int nodes, cudaStream_t s);

// The weighted accumulation of Eq. 3 fused with the output step of the last
// solves: with Z_e = base_e + Yn_e (normal solves, natural row order) and
// Z'_e = base_{nc+e} + P_e^T Ya_e (adjoint solves; P_e^T applied through
// pinv), Xf = sum_e 2 Re(w_e Z_e) for real S, or sum_e w_e Z_e + conj(w_e) Z'_e
// for complex S.  base (complex FP64, E = nc or 2 nc entries of n x m, ld n)
// may be null; Yn, Ya: nc entries of n x m (ld n) of the solve type F; Ya is
// unused for real S.
template <typename S, typename F>
void solve_accumulate(S* Xf, int64_t ldx, const c128* base, const F* Yn, const F* Ya, int64_t n, int64_t m, int nc,
                      const int32_t* pinv, const c128* w, cudaStream_t s);

}  // namespace feast
