// Small dense FP64 kernels around the filter: orthonormalisation (Gram,
// Cholesky, triangular inverse), the Jacobi reduced eigensolver, Ritz
// residual norms, column gathers, the weighted filter accumulation and the
// FP64 refinement residual.  S is the subspace scalar: double (real symmetric
// A) or c128 (complex Hermitian A).
#pragma once

#include "common.cuh"

namespace feast {

struct CoopWork {
  unsigned* counter;   // [1] monotone barrier counter
  int* status;         // [1] fatal status (DeviceStatus)
  int* info;           // [4] kernel-specific outputs (Cholesky column, sweeps, ...)
  double* partial;     // [>= 2*num_sms] partial sums
  unsigned* rotcount;  // [kMaxSweeps] CTAs that rotated in each sweep
  unsigned* roundcount;  // [kMaxSweeps * (kmax + 2)] CTAs that rotated in each round
  void* rot;           // rotation parameters, >= k/2+1 entries of (c, s, e s, e c)
};
constexpr int kMaxSweeps = 64;
size_t coop_work_bytes(int64_t kmax, int num_sms);
CoopWork coop_work_carve(void* base, int64_t kmax, int num_sms);

// H <- (H + H^H)/2 (k x k, ld)
template <typename S> void hermitize(S* H, int64_t k, int64_t ld, cudaStream_t s);

// In-place Cholesky G = R^H R, R in the upper triangle.  Returns through
// w.info[0] the first failing column + 1 (0 = success) after the stream syncs.
template <typename S>
void cholesky_upper(S* G, int64_t k, int64_t ld, const CoopWork& w, int num_sms, cudaStream_t s);

// Rinv = R^{-1} for upper-triangular R (k x k); the strict lower part of Rinv is zeroed.
template <typename S>
void tri_inverse_upper(const S* R, int64_t k, int64_t ld, S* Rinv, int64_t ldi, cudaStream_t s);

// Two-sided Jacobi with round-robin ordering on the Hermitian k x k matrix H
// (overwritten by its near-diagonal form); V receives the eigenvectors
// (unsorted).  Rotations skip |h_pq| <= tol ||H||_F; sweeps stop when a sweep
// rotates nothing or after max_sweeps.  Sweeps counted in w.info[1].  S may be
// double, c128 or, for a low-precision first phase, float / c64.  init_v =
// false continues from the current H and V (V not reset to the identity).
template <typename S>
void jacobi_eigh(S* H, int64_t k, int64_t ld, S* V, int64_t ldv, double tol, const CoopWork& w,
                 int num_sms, cudaStream_t s, int max_sweeps = kMaxSweeps, bool init_v = true);

// The same sweeps with H and V held as double-float values and every
// rotation applied on the FP32 pipes (converted in place from and back to
// FP64; S = double or c128); the diagonal is kept and updated in FP64 in dg
// (k doubles of scratch), so the eigenvalues keep FP64 accuracy while the
// off-diagonal entries and the vectors carry about 48 bits.
template <typename S>
void jacobi_eigh_df(S* H, int64_t k, int64_t ld, S* V, int64_t ldv, double* dg, double tol, const CoopWork& w,
                    int num_sms, cudaStream_t s, int max_sweeps = kMaxSweeps, bool init_v = true);
// Cluster finish of the FP64 Jacobi.  offdiag_scan lists the pairs i < j with
// |h_ij| > thr (absolute): *cnt (device) receives their number, list the
// first cap of them as (i, j).  cluster_jacobi diagonalises, for each of the
// nsets index sets idx[off[c] .. off[c+1]) (ascending, 2 .. kClusterMax
// entries, disjoint), the submatrix H[set, set] in place by cyclic Jacobi to
// the same threshold, and applies its unitary to V[:, set] (V: k x k, ld
// ldv).  Entries of H between a set and the rest are left as they are: they
// were at most thr when the sets were formed, and the set's rotation could
// make the true ones (not stored) up to sqrt(set size) times larger.  Scratch
// Ubuf: nsets kClusterMax^2 elements; sweeps_out: nsets ints (sweeps taken).
constexpr int kClusterMax = 64;
template <typename S>
void offdiag_scan(const S* H, int64_t k, int64_t ld, double thr, int* cnt, int* list, int cap, cudaStream_t s);
template <typename S>
void cluster_jacobi(S* H, int64_t k, int64_t ld, S* V, int64_t ldv, const int* idx, const int* off, int nsets,
                    double thr, S* Ubuf, int* sweeps_out, cudaStream_t s);

// Low-precision block Jacobi (F = float / c64) on the Hermitian k x k matrix
// H (FP64, ld k, not modified): block-pair rounds, each pair's 32 x 32
// subproblem diagonalised in shared memory, the unitaries applied to the whole
// working copy.  Rotations skip |h_pq| <= thr (absolute).  V (k x k, ld k)
// receives the accumulated eigenvectors; returns the sweeps taken (at most
// max_sweeps; the last one rotated nothing unless the limit was reached).
// Scratch: HP, VP of block_jacobi_pad(k)^2 elements, Ubuf of
// block_jacobi_u_bytes(k) bytes, d_rot one int.  Synchronises the stream once
// per sweep.
int64_t block_jacobi_pad(int64_t k);
size_t block_jacobi_u_bytes(int64_t kmax);
template <typename F, typename S>
int block_jacobi(const S* H, int64_t k, F* V, double thr, F* HP, F* VP, F* Ubuf, int* d_rot, int max_sweeps,
                 cudaStream_t s);

// dst (n x m, ld ldd) = src converted elementwise (FP64 <-> FP32, complex too)
template <typename To, typename From>
void convert_matrix(To* dst, int64_t ldd, const From* src, int64_t lds, int64_t n, int64_t m, cudaStream_t s);

// diag[i] = Re H[i,i]
template <typename S> void get_diag(const S* H, int64_t k, int64_t ld, double* diag, cudaStream_t s);

// out[j] = || X[:, j] ||_2^2
template <typename S> void col_norms2(const S* X, int64_t n, int64_t k, int64_t ld, double* out, cudaStream_t s);

// out[j] = || AX[:, j] - lam[j] X[:, j] ||_2^2
template <typename S>
void resid_norms2(const S* AX, const S* X, int64_t n, int64_t k, int64_t ld, const double* lam, double* out,
                  cudaStream_t s);

// out[j] = Re( X[:, j]^H Y[:, j] )
template <typename S>
void col_dots_re(const S* X, const S* Y, int64_t n, int64_t k, int64_t ld, double* out, cudaStream_t s);

// R[:, j] = AX[:, j] - lam[j] X[:, j]
template <typename S>
void ritz_residual(S* R, const S* AX, const S* X, int64_t n, int64_t k, int64_t ld, const double* lam, cudaStream_t s);

// dst[:, j] = src[:, idx[j]] * (scale ? scale[j] : 1)
template <typename S>
void gather_cols(S* dst, int64_t lddst, const S* src, int64_t ldsrc, int64_t n, const int* idx, int64_t k,
                 const double* scale, cudaStream_t s);

// dst (ks x ks, ld ks) = src[idx, idx] (ld lds); scatter_sub the reverse
template <typename S> void gather_sub(S* dst, const S* src, int64_t lds, const int* idx, int64_t ks, cudaStream_t s);
template <typename S> void scatter_sub(S* dst, int64_t ldd, const S* src, const int* idx, int64_t ks, cudaStream_t s);
// dst[:, idx[j]] = src[:, j] (n rows, k columns)
template <typename S>
void scatter_cols(S* dst, int64_t lddst, const S* src, int64_t ldsrc, int64_t n, const int* idx, int64_t k,
                  cudaStream_t s);
// X[:, j] *= scale[j]
template <typename S> void scale_cols(S* X, int64_t n, int64_t k, int64_t ld, const double* scale, cudaStream_t s);

// Xf = sum_e Re/complex weights:  real A: Xf = sum_j 2 Re(w_j Y_j);
// complex Hermitian: Xf = sum_j w_j Y_j + conj(w_j) Yadj_j.  Y holds the
// normal entries then (complex case) the adjoint entries, each n x m.
template <typename S>
void accumulate_filter(S* Xf, int64_t ld, const c128* Y, int64_t n, int64_t m, int nodes, const c128* w,
                       cudaStream_t s);

// R_e = X - z_e Y_e + AY_e for every entry e with active[e] != 0 (complex
// FP64); R_e = 0 for the others.
template <typename S>
void refine_residual(c128* R, const S* X, int64_t ldx, const c128* Y, const c128* AY, int64_t n, int64_t m,
                     int entries, const c128* z_e, const int* active, cudaStream_t s);


// ||R_e||_F^2 and ||Y_e||_F^2 per entry (out[2e], out[2e+1])
void entry_norms2(const c128* R, const c128* Y, int64_t n, int64_t m, int entries, double* out, cudaStream_t s);

// X0 = seeded N(0,1) (complex: independent N(0,1/2) parts), counter-based
template <typename S> void random_normal(S* X, int64_t n, int64_t m, int64_t ld, unsigned long long seed,
                                         cudaStream_t s);

// y = A x (FP64, A real or complex Hermitian) for the power-iteration norm estimate
template <typename S> void copy_matrix(S* dst, int64_t ldd, const S* src, int64_t lds, int64_t n, int64_t m,
                                       cudaStream_t s);
template <typename S> void set_identity(S* X, int64_t k, int64_t ld, cudaStream_t s);
// X = diag(d) (k x k)
template <typename S> void set_diag(S* X, int64_t k, int64_t ld, const double* d, cudaStream_t s);

// any non-finite entry in the n x m matrix -> *flag = 1
template <typename S> void check_finite(const S* X, int64_t n, int64_t m, int64_t ld, int* flag, cudaStream_t s);

}  // namespace feast
