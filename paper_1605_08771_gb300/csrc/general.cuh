// FEAST for a general (non-Hermitian) complex matrix: the kernels that the
// Hermitian path has no counterpart for.  The filter runs over the whole
// circle |z - c| = r (2 n_c shifted factorisations, no Hermitian mirror), and
// the reduced matrix Q^H A Q of the Rayleigh-Ritz step is a general k x k
// matrix, diagonalised here by Hessenberg reduction and shifted QR to Schur
// form (Golub & Van Loan, Matrix Computations, Sects. 7.4-7.5) followed by
// back substitution for the eigenvectors of the triangular factor.
#pragma once
#include "common.cuh"

namespace feast {

constexpr int kSchurMaxK = 2048;  // largest reduced dimension (one CTA, v in shared memory)

// Schur form of the complex k x k matrix H (column-major, ld k): H is
// overwritten by the upper-triangular T and Z (k x k, ld k) receives the
// unitary Schur vectors, H_in = Z T Z^H.  One CTA.  info[0]: 0 converged,
// 1 no convergence within 30 k QR sweeps, 2 the kernel's wall-clock limit
// (20 s) expired; info[1]: QR sweeps taken.
void schur_complex(c128* H, c128* Z, int k, int* info, cudaStream_t s);

// Eigenvectors of the upper-triangular T (k x k, ld k): column q of Y has
// Y[q, q] = 1, zeros below, and (T - T[q,q] I) y = 0 by back substitution;
// divisors smaller than `small` in modulus are replaced by `small`.
void triangular_eigvecs(const c128* T, c128* Y, int k, double small, cudaStream_t s);

// Y = sum_e w[e] W_e over `entries` blocks of nm elements (W_e = W + e nm).
void weighted_sum(c128* Y, const c128* W, int64_t nm, int entries, const c128* w, cudaStream_t s);

// out[j] = || AX[:, j] - lam[j] X[:, j] ||_2^2 with complex lam (n x k, ld n)
void resid_norms2_complex(const c128* AX, const c128* X, int64_t n, int64_t k, const c128* lam, double* out,
                          cudaStream_t s);

// *out = ||H||_F (k x k, ld k), one CTA
void frobenius_norm(const c128* H, int64_t k, double* out, cudaStream_t s);

}  // namespace feast
