/*
 * FEAST interval eigensolver for dense Hermitian / real symmetric matrices on
 * one NVIDIA GB300 (sm_103a).  C ABI: plain pointers and sizes only.
 *
 * Method (Gavin & Polizzi, "Enhancing the Performance and Robustness of the
 * FEAST Eigensolver", arXiv 1605.08771):
 *   - the spectral projector rho(A) = (1/2 pi i) \oint (zI - A)^{-1} dz
 *     (Sect. I, Eq. 2) applied to a subspace X by Gauss quadrature,
 *     rho(A) X ~ sum_j w_j (z_j I - A)^{-1} X (Eq. 3), one shifted LU and
 *     multi-right-hand-side solve per node;
 *   - subspace iteration with Rayleigh-Ritz (Appendix, FEAST Algorithm);
 *   - the two robustness variants: XFEAST, expanding the subspace with the
 *     previous filtered blocks (Sect. II-A, XFEAST Algorithm), and RFEAST,
 *     expanding it with Ritz residual vectors (Sect. II-B, RFEAST Algorithm).
 *
 * Conventions shared by every entry point:
 *   - matrices are column-major; complex data is interleaved (re, im) double
 *     precision, layout-compatible with C99 `double complex`;
 *   - pointers documented "device" must be device memory of the context's
 *     GPU, owned by the caller; pointers documented "host" are host memory;
 *   - every call is stream-ordered on the context's stream and returns only
 *     after its results are complete (it synchronises that stream);
 *   - return value: 0 success, > 0 warning, < 0 error (feast_strerror).
 *     On error the output buffers hold unspecified values.
 *   - the contour is the ellipse with centre (lmin+lmax)/2, horizontal
 *     semi-axis r = (lmax-lmin)/2 and vertical semi-axis aspect*r; n_c Gauss-
 *     Legendre nodes are placed on its upper half and the lower half is their
 *     mirror image, so n_c is also the number of shifted factorisations.
 */
#ifndef FEAST_GB300_H
#define FEAST_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct feast_ctx feast_ctx;

/* element type of A, X and eigenvectors */
enum { FEAST_R64 = 0, /* real symmetric, double */
       FEAST_C128 = 1 /* complex Hermitian, interleaved double complex */ };

/* iteration variant */
enum { FEAST_PLAIN = 0,  /* FEAST Algorithm (Appendix) */
       FEAST_XFEAST = 1, /* expanding subspace from previous filtered blocks (Sect. II-A) */
       FEAST_RFEAST = 2  /* expanding subspace with Ritz residuals (Sect. II-B) */ };

/* arithmetic of the shifted factorisations and solves */
enum { FEAST_PREC_F64 = 0,        /* complex FP64 LU and solves */
       FEAST_PREC_MIXED = 1,      /* complex FP32 LU and solves, FP64 iterative refinement; the
                                     GEMM updates of the LU and of the triangular solves on the
                                     bf16 tensor cores with FP32-exact operands (three-part bf16
                                     split, six split products, FP32 accumulate); the
                                     Rayleigh-Ritz products and the reduced eigensolver's polish
                                     in double-float arithmetic on the FP32 pipes (the polish's
                                     diagonal in FP64) */
       FEAST_PREC_MIXED_SIMT = 2  /* as FEAST_PREC_MIXED with those GEMM updates on the FP32
                                     SIMT pipes */ };

/* status codes */
#define FEAST_OK 0
#define FEAST_WARN_MAXITER 1        /* max_iter reached: best-effort pairs returned */
#define FEAST_ERR_ARG (-1)          /* invalid argument */
#define FEAST_ERR_NONFINITE (-2)    /* NaN or Inf in A or X */
#define FEAST_ERR_SINGULAR (-3)     /* exactly singular shifted matrix */
#define FEAST_ERR_ORTH (-4)         /* subspace could not be orthonormalised */
#define FEAST_ERR_M0 (-5)           /* every Ritz value inside I: m0 too small */
#define FEAST_ERR_CUDA (-6)         /* CUDA runtime error */
#define FEAST_ERR_NOMEM (-7)        /* device allocation failed */
#define FEAST_ERR_TIMEOUT (-8)      /* a bounded device wait gave up */

typedef struct {
  int variant;          /* FEAST_PLAIN (default), FEAST_XFEAST, FEAST_RFEAST */
  int s;                /* XFEAST window blocks / RFEAST Rayleigh-Ritz passes (default 3) */
  int prec;             /* FEAST_PREC_F64 (default), FEAST_PREC_MIXED or FEAST_PREC_MIXED_SIMT */
  int max_iter;         /* maximum outer iterations (default 100) */
  int refine_max;       /* mixed: maximum refinement steps per filter (default 10) */
  int refine_gemm;      /* mixed: the FP64-accurate products A Y of the refinement on the
                           tensor cores (0, default: bf16 digit split, Ozaki scheme) or
                           in double-float arithmetic on the FP32 pipes (1) */
  double aspect;        /* ellipse vertical / horizontal semi-axis (default 1: circle) */
  double anorm;         /* ||A||_2 when > 0; otherwise 40 power iterations estimate it */
  double refine_tol;    /* mixed: stop when ||R||_F <= refine_tol (||A|| + |z|) ||Y||_F;
                           0 = 16 eps sqrt(n) */
  unsigned long long seed; /* seed of the N(0,1) starting subspace when x0 == NULL */
  const void* x0;       /* optional device n x m0 starting subspace (leading dim n, dtype) */
  double refine_switch; /* mixed: while the previous iteration's max residual exceeds this and
                           fell at least tenfold, the next filter uses the FP32 solves without
                           FP64 refinement (default 0: always refine) */
  int rfeast_expand;    /* RFEAST step 2(iii) (Appendix, RFEAST Algorithm): 0 (default, the
                           paper) appends the residual R = A X - X Lambda of every selected
                           pair; 1 appends only those of selected pairs whose relative residual
                           is still above tol and ends the passes once none is (a converged
                           pair's residual is rounding noise whose direction adds spurious
                           Ritz pairs, Sect. II-B) */
  int response_stop;    /* 0 (default, the paper) stops on the step-3 check alone; 1 also stops
                           when every (selected) pair inside I whose filter response
                           Re(x^H rho(A) x) exceeds 1/2 has converged (rho > 1/2 exactly
                           inside I for the circle contour), returning those pairs: on spectra
                           with eigenvalues on both sides of I, mixtures of outside
                           eigenvectors give in-I Ritz values that never converge.  All three
                           variants (plain FEAST: the m0 - m outside directions of its
                           subspace are the ones that mix) */
  int reserved;
  const double* node_offsets; /* optional host array of n_c node offsets delta_j (NULL: the
                           Gauss-Legendre rule): the abscissae become
                           t_j' = tanh(atanh(t_j) + delta_j), which must stay strictly
                           increasing, and the weights those of the interpolatory rule on
                           them (exact for polynomials of degree < n_c); delta = 0 is the
                           Gauss rule (a placement the learned proposer may choose) */
} feast_opts;

/* Per-call statistics of the last feast_interval_solve on a context. */
typedef struct {
  int iterations;       /* outer iterations (Rayleigh-Ritz / check rounds) */
  int filters;          /* applications of rho(A): each solves n_c*m0 right-hand sides
                           per half-contour */
  int refine_steps;     /* mixed: total refinement steps */
  int m_expected;       /* XFEAST/RFEAST: count used by the stopping test */
  double factor_ms;     /* time of the shifted factorisations */
  double filter_ms;     /* total time of the filter applications */
  double total_ms;      /* whole solve */
  double max_residual;  /* max relative residual of the returned pairs */
  double history[128];  /* max residual per iteration (first 128) */
  double refine_gemm_ms;    /* mixed: summed device time (CUDA events) of the FP64-accurate
                               refinement GEMM launches */
  double refine_gemm_mac;   /* their real multiply-adds (M*N*K summed over launches) */
  int refine_gemm_launches; /* their number */
  int cgemm_launches;   /* mixed: launches of the complex-FP32 SIMT GEMM (LU trailing and
                           triangular-solve block updates) */
  double cgemm_ms;      /* their summed device time (CUDA events) */
  double cgemm_flop;    /* their real flops (8 per complex multiply-add) */
  int tcgemm_launches;  /* mixed: launches of the tensor-core complex-FP32 GEMM (the same
                           updates on the tensor cores) */
  double tcgemm_ms;     /* their summed device time (CUDA events) */
  double tcgemm_flop;   /* their real flops (8 per complex multiply-add) */
  int rr_passes;        /* Rayleigh-Ritz passes (reduced eigenproblems solved) */
  double rr_k_sum;      /* sum of their dimensions k */
  double rr_k3_sum;     /* sum of k^3 */
} feast_stats;

void feast_opts_default(feast_opts* opts);

/* Create a context on CUDA device `device`; `stream` is a cudaStream_t (NULL
 * = the legacy default stream).  The context owns its workspace (device
 * memory that grows to the largest problem seen).  Returns FEAST_OK,
 * FEAST_ERR_ARG or FEAST_ERR_CUDA. */
int feast_init(feast_ctx** ctx, int device, void* stream);
/* Release the context and its workspace. */
int feast_finalize(feast_ctx* ctx);
const char* feast_strerror(int code);

/* Number of CUDA kernels this library has launched in this process so far
 * (all contexts).  The difference across a call is its launch count. */
uint64_t feast_kernel_launches(void);

/* Contour nodes z_j and weights w_j of the upper half-contour (Eq. 3 with the
 * circle/ellipse reading above): z and w receive n_c complex values each
 * (host, 2*n_c doubles, interleaved).  Node j uses the j-th Gauss-Legendre
 * abscissa t_j in ascending order, theta_j = (pi/2)(1 - t_j),
 * z_j = c + r cos(theta_j) + i aspect r sin(theta_j),
 * w_j = (omega_j/4)(aspect r cos(theta_j) + i r sin(theta_j)). */
int feast_contour_nodes(double lmin, double lmax, int n_c, double aspect, double* z, double* w);

/* feast_contour_nodes with moved nodes: offsets (host, n_c doubles) as
 * feast_opts.node_offsets describes (NULL = Gauss).  Returns FEAST_ERR_ARG
 * when the moved abscissae are not strictly increasing inside (-1, 1). */
int feast_contour_nodes_offset(double lmin, double lmax, int n_c, double aspect, const double* offsets, double* z,
                               double* w);

/* Eigenpairs of the Hermitian n x n matrix A (device, leading dim lda >= n,
 * dtype FEAST_R64 or FEAST_C128, not modified) with eigenvalues in the open
 * interval (lmin, lmax).  m0 is the subspace size (more than the expected
 * count, at most n), n_c the number of upper-half quadrature nodes, tol the
 * stopping tolerance on max_k ||A x_k - lambda_k x_k|| / ||A||_2 over the
 * returned pairs (Appendix step 3).  Outputs: evals (host, >= m0 doubles,
 * ascending), evecs (device, n x m0, leading dim n, dtype; unit 2-norm
 * columns), res (host, >= m0 doubles, relative residuals), *m_found pairs,
 * *iterations outer iterations.  Only the first *m_found values/columns are
 * meaningful.  stats may be NULL.  Returns FEAST_OK, FEAST_WARN_MAXITER or an
 * error. */
int feast_interval_solve(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda,
                         double lmin, double lmax, int m0, int n_c, double tol,
                         const feast_opts* opts, double* evals, void* evecs, double* res,
                         int* m_found, int* iterations, feast_stats* stats);

/* The generalized problem A x = lambda B x with A Hermitian and B Hermitian
 * positive definite (the extension of FEAST to A x = lambda B x, Sect. I):
 * eigenpairs with lambda in (lmin, lmax).  B = R^H R (Cholesky) reduces it
 * to the standard problem C y = lambda y with C = R^{-H} A R^{-1}, which
 * feast_interval_solve solves (same options; opts.anorm is ignored, ||C|| is
 * estimated; opts.x0 must be NULL); the eigenvectors x = R^{-1} y are
 * returned B-orthonormal (x^H B x = 1).  B: device n x n, leading dim ldb,
 * dtype of A, not modified.  res: relative residuals of the reduced
 * problem, ||C y - lambda y|| / ||C||_2 = ||R^{-H}(A x - lambda B x)|| /
 * ||C||_2.  n * element size <= 200 KB (the Cholesky kernel keeps a column in
 * shared memory).  Returns FEAST_ERR_ARG when B is not numerically positive
 * definite; otherwise as feast_interval_solve. */
int feast_interval_solve_gen(feast_ctx* ctx, const void* A, const void* B, int dtype, int64_t n, int64_t lda,
                             int64_t ldb, double lmin, double lmax, int m0, int n_c, double tol,
                             const feast_opts* opts, double* evals, void* evecs, double* res, int* m_found,
                             int* iterations, feast_stats* stats);

/* One problem of a batch (feast_interval_solve_batch): inputs and outputs as
 * feast_interval_solve's, with its own device matrix, interval, m0 and n_c. */
typedef struct {
  const void* A;        /* device n x n, leading dim lda, dtype; not modified */
  int dtype;
  int64_t n, lda;
  double lmin, lmax, tol;
  int m0, n_c;
  double* evals;        /* host, >= m0 doubles */
  void* evecs;          /* device n x m0, leading dim n */
  double* res;          /* host, >= m0 doubles */
  int m_found, iterations, status;  /* outputs: pairs, outer iterations, return code */
  int route;            /* output: FEAST_PREC_* the autotuner chose (mixed requests) */
  double ms;            /* output: wall time of this problem's solve */
} feast_problem;

/* Many independent interval problems of uneven n and m0 (the intervals are
 * independent, Sect. I): `workers` host threads, each with its own CUDA
 * stream and context on `device`, take the problems largest first from a
 * shared queue, so small problems run concurrently and fill the GPU.  With
 * autotune != 0 and a mixed precision requested, the route of the complex-FP32
 * GEMM updates (tensor cores, FEAST_PREC_MIXED, or SIMT, FEAST_PREC_MIXED_SIMT)
 * is chosen per size bucket (n rounded up to 256) by timing both on a probe
 * factorisation the first time the bucket is met (cached for the process).
 * opts: shared by every problem (NULL = defaults; x0 must be NULL).  Returns
 * FEAST_OK when every problem returned >= 0, else the first negative status;
 * each problem's own status is in its `status`. */
int feast_interval_solve_batch(int device, int nproblems, feast_problem* problems, const feast_opts* opts,
                               int workers, int autotune);

/* Y = rho(A) X by the quadrature of Eq. 3 over both half-contours: real A:
 * sum_j 2 Re(w_j (z_j I - A)^{-1} X); complex Hermitian A:
 * sum_j [w_j (z_j I - A)^{-1} + conj(w_j) (conj(z_j) I - A)^{-1}] X.
 * X, Y: device n x m (leading dim n, dtype).  opts supplies prec, aspect,
 * refine_max, refine_tol, anorm (NULL = defaults). */
int feast_filter_apply(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda,
                       double lmin, double lmax, int n_c, const feast_opts* opts,
                       const void* X, int64_t m, void* Y);

/* LU with partial pivoting of M_e = z_e I - A for nz shifts z (host, 2*nz
 * doubles).  LU: device nz * n * n complex elements (complex double for
 * FEAST_PREC_F64, complex float for the mixed precisions), factor e at offset
 * e*n*n, unit-lower L below the diagonal, U on and above it.  perm: device
 * nz*n int32, perm[e*n + i] = row of M_e now at row i (P M_e = L U). */
int feast_shifted_lu(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda,
                     const double* z, int nz, int prec, void* LU, int32_t* perm);

/* Y_e = M_e^{-1} B (adjoint = 0) or M_e^{-H} B (adjoint = 1) from factors of
 * feast_shifted_lu (same prec), without refinement.  FEAST_PREC_MIXED_TC
 * also runs the block updates of the triangular solves on the tensor cores
 * (the route opts.tc_solve = 1 selects in the solver).  B: device n x m complex
 * double; Y: device nz * n * m complex double, solve e at offset e*n*m. */
int feast_shifted_solve(feast_ctx* ctx, const void* LU, const int32_t* perm, int64_t n, int nz,
                        int prec, int adjoint, const void* B, int64_t m, void* Y);

/* Orthonormalise the columns of X (device n x k, dtype, in place).
 * method 0: Cholesky-QR twice, Gram-eigendecomposition route on breakdown;
 * method 1: Gram-eigendecomposition X^H X = V S^2 V^H, U = X V S^{-1} over
 * the directions with s^2 >= 1e-12 s_1^2, then one Cholesky-QR pass
 * (Sect. II-A).  *rank receives the number of orthonormal columns written to
 * the front of X. */
int feast_orthonormalize(feast_ctx* ctx, int dtype, int64_t n, int64_t k, void* X, int method,
                         int* rank);

/* Eigenvalues (host, ascending) and eigenvectors (device k x k, leading dim
 * k) of the Hermitian k x k matrix H (device, leading dim k, not modified) by
 * two-sided Jacobi with round-robin ordering; *sweeps may be NULL. */
int feast_jacobi_eigh(feast_ctx* ctx, int dtype, int64_t k, const void* H, double* evals,
                      void* V, int* sweeps);

/* Rayleigh-Ritz on the orthonormal basis Q (device n x k): A' = Q^H A Q,
 * A' V = V Lambda, X = Q V (device n x k), relative residuals
 * ||A x_j - lambda_j x_j|| / anorm (host), Ritz values ascending (host). */
int feast_rayleigh_ritz(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda,
                        const void* Q, int64_t k, double anorm, double* evals, void* X,
                        double* res);

/* C = alpha op(A) op(B) + beta C, FP64-accurate, column major on the device:
 * dtype FEAST_R64 (double) or FEAST_C128 (interleaved complex double);
 * op(A) = A (transA = 0; A is M x K, lda >= M) or its conjugate transpose
 * (transA = 1; A is K x M, lda >= K); likewise op(B) (K x N) from B (ldb);
 * C is M x N (ldc >= M, not aliasing A or B); alpha, beta real.  This is the
 * FP64-accurate product that the mixed precision needs for its refinement
 * residual R = X - (zI - A) Y and uses for its Rayleigh-Ritz and
 * orthonormalisation products (the refinement itself is not in the paper,
 * which solves in full precision).
 * method 0: bf16 tensor cores with error-free digit splitting (Ozaki scheme:
 * six 8-bit digits per element under a per-row / per-column exponent, 21
 * digit products accumulated exactly in 128-long K chunks; complex by three
 * real products), error about 2^-47 sum_k 2^(e_i + f_j) per real product
 * where 2^e_i > max_k |op(A)_ik| and 2^f_j > max_k |op(B)_kj|.
 * method 1: double-float arithmetic on the FP32 pipes, error about
 * 2^-44 sum_k |A_ik| |B_kj|; real, transA = transB = 0 and beta = 0 only.
 * Scratch comes from the context.  Returns FEAST_ERR_ARG for bad sizes,
 * leading dimensions, flags or non-finite alpha/beta, FEAST_ERR_TIMEOUT when a
 * bounded device wait gave up. */
int feast_gemm_f64acc(feast_ctx* ctx, int method, int dtype, int transA, int transB, int64_t M, int64_t N, int64_t K,
                      double alpha, const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                      int64_t ldc);

/* ---- learned m0 / node proposer (spectrum estimation ahead of the solve,
 * which the paper names as future work, Sect. IV) ---- */

/* Stochastic-trace Chebyshev moments of the spectral density of the Hermitian
 * A (device, dtype, leading dim lda): mu_k = (1/(n nv)) sum_v Re(v^H T_k(B) v)
 * for k < M, B = (A - c I)/r, the T_k(B) v by the three-term recurrence
 * t_{k+1} = 2 B t_k - t_{k-1}.  The spectrum of A must lie in [c - r, c + r].
 * V: device n x nv probe vectors (leading dim n, dtype of A) with E[v v^H] = I
 * (N(0,1) or random signs); mu: host, M doubles.  1 <= M <= 4096. */
int feast_spectral_moments(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double c, double r,
                           const void* V, int64_t nv, int M, double* mu);

/* Host: eigenvalue count estimate of (a, b) from the moments of
 * feast_spectral_moments, n times the Jackson-damped kernel-polynomial
 * density integrated over (a, b):  n [g_0 mu_0 (th_a - th_b)/pi +
 * sum_{k>=1} g_k mu_k 2 (sin(k th_a) - sin(k th_b))/(k pi)], th = arccos((x - c)/r). */
double feast_moments_count(const double* mu, int M, double c, double r, double a, double b, int64_t n);

/* The proposer's multilayer perceptron, 64 -> 256 -> 256 -> 256 -> 9 with
 * ReLU on the hidden layers, FP32.  params: one device array of
 * feast_mlp_param_count() floats holding, layer by layer, W (d_out x d_in,
 * row major) then b (d_out).  X: device B x 64, Y: device B x 9, T: device
 * B x 9 targets, row major.  Scratch comes from the context. */
int feast_mlp_param_count(void);
int feast_mlp_forward(feast_ctx* ctx, const float* params, const float* X, int64_t B, float* Y);
/* grad (device, feast_mlp_param_count floats) of the mean squared error
 * (1/(9 B)) sum (Y - T)^2, whose value goes to *loss (host). */
int feast_mlp_gradient(feast_ctx* ctx, const float* params, const float* X, const float* T, int64_t B, float* grad,
                       double* loss);
/* One Adam step (Kingma & Ba; b1 = 0.9, b2 = 0.999, eps = 1e-8) on the mean
 * squared error of the batch: params, m, v (device, feast_mlp_param_count
 * floats each) updated in place; step counts from 1; *loss (host, may be NULL)
 * receives the loss before the step. */
int feast_mlp_train_step(feast_ctx* ctx, float* params, float* m, float* v, const float* X, const float* T, int64_t B,
                         int step, double lr, double* loss);

/* Allocation-free Jacobi eigensolver, for callers that cannot allocate device
 * memory at call time: services that reserve their whole memory budget up
 * front, frameworks whose caching allocator holds the free memory.  (The
 * paper has no counterpart; this is a deployment variant of
 * feast_jacobi_eigh.)  Same operation and outputs as feast_jacobi_eigh,
 * without a context: device is the CUDA device, stream a cudaStream_t (NULL
 * = legacy default stream), H device k x k (leading dim k, not modified),
 * evals host (k doubles, ascending), V device k x k.
 * All scratch lives in one static device array of 2.25 MiB inside the library
 * (held by every GPU that loads the library until the process exits), so k is
 * limited to 1 <= k <= 256; larger k returns FEAST_ERR_ARG.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  The first call on a
 * device looks up the array's device address (once per device).  The call
 * synchronises its stream and reads the eigenvalues back to the host to sort
 * them, so a stream that is being captured into a CUDA graph is refused with
 * FEAST_ERR_ARG before anything is enqueued on it (the capture stays valid).
 * The caller's current device is restored on return.  Every call reuses the
 * same array: calls that overlap on the GPU (other streams or host threads)
 * race. */
int feast_jacobi_eigh_noalloc(int device, void* stream, int dtype, int64_t k, const void* H,
                              double* evals, void* V, int* sweeps);

/* ------------------------------------------------------------------------
 * General (non-Hermitian) matrices.  Sect. I names the non-Hermitian problem
 * among the extensions FEAST takes directly; the paper gives no algorithm.
 * Reading: the contour is the whole circle |z - c| = r and the filter
 * sum_k w_k (z_k I - A)^{-1} X (Eq. 3) takes both half-circles (2 n_c
 * shifted factorisations, no Hermitian mirror); Rayleigh-Ritz uses an
 * orthonormal basis Q of the filtered block, A' = Q^H A Q is diagonalised
 * by Hessenberg reduction and shifted QR to Schur form, Ritz vectors
 * x = Q v have unit 2-norm; the check is max ||A x - lambda x|| / ||A||_2
 * over the Ritz values inside the disk (FEAST Algorithm step 3).  FP64
 * complex arithmetic throughout.  Complex numbers on the host are
 * interleaved (re, im) doubles.
 * ------------------------------------------------------------------------ */

/* The 2 n_c nodes and weights of the whole circle (host arrays of 2 n_c
 * complex numbers each): first the upper half-circle nodes of the Hermitian
 * rule, c + r e^{i theta_j}, theta_j = (pi/2)(1 - t_j) for the ascending
 * Gauss-Legendre abscissae t_j, with weights (omega_j / 4) r e^{i theta_j};
 * then their mirror images c + r e^{-i theta_j} with weights
 * (omega_j / 4) r e^{-i theta_j}.  1 <= n_c <= 64, r > 0.  Returns FEAST_OK
 * or FEAST_ERR_ARG. */
int feast_circle_nodes(double c_re, double c_im, double radius, int n_c, double* z, double* w);

/* Eigenpairs of the general complex k x k matrix H (device, column-major,
 * leading dim k, not modified), the reduced problem of the general
 * Rayleigh-Ritz step: Hessenberg reduction, implicit single-shift QR with
 * Wilkinson shifts to the Schur form H = Z T Z^H (one CTA), eigenvectors of
 * T by back substitution, V = Z Y with unit 2-norm columns.  evals: host,
 * k complex numbers in the order of T's diagonal; V: device k x k.
 * *sweeps (may be NULL): QR sweeps taken.  1 <= k <= 2048.  Returns
 * FEAST_ERR_NONFINITE for NaN/Inf in H, FEAST_ERR_ORTH when QR does not
 * converge within 30 k sweeps, FEAST_ERR_TIMEOUT when the kernel's 20 s
 * limit expires. */
int feast_eig_general(feast_ctx* ctx, int64_t k, const void* H, double* evals, void* V, int* sweeps);

/* Y = sum_k w_k (z_k I - A)^{-1} X over the 2 n_c nodes of feast_circle_nodes:
 * the filter of a general n x n matrix A (device, dtype FEAST_R64 or
 * FEAST_C128, leading dim lda) on the complex n x m block X (device, leading
 * dim n); Y: device complex n x m (leading dim n).  Scratch: 2 n_c complex
 * FP64 factors of n x n.  Returns FEAST_ERR_SINGULAR when a shifted matrix is
 * exactly singular (a node on an eigenvalue). */
int feast_filter_apply_general(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double c_re,
                               double c_im, double radius, int n_c, const void* X, int64_t m, void* Y);

/* Eigenpairs of the general n x n matrix A (device, dtype FEAST_R64 or
 * FEAST_C128, leading dim lda, not modified) with eigenvalues inside the open
 * disk |lambda - c| < r.  m0: subspace size (more than the expected count,
 * 1 <= m0 <= min(n, 2048)); n_c: nodes per half-circle; tol: stopping
 * tolerance on the relative residuals of the Ritz pairs inside the disk
 * (||A||_2 by 40 power iterations of A^H A).  x0: optional device complex
 * n x m0 starting block (NULL: seeded N(0, 1/2) + i N(0, 1/2)).  The next
 * iteration filters all m0 Ritz vectors.  Outputs: evals (host, >= 2 m0
 * doubles: complex eigenvalues ordered by real then imaginary part), X
 * (device complex n x m0, leading dim n; unit 2-norm eigenvectors), res
 * (host, >= m0 doubles), *m_found pairs, *iterations.  Stops with no pairs
 * when no Ritz value lies inside after two iterations.  When the filtered
 * block is numerically rank deficient the basis keeps the directions with
 * sigma^2 >= 1e-12 sigma_1^2 and the subspace shrinks to that rank.
 * Returns FEAST_OK, FEAST_WARN_MAXITER or an error. */
int feast_disk_solve(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double c_re, double c_im,
                     double radius, int m0, int n_c, double tol, int max_iter, const void* x0, double* evals,
                     void* X, double* res, int* m_found, int* iterations);

#ifdef __cplusplus
}
#endif

#endif /* FEAST_GB300_H */
