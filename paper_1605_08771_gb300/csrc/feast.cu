// Host driver of the FEAST interval eigensolver and the C ABI (include/feast.h).
//
// The driver follows the paper's Appendix: FEAST (filter, Rayleigh-Ritz,
// check), XFEAST (window of s filtered blocks, Sect. II-A) and RFEAST (s
// Rayleigh-Ritz passes expanding with Ritz residuals, Sect. II-B).  All
// arithmetic runs in the CUDA kernels of factor.cu, gemm.cu, oz_gemm.cu,
// tc_cgemm.cu and dense.cu; the host only sequences launches, reads back the
// k Ritz values and residuals it needs for the selection and stopping
// decisions and sorts them, and groups the FP64 polish's remaining
// above-threshold pairs into index sets.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/feast.h"
#include "dense.cuh"
#include "factor.cuh"
#include "gemm.cuh"
#include "general.cuh"
#include "oz_gemm.cuh"
#include "proposer.cuh"

using namespace feast;

// ---------------------------------------------------------------------------
// context and workspace
// ---------------------------------------------------------------------------
namespace {

struct Arena {
  struct Block { char* p; size_t cap, off; };
  std::vector<Block> blocks;
  void* alloc(size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    for (auto& b : blocks)
      if (b.cap - b.off >= bytes) {
        void* r = b.p + b.off;
        b.off += bytes;
        return r;
      }
    size_t cap = std::max(bytes, size_t(64) << 20);
    char* p = nullptr;
    cudaError_t e = cudaMalloc(&p, cap);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw std::bad_alloc();
    }
    blocks.push_back({p, cap, bytes});
    return p;
  }
  void reset() {
    for (auto& b : blocks) b.off = 0;
  }
  void release() {
    for (auto& b : blocks) cudaFree(b.p);
    blocks.clear();
  }
};

}  // namespace

struct feast_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  Arena arena;
  Arena aux;   // the generalized solve's reduction (kept across the inner solve's arena resets)
  feast_stats last{};
};

namespace {

struct FeastError {
  int code;
};

template <typename T> T* dalloc(feast_ctx* c, int64_t count) { return (T*)c->arena.alloc(sizeof(T) * (size_t)std::max<int64_t>(count, 1)); }

void sync(feast_ctx* c) { FEAST_CUDA_TRY(cudaStreamSynchronize(c->stream)); }

template <typename T> void to_host(feast_ctx* c, T* h, const T* d, int64_t count) {
  if (count <= 0) return;
  FEAST_CUDA_TRY(cudaMemcpyAsync(h, d, sizeof(T) * count, cudaMemcpyDeviceToHost, c->stream));
  sync(c);
}
template <typename T> void to_dev(feast_ctx* c, T* d, const T* h, int64_t count) {
  if (count <= 0) return;
  FEAST_CUDA_TRY(cudaMemcpyAsync(d, h, sizeof(T) * count, cudaMemcpyHostToDevice, c->stream));
  sync(c);  // the host vector may be reused right after
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// quadrature (Eq. 3 with the ellipse / Gauss-Legendre reading)
// ---------------------------------------------------------------------------
// Gauss-Legendre abscissae (ascending) and weights by Newton's method on
// P_n with the three-term recurrence, started from cos(pi (j - 1/4)/(n + 1/2)).
void gauss_legendre(int n, std::vector<double>& t, std::vector<double>& wt) {
  t.assign(n, 0.0);
  wt.assign(n, 0.0);
  for (int j = 1; j <= n; ++j) {
    double x = std::cos(M_PI * (j - 0.25) / (n + 0.5));
    double p = 0, dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      p = p1;
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = x;
      for (int k = 1; k < n; ++k) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
    }
    t[n - j] = x;  // cos estimate descends with j: store ascending
    wt[n - j] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

// Moved nodes t_j' = tanh(atanh(t_j) + delta_j) and the weights of the
// interpolatory rule on them: sum_j om_j P_p(t_j') = 2 [p == 0] for the
// Legendre polynomials P_p, p < n, by Gaussian elimination with partial
// pivoting.  false when the moved nodes are not strictly increasing.
bool offset_rule(int n, const double* delta, std::vector<double>& t, std::vector<double>& om) {
  std::vector<double> t0, w0;
  gauss_legendre(n, t0, w0);
  t.resize(n);
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(delta[j])) return false;
    t[j] = std::tanh(std::atanh(t0[j]) + delta[j]);
    if (!(std::fabs(t[j]) < 1.0) || (j > 0 && !(t[j] > t[j - 1]))) return false;
  }
  // G[p][j] = P_p(t_j), augmented with the right-hand side
  std::vector<double> G((size_t)n * (n + 1), 0.0);
  auto at = [&](int p, int j) -> double& { return G[(size_t)p * (n + 1) + j]; };
  for (int j = 0; j < n; ++j) {
    double pm = 1.0, pc = t[j];
    at(0, j) = 1.0;
    if (n > 1) at(1, j) = pc;
    for (int p = 1; p + 1 < n; ++p) {
      const double pn = ((2.0 * p + 1.0) * t[j] * pc - p * pm) / (p + 1.0);
      pm = pc;
      pc = pn;
      at(p + 1, j) = pn;
    }
  }
  at(0, n) = 2.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(at(r, col)) > std::fabs(at(piv, col))) piv = r;
    if (at(piv, col) == 0.0) return false;
    if (piv != col)
      for (int j = 0; j <= n; ++j) std::swap(at(piv, j), at(col, j));
    for (int r = col + 1; r < n; ++r) {
      const double f = at(r, col) / at(col, col);
      for (int j = col; j <= n; ++j) at(r, j) -= f * at(col, j);
    }
  }
  om.assign(n, 0.0);
  for (int col = n - 1; col >= 0; --col) {
    double v = at(col, n);
    for (int j = col + 1; j < n; ++j) v -= at(col, j) * om[j];
    om[col] = v / at(col, col);
  }
  return true;
}

void contour(double lmin, double lmax, int nc, double aspect, std::vector<c128>& z, std::vector<c128>& w,
             const double* offsets = nullptr) {
  std::vector<double> t, om;
  if (offsets) {
    if (!offset_rule(nc, offsets, t, om)) throw FeastError{FEAST_ERR_ARG};
  } else {
    gauss_legendre(nc, t, om);
  }
  const double c = 0.5 * (lmin + lmax), r = 0.5 * (lmax - lmin);
  z.resize(nc);
  w.resize(nc);
  for (int j = 0; j < nc; ++j) {
    const double th = 0.5 * M_PI * (1.0 - t[j]);
    z[j] = c128{c + r * std::cos(th), aspect * r * std::sin(th)};
    w[j] = c128{0.25 * om[j] * aspect * r * std::cos(th), 0.25 * om[j] * r * std::sin(th)};
  }
}

// ---------------------------------------------------------------------------
// selection rules (Sect. II-A end; Sect. II-B)
// ---------------------------------------------------------------------------
bool in_interval(double l, double a, double b) { return l > a && l < b; }

std::vector<int> select_pairs(const std::vector<double>& lam, const std::vector<double>& res, double a, double b,
                              int m0) {
  const int k = (int)lam.size();
  std::vector<int> ins, outs;
  for (int i = 0; i < k; ++i) (in_interval(lam[i], a, b) ? ins : outs).push_back(i);
  auto by_res = [&](int x, int y) { return res[x] < res[y] || (res[x] == res[y] && (lam[x] < lam[y] || (lam[x] == lam[y] && x < y))); };
  std::stable_sort(ins.begin(), ins.end(), by_res);
  std::stable_sort(outs.begin(), outs.end(), by_res);
  std::vector<int> sel(ins.begin(), ins.begin() + std::min<int>((int)ins.size(), m0));
  for (size_t i = 0; (int)sel.size() < m0 && i < outs.size(); ++i) sel.push_back(outs[i]);
  std::sort(sel.begin(), sel.end(), [&](int x, int y) { return lam[x] < lam[y] || (lam[x] == lam[y] && x < y); });
  return sel;
}

// ---------------------------------------------------------------------------
// solver
// ---------------------------------------------------------------------------
template <typename S>
struct Solver {
  static constexpr bool kCplx = is_cx<S>::value;
  feast_ctx* ctx;
  cudaStream_t st;
  const S* A;
  int64_t n, lda;
  double lmin, lmax;
  int nc;
  feast_opts o;
  double anorm = 0.0;
  int E = 0;  // solve entries per filter: nc (real) or 2 nc (complex)

  std::vector<c128> z, w;
  c128* d_w = nullptr;
  c128* d_ze = nullptr;
  void* M = nullptr;
  int32_t* ipiv = nullptr;
  int32_t* perm = nullptr;
  int32_t* pinv = nullptr;   // inverse row permutations (adjoint solves' output step)
  PanelWork pw{};
  CoopWork cw{};
  int64_t kmax = 0, mmax = 0;

  // filter scratch
  c128* Y = nullptr;
  c128* Yw = nullptr;   // F64: adjoint work; mixed: residual R
  c128* AY = nullptr;
  c64* Yc = nullptr;
  double* d_en = nullptr;
  int* d_act = nullptr;
  int refine_steps = 0;
  int rr_passes = 0;  // Rayleigh-Ritz passes and the sums of their k and k^3
  double rr_k_sum = 0.0, rr_k3_sum = 0.0;
  bool refine_now = true;      // mixed: refine the next filter application
  // two-phase reduced eigensolver scratch (FP32 Jacobi, FP64 polish)
  using F32 = typename std::conditional<std::is_same<S, c128>::value, c64, float>::type;
  static constexpr int64_t kEigMixedMin = 64;
  F32* H32 = nullptr;
  F32* V32 = nullptr;
  F32* HPb = nullptr;   // block Jacobi working copy (padded)
  F32* VPb = nullptr;
  F32* Ubj = nullptr;   // block Jacobi subproblem unitaries
  int* d_bjrot = nullptr;  // block Jacobi: set when a sweep rotated
  S* Ve = nullptr;
  S* Te = nullptr;
  S* T2e = nullptr;
  // cluster finish of the FP64 polish: pair list, index sets, their unitaries
  int* d_ccnt = nullptr;
  int* d_clist = nullptr;
  int* d_cidx = nullptr;
  int* d_coff = nullptr;
  int* d_csw = nullptr;
  S* Ucl = nullptr;
  int64_t ccap = 0;
  // sweeps restricted to the indices of the above-threshold pairs
  S *Hsub = nullptr, *Vsub = nullptr, *Tsub = nullptr, *Tsub2 = nullptr;
  double* d_dg = nullptr;  // FP64 diagonal of the double-float sweeps
  static constexpr int kPolishSweeps = 2;  // full FP64 sweeps before the cluster finish
  // mixed, opts.refine_gemm = 1: double-float planes of A (hi/lo of Re, Im,
  // Re + Im) and of the right-hand block of an A product
  float* Apl = nullptr;
  float* Bpl = nullptr;
  double* Tdf = nullptr;
  int64_t bpl_cols = 0;
  // mixed, opts.refine_gemm = 0: digit planes of A (Re, Im, Re + Im for
  // complex A) and buffers for those of the right operand
  bool use_oz = false;
  OzOperand Aoz[3];
  void* Boz[3] = {nullptr, nullptr, nullptr};
  // FEAST_PREC_MIXED: bf16 planes of the complex-FP32 factors for the
  // tensor-core block updates of the triangular solves
  SolvePlanes splanes;
  bool use_tc = false;
  // The Rayleigh-Ritz, orthonormalisation and eigensolver products are not
  // routed through the digit-split GEMM: its error is bounded by row/column
  // maxima, and on the graded filtered bases it held the n = 8192 RFEAST
  // residuals above 1e-10 ||A||.  Their op-N products take the double-float
  // GEMM (mm_df below); the Gram matrices of the filtered bases stay FP64.
  // Rayleigh-Ritz scratch
  S *Qb = nullptr, *Wb = nullptr, *Xr = nullptr, *AXr = nullptr, *T1 = nullptr, *T2 = nullptr;
  S *Ar0 = nullptr, *Ar = nullptr, *Vk = nullptr, *Gs = nullptr, *Ri = nullptr, *Cs = nullptr, *Cs2 = nullptr;
  S* part = nullptr;
  int64_t part_elems = 0;
  double *d_lam = nullptr, *d_nrm = nullptr, *d_scale = nullptr;
  int* d_idx = nullptr;
  int* d_flag = nullptr;

  std::vector<double> lam, res;  // last Rayleigh-Ritz
  int last_sweeps = 0;

  // phase timing (FEAST_PROFILE set): synchronises around each phase
  bool profile = std::getenv("FEAST_PROFILE") != nullptr;
  std::vector<std::pair<const char*, double>> phases;
  template <typename Fn> void phase(const char* name, Fn&& fn) {
    if (!profile) { fn(); return; }
    sync(ctx);
    const double t0 = now_ms();
    fn();
    sync(ctx);
    const double dt = now_ms() - t0;
    for (auto& p : phases)
      if (p.first == name) { p.second += dt; return; }
    phases.push_back({name, dt});
  }

  Solver(feast_ctx* c, const S* A_, int64_t n_, int64_t lda_, double a, double b, int nc_, const feast_opts& o_)
      : ctx(c), st(c->stream), A(A_), n(n_), lda(lda_), lmin(a), lmax(b), nc(nc_), o(o_) {
    E = kCplx ? 2 * nc : nc;
  }

  // ---- allocation ----
  void alloc_common(int64_t kmax_, int64_t mmax_) {
    kmax = std::max<int64_t>(kmax_, 1);
    mmax = std::max<int64_t>(mmax_, 1);
    use_oz = o.prec != FEAST_PREC_F64 && o.refine_gemm == 0;
    use_tc = o.prec == FEAST_PREC_MIXED;
    contour(lmin, lmax, nc, o.aspect, z, w, o.node_offsets);
    d_w = dalloc<c128>(ctx, nc);
    d_ze = dalloc<c128>(ctx, E);
    std::vector<c128> ze(E);
    for (int j = 0; j < nc; ++j) {
      ze[j] = z[j];
      if (kCplx) ze[nc + j] = conj(z[j]);
    }
    to_dev(ctx, d_w, w.data(), nc);
    to_dev(ctx, d_ze, ze.data(), E);
    cw = coop_work_carve(ctx->arena.alloc(coop_work_bytes(kmax, ctx->num_sms)), kmax, ctx->num_sms);
    d_flag = dalloc<int>(ctx, 4);  // [0]: status word of the tensor-core refinement GEMM
    FEAST_CUDA_TRY(cudaMemsetAsync(d_flag, 0, 4 * sizeof(int), st));
    d_en = dalloc<double>(ctx, 2 * E);
    d_act = dalloc<int>(ctx, E);
  }
  void alloc_factors() {
    const size_t eb = o.prec == FEAST_PREC_F64 ? sizeof(c128) : sizeof(c64);
    M = ctx->arena.alloc(eb * (size_t)nc * n * n);
    ipiv = dalloc<int32_t>(ctx, (int64_t)nc * n);
    perm = dalloc<int32_t>(ctx, (int64_t)nc * n);
    pinv = dalloc<int32_t>(ctx, (int64_t)nc * n);
    const int pmax = std::max(1, ctx->num_sms * 8);
    pw = panel_work_carve(ctx->arena.alloc(panel_work_bytes(nc, pmax, eb)), nc, pmax, eb);
    if (use_tc) pw.tc_planes = ctx->arena.alloc(lu_tc_planes_bytes(n, nc));
  }
  void alloc_filter(int64_t m) {
    const int64_t nm = n * m;
    Y = dalloc<c128>(ctx, E * nm);
    if (o.prec == FEAST_PREC_F64) {
      if (kCplx) Yw = dalloc<c128>(ctx, nc * nm);
    } else {
      Yw = dalloc<c128>(ctx, E * nm);
      AY = dalloc<c128>(ctx, E * nm);
      Yc = dalloc<c64>(ctx, E * nm);
      if (use_tc)
        splanes = solve_planes_carve(ctx->arena.alloc(solve_planes_bytes(n, m, nc, nc, kCplx)), n, m, nc, nc, kCplx);
      bpl_cols = std::max<int64_t>(E * m, kmax);
      if (use_oz) {
        // rows of A are read through its Hermitian symmetry, A(i, k) =
        // conj(A[k + i lda]), so every split reads contiguous columns
        if (kCplx) {
          for (int t = 0; t < 3; ++t) Aoz[t] = oz_operand(ctx->arena.alloc(oz_operand_bytes(n, n, true)), n, n, true);
          static const int modes[3] = {0, 3, 4};  // Re A(i, k), Im A(i, k), Re + Im
          oz_split_modes((const double*)A, 2, modes, 3, n, 1, lda, Aoz, st);
        } else {
          Aoz[0] = oz_operand(ctx->arena.alloc(oz_operand_bytes(n, n, true)), n, n, true);
          oz_split((const double*)A, 1, 0, n, 1, lda, Aoz[0], st);
        }
        for (int t = 0; t < (kCplx ? 3 : 2); ++t) Boz[t] = ctx->arena.alloc(oz_operand_bytes(bpl_cols, n, false));
      } else {
        const int apl = kCplx ? 6 : 2;
        Apl = dalloc<float>(ctx, (int64_t)apl * n * n);
        if (kCplx) {
          split_df32((const double*)A, n, n, lda, 2, 0, Apl, Apl + n * n, st);
          split_df32((const double*)A, n, n, lda, 2, 1, Apl + 2 * n * n, Apl + 3 * n * n, st);
          split_df32((const double*)A, n, n, lda, 2, 2, Apl + 4 * n * n, Apl + 5 * n * n, st);
        } else {
          split_df32((const double*)A, n, n, lda, 1, 0, Apl, Apl + n * n, st);
        }
        Bpl = dalloc<float>(ctx, 6 * n * bpl_cols);
      }
      if (kCplx) Tdf = dalloc<double>(ctx, n * bpl_cols);
    }
  }
  void alloc_rr() {
    Qb = dalloc<S>(ctx, n * kmax);
    Wb = dalloc<S>(ctx, n * kmax);
    Xr = dalloc<S>(ctx, n * kmax);
    AXr = dalloc<S>(ctx, n * kmax);
    T1 = dalloc<S>(ctx, n * kmax);
    T2 = dalloc<S>(ctx, n * kmax);
    const int64_t kk = kmax * kmax;
    Ar0 = dalloc<S>(ctx, kk); Ar = dalloc<S>(ctx, kk); Vk = dalloc<S>(ctx, kk); Gs = dalloc<S>(ctx, kk);
    Ri = dalloc<S>(ctx, kk); Cs = dalloc<S>(ctx, kk); Cs2 = dalloc<S>(ctx, kk);
    if (o.prec != FEAST_PREC_F64 && (double)n * kmax * kmax >= kDfMinWork) {
      Ldf = dalloc<float>(ctx, 4 * n * kmax);
      Rdf = dalloc<float>(ctx, 4 * n * kmax);
      Pdf = dalloc<double>(ctx, (int64_t)kDfMaxSplit * 2 * kk);
    }
    if (kmax >= kEigMixedMin) {
      H32 = dalloc<F32>(ctx, kk); V32 = dalloc<F32>(ctx, kk);
      const int64_t kp = block_jacobi_pad(kmax);
      HPb = dalloc<F32>(ctx, kp * kp); VPb = dalloc<F32>(ctx, kp * kp);
      Ubj = (F32*)ctx->arena.alloc(block_jacobi_u_bytes(kmax));
      d_bjrot = dalloc<int>(ctx, 1);
      Ve = dalloc<S>(ctx, kk); Te = dalloc<S>(ctx, kk); T2e = dalloc<S>(ctx, kk);
      ccap = 32 * kmax;
      d_ccnt = dalloc<int>(ctx, 1);
      d_clist = dalloc<int>(ctx, 2 * ccap);
      d_cidx = dalloc<int>(ctx, kmax);
      d_coff = dalloc<int>(ctx, kmax / 2 + 2);
      d_csw = dalloc<int>(ctx, kmax / 2 + 1);
      Ucl = dalloc<S>(ctx, (kmax / 2 + 1) * kClusterMax * kClusterMax);
      Hsub = dalloc<S>(ctx, kk); Vsub = dalloc<S>(ctx, kk); Tsub = dalloc<S>(ctx, kk); Tsub2 = dalloc<S>(ctx, kk);
      d_dg = dalloc<double>(ctx, kmax);
    }
    part_elems = 32 * kk;
    part = dalloc<S>(ctx, part_elems);
    d_lam = dalloc<double>(ctx, kmax);
    d_nrm = dalloc<double>(ctx, kmax);
    d_scale = dalloc<double>(ctx, kmax);
    d_idx = dalloc<int>(ctx, kmax);
  }

  // ---- small GEMM helpers ----
  // Mixed path: products C = alpha A B + beta C with op N on both sides (the
  // tall n x k products Q V, W V, X R^-1, Q C) and the reductions over n
  // below in double-float arithmetic on the FP32 pipes, several times the
  // FP64 rate of this GPU.  The low word of each product sum is accumulated in
  // FP32 and flushed to FP64 every 32 terms; the error stays within 2^-44 of
  // sum |a||b| (the parity tests' bound), against ~1e-16 sqrt(K) in FP64.  The
  // Gram matrices of the filtered bases stay FP64 (Cholesky-QR squares their
  // condition number); the eigensolver's k x k products use mm_eig.  Complex
  // products take the four real products (4M): the three-product form (3M)
  // forms Im as T3 - T1 - T2, whose cancellation made the n = 8192 RFEAST solve
  // take 4 iterations instead of 2; 4M keeps 2.
  float* Ldf = nullptr;  // 4 planes (Re hi/lo, Im hi/lo) of n x kmax
  float* Rdf = nullptr;  // 4 planes of n x kmax
  double* Pdf = nullptr; // split-K partial products of the reductions over n
  static constexpr double kDfMinWork = 1e6;
  static constexpr int kDfMaxSplit = 16;
  bool mm_df_ok(int64_t Mr, int64_t Nc, int64_t K, c128 alpha, c128 beta, int opA, int opB) const {
    if (!Ldf || opA != OP_N || opB != OP_N || alpha.im != 0.0 || beta.im != 0.0) return false;
    if ((double)Mr * (double)Nc * (double)K < kDfMinWork) return false;
    return Mr * K <= n * kmax && K * Nc <= n * kmax;
  }
  // Reductions over n, C = A^H B (C: Mr x Nc with Mr, Nc <= kmax, K = n:
  // Q^H W, Q^H R and the RFEAST blocks of A'), other than Gram matrices
  // (A == B, which Cholesky-QR needs in FP64): double-float 4M, the reduction
  // split into slices over all SMs.  At n = 8192 they keep the RFEAST solve at
  // 2 rounds once only unconverged pairs expand the subspace (appending every
  // residual, the noise they add stopped it from converging).
  bool mm_df_reduce_ok(int64_t Mr, int64_t Nc, int64_t K, const S* Am, int opA, const S* Bm, int opB) const {
    if (!Ldf || !Pdf || opA != OP_C || opB != OP_N || Am == Bm) return false;
    if ((double)Mr * (double)Nc * (double)K < kDfMinWork) return false;
    return Mr <= kmax && Nc <= kmax && Mr * K <= n * kmax && K * Nc <= n * kmax;
  }
  void mm_df_reduce(int64_t Mr, int64_t Nc, int64_t K, const S* Am, int64_t la, const S* Bm, int64_t lb, S* Cm,
                    int64_t lc) {
    const int64_t ak = Mr * K, bk = K * Nc;
    const int64_t tiles = cdiv(Mr, 64) * cdiv(Nc, 64);
    int ks = (int)std::min<int64_t>({(int64_t)kDfMaxSplit, std::max<int64_t>(1, K / 256),
                                     std::max<int64_t>(1, cdiv(3 * ctx->num_sms, tiles))});
    const int w = kCplx ? 2 : 1;
    const int64_t czs = (int64_t)w * Mr * Nc;
    if constexpr (std::is_same<S, c128>::value) {
      // planes of A^H: Re, then -Im (conjugate); of B: Re, Im
      split_df32_t((const double*)Am, Mr, K, la, 2, 0, false, Ldf, Ldf + ak, st);
      split_df32_t((const double*)Am, Mr, K, la, 2, 1, true, Ldf + 2 * ak, Ldf + 3 * ak, st);
      split_df32((const double*)Bm, K, Nc, lb, 2, 0, Rdf, Rdf + bk, st);
      split_df32((const double*)Bm, K, Nc, lb, 2, 1, Rdf + 2 * bk, Rdf + 3 * bk, st);
      double* P = Pdf;
      gemm_df32(Mr, Nc, K, 1.0, Ldf, Ldf + ak, Mr, Rdf, Rdf + bk, K, 0.0, P, Mr, 2, 0, st, -1, ks, czs);
      gemm_df32(Mr, Nc, K, -1.0, Ldf + 2 * ak, Ldf + 3 * ak, Mr, Rdf + 2 * bk, Rdf + 3 * bk, K, 1.0, P, Mr, 2, 0, st,
                -1, ks, czs);
      gemm_df32(Mr, Nc, K, 1.0, Ldf, Ldf + ak, Mr, Rdf + 2 * bk, Rdf + 3 * bk, K, 0.0, P, Mr, 2, 1, st, -1, ks, czs);
      gemm_df32(Mr, Nc, K, 1.0, Ldf + 2 * ak, Ldf + 3 * ak, Mr, Rdf, Rdf + bk, K, 1.0, P, Mr, 2, 1, st, -1, ks, czs);
    } else {
      split_df32_t((const double*)Am, Mr, K, la, 1, 0, false, Ldf, Ldf + ak, st);
      split_df32((const double*)Bm, K, Nc, lb, 1, 0, Rdf, Rdf + bk, st);
      gemm_df32(Mr, Nc, K, 1.0, Ldf, Ldf + ak, Mr, Rdf, Rdf + bk, K, 0.0, Pdf, Mr, 1, 0, st, -1, ks, czs);
    }
    sum_partials((double*)Cm, lc, Pdf, Mr, Nc, ks, kCplx, st);
  }
  // complex C = alpha A B + beta C by four real double-float products (4M)
  void mm_df(int64_t Mr, int64_t Nc, int64_t K, double alpha, const S* Am, int64_t la, const S* Bm, int64_t lb,
             double beta, S* Cm, int64_t lc) {
    const int64_t ak = Mr * K, bk = K * Nc;
    double* C = (double*)Cm;
    if constexpr (std::is_same<S, c128>::value) {
      split_df32((const double*)Am, Mr, K, la, 2, 0, Ldf, Ldf + ak, st);
      split_df32((const double*)Am, Mr, K, la, 2, 1, Ldf + 2 * ak, Ldf + 3 * ak, st);
      split_df32((const double*)Bm, K, Nc, lb, 2, 0, Rdf, Rdf + bk, st);
      split_df32((const double*)Bm, K, Nc, lb, 2, 1, Rdf + 2 * bk, Rdf + 3 * bk, st);
      // Re C = alpha (Ar Br - Ai Bi) + beta Re C ; Im C = alpha (Ar Bi + Ai Br) + beta Im C
      gemm_df32(Mr, Nc, K, alpha, Ldf, Ldf + ak, Mr, Rdf, Rdf + bk, K, beta, C, lc, 2, 0, st, -1);
      gemm_df32(Mr, Nc, K, -alpha, Ldf + 2 * ak, Ldf + 3 * ak, Mr, Rdf + 2 * bk, Rdf + 3 * bk, K, 1.0, C, lc, 2, 0, st, -1);
      gemm_df32(Mr, Nc, K, alpha, Ldf, Ldf + ak, Mr, Rdf + 2 * bk, Rdf + 3 * bk, K, beta, C, lc, 2, 1, st, -1);
      gemm_df32(Mr, Nc, K, alpha, Ldf + 2 * ak, Ldf + 3 * ak, Mr, Rdf, Rdf + bk, K, 1.0, C, lc, 2, 1, st, -1);
    } else {
      split_df32((const double*)Am, Mr, K, la, 1, 0, Ldf, Ldf + ak, st);
      split_df32((const double*)Bm, K, Nc, lb, 1, 0, Rdf, Rdf + bk, st);
      gemm_df32(Mr, Nc, K, alpha, Ldf, Ldf + ak, Mr, Rdf, Rdf + bk, K, beta, C, lc, 1, 0, st, -1);
    }
  }
  void mm(int64_t Mr, int64_t Nc, int64_t K, c128 alpha, const S* Am, int64_t la, int opA, const S* Bm, int64_t lb,
          int opB, c128 beta, S* Cm, int64_t lc) {
    if (mm_df_ok(Mr, Nc, K, alpha, beta, opA, opB) && (Cm != Am && Cm != Bm)) {
      mm_df(Mr, Nc, K, alpha.re, Am, la, Bm, lb, beta.re, Cm, lc);
      return;
    }
    gemm_simple<S, S, S>(Mr, Nc, K, alpha, Am, la, opA, Bm, lb, opB, beta, Cm, lc, st);
  }
  // C = op(A) op(B) for a k x k x k product of the eigensolver: split-K so
  // that the FP64 work spreads over every SM (k = 900 gives only 15 x 15
  // output tiles)
  void mm_square(int64_t k, const S* Am, int opA, const S* Bm, S* Cm) {
    const int64_t tiles = cdiv(k, 64) * cdiv(k, 64);
    int ks = (int)std::min<int64_t>({32, std::max<int64_t>(1, k / 64), cdiv(4 * ctx->num_sms, tiles)});
    while (ks > 1 && (int64_t)ks * k * k > part_elems) --ks;
    gemm_simple<S, S, S>(k, k, k, C1(1.0), Am, k, opA, Bm, k, OP_N, C1(0.0), Cm, k, st, ks,
                         ks > 1 ? (void*)part : nullptr);
  }
  // k x k products of the two-phase eigensolver on the mixed path in
  // double-float: their operands are unitary, nearly unitary or the reduced
  // matrix itself, so the error (2^-44 of sum |a||b|) stays near 1e-13 ||A||,
  // far below what the Ritz pairs need.  FP64 otherwise, and for k below 512,
  // where the double-float kernel's few output tiles leave most SMs idle and
  // the split-K FP64 product is faster
  void mm_eig(int64_t k, const S* Am, int opA, const S* Bm, S* Cm) {
    if (Ldf && Pdf && o.prec != FEAST_PREC_F64 && k >= 512 && Cm != Am && Cm != Bm) {
      if (opA == OP_N) {
        mm_df(k, k, k, 1.0, Am, k, Bm, k, 0.0, Cm, k);
        return;
      }
      if (opA == OP_C) {
        mm_df_reduce(k, k, k, Am, k, Bm, k, Cm, k);
        return;
      }
    }
    mm_square(k, Am, opA, Bm, Cm);
  }
  // C (Mr x Nc) = op(A) op(B) with a long reduction K: split-K
  void mm_reduce(int64_t Mr, int64_t Nc, int64_t K, const S* Am, int64_t la, int opA, const S* Bm, int64_t lb,
                 int opB, S* Cm, int64_t lc) {
    if (mm_df_reduce_ok(Mr, Nc, K, Am, opA, Bm, opB)) {
      mm_df_reduce(Mr, Nc, K, Am, la, Bm, lb, Cm, lc);
      return;
    }
    int ks = (int)std::max<int64_t>(1, std::min<int64_t>(32, K / 256));
    while (ks > 1 && (int64_t)ks * lc * Nc > part_elems) --ks;
    gemm_simple<S, S, S>(Mr, Nc, K, C1(1.0), Am, la, opA, Bm, lb, opB, C1(0.0), Cm, lc, st, ks,
                         ks > 1 ? (void*)part : nullptr);
  }
  // Out = A * B for an n x k block B (ld n) in double-float arithmetic on the
  // FP32 pipes: B complex (bcplx) or real; Out has B's element type.  Complex
  // A times complex B takes three real products (3M): T1 = Ar Br, T2 = Ai Bi,
  // T3 = (Ar + Ai)(Br + Bi), Re = T1 - T2, Im = T3 - T1 - T2.
  void apply_A_df(const double* B, bool bcplx, int64_t k, double* Out) {
    const int64_t nk = n * k, nn = n * n;
    float *Brh = Bpl, *Brl = Bpl + nk, *Bih = Bpl + 2 * nk, *Bil = Bpl + 3 * nk;
    float *Bsh = Bpl + 4 * nk, *Bsl = Bpl + 5 * nk;
    const float *Arh = Apl, *Arl = Apl + nn, *Aih = Apl + 2 * nn, *Ail = Apl + 3 * nn;
    const float *Ash = Apl + 4 * nn, *Asl = Apl + 5 * nn;
    const int cs = bcplx ? 2 : 1;
    split_df32(B, n, k, n, cs, 0, Brh, Brl, st);
    if (bcplx) split_df32(B, n, k, n, 2, 1, Bih, Bil, st);
    if (kCplx) {  // complex A, complex B (3M)
      split_df32(B, n, k, n, 2, 2, Bsh, Bsl, st);
      gemm_df32(n, k, n, 1.0, Arh, Arl, n, Brh, Brl, n, 0.0, Out, n, 2, 0, st);
      gemm_df32(n, k, n, 1.0, Aih, Ail, n, Bih, Bil, n, 0.0, Tdf, n, 1, 0, st);
      gemm_df32(n, k, n, 1.0, Ash, Asl, n, Bsh, Bsl, n, 0.0, Out, n, 2, 1, st);
      combine_3m(Out, Tdf, n, k, st);
    } else if (bcplx) {  // real A, complex B
      gemm_df32(n, k, n, 1.0, Arh, Arl, n, Brh, Brl, n, 0.0, Out, n, 2, 0, st);
      gemm_df32(n, k, n, 1.0, Arh, Arl, n, Bih, Bil, n, 0.0, Out, n, 2, 1, st);
    } else {  // real A, real B
      gemm_df32(n, k, n, 1.0, Arh, Arl, n, Brh, Brl, n, 0.0, Out, n, 1, 0, st);
    }
  }
  // Out = A * B on the tensor cores: each real product from digit planes
  // (oz_gemm), complex A by the same three products (3M) as apply_A_df
  void apply_A_oz(const double* B, bool bcplx, int64_t k, double* Out) {
    OzOperand Bo[3];
    const int nb = kCplx ? 3 : (bcplx ? 2 : 1);
    for (int t = 0; t < nb; ++t) Bo[t] = oz_operand(Boz[t], k, n, false);
    const int sms = ctx->num_sms;
    static const int modes[3] = {0, 1, 2};  // Re, Im, Re + Im
    if (kCplx) oz_split_modes(B, 2, modes, 3, n, 1, n, Bo, st);
    else oz_split_modes(B, bcplx ? 2 : 1, modes, bcplx ? 2 : 1, n, 1, n, Bo, st);
    if (kCplx) {
      oz_gemm(n, k, Aoz[0], Bo[0], Out, n, 2, 0, d_flag, sms, st);
      oz_gemm(n, k, Aoz[1], Bo[1], Tdf, n, 1, 0, d_flag, sms, st);
      oz_gemm(n, k, Aoz[2], Bo[2], Out, n, 2, 1, d_flag, sms, st);
      combine_3m(Out, Tdf, n, k, st);
    } else if (bcplx) {
      oz_gemm(n, k, Aoz[0], Bo[0], Out, n, 2, 0, d_flag, sms, st);
      oz_gemm(n, k, Aoz[0], Bo[1], Out, n, 2, 1, d_flag, sms, st);
    } else {
      oz_gemm(n, k, Aoz[0], Bo[0], Out, n, 1, 0, d_flag, sms, st);
    }
  }
  // FP64-accurate A times an n x k block on the mixed path
  void apply_A_acc(const double* B, bool bcplx, int64_t k, double* Out) {
    if (use_oz) apply_A_oz(B, bcplx, k, Out);
    else apply_A_df(B, bcplx, k, Out);
  }
  // a timed-out wait inside the tensor-core GEMM
  void check_oz_status() {
    int f = 0;
    to_host(ctx, &f, d_flag, 1);
    if (f == DEV_BARRIER_TIMEOUT) throw FeastError{FEAST_ERR_TIMEOUT};
  }
  // A times a block: FP64 on the FP64 path, FP64-accurate products on the mixed path
  void apply_A(const S* Xm, int64_t k, S* Out) {
    if (o.prec != FEAST_PREC_F64 && (Apl || use_oz) && k <= bpl_cols) {
      apply_A_acc((const double*)Xm, kCplx, k, (double*)Out);
      return;
    }
    mm(n, k, n, C1(1.0), A, lda, OP_N, Xm, n, OP_N, C1(0.0), Out, n);
  }

  // ---- norm estimate: power iteration from ones/sqrt(n) ----
  double estimate_norm() {
    S* v = T1;
    S* wv = T2;
    std::vector<S> ones(n, cvt<S>(1.0 / std::sqrt((double)n)));
    to_dev(ctx, v, ones.data(), n);
    double est = 0.0, nr2 = 0.0;
    for (int it = 0; it < 40; ++it) {
      apply_A(v, 1, wv);
      col_norms2<S>(wv, n, 1, n, d_nrm, st);
      to_host(ctx, &nr2, d_nrm, 1);
      est = std::sqrt(nr2);
      if (est == 0.0) return 0.0;
      double sc = 1.0 / est;
      to_dev(ctx, d_scale, &sc, 1);
      int zero = 0;
      to_dev(ctx, d_idx, &zero, 1);
      gather_cols<S>(v, n, wv, n, n, d_idx, 1, d_scale, st);
    }
    return est;
  }

  // ---- factorisation of all shifts ----
  template <typename F>
  void factor_t() {
    F* Mf = (F*)M;
    std::vector<c128> zf(z.begin(), z.end());
    c128* d_zf = dalloc<c128>(ctx, nc);
    to_dev(ctx, d_zf, zf.data(), nc);
    form_shifted<F, S>(Mf, n, n, n * n, nc, A, lda, d_zf, st);
    lu_factor_batched<F>(Mf, n, n, n * n, nc, ipiv, perm, pw, ctx->num_sms, st);
    invert_perm(perm, pinv, n, nc, st);
    if constexpr (std::is_same<F, c64>::value)
      if (use_tc && splanes.col) solve_planes_build(Mf, n, n, n * n, nc, splanes, st);
    int status = 0;
    std::vector<int> zp(nc);
    to_host(ctx, &status, pw.status, 1);
    to_host(ctx, zp.data(), pw.zero_pivot, nc);
    if (status == DEV_BARRIER_TIMEOUT) throw FeastError{FEAST_ERR_TIMEOUT};
    for (int j = 0; j < nc; ++j)
      if (zp[j]) throw FeastError{FEAST_ERR_SINGULAR};
  }
  void factor() {
    if (o.prec == FEAST_PREC_F64) factor_t<c128>();
    else factor_t<c64>();
  }

  // ---- filter: Xf = rho(A) X (Eq. 3) ----
  // the low-precision solves of both half-contours into Yc (before the
  // adjoint solves' output permutation)
  template <typename TB>
  void solve_lowp_core(const TB* B, int64_t ldb, int64_t bstride, int64_t m) {
    const int64_t nm = n * m;
    const c64* Mf = (const c64*)M;
    const SolvePlanes* sp = use_tc ? &splanes : nullptr;
    permute_in<c64, TB>(Yc, nm, B, ldb, bstride, n, m, perm, nc, false, st);
    lu_solve_batched<c64>(Mf, n, n, n * n, nc, Yc, m, nm, false, st, sp, d_flag, ctx->num_sms);
    if (kCplx) {
      permute_in<c64, TB>(Yc + nc * nm, nm, B + nc * bstride, ldb, bstride, n, m, perm, nc, true, st);
      lu_solve_batched<c64>(Mf, n, n, n * n, nc, Yc + nc * nm, m, nm, true, st, sp, d_flag, ctx->num_sms);
    }
  }
  // Y (+)= the solves' outputs in natural row order, in FP64
  void lowp_out(int64_t m, bool accumulate) {
    const int64_t nm = n * m;
    permute_out<c64, c128>(Y, nm, Yc, nm, n, m, perm, nc, false, accumulate, st);
    if (kCplx) permute_out<c64, c128>(Y + nc * nm, nm, Yc + nc * nm, nm, n, m, perm, nc, true, accumulate, st);
  }

  double filter_ms = 0.0;
  void filter(const S* X, int64_t m, S* Xf) {
    const double t0 = now_ms();
    filter_body(X, m, Xf);
    sync(ctx);
    check_oz_status();
    filter_ms += now_ms() - t0;
  }
  // Xf = sum of the weighted solves (Eq. 3).  The weighted accumulation is
  // fused with the output step of the last solves (solve_accumulate) except
  // when the refinement ends on a residual check, whose Y is final already.
  void filter_body(const S* X, int64_t m, S* Xf) {
    const int64_t nm = n * m;
    if (o.prec == FEAST_PREC_F64) {
      const c128* Mf = (const c128*)M;
      permute_in<c128, S>(Y, nm, X, n, 0, n, m, perm, nc, false, st);
      lu_solve_batched<c128>(Mf, n, n, n * n, nc, Y, m, nm, false, st);
      if (kCplx) {
        permute_in<c128, S>(Yw, nm, X, n, 0, n, m, perm, nc, true, st);
        lu_solve_batched<c128>(Mf, n, n, n * n, nc, Yw, m, nm, true, st);
      }
      solve_accumulate<S, c128>(Xf, n, nullptr, Y, kCplx ? Yw : Y, n, m, nc, pinv, d_w, st);
      return;
    }
    phase("c64 solves", [&] { solve_lowp_core<S>(X, n, 0, m); });
    if (!refine_now) {
      solve_accumulate<S, c64>(Xf, n, nullptr, Yc, Yc + (kCplx ? nc * nm : 0), n, m, nc, pinv, d_w, st);
      return;
    }
    phase("c64 solves", [&] { lowp_out(m, false); });
    // default target 16 eps sqrt(n): just above the accuracy floor of the
    // FP64-accurate residual
    const double rtol = o.refine_tol > 0 ? o.refine_tol : 16.0 * 2.220446049250313e-16 * std::sqrt((double)n);
    std::vector<double> en(2 * E), prev(E, -1.0);
    double worst_prev = -1.0;
    // entries whose residual met the target drop out of later steps: their
    // A*Y product is skipped and their residual set to zero
    std::vector<int> active(E, 1);
    for (int step = 0; step < o.refine_max; ++step) {
      // R_e = X - (z_e I - A) Y_e, FP64-accurate (double-float A Y)
      for (int e0 = 0; e0 < E;) {
        if (!active[e0]) { ++e0; continue; }
        int e1 = e0;
        while (e1 < E && active[e1]) ++e1;
        phase("refine A*Y", [&] { apply_A_acc((const double*)(Y + e0 * nm), true, (e1 - e0) * m, (double*)(AY + e0 * nm)); });
        e0 = e1;
      }
      to_dev(ctx, d_act, active.data(), E);
      refine_residual<S>(Yw, X, n, Y, AY, n, m, E, d_ze, d_act, st);
      entry_norms2(Yw, Y, n, m, E, d_en, st);
      to_host(ctx, en.data(), d_en, 2 * E);
      bool conv = true, stagnant = step > 0;
      double worst = 0.0;
      for (int e = 0; e < E; ++e) {
        if (!active[e]) continue;
        const c128 ze = e < nc ? z[e] : conj(z[e - nc]);
        const double rn = std::sqrt(en[2 * e]), yn = std::sqrt(en[2 * e + 1]);
        const double rel = rn / ((anorm + std::sqrt(abs2(ze))) * yn);
        if (rel <= rtol) {
          active[e] = 0;
        } else {
          conv = false;
          worst = std::max(worst, rel);
          if (prev[e] < 0 || rn < 0.5 * prev[e]) stagnant = false;
        }
        prev[e] = rn;
      }
      if (std::getenv("FEAST_LOG"))
        fprintf(stderr, "[feast] refine step %d: worst active relative residual %.3e (target %.3e), active %d/%d\n",
                step, worst, rtol, (int)std::count(active.begin(), active.end(), 1), E);
      if (conv || stagnant) break;
      // entries that met the target in this step still take this correction
      // (their residual is fresh); earlier ones have R = 0
      phase("c64 solves", [&] { solve_lowp_core<c128>(Yw, n, nm, m); });
      ++refine_steps;
      // when the observed contraction already puts the next residual below
      // the target, the correction just applied finishes the refinement
      // (saves one FP64-accurate A*Y product per filter); so does the last
      // allowed step.  Then Y + correction goes straight into Xf.
      const bool last = (worst_prev > 0.0 && worst * (worst / worst_prev) <= rtol) || step + 1 == o.refine_max;
      if (last) {
        solve_accumulate<S, c64>(Xf, n, Y, Yc, Yc + (kCplx ? nc * nm : 0), n, m, nc, pinv, d_w, st);
        return;
      }
      phase("c64 solves", [&] { lowp_out(m, true); });
      worst_prev = worst;
    }
    accumulate_filter<S>(Xf, n, Y, n, m, nc, d_w, st);
  }

  // ---- orthonormalisation ----
  // Qout = X R^{-1} with X^H X = R^H R.  X, Qout: nr x k (ld nr).  false on breakdown.
  bool cholqr_once(const S* X, int64_t nr, int64_t k, S* Qout) {
    phase("CholQR: Gram", [&] {
      mm_reduce(k, k, nr, X, nr, OP_C, X, nr, OP_N, Gs, k);
      hermitize<S>(Gs, k, k, st);
    });
    int info[2] = {0, 0};
    int status = 0;
    phase("CholQR: Cholesky", [&] {
      cholesky_upper<S>(Gs, k, k, cw, ctx->num_sms, st);
      to_host(ctx, info, cw.info, 1);
      to_host(ctx, &status, cw.status, 1);
    });
    if (status == DEV_BARRIER_TIMEOUT) throw FeastError{FEAST_ERR_TIMEOUT};
    if (info[0] != 0) return false;
    phase("CholQR: X R^-1", [&] {
      tri_inverse_upper<S>(Gs, k, k, Ri, k, st);
      mm(nr, k, k, C1(1.0), X, nr, OP_N, Ri, k, OP_N, C1(0.0), Qout, nr);
    });
    return true;
  }
  // Hermitian eigendecomposition of the k x k matrix H (ld k, overwritten);
  // eigenvalues unsorted in `ev`, vectors in Vk (ld k)
  void jacobi_status(int* sweeps) {
    int status = 0;
    to_host(ctx, &status, cw.status, 1);
    if (sweeps) to_host(ctx, sweeps, cw.info + 1, 1);
    if (status == DEV_BARRIER_TIMEOUT) throw FeastError{FEAST_ERR_TIMEOUT};
  }
  // Two-phase Hermitian eigendecomposition for k >= kEigMixedMin: block
  // Jacobi in FP32 (a 64x faster pipe on this GPU, and 32 x 32 subproblems
  // in shared memory instead of one grid barrier per pair round) down to
  // off-diagonals of a few FP32 ulps of ||H||_F; its vectors, made exactly orthonormal in FP64 by one
  // Cholesky-QR pass (V R^-1 with V^H V = R^H R), transform H to V^H H V,
  // which FP64 Jacobi finishes to the same threshold as the one-phase solver
  // (quadratic convergence: a few sweeps).  Vk = V V', the eigenvalues on the
  // diagonal of H.  Returns false (nothing changed in H) when the Cholesky
  // factorisation breaks down.
  bool eig_two_phase(S* H, int64_t k, int* sweeps) {
    std::vector<double> cn(k);
    col_norms2<S>(H, k, k, k, d_nrm, st);
    to_host(ctx, cn.data(), d_nrm, k);
    double fro2 = 0.0;
    for (double v : cn) fro2 += v;
    int sw32 = 0;
    phase("eig: FP32 block Jacobi", [&] {
      sw32 = block_jacobi<F32, S>(H, k, V32, 4e-7 * std::sqrt(fro2), HPb, VPb, Ubj, d_bjrot, 40, st);
    });
    int info = 0;
    phase("eig: Cholesky-QR of V", [&] {
      convert_matrix<S, F32>(Ve, k, V32, k, k, k, st);
      mm_eig(k, Ve, OP_C, Ve, Te);
      hermitize<S>(Te, k, k, st);
      cholesky_upper<S>(Te, k, k, cw, ctx->num_sms, st);
      to_host(ctx, &info, cw.info, 1);
      jacobi_status(nullptr);
    });
    if (info != 0) return false;
    phase("eig: V^H H V", [&] {
      tri_inverse_upper<S>(Te, k, k, T2e, k, st);
      mm_eig(k, Ve, OP_N, T2e, Te);   // Te: orthonormal V
      mm_eig(k, H, OP_N, Te, T2e);    // H V
      mm_eig(k, Te, OP_C, T2e, H);    // V^H H V
      hermitize<S>(H, k, k, st);
    });
    int sw64 = 0;
    phase("eig: FP64 Jacobi", [&] { sw64 = polish(H, k); });
    phase("eig: V V'", [&] { mm_eig(k, Te, OP_N, T2e, Vk); });
    *sweeps = sw32 + sw64;
    if (std::getenv("FEAST_LOG"))
      fprintf(stderr, "[feast] two-phase eig k=%lld: %d FP32 + %d FP64 sweeps\n", (long long)k, sw32, sw64);
    return true;
  }
  // FP64 Jacobi polish of the nearly diagonal k x k matrix H (ld k), vectors
  // into T2e: kPolishSweeps full sweeps, then while some off-diagonal entry
  // exceeds the threshold (1e-15 ||H||_F) and the entries that do link only
  // small index sets (at most kClusterMax, the groups of nearly equal diagonal
  // entries), each set is finished in shared memory (cluster_jacobi) instead
  // of by further sweeps, which would walk all k - 1 rounds to rotate a few
  // pairs.  Otherwise one more full sweep.  Returns the full sweeps taken.
  int polish(S* H, int64_t k) {
    const bool log = std::getenv("FEAST_LOG") != nullptr;
    int sweeps = 0, s1 = 0;
    // mixed path: the sweeps in double-float on the FP32 pipes (the diagonal
    // in FP64); the FP64 path keeps FP64 sweeps
    auto sweep = [&](S* Hm, int64_t km, S* Vm, double tol, int maxs, bool init) {
      if (o.prec != FEAST_PREC_F64 && d_dg)
        jacobi_eigh_df<S>(Hm, km, km, Vm, km, d_dg, tol, cw, ctx->num_sms, st, maxs, init);
      else
        jacobi_eigh<S>(Hm, km, km, Vm, km, tol, cw, ctx->num_sms, st, maxs, init);
    };
    sweep(H, k, T2e, 1e-15, kPolishSweeps, true);
    jacobi_status(&s1);
    sweeps += s1;
    if (!d_ccnt) {
      if (s1 >= kPolishSweeps) {
        sweep(H, k, T2e, 1e-15, kMaxSweeps, false);
        jacobi_status(&s1);
        sweeps += s1;
      }
      return sweeps;
    }
    std::vector<double> cn(k);
    col_norms2<S>(H, k, k, k, d_nrm, st);
    to_host(ctx, cn.data(), d_nrm, k);
    double fro2 = 0.0;
    for (double v : cn) fro2 += v;
    const double thr = 1e-15 * std::sqrt(fro2);
    std::vector<int> parent(k), list, setidx, setoff, swc;
    for (int pass = 0; pass < 16; ++pass) {
      // a hair above the kernels' threshold, so that a pair the scan reports
      // is one the Jacobi kernels rotate
      offdiag_scan<S>(H, k, k, thr * (1.0 + 1e-6), d_ccnt, d_clist, (int)ccap, st);
      int cnt = 0;
      to_host(ctx, &cnt, d_ccnt, 1);
      if (cnt == 0) return sweeps;
      bool sets_ok = cnt <= ccap;
      int nsets = 0, maxset = 0;
      std::vector<int> act;  // indices of the above-threshold pairs
      if (sets_ok) {
        list.resize(2 * (size_t)cnt);
        to_host(ctx, list.data(), d_clist, 2 * (int64_t)cnt);
        std::iota(parent.begin(), parent.end(), 0);
        auto find = [&](int x) {
          while (parent[x] != x) x = parent[x] = parent[parent[x]];
          return x;
        };
        for (int e = 0; e < cnt; ++e) {
          const int a = find(list[2 * e]), b = find(list[2 * e + 1]);
          if (a != b) parent[std::max(a, b)] = std::min(a, b);
        }
        // members of each set in ascending index order
        std::vector<int> root_of(k, -1), count;
        std::vector<char> used(k, 0);
        for (int e = 0; e < 2 * cnt; ++e) used[list[e]] = 1;
        for (int64_t i = 0; i < k; ++i)
          if (used[i]) act.push_back((int)i);
        std::vector<int> setid(k, -1);
        for (int64_t i = 0; i < k; ++i)
          if (used[i]) {
            const int r = find((int)i);
            if (root_of[r] < 0) {
              root_of[r] = nsets++;
              count.push_back(0);
            }
            setid[i] = root_of[r];
            ++count[setid[i]];
          }
        setoff.assign(nsets + 1, 0);
        for (int c = 0; c < nsets; ++c) {
          setoff[c + 1] = setoff[c] + count[c];
          maxset = std::max(maxset, count[c]);
        }
        sets_ok = maxset <= kClusterMax;
        if (sets_ok) {
          setidx.assign(setoff[nsets], 0);
          std::vector<int> fill(setoff.begin(), setoff.end() - 1);
          for (int64_t i = 0; i < k; ++i)
            if (setid[i] >= 0) setidx[fill[setid[i]]++] = (int)i;
        }
      }
      // a set too large for the shared-memory finish: one sweep restricted to
      // the indices of the above-threshold pairs (a sweep's cost is its
      // rounds, one per index); the entries between them and the other
      // indices are at most thr and stay as they are
      const int64_t ks = (int64_t)act.size();
      const bool restricted = !sets_ok && ks >= 2 && ks < k && Hsub != nullptr;
      if (log)
        fprintf(stderr, "[feast] FP64 polish k=%lld pass %d: %d pairs above threshold, %d sets, largest %d%s\n",
                (long long)k, pass, cnt, nsets, maxset,
                sets_ok ? "" : (restricted ? " -> sweep over the linked indices" : " -> full sweep"));
      if (sets_ok) {
        to_dev(ctx, d_cidx, setidx.data(), (int64_t)setidx.size());
        to_dev(ctx, d_coff, setoff.data(), (int64_t)nsets + 1);
        cluster_jacobi<S>(H, k, k, T2e, k, d_cidx, d_coff, nsets, thr, Ucl, d_csw, st);
        if (log) {
          swc.resize(nsets);
          to_host(ctx, swc.data(), d_csw, nsets);
          fprintf(stderr, "[feast] FP64 polish k=%lld: set sweeps max %d\n", (long long)k,
                  *std::max_element(swc.begin(), swc.end()));
        }
      } else if (restricted) {
        to_dev(ctx, d_cidx, act.data(), ks);
        gather_sub<S>(Hsub, H, k, d_cidx, ks, st);
        col_norms2<S>(Hsub, ks, ks, ks, d_nrm, st);
        std::vector<double> sn(ks);
        to_host(ctx, sn.data(), d_nrm, ks);
        double sub2 = 0.0;
        for (double v : sn) sub2 += v;
        // the same absolute threshold as the whole matrix's
        const double tol_sub = sub2 > 0.0 ? thr / std::sqrt(sub2) : 1e-15;
        sweep(Hsub, ks, Vsub, tol_sub, 1, true);
        jacobi_status(&s1);
        sweeps += s1;
        scatter_sub<S>(H, k, Hsub, d_cidx, ks, st);
        gather_cols<S>(Tsub, k, T2e, k, k, d_cidx, ks, nullptr, st);
        gemm_simple<S, S, S>(k, ks, ks, C1(1.0), Tsub, k, OP_N, Vsub, ks, OP_N, C1(0.0), Tsub2, k, st);
        scatter_cols<S>(T2e, k, Tsub2, k, k, d_cidx, ks, st);
      } else {
        sweep(H, k, T2e, 1e-15, 1, false);
        jacobi_status(&s1);
        sweeps += s1;
      }
    }
    // still not below the threshold: finish with full sweeps
    sweep(H, k, T2e, 1e-15, kMaxSweeps, false);
    jacobi_status(&s1);
    return sweeps + s1;
  }
  void eig(S* H, int64_t k, std::vector<double>& ev) {
    const bool log = std::getenv("FEAST_LOG") != nullptr;
    double t0 = 0.0;
    if (log) {
      sync(ctx);
      t0 = now_ms();
    }
    if (!(k >= kEigMixedMin && H32 && d_bjrot && k <= kmax && eig_two_phase(H, k, &last_sweeps))) {
      jacobi_eigh<S>(H, k, k, Vk, k, 1e-15, cw, ctx->num_sms, st);
      jacobi_status(&last_sweeps);
    }
    get_diag<S>(H, k, k, d_lam, st);
    ev.resize(k);
    to_host(ctx, ev.data(), d_lam, k);
    if (log) fprintf(stderr, "[feast] jacobi k=%lld sweeps=%d %.1f ms\n", (long long)k, last_sweeps, now_ms() - t0);
  }
  // Gram-eigendecomposition route (Sect. II-A): X^H X = V S^2 V^H, keep
  // s^2 >= trunc s_1^2, U = X V S^{-1}, then one Cholesky-QR pass.
  int64_t gram_eig_orth(const S* X, int64_t nr, int64_t k, S* Qout, S* tmp, double trunc) {
    mm_reduce(k, k, nr, X, nr, OP_C, X, nr, OP_N, Gs, k);
    hermitize<S>(Gs, k, k, st);
    std::vector<double> s2;
    eig(Gs, k, s2);
    std::vector<int> ord(k);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return s2[a] > s2[b]; });
    if (!(s2[ord[0]] > 0.0)) return 0;
    std::vector<int> keep;
    std::vector<double> sc;
    for (int i : ord)
      if (s2[i] >= trunc * s2[ord[0]]) {
        keep.push_back(i);
        sc.push_back(1.0 / std::sqrt(s2[i]));
      }
    const int64_t r = (int64_t)keep.size();
    to_dev(ctx, d_idx, keep.data(), r);
    to_dev(ctx, d_scale, sc.data(), r);
    gather_cols<S>(Cs, k, Vk, k, k, d_idx, r, d_scale, st);
    mm(nr, r, k, C1(1.0), X, nr, OP_N, Cs, k, OP_N, C1(0.0), tmp, nr);
    if (!cholqr_once(tmp, nr, r, Qout)) return 0;
    return r;
  }
  // Cholesky-QR twice; Gram route on breakdown.  Returns the rank (0 = failure).
  int64_t orthonormalize(const S* X, int64_t nr, int64_t k, S* Qout, S* tmp) {
    bool ok = false;
    phase("CholQR2", [&] { ok = cholqr_once(X, nr, k, tmp) && cholqr_once(tmp, nr, k, Qout); });
    if (ok) return k;
    return gram_eig_orth(X, nr, k, Qout, tmp, 1e-12);
  }

  // ---- Rayleigh-Ritz ----
  // W = A Q, A' = Q^H W (ld kmax) for the first k columns of Qb
  void rr_project(int64_t k) {
    phase("RR A*Q", [&] { apply_A(Qb, k, Wb); });
    phase("RR Q^H W", [&] {
      mm_reduce(k, k, n, Qb, n, OP_C, Wb, n, OP_N, Ar0, kmax);
      hermitize<S>(Ar0, k, kmax, st);
    });
  }
  // diagonalise A'[0:k, 0:k]: lam (ascending), Xr = Q V, AXr = W V, res
  void rr_solve(int64_t k) {
    ++rr_passes;
    rr_k_sum += (double)k;
    rr_k3_sum += (double)k * (double)k * (double)k;
    copy_matrix<S>(Ar, k, Ar0, kmax, k, k, st);
    std::vector<double> ev;
    phase("Jacobi (RR)", [&] { eig(Ar, k, ev); });
    std::vector<int> ord(k);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return ev[a] < ev[b]; });
    lam.resize(k);
    for (int64_t i = 0; i < k; ++i) lam[i] = ev[ord[i]];
    to_dev(ctx, d_idx, ord.data(), k);
    phase("RR X = QV, AX = WV", [&] {
      gather_cols<S>(Cs, k, Vk, k, k, d_idx, k, nullptr, st);
      mm(n, k, k, C1(1.0), Qb, n, OP_N, Cs, k, OP_N, C1(0.0), Xr, n);
      mm(n, k, k, C1(1.0), Wb, n, OP_N, Cs, k, OP_N, C1(0.0), AXr, n);
      to_dev(ctx, d_lam, lam.data(), k);
      resid_norms2<S>(AXr, Xr, n, k, n, d_lam, d_nrm, st);
    });
    res.resize(k);
    to_host(ctx, res.data(), d_nrm, k);
    for (auto& r : res) r = std::sqrt(r) / anorm;
  }

  // ---- drivers ----
  struct Out {
    int status = 0;
    std::vector<int> idx;       // returned pairs: columns of `src`, ascending lambda
    std::vector<double> ev, rs; // their eigenvalues and relative residuals
    const S* src = nullptr;     // device matrix holding the eigenvectors (ld n)
    int iterations = 0, filters = 0, m_expected = -1;
    std::vector<double> hist;
  };
  // Deferred stopping test of a round whose selected pairs are the columns of
  // the block that the next filter takes: those inside I with filter response
  // mu_k = Re(x_k^H rho(A) x_k) > 1/2 must all have converged (a mixture of
  // eigenvectors outside I has mu < 1/2; rho > 1/2 exactly inside I).
  struct Pending {
    bool valid = false;
    std::vector<int> in_cols;        // columns (within the block) of the pairs inside I
    std::vector<double> ev, rs;      // per column of the block
  };
  bool response_test(const Pending& pd, const S* Xb, const S* Xfb, int64_t cols, double tol, Out& out) {
    col_dots_re<S>(Xb, Xfb, n, cols, n, d_nrm, st);
    std::vector<double> mu(cols);
    to_host(ctx, mu.data(), d_nrm, cols);
    std::vector<int> keep;
    for (int c : pd.in_cols)
      if (mu[c] > 0.5) keep.push_back(c);
    if (std::getenv("FEAST_LOG")) {
      int unconv = 0;
      double worst = 0.0, mu_min = 1.0;
      for (int c : keep) {
        if (!(pd.rs[c] <= tol)) ++unconv;
        worst = std::max(worst, pd.rs[c]);
        mu_min = std::min(mu_min, mu[c]);
      }
      fprintf(stderr, "[feast] response test: %zu in-I pairs, %zu with mu > 1/2 (min mu %.6f), %d unconverged, "
              "max residual %.2e\n", pd.in_cols.size(), keep.size(), mu_min, unconv, worst);
    }
    if (keep.empty()) return false;
    for (int c : keep)
      if (!(pd.rs[c] <= tol)) return false;
    std::sort(keep.begin(), keep.end(), [&](int a, int b) { return pd.ev[a] < pd.ev[b] || (pd.ev[a] == pd.ev[b] && a < b); });
    out.idx = keep;
    out.ev.clear();
    out.rs.clear();
    for (int c : keep) {
      out.ev.push_back(pd.ev[c]);
      out.rs.push_back(pd.rs[c]);
    }
    out.src = Xb;
    return true;
  }
  Pending make_pending(const std::vector<int>& sel, double tol) {
    Pending pd;
    bool any_conv = false;
    for (size_t c = 0; c < sel.size(); ++c) {
      pd.ev.push_back(lam[sel[c]]);
      pd.rs.push_back(res[sel[c]]);
      if (in_interval(lam[sel[c]], lmin, lmax)) {
        pd.in_cols.push_back((int)c);
        any_conv = any_conv || res[sel[c]] <= tol;
      }
    }
    pd.valid = any_conv;
    return pd;
  }

  // mixed: skip the FP64-accurate refinement of the next filter while the
  // residual is above o.refine_switch and still falling at least tenfold per
  // iteration (a filter accurate to FP32 cannot be what limits it then)
  void update_refine(const std::vector<double>& hist) {
    if (o.prec == FEAST_PREC_F64 || o.refine_switch <= 0.0) { refine_now = true; return; }
    const double r = hist.back();
    const double prev = hist.size() >= 2 ? hist[hist.size() - 2] : INFINITY;
    refine_now = !(r > o.refine_switch && r < 0.1 * prev);
  }

  std::vector<int> in_sorted(const std::vector<int>& cand) {
    std::vector<int> v;
    for (int i : cand)
      if (in_interval(lam[i], lmin, lmax)) v.push_back(i);
    return v;
  }
  void finish(Out& out, std::vector<int> ins) {
    std::sort(ins.begin(), ins.end(), [&](int a, int b) { return lam[a] < lam[b] || (lam[a] == lam[b] && a < b); });
    out.idx = ins;
    out.ev.clear();
    out.rs.clear();
    for (int i : ins) {
      out.ev.push_back(lam[i]);
      out.rs.push_back(res[i]);
    }
    out.src = Xr;
  }
  std::vector<int> lowest_residual(std::vector<int> v, int m) {
    std::stable_sort(v.begin(), v.end(), [&](int a, int b) {
      return res[a] < res[b] || (res[a] == res[b] && (lam[a] < lam[b] || (lam[a] == lam[b] && a < b)));
    });
    if ((int)v.size() > m) v.resize(std::max(m, 0));
    return v;
  }
  double max_res(const std::vector<int>& v) {
    double r = 0.0;
    for (int i : v) r = std::max(r, res[i]);
    return v.empty() ? INFINITY : r;
  }

  Out run_plain(S* X, int m0, double tol) {
    Out out;
    int64_t kx = m0;
    S* Xf = T2;
    Pending pd;
    for (int it = 1; it <= o.max_iter; ++it) {
      filter(X, kx, Xf);
      ++out.filters;
      // response_stop: the previous round's in-I pairs with filter response
      // above 1/2 (read off this filter) have all converged
      if (pd.valid) {
        if (response_test(pd, X, Xf, kx, tol, out)) {
          out.iterations = it - 1;
          return out;
        }
        pd.valid = false;
      }
      const int64_t k = orthonormalize(Xf, n, kx, Qb, T1);
      if (k == 0) throw FeastError{FEAST_ERR_ORTH};
      rr_project(k);
      rr_solve(k);
      std::vector<int> all(k);
      std::iota(all.begin(), all.end(), 0);
      std::vector<int> ins = in_sorted(all);
      const double r = max_res(ins);
      out.hist.push_back(r);
      update_refine(out.hist);
      out.iterations = it;
      if ((!ins.empty() && r <= tol) || (ins.empty() && it >= 2)) {
        finish(out, ins);
        return out;
      }
      copy_matrix<S>(X, n, Xr, n, n, k, st);
      kx = k;
      if (o.response_stop) pd = make_pending(all, tol);
    }
    std::vector<int> all(lam.size());
    std::iota(all.begin(), all.end(), 0);
    finish(out, in_sorted(all));
    out.status = FEAST_WARN_MAXITER;
    return out;
  }

  // block QR of the window (see the XFEAST reading): returns k
  int64_t block_qr(const std::vector<S*>& blocks, int64_t mb) {
    int64_t kq = 0;
    std::vector<double> nr2(mb);
    for (S* B : blocks) {
      col_norms2<S>(B, n, mb, n, d_nrm, st);
      to_host(ctx, nr2.data(), d_nrm, mb);
      double bn = 0.0;
      for (double v : nr2) bn = std::max(bn, std::sqrt(v));
      if (bn == 0.0) continue;
      S* P = T1;
      copy_matrix<S>(P, n, B, n, n, mb, st);
      if (kq > 0)
        for (int rep = 0; rep < 2; ++rep) {
          mm_reduce(kq, mb, n, Qb, n, OP_C, P, n, OP_N, Cs2, kq);
          mm(n, mb, kq, C1(-1.0), Qb, n, OP_N, Cs2, kq, OP_N, C1(1.0), P, n);
        }
      mm_reduce(mb, mb, n, P, n, OP_C, P, n, OP_N, Gs, mb);
      hermitize<S>(Gs, mb, mb, st);
      std::vector<double> s2;
      eig(Gs, mb, s2);
      std::vector<int> ord(mb);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return s2[a] < s2[b]; });
      std::vector<int> keep;
      std::vector<double> sc;
      const double thr = (1e-13 * bn) * (1e-13 * bn);
      for (int i : ord)
        if (s2[i] >= thr) {
          keep.push_back(i);
          sc.push_back(1.0 / std::sqrt(s2[i]));
        }
      const int64_t r = (int64_t)keep.size();
      if (r == 0) continue;
      to_dev(ctx, d_idx, keep.data(), r);
      to_dev(ctx, d_scale, sc.data(), r);
      gather_cols<S>(Cs, mb, Vk, mb, mb, d_idx, r, d_scale, st);
      S* U = T2;
      mm(n, r, mb, C1(1.0), P, n, OP_N, Cs, mb, OP_N, C1(0.0), U, n);
      if (kq > 0) {
        mm_reduce(kq, r, n, Qb, n, OP_C, U, n, OP_N, Cs2, kq);
        mm(n, r, kq, C1(-1.0), Qb, n, OP_N, Cs2, kq, OP_N, C1(1.0), U, n);
      }
      if (!cholqr_once(U, n, r, Qb + kq * n)) throw FeastError{FEAST_ERR_ORTH};
      kq += r;
    }
    return kq;
  }

  Out run_xfeast(S* X0, int m0, double tol, int s) {
    Out out;
    std::vector<S*> ring(s);
    for (int i = 0; i < s; ++i) ring[i] = dalloc<S>(ctx, n * m0);
    // step 0: X_0 with unit columns, then X_i = rho(A)^i X_0
    col_norms2<S>(X0, n, m0, n, d_nrm, st);
    std::vector<double> nr2(m0), sc(m0);
    std::vector<int> iden(m0);
    to_host(ctx, nr2.data(), d_nrm, m0);
    for (int j = 0; j < m0; ++j) {
      sc[j] = nr2[j] > 0 ? 1.0 / std::sqrt(nr2[j]) : 1.0;
      iden[j] = j;
    }
    to_dev(ctx, d_scale, sc.data(), m0);
    to_dev(ctx, d_idx, iden.data(), m0);
    gather_cols<S>(ring[0], n, X0, n, n, d_idx, m0, d_scale, st);
    for (int i = 1; i < s; ++i) {
      filter(ring[i - 1], m0, ring[i]);
      ++out.filters;
    }
    S* Xsel = dalloc<S>(ctx, n * m0);
    std::vector<int> ins;
    for (int it = 1; it <= o.max_iter; ++it) {
      const int64_t k = block_qr(ring, m0);                       // step 1
      if (k == 0) throw FeastError{FEAST_ERR_ORTH};
      rr_project(k);                                              // step 2(i)
      rr_solve(k);
      std::vector<int> sel = select_pairs(lam, res, lmin, lmax, m0);   // step 2(ii)
      ins = in_sorted(sel);                                       // step 3
      const double r = max_res(ins);
      out.hist.push_back(r);
      update_refine(out.hist);
      out.iterations = it;
      if ((!ins.empty() && r <= tol) || (ins.empty() && it >= 2)) {
        finish(out, ins);
        return out;
      }
      if (it == o.max_iter) break;
      const int64_t ms = (int64_t)sel.size();
      to_dev(ctx, d_idx, sel.data(), ms);
      gather_cols<S>(Xsel, n, Xr, n, n, d_idx, ms, nullptr, st);
      S* oldest = ring[0];
      filter(Xsel, ms, oldest);                                   // step 4(i)
      ++out.filters;
      if (o.response_stop) {
        Pending pd = make_pending(sel, tol);
        if (pd.valid && response_test(pd, Xsel, oldest, ms, tol, out)) return out;
      }
      std::rotate(ring.begin(), ring.begin() + 1, ring.end());    // step 4(ii)
    }
    finish(out, ins);
    out.status = FEAST_WARN_MAXITER;
    return out;
  }

  Out run_rfeast(S* X, int m0, double tol, int s) {
    Out out;
    S* Xf = dalloc<S>(ctx, n * m0);
    S* AXs = dalloc<S>(ctx, n * m0);
    std::vector<int> ins;
    int64_t kx = m0;
    Pending pd;
    for (int it = 1; it <= o.max_iter; ++it) {
      filter(X, kx, Xf);                                          // step 1
      ++out.filters;
      if (pd.valid) {
        if (response_test(pd, X, Xf, kx, tol, out)) {
          out.iterations = it - 1;
          return out;
        }
        pd.valid = false;
      }
      int64_t k = orthonormalize(Xf, n, kx, Qb, T1);
      if (k == 0) throw FeastError{FEAST_ERR_ORTH};
      rr_project(k);
      int mexp = 0;
      std::vector<int> sel;
      for (int j = 1; j <= s; ++j) {
        rr_solve(k);
        if (j == 1) {
          mexp = 0;
          for (double v : lam) mexp += in_interval(v, lmin, lmax);
        }
        sel = select_pairs(lam, res, lmin, lmax, m0);
        const int64_t ms = (int64_t)sel.size();
        to_dev(ctx, d_idx, sel.data(), ms);
        gather_cols<S>(X, n, Xr, n, n, d_idx, ms, nullptr, st);
        kx = ms;
        if (j < s && k + ms <= kmax) {
          gather_cols<S>(AXs, n, AXr, n, n, d_idx, ms, nullptr, st);
          std::vector<double> ls(ms);
          for (int64_t i = 0; i < ms; ++i) ls[i] = lam[sel[i]];
          to_dev(ctx, d_lam, ls.data(), ms);
          S* R = T1;
          ritz_residual<S>(R, AXs, X, n, ms, n, d_lam, st);
          col_norms2<S>(R, n, ms, n, d_nrm, st);
          std::vector<double> nr2(ms), sc(ms);
          to_host(ctx, nr2.data(), d_nrm, ms);
          // step 2(iii): the residual of every selected pair (the paper), or
          // with rfeast_expand = 1 only of those that have not converged: a
          // converged pair's residual is at the rounding level of A X, and its
          // normalised direction would add spurious Ritz pairs, not information
          std::vector<int> act;
          for (int64_t i = 0; i < ms; ++i)
            if (nr2[i] > 0 && (o.rfeast_expand == 0 || res[sel[i]] > tol)) act.push_back((int)i);
          const int64_t ma = (int64_t)act.size();
          if (std::getenv("FEAST_LOG"))
            fprintf(stderr, "[feast] rfeast it %d j %d: %lld of %lld residuals appended\n", it, j, (long long)ma,
                    (long long)ms);
          if (ma == 0) break;  // nothing to append (every selected pair converged)
          for (int64_t c = 0; c < ma; ++c) sc[c] = 1.0 / std::sqrt(nr2[act[c]]);
          to_dev(ctx, d_scale, sc.data(), ma);
          to_dev(ctx, d_idx, act.data(), ma);
          gather_cols<S>(AXs, n, T1, n, n, d_idx, ma, d_scale, st);
          R = AXs;
          // continue in the Ritz basis of this pass (same span): Q <- X, W <- A X,
          // A' <- diag(lambda), so the next Jacobi starts from a matrix whose
          // leading block is already diagonal
          copy_matrix<S>(Qb, n, Xr, n, n, k, st);
          copy_matrix<S>(Wb, n, AXr, n, n, k, st);
          to_dev(ctx, d_lam, lam.data(), k);
          set_diag<S>(Ar0, k, kmax, d_lam, st);
          phase("RFEAST R - Q Q^H R", [&] {
            for (int rep = 0; rep < 2; ++rep) {
              mm_reduce(k, ma, n, Qb, n, OP_C, R, n, OP_N, Cs2, k);
              mm(n, ma, k, C1(-1.0), Qb, n, OP_N, Cs2, k, OP_N, C1(1.0), R, n);
            }
          });
          S* U = Qb + k * n;
          const int64_t ku = orthonormalize(R, n, ma, U, T2);
          if (ku == 0) break;  // nothing new to append
          S* WU = Wb + k * n;
          phase("RR A*Q", [&] { apply_A(U, ku, WU); });
          // A' blocks: [Q U]^H A [Q U] from the new columns only
          phase("RFEAST A' blocks", [&] {
            mm_reduce(k, ku, n, Qb, n, OP_C, WU, n, OP_N, Ar0 + k * kmax, kmax);
            mm_reduce(ku, k, n, U, n, OP_C, Wb, n, OP_N, Ar0 + k, kmax);
            mm_reduce(ku, ku, n, U, n, OP_C, WU, n, OP_N, Ar0 + k + k * kmax, kmax);
            hermitize<S>(Ar0, k + ku, kmax, st);
          });
          k += ku;
        } else if (j < s) {
          break;
        }
      }
      out.m_expected = mexp;
      const std::vector<int> all_in = in_sorted(sel);
      ins = lowest_residual(all_in, mexp);
      const double r = max_res(ins);
      if (std::getenv("FEAST_LOG")) {
        std::vector<double> rr;
        for (int i : all_in) rr.push_back(res[i]);
        std::sort(rr.begin(), rr.end());
        fprintf(stderr, "[feast] rfeast it %d: k %lld, m_exp %d, in-I selected %zu, max over m_exp %.2e, in-I residuals:",
                it, (long long)k, mexp, all_in.size(), r);
        for (size_t q = rr.size() > 8 ? rr.size() - 8 : 0; q < rr.size(); ++q) fprintf(stderr, " %.1e", rr[q]);
        fprintf(stderr, "\n");
      }
      out.hist.push_back(r);
      update_refine(out.hist);
      out.iterations = it;
      if ((!ins.empty() && r <= tol) || (ins.empty() && it >= 2)) {
        finish(out, ins);
        return out;
      }
      if (o.response_stop) pd = make_pending(sel, tol);
    }
    finish(out, ins);
    out.status = FEAST_WARN_MAXITER;
    return out;
  }
};

int check_common(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double lmin, double lmax,
                 int n_c) {
  if (!ctx || !A || n < 1 || lda < n || n_c < 1 || n_c > 256) return FEAST_ERR_ARG;
  if (dtype != FEAST_R64 && dtype != FEAST_C128) return FEAST_ERR_ARG;
  if (!std::isfinite(lmin) || !std::isfinite(lmax) || !(lmin < lmax)) return FEAST_ERR_ARG;
  if (n > INT32_MAX / 2) return FEAST_ERR_ARG;
  return FEAST_OK;
}

template <typename Fn>
int guarded(feast_ctx* ctx, Fn&& fn) {
  try {
    int r = fn();
    return r;
  } catch (const FeastError& e) {
    if (ctx) cudaStreamSynchronize(ctx->stream);
    cudaGetLastError();
    return e.code;
  } catch (const CudaFailure& e) {
    if (e.err == cudaErrorMemoryAllocation) { cudaGetLastError(); return FEAST_ERR_NOMEM; }
    return FEAST_ERR_CUDA;
  } catch (const std::bad_alloc&) {
    cudaGetLastError();
    return FEAST_ERR_NOMEM;
  }
}

template <typename S>
int check_finite_dev(feast_ctx* ctx, const S* X, int64_t n, int64_t m, int64_t ld) {
  int* flag = dalloc<int>(ctx, 1);
  FEAST_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  check_finite<S>(X, n, m, ld, flag, ctx->stream);
  int h = 0;
  to_host(ctx, &h, flag, 1);
  return h ? FEAST_ERR_NONFINITE : FEAST_OK;
}

template <typename S>
int solve_t(feast_ctx* ctx, const S* A, int64_t n, int64_t lda, double lmin, double lmax, int m0, int n_c,
            double tol, const feast_opts& o, double* evals, S* evecs, double* resout, int* m_found, int* iters,
            feast_stats* stats) {
  const double t0 = now_ms();
  ctx->arena.reset();
  if (int r = check_finite_dev<S>(ctx, A, n, n, lda)) return r;
  Solver<S> sv(ctx, A, n, lda, lmin, lmax, n_c, o);
  const int s = std::max(1, o.s);
  const int64_t kmax = (o.variant == FEAST_PLAIN) ? m0 : (int64_t)s * m0;
  sv.alloc_common(kmax, m0);
  sv.alloc_rr();
  sv.alloc_filter(m0);
  sv.alloc_factors();
  sv.anorm = o.anorm > 0 ? o.anorm : sv.estimate_norm();
  if (!(sv.anorm > 0)) sv.anorm = 1.0;
  sv.refine_now = !(o.prec != FEAST_PREC_F64 && o.refine_switch > 0.0);
  S* X = dalloc<S>(ctx, n * m0);
  if (o.x0) {
    copy_matrix<S>(X, n, (const S*)o.x0, n, n, m0, ctx->stream);
    if (int r = check_finite_dev<S>(ctx, X, n, m0, n)) return r;
  } else {
    random_normal<S>(X, n, m0, n, o.seed, ctx->stream);
  }
  sync(ctx);
  kernel_timer_begin();
  const double tf0 = now_ms();
  sv.factor();
  sync(ctx);
  const double tf1 = now_ms();
  typename Solver<S>::Out out;
  if (o.variant == FEAST_XFEAST) out = sv.run_xfeast(X, m0, tol, s);
  else if (o.variant == FEAST_RFEAST) out = sv.run_rfeast(X, m0, tol, s);
  else out = sv.run_plain(X, m0, tol);
  const int mf = (int)out.idx.size();
  const std::vector<double>& ev = out.ev;
  const std::vector<double>& rs = out.rs;
  if (mf > 0) {
    to_dev(ctx, sv.d_idx, out.idx.data(), mf);
    gather_cols<S>(evecs, n, out.src, n, n, sv.d_idx, mf, nullptr, ctx->stream);
  }
  sync(ctx);
  for (int i = 0; i < mf; ++i) {
    evals[i] = ev[i];
    resout[i] = rs[i];
  }
  *m_found = mf;
  *iters = out.iterations;
  feast_stats st{};
  st.iterations = out.iterations;
  st.filters = out.filters;
  st.refine_steps = sv.refine_steps;
  st.m_expected = out.m_expected;
  st.rr_passes = sv.rr_passes;
  st.rr_k_sum = sv.rr_k_sum;
  st.rr_k3_sum = sv.rr_k3_sum;
  st.factor_ms = tf1 - tf0;
  st.filter_ms = sv.filter_ms;
  kernel_timer_end(TIMER_REFINE_GEMM, &st.refine_gemm_ms, &st.refine_gemm_mac, &st.refine_gemm_launches);
  kernel_timer_end(TIMER_CGEMM, &st.cgemm_ms, &st.cgemm_flop, &st.cgemm_launches);
  kernel_timer_end(TIMER_TCGEMM, &st.tcgemm_ms, &st.tcgemm_flop, &st.tcgemm_launches);
  sv.check_oz_status();
  st.total_ms = now_ms() - t0;
  st.max_residual = 0.0;
  for (double r : rs) st.max_residual = std::max(st.max_residual, r);
  for (size_t i = 0; i < out.hist.size() && i < 128; ++i) st.history[i] = out.hist[i];
  ctx->last = st;
  if (stats) *stats = st;
  if (sv.profile) {
    fprintf(stderr, "[feast] phases (ms):");
    for (auto& p : sv.phases) fprintf(stderr, " %s=%.1f", p.first, p.second);
    fprintf(stderr, " factor=%.1f total=%.1f\n", st.factor_ms, st.total_ms);
  }
  return out.status;
}

// ---------------------------------------------------------------------------
// general (non-Hermitian) matrices: FEAST on the whole circle |z - c| = r
// (Sect. I names the extension; the reading: 2 n_c Gauss nodes, the filter
// without the Hermitian mirror, Rayleigh-Ritz on an orthonormal basis with
// the reduced general eigenproblem by Schur form)
// ---------------------------------------------------------------------------
// Upper half-circle nodes of the Hermitian rule, then their mirror images
// c + r e^{-i theta_j} with weights (omega_j / 4) r e^{-i theta_j}.
void circle(c128 center, double r, int nc, std::vector<c128>& z, std::vector<c128>& w) {
  std::vector<double> t, om;
  gauss_legendre(nc, t, om);
  z.resize(2 * nc);
  w.resize(2 * nc);
  for (int j = 0; j < nc; ++j) {
    const double th = 0.5 * M_PI * (1.0 - t[j]), cs = std::cos(th), sn = std::sin(th);
    z[j] = c128{center.re + r * cs, center.im + r * sn};
    w[j] = c128{0.25 * om[j] * r * cs, 0.25 * om[j] * r * sn};
    z[nc + j] = c128{center.re + r * cs, center.im - r * sn};
    w[nc + j] = c128{0.25 * om[j] * r * cs, -0.25 * om[j] * r * sn};
  }
}

struct General {
  feast_ctx* ctx;
  cudaStream_t st;
  int64_t n = 0, mmax = 0;
  int nc = 0, E = 0;
  c128* A = nullptr;  // complex copy of the input, ld n
  c128* M = nullptr;  // E shifted factors
  int32_t *ipiv = nullptr, *perm = nullptr;
  PanelWork pw{};
  CoopWork cw{};
  c128* d_w = nullptr;
  c128* Wsol = nullptr;  // E n x mmax solutions
  c128 *G = nullptr, *Ri = nullptr, *Vg = nullptr, *Cg = nullptr, *part = nullptr, *tmp = nullptr;
  c128 *Q = nullptr, *Wq = nullptr, *Hr = nullptr, *Zs = nullptr, *Ys = nullptr, *Vr = nullptr;
  c128 *X = nullptr, *AX = nullptr, *d_lam = nullptr;
  double *d_nrm = nullptr, *d_scale = nullptr;
  int* d_idx = nullptr;
  int* d_info = nullptr;
  int64_t part_elems = 0;
  double anorm = 1.0;
  int last_sweeps = 0;

  General(feast_ctx* c) : ctx(c), st(c->stream) {}

  // scratch of the k x k steps, k <= kmax
  void setup_small(int64_t kmax) {
    mmax = kmax;
    cw = coop_work_carve(ctx->arena.alloc(coop_work_bytes(kmax, ctx->num_sms)), kmax, ctx->num_sms);
    const int64_t kk = kmax * kmax;
    G = dalloc<c128>(ctx, kk);
    Ri = dalloc<c128>(ctx, kk);
    Vg = dalloc<c128>(ctx, kk);
    Cg = dalloc<c128>(ctx, kk);
    Hr = dalloc<c128>(ctx, kk);
    Zs = dalloc<c128>(ctx, kk);
    Ys = dalloc<c128>(ctx, kk);
    Vr = dalloc<c128>(ctx, kk);
    part_elems = 32 * kk;
    part = dalloc<c128>(ctx, part_elems);
    d_lam = dalloc<c128>(ctx, kmax);
    d_nrm = dalloc<double>(ctx, kmax);
    d_scale = dalloc<double>(ctx, kmax);
    d_idx = dalloc<int>(ctx, kmax);
    d_info = dalloc<int>(ctx, 2);
  }
  // A (dtype R64 or C128, ld lda) -> complex copy (ld n)
  void setup_matrix(const void* Ain, int dtype, int64_t n_, int64_t lda) {
    n = n_;
    A = dalloc<c128>(ctx, n * n);
    if (dtype == FEAST_R64) convert_matrix<c128, double>(A, n, (const double*)Ain, lda, n, n, st);
    else copy_matrix<c128>(A, n, (const c128*)Ain, lda, n, n, st);
  }
  // n x mmax blocks of the Rayleigh-Ritz step
  void setup_blocks() {
    tmp = dalloc<c128>(ctx, n * mmax);
    Q = dalloc<c128>(ctx, n * mmax);
    Wq = dalloc<c128>(ctx, n * mmax);
    X = dalloc<c128>(ctx, n * mmax);
    AX = dalloc<c128>(ctx, n * mmax);
  }
  // ||A||_2 by 40 power iterations of A^H A from ones / sqrt(n)
  double norm_estimate() {
    c128* v = dalloc<c128>(ctx, n);
    c128* u = dalloc<c128>(ctx, n);
    c128* wv = dalloc<c128>(ctx, n);
    double* nr = dalloc<double>(ctx, 1);
    std::vector<c128> h(n, c128{1.0 / std::sqrt((double)n), 0.0});
    to_dev(ctx, v, h.data(), n);
    double est = 0.0;
    for (int it = 0; it < 40; ++it) {
      gemm_simple<c128, c128, c128>(n, 1, n, C1(1.0), A, n, OP_N, v, n, OP_N, C1(0.0), u, n, st);
      gemm_simple<c128, c128, c128>(n, 1, n, C1(1.0), A, n, OP_C, u, n, OP_N, C1(0.0), wv, n, st);
      col_norms2<c128>(wv, n, 1, n, nr, st);
      double nw2 = 0.0;
      to_host(ctx, &nw2, nr, 1);
      const double nw = std::sqrt(nw2);
      if (!(nw > 0.0)) return 0.0;
      est = std::sqrt(nw);
      const double inv = 1.0 / nw;
      to_dev(ctx, d_scale, &inv, 1);
      copy_matrix<c128>(v, n, wv, n, n, 1, st);
      scale_cols<c128>(v, n, 1, n, d_scale, st);
    }
    return est;
  }
  void factor(c128 center, double r, int nc_) {
    nc = nc_;
    E = 2 * nc;
    std::vector<c128> z, w;
    circle(center, r, nc, z, w);
    d_w = dalloc<c128>(ctx, E);
    c128* dz = dalloc<c128>(ctx, E);
    to_dev(ctx, d_w, w.data(), E);
    to_dev(ctx, dz, z.data(), E);
    M = dalloc<c128>(ctx, (int64_t)E * n * n);
    ipiv = dalloc<int32_t>(ctx, (int64_t)E * n);
    perm = dalloc<int32_t>(ctx, (int64_t)E * n);
    const int pmax = std::max(1, ctx->num_sms * 8);
    pw = panel_work_carve(ctx->arena.alloc(panel_work_bytes(E, pmax, sizeof(c128))), E, pmax, sizeof(c128));
    Wsol = dalloc<c128>(ctx, (int64_t)E * n * mmax);
    form_shifted<c128, c128>(M, n, n, n * n, E, A, n, dz, st);
    lu_factor_batched<c128>(M, n, n, n * n, E, ipiv, perm, pw, ctx->num_sms, st);
    int status = 0;
    std::vector<int> zp(E);
    to_host(ctx, &status, pw.status, 1);
    to_host(ctx, zp.data(), pw.zero_pivot, E);
    if (status == DEV_BARRIER_TIMEOUT) throw FeastError{FEAST_ERR_TIMEOUT};
    for (int v : zp)
      if (v) throw FeastError{FEAST_ERR_SINGULAR};
  }
  // Y = sum_k w_k (z_k I - A)^{-1} Xin (n x m)
  void filter(const c128* Xin, int64_t m, c128* Y) {
    const int64_t nm = n * m;
    permute_in<c128, c128>(Wsol, nm, Xin, n, 0, n, m, perm, E, false, st);
    lu_solve_batched<c128>(M, n, n, n * n, E, Wsol, m, nm, false, st, nullptr, nullptr, ctx->num_sms);
    weighted_sum(Y, Wsol, nm, E, d_w, st);
  }
  // C (r x c) = X^H Y with the long reduction over n split
  void reduce(int64_t r, int64_t c, const c128* Xm, const c128* Ym, c128* C) {
    int ks = (int)std::max<int64_t>(1, std::min<int64_t>(32, n / 256));
    while (ks > 1 && (int64_t)ks * r * c > part_elems) --ks;
    gemm_simple<c128, c128, c128>(r, c, n, C1(1.0), Xm, n, OP_C, Ym, n, OP_N, C1(0.0), C, r, st, ks,
                                  ks > 1 ? (void*)part : nullptr);
  }
  bool cholqr_once(const c128* Xm, int64_t k, c128* Qout) {
    reduce(k, k, Xm, Xm, G);
    hermitize<c128>(G, k, k, st);
    cholesky_upper<c128>(G, k, k, cw, ctx->num_sms, st);
    int info = 0, status = 0;
    to_host(ctx, &info, cw.info, 1);
    to_host(ctx, &status, cw.status, 1);
    if (status == DEV_BARRIER_TIMEOUT) throw FeastError{FEAST_ERR_TIMEOUT};
    if (info != 0) return false;
    tri_inverse_upper<c128>(G, k, k, Ri, k, st);
    gemm_simple<c128, c128, c128>(n, k, k, C1(1.0), Xm, n, OP_N, Ri, k, OP_N, C1(0.0), Qout, n, st);
    return true;
  }
  // orthonormal basis of span(Y) (n x k): Cholesky-QR twice, else the Gram
  // eigendecomposition route (keep sigma^2 >= 1e-12 sigma_1^2, then one
  // Cholesky-QR pass); returns the rank
  int64_t orth(const c128* Y, int64_t k, c128* Qout) {
    if (cholqr_once(Y, k, tmp) && cholqr_once(tmp, k, Qout)) return k;
    reduce(k, k, Y, Y, G);
    hermitize<c128>(G, k, k, st);
    jacobi_eigh<c128>(G, k, k, Vg, k, 1e-15, cw, ctx->num_sms, st);
    int status = 0;
    to_host(ctx, &status, cw.status, 1);
    if (status == DEV_BARRIER_TIMEOUT) throw FeastError{FEAST_ERR_TIMEOUT};
    get_diag<c128>(G, k, k, d_nrm, st);
    std::vector<double> s2(k);
    to_host(ctx, s2.data(), d_nrm, k);
    std::vector<int> ord(k);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return s2[a] > s2[b]; });
    if (!(s2[ord[0]] > 0.0)) throw FeastError{FEAST_ERR_ORTH};
    std::vector<int> keep;
    std::vector<double> sc;
    for (int i : ord)
      if (s2[i] >= 1e-12 * s2[ord[0]]) {
        keep.push_back(i);
        sc.push_back(1.0 / std::sqrt(s2[i]));
      }
    const int64_t r = (int64_t)keep.size();
    to_dev(ctx, d_idx, keep.data(), r);
    to_dev(ctx, d_scale, sc.data(), r);
    gather_cols<c128>(Cg, k, Vg, k, k, d_idx, r, d_scale, st);
    gemm_simple<c128, c128, c128>(n, r, k, C1(1.0), Y, n, OP_N, Cg, k, OP_N, C1(0.0), tmp, n, st);
    if (!cholqr_once(tmp, r, Qout)) throw FeastError{FEAST_ERR_ORTH};
    return r;
  }
  // eigenpairs of the general k x k matrix H (ld k, overwritten): values in
  // ev, unit-norm vectors in Vr (ld k)
  void eig(c128* H, int64_t k, std::vector<c128>& ev) {
    frobenius_norm(H, k, d_nrm, st);
    double hn = 0.0;
    to_host(ctx, &hn, d_nrm, 1);
    FEAST_CUDA_TRY(cudaMemsetAsync(d_info, 0, 2 * sizeof(int), st));
    schur_complex(H, Zs, (int)k, d_info, st);
    int info[2] = {0, 0};
    to_host(ctx, info, d_info, 2);
    if (info[0] == 2) throw FeastError{FEAST_ERR_TIMEOUT};
    if (info[0] != 0) throw FeastError{FEAST_ERR_ORTH};
    last_sweeps = info[1];
    triangular_eigvecs(H, Ys, (int)k, std::max(2.220446049250313e-16 * hn, 1e-300), st);
    gemm_simple<c128, c128, c128>(k, k, k, C1(1.0), Zs, k, OP_N, Ys, k, OP_N, C1(0.0), Vr, k, st);
    col_norms2<c128>(Vr, k, k, k, d_nrm, st);
    std::vector<double> nr(k);
    to_host(ctx, nr.data(), d_nrm, k);
    for (auto& x : nr) x = x > 0.0 ? 1.0 / std::sqrt(x) : 1.0;
    to_dev(ctx, d_scale, nr.data(), k);
    scale_cols<c128>(Vr, k, k, k, d_scale, st);
    ev.resize(k);  // the diagonal of T, stride k + 1
    FEAST_CUDA_TRY(cudaMemcpy2DAsync(ev.data(), sizeof(c128), H, (k + 1) * sizeof(c128), sizeof(c128), k,
                                     cudaMemcpyDeviceToHost, st));
    sync(ctx);
  }
  // Rayleigh-Ritz on the orthonormal Q (n x k): ev, X = Q V (unit columns),
  // AX, relative residuals
  void rayleigh_ritz(int64_t k, std::vector<c128>& ev, std::vector<double>& res) {
    gemm_simple<c128, c128, c128>(n, k, n, C1(1.0), A, n, OP_N, Q, n, OP_N, C1(0.0), Wq, n, st);
    reduce(k, k, Q, Wq, Hr);
    eig(Hr, k, ev);
    gemm_simple<c128, c128, c128>(n, k, k, C1(1.0), Q, n, OP_N, Vr, k, OP_N, C1(0.0), X, n, st);
    gemm_simple<c128, c128, c128>(n, k, k, C1(1.0), Wq, n, OP_N, Vr, k, OP_N, C1(0.0), AX, n, st);
    col_norms2<c128>(X, n, k, n, d_nrm, st);
    std::vector<double> nr(k);
    to_host(ctx, nr.data(), d_nrm, k);
    for (auto& x : nr) x = x > 0.0 ? 1.0 / std::sqrt(x) : 1.0;
    to_dev(ctx, d_scale, nr.data(), k);
    scale_cols<c128>(X, n, k, n, d_scale, st);
    scale_cols<c128>(AX, n, k, n, d_scale, st);
    to_dev(ctx, d_lam, ev.data(), k);
    resid_norms2_complex(AX, X, n, k, d_lam, d_nrm, st);
    res.resize(k);
    to_host(ctx, res.data(), d_nrm, k);
    for (auto& r : res) r = std::sqrt(r) / anorm;
  }
};

bool in_disk(c128 l, c128 c, double r) { return std::hypot(l.re - c.re, l.im - c.im) < r; }

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void feast_opts_default(feast_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->variant = FEAST_PLAIN;
  o->s = 3;
  o->prec = FEAST_PREC_F64;
  o->max_iter = 100;
  o->refine_max = 10;
  o->refine_gemm = 0;
  o->aspect = 1.0;
  o->anorm = 0.0;
  o->refine_tol = 0.0;
  o->seed = 0x1605087710ull;
  o->x0 = nullptr;
  o->refine_switch = 0.0;
}

int feast_init(feast_ctx** ctx, int device, void* stream) {
  if (!ctx) return FEAST_ERR_ARG;
  *ctx = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return FEAST_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return FEAST_ERR_CUDA;
  feast_ctx* c = new (std::nothrow) feast_ctx();
  if (!c) return FEAST_ERR_NOMEM;
  c->device = device;
  c->stream = (cudaStream_t)stream;
  if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    return FEAST_ERR_CUDA;
  }
  *ctx = c;
  return FEAST_OK;
}

int feast_finalize(feast_ctx* ctx) {
  if (!ctx) return FEAST_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  ctx->arena.release();
  ctx->aux.release();
  delete ctx;
  return FEAST_OK;
}

uint64_t feast_kernel_launches(void) { return (uint64_t)feast::launch_count(); }

const char* feast_strerror(int code) {
  switch (code) {
    case FEAST_OK: return "success";
    case FEAST_WARN_MAXITER: return "maximum number of iterations reached before convergence";
    case FEAST_ERR_ARG: return "invalid argument";
    case FEAST_ERR_NONFINITE: return "NaN or Inf in the input matrix or subspace";
    case FEAST_ERR_SINGULAR: return "a shifted matrix z_j I - A is exactly singular";
    case FEAST_ERR_ORTH: return "the subspace could not be orthonormalised";
    case FEAST_ERR_M0: return "subspace size m0 too small for the interval";
    case FEAST_ERR_CUDA: return "CUDA runtime error";
    case FEAST_ERR_NOMEM: return "device memory allocation failed";
    case FEAST_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    default: return "unknown status";
  }
}

int feast_contour_nodes(double lmin, double lmax, int n_c, double aspect, double* z, double* w) {
  if (!z || !w || n_c < 1 || n_c > 256 || !(lmin < lmax) || !(aspect > 0)) return FEAST_ERR_ARG;
  std::vector<c128> zz, ww;
  contour(lmin, lmax, n_c, aspect, zz, ww);
  for (int j = 0; j < n_c; ++j) {
    z[2 * j] = zz[j].re;
    z[2 * j + 1] = zz[j].im;
    w[2 * j] = ww[j].re;
    w[2 * j + 1] = ww[j].im;
  }
  return FEAST_OK;
}

int feast_contour_nodes_offset(double lmin, double lmax, int n_c, double aspect, const double* offsets, double* z,
                               double* w) {
  if (!z || !w || n_c < 1 || n_c > 256 || !(lmin < lmax) || !(aspect > 0)) return FEAST_ERR_ARG;
  std::vector<c128> zz, ww;
  try {
    contour(lmin, lmax, n_c, aspect, zz, ww, offsets);
  } catch (const FeastError& e) {
    return e.code;
  }
  for (int j = 0; j < n_c; ++j) {
    z[2 * j] = zz[j].re;
    z[2 * j + 1] = zz[j].im;
    w[2 * j] = ww[j].re;
    w[2 * j + 1] = ww[j].im;
  }
  return FEAST_OK;
}

int feast_spectral_moments(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double c, double r,
                           const void* V, int64_t nv, int M, double* mu) {
  if (int e = check_common(ctx, A, dtype, n, lda, -1.0, 1.0, 1)) return e;
  if (!V || !mu || nv < 1 || M < 1 || M > 4096 || !std::isfinite(c) || !(r > 0) || !std::isfinite(r))
    return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    auto run = [&](auto tag) {
      using S = decltype(tag);
      S* T0 = dalloc<S>(ctx, n * nv);
      S* T1 = dalloc<S>(ctx, n * nv);
      S* AT = dalloc<S>(ctx, n * nv);
      double* part = dalloc<double>(ctx, (int64_t)M * kMomentBlocks);
      chebyshev_moments<S>((const S*)A, n, lda, c, r, (const S*)V, nv, M, T0, T1, AT, part, nullptr, ctx->stream);
      std::vector<double> h((size_t)M * kMomentBlocks);
      to_host(ctx, h.data(), part, (int64_t)M * kMomentBlocks);
      for (int k = 0; k < M; ++k) {
        double acc = 0.0;
        for (int b = 0; b < kMomentBlocks; ++b) acc += h[(size_t)k * kMomentBlocks + b];
        mu[k] = acc / ((double)n * (double)nv);
      }
      return FEAST_OK;
    };
    if (dtype == FEAST_R64) return run(double{});
    return run(c128{});
  });
}

double feast_moments_count(const double* mu, int M, double c, double r, double a, double b, int64_t n) {
  if (!mu || M < 1 || !(r > 0)) return NAN;
  auto theta = [&](double x) { return std::acos(std::min(1.0, std::max(-1.0, (x - c) / r))); };
  const double ta = theta(a), tb = theta(b), q = M_PI / (M + 1);
  double sum = 0.0;
  for (int k = 0; k < M; ++k) {
    // Jackson damping
    const double g = ((M - k + 1) * std::cos(q * k) + std::sin(q * k) / std::tan(q)) / (M + 1);
    const double ik = k == 0 ? (ta - tb) / M_PI : 2.0 * (std::sin(k * ta) - std::sin(k * tb)) / (k * M_PI);
    sum += g * mu[k] * ik;
  }
  return (double)n * sum;
}

int feast_mlp_param_count(void) { return (int)mlp_param_count(); }

int feast_mlp_forward(feast_ctx* ctx, const float* params, const float* X, int64_t B, float* Y) {
  if (!ctx || !params || !X || !Y || B < 1 || B > (1 << 22)) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    float* acts = dalloc<float>(ctx, (int64_t)mlp_act_floats(B));
    mlp_forward(params, X, B, acts, ctx->stream);
    const int64_t out = (int64_t)mlp_act_floats(B) - B * kMlpDims[kMlpLayers];
    FEAST_CUDA_TRY(cudaMemcpyAsync(Y, acts + out, sizeof(float) * B * kMlpDims[kMlpLayers], cudaMemcpyDeviceToDevice,
                                   ctx->stream));
    sync(ctx);
    return FEAST_OK;
  });
}

namespace {
// forward + backward into grad; the loss (mean squared error) to the host
double mlp_grad_run(feast_ctx* ctx, const float* params, const float* X, const float* T, int64_t B, float* grad) {
  float* acts = dalloc<float>(ctx, (int64_t)mlp_act_floats(B));
  float* d0 = dalloc<float>(ctx, B * 256);
  float* d1 = dalloc<float>(ctx, B * 256);
  const int dlast = kMlpDims[kMlpLayers];
  float* sq = dalloc<float>(ctx, B * dlast);
  mlp_forward(params, X, B, acts, ctx->stream);
  mlp_backward(params, acts, T, B, grad, d0, d1, sq, ctx->stream);
  std::vector<float> h((size_t)B * dlast);
  to_host(ctx, h.data(), sq, B * dlast);
  double acc = 0.0;
  for (float v : h) acc += v;
  return acc / ((double)B * dlast);
}
}  // namespace

int feast_mlp_gradient(feast_ctx* ctx, const float* params, const float* X, const float* T, int64_t B, float* grad,
                       double* loss) {
  if (!ctx || !params || !X || !T || !grad || B < 1 || B > (1 << 22)) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    const double l = mlp_grad_run(ctx, params, X, T, B, grad);
    if (loss) *loss = l;
    return FEAST_OK;
  });
}

int feast_mlp_train_step(feast_ctx* ctx, float* params, float* m, float* v, const float* X, const float* T, int64_t B,
                         int step, double lr, double* loss) {
  if (!ctx || !params || !m || !v || !X || !T || B < 1 || B > (1 << 22) || step < 1 || !(lr > 0)) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    float* grad = dalloc<float>(ctx, (int64_t)mlp_param_count());
    const double l = mlp_grad_run(ctx, params, X, T, B, grad);
    adam_update(params, grad, m, v, (int64_t)mlp_param_count(), step, (float)lr, ctx->stream);
    sync(ctx);
    if (loss) *loss = l;
    return FEAST_OK;
  });
}

int feast_interval_solve(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double lmin, double lmax,
                         int m0, int n_c, double tol, const feast_opts* opts, double* evals, void* evecs,
                         double* res, int* m_found, int* iterations, feast_stats* stats) {
  if (int r = check_common(ctx, A, dtype, n, lda, lmin, lmax, n_c)) return r;
  if (m0 < 1 || m0 > n || !(tol > 0) || !evals || !evecs || !res || !m_found || !iterations) return FEAST_ERR_ARG;
  feast_opts o;
  if (opts) o = *opts; else feast_opts_default(&o);
  if (o.variant < 0 || o.variant > 2 || o.prec < 0 || o.prec > 2 || o.max_iter < 1 || !(o.aspect > 0)) return FEAST_ERR_ARG;
  if (o.variant != FEAST_PLAIN && (o.s < 1 || (int64_t)o.s * m0 > 65536)) return FEAST_ERR_ARG;
  if (o.refine_max < 0 || !(o.refine_switch >= 0.0) || o.refine_gemm < 0 || o.refine_gemm > 1) return FEAST_ERR_ARG;
  if (o.rfeast_expand < 0 || o.rfeast_expand > 1 || o.response_stop < 0 || o.response_stop > 1) return FEAST_ERR_ARG;
  *m_found = 0;
  *iterations = 0;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    if (dtype == FEAST_R64)
      return solve_t<double>(ctx, (const double*)A, n, lda, lmin, lmax, m0, n_c, tol, o, evals, (double*)evecs, res,
                             m_found, iterations, stats);
    return solve_t<c128>(ctx, (const c128*)A, n, lda, lmin, lmax, m0, n_c, tol, o, evals, (c128*)evecs, res, m_found,
                         iterations, stats);
  });
}

int feast_interval_solve_gen(feast_ctx* ctx, const void* A, const void* B, int dtype, int64_t n, int64_t lda,
                             int64_t ldb, double lmin, double lmax, int m0, int n_c, double tol, const feast_opts* opts,
                             double* evals, void* evecs, double* res, int* m_found, int* iterations,
                             feast_stats* stats) {
  if (int r = check_common(ctx, A, dtype, n, lda, lmin, lmax, n_c)) return r;
  if (!B || ldb < n || m0 < 1 || m0 > n || !(tol > 0) || !evals || !evecs || !res || !m_found || !iterations)
    return FEAST_ERR_ARG;
  const size_t es = dtype == FEAST_R64 ? sizeof(double) : sizeof(c128);
  if (es * (size_t)n > 200 * 1024) return FEAST_ERR_ARG;  // the Cholesky kernel keeps a column in shared memory
  feast_opts o;
  if (opts) o = *opts; else feast_opts_default(&o);
  o.anorm = 0.0;   // ||C|| is estimated for the reduced matrix
  if (o.x0) return FEAST_ERR_ARG;
  *m_found = 0;
  *iterations = 0;
  int status = guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->aux.reset();
    auto run = [&](auto tag) -> int {
      using S = decltype(tag);
      auto aux = [&](int64_t count) { return (S*)ctx->aux.alloc(sizeof(S) * (size_t)std::max<int64_t>(count, 1)); };
      const cudaStream_t st = ctx->stream;
      if (int r = check_finite_dev<S>(ctx, (const S*)B, n, n, ldb)) return r;
      // B = R^H R (Cholesky, upper), Ri = R^{-1}, C = Ri^H A Ri
      S* Rb = aux(n * n);
      S* Ri = aux(n * n);
      S* T = aux(n * n);
      S* C = aux(n * n);
      CoopWork cw = coop_work_carve(ctx->aux.alloc(coop_work_bytes(n, ctx->num_sms)), n, ctx->num_sms);
      copy_matrix<S>(Rb, n, (const S*)B, ldb, n, n, st);
      cholesky_upper<S>(Rb, n, n, cw, ctx->num_sms, st);
      int info = 0, cst = 0;
      to_host(ctx, &info, cw.info, 1);
      to_host(ctx, &cst, cw.status, 1);
      if (cst == DEV_BARRIER_TIMEOUT) return FEAST_ERR_TIMEOUT;
      if (info != 0) return FEAST_ERR_ARG;   // B not numerically positive definite
      tri_inverse_upper<S>(Rb, n, n, Ri, n, st);
      gemm_simple<S, S, S>(n, n, n, C1(1.0), (const S*)A, lda, OP_N, Ri, n, OP_N, C1(0.0), T, n, st);
      gemm_simple<S, S, S>(n, n, n, C1(1.0), Ri, n, OP_C, T, n, OP_N, C1(0.0), C, n, st);
      hermitize<S>(C, n, n, st);
      sync(ctx);
      // the standard problem C y = lambda y, then x = Ri y (B-orthonormal)
      S* Y = aux(n * m0);
      const int r = solve_t<S>(ctx, C, n, n, lmin, lmax, m0, n_c, tol, o, evals, Y, res, m_found, iterations, stats);
      if (r < 0) return r;
      if (*m_found > 0)
        gemm_simple<S, S, S>(n, *m_found, n, C1(1.0), Ri, n, OP_N, Y, n, OP_N, C1(0.0), (S*)evecs, n, st);
      sync(ctx);
      return r;
    };
    if (dtype == FEAST_R64) return run(double{});
    return run(c128{});
  });
  return status;
}

int feast_filter_apply(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double lmin, double lmax,
                       int n_c, const feast_opts* opts, const void* X, int64_t m, void* Y) {
  if (int r = check_common(ctx, A, dtype, n, lda, lmin, lmax, n_c)) return r;
  if (!X || !Y || m < 1) return FEAST_ERR_ARG;
  feast_opts o;
  if (opts) o = *opts; else feast_opts_default(&o);
  if (o.prec < 0 || o.prec > 2 || !(o.aspect > 0) || o.refine_max < 0 || o.refine_gemm < 0 || o.refine_gemm > 1)
    return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    auto run = [&](auto tag) {
      using S = decltype(tag);
      Solver<S> sv(ctx, (const S*)A, n, lda, lmin, lmax, n_c, o);
      sv.alloc_common(1, m);
      sv.alloc_filter(m);
      sv.alloc_factors();
      sv.kmax = 1;
      sv.T1 = dalloc<S>(ctx, n);
      sv.T2 = dalloc<S>(ctx, n);
      sv.d_nrm = dalloc<double>(ctx, 1);
      sv.d_scale = dalloc<double>(ctx, 1);
      sv.d_idx = dalloc<int>(ctx, 1);
      sv.anorm = o.anorm > 0 ? o.anorm : (o.prec != FEAST_PREC_F64 ? sv.estimate_norm() : 1.0);
      sv.factor();
      sv.filter((const S*)X, m, (S*)Y);
      sync(ctx);
      ctx->last = feast_stats{};
      ctx->last.refine_steps = sv.refine_steps;
      return FEAST_OK;
    };
    if (dtype == FEAST_R64) return run(double{});
    return run(c128{});
  });
}

int feast_shifted_lu(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, const double* z, int nz,
                     int prec, void* LU, int32_t* perm) {
  if (int r = check_common(ctx, A, dtype, n, lda, -1.0, 1.0, nz)) return r;
  if (!z || !LU || !perm || (prec < FEAST_PREC_F64 || prec > FEAST_PREC_MIXED_SIMT)) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    const size_t eb = prec == FEAST_PREC_F64 ? sizeof(c128) : sizeof(c64);
    const int pmax = std::max(1, ctx->num_sms * 8);
    PanelWork pw = panel_work_carve(ctx->arena.alloc(panel_work_bytes(nz, pmax, eb)), nz, pmax, eb);
    if (prec == FEAST_PREC_MIXED) pw.tc_planes = ctx->arena.alloc(lu_tc_planes_bytes(n, nz));
    c128* dz = dalloc<c128>(ctx, nz);
    to_dev(ctx, dz, (const c128*)z, nz);
    int32_t* ipiv = dalloc<int32_t>(ctx, (int64_t)nz * n);
    auto go = [&](auto ftag) {
      using F = decltype(ftag);
      if (dtype == FEAST_R64) form_shifted<F, double>((F*)LU, n, n, n * n, nz, (const double*)A, lda, dz, ctx->stream);
      else form_shifted<F, c128>((F*)LU, n, n, n * n, nz, (const c128*)A, lda, dz, ctx->stream);
      lu_factor_batched<F>((F*)LU, n, n, n * n, nz, ipiv, perm, pw, ctx->num_sms, ctx->stream);
    };
    if (prec == FEAST_PREC_F64) go(c128{});
    else go(c64{});
    int status = 0;
    std::vector<int> zp(nz);
    to_host(ctx, &status, pw.status, 1);
    to_host(ctx, zp.data(), pw.zero_pivot, nz);
    if (status == DEV_BARRIER_TIMEOUT) return FEAST_ERR_TIMEOUT;
    for (int v : zp)
      if (v) return FEAST_ERR_SINGULAR;
    return FEAST_OK;
  });
}

int feast_shifted_solve(feast_ctx* ctx, const void* LU, const int32_t* perm, int64_t n, int nz, int prec, int adjoint,
                        const void* B, int64_t m, void* Y) {
  if (!ctx || !LU || !perm || !B || !Y || n < 1 || nz < 1 || m < 1) return FEAST_ERR_ARG;
  if (prec < FEAST_PREC_F64 || prec > FEAST_PREC_MIXED_SIMT) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    const int64_t nm = n * m;
    auto go = [&](auto ftag) {
      using F = decltype(ftag);
      F* W = dalloc<F>(ctx, nz * nm);
      // FEAST_PREC_MIXED: block updates on the tensor cores from bf16 planes of the factors
      const SolvePlanes* planes = nullptr;
      SolvePlanes sp;
      int* flag = dalloc<int>(ctx, 1);
      FEAST_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
      if constexpr (std::is_same<F, c64>::value) {
        if (prec == FEAST_PREC_MIXED) {
          sp = solve_planes_carve(ctx->arena.alloc(solve_planes_bytes(n, m, nz, nz, adjoint != 0)), n, m, nz, nz,
                                  adjoint != 0);
          if (!adjoint) sp.row = nullptr;
          solve_planes_build((const c64*)LU, n, n, n * n, nz, sp, ctx->stream);
          planes = &sp;
        }
      }
      permute_in<F, c128>(W, nm, (const c128*)B, n, 0, n, m, perm, nz, adjoint != 0, ctx->stream);
      lu_solve_batched<F>((const F*)LU, n, n, n * n, nz, W, m, nm, adjoint != 0, ctx->stream, planes, flag,
                          ctx->num_sms);
      permute_out<F, c128>((c128*)Y, nm, W, nm, n, m, perm, nz, adjoint != 0, false, ctx->stream);
      int f = 0;
      to_host(ctx, &f, flag, 1);
      return f == DEV_BARRIER_TIMEOUT ? FEAST_ERR_TIMEOUT : FEAST_OK;
    };
    const int r = prec == FEAST_PREC_F64 ? go(c128{}) : go(c64{});
    sync(ctx);
    return r;
  });
}

int feast_orthonormalize(feast_ctx* ctx, int dtype, int64_t n, int64_t k, void* X, int method, int* rank) {
  if (!ctx || !X || !rank || n < 1 || k < 1 || k > n || (dtype != FEAST_R64 && dtype != FEAST_C128)) return FEAST_ERR_ARG;
  if (method < 0 || method > 1) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    auto run = [&](auto tag) {
      using S = decltype(tag);
      feast_opts o;
      feast_opts_default(&o);
      Solver<S> sv(ctx, nullptr, n, n, -1.0, 1.0, 1, o);
      sv.kmax = k;
      sv.cw = coop_work_carve(ctx->arena.alloc(coop_work_bytes(k, ctx->num_sms)), k, ctx->num_sms);
      const int64_t kk = k * k;
      sv.Gs = dalloc<S>(ctx, kk); sv.Ri = dalloc<S>(ctx, kk); sv.Vk = dalloc<S>(ctx, kk); sv.Cs = dalloc<S>(ctx, kk);
      sv.part_elems = 32 * kk;
      sv.part = dalloc<S>(ctx, sv.part_elems);
      sv.d_lam = dalloc<double>(ctx, k); sv.d_scale = dalloc<double>(ctx, k); sv.d_idx = dalloc<int>(ctx, k);
      S* Q = dalloc<S>(ctx, n * k);
      S* T = dalloc<S>(ctx, n * k);
      int64_t r = method == 0 ? sv.orthonormalize((S*)X, n, k, Q, T) : sv.gram_eig_orth((S*)X, n, k, Q, T, 1e-12);
      if (r == 0) return FEAST_ERR_ORTH;
      copy_matrix<S>((S*)X, n, Q, n, n, r, ctx->stream);
      sync(ctx);
      *rank = (int)r;
      return FEAST_OK;
    };
    if (dtype == FEAST_R64) return run(double{});
    return run(c128{});
  });
}

int feast_jacobi_eigh(feast_ctx* ctx, int dtype, int64_t k, const void* H, double* evals, void* V, int* sweeps) {
  if (!ctx || !H || !evals || !V || k < 1 || (dtype != FEAST_R64 && dtype != FEAST_C128)) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    auto run = [&](auto tag) {
      using S = decltype(tag);
      feast_opts o;
      feast_opts_default(&o);
      Solver<S> sv(ctx, nullptr, 1, 1, -1.0, 1.0, 1, o);
      sv.kmax = k;
      sv.cw = coop_work_carve(ctx->arena.alloc(coop_work_bytes(k, ctx->num_sms)), k, ctx->num_sms);
      sv.Vk = dalloc<S>(ctx, k * k);
      sv.Cs = dalloc<S>(ctx, k * k);
      sv.d_lam = dalloc<double>(ctx, k);
      sv.d_idx = dalloc<int>(ctx, k);
      S* Hw = dalloc<S>(ctx, k * k);
      copy_matrix<S>(Hw, k, (const S*)H, k, k, k, ctx->stream);
      std::vector<double> ev;
      sv.eig(Hw, k, ev);
      std::vector<int> ord(k);
      std::iota(ord.begin(), ord.end(), 0);
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return ev[a] < ev[b]; });
      to_dev(ctx, sv.d_idx, ord.data(), k);
      gather_cols<S>((S*)V, k, sv.Vk, k, k, sv.d_idx, k, nullptr, ctx->stream);
      sync(ctx);
      for (int64_t i = 0; i < k; ++i) evals[i] = ev[ord[i]];
      if (sweeps) *sweeps = sv.last_sweeps;
      return FEAST_OK;
    };
    if (dtype == FEAST_R64) return run(double{});
    return run(c128{});
  });
}

int feast_rayleigh_ritz(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, const void* Q, int64_t k,
                        double anorm, double* evals, void* X, double* res) {
  if (int r = check_common(ctx, A, dtype, n, lda, -1.0, 1.0, 1)) return r;
  if (!Q || !evals || !X || !res || k < 1 || k > n || !(anorm > 0)) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    auto run = [&](auto tag) {
      using S = decltype(tag);
      feast_opts o;
      feast_opts_default(&o);
      Solver<S> sv(ctx, (const S*)A, n, lda, -1.0, 1.0, 1, o);
      sv.kmax = k;
      sv.cw = coop_work_carve(ctx->arena.alloc(coop_work_bytes(k, ctx->num_sms)), k, ctx->num_sms);
      sv.alloc_rr();
      sv.anorm = anorm;
      copy_matrix<S>(sv.Qb, n, (const S*)Q, n, n, k, ctx->stream);
      sv.rr_project(k);
      sv.rr_solve(k);
      copy_matrix<S>((S*)X, n, sv.Xr, n, n, k, ctx->stream);
      sync(ctx);
      for (int64_t i = 0; i < k; ++i) {
        evals[i] = sv.lam[i];
        res[i] = sv.res[i];
      }
      return FEAST_OK;
    };
    if (dtype == FEAST_R64) return run(double{});
    return run(c128{});
  });
}

int feast_gemm_f64acc(feast_ctx* ctx, int method, int dtype, int transA, int transB, int64_t M, int64_t N, int64_t K,
                      double alpha, const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C,
                      int64_t ldc) {
  if (!ctx || !A || !B || !C || M < 1 || N < 1 || K < 1 || ldc < M) return FEAST_ERR_ARG;
  if (dtype != FEAST_R64 && dtype != FEAST_C128) return FEAST_ERR_ARG;
  if ((transA != 0 && transA != 1) || (transB != 0 && transB != 1)) return FEAST_ERR_ARG;
  if (lda < (transA ? K : M) || ldb < (transB ? N : K)) return FEAST_ERR_ARG;
  if (!std::isfinite(alpha) || !std::isfinite(beta)) return FEAST_ERR_ARG;
  if (method != 0 && method != 1) return FEAST_ERR_ARG;
  // the double-float route: real, no transposes, C = alpha A B
  if (method == 1 && (dtype != FEAST_R64 || transA || transB || beta != 0.0)) return FEAST_ERR_ARG;
  if (M > INT32_MAX / kOzDigits || N > INT32_MAX / kOzDigits) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    cudaStream_t st = ctx->stream;
    const bool cplx = dtype == FEAST_C128;
    if (method == 0) {
      int* flag = dalloc<int>(ctx, 1);
      FEAST_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
      OzScratch w{};
      for (int t = 0; t < (cplx ? 3 : 1); ++t) {
        w.L[t] = ctx->arena.alloc(oz_operand_bytes(M, K, true));
        w.R[t] = ctx->arena.alloc(oz_operand_bytes(N, K, false));
      }
      w.T = dalloc<double>(ctx, (cplx ? 2 : 1) * M * N);
      w.T2 = cplx ? dalloc<double>(ctx, M * N) : nullptr;
      oz_gemm_op(cplx, M, N, K, alpha, (const double*)A, lda, transA != 0, (const double*)B, ldb, transB != 0, beta,
                 (double*)C, ldc, w, flag, ctx->num_sms, st);
      int f = 0;
      to_host(ctx, &f, flag, 1);
      if (f == DEV_BARRIER_TIMEOUT) return FEAST_ERR_TIMEOUT;
    } else {
      float* Ap = dalloc<float>(ctx, 2 * M * K);
      float* Bp = dalloc<float>(ctx, 2 * K * N);
      split_df32((const double*)A, M, K, lda, 1, 0, Ap, Ap + M * K, st);
      split_df32((const double*)B, K, N, ldb, 1, 0, Bp, Bp + K * N, st);
      gemm_df32(M, N, K, alpha, Ap, Ap + M * K, M, Bp, Bp + K * N, K, 0.0, (double*)C, ldc, 1, 0, st);
      sync(ctx);
    }
    return FEAST_OK;
  });
}

// ---------------------------------------------------------------------------
// general (non-Hermitian) matrices
// ---------------------------------------------------------------------------
int feast_circle_nodes(double c_re, double c_im, double radius, int n_c, double* z, double* w) {
  if (!z || !w || n_c < 1 || n_c > 64 || !std::isfinite(c_re) || !std::isfinite(c_im) || !(radius > 0.0) ||
      !std::isfinite(radius))
    return FEAST_ERR_ARG;
  std::vector<c128> zz, ww;
  circle(c128{c_re, c_im}, radius, n_c, zz, ww);
  for (int j = 0; j < 2 * n_c; ++j) {
    z[2 * j] = zz[j].re;
    z[2 * j + 1] = zz[j].im;
    w[2 * j] = ww[j].re;
    w[2 * j + 1] = ww[j].im;
  }
  return FEAST_OK;
}

int feast_eig_general(feast_ctx* ctx, int64_t k, const void* H, double* evals, void* V, int* sweeps) {
  if (!ctx || !H || !evals || !V || k < 1 || k > kSchurMaxK) return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    General g(ctx);
    g.setup_small(k);
    c128* Hw = dalloc<c128>(ctx, k * k);
    copy_matrix<c128>(Hw, k, (const c128*)H, k, k, k, ctx->stream);
    if (int r = check_finite_dev<c128>(ctx, Hw, k, k, k)) return r;
    std::vector<c128> ev;
    g.eig(Hw, k, ev);
    copy_matrix<c128>((c128*)V, k, g.Vr, k, k, k, ctx->stream);
    sync(ctx);
    for (int64_t i = 0; i < k; ++i) {
      evals[2 * i] = ev[i].re;
      evals[2 * i + 1] = ev[i].im;
    }
    if (sweeps) *sweeps = g.last_sweeps;
    return FEAST_OK;
  });
}

int feast_filter_apply_general(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double c_re,
                               double c_im, double radius, int n_c, const void* X, int64_t m, void* Y) {
  if (!ctx || !A || !X || !Y || n < 1 || lda < n || m < 1 || n_c < 1 || n_c > 64) return FEAST_ERR_ARG;
  if ((dtype != FEAST_R64 && dtype != FEAST_C128) || !(radius > 0.0) || !std::isfinite(radius) ||
      !std::isfinite(c_re) || !std::isfinite(c_im))
    return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    if (dtype == FEAST_R64) {
      if (int r = check_finite_dev<double>(ctx, (const double*)A, n, n, lda)) return r;
    } else if (int r = check_finite_dev<c128>(ctx, (const c128*)A, n, n, lda)) {
      return r;
    }
    if (int r = check_finite_dev<c128>(ctx, (const c128*)X, n, m, n)) return r;
    General g(ctx);
    g.mmax = m;
    g.setup_matrix(A, dtype, n, lda);
    g.factor(c128{c_re, c_im}, radius, n_c);
    g.filter((const c128*)X, m, (c128*)Y);
    sync(ctx);
    return FEAST_OK;
  });
}

int feast_disk_solve(feast_ctx* ctx, const void* A, int dtype, int64_t n, int64_t lda, double c_re, double c_im,
                     double radius, int m0, int n_c, double tol, int max_iter, const void* x0, double* evals,
                     void* X, double* res, int* m_found, int* iterations) {
  if (!ctx || !A || !evals || !X || !res || !m_found || !iterations) return FEAST_ERR_ARG;
  if ((dtype != FEAST_R64 && dtype != FEAST_C128) || n < 1 || lda < n || m0 < 1 || m0 > n || m0 > kSchurMaxK ||
      n_c < 1 || n_c > 64 || max_iter < 1 || !(tol > 0.0) || !(radius > 0.0) || !std::isfinite(radius) ||
      !std::isfinite(c_re) || !std::isfinite(c_im))
    return FEAST_ERR_ARG;
  return guarded(ctx, [&]() {
    FEAST_CUDA_TRY(cudaSetDevice(ctx->device));
    ctx->arena.reset();
    cudaStream_t st = ctx->stream;
    if (dtype == FEAST_R64) {
      if (int r = check_finite_dev<double>(ctx, (const double*)A, n, n, lda)) return r;
    } else if (int r = check_finite_dev<c128>(ctx, (const c128*)A, n, n, lda)) {
      return r;
    }
    const c128 center{c_re, c_im};
    General g(ctx);
    g.setup_small(m0);
    g.setup_matrix(A, dtype, n, lda);
    g.setup_blocks();
    g.anorm = g.norm_estimate();
    if (!(g.anorm > 0.0)) g.anorm = 1.0;
    g.factor(center, radius, n_c);
    c128* X0 = dalloc<c128>(ctx, n * m0);
    c128* Yf = dalloc<c128>(ctx, n * m0);
    if (x0) {
      copy_matrix<c128>(X0, n, (const c128*)x0, n, n, m0, st);
      if (int r = check_finite_dev<c128>(ctx, X0, n, m0, n)) return r;
    } else {
      random_normal<c128>(X0, n, m0, n, 0x5eedull, st);
    }
    const c128* Xcur = X0;
    int64_t k = m0;
    std::vector<c128> ev;
    std::vector<double> rs;
    std::vector<int> ins;
    int status = FEAST_WARN_MAXITER, it = 0;
    for (it = 1; it <= max_iter; ++it) {
      g.filter(Xcur, k, Yf);
      k = g.orth(Yf, k, g.Q);
      g.rayleigh_ritz(k, ev, rs);
      ins.clear();
      double r = 0.0;
      for (int64_t i = 0; i < k; ++i)
        if (in_disk(ev[i], center, radius)) {
          ins.push_back((int)i);
          r = std::max(r, rs[i]);
        }
      if ((!ins.empty() && r <= tol) || (ins.empty() && it >= 2)) {
        status = FEAST_OK;
        break;
      }
      Xcur = g.X;
    }
    if (it > max_iter) it = max_iter;
    std::stable_sort(ins.begin(), ins.end(), [&](int a, int b) {
      return ev[a].re < ev[b].re || (ev[a].re == ev[b].re && ev[a].im < ev[b].im);
    });
    const int mf = (int)ins.size();
    if (mf > 0) {
      to_dev(ctx, g.d_idx, ins.data(), mf);
      gather_cols<c128>((c128*)X, n, g.X, n, n, g.d_idx, mf, nullptr, st);
    }
    sync(ctx);
    for (int i = 0; i < mf; ++i) {
      evals[2 * i] = ev[ins[i]].re;
      evals[2 * i + 1] = ev[ins[i]].im;
      res[i] = rs[ins[i]];
    }
    *m_found = mf;
    *iterations = it;
    return status;
  });
}
}  // extern "C"
