// Kernels of FEAST for a general (non-Hermitian) complex matrix: the reduced
// eigensolver (Hessenberg reduction, shifted QR to Schur form, triangular
// eigenvectors), the weighted sum of the whole-circle filter and the residual
// norms with complex Ritz values.
//
// Reduced eigensolver.  The Rayleigh-Ritz matrix Q^H A Q is small (k <= m0)
// and its QR iteration is a chain of dependent plane rotations, so one CTA
// takes it: one thread decides (deflation test, shift, rotation), all threads
// apply each rotation to the rows and columns it touches.
//   * Hessenberg reduction by Householder reflections P = I - tau v v^H that
//     map column j below the subdiagonal to alpha e_1 (alpha = -e^{i arg x_0}
//     ||x||), applied from the left (one warp per column) and the right (one
//     thread per row, column-major rows are coalesced), accumulated into Z.
//   * Implicit single-shift QR on the active window [lo, hi]: Wilkinson
//     shift (the eigenvalue of the trailing 2 x 2 block nearer its last
//     diagonal entry; an ad hoc shift every tenth sweep without deflation),
//     the bulge chased by Givens rotations G = [c s; -conj(s) c] with real c,
//     applied to the whole rows (up to column k - 1) and columns (from row
//     0) so that the full triangular factor T = Z^H H Z is formed.  A
//     subdiagonal entry is set to zero when it is at most 2^-52 times the sum
//     of the moduli of its two diagonal neighbours.
// Every loop is bounded: at most 30 k sweeps and a 20 s wall-clock limit,
// after which the kernel reports through info and returns.
#include "general.cuh"

namespace feast {
namespace {

constexpr int kSchurThreads = 512;
constexpr int kSchurWarps = kSchurThreads / 32;
constexpr unsigned long long kSchurLimitNs = 20ull * 1000000000ull;
constexpr double kEps = 2.220446049250313e-16;  // 2^-52

__device__ __forceinline__ double cmod(c128 a) { return hypot(a.re, a.im); }

// principal square root
__device__ __forceinline__ c128 csqrt_principal(c128 a) {
  const double r = cmod(a);
  if (r == 0.0) return c128{0.0, 0.0};
  if (a.re >= 0.0) {
    const double re = sqrt(0.5 * (r + a.re));
    return c128{re, a.im / (2.0 * re)};
  }
  const double im = copysign(sqrt(0.5 * (r - a.re)), a.im);
  return c128{a.im / (2.0 * im), im};
}

// sum over the CTA; every thread receives it
__device__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red is free (its previous readers have passed)
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(kSchurThreads) schur_kernel(c128* __restrict__ H, c128* __restrict__ Z, int k,
                                                              int* __restrict__ info) {
  __shared__ c128 v[kSchurMaxK];
  __shared__ double red[kSchurWarps];
  __shared__ c128 s_alpha, s_sn, s_mu;
  __shared__ double s_tau, s_c;
  __shared__ int s_ctl[3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long t0 = globaltimer_ns();
  auto at = [&](int i, int j) -> c128& { return H[(int64_t)i + (int64_t)j * k]; };
  const int64_t kk = (int64_t)k * k;

  double part = 0.0;
  for (int64_t idx = tid; idx < kk; idx += blockDim.x) {
    Z[idx] = c128{(idx % k) == (idx / k) ? 1.0 : 0.0, 0.0};
    part += abs2(H[idx]);
  }
  const double hnorm = sqrt(cta_sum(part, red));

  // ---- Hessenberg reduction ----
  for (int col = 0; col + 2 < k; ++col) {
    const int len = k - col - 1;
    double p = 0.0;
    for (int i = tid; i < len; i += blockDim.x) {
      const c128 x = at(col + 1 + i, col);
      v[i] = x;
      p += abs2(x);
    }
    const double norm2 = cta_sum(p, red);
    if (tid == 0) {
      double tau = 0.0;
      c128 alpha = v[0];
      const double nrm = sqrt(norm2);
      if (nrm > 0.0) {
        const c128 x0 = v[0];
        const double a0 = cmod(x0);
        const c128 ph = a0 > 0.0 ? c128{x0.re / a0, x0.im / a0} : c128{1.0, 0.0};
        alpha = c128{-ph.re * nrm, -ph.im * nrm};
        v[0] = x0 - alpha;
        tau = 1.0 / (norm2 + a0 * nrm);  // 2 / (v^H v), v^H v = 2 (||x||^2 + |x_0| ||x||)
      }
      s_tau = tau;
      s_alpha = alpha;
    }
    __syncthreads();
    const double tau = s_tau;
    if (tau == 0.0) continue;  // column already reduced (uniform branch)
    // left: rows col+1.., columns col+1..k-1; one warp per column
    for (int j = col + 1 + warp; j < k; j += kSchurWarps) {
      c128 d{0.0, 0.0};
      for (int i = lane; i < len; i += 32) d = d + conj(v[i]) * at(col + 1 + i, j);
      for (int o = 16; o > 0; o >>= 1) {
        d.re += __shfl_xor_sync(0xffffffffu, d.re, o);
        d.im += __shfl_xor_sync(0xffffffffu, d.im, o);
      }
      const c128 f = d * tau;
      for (int i = lane; i < len; i += 32) at(col + 1 + i, j) = at(col + 1 + i, j) - v[i] * f;
    }
    __syncthreads();
    // right: every row of H and Z, columns col+1..k-1
    for (int r = tid; r < k; r += blockDim.x) {
      c128 t{0.0, 0.0}, tz{0.0, 0.0};
      for (int i = 0; i < len; ++i) {
        t = t + at(r, col + 1 + i) * v[i];
        tz = tz + Z[r + (int64_t)(col + 1 + i) * k] * v[i];
      }
      const c128 f = t * tau, fz = tz * tau;
      for (int i = 0; i < len; ++i) {
        at(r, col + 1 + i) = at(r, col + 1 + i) - f * conj(v[i]);
        c128& zr = Z[r + (int64_t)(col + 1 + i) * k];
        zr = zr - fz * conj(v[i]);
      }
    }
    __syncthreads();
    for (int i = tid; i < len; i += blockDim.x) at(col + 1 + i, col) = i == 0 ? s_alpha : c128{0.0, 0.0};
    __syncthreads();
  }

  // ---- shifted QR to Schur form ----
  int hi = k - 1, its = 0, sweeps = 0;  // used by thread 0 only
  const int max_sweeps = 30 * k;
  while (true) {
    if (tid == 0) {
      int action = 1, lo = 0;
      while (hi > 0) {
        int l = hi;
        for (; l > 0; --l) {
          double thr = kEps * (cmod(at(l, l)) + cmod(at(l - 1, l - 1)));
          if (thr == 0.0) thr = kEps * hnorm;
          if (cmod(at(l, l - 1)) <= thr) {
            at(l, l - 1) = c128{0.0, 0.0};
            break;
          }
        }
        if (l == hi) {
          --hi;
          its = 0;
          continue;
        }
        lo = l;
        break;
      }
      if (hi <= 0) {
        action = 0;
      } else if (sweeps >= max_sweeps) {
        action = 2;
      } else if (globaltimer_ns() - t0 > kSchurLimitNs) {
        action = 3;
      } else {
        const c128 d = at(hi, hi);
        c128 mu;
        if (its > 0 && its % 10 == 0) {
          mu = d + c128{0.75 * cmod(at(hi, hi - 1)), 0.0};
        } else {
          const c128 a = at(hi - 1, hi - 1), b = at(hi - 1, hi), c = at(hi, hi - 1);
          const c128 p = (a - d) * 0.5;
          const c128 bc = b * c;
          const c128 disc = csqrt_principal(p * p + bc);
          const c128 q1 = p + disc, q2 = p - disc;
          const c128 q = abs2(q1) >= abs2(q2) ? q1 : q2;
          // the shifted roots u of u^2 - 2 p u - bc = 0 are q and -bc / q
          mu = abs2(q) > 0.0 ? d - bc * recip(q) : d;
        }
        ++its;
        ++sweeps;
        s_mu = mu;
      }
      s_ctl[0] = action;
      s_ctl[1] = lo;
      s_ctl[2] = hi;
      if (action != 1) {
        info[0] = action == 0 ? 0 : (action == 2 ? 1 : 2);
        info[1] = sweeps;
      }
    }
    __syncthreads();
    if (s_ctl[0] != 1) break;
    const int lo = s_ctl[1], hh = s_ctl[2];
    const c128 mu = s_mu;
    for (int j = lo; j < hh; ++j) {
      if (tid == 0) {
        c128 x, y;
        if (j == lo) {
          x = at(lo, lo) - mu;
          y = at(lo + 1, lo);
        } else {
          x = at(j, j - 1);
          y = at(j + 1, j - 1);
        }
        const double ax = cmod(x), ay = cmod(y);
        double c = 1.0;
        c128 sn{0.0, 0.0};
        if (ay > 0.0) {
          if (ax == 0.0) {
            c = 0.0;
            sn = c128{1.0, 0.0};
          } else {
            const double r = hypot(ax, ay);
            c = ax / r;
            sn = c128{x.re / ax, x.im / ax} * conj(y) * (1.0 / r);
          }
        }
        s_c = c;
        s_sn = sn;
      }
      __syncthreads();
      const double c = s_c;
      const c128 sn = s_sn;
      // rows j, j+1 from G on the left
      for (int q = (j == lo ? lo : j - 1) + tid; q < k; q += blockDim.x) {
        const c128 a = at(j, q), b = at(j + 1, q);
        at(j, q) = c * a + sn * b;
        at(j + 1, q) = c * b - conj(sn) * a;
      }
      __syncthreads();
      if (tid == 0 && j > lo) at(j + 1, j - 1) = c128{0.0, 0.0};
      // columns j, j+1 from G^H on the right (rows to the bulge), and Z
      const int rmax = min(j + 2, hh);
      for (int r = tid; r <= rmax; r += blockDim.x) {
        const c128 a = at(r, j), b = at(r, j + 1);
        at(r, j) = c * a + conj(sn) * b;
        at(r, j + 1) = c * b - sn * a;
      }
      for (int r = tid; r < k; r += blockDim.x) {
        c128& za = Z[r + (int64_t)j * k];
        c128& zb = Z[r + (int64_t)(j + 1) * k];
        const c128 a = za, b = zb;
        za = c * a + conj(sn) * b;
        zb = c * b - sn * a;
      }
      __syncthreads();
    }
  }
}

// one thread per eigenvector: back substitution on the triangular factor
__global__ void trevec_kernel(const c128* __restrict__ T, c128* __restrict__ Y, int k, double small) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k) return;
  c128* y = Y + (int64_t)q * k;
  for (int i = q + 1; i < k; ++i) y[i] = c128{0.0, 0.0};
  y[q] = c128{1.0, 0.0};
  const c128 lam = T[(int64_t)q + (int64_t)q * k];
  for (int i = q - 1; i >= 0; --i) {
    c128 s{0.0, 0.0};
    for (int j = i + 1; j <= q; ++j) s = s + T[(int64_t)i + (int64_t)j * k] * y[j];
    c128 d = T[(int64_t)i + (int64_t)i * k] - lam;
    if (cmod(d) < small) d = c128{small, 0.0};
    y[i] = -(s * recip(d));
    if (cmod(y[i]) > 1e150)  // keep the growing components finite (normalised later)
      for (int j = i; j <= q; ++j) y[j] = y[j] * 1e-150;
  }
}

__global__ void weighted_sum_kernel(c128* __restrict__ Y, const c128* __restrict__ W, int64_t nm, int entries,
                                    const c128* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nm; i += (int64_t)gridDim.x * blockDim.x) {
    c128 acc{0.0, 0.0};
    for (int e = 0; e < entries; ++e) acc = acc + w[e] * W[(int64_t)e * nm + i];
    Y[i] = acc;
  }
}

__global__ void resid_complex_kernel(const c128* __restrict__ AX, const c128* __restrict__ X, int64_t n,
                                     const c128* __restrict__ lam, double* __restrict__ out) {
  __shared__ double red[32];
  const int64_t j = blockIdx.x;
  const c128 l = lam[j];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += abs2(AX[i + j * n] - l * X[i + j * n]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[j] = t;
  }
}

__global__ void frobenius_kernel(const c128* __restrict__ H, int64_t kk, double* __restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < kk; i += blockDim.x) s += abs2(H[i]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    *out = sqrt(t);
  }
}

}  // namespace

void schur_complex(c128* H, c128* Z, int k, int* info, cudaStream_t s) {
  if (k < 1 || k > kSchurMaxK) throw CudaFailure(cudaErrorInvalidValue);
  schur_kernel<<<1, kSchurThreads, 0, s>>>(H, Z, k, info);
  FEAST_LAUNCH_CHECK();
}

void triangular_eigvecs(const c128* T, c128* Y, int k, double small, cudaStream_t s) {
  if (k < 1) return;
  trevec_kernel<<<(k + 127) / 128, 128, 0, s>>>(T, Y, k, small);
  FEAST_LAUNCH_CHECK();
}

void weighted_sum(c128* Y, const c128* W, int64_t nm, int entries, const c128* w, cudaStream_t s) {
  if (nm <= 0) return;
  const int64_t blocks = std::min<int64_t>((nm + 255) / 256, 152 * 16);
  weighted_sum_kernel<<<(unsigned)blocks, 256, 0, s>>>(Y, W, nm, entries, w);
  FEAST_LAUNCH_CHECK();
}

void resid_norms2_complex(const c128* AX, const c128* X, int64_t n, int64_t k, const c128* lam, double* out,
                          cudaStream_t s) {
  if (k <= 0) return;
  resid_complex_kernel<<<(unsigned)k, 256, 0, s>>>(AX, X, n, lam, out);
  FEAST_LAUNCH_CHECK();
}

void frobenius_norm(const c128* H, int64_t k, double* out, cudaStream_t s) {
  frobenius_kernel<<<1, 1024, 0, s>>>(H, k * k, out);
  FEAST_LAUNCH_CHECK();
}

}  // namespace feast
