// Dense FP64 kernels of the Rayleigh-Ritz side (see dense.cuh).
//
// Cholesky and Jacobi are single cooperative launches whose CTAs meet at the
// bounded group barrier of common.cuh; every value read after a barrier that
// another CTA may have written goes through L2 (ld.global.cg).
#include "dense.cuh"

#include <algorithm>

#include "dfloat.cuh"

namespace feast {

namespace {

template <typename S> __device__ __forceinline__ S ldcg(const S* p);
template <> __device__ __forceinline__ double ldcg<double>(const double* p) { return __ldcg(p); }
template <> __device__ __forceinline__ c128 ldcg<c128>(const c128* p) {
  double2 v = __ldcg((const double2*)p);
  return c128{v.x, v.y};
}
template <> __device__ __forceinline__ float ldcg<float>(const float* p) { return __ldcg(p); }
template <> __device__ __forceinline__ c64 ldcg<c64>(const c64* p) {
  float2 v = __ldcg((const float2*)p);
  return c64{v.x, v.y};
}
template <typename S> __device__ __forceinline__ S one();
template <> __device__ __forceinline__ double one<double>() { return 1.0; }
template <> __device__ __forceinline__ c128 one<c128>() { return c128{1.0, 0.0}; }
template <> __device__ __forceinline__ float one<float>() { return 1.0f; }
template <> __device__ __forceinline__ c64 one<c64>() { return c64{1.0f, 0.0f}; }

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}
__device__ double block_sum(double v) {
  __shared__ double sh[32];
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
    sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

inline unsigned grid1d(int64_t total, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, threads), 16384));
}

// ---------------------------------------------------------------------------
template <typename S>
__global__ void hermitize_kernel(S* H, int64_t k, int64_t ld) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    int64_t i = idx % k, j = idx / k;
    if (i > j) continue;
    S a = H[i + j * ld], b = H[j + i * ld];
    if (i == j) {
      H[i + i * ld] = cvt<S>(real_part(a));
    } else {
      S m = (a + conj(b)) * 0.5;
      H[i + j * ld] = m;
      H[j + i * ld] = conj(m);
    }
  }
}

// ---------------------------------------------------------------------------
// Right-looking Cholesky, one column per step, two group barriers per column.
template <typename S>
__global__ void __launch_bounds__(256) chol_kernel(S* G, int64_t k, int64_t ld, CoopWork w, int P) {
  extern __shared__ unsigned char smem_raw[];
  S* row = (S*)smem_raw;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NT = (int64_t)P * blockDim.x;
  const int64_t gw = gt >> 5, nw = NT >> 5;
  const int lane = threadIdx.x & 31;
  unsigned nb = 0;
  for (int64_t j = 0; j < k; ++j) {
    const double gjj = real_part(ldcg(&G[j + j * ld]));
    if (!(gjj > 0.0) || !isfinite(gjj)) {
      if (gt == 0) atomicCAS(&w.info[0], 0, (int)j + 1);
      return;  // every CTA reads the same value and leaves together
    }
    const double rjj = sqrt(gjj);
    const double inv = 1.0 / rjj;
    for (int64_t l = j + 1 + gt; l < k; l += NT) G[j + l * ld] = ldcg(&G[j + l * ld]) * inv;
    if (gt == 0) G[j + j * ld] = cvt<S>(rjj);
    if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
    for (int64_t l = j + 1 + threadIdx.x; l < k; l += blockDim.x) row[l] = ldcg(&G[j + l * ld]);
    __syncthreads();
    for (int64_t l2 = j + 1 + gw; l2 < k; l2 += nw) {
      const S r2 = row[l2];
      for (int64_t l1 = j + 1 + lane; l1 <= l2; l1 += 32) {
        S* g = &G[l1 + l2 * ld];
        *g = ldcg(g) - conj(row[l1]) * r2;
      }
    }
    if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
  }
}

// ---------------------------------------------------------------------------
template <typename S>
__global__ void tri_inv_kernel(const S* R, int64_t k, int64_t ld, S* Ri, int64_t ldi) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= k) return;
  S* x = Ri + c * ldi;
  for (int64_t i = c + 1 + lane; i < k; i += 32) x[i] = num<S>::zero();
  if (lane == 0) x[c] = recip(R[c + c * ld]);
  __syncwarp();
  for (int64_t i = c - 1; i >= 0; --i) {
    S acc = num<S>::zero();
    for (int64_t l = i + 1 + lane; l <= c; l += 32) acc = acc + R[i + l * ld] * x[l];
    if constexpr (std::is_same<S, double>::value) {
      acc = warp_sum(acc);
    } else {
      acc.re = warp_sum(acc.re);
      acc.im = warp_sum(acc.im);
    }
    if (lane == 0) x[i] = -(acc * recip(R[i + i * ld]));
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Jacobi, round-robin (circle-method) ordering: in round r the k/2 disjoint
// pairs are (r, kk-1) and (r+i, r-i) mod (kk-1), i = 1..kk/2-1, kk = k
// rounded up to even (index k is a dummy when k is odd).
template <typename S>
__global__ void __launch_bounds__(256)
jacobi_kernel(S* H, int64_t k, int64_t ld, S* V, int64_t ldv, double tol, CoopWork w, int P, int max_sweeps,
              int init_v) {
  using R = real_t<S>;  // rotations in the working precision (FP32 or FP64)
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NT = (int64_t)P * blockDim.x;
  unsigned nb = 0;
  const int64_t kk = k + (k & 1), np = kk / 2, m1 = kk - 1;
  R* rc = (R*)w.rot;
  R* rs = rc + np;
  S* rse = (S*)(rs + np);  // e s and e c of each pair's rotation
  S* rce = rse + np;
  int* ron = (int*)(rce + np);
  int* rpp = ron + np;
  int* rqq = rpp + np;

  double part = 0.0;
  for (int64_t idx = gt; idx < k * k; idx += NT) {
    const int64_t i = idx % k, j = idx / k;
    if (init_v) V[i + j * ldv] = (i == j) ? one<S>() : num<S>::zero();
    part += abs2(H[i + j * ld]);
  }
  part = block_sum(part);
  if (threadIdx.x == 0) w.partial[blockIdx.x] = part;
  if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
  double fro2 = 0.0;
  for (int q = 0; q < P; ++q) fro2 += __ldcg(&w.partial[q]);
  const R thr = (R)(tol * sqrt(fro2));

  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int64_t r = 0; r < m1; ++r) {
      int any_on = 0;
      for (int64_t i = gt; i < np; i += NT) {
        int64_t a, b;
        if (i == 0) { a = r % m1; b = m1; }
        else { a = (r + i) % m1; b = ((r - i) % m1 + m1) % m1; }
        const int64_t p = a < b ? a : b, q = a < b ? b : a;
        R c = R(1), s = R(0);
        S se = num<S>::zero(), ce = one<S>();
        int on = 0;
        if (q < k) {
          const S apq = ldcg(&H[p + q * ld]);
          const R g = sqrt(abs2(apq));
          if (g > thr) {
            const R app = real_part(ldcg(&H[p + p * ld]));
            const R aqq = real_part(ldcg(&H[q + q * ld]));
            const S e = conj(apq) * (R(1) / g);
            const R tau = (aqq - app) / (R(2) * g);
            const R t = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + hypot(R(1), tau));
            c = R(1) / hypot(R(1), t);
            s = t * c;
            se = e * s;
            ce = e * c;
            on = 1;
          }
        }
        any_on |= on;
        rc[i] = c; rs[i] = s; rse[i] = se; rce[i] = ce; ron[i] = on; rpp[i] = (int)p; rqq[i] = (int)q;
      }
      // a round that rotates no pair skips its update phase and second barrier
      // (late sweeps rotate few pairs): one count per round, read after the barrier
      const int64_t gr = (int64_t)sweep * m1 + r;
      if (__syncthreads_or(any_on) && threadIdx.x == 0) {
        atomicAdd(&w.roundcount[gr], 1u);
        atomicAdd(&w.rotcount[sweep], 1u);
      }
      if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
      if (__ldcg(&w.roundcount[gr]) == 0u) continue;
      const int64_t nblk = np * np;
      for (int64_t task = gt; task < nblk + k * np; task += NT) {
        if (task < nblk) {
          // H stays exactly Hermitian: block (I, J) with I <= J is rotated and
          // written with its mirror (J, I)
          const int64_t I = task % np, J = task / np;
          if (I > J) continue;
          const int onI = __ldcg(&ron[I]), onJ = __ldcg(&ron[J]);
          if (!onI && !onJ) continue;
          const int pI = __ldcg(&rpp[I]), qI = __ldcg(&rqq[I]);
          const int pJ = __ldcg(&rpp[J]), qJ = __ldcg(&rqq[J]);
          const bool vqI = qI < k, vqJ = qJ < k;
          S b00 = ldcg(&H[pI + (int64_t)pJ * ld]);
          S b01 = vqJ ? ldcg(&H[pI + (int64_t)qJ * ld]) : num<S>::zero();
          S b10 = vqI ? ldcg(&H[qI + (int64_t)pJ * ld]) : num<S>::zero();
          S b11 = (vqI && vqJ) ? ldcg(&H[qI + (int64_t)qJ * ld]) : num<S>::zero();
          if (onJ) {
            const R c = __ldcg(&rc[J]), s = __ldcg(&rs[J]);
            const S se = ldcg(&rse[J]), ce = ldcg(&rce[J]);
            S n00 = b00 * c - b01 * se, n01 = b00 * s + b01 * ce;
            S n10 = b10 * c - b11 * se, n11 = b10 * s + b11 * ce;
            b00 = n00; b01 = n01; b10 = n10; b11 = n11;
          }
          if (onI) {
            const R c = __ldcg(&rc[I]), s = __ldcg(&rs[I]);
            const S sec = conj(ldcg(&rse[I])), cec = conj(ldcg(&rce[I]));
            S n00 = b00 * c - b10 * sec, n10 = b00 * s + b10 * cec;
            S n01 = b01 * c - b11 * sec, n11 = b01 * s + b11 * cec;
            b00 = n00; b01 = n01; b10 = n10; b11 = n11;
          }
          if (I == J && onI) {
            b01 = num<S>::zero();
            b10 = num<S>::zero();
            b00 = cvt<S>(real_part(b00));
            b11 = cvt<S>(real_part(b11));
          }
          H[pI + (int64_t)pJ * ld] = b00;
          if (vqJ) H[pI + (int64_t)qJ * ld] = b01;
          if (vqI) H[qI + (int64_t)pJ * ld] = b10;
          if (vqI && vqJ) H[qI + (int64_t)qJ * ld] = b11;
          if (I != J) {
            H[pJ + (int64_t)pI * ld] = conj(b00);
            if (vqJ) H[qJ + (int64_t)pI * ld] = conj(b01);
            if (vqI) H[pJ + (int64_t)qI * ld] = conj(b10);
            if (vqI && vqJ) H[qJ + (int64_t)qI * ld] = conj(b11);
          }
        } else {
          const int64_t tv = task - nblk;
          const int64_t row = tv % k, J = tv / k;
          if (!__ldcg(&ron[J])) continue;
          const int pJ = __ldcg(&rpp[J]), qJ = __ldcg(&rqq[J]);
          const R c = __ldcg(&rc[J]), s = __ldcg(&rs[J]);
          const S se = ldcg(&rse[J]), ce = ldcg(&rce[J]);
          S* vp = &V[row + (int64_t)pJ * ldv];
          S* vq = &V[row + (int64_t)qJ * ldv];
          const S a = ldcg(vp), b = ldcg(vq);
          *vp = a * c - b * se;
          *vq = a * s + b * ce;
        }
      }
      if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
    }
    sweeps = sweep + 1;
    if (__ldcg(&w.rotcount[sweep]) == 0u) break;
  }
  if (gt == 0) w.info[1] = sweeps;
}

// ---------------------------------------------------------------------------
template <typename S>
__global__ void get_diag_kernel(const S* H, int64_t k, int64_t ld, double* d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = real_part(H[i + i * ld]);
}

template <typename S>
__global__ void col_norms2_kernel(const S* X, int64_t n, int64_t ld, double* out) {
  const int64_t j = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += abs2(X[i + j * ld]);
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

template <typename S>
__global__ void col_dots_kernel(const S* X, const S* Y, int64_t n, int64_t ld, double* out) {
  const int64_t j = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += real_part(conj(X[i + j * ld]) * Y[i + j * ld]);
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

template <typename S>
__global__ void resid_norms2_kernel(const S* AX, const S* X, int64_t n, int64_t ld, const double* lam, double* out) {
  const int64_t j = blockIdx.x;
  const double l = lam[j];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += abs2(AX[i + j * ld] - X[i + j * ld] * l);
  s = block_sum(s);
  if (threadIdx.x == 0) out[j] = s;
}

template <typename S>
__global__ void ritz_residual_kernel(S* R, const S* AX, const S* X, int64_t n, int64_t k, int64_t ld,
                                     const double* lam) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    R[i + j * ld] = AX[i + j * ld] - X[i + j * ld] * lam[j];
  }
}

template <typename S>
__global__ void gather_cols_kernel(S* dst, int64_t lddst, const S* src, int64_t ldsrc, int64_t n, const int* idx,
                                   int64_t k, const double* scale) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    S v = src[i + (int64_t)idx[j] * ldsrc];
    if (scale) v = v * scale[j];
    dst[i + j * lddst] = v;
  }
}

// dst (ks x ks, ld ks) = src[idx, idx] (src ld lds)
template <typename S>
__global__ void gather_sub_kernel(S* dst, const S* src, int64_t lds, const int* idx, int64_t ks) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ks * ks; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t % ks, b = t / ks;
    dst[t] = src[idx[a] + (int64_t)idx[b] * lds];
  }
}

// dst[idx, idx] (ld ldd) = src (ks x ks, ld ks)
template <typename S>
__global__ void scatter_sub_kernel(S* dst, int64_t ldd, const S* src, const int* idx, int64_t ks) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ks * ks; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t a = t % ks, b = t / ks;
    dst[idx[a] + (int64_t)idx[b] * ldd] = src[t];
  }
}

// dst[:, idx[j]] = src[:, j]
template <typename S>
__global__ void scatter_cols_kernel(S* dst, int64_t lddst, const S* src, int64_t ldsrc, int64_t n, const int* idx,
                                    int64_t k) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    dst[i + (int64_t)idx[j] * lddst] = src[i + j * ldsrc];
  }
}

template <typename S>
__global__ void scale_cols_kernel(S* X, int64_t n, int64_t k, int64_t ld, const double* scale) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    X[i + j * ld] = X[i + j * ld] * scale[j];
  }
}

template <typename S>
__global__ void accumulate_kernel(S* Xf, int64_t ld, const c128* Y, int64_t n, int64_t m, int nodes,
                                  const c128* w) {
  const int64_t nm = n * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nm; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    if constexpr (std::is_same<S, double>::value) {
      double acc = 0.0;
      for (int j = 0; j < nodes; ++j) acc += 2.0 * (w[j] * Y[(int64_t)j * nm + t]).re;
      Xf[i + c * ld] = acc;
    } else {
      c128 acc{0.0, 0.0};
      for (int j = 0; j < nodes; ++j) {
        acc = acc + w[j] * Y[(int64_t)j * nm + t];
        acc = acc + conj(w[j]) * Y[(int64_t)(nodes + j) * nm + t];
      }
      Xf[i + c * ld] = acc;
    }
  }
}

template <typename S>
__global__ void refine_residual_kernel(c128* R, const S* X, int64_t ldx, const c128* Y, const c128* AY, int64_t n,
                                       int64_t m, const c128* z_e, const int* active) {
  const int e = blockIdx.y;
  const int64_t nm = n * m;
  const c128 z = z_e[e];
  const bool on = active[e] != 0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nm; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    const int64_t o = (int64_t)e * nm + t;
    R[o] = on ? cvt<c128>(X[i + c * ldx]) - z * Y[o] + AY[o] : c128{0.0, 0.0};
  }
}


__global__ void entry_norms2_kernel(const c128* R, const c128* Y, int64_t nm, double* out) {
  const int e = blockIdx.y;
  double sr = 0.0, sy = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nm; t += (int64_t)gridDim.x * blockDim.x) {
    sr += abs2(R[(int64_t)e * nm + t]);
    sy += abs2(Y[(int64_t)e * nm + t]);
  }
  sr = block_sum(sr);
  sy = block_sum(sy);
  if (threadIdx.x == 0) {
    atomicAdd(&out[2 * e], sr);
    atomicAdd(&out[2 * e + 1], sy);
  }
}

// splitmix64 (Steele, Lea & Flood 2014) as a counter-based generator
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

template <typename S>
__global__ void random_normal_kernel(S* X, int64_t n, int64_t m, int64_t ld, unsigned long long seed) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    const unsigned long long h1 = splitmix64(seed ^ splitmix64(2ull * (unsigned long long)t));
    const unsigned long long h2 = splitmix64(seed ^ splitmix64(2ull * (unsigned long long)t + 1ull));
    const double u1 = ((double)(h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double u2 = ((double)(h2 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    if constexpr (std::is_same<S, double>::value) {
      X[i + c * ld] = rad * cs;
    } else {
      X[i + c * ld] = c128{rad * cs * 0.7071067811865476, rad * sn * 0.7071067811865476};
    }
  }
}

template <typename S>
__global__ void copy_matrix_kernel(S* dst, int64_t ldd, const S* src, int64_t lds, int64_t n, int64_t m) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    dst[i + c * ldd] = src[i + c * lds];
  }
}

template <typename S>
__global__ void set_diag_kernel(S* X, int64_t k, int64_t ld, const double* d) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % k, c = t / k;
    X[i + c * ld] = (i == c) ? cvt<S>(d[i]) : num<S>::zero();
  }
}

template <typename S>
__global__ void set_identity_kernel(S* X, int64_t k, int64_t ld) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % k, c = t / k;
    X[i + c * ld] = (i == c) ? one<S>() : num<S>::zero();
  }
}

template <typename S>
__global__ void check_finite_kernel(const S* X, int64_t n, int64_t m, int64_t ld, int* flag) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    if (!isfinite(abs2(X[i + c * ld]))) { *flag = 1; return; }
  }
}

}  // namespace

// ---------------------------------------------------------------------------
size_t coop_work_bytes(int64_t kmax, int num_sms) {
  const int64_t np = (kmax + 2) / 2;
  return 256 * 4 + sizeof(double) * 2 * (size_t)std::max(num_sms, 1024) + 256 +
         sizeof(unsigned) * kMaxSweeps + 256 + sizeof(unsigned) * kMaxSweeps * (size_t)(kmax + 2) + 256 +
         (size_t)np * (2 * sizeof(double) + 2 * sizeof(c128) + 3 * sizeof(int)) + 256;
}

CoopWork coop_work_carve(void* base, int64_t kmax, int num_sms) {
  char* p = (char*)base;
  CoopWork w{};
  w.counter = (unsigned*)p; p += 256;
  w.status = (int*)p; p += 256;
  w.info = (int*)p; p += 256;
  p += 256;
  w.partial = (double*)p; p += ((sizeof(double) * 2 * (size_t)std::max(num_sms, 1024) + 255) & ~size_t(255));
  w.rotcount = (unsigned*)p; p += ((sizeof(unsigned) * kMaxSweeps + 255) & ~size_t(255));
  w.roundcount = (unsigned*)p; p += ((sizeof(unsigned) * kMaxSweeps * (size_t)(kmax + 2) + 255) & ~size_t(255));
  w.rot = p;
  return w;
}

template <typename S> void hermitize(S* H, int64_t k, int64_t ld, cudaStream_t s) {
  hermitize_kernel<S><<<grid1d(k * k), 256, 0, s>>>(H, k, ld);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void cholesky_upper(S* G, int64_t k, int64_t ld, const CoopWork& w, int num_sms, cudaStream_t s) {
  FEAST_CUDA_TRY(cudaMemsetAsync(w.counter, 0, 256 * 3, s));
  const size_t smem = sizeof(S) * (size_t)k;
  if (smem > 48 * 1024)
    FEAST_CUDA_TRY(cudaFuncSetAttribute(chol_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int occ = 0;
  FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, chol_kernel<S>, 256, smem));
  int P = (int)std::min<int64_t>((int64_t)std::max(1, occ) * num_sms, cdiv(k * k / 2 + 1, 256 * 16));
  P = std::max(1, std::min(P, num_sms));
  CoopWork wl = w;
  void* args[] = {&G, &k, &ld, &wl, &P};
  FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)chol_kernel<S>, dim3(P), dim3(256), args, smem, s));
  note_launch();
}

template <typename S>
void tri_inverse_upper(const S* R, int64_t k, int64_t ld, S* Rinv, int64_t ldi, cudaStream_t s) {
  tri_inv_kernel<S><<<(unsigned)cdiv(k * 32, 256), 256, 0, s>>>(R, k, ld, Rinv, ldi);
  FEAST_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Jacobi in double-float arithmetic (FP64-accurate polish on the FP32 pipes).
// The same round-robin sweeps as jacobi_kernel, with H and V stored as
// double-float values (T = dfr for real symmetric, dfc for complex Hermitian
// matrices; 8 or 16 bytes, like double and c128) and every rotation applied
// in double-float.  The rotation parameters are computed in FP64 from the
// pair's entry and the diagonal, which lives in FP64 (dg) and is updated
// there by the closed form d_p - t |h_pq|, d_q + t |h_pq|, so the
// eigenvalues keep FP64 accuracy; the stored diagonal entries are not used.
// ---------------------------------------------------------------------------
template <typename T> struct df_of;
template <> struct df_of<dfr> { using D = double; };
template <> struct df_of<dfc> { using D = c128; };
__device__ __forceinline__ double df_to_d(dfr a) { return a.to_double(); }
__device__ __forceinline__ c128 df_to_d(dfc a) { return c128{a.re.to_double(), a.im.to_double()}; }
__device__ __forceinline__ dfr df_from_d(double x) { return dfr(x); }
__device__ __forceinline__ dfc df_from_d(c128 x) { return dfc{dfr(x.re), dfr(x.im)}; }
__device__ __forceinline__ dfr df_ldcg(const dfr* p) {
  const float2 v = __ldcg((const float2*)p);
  return dfr(v.x, v.y);
}
__device__ __forceinline__ dfc df_ldcg(const dfc* p) {
  const float4 v = __ldcg((const float4*)p);
  return dfc{dfr(v.x, v.y), dfr(v.z, v.w)};
}
__device__ __forceinline__ dfr df_zero(dfr) { return dfr(0.0f, 0.0f); }
__device__ __forceinline__ dfc df_zero(dfc) { return dfc{dfr(0.0f, 0.0f), dfr(0.0f, 0.0f)}; }
__device__ __forceinline__ dfr df_one(dfr) { return dfr(1.0f, 0.0f); }
__device__ __forceinline__ dfc df_one(dfc) { return dfc{dfr(1.0f, 0.0f), dfr(0.0f, 0.0f)}; }
__device__ __forceinline__ dfr df_conj(dfr a) { return a; }
__device__ __forceinline__ dfc df_conj(dfc a) { return dfc{a.re, -a.im}; }
// x c - y u and x s + y v (c, s real; u, v of the storage type)
__device__ __forceinline__ dfr df_mulr(dfr x, dfr c) { return x * c; }
__device__ __forceinline__ dfc df_mulr(dfc x, dfr c) { return dfc{x.re * c, x.im * c}; }
__device__ __forceinline__ dfr df_mul(dfr x, dfr u) { return x * u; }
__device__ __forceinline__ dfc df_mul(dfc x, dfc u) {
  return dfc{x.re * u.re - x.im * u.im, x.re * u.im + x.im * u.re};
}
__device__ __forceinline__ dfr df_sub(dfr a, dfr b) { return a - b; }
__device__ __forceinline__ dfc df_sub(dfc a, dfc b) { return dfc{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ dfr df_add(dfr a, dfr b) { return a + b; }
__device__ __forceinline__ dfc df_add(dfc a, dfc b) { return dfc{a.re + b.re, a.im + b.im}; }

template <typename T>
__global__ void __launch_bounds__(256)
jacobi_df_kernel(T* H, int64_t k, int64_t ld, T* V, int64_t ldv, double* dg, double tol, CoopWork w, int P,
                 int max_sweeps, int init_v) {
  using D = typename df_of<T>::D;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t NT = (int64_t)P * blockDim.x;
  unsigned nb = 0;
  const int64_t kk = k + (k & 1), np = kk / 2, m1 = kk - 1;
  dfr* rc = (dfr*)w.rot;
  dfr* rs = rc + np;
  T* rse = (T*)(rs + np);
  T* rce = rse + np;
  int* ron = (int*)(rce + np);
  int* rpp = ron + np;
  int* rqq = rpp + np;

  double part = 0.0;
  for (int64_t idx = gt; idx < k * k; idx += NT) {
    const int64_t i = idx % k, j = idx / k;
    if (init_v) V[i + j * ldv] = (i == j) ? df_one(T{}) : df_zero(T{});
    const D h = df_to_d(H[i + j * ld]);
    part += abs2(h);
    if (i == j) dg[i] = real_part(h);
  }
  part = block_sum(part);
  if (threadIdx.x == 0) w.partial[blockIdx.x] = part;
  if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
  double fro2 = 0.0;
  for (int q = 0; q < P; ++q) fro2 += __ldcg(&w.partial[q]);
  const double thr = tol * sqrt(fro2);

  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int64_t r = 0; r < m1; ++r) {
      int any_on = 0;
      for (int64_t i = gt; i < np; i += NT) {
        int64_t a, b;
        if (i == 0) { a = r % m1; b = m1; }
        else { a = (r + i) % m1; b = ((r - i) % m1 + m1) % m1; }
        const int64_t p = a < b ? a : b, q = a < b ? b : a;
        double c = 1.0, sn = 0.0;
        D se = cvt<D>(0.0), ce = cvt<D>(1.0);
        int on = 0;
        if (q < k) {
          const D apq = df_to_d(df_ldcg(&H[p + q * ld]));
          const double g = sqrt(abs2(apq));
          if (g > thr) {
            const double app = __ldcg(&dg[p]), aqq = __ldcg(&dg[q]);
            const D e = conj(apq) * (1.0 / g);
            const double tau = (aqq - app) / (2.0 * g);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + hypot(1.0, tau));
            c = 1.0 / hypot(1.0, t);
            sn = t * c;
            se = e * sn;
            ce = e * c;
            dg[p] = app - t * g;
            dg[q] = aqq + t * g;
            on = 1;
          }
        }
        any_on |= on;
        rc[i] = dfr(c); rs[i] = dfr(sn); rse[i] = df_from_d(se); rce[i] = df_from_d(ce);
        ron[i] = on; rpp[i] = (int)p; rqq[i] = (int)q;
      }
      const int64_t gr = (int64_t)sweep * m1 + r;
      if (__syncthreads_or(any_on) && threadIdx.x == 0) {
        atomicAdd(&w.roundcount[gr], 1u);
        atomicAdd(&w.rotcount[sweep], 1u);
      }
      if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
      if (__ldcg(&w.roundcount[gr]) == 0u) continue;
      const int64_t nblk = np * np;
      for (int64_t task = gt; task < nblk + k * np; task += NT) {
        if (task < nblk) {
          const int64_t I = task % np, J = task / np;
          if (I > J) continue;
          const int onI = __ldcg(&ron[I]), onJ = __ldcg(&ron[J]);
          if (!onI && !onJ) continue;
          const int pI = __ldcg(&rpp[I]), qI = __ldcg(&rqq[I]);
          const int pJ = __ldcg(&rpp[J]), qJ = __ldcg(&rqq[J]);
          const bool vqI = qI < k, vqJ = qJ < k;
          if (I == J) {  // the pair's own 2 x 2 block: diagonal from dg, the pair annihilated
            H[pI + (int64_t)pI * ld] = df_from_d(cvt<D>(__ldcg(&dg[pI])));
            if (vqI) {
              H[qI + (int64_t)qI * ld] = df_from_d(cvt<D>(__ldcg(&dg[qI])));
              H[pI + (int64_t)qI * ld] = df_zero(T{});
              H[qI + (int64_t)pI * ld] = df_zero(T{});
            }
            continue;
          }
          T b00 = df_ldcg(&H[pI + (int64_t)pJ * ld]);
          T b01 = vqJ ? df_ldcg(&H[pI + (int64_t)qJ * ld]) : df_zero(T{});
          T b10 = vqI ? df_ldcg(&H[qI + (int64_t)pJ * ld]) : df_zero(T{});
          T b11 = (vqI && vqJ) ? df_ldcg(&H[qI + (int64_t)qJ * ld]) : df_zero(T{});
          if (onJ) {
            const dfr c = df_ldcg(&rc[J]), sn = df_ldcg(&rs[J]);
            const T se = df_ldcg(&rse[J]), ce = df_ldcg(&rce[J]);
            const T n00 = df_sub(df_mulr(b00, c), df_mul(b01, se)), n01 = df_add(df_mulr(b00, sn), df_mul(b01, ce));
            const T n10 = df_sub(df_mulr(b10, c), df_mul(b11, se)), n11 = df_add(df_mulr(b10, sn), df_mul(b11, ce));
            b00 = n00; b01 = n01; b10 = n10; b11 = n11;
          }
          if (onI) {
            const dfr c = df_ldcg(&rc[I]), sn = df_ldcg(&rs[I]);
            const T sec = df_conj(df_ldcg(&rse[I])), cec = df_conj(df_ldcg(&rce[I]));
            const T n00 = df_sub(df_mulr(b00, c), df_mul(b10, sec)), n10 = df_add(df_mulr(b00, sn), df_mul(b10, cec));
            const T n01 = df_sub(df_mulr(b01, c), df_mul(b11, sec)), n11 = df_add(df_mulr(b01, sn), df_mul(b11, cec));
            b00 = n00; b01 = n01; b10 = n10; b11 = n11;
          }
          H[pI + (int64_t)pJ * ld] = b00;
          if (vqJ) H[pI + (int64_t)qJ * ld] = b01;
          if (vqI) H[qI + (int64_t)pJ * ld] = b10;
          if (vqI && vqJ) H[qI + (int64_t)qJ * ld] = b11;
          H[pJ + (int64_t)pI * ld] = df_conj(b00);
          if (vqJ) H[qJ + (int64_t)pI * ld] = df_conj(b01);
          if (vqI) H[pJ + (int64_t)qI * ld] = df_conj(b10);
          if (vqI && vqJ) H[qJ + (int64_t)qI * ld] = df_conj(b11);
        } else {
          const int64_t tv = task - nblk;
          const int64_t row = tv % k, J = tv / k;
          if (!__ldcg(&ron[J])) continue;
          const int pJ = __ldcg(&rpp[J]), qJ = __ldcg(&rqq[J]);
          const dfr c = df_ldcg(&rc[J]), sn = df_ldcg(&rs[J]);
          const T se = df_ldcg(&rse[J]), ce = df_ldcg(&rce[J]);
          T* vp = &V[row + (int64_t)pJ * ldv];
          T* vq = &V[row + (int64_t)qJ * ldv];
          const T a = df_ldcg(vp), b = df_ldcg(vq);
          *vp = df_sub(df_mulr(a, c), df_mul(b, se));
          *vq = df_add(df_mulr(a, sn), df_mul(b, ce));
        }
      }
      if (!group_barrier(w.counter, (++nb) * (unsigned)P, w.status)) return;
    }
    sweeps = sweep + 1;
    if (__ldcg(&w.rotcount[sweep]) == 0u) break;
  }
  if (gt == 0) w.info[1] = sweeps;
}

// in place: FP64 storage <-> double-float storage (same bytes per element)
template <typename S, typename T>
__global__ void to_df_kernel(S* X, int64_t k, int64_t ld) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % k, j = t / k;
    S* e = &X[i + j * ld];
    const T v = df_from_d(*e);
    *reinterpret_cast<T*>(e) = v;
  }
}
template <typename S, typename T>
__global__ void from_df_kernel(S* X, int64_t k, int64_t ld, const double* dg) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < k * k; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % k, j = t / k;
    S* e = &X[i + j * ld];
    const T v = *reinterpret_cast<const T*>(e);
    *e = (dg && i == j) ? cvt<S>(dg[i]) : df_to_d(v);
  }
}

template <typename S>
void jacobi_eigh(S* H, int64_t k, int64_t ld, S* V, int64_t ldv, double tol, const CoopWork& w, int num_sms,
                 cudaStream_t s, int max_sweeps, bool init_v) {
  FEAST_CUDA_TRY(cudaMemsetAsync(w.counter, 0, 256 * 3, s));
  FEAST_CUDA_TRY(cudaMemsetAsync(w.rotcount, 0, sizeof(unsigned) * kMaxSweeps, s));
  FEAST_CUDA_TRY(cudaMemsetAsync(w.roundcount, 0, sizeof(unsigned) * kMaxSweeps * (size_t)(k + 2), s));
  int occ = 0;
  FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_kernel<S>, 256, 0));
  const int64_t tasks = (k / 2 + 1) * (k / 2 + 1) + k * (k / 2 + 1);
  int P = (int)std::min<int64_t>((int64_t)std::max(1, occ) * num_sms, cdiv(tasks, 256 * 8));
  P = std::max(1, std::min(P, num_sms));
  int maxs = std::max(1, std::min(max_sweeps, kMaxSweeps));
  int iv = init_v ? 1 : 0;
  CoopWork wl = w;
  void* args[] = {&H, &k, &ld, &V, &ldv, &tol, &wl, &P, &maxs, &iv};
  FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_kernel<S>, dim3(P), dim3(256), args, 0, s));
  note_launch();
}

template <typename S>
void jacobi_eigh_df(S* H, int64_t k, int64_t ld, S* V, int64_t ldv, double* dg, double tol, const CoopWork& w,
                    int num_sms, cudaStream_t s, int max_sweeps, bool init_v) {
  using T = typename std::conditional<is_cx<S>::value, dfc, dfr>::type;
  static_assert(sizeof(T) == sizeof(S), "double-float storage takes the FP64 element's bytes");
  FEAST_CUDA_TRY(cudaMemsetAsync(w.counter, 0, 256 * 3, s));
  FEAST_CUDA_TRY(cudaMemsetAsync(w.rotcount, 0, sizeof(unsigned) * kMaxSweeps, s));
  FEAST_CUDA_TRY(cudaMemsetAsync(w.roundcount, 0, sizeof(unsigned) * kMaxSweeps * (size_t)(k + 2), s));
  to_df_kernel<S, T><<<grid1d(k * k), 256, 0, s>>>(H, k, ld);
  FEAST_LAUNCH_CHECK();
  if (!init_v) {
    to_df_kernel<S, T><<<grid1d(k * k), 256, 0, s>>>(V, k, ldv);
    FEAST_LAUNCH_CHECK();
  }
  int occ = 0;
  FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, jacobi_df_kernel<T>, 256, 0));
  const int64_t tasks = (k / 2 + 1) * (k / 2 + 1) + k * (k / 2 + 1);
  int P = (int)std::min<int64_t>((int64_t)std::max(1, occ) * num_sms, cdiv(tasks, 256 * 8));
  P = std::max(1, std::min(P, num_sms));
  int maxs = std::max(1, std::min(max_sweeps, kMaxSweeps));
  int iv = init_v ? 1 : 0;
  CoopWork wl = w;
  T* Ht = reinterpret_cast<T*>(H);
  T* Vt = reinterpret_cast<T*>(V);
  void* args[] = {&Ht, &k, &ld, &Vt, &ldv, &dg, &tol, &wl, &P, &maxs, &iv};
  FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)jacobi_df_kernel<T>, dim3(P), dim3(256), args, 0, s));
  note_launch();
  from_df_kernel<S, T><<<grid1d(k * k), 256, 0, s>>>(H, k, ld, dg);
  FEAST_LAUNCH_CHECK();
  from_df_kernel<S, T><<<grid1d(k * k), 256, 0, s>>>(V, k, ldv, nullptr);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void get_diag(const S* H, int64_t k, int64_t ld, double* d, cudaStream_t s) {
  get_diag_kernel<S><<<grid1d(k), 256, 0, s>>>(H, k, ld, d);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void col_norms2(const S* X, int64_t n, int64_t k, int64_t ld, double* out, cudaStream_t s) {
  if (k <= 0) return;
  col_norms2_kernel<S><<<(unsigned)k, 256, 0, s>>>(X, n, ld, out);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void col_dots_re(const S* X, const S* Y, int64_t n, int64_t k, int64_t ld, double* out, cudaStream_t s) {
  if (k <= 0) return;
  col_dots_kernel<S><<<(unsigned)k, 256, 0, s>>>(X, Y, n, ld, out);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void resid_norms2(const S* AX, const S* X, int64_t n, int64_t k, int64_t ld, const double* lam, double* out,
                  cudaStream_t s) {
  if (k <= 0) return;
  resid_norms2_kernel<S><<<(unsigned)k, 256, 0, s>>>(AX, X, n, ld, lam, out);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void ritz_residual(S* R, const S* AX, const S* X, int64_t n, int64_t k, int64_t ld, const double* lam, cudaStream_t s) {
  ritz_residual_kernel<S><<<grid1d(n * k), 256, 0, s>>>(R, AX, X, n, k, ld, lam);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void gather_cols(S* dst, int64_t lddst, const S* src, int64_t ldsrc, int64_t n, const int* idx, int64_t k,
                 const double* scale, cudaStream_t s) {
  if (k <= 0) return;
  gather_cols_kernel<S><<<grid1d(n * k), 256, 0, s>>>(dst, lddst, src, ldsrc, n, idx, k, scale);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void gather_sub(S* dst, const S* src, int64_t lds, const int* idx, int64_t ks, cudaStream_t s) {
  if (ks <= 0) return;
  gather_sub_kernel<S><<<grid1d(ks * ks), 256, 0, s>>>(dst, src, lds, idx, ks);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void scatter_sub(S* dst, int64_t ldd, const S* src, const int* idx, int64_t ks, cudaStream_t s) {
  if (ks <= 0) return;
  scatter_sub_kernel<S><<<grid1d(ks * ks), 256, 0, s>>>(dst, ldd, src, idx, ks);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void scatter_cols(S* dst, int64_t lddst, const S* src, int64_t ldsrc, int64_t n, const int* idx, int64_t k,
                  cudaStream_t s) {
  if (k <= 0) return;
  scatter_cols_kernel<S><<<grid1d(n * k), 256, 0, s>>>(dst, lddst, src, ldsrc, n, idx, k);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void scale_cols(S* X, int64_t n, int64_t k, int64_t ld, const double* scale, cudaStream_t s) {
  if (k <= 0) return;
  scale_cols_kernel<S><<<grid1d(n * k), 256, 0, s>>>(X, n, k, ld, scale);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void accumulate_filter(S* Xf, int64_t ld, const c128* Y, int64_t n, int64_t m, int nodes, const c128* w,
                       cudaStream_t s) {
  accumulate_kernel<S><<<grid1d(n * m), 256, 0, s>>>(Xf, ld, Y, n, m, nodes, w);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void refine_residual(c128* R, const S* X, int64_t ldx, const c128* Y, const c128* AY, int64_t n, int64_t m,
                     int entries, const c128* z_e, const int* active, cudaStream_t s) {
  dim3 g(grid1d(n * m), entries);
  refine_residual_kernel<S><<<g, 256, 0, s>>>(R, X, ldx, Y, AY, n, m, z_e, active);
  FEAST_LAUNCH_CHECK();
}


void entry_norms2(const c128* R, const c128* Y, int64_t n, int64_t m, int entries, double* out, cudaStream_t s) {
  FEAST_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double) * 2 * entries, s));
  dim3 g((unsigned)std::min<int64_t>(cdiv(n * m, 256), 512), entries);
  entry_norms2_kernel<<<g, 256, 0, s>>>(R, Y, n * m, out);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void random_normal(S* X, int64_t n, int64_t m, int64_t ld, unsigned long long seed,
                                         cudaStream_t s) {
  random_normal_kernel<S><<<grid1d(n * m), 256, 0, s>>>(X, n, m, ld, seed);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void copy_matrix(S* dst, int64_t ldd, const S* src, int64_t lds, int64_t n, int64_t m,
                                       cudaStream_t s) {
  if (n <= 0 || m <= 0) return;
  copy_matrix_kernel<S><<<grid1d(n * m), 256, 0, s>>>(dst, ldd, src, lds, n, m);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void set_diag(S* X, int64_t k, int64_t ld, const double* d, cudaStream_t s) {
  set_diag_kernel<S><<<grid1d(k * k), 256, 0, s>>>(X, k, ld, d);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void set_identity(S* X, int64_t k, int64_t ld, cudaStream_t s) {
  set_identity_kernel<S><<<grid1d(k * k), 256, 0, s>>>(X, k, ld);
  FEAST_LAUNCH_CHECK();
}

template <typename S> void check_finite(const S* X, int64_t n, int64_t m, int64_t ld, int* flag, cudaStream_t s) {
  check_finite_kernel<S><<<grid1d(n * m), 256, 0, s>>>(X, n, m, ld, flag);
  FEAST_LAUNCH_CHECK();
}

// ---------------------------------------------------------------------------
// Block Jacobi (low-precision first phase of the two-phase eigensolver).
// Rows are grouped in blocks of BJ_B; in round r the blocks are paired by the
// same round-robin schedule as the scalar kernel.  One CTA per pair
// diagonalises its (2 BJ_B)-square subproblem in shared memory with one
// cyclic Jacobi sweep and writes the accumulated unitary U; a second launch
// forms U_P^H H[P, Q] U_Q for every pair of pairs and V[:, P] U_P.  Each
// output tile reads only its own input tile, so the rounds need no grid-wide
// barrier; a sweep is nb - 1 rounds instead of k - 1.
constexpr int BJ_B = 16, BJ_P = 2 * BJ_B;

__device__ __forceinline__ void bj_pair(int ip, int r, int nbe, int& I, int& J) {
  const int m1 = nbe - 1;
  int a, b;
  if (ip == 0) { a = r % m1; b = m1; }
  else { a = (r + ip) % m1; b = ((r - ip) % m1 + m1) % m1; }
  I = a < b ? a : b;
  J = a < b ? b : a;
}
// global row of subproblem index t of pair (I, J), or -1 (dummy block)
__device__ __forceinline__ int bj_row(int t, int I, int J, int nb) {
  const int blk = t < BJ_B ? I : J;
  return blk < nb ? blk * BJ_B + (t % BJ_B) : -1;
}

template <typename S>
__global__ void __launch_bounds__(256) bj_solve_kernel(const S* __restrict__ HP, int64_t ld, int nb, int nbe, int r,
                                                       float thr, S* __restrict__ U, int* rotated) {
  using R = real_t<S>;
  __shared__ S A[BJ_P][BJ_P + 1];
  __shared__ S Us[BJ_P][BJ_P + 1];
  __shared__ R pc[BJ_B], ps[BJ_B];
  __shared__ S pe[BJ_B];
  __shared__ int pon[BJ_B], pp[BJ_B], pq[BJ_B];
  __shared__ int any;
  const int ip = blockIdx.x, t = threadIdx.x;
  int I, J;
  bj_pair(ip, r, nbe, I, J);
  for (int l = t; l < BJ_P * BJ_P; l += blockDim.x) {
    const int i = l % BJ_P, j = l / BJ_P;
    const int gi = bj_row(i, I, J, nb), gj = bj_row(j, I, J, nb);
    A[i][j] = (gi >= 0 && gj >= 0) ? HP[gi + (int64_t)gj * ld] : num<S>::zero();
    Us[i][j] = i == j ? one<S>() : num<S>::zero();
  }
  if (t == 0) any = 0;
  __syncthreads();
  constexpr int m1 = BJ_P - 1;
  for (int rr = 0; rr < m1; ++rr) {
    if (t < BJ_B) {
      int a, b;
      if (t == 0) { a = rr % m1; b = m1; }
      else { a = (rr + t) % m1; b = ((rr - t) % m1 + m1) % m1; }
      const int p = a < b ? a : b, q = a < b ? b : a;
      R c = R(1), sn = R(0);
      S e = one<S>();
      int on = 0;
      const S apq = A[p][q];
      const R g = sqrt(abs2(apq));
      if (g > thr) {
        const R app = real_part(A[p][p]), aqq = real_part(A[q][q]);
        e = conj(apq) * (R(1) / g);
        const R tau = (aqq - app) / (R(2) * g);
        const R tt = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + hypot(R(1), tau));
        c = R(1) / hypot(R(1), tt);
        sn = tt * c;
        on = 1;
        any = 1;
      }
      pc[t] = c; ps[t] = sn; pe[t] = e; pon[t] = on; pp[t] = p; pq[t] = q;
    }
    __syncthreads();
    {
      // 2 x 2 block (I', J') of the rows of pair I' and the columns of pair J'
      const int bI = t % BJ_B, bJ = t / BJ_B;
      const int onI = pon[bI], onJ = pon[bJ];
      if (onI || onJ) {
        const int pI = pp[bI], qI = pq[bI], pJ = pp[bJ], qJ = pq[bJ];
        S b00 = A[pI][pJ], b01 = A[pI][qJ], b10 = A[qI][pJ], b11 = A[qI][qJ];
        if (onJ) {
          const R c = pc[bJ], sn = ps[bJ];
          const S se = pe[bJ] * sn, ce = pe[bJ] * c;
          S n00 = b00 * c - b01 * se, n01 = b00 * sn + b01 * ce;
          S n10 = b10 * c - b11 * se, n11 = b10 * sn + b11 * ce;
          b00 = n00; b01 = n01; b10 = n10; b11 = n11;
        }
        if (onI) {
          const R c = pc[bI], sn = ps[bI];
          const S ec = conj(pe[bI]);
          const S sec = ec * sn, cec = ec * c;
          S n00 = b00 * c - b10 * sec, n10 = b00 * sn + b10 * cec;
          S n01 = b01 * c - b11 * sec, n11 = b01 * sn + b11 * cec;
          b00 = n00; b01 = n01; b10 = n10; b11 = n11;
        }
        if (bI == bJ && onI) {
          b01 = num<S>::zero();
          b10 = num<S>::zero();
          b00 = cvt<S>(real_part(b00));
          b11 = cvt<S>(real_part(b11));
        }
        A[pI][pJ] = b00; A[pI][qJ] = b01; A[qI][pJ] = b10; A[qI][qJ] = b11;
      }
      // U <- U G_J' for the columns of each rotated pair
      for (int l = t; l < BJ_P * BJ_B; l += blockDim.x) {
        const int row = l % BJ_P, j = l / BJ_P;
        if (!pon[j]) continue;
        const int p = pp[j], q = pq[j];
        const R c = pc[j], sn = ps[j];
        const S e = pe[j];
        const S a = Us[row][p], b = Us[row][q];
        Us[row][p] = a * c - b * (e * sn);
        Us[row][q] = a * sn + b * (e * c);
      }
    }
    __syncthreads();
  }
  for (int l = t; l < BJ_P * BJ_P; l += blockDim.x) {
    const int i = l % BJ_P, j = l / BJ_P;
    U[(int64_t)ip * BJ_P * BJ_P + i + j * BJ_P] = Us[i][j];
  }
  if (t == 0 && any) atomicOr(rotated, 1);
}

// H[P, Q] <- U_P^H H[P, Q] U_Q for pair tiles (P, Q) (grid npairs x npairs)
template <typename S>
__global__ void __launch_bounds__(256) bj_apply_h_kernel(S* HP, int64_t ld, int nb, int nbe, int r,
                                                         const S* __restrict__ U) {
  __shared__ S T[BJ_P][BJ_P + 1];
  __shared__ S X[BJ_P][BJ_P + 1];
  __shared__ S UPs[BJ_P][BJ_P + 1];
  __shared__ S UQs[BJ_P][BJ_P + 1];
  const int P = blockIdx.x, Q = blockIdx.y, t = threadIdx.x;
  int IP, JP, IQ, JQ;
  bj_pair(P, r, nbe, IP, JP);
  bj_pair(Q, r, nbe, IQ, JQ);
  for (int l = t; l < BJ_P * BJ_P; l += blockDim.x) {
    const int i = l % BJ_P, j = l / BJ_P;
    const int gi = bj_row(i, IP, JP, nb), gj = bj_row(j, IQ, JQ, nb);
    T[i][j] = (gi >= 0 && gj >= 0) ? HP[gi + (int64_t)gj * ld] : num<S>::zero();
    UPs[i][j] = U[(int64_t)P * BJ_P * BJ_P + l];
    UQs[i][j] = U[(int64_t)Q * BJ_P * BJ_P + l];
  }
  __syncthreads();
  for (int l = t; l < BJ_P * BJ_P; l += blockDim.x) {
    const int i = l % BJ_P, j = l / BJ_P;
    S acc = num<S>::zero();
#pragma unroll 8
    for (int m = 0; m < BJ_P; ++m) acc = acc + T[i][m] * UQs[m][j];
    X[i][j] = acc;
  }
  __syncthreads();
  for (int l = t; l < BJ_P * BJ_P; l += blockDim.x) {
    const int i = l % BJ_P, j = l / BJ_P;
    const int gi = bj_row(i, IP, JP, nb), gj = bj_row(j, IQ, JQ, nb);
    if (gi < 0 || gj < 0) continue;
    S acc = num<S>::zero();
#pragma unroll 8
    for (int m = 0; m < BJ_P; ++m) acc = acc + conj(UPs[m][i]) * X[m][j];
    HP[gi + (int64_t)gj * ld] = acc;
  }
}

// V[rows, P] <- V[rows, P] U_P for 32-row chunks (grid npairs x kp / 32)
template <typename S>
__global__ void __launch_bounds__(256) bj_apply_v_kernel(S* VP, int64_t ld, int kp, int nb, int nbe, int r,
                                                         const S* __restrict__ U) {
  __shared__ S W[BJ_P][BJ_P + 1];
  __shared__ S UPs[BJ_P][BJ_P + 1];
  const int P = blockIdx.x, t = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.y * BJ_P;
  int IP, JP;
  bj_pair(P, r, nbe, IP, JP);
  for (int l = t; l < BJ_P * BJ_P; l += blockDim.x) {
    const int i = l % BJ_P, j = l / BJ_P;
    const int gj = bj_row(j, IP, JP, nb);
    W[i][j] = (gj >= 0 && r0 + i < kp) ? VP[(r0 + i) + (int64_t)gj * ld] : num<S>::zero();
    UPs[i][j] = U[(int64_t)P * BJ_P * BJ_P + l];
  }
  __syncthreads();
  for (int l = t; l < BJ_P * BJ_P; l += blockDim.x) {
    const int i = l % BJ_P, j = l / BJ_P;
    const int gj = bj_row(j, IP, JP, nb);
    if (gj < 0 || r0 + i >= kp) continue;
    S acc = num<S>::zero();
#pragma unroll 8
    for (int m = 0; m < BJ_P; ++m) acc = acc + W[i][m] * UPs[m][j];
    VP[(r0 + i) + (int64_t)gj * ld] = acc;
  }
}

// HP (kp x kp) <- H (k x k, ld k) converted and zero-padded; VP <- I
template <typename F, typename S>
__global__ void bj_load_kernel(F* HP, F* VP, int64_t kp, const S* H, int64_t k) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < kp * kp;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % kp, j = idx / kp;
    HP[idx] = (i < k && j < k) ? cvt<F>(H[i + j * k]) : num<F>::zero();
    VP[idx] = i == j ? one<F>() : num<F>::zero();
  }
}

template <typename F>
__global__ void bj_store_kernel(F* V, int64_t k, const F* VP, int64_t kp) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % k, j = idx / k;
    V[idx] = VP[i + j * kp];
  }
}

template <typename To, typename From>
__global__ void convert_matrix_kernel(To* dst, int64_t ldd, const From* src, int64_t lds, int64_t n, int64_t m) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    dst[i + c * ldd] = cvt<To>(src[i + c * lds]);
  }
}

template <typename To, typename From>
void convert_matrix(To* dst, int64_t ldd, const From* src, int64_t lds, int64_t n, int64_t m, cudaStream_t s) {
  if (n <= 0 || m <= 0) return;
  convert_matrix_kernel<To, From><<<grid1d(n * m), 256, 0, s>>>(dst, ldd, src, lds, n, m);
  FEAST_LAUNCH_CHECK();
}
template void convert_matrix<float, double>(float*, int64_t, const double*, int64_t, int64_t, int64_t, cudaStream_t);
template void convert_matrix<double, float>(double*, int64_t, const float*, int64_t, int64_t, int64_t, cudaStream_t);
template void convert_matrix<c64, c128>(c64*, int64_t, const c128*, int64_t, int64_t, int64_t, cudaStream_t);
template void convert_matrix<c128, c64>(c128*, int64_t, const c64*, int64_t, int64_t, int64_t, cudaStream_t);
template void convert_matrix<c128, double>(c128*, int64_t, const double*, int64_t, int64_t, int64_t, cudaStream_t);
template void jacobi_eigh<float>(float*, int64_t, int64_t, float*, int64_t, double, const CoopWork&, int, cudaStream_t,
                                 int, bool);
template void jacobi_eigh<c64>(c64*, int64_t, int64_t, c64*, int64_t, double, const CoopWork&, int, cudaStream_t, int,
                               bool);

int64_t block_jacobi_pad(int64_t k) { return cdiv(k, BJ_B) * BJ_B; }
size_t block_jacobi_u_bytes(int64_t kmax) {
  const int64_t nb = cdiv(kmax, BJ_B), nbe = nb + (nb & 1);
  return (size_t)(nbe / 2) * BJ_P * BJ_P * sizeof(c128);
}

template <typename F, typename S>
int block_jacobi(const S* H, int64_t k, F* V, double thr, F* HP, F* VP, F* Ubuf, int* d_rot, int max_sweeps,
                 cudaStream_t s) {
  const int64_t kp = block_jacobi_pad(k);
  const int nb = (int)(kp / BJ_B), nbe = nb + (nb & 1), npairs = nbe / 2, rounds = nbe - 1;
  bj_load_kernel<F, S><<<grid1d(kp * kp), 256, 0, s>>>(HP, VP, kp, H, k);
  FEAST_LAUNCH_CHECK();
  int sweeps = 0;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    FEAST_CUDA_TRY(cudaMemsetAsync(d_rot, 0, sizeof(int), s));
    for (int r = 0; r < rounds; ++r) {
      bj_solve_kernel<F><<<npairs, 256, 0, s>>>(HP, kp, nb, nbe, r, (float)thr, Ubuf, d_rot);
      FEAST_LAUNCH_CHECK();
      bj_apply_h_kernel<F><<<dim3(npairs, npairs), 256, 0, s>>>(HP, kp, nb, nbe, r, Ubuf);
      FEAST_LAUNCH_CHECK();
      bj_apply_v_kernel<F><<<dim3(npairs, (unsigned)(kp / BJ_P + (kp % BJ_P != 0))), 256, 0, s>>>(VP, kp, (int)kp, nb,
                                                                                                 nbe, r, Ubuf);
      FEAST_LAUNCH_CHECK();
    }
    ++sweeps;
    int rot = 0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(&rot, d_rot, sizeof(int), cudaMemcpyDeviceToHost, s));
    FEAST_CUDA_TRY(cudaStreamSynchronize(s));
    if (!rot) break;
  }
  bj_store_kernel<F><<<grid1d(k * k), 256, 0, s>>>(V, k, VP, kp);
  FEAST_LAUNCH_CHECK();
  return sweeps;
}
template int block_jacobi<float, double>(const double*, int64_t, float*, double, float*, float*, float*, int*, int,
                                         cudaStream_t);
template int block_jacobi<c64, c128>(const c128*, int64_t, c64*, double, c64*, c64*, c64*, int*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Cluster finish of the FP64 Jacobi.  Once only pairs inside groups of nearly
// equal diagonal entries still exceed the threshold, a full sweep walks every
// round (with a grid barrier each) to rotate a few pairs.  Instead, the
// above-threshold pairs are listed, grouped into connected index sets on the
// host, and each set's submatrix is diagonalised by cyclic Jacobi in one CTA's
// shared memory; its unitary then updates the set's columns of V.

// pairs (i < j) with |h_ij| > thr: count in *cnt, the first cap in list
template <typename S>
__global__ void offdiag_scan_kernel(const S* H, int64_t k, int64_t ld, double thr2, int* cnt, int* list, int cap) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < k * k;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % k, j = idx / k;
    if (i < j && abs2(H[i + j * ld]) > thr2) {
      const int pos = atomicAdd(cnt, 1);
      if (pos < cap) {
        list[2 * pos] = (int)i;
        list[2 * pos + 1] = (int)j;
      }
    }
  }
}

constexpr int CJ_LD = kClusterMax + 1;

// one CTA per index set c = idx[off[c] .. off[c+1]) (ascending, size <= kClusterMax)
template <typename S>
__global__ void __launch_bounds__(256) cluster_jacobi_kernel(S* H, int64_t ld, const int* __restrict__ idx,
                                                             const int* __restrict__ off, double thr, int max_sweeps,
                                                             S* __restrict__ Ubuf, int* sweeps_out) {
  using R = real_t<S>;
  extern __shared__ unsigned char cj_smem[];
  S* A = reinterpret_cast<S*>(cj_smem);                 // m x m, row stride CJ_LD
  S* U = A + kClusterMax * CJ_LD;
  __shared__ R pc[kClusterMax / 2], ps[kClusterMax / 2];
  __shared__ S pe[kClusterMax / 2];
  __shared__ int pon[kClusterMax / 2], pp[kClusterMax / 2], pq[kClusterMax / 2];
  __shared__ int any;
  const int c = blockIdx.x, t = threadIdx.x;
  const int* ix = idx + off[c];
  const int m = off[c + 1] - off[c];
  const int mm = m + (m & 1), np = mm / 2, m1 = mm - 1;
  for (int l = t; l < m * m; l += blockDim.x) {
    const int i = l % m, j = l / m;
    A[i * CJ_LD + j] = H[ix[i] + (int64_t)ix[j] * ld];
    U[i * CJ_LD + j] = i == j ? one<S>() : num<S>::zero();
  }
  __syncthreads();
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    if (t == 0) any = 0;
    __syncthreads();
    for (int r = 0; r < m1; ++r) {
      if (t < np) {
        int a, b;
        if (t == 0) { a = r % m1; b = m1; }
        else { a = (r + t) % m1; b = ((r - t) % m1 + m1) % m1; }
        const int p = a < b ? a : b, q = a < b ? b : a;
        R cs = R(1), sn = R(0);
        S e = one<S>();
        int on = 0;
        if (q < m) {
          const S apq = A[p * CJ_LD + q];
          const R g = sqrt(abs2(apq));
          if (g > thr) {
            const R app = real_part(A[p * CJ_LD + p]), aqq = real_part(A[q * CJ_LD + q]);
            e = conj(apq) * (R(1) / g);
            const R tau = (aqq - app) / (R(2) * g);
            const R tt = (tau >= R(0) ? R(1) : R(-1)) / (fabs(tau) + hypot(R(1), tau));
            cs = R(1) / hypot(R(1), tt);
            sn = tt * cs;
            on = 1;
            any = 1;
          }
        }
        pc[t] = cs; ps[t] = sn; pe[t] = e; pon[t] = on; pp[t] = p; pq[t] = q;
      }
      __syncthreads();
      // 2 x 2 blocks (rows of pair I, columns of pair J), as in jacobi_kernel
      for (int task = t; task < np * np; task += blockDim.x) {
        const int I = task % np, J = task / np;
        const int onI = pon[I], onJ = pon[J];
        if (!onI && !onJ) continue;
        const int pI = pp[I], qI = pq[I], pJ = pp[J], qJ = pq[J];
        const bool vqI = qI < m, vqJ = qJ < m;
        S b00 = A[pI * CJ_LD + pJ];
        S b01 = vqJ ? A[pI * CJ_LD + qJ] : num<S>::zero();
        S b10 = vqI ? A[qI * CJ_LD + pJ] : num<S>::zero();
        S b11 = (vqI && vqJ) ? A[qI * CJ_LD + qJ] : num<S>::zero();
        if (onJ) {
          const R cs = pc[J], sn = ps[J];
          const S se = pe[J] * sn, ce = pe[J] * cs;
          S n00 = b00 * cs - b01 * se, n01 = b00 * sn + b01 * ce;
          S n10 = b10 * cs - b11 * se, n11 = b10 * sn + b11 * ce;
          b00 = n00; b01 = n01; b10 = n10; b11 = n11;
        }
        if (onI) {
          const R cs = pc[I], sn = ps[I];
          const S ec = conj(pe[I]);
          const S sec = ec * sn, cec = ec * cs;
          S n00 = b00 * cs - b10 * sec, n10 = b00 * sn + b10 * cec;
          S n01 = b01 * cs - b11 * sec, n11 = b01 * sn + b11 * cec;
          b00 = n00; b01 = n01; b10 = n10; b11 = n11;
        }
        if (I == J && onI) {
          b01 = num<S>::zero();
          b10 = num<S>::zero();
          b00 = cvt<S>(real_part(b00));
          b11 = cvt<S>(real_part(b11));
        }
        A[pI * CJ_LD + pJ] = b00;
        if (vqJ) A[pI * CJ_LD + qJ] = b01;
        if (vqI) A[qI * CJ_LD + pJ] = b10;
        if (vqI && vqJ) A[qI * CJ_LD + qJ] = b11;
      }
      // U <- U G_J for the columns of each rotated pair
      for (int task = t; task < m * np; task += blockDim.x) {
        const int row = task % m, J = task / m;
        if (!pon[J]) continue;
        const int p = pp[J], q = pq[J];
        const R cs = pc[J], sn = ps[J];
        const S e = pe[J];
        const S a = U[row * CJ_LD + p], b = U[row * CJ_LD + q];
        U[row * CJ_LD + p] = a * cs - b * (e * sn);
        U[row * CJ_LD + q] = a * sn + b * (e * cs);
      }
      __syncthreads();
    }
    const int rotated = any;
    __syncthreads();
    if (!rotated) break;
  }
  for (int l = t; l < m * m; l += blockDim.x) {
    const int i = l % m, j = l / m;
    H[ix[i] + (int64_t)ix[j] * ld] = A[i * CJ_LD + j];
    Ubuf[(int64_t)c * kClusterMax * kClusterMax + i + (int64_t)j * kClusterMax] = U[i * CJ_LD + j];
  }
  if (t == 0) sweeps_out[c] = sweep + (sweep < max_sweeps ? 1 : 0);
}

// V[rows, set c] <- V[rows, set c] U_c for 64-row chunks (grid nsets x ceil(k / 64))
template <typename S>
__global__ void __launch_bounds__(256) cluster_apply_v_kernel(S* V, int64_t k, int64_t ldv, const int* __restrict__ idx,
                                                              const int* __restrict__ off, const S* __restrict__ Ubuf) {
  extern __shared__ unsigned char cj_smem[];
  S* W = reinterpret_cast<S*>(cj_smem);                 // 64 rows x m, row stride CJ_LD
  S* U = W + 64 * CJ_LD;                                // m x m, row stride CJ_LD
  const int c = blockIdx.x, t = threadIdx.x;
  const int* ix = idx + off[c];
  const int m = off[c + 1] - off[c];
  const int64_t r0 = (int64_t)blockIdx.y * 64;
  for (int l = t; l < m * m; l += blockDim.x) {
    const int i = l % m, j = l / m;
    U[i * CJ_LD + j] = Ubuf[(int64_t)c * kClusterMax * kClusterMax + i + (int64_t)j * kClusterMax];
  }
  for (int l = t; l < 64 * m; l += blockDim.x) {
    const int rr = l % 64, j = l / 64;
    W[rr * CJ_LD + j] = (r0 + rr < k) ? V[(r0 + rr) + (int64_t)ix[j] * ldv] : num<S>::zero();
  }
  __syncthreads();
  for (int l = t; l < 64 * m; l += blockDim.x) {
    const int rr = l % 64, j = l / 64;
    if (r0 + rr >= k) continue;
    S acc = num<S>::zero();
    for (int q = 0; q < m; ++q) acc = acc + W[rr * CJ_LD + q] * U[q * CJ_LD + j];
    V[(r0 + rr) + (int64_t)ix[j] * ldv] = acc;
  }
}

template <typename S>
void offdiag_scan(const S* H, int64_t k, int64_t ld, double thr, int* cnt, int* list, int cap, cudaStream_t s) {
  FEAST_CUDA_TRY(cudaMemsetAsync(cnt, 0, sizeof(int), s));
  if (k < 2) return;
  offdiag_scan_kernel<S><<<grid1d(k * k), 256, 0, s>>>(H, k, ld, thr * thr, cnt, list, cap);
  FEAST_LAUNCH_CHECK();
}

template <typename S>
void cluster_jacobi(S* H, int64_t k, int64_t ld, S* V, int64_t ldv, const int* idx, const int* off, int nsets,
                    double thr, S* Ubuf, int* sweeps_out, cudaStream_t s) {
  if (nsets <= 0) return;
  const int smem = 2 * kClusterMax * CJ_LD * (int)sizeof(S);
  static bool attr = [] {
    cudaFuncSetAttribute(cluster_jacobi_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         2 * kClusterMax * CJ_LD * (int)sizeof(S));
    cudaFuncSetAttribute(cluster_apply_v_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (64 + kClusterMax) * CJ_LD * (int)sizeof(S));
    return true;
  }();
  (void)attr;
  cluster_jacobi_kernel<S><<<nsets, 256, smem, s>>>(H, ld, idx, off, thr, kMaxSweeps, Ubuf, sweeps_out);
  FEAST_LAUNCH_CHECK();
  cluster_apply_v_kernel<S><<<dim3((unsigned)nsets, (unsigned)cdiv(k, 64)), 256,
                              (64 + kClusterMax) * CJ_LD * (int)sizeof(S), s>>>(V, k, ldv, idx, off, Ubuf);
  FEAST_LAUNCH_CHECK();
}

#define INST_S(S)                                                                                          \
  template void hermitize<S>(S*, int64_t, int64_t, cudaStream_t);                                          \
  template void cholesky_upper<S>(S*, int64_t, int64_t, const CoopWork&, int, cudaStream_t);               \
  template void tri_inverse_upper<S>(const S*, int64_t, int64_t, S*, int64_t, cudaStream_t);               \
  template void jacobi_eigh<S>(S*, int64_t, int64_t, S*, int64_t, double, const CoopWork&, int, cudaStream_t, int,  \
                               bool);                                                                     \
  template void get_diag<S>(const S*, int64_t, int64_t, double*, cudaStream_t);                            \
  template void col_norms2<S>(const S*, int64_t, int64_t, int64_t, double*, cudaStream_t);                 \
  template void col_dots_re<S>(const S*, const S*, int64_t, int64_t, int64_t, double*, cudaStream_t);      \
  template void resid_norms2<S>(const S*, const S*, int64_t, int64_t, int64_t, const double*, double*,     \
                                cudaStream_t);                                                            \
  template void ritz_residual<S>(S*, const S*, const S*, int64_t, int64_t, int64_t, const double*,         \
                                 cudaStream_t);                                                           \
  template void gather_cols<S>(S*, int64_t, const S*, int64_t, int64_t, const int*, int64_t, const double*, \
                               cudaStream_t);                                                             \
  template void scale_cols<S>(S*, int64_t, int64_t, int64_t, const double*, cudaStream_t);                 \
  template void jacobi_eigh_df<S>(S*, int64_t, int64_t, S*, int64_t, double*, double, const CoopWork&, int,  \
                                  cudaStream_t, int, bool);                                                \
  template void gather_sub<S>(S*, const S*, int64_t, const int*, int64_t, cudaStream_t);                   \
  template void scatter_sub<S>(S*, int64_t, const S*, const int*, int64_t, cudaStream_t);                  \
  template void scatter_cols<S>(S*, int64_t, const S*, int64_t, int64_t, const int*, int64_t, cudaStream_t); \
  template void accumulate_filter<S>(S*, int64_t, const c128*, int64_t, int64_t, int, const c128*,         \
                                     cudaStream_t);                                                       \
  template void refine_residual<S>(c128*, const S*, int64_t, const c128*, const c128*, int64_t, int64_t,   \
                                   int, const c128*, const int*, cudaStream_t);                           \
  template void random_normal<S>(S*, int64_t, int64_t, int64_t, unsigned long long, cudaStream_t);         \
  template void copy_matrix<S>(S*, int64_t, const S*, int64_t, int64_t, int64_t, cudaStream_t);            \
  template void set_identity<S>(S*, int64_t, int64_t, cudaStream_t);                                       \
  template void set_diag<S>(S*, int64_t, int64_t, const double*, cudaStream_t);                            \
  template void check_finite<S>(const S*, int64_t, int64_t, int64_t, int*, cudaStream_t);                  \
  template void offdiag_scan<S>(const S*, int64_t, int64_t, double, int*, int*, int, cudaStream_t);        \
  template void cluster_jacobi<S>(S*, int64_t, int64_t, S*, int64_t, const int*, const int*, int, double,  \
                                  S*, int*, cudaStream_t);

INST_S(double)
INST_S(c128)

}  // namespace feast
