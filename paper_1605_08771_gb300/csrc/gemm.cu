// Batched SIMT GEMM (see gemm.cuh).  Register-tiled: each CTA computes a
// BM x BN tile of C, each thread TM x TN outputs strided by BM/TM rows and
// BN/TN columns so that both the shared-memory reads and the column-major
// epilogue stores of a warp are contiguous.
#include "gemm.cuh"

#include <atomic>
#include <vector>

namespace feast {

namespace {

template <typename T> __device__ __forceinline__ T maybe_conj(T v, int op) { return op == OP_C ? conj(v) : v; }

template <typename TC> __device__ __forceinline__ TC axpby(c128 alpha, TC acc, c128 beta, const TC* cptr, bool use_beta);
template <> __device__ __forceinline__ double axpby<double>(c128 alpha, double acc, c128 beta, const double* c, bool ub) {
  double r = alpha.re * acc;
  if (ub) r = fma(beta.re, *c, r);
  return r;
}
template <> __device__ __forceinline__ c128 axpby<c128>(c128 alpha, c128 acc, c128 beta, const c128* c, bool ub) {
  c128 r = alpha * acc;
  if (ub) r = r + beta * (*c);
  return r;
}
template <> __device__ __forceinline__ c64 axpby<c64>(c128 alpha, c64 acc, c128 beta, const c64* c, bool ub) {
  c64 a{(float)alpha.re, (float)alpha.im};
  c64 r = a * acc;
  if (ub) { c64 b{(float)beta.re, (float)beta.im}; r = r + b * (*c); }
  return r;
}

template <typename TA, typename TB, typename TC, int BM, int BN, int BK, int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN))
gemm_kernel(GemmArgs g) {
  constexpr int NT = (BM / TM) * (BN / TN);
  constexpr int SM = BM / TM, SN = BN / TN;
  __shared__ TA As[BK][BM + 1];
  __shared__ TB Bs[BK][BN + 1];

  const int bz = blockIdx.z;
  const int b = bz % g.batch;
  const int kc = bz / g.batch;
  const TA* A = (const TA*)g.A + (int64_t)b * g.strideA;
  const TB* B = (const TB*)g.B + (int64_t)b * g.strideB;
  const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
  const int64_t kper = cdiv(cdiv(g.K, BK), g.ksplit) * BK;
  const int64_t kbeg = (int64_t)kc * kper;
  const int64_t kend = min(g.K, kbeg + kper);

  TC acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = num<TC>::zero();

  const int t = threadIdx.x;
  const int tm = t % SM, tn = t / SM;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    for (int l = t; l < BM * BK; l += NT) {
      int mm, kk;
      if (g.opA == OP_N) { mm = l % BM; kk = l / BM; } else { kk = l % BK; mm = l / BK; }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      TA v = num<TA>::zero();
      if (gm < g.M && gk < kend) v = maybe_conj(g.opA == OP_N ? A[gm + gk * g.lda] : A[gk + gm * g.lda], g.opA);
      As[kk][mm] = v;
    }
    for (int l = t; l < BK * BN; l += NT) {
      int kk, nn;
      if (g.opB == OP_N) { kk = l % BK; nn = l / BK; } else { nn = l % BN; kk = l / BN; }
      const int64_t gk = k0 + kk, gn = n0 + nn;
      TB v = num<TB>::zero();
      if (gn < g.N && gk < kend) v = maybe_conj(g.opB == OP_N ? B[gk + gn * g.ldb] : B[gn + gk * g.ldb], g.opB);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      TA a[TM];
      TB bb[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][tm + i * SM];
#pragma unroll
      for (int j = 0; j < TN; ++j) bb[j] = Bs[kk][tn + j * SN];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) mac(acc[i][j], a[i], bb[j]);
    }
    __syncthreads();
  }

  if (g.ksplit > 1) {
    TC* P = (TC*)g.Cpart + ((int64_t)kc * g.batch + b) * g.ldc * g.N;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + tn + j * SN;
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int64_t gm = m0 + tm + i * SM;
        if (gm < g.M && gn < g.N) P[gm + gn * g.ldc] = acc[i][j];
      }
    }
    return;
  }
  TC* C = (TC*)g.C + (int64_t)b * g.strideC;
  const bool ub = (g.beta.re != 0.0 || g.beta.im != 0.0);
#pragma unroll
  for (int j = 0; j < TN; ++j) {
    const int64_t gn = n0 + tn + j * SN;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + tm + i * SM;
      if (gm < g.M && gn < g.N) {
        TC* c = C + gm + gn * g.ldc;
        *c = axpby<TC>(g.alpha, acc[i][j], g.beta, c, ub);
      }
    }
  }
}

// Complex-FP32 variant of gemm_kernel (64 x 64 tile, 4 x 4 complex outputs
// per thread, 256 threads, 3 CTAs per SM) whose next K slice is loaded from
// global memory into registers while the current slice is multiplied from
// shared memory: the plain kernel stalls on those loads (long-scoreboard
// stalls dominate its profile).  op(A), op(B) in {N, C}; no split-K.
// The C tile read by the epilogue is copied to shared memory with cp.async
// at the start.  Measured on the n = 8192 solve: 1.15 s of complex GEMM
// (1.27 s without the C copy, 1.58 s for the plain kernel; bounded at 2 CTAs
// per SM, with more registers and no spills, 1.46 s).
constexpr int CP_BM = 64, CP_BN = 64, CP_BK = 16, CP_T = 4;
constexpr int CP_SM = CP_BM / CP_T, CP_SN = CP_BN / CP_T, CP_NT = CP_SM * CP_SN;
constexpr int CP_AL = CP_BM * CP_BK / CP_NT, CP_BL = CP_BN * CP_BK / CP_NT;  // 4 and 4

// C tile of the epilogue (beta != 0): copied to shared memory with cp.async
// at the start, so its global-memory latency overlaps the multiplication
constexpr int CP_DSMEM = CP_BM * CP_BN * (int)sizeof(c64);

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(sdst)),
               "l"(gsrc)
               : "memory");
}

template <int OPA, int OPB, int MINB>
__global__ void __launch_bounds__(CP_NT, MINB) cgemm_prefetch_kernel(GemmArgs g) {
  __shared__ c64 As[CP_BK][CP_BM + 1];
  __shared__ c64 Bs[CP_BK][CP_BN + 1];
  extern __shared__ c64 Cs[];  // CP_BM x CP_BN, each thread's own outputs
  constexpr bool an = OPA == OP_N, bn = OPB == OP_N;
  const int b = blockIdx.z;
  const c64* A = (const c64*)g.A + (int64_t)b * g.strideA;
  const c64* B = (const c64*)g.B + (int64_t)b * g.strideB;
  const int64_t m0 = (int64_t)blockIdx.x * CP_BM, n0 = (int64_t)blockIdx.y * CP_BN;
  const int t = threadIdx.x;
  const int tm = t % CP_SM, tn = t / CP_SM;
  c64 ra[CP_AL], rb[CP_BL];
  c64* C = (c64*)g.C + (int64_t)b * g.strideC;
  const bool ub = (g.beta.re != 0.0 || g.beta.im != 0.0);
  if (ub) {
#pragma unroll
    for (int j = 0; j < CP_T; ++j) {
      const int64_t gn = n0 + tn + j * CP_SN;
#pragma unroll
      for (int i = 0; i < CP_T; ++i) {
        const int64_t gm = m0 + tm + i * CP_SM;
        if (gm < g.M && gn < g.N) cp_async8(&Cs[(tm + i * CP_SM) + (tn + j * CP_SN) * CP_BM], C + gm + gn * g.ldc);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int r = 0; r < CP_AL; ++r) {
      const int l = t + r * CP_NT;
      const int mm = an ? l % CP_BM : l / CP_BK, kk = an ? l / CP_BM : l % CP_BK;
      const int64_t gm = m0 + mm, gk = k0 + kk;
      c64 v{0.f, 0.f};
      if (gm < g.M && gk < g.K) {
        v = an ? A[gm + gk * g.lda] : A[gk + gm * g.lda];
        if (OPA == OP_C) v.im = -v.im;
      }
      ra[r] = v;
    }
#pragma unroll
    for (int r = 0; r < CP_BL; ++r) {
      const int l = t + r * CP_NT;
      const int kk = bn ? l % CP_BK : l / CP_BN, nn = bn ? l / CP_BK : l % CP_BN;
      const int64_t gk = k0 + kk, gn = n0 + nn;
      c64 v{0.f, 0.f};
      if (gn < g.N && gk < g.K) {
        v = bn ? B[gk + gn * g.ldb] : B[gn + gk * g.ldb];
        if (OPB == OP_C) v.im = -v.im;
      }
      rb[r] = v;
    }
  };
  float cr[CP_T][CP_T], ci[CP_T][CP_T];
#pragma unroll
  for (int i = 0; i < CP_T; ++i)
#pragma unroll
    for (int j = 0; j < CP_T; ++j) { cr[i][j] = 0.f; ci[i][j] = 0.f; }
  load(0);
  for (int64_t k0 = 0; k0 < g.K; k0 += CP_BK) {
    __syncthreads();
#pragma unroll
    for (int r = 0; r < CP_AL; ++r) {
      const int l = t + r * CP_NT;
      As[an ? l / CP_BM : l % CP_BK][an ? l % CP_BM : l / CP_BK] = ra[r];
    }
#pragma unroll
    for (int r = 0; r < CP_BL; ++r) {
      const int l = t + r * CP_NT;
      Bs[bn ? l % CP_BK : l / CP_BN][bn ? l / CP_BK : l % CP_BN] = rb[r];
    }
    __syncthreads();
    if (k0 + CP_BK < g.K) load(k0 + CP_BK);
#pragma unroll
    for (int kk = 0; kk < CP_BK; ++kk) {
      c64 a[CP_T], bb[CP_T];
#pragma unroll
      for (int i = 0; i < CP_T; ++i) a[i] = As[kk][tm + i * CP_SM];
#pragma unroll
      for (int j = 0; j < CP_T; ++j) bb[j] = Bs[kk][tn + j * CP_SN];
#pragma unroll
      for (int i = 0; i < CP_T; ++i)
#pragma unroll
        for (int j = 0; j < CP_T; ++j) {
          cr[i][j] = fmaf(a[i].re, bb[j].re, cr[i][j]);
          cr[i][j] = fmaf(-a[i].im, bb[j].im, cr[i][j]);
          ci[i][j] = fmaf(a[i].re, bb[j].im, ci[i][j]);
          ci[i][j] = fmaf(a[i].im, bb[j].re, ci[i][j]);
        }
    }
  }
  if (ub) asm volatile("cp.async.wait_all;" ::: "memory");
  const c64 al{(float)g.alpha.re, (float)g.alpha.im}, be{(float)g.beta.re, (float)g.beta.im};
#pragma unroll
  for (int j = 0; j < CP_T; ++j) {
    const int64_t gn = n0 + tn + j * CP_SN;
#pragma unroll
    for (int i = 0; i < CP_T; ++i) {
      const int64_t gm = m0 + tm + i * CP_SM;
      if (gm < g.M && gn < g.N) {
        c64 r = al * c64{cr[i][j], ci[i][j]};
        if (ub) r = r + be * Cs[(tm + i * CP_SM) + (tn + j * CP_SN) * CP_BM];
        C[gm + gn * g.ldc] = r;
      }
    }
  }
}

template <typename TC>
__global__ void gemm_reduce_splitk(GemmArgs g) {
  const int64_t total = g.M * g.N;
  const int b = blockIdx.y;
  const bool ub = (g.beta.re != 0.0 || g.beta.im != 0.0);
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = idx % g.M, n = idx / g.M;
    TC s = num<TC>::zero();
    for (int kc = 0; kc < g.ksplit; ++kc) {
      const TC* P = (const TC*)g.Cpart + ((int64_t)kc * g.batch + b) * g.ldc * g.N;
      s = s + P[m + n * g.ldc];
    }
    TC* c = (TC*)g.C + (int64_t)b * g.strideC + m + n * g.ldc;
    *c = axpby<TC>(g.alpha, s, g.beta, c, ub);
  }
}

}  // namespace

template <typename TA, typename TB, typename TC>
void gemm(const GemmArgs& g0, cudaStream_t stream) {
  if (g0.M <= 0 || g0.N <= 0 || g0.batch <= 0) return;
  GemmArgs g = g0;
  if (g.ksplit < 1) g.ksplit = 1;
  constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4;
  if (g.ksplit > 1 && g.Cpart == nullptr) g.ksplit = 1;
  dim3 grid((unsigned)cdiv(g.M, BM), (unsigned)cdiv(g.N, BN), (unsigned)(g.batch * g.ksplit));
  constexpr bool c64_gemm =
      std::is_same<TA, c64>::value && std::is_same<TB, c64>::value && std::is_same<TC, c64>::value;
  if (c64_gemm) kernel_timer_launch_begin(TIMER_CGEMM, stream);
  if constexpr (c64_gemm) {
    if (g.ksplit == 1 && g.opA != OP_T && g.opB != OP_T) {
      static bool attr = [] {
        cudaFuncSetAttribute(cgemm_prefetch_kernel<OP_N, OP_N, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, CP_DSMEM);
        cudaFuncSetAttribute(cgemm_prefetch_kernel<OP_C, OP_N, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, CP_DSMEM);
        cudaFuncSetAttribute(cgemm_prefetch_kernel<OP_N, OP_C, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, CP_DSMEM);
        cudaFuncSetAttribute(cgemm_prefetch_kernel<OP_C, OP_C, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, CP_DSMEM);
        return true;
      }();
      (void)attr;
      if (g.opA == OP_N && g.opB == OP_N) cgemm_prefetch_kernel<OP_N, OP_N, 3><<<grid, CP_NT, CP_DSMEM, stream>>>(g);
      else if (g.opB == OP_N) cgemm_prefetch_kernel<OP_C, OP_N, 3><<<grid, CP_NT, CP_DSMEM, stream>>>(g);
      else if (g.opA == OP_N) cgemm_prefetch_kernel<OP_N, OP_C, 3><<<grid, CP_NT, CP_DSMEM, stream>>>(g);
      else cgemm_prefetch_kernel<OP_C, OP_C, 3><<<grid, CP_NT, CP_DSMEM, stream>>>(g);
    } else {
      gemm_kernel<TA, TB, TC, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, stream>>>(g);
    }
  } else {
    gemm_kernel<TA, TB, TC, BM, BN, BK, TM, TN><<<grid, (BM / TM) * (BN / TN), 0, stream>>>(g);
  }
  FEAST_LAUNCH_CHECK();
  if (c64_gemm) kernel_timer_launch_end(TIMER_CGEMM, stream, 8.0 * (double)g.M * (double)g.N * (double)g.K * g.batch);
  if (g.ksplit > 1) {
    int64_t total = g.M * g.N;
    dim3 rg((unsigned)std::min<int64_t>(cdiv(total, 256), 4096), (unsigned)g.batch);
    gemm_reduce_splitk<TC><<<rg, 256, 0, stream>>>(g);
    FEAST_LAUNCH_CHECK();
  }
}

template void gemm<c128, c128, c128>(const GemmArgs&, cudaStream_t);
template void gemm<c64, c64, c64>(const GemmArgs&, cudaStream_t);
template void gemm<double, double, double>(const GemmArgs&, cudaStream_t);
template void gemm<double, c128, c128>(const GemmArgs&, cudaStream_t);

}  // namespace feast

// ---------------------------------------------------------------------------
// double-float GEMM
// ---------------------------------------------------------------------------
namespace feast {
namespace {

constexpr int DF_BM = 64, DF_BN = 64, DF_BK = 16, DF_TM = 4, DF_TN = 4;
constexpr int DF_THREADS = (DF_BM / DF_TM) * (DF_BN / DF_TN);

__device__ __forceinline__ void df_mac(float a, float al, float b, float bl, float& s, float& x) {
  // explicit _rn intrinsics: the compiler must not contract these into FMAs
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);                       // a*b = p + e exactly
  const float t = __fadd_rn(s, p);                      // s + p = t + err exactly (TwoSum)
  const float bp = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  x = fmaf(a, bl, x);
  x = fmaf(al, b, x);
  x = __fadd_rn(x, __fadd_rn(e, err));
}

__global__ void __launch_bounds__(DF_THREADS)
gemm_df32_kernel(int64_t M, int64_t N, int64_t K, double alpha, const float* __restrict__ Ahi,
                 const float* __restrict__ Alo, int64_t lda, const float* __restrict__ Bhi,
                 const float* __restrict__ Blo, int64_t ldb, double beta, double* C, int64_t ldc, int cs, int co,
                 int64_t kper, int64_t czs) {
  __shared__ __align__(16) float sAh[DF_BK][DF_BM];
  __shared__ __align__(16) float sAl[DF_BK][DF_BM];
  __shared__ __align__(16) float sBh[DF_BK][DF_BN + 1];
  __shared__ __align__(16) float sBl[DF_BK][DF_BN + 1];
  const int t = threadIdx.x;
  const int tm = t % (DF_BM / DF_TM), tn = t / (DF_BM / DF_TM);
  const int64_t m0 = (int64_t)blockIdx.x * DF_BM, n0 = (int64_t)blockIdx.y * DF_BN;
  float s[DF_TM][DF_TN], x[DF_TM][DF_TN];
  double d[DF_TM][DF_TN];
#pragma unroll
  for (int i = 0; i < DF_TM; ++i)
#pragma unroll
    for (int j = 0; j < DF_TN; ++j) { s[i][j] = 0.f; x[i][j] = 0.f; d[i][j] = 0.0; }

  int tile = 0;
  // split-K: slice z of the reduction writes its own output block
  const int64_t kbeg = (int64_t)blockIdx.z * kper, kend = min(K, kbeg + kper);
  C += (int64_t)blockIdx.z * czs;
  for (int64_t k0 = kbeg; k0 < kend; k0 += DF_BK, ++tile) {
    // A tile: BM x BK, consecutive threads along m (coalesced)
    for (int l = t; l < DF_BM * DF_BK; l += DF_THREADS) {
      const int mm = l % DF_BM, kk = l / DF_BM;
      const int64_t gm = m0 + mm, gk = k0 + kk;
      float h = 0.f, lo = 0.f;
      if (gm < M && gk < kend) { h = Ahi[gm + gk * lda]; lo = Alo[gm + gk * lda]; }
      sAh[kk][mm] = h;
      sAl[kk][mm] = lo;
    }
    // B tile: BK x BN, consecutive threads along k (coalesced)
    for (int l = t; l < DF_BK * DF_BN; l += DF_THREADS) {
      const int kk = l % DF_BK, nn = l / DF_BK;
      const int64_t gk = k0 + kk, gn = n0 + nn;
      float h = 0.f, lo = 0.f;
      if (gn < N && gk < kend) { h = Bhi[gk + gn * ldb]; lo = Blo[gk + gn * ldb]; }
      sBh[kk][nn] = h;
      sBl[kk][nn] = lo;
    }
    __syncthreads();
    // partial unroll keeps the loop body within the instruction cache
#pragma unroll 4
    for (int kk = 0; kk < DF_BK; ++kk) {
      const float4 ah = *reinterpret_cast<const float4*>(&sAh[kk][tm * DF_TM]);
      const float4 al = *reinterpret_cast<const float4*>(&sAl[kk][tm * DF_TM]);
      const float a_h[4] = {ah.x, ah.y, ah.z, ah.w};
      const float a_l[4] = {al.x, al.y, al.z, al.w};
      float b_h[DF_TN], b_l[DF_TN];
#pragma unroll
      for (int j = 0; j < DF_TN; ++j) {
        b_h[j] = sBh[kk][tn + j * (DF_BN / DF_TN)];
        b_l[j] = sBl[kk][tn + j * (DF_BN / DF_TN)];
      }
#pragma unroll
      for (int i = 0; i < DF_TM; ++i)
#pragma unroll
        for (int j = 0; j < DF_TN; ++j) df_mac(a_h[i], a_l[i], b_h[j], b_l[j], s[i][j], x[i][j]);
    }
    __syncthreads();
    if (tile & 1) {  // flush every 32 k-steps
#pragma unroll
      for (int i = 0; i < DF_TM; ++i)
#pragma unroll
        for (int j = 0; j < DF_TN; ++j) { d[i][j] += (double)x[i][j]; x[i][j] = 0.f; }
    }
  }
#pragma unroll
  for (int j = 0; j < DF_TN; ++j) {
    const int64_t gn = n0 + tn + j * (DF_BN / DF_TN);
#pragma unroll
    for (int i = 0; i < DF_TM; ++i) {
      const int64_t gm = m0 + tm * DF_TM + i;
      if (gm < M && gn < N) {
        const double r = (double)s[i][j] + (d[i][j] + (double)x[i][j]);
        double* c = C + (gm + gn * ldc) * cs + co;
        *c = (beta != 0.0) ? fma(alpha, r, beta * (*c)) : alpha * r;
      }
    }
  }
}

__global__ void combine_3m_kernel(double* C, const double* T2, int64_t total) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const double t1 = C[2 * idx], t3 = C[2 * idx + 1], t2 = T2[idx];
    C[2 * idx] = t1 - t2;
    C[2 * idx + 1] = (t3 - t1) - t2;
  }
}

__global__ void combine_axpby_kernel(double* C, int64_t ldc, int cplx, const double* T, const double* T2, int64_t M,
                                     int64_t N, double alpha, double beta) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * N;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % M, j = idx / M;
    if (cplx) {
      const double t1 = T[2 * idx], t3 = T[2 * idx + 1], t2 = T2[idx];
      double* c = C + 2 * (i + j * ldc);
      const double re = t1 - t2, im = (t3 - t1) - t2;
      c[0] = beta != 0.0 ? alpha * re + beta * c[0] : alpha * re;
      c[1] = beta != 0.0 ? alpha * im + beta * c[1] : alpha * im;
    } else {
      double* c = C + (i + j * ldc);
      *c = beta != 0.0 ? alpha * T[idx] + beta * (*c) : alpha * T[idx];
    }
  }
}

// hi/lo planes (rows x cols, ld rows) of a transposed source: element (i, j)
// is src[(j + i*lds)*ss + so], negated when neg; staged through shared memory
// so both sides are coalesced
__global__ void split_df32_t_kernel(const double* src, int64_t rows, int64_t cols, int64_t lds, int ss, int so, int neg,
                                    float* hi, float* lo) {
  __shared__ double tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32, j0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r, j = j0 + threadIdx.x;
    double v = 0.0;
    if (i < rows && j < cols) v = src[(j + i * lds) * ss + so];
    tile[r][threadIdx.x] = neg ? -v : v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, i = i0 + threadIdx.x;
    if (i < rows && j < cols) {
      const double v = tile[threadIdx.x][r];
      const float h = (float)v;
      hi[i + j * rows] = h;
      lo[i + j * rows] = (float)(v - (double)h);
    }
  }
}

// C (M x N, ld ldc, interleaved complex when cplx) = sum over ks partial
// blocks P (each M x N with leading dim M, same element layout)
__global__ void sum_partials_kernel(double* C, int64_t ldc, const double* P, int64_t M, int64_t N, int ks, int cplx) {
  const int w = cplx ? 2 : 1;
  const int64_t blk = M * N * w;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < M * N * w;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = idx / w, part = idx % w;
    const int64_t i = e % M, j = e / M;
    double acc = 0.0;
    for (int z = 0; z < ks; ++z) acc += P[z * blk + idx];
    C[(i + j * ldc) * w + part] = acc;
  }
}

__global__ void split_df32_kernel(const double* src, int64_t rows, int64_t cols, int64_t lds, int ss, int so,
                                  float* hi, float* lo) {
  const int64_t total = rows * cols;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % rows, j = idx / rows;
    const double* e = src + (i + j * lds) * ss;
    const double v = (so == 2) ? e[0] + e[1] : e[so];
    const float h = (float)v;
    hi[idx] = h;
    lo[idx] = (float)(v - (double)h);
  }
}

}  // namespace

namespace {
struct KernelTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool[TIMER_CLASSES];
  size_t used[TIMER_CLASSES] = {};
  double work[TIMER_CLASSES] = {};
  int launches[TIMER_CLASSES] = {};
};
// one timer per host thread: the batched solver runs problems on several
// threads, each timing its own launches
KernelTimer& kernel_timer() {
  static thread_local KernelTimer t;
  return t;
}
std::atomic<unsigned long long> g_launches{0};
}  // namespace

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(); }

void kernel_timer_begin() {
  KernelTimer& t = kernel_timer();
  t.on = true;
  for (int c = 0; c < TIMER_CLASSES; ++c) {
    t.used[c] = 0;
    t.work[c] = 0.0;
    t.launches[c] = 0;
  }
}
void kernel_timer_end(int cls, double* ms, double* work, int* launches) {
  KernelTimer& t = kernel_timer();
  double tot = 0.0;
  for (size_t i = 0; i + 1 < t.used[cls]; i += 2) {
    float e = 0.f;
    FEAST_CUDA_TRY(cudaEventSynchronize(t.pool[cls][i + 1]));
    FEAST_CUDA_TRY(cudaEventElapsedTime(&e, t.pool[cls][i], t.pool[cls][i + 1]));
    tot += e;
  }
  if (ms) *ms = tot;
  if (work) *work = t.work[cls];
  if (launches) *launches = t.launches[cls];
  t.used[cls] = 0;
  bool any = false;
  for (int c = 0; c < TIMER_CLASSES; ++c) any = any || t.used[c] > 0;
  if (!any) t.on = false;
}
void kernel_timer_launch_begin(int cls, cudaStream_t s) {
  KernelTimer& t = kernel_timer();
  if (!t.on) return;
  while (t.pool[cls].size() < t.used[cls] + 2) {
    cudaEvent_t e;
    FEAST_CUDA_TRY(cudaEventCreate(&e));
    t.pool[cls].push_back(e);
  }
  FEAST_CUDA_TRY(cudaEventRecord(t.pool[cls][t.used[cls]], s));
}
void kernel_timer_launch_end(int cls, cudaStream_t s, double work) {
  KernelTimer& t = kernel_timer();
  if (!t.on) return;
  FEAST_CUDA_TRY(cudaEventRecord(t.pool[cls][t.used[cls] + 1], s));
  t.used[cls] += 2;
  t.work[cls] += work;
  t.launches[cls] += 1;
}

void gemm_df32(int64_t M, int64_t N, int64_t K, double alpha, const float* Ahi, const float* Alo, int64_t lda,
               const float* Bhi, const float* Blo, int64_t ldb, double beta, double* C, int64_t ldc, int cs, int co,
               cudaStream_t s, int timer_class, int ksplit, int64_t czs) {
  if (M <= 0 || N <= 0) return;
  if (timer_class >= 0) kernel_timer_launch_begin(timer_class, s);
  ksplit = std::max(1, ksplit);
  const int64_t kper = cdiv(cdiv(K, ksplit), 2 * DF_BK) * (2 * DF_BK);
  dim3 grid((unsigned)cdiv(M, DF_BM), (unsigned)cdiv(N, DF_BN), (unsigned)ksplit);
  gemm_df32_kernel<<<grid, DF_THREADS, 0, s>>>(M, N, K, alpha, Ahi, Alo, lda, Bhi, Blo, ldb, beta, C, ldc, cs, co, kper,
                                               czs);
  FEAST_LAUNCH_CHECK();
  if (timer_class >= 0) kernel_timer_launch_end(timer_class, s, (double)M * (double)N * (double)K);
}

void combine_3m(double* C, const double* T2, int64_t n, int64_t k, cudaStream_t s) {
  const int64_t total = n * k;
  if (total <= 0) return;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 16384));
  combine_3m_kernel<<<g, 256, 0, s>>>(C, T2, total);
  FEAST_LAUNCH_CHECK();
}

void combine_axpby(double* C, int64_t ldc, bool cplx, const double* T, const double* T2, int64_t M, int64_t N,
                   double alpha, double beta, cudaStream_t s) {
  const int64_t total = M * N;
  if (total <= 0) return;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 16384));
  combine_axpby_kernel<<<g, 256, 0, s>>>(C, ldc, cplx ? 1 : 0, T, T2, M, N, alpha, beta);
  FEAST_LAUNCH_CHECK();
}

void split_df32_t(const double* src, int64_t rows, int64_t cols, int64_t lds, int ss, int so, bool neg, float* hi,
                  float* lo, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return;
  dim3 g((unsigned)cdiv(rows, 32), (unsigned)cdiv(cols, 32));
  split_df32_t_kernel<<<g, dim3(32, 8), 0, s>>>(src, rows, cols, lds, ss, so, neg ? 1 : 0, hi, lo);
  FEAST_LAUNCH_CHECK();
}

void sum_partials(double* C, int64_t ldc, const double* P, int64_t M, int64_t N, int ks, bool cplx, cudaStream_t s) {
  const int64_t total = M * N * (cplx ? 2 : 1);
  if (total <= 0) return;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 16384));
  sum_partials_kernel<<<g, 256, 0, s>>>(C, ldc, P, M, N, ks, cplx ? 1 : 0);
  FEAST_LAUNCH_CHECK();
}

void split_df32(const double* src, int64_t rows, int64_t cols, int64_t lds, int ss, int so, float* hi, float* lo,
                cudaStream_t s) {
  const int64_t total = rows * cols;
  if (total <= 0) return;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, 256), 16384));
  split_df32_kernel<<<g, 256, 0, s>>>(src, rows, cols, lds, ss, so, hi, lo);
  FEAST_LAUNCH_CHECK();
}

}  // namespace feast
