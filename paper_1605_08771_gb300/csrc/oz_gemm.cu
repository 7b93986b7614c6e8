// FP64-accurate real GEMM on the bf16 tensor cores (sm_103a tcgen05) by
// error-free digit splitting -- the Ozaki scheme (Ozaki, Ogita, Oishi & Rump,
// Numer. Algorithms 59, 2012) with the chunked exact accumulation of its
// low-precision tensor-core variants.
//
// Splitting.  Each row i of A (and each column j of B) gets an exponent e with
// max |x| < 2^e and is written as x = 2^(e-8) sum_{p<6} d_p 2^(-8p) + r with
// |r| <= 2^(e-49): X = x 2^(48-e) rounded to the nearest integer, then its
// balanced base-256 digits from the top (each rounded to nearest, so
// |d_0| <= 256, |d_p| <= 128).  Plane p stores d_p 2^(-8p), exact in bf16 (at
// most 8 significant bits).  Then
//     (A B)_ij = 2^(eA_i + eB_j - 16) sum_{p,q} sum_k a_p(i,k) b_q(k,j),
// and the 21 plane products with p + q <= 5 keep about 47 bits; the rest are
// below 2^-48 relative to sum_k 2^(eA_i + eB_j).
//
// Exact accumulation.  The products of one level l = p + q are integers times
// 2^(-8l) and over 128 consecutive k their sum stays below 2^24 times that
// unit (|d_0 d_0| <= 2^16; a level l >= 1 term is at most 2^14 (l + 3)), so
// an FP32 tensor-core accumulator holds it exactly.  Levels 0-3 therefore
// accumulate in four TMEM accumulators over one 128-wide K chunk at a time;
// after each chunk the epilogue warps read them and add them into a running
// double-float (hi, lo) pair per output with TwoSum (Knuth), so no bit is lost.
// Levels 4-5 are 2^-32 smaller: they share a fifth accumulator over the whole
// K, whose FP32 rounding stays near 2^-50 of the result.
//
// Kernel: persistent, one 128 x 96 output tile at a time per CTA.  Warp 0
// issues the TMA loads (K-major, 64B swizzle, 32 k of all 12 digit planes per
// stage, two stages); one thread of warp 1 issues tcgen05.mma kind::f16
// (M = 128, N = 96, K = 16); warps 2-9 drain the accumulators (lane = output
// row, each warp half of the columns).  The MMAs into the shared level-4/5
// accumulator come first in each stage, so the tensor cores keep working
// while the previous chunk is drained.  Every wait is bounded; on expiry the
// kernel records the failure, lets the issued MMAs and loads complete, frees
// its TMEM and skips the stores.
#include <mutex>

#include "gemm.cuh"
#include "oz_gemm.cuh"
#include "tcgen05.cuh"

namespace feast {

namespace {

constexpr int OZ_D = kOzDigits;
constexpr int OZ_BM = kOzTileM, OZ_BN = kOzTileN, OZ_BK = kOzTileK;  // BK bf16 = 64 bytes = one swizzle row
constexpr int OZ_CHUNK = 4;                                           // stages per exact chunk (128 k)
constexpr int OZ_STAGES = 2;
constexpr int OZ_A_TILE = OZ_BM * OZ_BK * 2;  // 8 KB
constexpr int OZ_B_TILE = OZ_BN * OZ_BK * 2;  // 6 KB
constexpr int OZ_STAGE_BYTES = OZ_D * (OZ_A_TILE + OZ_B_TILE);
constexpr int OZ_LO_BYTES = OZ_BM * OZ_BN * 4;  // low halves of the running double-float sums
constexpr int OZ_SMEM = OZ_STAGES * OZ_STAGE_BYTES + OZ_LO_BYTES + 1024 + 256;
constexpr int OZ_EXACT = 4;                   // levels drained per chunk
constexpr int OZ_MERGED_COL = OZ_EXACT * OZ_BN;
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_EPI_WARPS = 8;
constexpr int OZ_THREADS = 32 * (2 + OZ_EPI_WARPS);
constexpr int OZ_COLS_PER_WARP = OZ_BN / 2;   // 48
constexpr int OZ_GROUP_M = 8;                 // tile raster: groups of 8 row tiles

static_assert(OZ_MERGED_COL + OZ_BN <= OZ_TMEM_COLS, "TMEM columns");
static_assert(OZ_SMEM <= 227 * 1024, "shared memory");
static_assert(OZ_COLS_PER_WARP % 16 == 0, "column groups of 16");

// kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9, 10-12 = 1), both K-major, N >> 3 in 17-22, M >> 4 in 24-28.
constexpr uint32_t kIdescBf16 =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(OZ_BN >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem), "l"(da), "l"(db), "r"(kIdescBf16), "r"(accum)
      : "memory");
}

// TwoSum (Knuth): s + e == a + b exactly; explicit _rn keeps the compiler
// from reassociating or contracting
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// x 2^k: one exact multiplication when 2^k is a normal double
__device__ __forceinline__ double pow2_scale(double x, int k) {
  if (k >= -1022 && k <= 1023) return x * __longlong_as_double((long long)(k + 1023) << 52);
  return ldexp(x, k);
}

__device__ __forceinline__ void tile_coords(int t, int mtiles, int ntiles, int& mt, int& nt) {
  const int per = OZ_GROUP_M * ntiles;
  const int first = (t / per) * OZ_GROUP_M;
  const int gm = min(mtiles - first, OZ_GROUP_M);
  const int r = t % per;
  mt = first + r % gm;
  nt = r / gm;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
               int Mpad, int Npad, int kstages, const int* __restrict__ eA, const int* __restrict__ eB, double* C,
               int64_t ldc, int cs, int co, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* lo_sm = (float*)(smem + OZ_STAGES * OZ_STAGE_BYTES);        // [column][row]
  uint64_t* bars = (uint64_t*)(smem + OZ_STAGES * OZ_STAGE_BYTES + OZ_LO_BYTES);  // full[2] empty[2] chunk drained final
  uint32_t* tmem_slot = (uint32_t*)(bars + 8);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar_full = smem_u32(&bars[0]), bar_empty = smem_u32(&bars[2]);
  const uint32_t bar_chunk = smem_u32(&bars[4]), bar_drained = smem_u32(&bars[5]), bar_final = smem_u32(&bars[6]);
  const int mtiles = Mpad / OZ_BM, ntiles = Npad / OZ_BN;
  const int tiles = mtiles * ntiles;
  const int nchunks = (kstages + OZ_CHUNK - 1) / OZ_CHUNK;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < OZ_STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    mbar_init(bar_chunk, 1);
    mbar_init(bar_drained, OZ_EPI_WARPS);
    mbar_init(bar_final, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* fail = &s_fail;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: the 12 digit-plane tiles of every stage ----
      int g = 0;
      for (int tile = blockIdx.x; tile < tiles && !*fail; tile += gridDim.x) {
        int mt, nt;
        tile_coords(tile, mtiles, ntiles, mt, nt);
        for (int ks = 0; ks < kstages; ++ks, ++g) {
          const int st = g % OZ_STAGES;
          if (g >= OZ_STAGES && !mbar_wait(bar_empty + 8 * st, ((g / OZ_STAGES) - 1) & 1)) {
            atomicExch(&s_fail, 1);
            break;
          }
          if (*fail) break;
          const uint32_t base = smem_u32(smem + st * OZ_STAGE_BYTES);
          mbar_expect_tx(bar_full + 8 * st, OZ_STAGE_BYTES);
          const int x = ks * OZ_BK;
#pragma unroll
          for (int p = 0; p < OZ_D; ++p)
            tma_load_2d(base + p * OZ_A_TILE, &tmA, x, p * Mpad + mt * OZ_BM, bar_full + 8 * st);
#pragma unroll
          for (int q = 0; q < OZ_D; ++q)
            tma_load_2d(base + OZ_D * OZ_A_TILE + q * OZ_B_TILE, &tmB, x, q * Npad + nt * OZ_BN, bar_full + 8 * st);
        }
      }
      // loads still in flight land before the CTA leaves
      for (int h = g - OZ_STAGES; h < g; ++h)
        if (h >= 0) mbar_wait(bar_full + 8 * (h % OZ_STAGES), (h / OZ_STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      int g = 0, q = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < tiles && ok; tile += gridDim.x) {
        for (int c = 0; c < nchunks && ok; ++c, ++q) {
          const int s0 = c * OZ_CHUNK, s1 = min(kstages, s0 + OZ_CHUNK);
          for (int ks = s0; ks < s1; ++ks, ++g) {
            const int st = g % OZ_STAGES;
            if (*fail || !mbar_wait(bar_full + 8 * st, (g / OZ_STAGES) & 1)) { ok = false; break; }
            tc_fence_after();
            const bool tile_first = ks == 0, chunk_first = ks == s0;
            // the previous tile's accumulators, the shared one included, must be read first
            if (tile_first && q > 0) {
              if (!mbar_wait(bar_drained, (q - 1) & 1)) { ok = false; break; }
              tc_fence_after();
            }
            const uint32_t abase = smem_u32(smem + st * OZ_STAGE_BYTES);
            const uint32_t bbase = abase + OZ_D * OZ_A_TILE;
            // levels 4 and 5 into the shared accumulator
            bool first = tile_first;
#pragma unroll
            for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
              for (int p = 0; p < OZ_D; ++p) {
#pragma unroll
                for (int qq = 0; qq < OZ_D; ++qq) {
                  if (p + qq < OZ_EXACT || p + qq > OZ_D - 1) continue;
                  mma_bf16(tmem + OZ_MERGED_COL, sw64_desc(abase + p * OZ_A_TILE + kk * 32),
                           sw64_desc(bbase + qq * OZ_B_TILE + kk * 32), first ? 0u : 1u);
                  first = false;
                }
              }
            }
            // levels 0-3 restart at each chunk: wait for the previous chunk's drain
            if (chunk_first && !tile_first && q > 0) {
              if (!mbar_wait(bar_drained, (q - 1) & 1)) { ok = false; break; }
              tc_fence_after();
            }
#pragma unroll
            for (int kk = 0; kk < OZ_BK / 16; ++kk) {
#pragma unroll
              for (int l = 0; l < OZ_EXACT; ++l) {
#pragma unroll
                for (int p = 0; p <= l; ++p) {
                  const bool restart = chunk_first && kk == 0 && p == 0;
                  mma_bf16(tmem + l * OZ_BN, sw64_desc(abase + p * OZ_A_TILE + kk * 32),
                           sw64_desc(bbase + (l - p) * OZ_B_TILE + kk * 32), restart ? 0u : 1u);
                }
              }
            }
            mma_commit(bar_empty + 8 * st);  // frees the stage once these MMAs are done
          }
          if (ok) mma_commit(bar_chunk);     // the chunk's sums are complete in TMEM
        }
      }
      if (!ok) atomicExch(&s_fail, 1);
      // every issued MMA completes before TMEM is released
      mma_commit(bar_final);
      mbar_wait(bar_final, 0);
    }
  } else {
    // ---- epilogue: drain the exact levels after every chunk ----
    const int quad = warp & 3;                 // TMEM lanes this warp may access
    const int half = (warp - 2) >> 2;          // column half
    const int row = quad * 32 + lane;          // output row within the tile
    const uint32_t tbase = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(half * OZ_COLS_PER_WARP);
    int q = 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
      int mt, nt;
      tile_coords(tile, mtiles, ntiles, mt, nt);
      // running sum of output (row, column j) = H[j] + Lo[j]; the high parts
      // live in registers, the low parts in shared memory (one word per thread
      // and column, consecutive rows adjacent)
      float H[OZ_COLS_PER_WARP];
      float* Lo = lo_sm + (size_t)half * OZ_COLS_PER_WARP * OZ_BM + row;
#pragma unroll
      for (int j = 0; j < OZ_COLS_PER_WARP; ++j) { H[j] = 0.f; Lo[j * OZ_BM] = 0.f; }
      bool ok = true;
      for (int c = 0; c < nchunks; ++c, ++q) {
        if (*fail || !mbar_wait(bar_chunk, q & 1)) { ok = false; break; }
        tc_fence_after();
#pragma unroll
        for (int gcol = 0; gcol < OZ_COLS_PER_WARP / 16; ++gcol) {
          uint32_t va[16], vb[16];
          const uint32_t ta = tbase + gcol * 16;
          tmem_ld16(ta, va);
          tmem_ld16(ta + OZ_BN, vb);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float& h = H[gcol * 16 + j];
            float e0, e1;
            two_sum(h, __uint_as_float(va[j]), h, e0);
            two_sum(h, __uint_as_float(vb[j]), h, e1);
            float& lo = Lo[(gcol * 16 + j) * OZ_BM];
            lo = __fadd_rn(lo, __fadd_rn(e0, e1));
          }
          tmem_ld16(ta + 2 * OZ_BN, va);
          tmem_ld16(ta + 3 * OZ_BN, vb);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float& h = H[gcol * 16 + j];
            float e2;
            two_sum(h, __uint_as_float(va[j]), h, e2);
            float& lo = Lo[(gcol * 16 + j) * OZ_BM];
            lo = __fadd_rn(lo, __fadd_rn(e2, __uint_as_float(vb[j])));
          }
        }
        if (c == nchunks - 1) {
#pragma unroll
          for (int gcol = 0; gcol < OZ_COLS_PER_WARP / 16; ++gcol) {
            uint32_t v[16];
            tmem_ld16(tbase + OZ_MERGED_COL + gcol * 16, v);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              float& lo = Lo[(gcol * 16 + j) * OZ_BM];
              lo = __fadd_rn(lo, __uint_as_float(v[j]));
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_drained);
      }
      if (!ok) {
        atomicExch(&s_fail, 1);
        break;
      }
      const int i = mt * OZ_BM + row;
      if (i < M) {
        const int ei = eA[i] - 16;
#pragma unroll
        for (int j = 0; j < OZ_COLS_PER_WARP; ++j) {
          const int col = nt * OZ_BN + half * OZ_COLS_PER_WARP + j;
          if (col < N)
            C[((int64_t)i + (int64_t)col * ldc) * cs + co] = pow2_scale((double)H[j] + (double)Lo[j * OZ_BM], ei + eB[col]);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS));
  if (threadIdx.x == 0 && s_fail) atomicExch(status, DEV_BARRIER_TIMEOUT);
}

// Split kernel.  One CTA per vector, up to three combinations (modes) of the
// same source elements per launch, so a complex operand is read once for its
// Re, Im and Re +- Im planes.  The exponent comes from the vector's max |x|
// (an integer max over the FP64 bit patterns); the digits of x are taken with
// integer arithmetic from its bit pattern: X = x 2^(48-e) rounded to the
// nearest integer (ties to even), |X| <= 2^48, then balanced base-256 digits
// from the top.  The only FP64 instruction is the add of the Re +- Im modes:
// FP64 arithmetic is slow on this part, and an FP64 digit loop made the split
// compute-bound.  Padded vectors and the K padding are zero.
constexpr int OZ_SPLIT_THREADS = 256;
constexpr int OZ_SPLIT_VEC = 4;  // consecutive k per thread (one 8-byte store per plane)

struct OzSplitOut {
  uint16_t* planes[3];
  int* exps[3];
  int mode[3];
};

__device__ __forceinline__ double oz_mode_value(int mode, double re, double im) {
  switch (mode) {
    case 1: return im;
    case 2: return re + im;
    case 3: return -im;
    case 4: return re - im;
    default: return re;
  }
}

// round(|x| 2^(48-e)) with ties to even, signed; requires |x| < 2^e
__device__ __forceinline__ long long oz_fixed48(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  unsigned long long mant = b & 0x000fffffffffffffull;
  if (E != 0) mant |= 0x0010000000000000ull;
  if (mant == 0) return 0;
  // |x| = mant 2^(max(E, 1) - 1075); |x| 2^(48 - e) = mant 2^(-s)
  const int s = 1027 + e - (E != 0 ? E : 1);
  unsigned long long q;
  if (s <= 0) {
    q = mant << (-s);  // subnormal vectors only; q < 2^48 since |x| < 2^e
  } else if (s >= 55) {
    q = 0;             // mant < 2^53 <= 2^(s-2): below half a unit
  } else {
    q = mant >> s;
    const unsigned long long r = mant & ((1ull << s) - 1), half = 1ull << (s - 1);
    q += (r > half || (r == half && (q & 1ull))) ? 1ull : 0ull;
  }
  return (b >> 63) ? -(long long)q : (long long)q;
}

// bf16 pattern of the integer digit d (|d| <= 256) times 2^(-8p): exact, the
// upper half of the FP32 pattern
__device__ __forceinline__ uint16_t oz_digit_bf16(long long d, float scale) {
  return (uint16_t)(__float_as_uint((float)d * scale) >> 16);
}

template <int NM>
__global__ void __launch_bounds__(OZ_SPLIT_THREADS, 3)
oz_split_kernel(const double* __restrict__ src, int ss, int64_t K, int64_t se, int64_t sv, int64_t nvec,
                int64_t vpad, int64_t kpad, OzSplitOut out) {
  const int64_t v = blockIdx.x;
  const int64_t plane = vpad * kpad;
  const int64_t step = (int64_t)OZ_SPLIT_VEC * blockDim.x;
  if (v >= nvec) {
    for (int t = 0; t < NM; ++t) {
      uint16_t* o = out.planes[t] + v * kpad;
      for (int64_t k = (int64_t)OZ_SPLIT_VEC * threadIdx.x; k < kpad; k += step)
        for (int p = 0; p < OZ_D; ++p) *reinterpret_cast<uint2*>(o + p * plane + k) = make_uint2(0u, 0u);
      if (threadIdx.x == 0) out.exps[t][v] = 0;
    }
    return;
  }
  auto load = [&](int64_t k, double& re, double& im) {
    re = 0.0;
    im = 0.0;
    if (k < K) {
      const double* e = src + (k * se + v * sv) * ss;
      if (ss == 2) {
        const double2 z = *reinterpret_cast<const double2*>(e);
        re = z.x;
        im = z.y;
      } else {
        re = e[0];
      }
    }
  };
  // pass 1: max |x| per mode over the bit patterns (finite doubles order as
  // their magnitudes' patterns)
  unsigned long long amax[NM];
#pragma unroll
  for (int t = 0; t < NM; ++t) amax[t] = 0;
  for (int64_t k0 = (int64_t)OZ_SPLIT_VEC * threadIdx.x; k0 < K; k0 += step) {
#pragma unroll
    for (int j = 0; j < OZ_SPLIT_VEC; ++j) {
      double re, im;
      load(k0 + j, re, im);
#pragma unroll
      for (int t = 0; t < NM; ++t) {
        const unsigned long long m =
            (unsigned long long)__double_as_longlong(oz_mode_value(out.mode[t], re, im)) & 0x7fffffffffffffffull;
        amax[t] = m > amax[t] ? m : amax[t];
      }
    }
  }
  __shared__ unsigned long long red[NM][OZ_SPLIT_THREADS / 32];
  __shared__ int s_e[NM];
#pragma unroll
  for (int t = 0; t < NM; ++t) {
    unsigned long long m = amax[t];
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long x = __shfl_xor_sync(0xffffffffu, m, o);
      m = x > m ? x : m;
    }
    if ((threadIdx.x & 31) == 0) red[t][threadIdx.x >> 5] = m;
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < NM; ++t) {
    if (threadIdx.x == t) {
      unsigned long long m = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = red[t][w] > m ? red[t][w] : m;
      int e = 0;
      if (m != 0) frexp(__longlong_as_double((long long)m), &e);  // max |x| < 2^e
      s_e[t] = e;
      out.exps[t][v] = e;
    }
  }
  __syncthreads();
  int ev[NM];
#pragma unroll
  for (int t = 0; t < NM; ++t) ev[t] = s_e[t];
  // pass 2: digits (the vector is re-read, mostly from L2)
  for (int64_t k0 = (int64_t)OZ_SPLIT_VEC * threadIdx.x; k0 < kpad; k0 += step) {
    double re[OZ_SPLIT_VEC], im[OZ_SPLIT_VEC];
#pragma unroll
    for (int j = 0; j < OZ_SPLIT_VEC; ++j) load(k0 + j, re[j], im[j]);
#pragma unroll
    for (int t = 0; t < NM; ++t) {
      long long X[OZ_SPLIT_VEC];
#pragma unroll
      for (int j = 0; j < OZ_SPLIT_VEC; ++j) X[j] = oz_fixed48(oz_mode_value(out.mode[t], re[j], im[j]), ev[t]);
      uint16_t* o = out.planes[t] + v * kpad + k0;
      float scale = 1.0f;
#pragma unroll
      for (int p = 0; p < OZ_D; ++p) {
        uint16_t d16[OZ_SPLIT_VEC];
#pragma unroll
        for (int j = 0; j < OZ_SPLIT_VEC; ++j) {
          long long d;
          if (p < OZ_D - 1) {
            const int sh = 8 * (OZ_D - 1 - p);  // 40, 32, ..., 8
            d = (X[j] + (1ll << (sh - 1))) >> sh;
            X[j] -= d << sh;
          } else {
            d = X[j];
          }
          d16[j] = oz_digit_bf16(d, scale);
        }
        *reinterpret_cast<uint2*>(o + p * plane) =
            make_uint2((uint32_t)d16[0] | ((uint32_t)d16[1] << 16), (uint32_t)d16[2] | ((uint32_t)d16[3] << 16));
        scale *= 0.00390625f;  // 2^-8
      }
    }
  }
}

void make_map_bf16(CUtensorMap* map, const uint16_t* base, int64_t rows, int64_t kpad, int box_rows) {
  auto fn = tensor_map_encode_fn();
  if (!fn) throw CudaFailure(cudaErrorNotSupported);
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaFailure(cudaErrorInvalidValue);
}

}  // namespace

OzOperand oz_operand(void* buf, int64_t nvec, int64_t K, bool left) {
  OzOperand op;
  op.nvec = nvec;
  op.vpad = oz_vpad(nvec, left);
  op.K = K;
  op.kpad = oz_kpad(K);
  op.planes = (uint16_t*)buf;
  op.exps = (int*)((char*)buf + (size_t)OZ_D * op.vpad * op.kpad * 2);
  return op;
}

void oz_split_modes(const double* src, int ss, const int* modes, int nm, int64_t K, int64_t se, int64_t sv,
                    const OzOperand* ops, cudaStream_t s) {
  if (nm < 1 || nm > 3) throw CudaFailure(cudaErrorInvalidValue);
  const OzOperand& op = ops[0];
  if (op.vpad <= 0) return;
  OzSplitOut out{};
  for (int t = 0; t < nm; ++t) {
    if (ops[t].vpad != op.vpad || ops[t].kpad != op.kpad || ops[t].nvec != op.nvec || ops[t].K != op.K ||
        op.kpad % OZ_SPLIT_VEC)
      throw CudaFailure(cudaErrorInvalidValue);
    out.planes[t] = ops[t].planes;
    out.exps[t] = ops[t].exps;
    out.mode[t] = modes[t];
  }
  const dim3 grid((unsigned)op.vpad);
  switch (nm) {
    case 1: oz_split_kernel<1><<<grid, OZ_SPLIT_THREADS, 0, s>>>(src, ss, K, se, sv, op.nvec, op.vpad, op.kpad, out); break;
    case 2: oz_split_kernel<2><<<grid, OZ_SPLIT_THREADS, 0, s>>>(src, ss, K, se, sv, op.nvec, op.vpad, op.kpad, out); break;
    default: oz_split_kernel<3><<<grid, OZ_SPLIT_THREADS, 0, s>>>(src, ss, K, se, sv, op.nvec, op.vpad, op.kpad, out); break;
  }
  FEAST_LAUNCH_CHECK();
}

void oz_split(const double* src, int ss, int mode, int64_t K, int64_t se, int64_t sv, const OzOperand& op,
              cudaStream_t s) {
  oz_split_modes(src, ss, &mode, 1, K, se, sv, &op, s);
}

void oz_gemm(int64_t M, int64_t N, const OzOperand& A, const OzOperand& B, double* C, int64_t ldc, int cs, int co,
             int* status, int num_sms, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  if (A.K != B.K || A.kpad != B.kpad || A.vpad % OZ_BM || B.vpad % OZ_BN || A.kpad % OZ_BK || M > A.nvec || N > B.nvec)
    throw CudaFailure(cudaErrorInvalidValue);
  CUtensorMap mA, mB;
  make_map_bf16(&mA, A.planes, (int64_t)OZ_D * A.vpad, A.kpad, OZ_BM);
  make_map_bf16(&mB, B.planes, (int64_t)OZ_D * B.vpad, B.kpad, OZ_BN);
  static std::once_flag attr;
  cudaError_t aerr = cudaSuccess;
  std::call_once(attr, [&] {
    aerr = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM);
  });
  FEAST_CUDA_TRY(aerr);
  const int64_t tiles = (A.vpad / OZ_BM) * (B.vpad / OZ_BN);
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, num_sms);
  kernel_timer_launch_begin(TIMER_REFINE_GEMM, s);
  oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, s>>>(mA, mB, (int)M, (int)N, (int)A.vpad, (int)B.vpad,
                                                   (int)(A.kpad / OZ_BK), A.exps, B.exps, C, ldc, cs, co, status);
  FEAST_LAUNCH_CHECK();
  kernel_timer_launch_end(TIMER_REFINE_GEMM, s, (double)M * (double)N * (double)A.K);
}

void oz_gemm_op(bool cplx, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t lda, bool transA,
                const double* B, int64_t ldb, bool transB, double beta, double* C, int64_t ldc, const OzScratch& w,
                int* status, int num_sms, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  OzOperand L[3], R[3];
  const int parts = cplx ? 3 : 1;
  for (int t = 0; t < parts; ++t) {
    L[t] = oz_operand(w.L[t], M, K, true);
    R[t] = oz_operand(w.R[t], N, K, false);
  }
  // vectors: rows of op(A), columns of op(B).  Row i of A is strided by lda;
  // row i of A^H is column i of A, conjugated (imaginary part negated).
  const int64_t lse = transA ? 1 : lda, lsv = transA ? lda : 1;
  const int64_t rse = transB ? ldb : 1, rsv = transB ? 1 : ldb;
  if (cplx) {
    static const int plain[3] = {0, 1, 2}, conjugated[3] = {0, 3, 4};  // Re, Im, Re + Im
    const int* lm = transA ? conjugated : plain;
    const int* rm = transB ? conjugated : plain;
    oz_split_modes(A, 2, lm, 3, K, lse, lsv, L, s);
    oz_split_modes(B, 2, rm, 3, K, rse, rsv, R, s);
    oz_gemm(M, N, L[0], R[0], w.T, M, 2, 0, status, num_sms, s);   // T1 in the real slots
    oz_gemm(M, N, L[1], R[1], w.T2, M, 1, 0, status, num_sms, s);  // T2
    oz_gemm(M, N, L[2], R[2], w.T, M, 2, 1, status, num_sms, s);   // T3 in the imaginary slots
  } else {
    oz_split(A, 1, 0, K, lse, lsv, L[0], s);
    oz_split(B, 1, 0, K, rse, rsv, R[0], s);
    oz_gemm(M, N, L[0], R[0], w.T, M, 1, 0, status, num_sms, s);
  }
  combine_axpby(C, ldc, cplx, w.T, w.T2, M, N, alpha, beta, s);
}

}  // namespace feast
