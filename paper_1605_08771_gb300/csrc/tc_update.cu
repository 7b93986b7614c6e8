// Tensor-core (tcgen05) complex-FP32 rank-kb update C -= A B for every
// quadrature node, on the 5th-generation tensor cores of sm_103a.  It serves
// the trailing update of the shifted LU (A22 -= L21 U12) and the block
// updates of the triangular solves (Y2 -= L21 Y1, Y1 -= U12 Y2, and the same
// with conjugate-transposed factor blocks for the adjoint solves).
//
// Complex products become one real GEMM through the 2x2 real embedding with
// interleaved rows: row 2i of the real left operand holds [Re L_i, -Im L_i],
// row 2i+1 holds [Im L_i, Re L_i], and the right operand is [Re U; Im U], so
// real row 2i of the product is Re(L U)_i and row 2i+1 is Im(L U)_i -- the
// interleaved complex layout of A22 itself.  Each FP32 operand is split into
// three TF32 parts, hi = rna(a), mid = rna(a - hi), lo = rna(a - hi - mid);
// the subtractions are exact and 3 x 11 significand bits cover FP32's 24, so
// hi + mid + lo == a.  Six TF32 products -- hi*hi, hi*mid, mid*hi, hi*lo,
// lo*hi, mid*mid -- accumulate in FP32 in tensor memory; the dropped ones are
// below 2^-32 |a||b|.  (A two-part split, hi + rna(a - hi), keeps only about
// 22 bits of each operand: measured on the n = 8192 workload its factors
// made the first refined residual 3.5x larger than FP32 factors do, with or
// without the lo*lo product, and cost an extra refinement step.)
//
// Kernel: 128 x 128 output tiles, persistent CTAs of four warps.  Thread 0 issues the
// TMA loads of the 128B-swizzled K-major operand tiles, thread 32 issues the
// tcgen05.mma instructions (M = 128, N = 128, K = 8) into a 128-column TMEM
// accumulator, and all four warps read the accumulator back with tcgen05.ld
// for the epilogue C -= D.  Every mbarrier wait is bounded by a wall-clock
// limit; on expiry the kernel records the failure, lets the issued MMAs
// complete, frees its TMEM and skips the stores.
#include <mutex>

#include "factor.cuh"
#include "tc_update.cuh"
#include "tcgen05.cuh"

namespace feast {

namespace {

constexpr int TC_BM = 128, TC_BN = 128, TC_BK = 32;  // BK fp32 = 128 bytes = one swizzle row
constexpr int TC_STAGES = 2;
constexpr int TC_TILE_BYTES = TC_BM * TC_BK * 4;     // 16 KB per operand tile (BN == BM)
constexpr int TC_STAGE_BYTES = 6 * TC_TILE_BYTES;    // A hi/mid/lo, B hi/mid/lo
constexpr int TC_SMEM_BYTES = TC_STAGES * TC_STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;
constexpr int TC_TMEM_COLS = 128;
// Instruction descriptor, kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in 17-22,
// M >> 4 in 24-28.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                                ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t da, uint64_t db, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem), "l"(da), "l"(db), "r"(kIdescTf32), "r"(accum)
      : "memory");
}

__global__ void __launch_bounds__(128, 1)
tc_update_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, c64* Cm,
                 int64_t ldc, int64_t cstride, int64_t c_r0, int64_t c_c0, int64_t R, int64_t C, int rows_pad,
                 int cols_pad,
                 int ksteps, int nodes, int a_part_rows, int b_part_rows, int* status) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + TC_STAGES * TC_STAGE_BYTES);  // full[2], empty[2], done
  uint32_t* tmem_slot = (uint32_t*)(bars + 8);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar_full = smem_u32(&bars[0]), bar_empty = smem_u32(&bars[2]), bar_done = smem_u32(&bars[4]);
  const int mtiles = rows_pad / TC_BM, ntiles = cols_pad / TC_BN;
  const int64_t total = (int64_t)mtiles * ntiles * nodes;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_full + 8 * s));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_empty + 8 * s));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_done));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // persistent loop over output tiles; k-steps are numbered globally (g) so
  // the stage parities carry over from tile to tile
  int it = 0;
  for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x, ++it) {
    const int node = (int)(tile / ((int64_t)mtiles * ntiles));
    const int rem = (int)(tile % ((int64_t)mtiles * ntiles));
    const int mt = rem % mtiles, nt = rem / mtiles;
    const int row0 = node * rows_pad + mt * TC_BM;  // TMA row of the left operand
    const int col0 = node * cols_pad + nt * TC_BN;  // TMA row of the right operand
    const int gbase = it * ksteps;
    if (threadIdx.x == 0 && !s_fail) {
      // producer: TMA loads of the six operand tiles of each k-step (the
      // three parts of each operand are consecutive row blocks of one map)
      for (int ks = 0; ks < ksteps; ++ks) {
        const int g = gbase + ks, s = g % TC_STAGES;
        if (g >= TC_STAGES && !mbar_wait(bar_empty + 8 * s, ((g / TC_STAGES) - 1) & 1)) {
          atomicExch(&s_fail, 1);
          break;
        }
        uint8_t* st = smem + s * TC_STAGE_BYTES;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_full + 8 * s),
                     "r"(TC_STAGE_BYTES)
                     : "memory");
        const int x = ks * TC_BK;
#pragma unroll
        for (int part = 0; part < 3; ++part) {
          tma_load_2d(smem_u32(st + part * TC_TILE_BYTES), &tmA, x, part * a_part_rows + row0, bar_full + 8 * s);
          tma_load_2d(smem_u32(st + (3 + part) * TC_TILE_BYTES), &tmB, x, part * b_part_rows + col0,
                      bar_full + 8 * s);
        }
      }
    } else if (threadIdx.x == 32) {
      // MMA issuer: 4 k-steps of 8 per stage, 6 split products each
      for (int ks = 0; ks < ksteps && !s_fail; ++ks) {
        const int g = gbase + ks, s = g % TC_STAGES;
        if (!mbar_wait(bar_full + 8 * s, (g / TC_STAGES) & 1)) {
          atomicExch(&s_fail, 1);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(smem + s * TC_STAGE_BYTES);
#pragma unroll
        for (int kk = 0; kk < TC_BK / 8; ++kk) {
          const uint32_t off = kk * 32;  // 8 tf32 = 32 bytes along K inside the swizzle row
          const uint64_t ah = sw128_desc(base + off), am = sw128_desc(base + TC_TILE_BYTES + off),
                         al = sw128_desc(base + 2 * TC_TILE_BYTES + off);
          const uint64_t bh = sw128_desc(base + 3 * TC_TILE_BYTES + off),
                         bm = sw128_desc(base + 4 * TC_TILE_BYTES + off),
                         bl = sw128_desc(base + 5 * TC_TILE_BYTES + off);
          mma_tf32(tmem, ah, bh, (ks > 0 || kk > 0) ? 1u : 0u);
          mma_tf32(tmem, ah, bm, 1u);
          mma_tf32(tmem, am, bh, 1u);
          mma_tf32(tmem, ah, bl, 1u);
          mma_tf32(tmem, al, bh, 1u);
          mma_tf32(tmem, am, bm, 1u);
        }
        mma_commit(bar_empty + 8 * s);  // frees the stage when these MMAs are done
      }
      mma_commit(bar_done);  // completion of every MMA issued for this tile
    }
    __syncwarp();

    // epilogue: A22 -= D, read back from TMEM lane by lane (lane = real row)
    const bool ok = mbar_wait(bar_done, it & 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!ok) atomicExch(&s_fail, 1);
    __syncthreads();
    const bool fail = s_fail != 0;
    const int64_t rr = (int64_t)mt * TC_BM + warp * 32 + lane;  // real row within this node
    const int64_t i = rr >> 1;
    const int part = (int)(rr & 1);
    float* Cb = (float*)(Cm + (int64_t)node * cstride);
#pragma unroll 1
    for (int cc = 0; cc < TC_BN / 32; ++cc) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (!fail && i < R) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int64_t j = (int64_t)nt * TC_BN + cc * 32 + c;
          if (j < C) {
            float* p = Cb + 2 * ((c_r0 + i) + (c_c0 + j) * ldc) + part;
            *p = *p - __uint_as_float(v[c]);
          }
        }
      }
    }
    // the accumulator is read: the next tile's MMAs may overwrite it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (fail) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  if (threadIdx.x == 0 && s_fail) atomicExch(status, DEV_BARRIER_TIMEOUT);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// three-part TF32 split of an FP32 value: hi + mid + lo == x exactly
__device__ __forceinline__ void tf32_split3(float x, float& h, float& m, float& l) {
  h = tf32_rna(x);
  const float r = x - h;  // exact
  m = tf32_rna(r);
  l = tf32_rna(r - m);    // r - m exact, and it has at most 11 significant bits
}

// Operand packing into three TF32 planes (hi, mid, lo; plane stride a_part /
// b_part floats), K contiguous (Kp >= 2 kb).  Left operand: rows_pad real
// rows, row 2i = [Re A_i, -Im A_i], row 2i+1 = [Im A_i, Re A_i]; right
// operand: cols_pad rows, row j = [Re B_:j ; Im B_:j].  Each source block is
// read through TcSrc (conjugate transposes included); 32 x 32 complex tiles
// are staged through shared memory, the global reads running along the
// source's leading dimension.
__device__ __forceinline__ c64 tc_src_load(const TcSrc& src, int node, int64_t v, int64_t k) {
  const c64* b = src.base + (int64_t)node * src.node_stride;
  if (!src.conj_t) return b[(src.r0 + (src.vec_rows ? v : k)) + (src.c0 + (src.vec_rows ? k : v)) * src.ld];
  const c64 x = b[(src.r0 + (src.vec_rows ? v : k)) + (src.c0 + (src.vec_rows ? k : v)) * src.ld];
  return c64{x.re, -x.im};
}

__global__ void tc_pack_kernel(TcSrc sa, TcSrc sb, int kb, int64_t R, int64_t C, int rows_pad, int cols_pad, int Kp,
                               float* A, int64_t a_part, float* B, int64_t b_part) {
  __shared__ c64 tile[32][33];
  const int node = blockIdx.z;
  const bool left = blockIdx.y == 0;
  const TcSrc& src = left ? sa : sb;
  const int64_t base = (int64_t)blockIdx.x * 32;  // complex rows (left) or columns (right)
  const int64_t lim = left ? R : C;
  if (base >= (left ? rows_pad / 2 : cols_pad)) return;
  for (int kc = 0; kc < Kp / 2; kc += 32) {       // k-chunks of the complex operand
    __syncthreads();
    for (int t = threadIdx.x; t < 32 * 32; t += blockDim.x) {
      int q, k;  // consecutive threads along the source's leading dimension
      if (src.vec_rows) { q = t % 32; k = t / 32; } else { k = t % 32; q = t / 32; }
      c64 v{0.f, 0.f};
      if (base + q < lim && kc + k < kb) v = tc_src_load(src, node, base + q, kc + k);
      tile[q][k] = v;
    }
    __syncthreads();
    if (left) {
      // 64 real rows x (32 real-part columns + 32 imaginary-part columns)
      for (int t = threadIdx.x; t < 64 * 64; t += blockDim.x) {
        const int c = t % 64, rl = t / 64;
        const int q = rl >> 1, part = rl & 1, k = c % 32;
        const c64 L = tile[q][k];
        float val;
        int kk;
        if (c < 32) { val = part ? L.im : L.re; kk = kc + k; }
        else { val = part ? L.re : -L.im; kk = kb + kc + k; }
        if (kc + k >= kb) continue;
        const int64_t o = ((int64_t)node * rows_pad + 2 * base + rl) * Kp + kk;
        tf32_split3(val, A[o], A[a_part + o], A[2 * a_part + o]);
      }
    } else {
      for (int t = threadIdx.x; t < 32 * 64; t += blockDim.x) {
        const int c = t % 64, q = t / 64, k = c % 32;
        if (kc + k >= kb) continue;
        const c64 U = tile[q][k];
        const float val = (c < 32) ? U.re : U.im;
        const int kk = (c < 32) ? kc + k : kb + kc + k;
        const int64_t o = ((int64_t)node * cols_pad + base + q) * Kp + kk;
        tf32_split3(val, B[o], B[b_part + o], B[2 * b_part + o]);
      }
    }
  }
  // zero the K padding [2 kb, Kp)
  if (2 * kb < Kp) {
    const int rowsb = left ? 64 : 32;
    const int64_t rbase = left ? (int64_t)node * rows_pad + 2 * base : (int64_t)node * cols_pad + base;
    float* P = left ? A : B;
    const int64_t ps = left ? a_part : b_part;
    for (int t = threadIdx.x; t < rowsb * (Kp - 2 * kb); t += blockDim.x) {
      const int kk = 2 * kb + t % (Kp - 2 * kb), rl = t / (Kp - 2 * kb);
      const int64_t o = (rbase + rl) * Kp + kk;
      P[o] = 0.f;
      P[ps + o] = 0.f;
      P[2 * ps + o] = 0.f;
    }
  }
}

void make_map(CUtensorMap* map, float* base, int64_t rows, int Kp) {
  auto fn = tensor_map_encode_fn();
  if (!fn) throw CudaFailure(cudaErrorNotSupported);
  cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)TC_BM};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaFailure(cudaErrorInvalidValue);
}

}  // namespace

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

size_t tc_update_planes_bytes(int64_t rows, int64_t cols, int nodes) {
  const int64_t rp = cdiv(2 * rows, TC_BM) * TC_BM, cp = cdiv(cols, TC_BN) * TC_BN;
  const int64_t Kp = cdiv(2 * kTcBlock, TC_BK) * TC_BK;
  return (size_t)4 * 3 * (size_t)nodes * (size_t)(rp + cp) * (size_t)Kp + 4096;
}

void tc_block_update(const TcSrc& a, const TcSrc& b, int kb, int64_t R, int64_t C, c64* Cm, int64_t ldc,
                     int64_t cstride, int64_t c_r0, int64_t c_c0, int nodes, void* planes, int* status, int num_sms,
                     cudaStream_t s) {
  if (R <= 0 || C <= 0 || kb <= 0) return;
  if (kb > kTcBlock) throw CudaFailure(cudaErrorInvalidValue);
  const int rows_pad = (int)(cdiv(2 * R, TC_BM) * TC_BM);
  const int cols_pad = (int)(cdiv(C, TC_BN) * TC_BN);
  const int Kp = (int)(cdiv(2 * kb, TC_BK) * TC_BK);
  const int64_t a_rows = (int64_t)nodes * rows_pad, b_rows = (int64_t)nodes * cols_pad;
  float* A = (float*)planes;           // 3 planes of a_rows x Kp
  float* B = A + 3 * a_rows * Kp;      // 3 planes of b_rows x Kp
  {
    const int64_t blocks = std::max<int64_t>(rows_pad / 64, cols_pad / 32);
    dim3 g((unsigned)blocks, 2, nodes);
    tc_pack_kernel<<<g, 256, 0, s>>>(a, b, kb, R, C, rows_pad, cols_pad, Kp, A, a_rows * Kp, B, b_rows * Kp);
    FEAST_LAUNCH_CHECK();
  }
  CUtensorMap mA, mB;
  make_map(&mA, A, 3 * a_rows, Kp);
  make_map(&mB, B, 3 * b_rows, Kp);
  static std::once_flag attr;
  cudaError_t aerr = cudaSuccess;
  std::call_once(attr, [&] {
    aerr = cudaFuncSetAttribute(tc_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_BYTES);
  });
  FEAST_CUDA_TRY(aerr);
  const int64_t tiles = (int64_t)(rows_pad / TC_BM) * (cols_pad / TC_BN) * nodes;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, num_sms);
  tc_update_kernel<<<grid, 128, TC_SMEM_BYTES, s>>>(mA, mB, Cm, ldc, cstride, c_r0, c_c0, R, C, rows_pad, cols_pad,
                                                    Kp / TC_BK, nodes, (int)a_rows, (int)b_rows, status);
  FEAST_LAUNCH_CHECK();
}

void tc_trailing_update(c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, int64_t k0, int kb, void* planes,
                        int* status, int num_sms, cudaStream_t s) {
  const int64_t r1 = k0 + kb;
  // A22 -= L21 U12: L21 = M[r1:, k0:r1] (vectors along rows), U12 = M[k0:r1, r1:]
  const TcSrc a{M, stride, ld, r1, k0, true, false};
  const TcSrc b{M, stride, ld, k0, r1, false, false};
  tc_block_update(a, b, kb, n - r1, n - r1, M, ld, stride, r1, r1, nodes, planes, status, num_sms, s);
}

}  // namespace feast
