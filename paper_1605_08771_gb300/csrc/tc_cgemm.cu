// Tensor-core (tcgen05, sm_103a) complex-FP32 block update C -= A B: the
// trailing updates of the shifted LU (A22 -= L21 U12) and the block updates
// of the triangular solves (Y2 -= L21 Y1, Y1 -= U12 Y2, and the adjoint
// solves' updates with conjugate-transposed factor blocks), i.e. the GEMM
// part of the shifted factorisations and solves of Eq. 3.
//
// FP32-exact operands on the bf16 tensor cores.  Every FP32 value x is split
// into three bf16 parts, x0 = bf16(x), x1 = bf16(x - x0), x2 = x - x0 - x1:
// the subtractions are exact, and 3 x 8 significant bits cover FP32's 24, so
// x0 + x1 + x2 == x.  A real product a b keeps the six part products whose
// size is at least 2^-18 |a||b| (a0 b0, a0 b1, a1 b0, a0 b2, a1 b1, a2 b0);
// the dropped ones are below 2^-26 |a||b|, under FP32 rounding.  bf16 x bf16
// products are exact in the FP32 tensor-memory accumulator.  A complex
// product takes four real products (Re = Ar Br - Ai Bi, Im = Ar Bi + Ai Br,
// the minus sign by the instruction's negate-A bit), so one complex
// multiply-add costs 24 bf16 multiply-adds: the rate is 1/6 of the dense bf16
// rate in complex-FP32 flops (8 per complex multiply-add).
//
// Operands are split once into K-major bf16 planes (cg_split; the factor
// panels of the solves once per factorisation) and loaded by TMA.
//
// Kernel: persistent, one 128 x BN complex output tile at a time per CTA
// (BN = 128, or 112 when that pads fewer columns), six warps.  Warp 0 issues the TMA loads (64B swizzle, 32 k of all twelve
// planes per stage, two stages); one thread of warp 1 issues tcgen05.mma
// kind::f16 (M = 128, N = BN, K = 16) into a Re and an Im accumulator of
// BN TMEM columns each, double-buffered across tiles so the next tile's
// products overlap this tile's epilogue; warps 2-5 read the accumulators
// back (lane = output row) and apply C -= D to the complex-FP32 C in place.
// Every mbarrier wait is bounded; on expiry the kernel records the failure,
// lets the issued MMAs and loads complete, frees its TMEM and skips the rest.
#include <cuda_bf16.h>

#include <mutex>

#include "tc_cgemm.cuh"
#include "tcgen05.cuh"

namespace feast {

namespace {

constexpr int CG_BM = kCgTileM, CG_BK = kCgChunk;
constexpr int CG_P = kCgPlanes;
constexpr int CG_STAGES = 2;
constexpr int CG_A_TILE = CG_BM * CG_BK * 2;                     // 8 KB
constexpr int CG_TMEM_COLS = 512;                                // 2 buffers x (Re, Im) x BN
constexpr int CG_EPI_WARPS = 4;
constexpr int CG_THREADS = 32 * (2 + CG_EPI_WARPS);

// Tile width BN (128, or 112 for the solves' 300 right-hand sides: 3 tiles
// of 112 compute 336 columns, 3 of 128 compute 384)
template <int BN> struct CgTile {
  static constexpr int B_TILE = BN * CG_BK * 2;                  // 8 KB or 7 KB
  static constexpr int STAGE_BYTES = CG_P * (CG_A_TILE + B_TILE);
  static constexpr int SMEM = CG_STAGES * STAGE_BYTES + 1024 + 256;
  // kind::f16 instruction descriptor: D = F32 (bits 4-5 = 1), A = B = BF16
  // (bits 7-9, 10-12 = 1), both K-major, N >> 3 in 17-22, M >> 4 in 24-28;
  // bit 13 negates A.
  static constexpr uint32_t IDESC =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(CG_BM >> 4) << 24);
  static_assert(4 * BN <= CG_TMEM_COLS, "TMEM columns");
  static_assert(SMEM <= 227 * 1024, "shared memory");
  static_assert(BN % 16 == 0 && B_TILE % 512 == 0, "MMA N and 64B-swizzle alignment");
};
constexpr uint32_t kNegA = 1u << 13;

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(accum)
      : "memory");
}

// TMA row of an operand tile: base + node + slab of chunk c + plane
struct OpCoords {
  int base_row, node_rows, slab_rows, plane_rows, cps, base_x;  // cps: 32-wide k chunks per slab
};

template <int CG_BN>
__global__ void __launch_bounds__(CG_THREADS, 1)
cg_update_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OpCoords ca,
                 OpCoords cb, int kchunks, int R, int N, int mtiles, int ntiles, int nodes, c64* C, int64_t ldc,
                 int64_t cstride, int* status) {
  constexpr int CG_B_TILE = CgTile<CG_BN>::B_TILE;
  constexpr int CG_STAGE_BYTES = CgTile<CG_BN>::STAGE_BYTES;
  constexpr uint32_t kIdesc = CgTile<CG_BN>::IDESC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + CG_STAGES * CG_STAGE_BYTES);  // full[2] empty[2] tfull[2] tempty[2] final
  uint32_t* tmem_slot = (uint32_t*)(bars + 10);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bar_full = smem_u32(&bars[0]), bar_empty = smem_u32(&bars[2]);
  const uint32_t bar_tfull = smem_u32(&bars[4]), bar_tempty = smem_u32(&bars[6]), bar_final = smem_u32(&bars[8]);
  const int per_node = mtiles * ntiles;
  const int tiles = per_node * nodes;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < CG_STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar_tfull + 8 * b, 1);
      mbar_init(bar_tempty + 8 * b, CG_EPI_WARPS);
    }
    mbar_init(bar_final, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(CG_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int* fail = &s_fail;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: the twelve plane tiles of every stage ----
      int g = 0;
      for (int t = blockIdx.x; t < tiles && !*fail; t += gridDim.x) {
        const int e = t / per_node, r = t % per_node;
        const int mt = r % mtiles, nt = r / mtiles;
        for (int c = 0; c < kchunks; ++c, ++g) {
          const int st = g % CG_STAGES;
          if (g >= CG_STAGES && !mbar_wait(bar_empty + 8 * st, ((g / CG_STAGES) - 1) & 1)) {
            atomicExch(&s_fail, 1);
            break;
          }
          if (*fail) break;
          const uint32_t base = smem_u32(smem + st * CG_STAGE_BYTES);
          mbar_expect_tx(bar_full + 8 * st, CG_STAGE_BYTES);
          const int xa = ca.base_x + (c % ca.cps) * CG_BK, xb = cb.base_x + (c % cb.cps) * CG_BK;
          const int ya = ca.base_row + e * ca.node_rows + (c / ca.cps) * ca.slab_rows + mt * CG_BM;
          const int yb = cb.base_row + e * cb.node_rows + (c / cb.cps) * cb.slab_rows + nt * CG_BN;
#pragma unroll
          for (int p = 0; p < CG_P; ++p)
            tma_load_2d(base + p * CG_A_TILE, &tmA, xa, ya + p * ca.plane_rows, bar_full + 8 * st);
#pragma unroll
          for (int q = 0; q < CG_P; ++q)
            tma_load_2d(base + CG_P * CG_A_TILE + q * CG_B_TILE, &tmB, xb, yb + q * cb.plane_rows,
                        bar_full + 8 * st);
        }
      }
      // loads still in flight land before the CTA leaves
      for (int h = g - CG_STAGES; h < g; ++h)
        if (h >= 0) mbar_wait(bar_full + 8 * (h % CG_STAGES), (h / CG_STAGES) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      // split-part pairs (x, y) of each real product: a_x b_y
      constexpr int px[6] = {0, 0, 1, 0, 1, 2};
      constexpr int py[6] = {0, 1, 0, 2, 1, 0};
      int g = 0, it = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++it) {
        const int buf = it & 1;
        const uint32_t dre = tmem + (uint32_t)(buf * 2 * CG_BN), dim = dre + CG_BN;
        // the epilogue must have read this buffer's previous tile
        if (it >= 2) {
          if (*fail || !mbar_wait(bar_tempty + 8 * buf, ((it >> 1) - 1) & 1)) { ok = false; break; }
          tc_fence_after();
        }
        for (int c = 0; c < kchunks; ++c, ++g) {
          const int st = g % CG_STAGES;
          if (*fail || !mbar_wait(bar_full + 8 * st, (g / CG_STAGES) & 1)) { ok = false; break; }
          tc_fence_after();
          const uint32_t abase = smem_u32(smem + st * CG_STAGE_BYTES);
          const uint32_t bbase = abase + CG_P * CG_A_TILE;
#pragma unroll
          for (int kk = 0; kk < CG_BK / 16; ++kk) {
            const uint32_t off = kk * 32;  // 16 bf16 along K inside the 64-byte swizzle row
            uint64_t a[CG_P], b[CG_P];
#pragma unroll
            for (int p = 0; p < CG_P; ++p) {
              a[p] = sw64_desc(abase + p * CG_A_TILE + off);
              b[p] = sw64_desc(bbase + p * CG_B_TILE + off);
            }
            const bool first = c == 0 && kk == 0;
#pragma unroll
            for (int s = 0; s < 6; ++s) {
              const uint32_t acc = (first && s == 0) ? 0u : 1u;
              const int x = px[s], y = py[s];
              mma(dre, a[x], b[y], kIdesc, acc);                 // + Re a Re b
              mma(dre, a[3 + x], b[3 + y], kIdesc | kNegA, 1u);  // - Im a Im b
              mma(dim, a[x], b[3 + y], kIdesc, acc);             // + Re a Im b
              mma(dim, a[3 + x], b[y], kIdesc, 1u);              // + Im a Re b
            }
          }
          mma_commit(bar_empty + 8 * st);  // frees the stage once these MMAs are done
        }
        if (!ok) break;
        mma_commit(bar_tfull + 8 * buf);   // the tile's sums are complete in TMEM
      }
      if (!ok) atomicExch(&s_fail, 1);
      // every issued MMA completes before TMEM is released
      mma_commit(bar_final);
      mbar_wait(bar_final, 0);
    }
  } else {
    // ---- epilogue: C -= D, lane = output row ----
    const int quad = warp & 3;  // TMEM lanes this warp may access
    const int row = quad * 32 + lane;
    int it = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++it) {
      const int e = t / per_node, r = t % per_node;
      const int mt = r % mtiles, nt = r / mtiles;
      const int buf = it & 1;
      if (*fail || !mbar_wait(bar_tfull + 8 * buf, (it >> 1) & 1)) {
        atomicExch(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const int i = mt * CG_BM + row;
      float2* Ce = (float2*)(C + (int64_t)e * cstride);
      const uint32_t tb = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * 2 * CG_BN);
#pragma unroll 1
      for (int g16 = 0; g16 < CG_BN / 16; ++g16) {
        uint32_t vr[16], vi[16];
        tmem_ld16(tb + g16 * 16, vr);
        tmem_ld16(tb + CG_BN + g16 * 16, vi);
        tmem_wait_ld();
        if (i < R) {
          const int j0 = nt * CG_BN + g16 * 16;
          float2 cv[16];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j0 + j < N) cv[j] = Ce[(int64_t)i + (int64_t)(j0 + j) * ldc];
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (j0 + j < N) {
              cv[j].x -= __uint_as_float(vr[j]);
              cv[j].y -= __uint_as_float(vi[j]);
              Ce[(int64_t)i + (int64_t)(j0 + j) * ldc] = cv[j];
            }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_tempty + 8 * buf);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CG_TMEM_COLS));
  if (threadIdx.x == 0 && s_fail) atomicExch(status, DEV_BARRIER_TIMEOUT);
}

// 32 x 32 (v, k) tile per CTA of 32 x 8 threads: read coalesced along the
// source's contiguous dimension, transpose in shared memory, write the six
// planes coalesced along k.
__global__ void __launch_bounds__(256)
cg_split_kernel(const c64* __restrict__ src, int64_t node_stride, int64_t slab_src, int64_t ld, int64_t r0,
                int64_t c0, int vec_rows, int conj_src, int64_t V, int64_t K, int kslab, int64_t slabs, int64_t vpad,
                int64_t kdim, uint16_t* __restrict__ out) {
  __shared__ c64 tile[32][33];  // [k][v]
  const int64_t z = blockIdx.z;
  const int64_t e = z / slabs, b = z % slabs;
  const int64_t v0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 32;
  const int64_t Kb = min((int64_t)kslab, K - b * kslab);
  const c64* base = src + e * node_stride + b * slab_src;
  const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    c64 x{0.f, 0.f};
    if (vec_rows) {
      const int64_t v = v0 + tx, k = k0 + r;
      if (v < V && k < Kb) x = base[(r0 + v) + (c0 + k) * ld];
      tile[r][tx] = x;
    } else {
      const int64_t k = k0 + tx, v = v0 + r;
      if (v < V && k < Kb) x = base[(r0 + k) + (c0 + v) * ld];
      tile[tx][r] = x;
    }
  }
  __syncthreads();
  const int64_t plane = vpad * kdim;
  uint16_t* o = out + z * (int64_t)CG_P * plane;
#pragma unroll
  for (int r = ty; r < 32; r += 8) {
    const int64_t v = v0 + r, k = k0 + tx;
    if (v >= vpad || k >= kdim) continue;
    c64 x = tile[tx][r];
    if (conj_src) x.im = -x.im;
    uint16_t a0, a1, a2, b0, b1, b2;
    cg_split3(x.re, a0, a1, a2);
    cg_split3(x.im, b0, b1, b2);
    const int64_t at = v * kdim + k;
    o[at] = a0;
    o[plane + at] = a1;
    o[2 * plane + at] = a2;
    o[3 * plane + at] = b0;
    o[4 * plane + at] = b1;
    o[5 * plane + at] = b2;
  }
}

void make_map(CUtensorMap* map, const uint16_t* base, int64_t rows, int64_t kdim, int box_rows) {
  auto fn = tensor_map_encode_fn();
  if (!fn) throw CudaFailure(cudaErrorNotSupported);
  cuuint64_t dims[2] = {(cuuint64_t)kdim, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kdim * 2};
  cuuint32_t box[2] = {(cuuint32_t)CG_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw CudaFailure(cudaErrorInvalidValue);
}

OpCoords coords(const CgOperand& o) {
  return OpCoords{(int)o.base_row, (int)o.node_rows, (int)o.slab_rows, (int)o.plane_rows, o.kslab / CG_BK, o.base_x};
}

}  // namespace

// the driver's cuTensorMapEncodeTiled, looked up once through the runtime
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

void cg_split(const c64* src, int64_t node_stride, int64_t slab_src, int64_t ld, int64_t r0, int64_t c0,
              bool vec_rows, bool conj_src, int64_t V, int64_t K, int kslab, int64_t slabs, int64_t vpad,
              int64_t kdim, int nodes, uint16_t* out, cudaStream_t s) {
  if (nodes <= 0 || slabs <= 0 || vpad <= 0 || kdim <= 0) return;
  if (vpad % 32 || kdim % 32 || kslab > kdim || (int64_t)nodes * slabs > 65535)
    throw CudaFailure(cudaErrorInvalidValue);
  dim3 grid((unsigned)(vpad / 32), (unsigned)(kdim / 32), (unsigned)(nodes * slabs));
  cg_split_kernel<<<grid, dim3(32, 8), 0, s>>>(src, node_stride, slab_src, ld, r0, c0, vec_rows ? 1 : 0,
                                               conj_src ? 1 : 0, V, K, kslab, slabs, vpad, kdim, out);
  FEAST_LAUNCH_CHECK();
}

void cg_update(const CgOperand& A, const CgOperand& B, int64_t K, int64_t R, int64_t N, c64* C, int64_t ldc,
               int64_t cstride, int nodes, int* status, int num_sms, cudaStream_t s) {
  if (R <= 0 || N <= 0 || K <= 0 || nodes <= 0) return;
  const int kchunks = (int)cdiv(K, CG_BK);
  const int64_t lim = (int64_t)1 << 31;
  if (A.total_rows + CG_BM >= lim || B.total_rows + 128 >= lim || A.kdim % CG_BK || B.kdim % CG_BK ||
      A.kslab % CG_BK || B.kslab % CG_BK || A.kslab <= 0 || B.kslab <= 0 || R >= lim || N >= lim ||
      A.base_x % CG_BK || B.base_x % CG_BK ||
      A.base_x + std::min<int64_t>(A.kslab, cdiv(K, CG_BK) * CG_BK) > A.kdim ||
      B.base_x + std::min<int64_t>(B.kslab, cdiv(K, CG_BK) * CG_BK) > B.kdim)
    throw CudaFailure(cudaErrorInvalidValue);
  // the tile width that computes the fewest padded columns (ties: 128)
  const int bn = (cdiv(N, 112) * 112 < cdiv(N, 128) * 128) ? 112 : 128;
  CUtensorMap mA, mB;
  make_map(&mA, A.planes, A.total_rows, A.kdim, CG_BM);
  make_map(&mB, B.planes, B.total_rows, B.kdim, bn);
  static std::once_flag attr;
  cudaError_t aerr = cudaSuccess;
  std::call_once(attr, [&] {
    aerr = cudaFuncSetAttribute(cg_update_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, CgTile<128>::SMEM);
    if (aerr == cudaSuccess)
      aerr = cudaFuncSetAttribute(cg_update_kernel<112>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  CgTile<112>::SMEM);
  });
  FEAST_CUDA_TRY(aerr);
  const int mtiles = (int)cdiv(R, CG_BM), ntiles = (int)cdiv(N, bn);
  const int64_t tiles = (int64_t)mtiles * ntiles * nodes;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, num_sms);
  kernel_timer_launch_begin(TIMER_TCGEMM, s);
  if (bn == 112)
    cg_update_kernel<112><<<grid, CG_THREADS, CgTile<112>::SMEM, s>>>(mA, mB, coords(A), coords(B), kchunks, (int)R,
                                                                      (int)N, mtiles, ntiles, nodes, C, ldc, cstride,
                                                                      status);
  else
    cg_update_kernel<128><<<grid, CG_THREADS, CgTile<128>::SMEM, s>>>(mA, mB, coords(A), coords(B), kchunks, (int)R,
                                                                      (int)N, mtiles, ntiles, nodes, C, ldc, cstride,
                                                                      status);
  FEAST_LAUNCH_CHECK();
  kernel_timer_launch_end(TIMER_TCGEMM, s, 8.0 * (double)R * (double)N * (double)K * nodes);
}

}  // namespace feast
