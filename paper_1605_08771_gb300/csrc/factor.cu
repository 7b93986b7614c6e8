// Shifted LU with partial pivoting and the blocked triangular solves.
//
// Right-looking blocked LU (panel width kPanel), all quadrature nodes in the
// same launches:
//   1. panel_lu_kernel: a cooperative launch, `P` CTAs per node each owning a
//      contiguous slice of the panel's rows.  Per column: every CTA publishes
//      its local pivot candidate (value, row, and the full panel row), one
//      bounded group barrier, then every CTA picks the same winner, swaps the
//      pivot row with the diagonal row where it owns them, scales its part of
//      the column and applies the rank-1 update to the rest of the panel,
//      tracking the next column's local maximum on the way.  When every
//      node's rows fit in co-resident CTAs of at most kPanelCacheRows rows,
//      each CTA keeps its rows of the panel in shared memory for the whole
//      panel (loaded once, written back once).  When a node's panel fits in
//      the shared memory of one 16-CTA thread-block cluster (complex FP32 up to
//      8192 rows), panel_lu_cluster_kernel takes it instead: candidates and
//      rows go through distributed shared memory and hardware cluster
//      barriers.
//   2. laswp_trsm_kernel: the panel's row interchanges applied to every column
//      outside the panel (as a gather of at most 2*kPanel touched rows), and
//      U12 = L11^{-1} A12 by a warp-per-column forward substitution.
//   3. A22 -= L21 U12 with the batched GEMM.
// The pivot choice is the first row of largest |m_ik|^2, as in the oracle.
#include "factor.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>
#include <climits>

namespace feast {

namespace {

constexpr int kPanelThreads = 256;
constexpr int kPanelCacheRows = 128;  // rows per CTA of the shared-memory panel

template <typename F>
__device__ __forceinline__ void argmax_merge(double& v, int& i, double v2, int i2) {
  if (v2 > v || (v2 == v && i2 >= 0 && (i < 0 || i2 < i))) { v = v2; i = i2; }
}

template <typename F>
__device__ void block_argmax(double& v, int& i) {
  __shared__ double sv[kPanelThreads / 32];
  __shared__ int si[kPanelThreads / 32];
  for (int off = 16; off > 0; off >>= 1) {
    double v2 = __shfl_down_sync(0xffffffffu, v, off);
    int i2 = __shfl_down_sync(0xffffffffu, i, off);
    argmax_merge<F>(v, i, v2, i2);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) { sv[w] = v; si[w] = i; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kPanelThreads / 32; ++k) argmax_merge<F>(sv[0], si[0], sv[k], si[k]);
  }
  __syncthreads();
  v = sv[0];
  i = si[0];
}

// net effect of a panel's interchanges on the rows it touched: after the
// swaps, row dst holds the former row src (one thread)
__device__ void panel_swap_summary(int b, int64_t n, int k0, int jb, const int32_t* ipiv, const PanelWork& w) {
  int rows[2 * kPanel], content[2 * kPanel];
  int cnt = 0;
  auto slot_of = [&](int r) {
    for (int q = 0; q < cnt; ++q)
      if (rows[q] == r) return q;
    rows[cnt] = r;
    content[cnt] = r;
    return cnt++;
  };
  for (int j = 0; j < jb; ++j) {
    int a = slot_of(k0 + j);
    int bb = slot_of(ipiv[(int64_t)b * n + k0 + j]);
    int tmp = content[a];
    content[a] = content[bb];
    content[bb] = tmp;
  }
  int out = 0;
  for (int q = 0; q < cnt; ++q)
    if (content[q] != rows[q]) {
      w.swap_dst[b * 2 * kPanel + out] = rows[q];
      w.swap_src[b * 2 * kPanel + out] = content[q];
      ++out;
    }
  w.swap_cnt[b] = out;
}

// CACHE: the CTA's rows of the panel stay in shared memory (R x jb, dynamic)
// for the whole panel instead of being re-read from L2 every column.
template <typename F, bool CACHE>
__global__ void __launch_bounds__(kPanelThreads)
panel_lu_kernel(F* M, int64_t n, int64_t ld, int64_t stride, int k0, int jb, int P, int64_t R,
                int32_t* ipiv, PanelWork w, unsigned base) {
  const int b = blockIdx.x / P;
  const int c = blockIdx.x % P;
  const int t = threadIdx.x;
  F* Mb = M + (int64_t)b * stride;
  const int64_t row_lo = k0 + (int64_t)c * R;
  const int64_t row_hi = min(n, row_lo + R);
  unsigned* ctr = w.counters + b;
  F* cand_row = (F*)w.cand_row;
  F* diag_row = (F*)w.diag_row;
  __shared__ F s_u[kPanel];
  __shared__ F s_d[kPanel];
  __shared__ int s_p;
  __shared__ int s_win;
  extern __shared__ __align__(16) unsigned char panel_smem[];
  F* T = reinterpret_cast<F*>(panel_smem);
  // element (row i, panel column cc) of a row this CTA owns
  auto at = [&](int64_t i, int cc) -> F& {
    if constexpr (CACHE) return T[(i - row_lo) + (int64_t)cc * R];
    else return Mb[i + (int64_t)(k0 + cc) * ld];
  };
  if constexpr (CACHE) {
    const int64_t nr = row_hi - row_lo;
    for (int64_t l = t; l < nr * jb; l += kPanelThreads) {
      const int64_t i = l % nr, cc = l / nr;
      T[i + cc * R] = Mb[(row_lo + i) + (k0 + cc) * ld];
    }
    __syncthreads();
  }

  // local maximum of column k0
  double v = -1.0;
  int vi = -1;
  for (int64_t i = row_lo + t; i < row_hi; i += kPanelThreads) {
    double a = (double)abs2(at(i, 0));
    argmax_merge<F>(v, vi, a, (int)i);
  }
  block_argmax<F>(v, vi);

  for (int j = 0; j < jb; ++j) {
    const int64_t d = k0 + j;
    const int64_t col = k0 + j;
    const int par = j & 1;
    const int64_t slot = ((int64_t)b * 2 + par) * w.pmax + c;
    if (t == 0) {
      w.cand_val[slot] = v;
      w.cand_idx[slot] = vi;
    }
    if (vi >= 0)
      for (int cc = t; cc < jb; cc += kPanelThreads)
        cand_row[slot * kPanel + cc] = at(vi, cc);
    if (d >= row_lo && d < row_hi)
      for (int cc = t; cc < jb; cc += kPanelThreads)
        diag_row[((int64_t)b * 2 + par) * kPanel + cc] = at(d, cc);
    if (!group_barrier(ctr, base + (unsigned)(j + 1) * (unsigned)P, w.status)) return;

    if (t < 32) {
      // warp 0 reads the P candidates in parallel and reduces them
      double bv = -1.0;
      int bi = -1, bq = -1;
      const int64_t s0 = ((int64_t)b * 2 + par) * w.pmax;
      for (int q = t; q < P; q += 32) {
        const double cv = __ldcg(&w.cand_val[s0 + q]);
        const int ci = __ldcg(&w.cand_idx[s0 + q]);
        if (ci >= 0 && (cv > bv || (cv == bv && (bi < 0 || ci < bi)))) {
          bv = cv;
          bi = ci;
          bq = q;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, bv, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        const int q2 = __shfl_down_sync(0xffffffffu, bq, off);
        if (i2 >= 0 && (v2 > bv || (v2 == bv && (bi < 0 || i2 < bi)))) {
          bv = v2;
          bi = i2;
          bq = q2;
        }
      }
      if (t == 0) {
        s_p = bi;
        s_win = bq;
      }
    }
    __syncthreads();
    const int p = s_p;
    const int win = s_win;
    if (p < 0) return;  // cannot happen for jb <= rows; defensive
    for (int cc = t; cc < jb; cc += kPanelThreads) {
      const int64_t ws = ((int64_t)b * 2 + par) * w.pmax + win;
      const F* src = cand_row + ws * kPanel + cc;
      const F* dsrc = diag_row + ((int64_t)b * 2 + par) * kPanel + cc;
      F u, dd;
      if constexpr (sizeof(F) == 16) {
        double2 x = __ldcg((const double2*)src);
        double2 y = __ldcg((const double2*)dsrc);
        u = F{x.x, x.y};
        dd = F{y.x, y.y};
      } else {
        float2 x = __ldcg((const float2*)src);
        float2 y = __ldcg((const float2*)dsrc);
        u = F{x.x, x.y};
        dd = F{y.x, y.y};
      }
      s_u[cc] = u;
      s_d[cc] = dd;
    }
    __syncthreads();
    const F piv = s_u[j];
    F inv;
    if (abs2(piv) == 0) {
      inv = num<F>::zero();
      if (c == 0 && t == 0) atomicCAS(&w.zero_pivot[b], 0, (int)col + 1);
    } else {
      inv = recip(piv);
    }
    if (d >= row_lo && d < row_hi)
      for (int cc = t; cc < jb; cc += kPanelThreads) at(d, cc) = s_u[cc];
    if (p != d && p >= row_lo && p < row_hi)
      for (int cc = t; cc < jb; cc += kPanelThreads) at(p, cc) = s_d[cc];
    if (c == 0 && t == 0) ipiv[(int64_t)b * n + d] = p;
    __syncthreads();

    v = -1.0;
    vi = -1;
    const int64_t lo = max(row_lo, d + 1);
    for (int64_t i = lo + t; i < row_hi; i += kPanelThreads) {
      F l = at(i, j) * inv;
      at(i, j) = l;
      for (int cc = j + 1; cc < jb; ++cc) {
        F x = at(i, cc) - l * s_u[cc];
        at(i, cc) = x;
        if (cc == j + 1) argmax_merge<F>(v, vi, (double)abs2(x), (int)i);
      }
    }
    if (j + 1 < jb) block_argmax<F>(v, vi);
    else __syncthreads();
  }
  if constexpr (CACHE) {
    const int64_t nr = row_hi - row_lo;
    for (int64_t l = t; l < nr * jb; l += kPanelThreads) {
      const int64_t i = l % nr, cc = l / nr;
      Mb[(row_lo + i) + (k0 + cc) * ld] = T[i + cc * R];
    }
  }

  if (c == 0 && t == 0) panel_swap_summary(b, n, k0, jb, ipiv, w);
}

// The panel factored by one thread-block cluster per node: the cluster's
// kPanelCluster CTAs hold all of the panel's rows in their shared memory
// (distributed shared memory, R <= kPanelClusterRows rows each), so a column
// step exchanges its pivot candidates and the pivot and diagonal rows through
// the cluster's shared memory with two hardware cluster barriers, instead of
// global memory and a software barrier.  Same arithmetic and pivot choice as
// panel_lu_kernel.  Clusters (nodes) are independent of one another.
constexpr int kPanelCluster = 16;
constexpr int kPanelClusterRows = 512;

template <typename F>
__global__ void __launch_bounds__(kPanelThreads, 1)
panel_lu_cluster_kernel(F* M, int64_t n, int64_t ld, int64_t stride, int k0, int jb, int64_t R, int32_t* ipiv,
                        PanelWork w) {
  namespace cgx = cooperative_groups;
  cgx::cluster_group cluster = cgx::this_cluster();
  const int b = blockIdx.x / kPanelCluster;
  const int c = (int)cluster.block_rank();
  const int t = threadIdx.x;
  F* Mb = M + (int64_t)b * stride;
  const int64_t row_lo = k0 + (int64_t)c * R;
  const int64_t row_hi = min(n, row_lo + R);
  const int64_t nr = row_hi > row_lo ? row_hi - row_lo : 0;
  extern __shared__ __align__(16) unsigned char cpanel_smem[];
  F* T = reinterpret_cast<F*>(cpanel_smem);
  __shared__ double s_cv;   // this CTA's pivot candidate (read by the cluster)
  __shared__ int s_ci;
  __shared__ F s_u[kPanel];
  __shared__ F s_d[kPanel];
  __shared__ int s_p;
  auto at = [&](int64_t i, int cc) -> F& { return T[(i - row_lo) + (int64_t)cc * R]; };
  for (int64_t l = t; l < nr * jb; l += kPanelThreads) {
    const int64_t i = l % nr, cc = l / nr;
    T[i + cc * R] = Mb[(row_lo + i) + (k0 + cc) * ld];
  }
  __syncthreads();
  double v = -1.0;
  int vi = -1;
  for (int64_t i = row_lo + t; i < row_hi; i += kPanelThreads) argmax_merge<F>(v, vi, (double)abs2(at(i, 0)), (int)i);
  block_argmax<F>(v, vi);

  for (int j = 0; j < jb; ++j) {
    const int64_t d = k0 + j;
    if (t == 0) {
      s_cv = v;
      s_ci = vi;
    }
    cluster.sync();  // every CTA's candidate is in place
    if (t < 32) {
      double bv = -1.0;
      int bi = -1;
      if (t < kPanelCluster) {
        bv = *cluster.map_shared_rank(&s_cv, t);
        bi = *cluster.map_shared_rank(&s_ci, t);
      }
      for (int off = 16; off > 0; off >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, bv, off);
        const int i2 = __shfl_down_sync(0xffffffffu, bi, off);
        if (i2 >= 0 && (v2 > bv || (v2 == bv && (bi < 0 || i2 < bi)))) {
          bv = v2;
          bi = i2;
        }
      }
      if (t == 0) s_p = bi;
    }
    __syncthreads();
    const int p = s_p;
    // the pivot row and the diagonal row from the CTAs that hold them
    if (p >= 0 && t < jb) {
      const int op = (int)((p - k0) / R), od = (int)((d - k0) / R);
      F* Tp = cluster.map_shared_rank(T, op);
      F* Td = cluster.map_shared_rank(T, od);
      const int64_t lp = p - (k0 + (int64_t)op * R), ldd = d - (k0 + (int64_t)od * R);
      s_u[t] = Tp[lp + (int64_t)t * R];
      s_d[t] = Td[ldd + (int64_t)t * R];
    }
    cluster.sync();  // every CTA has read both rows before their owners overwrite them
    if (p < 0) continue;  // cannot happen for jb <= rows (uniform across the cluster)
    const F piv = s_u[j];
    F inv;
    if (abs2(piv) == 0) {
      inv = num<F>::zero();
      if (c == 0 && t == 0) atomicCAS(&w.zero_pivot[b], 0, (int)d + 1);
    } else {
      inv = recip(piv);
    }
    if (d >= row_lo && d < row_hi)
      for (int cc = t; cc < jb; cc += kPanelThreads) at(d, cc) = s_u[cc];
    if (p != d && p >= row_lo && p < row_hi)
      for (int cc = t; cc < jb; cc += kPanelThreads) at(p, cc) = s_d[cc];
    if (c == 0 && t == 0) ipiv[(int64_t)b * n + d] = p;
    __syncthreads();
    v = -1.0;
    vi = -1;
    const int64_t lo = max(row_lo, d + 1);
    for (int64_t i = lo + t; i < row_hi; i += kPanelThreads) {
      F l = at(i, j) * inv;
      at(i, j) = l;
      for (int cc = j + 1; cc < jb; ++cc) {
        F x = at(i, cc) - l * s_u[cc];
        at(i, cc) = x;
        if (cc == j + 1) argmax_merge<F>(v, vi, (double)abs2(x), (int)i);
      }
    }
    if (j + 1 < jb) block_argmax<F>(v, vi);
    else __syncthreads();
  }
  for (int64_t l = t; l < nr * jb; l += kPanelThreads) {
    const int64_t i = l % nr, cc = l / nr;
    Mb[(row_lo + i) + (k0 + cc) * ld] = T[i + cc * R];
  }
  if (c == 0 && t == 0) panel_swap_summary(b, n, k0, jb, ipiv, w);
  cluster.sync();  // no CTA leaves while another may still read its shared memory
}

constexpr int kSwapWarps = 8;

template <typename F>
__global__ void __launch_bounds__(kSwapWarps * 32)
laswp_trsm_kernel(F* M, int64_t n, int64_t ld, int64_t stride, int k0, int jb,
                  const int* swap_src, const int* swap_dst, const int* swap_cnt) {
  const int b = blockIdx.y;
  F* Mb = M + (int64_t)b * stride;
  __shared__ F L11[kPanel][kPanel + 1];
  for (int l = threadIdx.x; l < jb * jb; l += blockDim.x) {
    int i = l % jb, j = l / jb;
    L11[i][j] = Mb[(k0 + i) + (int64_t)(k0 + j) * ld];
  }
  __syncthreads();
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t idx = (int64_t)blockIdx.x * kSwapWarps + wp;
  if (idx >= n - jb) return;
  const int64_t c = idx < k0 ? idx : idx + jb;
  F* colp = Mb + c * ld;
  const int cnt = swap_cnt[b];
  const int* src = swap_src + b * 2 * kPanel;
  const int* dst = swap_dst + b * 2 * kPanel;
  F v0 = num<F>::zero(), v1 = num<F>::zero();
  if (lane < cnt) v0 = colp[src[lane]];
  if (lane + 32 < cnt) v1 = colp[src[lane + 32]];
  __syncwarp();
  if (lane < cnt) colp[dst[lane]] = v0;
  if (lane + 32 < cnt) colp[dst[lane + 32]] = v1;
  __syncwarp();
  if (c >= k0 + jb) {
    F x = lane < jb ? colp[k0 + lane] : num<F>::zero();
    for (int j = 0; j < jb - 1; ++j) {
      F xj = shfl(x, j);
      if (lane > j && lane < jb) x = x - L11[lane][j] * xj;
    }
    if (lane < jb) colp[k0 + lane] = x;
  }
}

// Net effect of the row interchanges ipiv[r0 .. r0+cnt) (cnt <= kTcBlock) of
// every node on the rows they touch: after the swaps, row dst holds the
// former row src.  One warp per node: rows r0 .. r0+cnt-1 are indexed
// directly, pivot rows beyond them go to a short list searched by the warp.
// Pivot rows never lie above their step's row, so each swap is O(1) plus a
// ballot search.
__global__ void block_swap_summary_kernel(const int32_t* ipiv, int64_t n, int64_t r0, int cnt, int* src, int* dst,
                                          int* cntp, int cap) {
  const int b = blockIdx.x;
  const int lane = threadIdx.x;
  __shared__ int piv[kTcBlock];
  __shared__ int inner[kTcBlock];        // original row now held by row r0 + j
  __shared__ int ext_row[kTcBlock], ext_cont[kTcBlock];
  __shared__ int s_next;
  for (int j = lane; j < cnt; j += 32) {
    piv[j] = ipiv[(int64_t)b * n + r0 + j];
    inner[j] = (int)(r0 + j);
  }
  if (lane == 0) s_next = 0;
  __syncwarp();
  const int64_t r1 = r0 + cnt;
  for (int j = 0; j < cnt; ++j) {
    const int p = piv[j];
    if (p < r1) {
      if (lane == 0 && p != r0 + j) {
        const int t = inner[j];
        inner[j] = inner[p - r0];
        inner[p - r0] = t;
      }
    } else {
      const int m = s_next;
      int slot = -1;
      for (int q0 = 0; q0 < m; q0 += 32) {
        const int q = q0 + lane;
        const unsigned hit = __ballot_sync(0xffffffffu, q < m && ext_row[q] == p);
        if (hit) { slot = q0 + __ffs(hit) - 1; break; }
      }
      if (lane == 0) {
        if (slot < 0) {
          slot = m;
          ext_row[m] = p;
          ext_cont[m] = p;
          s_next = m + 1;
        }
        const int t = inner[j];
        inner[j] = ext_cont[slot];
        ext_cont[slot] = t;
      }
    }
    __syncwarp();
  }
  // compacted lists of the rows that moved
  if (lane == 0) {
    int out = 0;
    int* d = dst + (int64_t)b * cap;
    int* sr = src + (int64_t)b * cap;
    for (int j = 0; j < cnt; ++j)
      if (inner[j] != r0 + j) { d[out] = (int)(r0 + j); sr[out] = inner[j]; ++out; }
    for (int q = 0; q < s_next; ++q)
      if (ext_cont[q] != ext_row[q]) { d[out] = ext_row[q]; sr[out] = ext_cont[q]; ++out; }
    cntp[b] = out;
  }
}

// Apply a per-node row permutation list (row dst <- former row src, at most
// MAXS entries) to the columns [c0, c1) outside [s0, s1): warp per column.
template <typename F, int MAXS>
__global__ void __launch_bounds__(kSwapWarps * 32)
row_gather_kernel(F* M, int64_t ld, int64_t stride, int64_t c0, int64_t c1, int64_t s0, int64_t s1,
                  const int* src, const int* dst, const int* cntp, int cap) {
  const int b = blockIdx.y;
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t ncols = (c1 - c0) - (s1 - s0);
  const int64_t idx = (int64_t)blockIdx.x * kSwapWarps + wp;
  if (idx >= ncols) return;
  const int64_t c = (c0 + idx < s0) ? c0 + idx : c0 + idx + (s1 - s0);
  F* colp = M + (int64_t)b * stride + c * ld;
  const int cnt = cntp[b];
  const int* sr = src + (int64_t)b * cap;
  const int* ds = dst + (int64_t)b * cap;
  constexpr int PER = MAXS / 32;
  F v[PER];
#pragma unroll
  for (int q = 0; q < PER; ++q) v[q] = (lane + 32 * q < cnt) ? colp[sr[lane + 32 * q]] : num<F>::zero();
  __syncwarp();
#pragma unroll
  for (int q = 0; q < PER; ++q)
    if (lane + 32 * q < cnt) colp[ds[lane + 32 * q]] = v[q];
}

// U <- L11^{-1} U on the rows [r0, r0 + jb) of the columns [c0, c1), L11 the
// unit-lower diagonal block at (r0, r0): warp per column.
template <typename F>
__global__ void __launch_bounds__(kSwapWarps * 32)
trsm_rows_kernel(F* M, int64_t ld, int64_t stride, int64_t r0, int jb, int64_t c0, int64_t c1) {
  const int b = blockIdx.y;
  F* Mb = M + (int64_t)b * stride;
  __shared__ F L11[kPanel][kPanel + 1];
  for (int l = threadIdx.x; l < jb * jb; l += blockDim.x) {
    const int i = l % jb, j = l / jb;
    L11[i][j] = Mb[(r0 + i) + (r0 + j) * ld];
  }
  __syncthreads();
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t c = c0 + (int64_t)blockIdx.x * kSwapWarps + wp;
  if (c >= c1) return;
  F* colp = Mb + c * ld;
  F x = lane < jb ? colp[r0 + lane] : num<F>::zero();
  for (int j = 0; j < jb - 1; ++j) {
    const F xj = shfl(x, j);
    if (lane > j && lane < jb) x = x - L11[lane][j] * xj;
  }
  if (lane < jb) colp[r0 + lane] = x;
}

__global__ void build_perm_kernel(const int32_t* ipiv, int32_t* perm, int64_t n) {
  extern __shared__ int32_t sp[];
  const int b = blockIdx.x;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) sp[i] = (int32_t)i;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int32_t* ip = ipiv + (int64_t)b * n;
    for (int64_t k = 0; k < n; ++k) {
      int32_t p = ip[k];
      if (p != k) {
        int32_t tmp = sp[k];
        sp[k] = sp[p];
        sp[p] = tmp;
      }
    }
  }
  __syncthreads();
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) perm[(int64_t)b * n + i] = sp[i];
}

template <typename F, typename TA>
__global__ void form_shifted_kernel(F* M, int64_t n, int64_t ld, int64_t stride,
                                    const TA* A, int64_t lda, const c128* z) {
  const int b = blockIdx.y;
  const c128 zb = z[b];
  F* Mb = M + (int64_t)b * stride;
  const int64_t total = n * n;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, j = idx / n;
    c128 v = -cvt<c128>(A[i + j * lda]);
    if (i == j) v = v + zb;
    Mb[i + j * ld] = cvt<F>(v);
  }
}

// Triangular solve on a TB x TB diagonal block, warp per right-hand-side
// column, TB/32 rows per lane.  mode 0: L (unit lower, stored), 1: U^H
// (lower, from the stored U), 2: U (upper, stored), 3: L^H (unit upper, from
// the stored L).
template <typename F, int TB>
__global__ void __launch_bounds__(256)
trsm_diag_kernel(const F* M, int64_t ld, int64_t stride, F* Y, int64_t n, int64_t m,
                 int64_t ystride, int64_t r0, int bs, int mode) {
  constexpr int R = TB / 32;
  const int b = blockIdx.y;
  const F* Mb = M + (int64_t)b * stride;
  __shared__ F T[TB][TB + 1];
  for (int l = threadIdx.x; l < bs * bs; l += blockDim.x) {
    if (mode == 0 || mode == 2) {
      int i = l % bs, j = l / bs;
      T[i][j] = Mb[(r0 + i) + (r0 + j) * ld];
    } else {
      int j = l % bs, i = l / bs;
      T[i][j] = conj(Mb[(r0 + j) + (r0 + i) * ld]);
    }
  }
  __syncthreads();
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t cidx = (int64_t)blockIdx.x * 8 + wp;
  if (cidx >= m) return;
  F* y = Y + (int64_t)b * ystride + cidx * n + r0;
  F x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = (lane + 32 * r < bs) ? y[lane + 32 * r] : num<F>::zero();
  if (mode <= 1) {
    for (int j = 0; j < bs; ++j) {
      const int jl = j & 31, jr = j >> 5;
      if (mode == 1 && lane == jl) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == jr) x[r] = x[r] * recip(T[j][j]);
      }
      F xs = num<F>::zero();
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r == jr) xs = x[r];
      const F xj = shfl(xs, jl);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = lane + 32 * r;
        if (row > j && row < bs) x[r] = x[r] - T[row][j] * xj;
      }
    }
  } else {
    for (int j = bs - 1; j >= 0; --j) {
      const int jl = j & 31, jr = j >> 5;
      if (mode == 2 && lane == jl) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (r == jr) x[r] = x[r] * recip(T[j][j]);
      }
      F xs = num<F>::zero();
#pragma unroll
      for (int r = 0; r < R; ++r)
        if (r == jr) xs = x[r];
      const F xj = shfl(xs, jl);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int row = lane + 32 * r;
        if (row < j) x[r] = x[r] - T[row][j] * xj;
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (lane + 32 * r < bs) y[lane + 32 * r] = x[r];
}

// Triangular solve on a whole outer block (bs <= 256 rows) for the
// tensor-core route: one launch replaces the four 64-row diagonal solves and
// the three inner block updates of the outer block.  Warp per right-hand-side
// column with the column's 256 entries in registers (8 per lane, register r
// holding rows 32 r + lane); the block's triangle goes through shared memory
// in 32-column panels (column-major, zero outside the triangle and past bs),
// the next panel loaded into registers while the current one is used.  Panel
// p holds the columns of register p, so every register index is a
// compile-time constant and the rows a step cannot touch are skipped whole.
// Modes as trsm_diag_kernel; a non-unit diagonal is stored as its reciprocal.
// The solved block also goes out as the six bf16 planes of the outer update's
// right operand (K index = row within the outer block, zero past bs).
constexpr int kTrsmOuterWarps = 16;
constexpr int kTrsmOuterThreads = kTrsmOuterWarps * 32;
constexpr int kTrsmOuterLd = kSolveOuter + 1;  // padded panel column
constexpr size_t kTrsmOuterSmem = sizeof(c64) * 32 * kTrsmOuterLd;

template <int MODE>
__global__ void __launch_bounds__(kTrsmOuterThreads, 1)
trsm_outer_kernel(const c64* __restrict__ M, int64_t ld, int64_t stride, c64* __restrict__ Y, int64_t n, int64_t m,
                  int64_t ystride, int64_t R0, int bs, uint16_t* __restrict__ planes, int64_t mpad) {
  constexpr int OB = kSolveOuter, LDP = kTrsmOuterLd, R = OB / 32;
  constexpr int PER = 32 * OB / kTrsmOuterThreads;  // panel elements per thread
  constexpr bool kFwd = MODE <= 1, kStored = MODE == 0 || MODE == 2, kUnit = MODE == 0 || MODE == 3;
  extern __shared__ __align__(16) unsigned char trsm_smem[];
  c64* P = reinterpret_cast<c64*>(trsm_smem);
  const int b = blockIdx.y;
  const c64* Mb = M + (int64_t)b * stride;
  const int tid = threadIdx.x, wp = tid >> 5, lane = tid & 31;
  const int64_t cidx = (int64_t)blockIdx.x * kTrsmOuterWarps + wp;
  const bool active = cidx < m;
  c64* y = Y + (int64_t)b * ystride + cidx * n + R0;
  c64 x[R];
#pragma unroll
  for (int r = 0; r < R; ++r) x[r] = (active && lane + 32 * r < bs) ? y[lane + 32 * r] : num<c64>::zero();
  // T[rr][cc] of panel p (columns 32 p .. 32 p + 31) into registers: the rows a
  // forward step reaches are [32 p, bs), a backward one [0, 32 p + 32)
  c64 pre[PER];
  auto fetch = [&](int p) {
    const int c0 = 32 * p;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int l = tid + kTrsmOuterThreads * i;
      int rr, cc;
      if (kStored) {  // rows fastest: contiguous in the stored factor
        rr = l & (OB - 1);
        cc = c0 + (l >> 8);
      } else {        // columns fastest: contiguous in the stored row of the transpose
        cc = c0 + (l & 31);
        rr = l >> 5;
      }
      const bool in = rr < bs && cc < bs && (kFwd ? rr >= c0 : rr < c0 + 32);
      c64 v = num<c64>::zero();
      if (in) v = kStored ? Mb[(R0 + rr) + (R0 + cc) * ld] : conj(Mb[(R0 + cc) + (R0 + rr) * ld]);
      pre[i] = v;
    }
  };
  auto stash = [&](int p) {
    const int c0 = 32 * p;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int l = tid + kTrsmOuterThreads * i;
      const int rr = kStored ? (l & (OB - 1)) : (l >> 5);
      const int cc = kStored ? (c0 + (l >> 8)) : (c0 + (l & 31));
      // non-unit diagonal: its reciprocal, the only use of the entry
      P[(cc - c0) * LDP + rr] = (!kUnit && rr == cc) ? recip(pre[i]) : pre[i];
    }
  };
  const int np = (bs + 31) / 32;
  fetch(kFwd ? 0 : np - 1);
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int p = kFwd ? q : R - 1 - q;  // panel = register index (compile-time)
    if (p >= np) continue;              // panels past bs (uniform)
    __syncthreads();                    // the previous panel has been used
    stash(p);
    __syncthreads();
    const int pn = kFwd ? p + 1 : p - 1;
    if (kFwd ? pn < np : pn >= 0) fetch(pn);  // in flight during this panel
    if (!active) continue;
    const int jend = min(32, bs - 32 * p);
    for (int t = 0; t < jend; ++t) {
      const int jl = kFwd ? t : jend - 1 - t;
      const c64* Tj = P + jl * LDP;
      c64 xj = shfl(x[p], jl);
      if (!kUnit) {  // every lane scales the broadcast value; lane jl keeps it
        xj = xj * Tj[32 * p + jl];
        if (lane == jl) x[p] = xj;
      }
      if (kFwd) {
        if (lane > jl) x[p] = x[p] - Tj[32 * p + lane] * xj;
#pragma unroll
        for (int r = p + 1; r < R; ++r) x[r] = x[r] - Tj[32 * r + lane] * xj;
      } else {
        if (lane < jl) x[p] = x[p] - Tj[32 * p + lane] * xj;
#pragma unroll
        for (int r = 0; r < p; ++r) x[r] = x[r] - Tj[32 * r + lane] * xj;
      }
    }
  }
  if (!active) return;
#pragma unroll
  for (int r = 0; r < R; ++r)
    if (lane + 32 * r < bs) y[lane + 32 * r] = x[r];
  const int64_t plane = mpad * OB;
  uint16_t* o = planes + (int64_t)b * 6 * plane + cidx * OB;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int t = lane + 32 * r;
    const c64 v = t < bs ? x[r] : num<c64>::zero();
    uint16_t a0, a1, a2, b0, b1, b2;
    cg_split3(v.re, a0, a1, a2);
    cg_split3(v.im, b0, b1, b2);
    o[t] = a0;
    o[plane + t] = a1;
    o[2 * plane + t] = a2;
    o[3 * plane + t] = b0;
    o[4 * plane + t] = b1;
    o[5 * plane + t] = b2;
  }
}

// solve block rows: 64 for complex-FP32 factors, 32 for complex-FP64 (whose
// 64 x 64 shared tile would exceed the static shared-memory limit)
template <typename F> struct SolveBlock { static constexpr int value = 64; };
static_assert(kSolveBlock == 64, "tensor-core solve planes use the complex-FP32 diagonal block");
template <> struct SolveBlock<c128> { static constexpr int value = 32; };

template <typename F, typename TB>
__global__ void permute_in_kernel(F* Y, int64_t ystride, const TB* B, int64_t ldb, int64_t bstride, int64_t n, int64_t m,
                                  const int32_t* perm, bool adjoint) {
  const int b = blockIdx.y;
  const int64_t total = n * m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, c = idx / n;
    const int64_t src = adjoint ? i : perm[(int64_t)b * n + i];
    Y[(int64_t)b * ystride + idx] = cvt<F>(B[(int64_t)b * bstride + src + c * ldb]);
  }
}

template <typename F, typename TO>
__global__ void permute_out_kernel(TO* Out, int64_t ostride, const F* Y, int64_t ystride, int64_t n,
                                   int64_t m, const int32_t* perm, bool adjoint, bool accumulate) {
  const int b = blockIdx.y;
  const int64_t total = n * m;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx % n, c = idx / n;
    const int64_t dst = adjoint ? perm[(int64_t)b * n + i] : i;
    TO* o = Out + (int64_t)b * ostride + dst + c * n;
    TO v = cvt<TO>(Y[(int64_t)b * ystride + idx]);
    *o = accumulate ? (*o + v) : v;
  }
}

__global__ void invert_perm_kernel(const int32_t* perm, int32_t* pinv, int64_t n) {
  const int64_t b = blockIdx.y;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    pinv[b * n + perm[b * n + i]] = (int32_t)i;
}

template <typename S, typename F>
__global__ void solve_accumulate_kernel(S* Xf, int64_t ldx, const c128* base, const F* Yn, const F* Ya, int64_t n,
                                        int64_t m, int nc, const int32_t* pinv, const c128* w) {
  const int64_t nm = n * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nm; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, c = t / n;
    c128 acc{0.0, 0.0};
    for (int e = 0; e < nc; ++e) {
      c128 z = cvt<c128>(Yn[(int64_t)e * nm + t]);
      if (base) z = z + base[(int64_t)e * nm + t];
      acc = acc + w[e] * z;
      if constexpr (is_cx<S>::value) {
        c128 za = cvt<c128>(Ya[(int64_t)e * nm + pinv[(int64_t)e * n + i] + c * n]);
        if (base) za = za + base[(int64_t)(nc + e) * nm + t];
        acc = acc + conj(w[e]) * za;
      }
    }
    if constexpr (is_cx<S>::value) Xf[i + c * ldx] = acc;
    else Xf[i + c * ldx] = 2.0 * acc.re;
  }
}

inline unsigned grid1d(int64_t total, int threads = 256) {
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(cdiv(total, threads), 8192));
}

}  // namespace

size_t panel_work_bytes(int nodes, int pmax, size_t eb) {
  size_t s = 0;
  auto add = [&](size_t bytes) { s += (bytes + 255) & ~size_t(255); };
  add(sizeof(unsigned) * nodes);
  add(sizeof(int));
  add(sizeof(int) * nodes);
  add(sizeof(double) * nodes * 2 * pmax);
  add(sizeof(int) * nodes * 2 * pmax);
  add(eb * nodes * 2 * pmax * kPanel);
  add(eb * nodes * 2 * kPanel);
  add(sizeof(int) * nodes * 2 * kPanel);
  add(sizeof(int) * nodes * 2 * kPanel);
  add(sizeof(int) * nodes);
  add(sizeof(int) * nodes * 2 * kTcBlock);
  add(sizeof(int) * nodes * 2 * kTcBlock);
  add(sizeof(int) * nodes);
  return s;
}

PanelWork panel_work_carve(void* base, int nodes, int pmax, size_t eb) {
  char* p = (char*)base;
  auto take = [&](size_t bytes) { char* r = p; p += (bytes + 255) & ~size_t(255); return (void*)r; };
  PanelWork w{};
  w.counters = (unsigned*)take(sizeof(unsigned) * nodes);
  w.status = (int*)take(sizeof(int));
  w.zero_pivot = (int*)take(sizeof(int) * nodes);
  w.cand_val = (double*)take(sizeof(double) * nodes * 2 * pmax);
  w.cand_idx = (int*)take(sizeof(int) * nodes * 2 * pmax);
  w.cand_row = take(eb * nodes * 2 * pmax * kPanel);
  w.diag_row = take(eb * nodes * 2 * kPanel);
  w.swap_src = (int*)take(sizeof(int) * nodes * 2 * kPanel);
  w.swap_dst = (int*)take(sizeof(int) * nodes * 2 * kPanel);
  w.swap_cnt = (int*)take(sizeof(int) * nodes);
  w.blk_src = (int*)take(sizeof(int) * nodes * 2 * kTcBlock);
  w.blk_dst = (int*)take(sizeof(int) * nodes * 2 * kTcBlock);
  w.blk_cnt = (int*)take(sizeof(int) * nodes);
  w.pmax = pmax;
  w.tc_planes = nullptr;
  return w;
}

template <typename F, typename TA>
void form_shifted(F* M, int64_t n, int64_t ld, int64_t stride, int nodes,
                  const TA* A, int64_t lda, const c128* z, cudaStream_t s) {
  dim3 grid(grid1d(n * n), nodes);
  form_shifted_kernel<F, TA><<<grid, 256, 0, s>>>(M, n, ld, stride, A, lda, z);
  FEAST_LAUNCH_CHECK();
}

void lu_tc_trailing_update(c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, int64_t k0, int kb, void* planes,
                           int* status, int num_sms, cudaStream_t s);

template <typename F>
void lu_factor_batched(F* M, int64_t n, int64_t ld, int64_t stride, int nodes,
                       int32_t* ipiv, int32_t* perm, const PanelWork& w,
                       int num_sms, cudaStream_t s) {
  FEAST_CUDA_TRY(cudaMemsetAsync(w.counters, 0, sizeof(unsigned) * nodes, s));
  FEAST_CUDA_TRY(cudaMemsetAsync(w.status, 0, sizeof(int), s));
  FEAST_CUDA_TRY(cudaMemsetAsync(w.zero_pivot, 0, sizeof(int) * nodes, s));
  int occ = 0;
  FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, panel_lu_kernel<F, false>, kPanelThreads, 0));
  const int max_coop = std::max(1, occ) * num_sms;
  // the shared-memory variant: at most kPanelCacheRows rows per CTA
  const size_t cache_max = sizeof(F) * (size_t)kPanelCacheRows * kPanel;
  FEAST_CUDA_TRY(cudaFuncSetAttribute(panel_lu_kernel<F, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)cache_max));
  int occ_c = 0;
  FEAST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, panel_lu_kernel<F, true>, kPanelThreads,
                                                               cache_max));
  const int max_coop_c = occ_c * num_sms;
  // the cluster variant: can a cluster of kPanelCluster CTAs with the largest
  // panel slice be resident at all?
  const size_t cl_max = sizeof(F) * (size_t)kPanelClusterRows * kPanel;
  bool cluster_ok = cl_max <= 200 * 1024;
  if (cluster_ok) {
    FEAST_CUDA_TRY(cudaFuncSetAttribute(panel_lu_cluster_kernel<F>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    FEAST_CUDA_TRY(cudaFuncSetAttribute(panel_lu_cluster_kernel<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)cl_max));
    cudaLaunchConfig_t q{};
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = kPanelCluster;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.gridDim = dim3(kPanelCluster);
    q.blockDim = dim3(kPanelThreads);
    q.dynamicSmemBytes = cl_max;
    q.attrs = qa;
    q.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, panel_lu_cluster_kernel<F>, &q) != cudaSuccess) {
      cudaGetLastError();
      nclusters = 0;
    }
    cluster_ok = nclusters > 0;
  }
  unsigned base = 0;
  // complex-FP32 factors with tensor-core scratch: two-level blocking, outer
  // blocks of kTcBlock columns whose trailing update runs on the tensor cores,
  // each factored by kPanel-wide panels with CUDA-core updates restricted to
  // the block's columns and its row band; otherwise one level of kPanel.
  bool tc = false;
  if constexpr (std::is_same<F, c64>::value) tc = w.tc_planes != nullptr;
  const int64_t NB = tc ? kTcBlock : kPanel;
  auto gemm_update = [&](int64_t rows0, int64_t rows1, int64_t cols0, int64_t cols1, int64_t kc, int kw) {
    if (rows1 <= rows0 || cols1 <= cols0) return;
    GemmArgs g{};
    g.M = rows1 - rows0; g.N = cols1 - cols0; g.K = kw;
    g.A = M + rows0 + kc * ld; g.lda = ld; g.strideA = stride; g.opA = OP_N;
    g.B = M + kc + cols0 * ld; g.ldb = ld; g.strideB = stride; g.opB = OP_N;
    g.C = M + rows0 + cols0 * ld; g.ldc = ld; g.strideC = stride;
    g.alpha = C1(-1.0); g.beta = C1(1.0); g.batch = nodes; g.ksplit = 1;
    gemm<F, F, F>(g, s);
  };
  auto panel = [&](int64_t k1, int jb) {
    const int64_t H = n - k1;
    int k1i = (int)k1;
    PanelWork wl = w;
    // one cluster per node holding the whole panel in its shared memory
    if (cluster_ok && cdiv(H, kPanelCluster) <= kPanelClusterRows) {
      int64_t Rc = cdiv(H, kPanelCluster);
      cudaLaunchConfig_t q{};
      cudaLaunchAttribute qa[1];
      qa[0].id = cudaLaunchAttributeClusterDimension;
      qa[0].val.clusterDim.x = kPanelCluster;
      qa[0].val.clusterDim.y = 1;
      qa[0].val.clusterDim.z = 1;
      q.gridDim = dim3((unsigned)(nodes * kPanelCluster));
      q.blockDim = dim3(kPanelThreads);
      q.dynamicSmemBytes = sizeof(F) * (size_t)Rc * kPanel;
      q.stream = s;
      q.attrs = qa;
      q.numAttrs = 1;
      FEAST_CUDA_TRY(cudaLaunchKernelEx(&q, panel_lu_cluster_kernel<F>, M, n, ld, stride, k1i, jb, Rc, ipiv, wl));
      note_launch();
      return;
    }
    // rows of the panel in shared memory when every node's rows fit in
    // co-resident CTAs of at most kPanelCacheRows rows each
    int Pc = (int)std::min<int64_t>({cdiv(H, 64), (int64_t)(max_coop_c / nodes), (int64_t)w.pmax});
    if (Pc >= 1 && cdiv(H, Pc) <= kPanelCacheRows) {
      const int64_t Rc = cdiv(H, Pc);
      int P = (int)cdiv(H, Rc);
      void* args[] = {&M, &n, &ld, &stride, &k1i, (void*)&jb, &P, (void*)&Rc, &ipiv, &wl, &base};
      FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)panel_lu_kernel<F, true>, dim3(nodes * P),
                                                 dim3(kPanelThreads), args, sizeof(F) * (size_t)Rc * kPanel, s));
      note_launch();
      base += (unsigned)jb * (unsigned)P;
      return;
    }
    int P = (int)std::min<int64_t>(cdiv(H, 64), std::max(1, max_coop / nodes));
    P = std::max(1, std::min(P, w.pmax));
    const int64_t R = cdiv(H, P);
    P = (int)cdiv(H, R);  // no empty CTAs
    void* args[] = {&M, &n, &ld, &stride, &k1i, (void*)&jb, &P, (void*)&R, &ipiv, &wl, &base};
    FEAST_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)panel_lu_kernel<F, false>, dim3(nodes * P),
                                               dim3(kPanelThreads), args, 0, s));
    note_launch();
    base += (unsigned)jb * (unsigned)P;
  };
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int64_t nbo = std::min<int64_t>(NB, n - k0);
    const int64_t blk_end = k0 + nbo;
    if (!tc) {
      // one level: panel, interchanges + U12 for every other column, trailing update
      const int jb = (int)nbo;
      panel(k0, jb);
      if (n - jb > 0) {
        dim3 g2((unsigned)cdiv(n - jb, kSwapWarps), nodes);
        laswp_trsm_kernel<F><<<g2, kSwapWarps * 32, 0, s>>>(M, n, ld, stride, (int)k0, jb, w.swap_src, w.swap_dst,
                                                             w.swap_cnt);
        FEAST_LAUNCH_CHECK();
      }
      gemm_update(blk_end, n, blk_end, n, k0, jb);
      continue;
    }
    // two levels: factor the tall block [k0, n) x [k0, blk_end) panel by panel,
    // interchanges and updates confined to the block's columns
    for (int64_t k1 = k0; k1 < blk_end; k1 += kPanel) {
      const int jb = (int)std::min<int64_t>(kPanel, blk_end - k1);
      const int64_t r1 = k1 + jb;
      panel(k1, jb);
      if (nbo > jb) {
        dim3 g2((unsigned)cdiv(nbo - jb, kSwapWarps), nodes);
        row_gather_kernel<F, 2 * kPanel><<<g2, kSwapWarps * 32, 0, s>>>(M, ld, stride, k0, blk_end, k1, r1,
                                                                         w.swap_src, w.swap_dst, w.swap_cnt,
                                                                         2 * kPanel);
        FEAST_LAUNCH_CHECK();
      }
      if (r1 < blk_end) {
        dim3 g3((unsigned)cdiv(blk_end - r1, kSwapWarps), nodes);
        trsm_rows_kernel<F><<<g3, kSwapWarps * 32, 0, s>>>(M, ld, stride, k1, jb, r1, blk_end);
        FEAST_LAUNCH_CHECK();
      }
      gemm_update(r1, n, r1, blk_end, k1, jb);
    }
    // the block's interchanges on the columns left and right of it
    block_swap_summary_kernel<<<nodes, 32, 0, s>>>(ipiv, n, k0, (int)nbo, w.blk_src, w.blk_dst, w.blk_cnt,
                                                    2 * kTcBlock);
    FEAST_LAUNCH_CHECK();
    if (n - nbo > 0) {
      dim3 g4((unsigned)cdiv(n - nbo, kSwapWarps), nodes);
      row_gather_kernel<F, 2 * kTcBlock><<<g4, kSwapWarps * 32, 0, s>>>(M, ld, stride, 0, n, k0, blk_end, w.blk_src,
                                                                         w.blk_dst, w.blk_cnt, 2 * kTcBlock);
      FEAST_LAUNCH_CHECK();
    }
    if (blk_end < n) {
      // U12 = L11^{-1} A12 for the block's row band, panel by panel
      for (int64_t k1 = k0; k1 < blk_end; k1 += kPanel) {
        const int jb = (int)std::min<int64_t>(kPanel, blk_end - k1);
        dim3 g5((unsigned)cdiv(n - blk_end, kSwapWarps), nodes);
        trsm_rows_kernel<F><<<g5, kSwapWarps * 32, 0, s>>>(M, ld, stride, k1, jb, blk_end, n);
        FEAST_LAUNCH_CHECK();
        gemm_update(k1 + jb, blk_end, blk_end, n, k1, jb);
      }
      if constexpr (std::is_same<F, c64>::value)
        lu_tc_trailing_update(M, n, ld, stride, nodes, k0, (int)nbo, w.tc_planes, w.status, num_sms, s);
    }
  }
  const size_t smem = sizeof(int32_t) * (size_t)n;
  if (smem > 48 * 1024)
    FEAST_CUDA_TRY(cudaFuncSetAttribute(build_perm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  build_perm_kernel<<<nodes, 256, smem, s>>>(ipiv, perm, n);
  FEAST_LAUNCH_CHECK();
}

template <typename F>
void lu_solve_batched(const F* M, int64_t n, int64_t ld, int64_t stride, int nodes,
                      F* Y, int64_t m, int64_t ystride, bool adjoint, cudaStream_t s, const SolvePlanes* sp,
                      int* status, int num_sms) {
  if (m <= 0) return;
  constexpr int TBK = SolveBlock<F>::value;
  dim3 gd((unsigned)cdiv(m, 8), nodes);
  bool tc = false;
  if constexpr (std::is_same<F, c64>::value) tc = sp != nullptr && (!adjoint || sp->row) && m <= sp->mpad;
  // SIMT block update Y[c_off + i] -= op(block of the factor at a) Y[k_off + j]
  auto update = [&](int64_t rows, int64_t k, const F* a, int opA, int64_t c_off, int64_t k_off) {
    GemmArgs g{};
    g.M = rows; g.N = m; g.K = k;
    g.A = a; g.opA = opA; g.lda = ld; g.strideA = stride;
    g.B = Y + k_off; g.ldb = n; g.strideB = ystride; g.opB = OP_N;
    g.C = Y + c_off; g.ldc = n; g.strideC = ystride;
    g.alpha = C1(-1.0); g.beta = C1(1.0); g.batch = nodes; g.ksplit = 1;
    gemm<F, F, F>(g, s);
  };
  auto diag = [&](int64_t r0, int bs, int mode) {
    trsm_diag_kernel<F, TBK><<<gd, 256, 0, s>>>(M, ld, stride, Y, n, m, ystride, r0, bs, mode);
    FEAST_LAUNCH_CHECK();
  };
  // forward (L, or U^H for the adjoint) over rows [b0, b1), top down; the
  // updates reach rows [r1, upd_end)
  auto forward_rows = [&](int64_t b0, int64_t b1, int64_t upd_end) {
    for (int64_t r0 = b0; r0 < b1; r0 += TBK) {
      const int bs = (int)std::min<int64_t>(TBK, b1 - r0);
      const int64_t r1 = r0 + bs;
      diag(r0, bs, adjoint ? 1 : 0);
      if (r1 < upd_end) {
        if (!adjoint) update(upd_end - r1, bs, M + r1 + r0 * ld, OP_N, r1, r0);
        else update(upd_end - r1, bs, M + r0 + r1 * ld, OP_C, r1, r0);
      }
    }
  };
  // backward (U, or L^H for the adjoint) over rows [b0, b1), bottom up; the
  // updates reach rows [upd_begin, r0)
  auto backward_rows = [&](int64_t b0, int64_t b1, int64_t upd_begin) {
    for (int64_t r0 = b0 + ((b1 - b0 - 1) / TBK) * TBK; r0 >= b0; r0 -= TBK) {
      const int bs = (int)std::min<int64_t>(TBK, b1 - r0);
      diag(r0, bs, adjoint ? 3 : 2);
      if (r0 > upd_begin) {
        if (!adjoint) update(r0 - upd_begin, bs, M + upd_begin + r0 * ld, OP_N, upd_begin, r0);
        else update(r0 - upd_begin, bs, M + r0 + upd_begin * ld, OP_C, upd_begin, r0);
      }
    }
  };
  if (!tc) {
    forward_rows(0, n, n);
    backward_rows(0, n, 0);
    return;
  }
  if constexpr (std::is_same<F, c64>::value) {
    // two levels on the tensor cores: each 256-row outer block solved in one
    // launch (trsm_outer_kernel: its diagonal blocks and the updates inside
    // it), then one rank-256 update of every row past it on the tensor cores.
    // The outer-block solve writes its block as bf16 planes into the outer
    // update's right-operand buffer: no separate split launches.
    const int64_t OB = kSolveOuter;
    const CgOperand Abase = cg_operand(adjoint ? sp->row : sp->col, sp->npad, kSolveBlock, nodes, sp->nblk,
                                       kSolveBlock);
    // Y[c_off .. c_off + rows) -= A_rows(blocks from R0 / 64, K = k) B(K offset kx)
    auto tc_update = [&](int64_t R0, int64_t kx, int64_t k, int64_t rows, int64_t c_off) {
      CgOperand B = cg_operand(sp->rhs, sp->mpad, kSolveOuter, nodes);
      B.base_x = (int)kx;
      CgOperand A = Abase;
      A.base_row = ((R0 + kx) / kSolveBlock) * A.slab_rows + c_off;
      cg_update(A, B, k, rows, m, Y + c_off, n, ystride, nodes, status, num_sms, s);
    };
    const dim3 go((unsigned)cdiv(m, kTrsmOuterWarps), nodes);
    auto solve_outer = [&](int64_t R0, int bs, int mode) {
      auto launch = [&](auto kernel) {
        FEAST_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrsmOuterSmem));
        kernel<<<go, kTrsmOuterThreads, kTrsmOuterSmem, s>>>(M, ld, stride, Y, n, m, ystride, R0, bs, sp->rhs,
                                                             sp->mpad);
      };
      switch (mode) {
        case 0: launch(trsm_outer_kernel<0>); break;
        case 1: launch(trsm_outer_kernel<1>); break;
        case 2: launch(trsm_outer_kernel<2>); break;
        default: launch(trsm_outer_kernel<3>); break;
      }
      FEAST_LAUNCH_CHECK();
    };
    for (int64_t R0 = 0; R0 < n; R0 += OB) {
      const int64_t R1 = std::min(n, R0 + OB);
      solve_outer(R0, (int)(R1 - R0), adjoint ? 1 : 0);
      if (R1 < n) tc_update(R0, 0, R1 - R0, n - R1, R1);
    }
    for (int64_t R0 = ((n - 1) / OB) * OB; R0 >= 0; R0 -= OB) {
      const int64_t R1 = std::min(n, R0 + OB);
      solve_outer(R0, (int)(R1 - R0), adjoint ? 3 : 2);
      if (R0 > 0) tc_update(R0, 0, R1 - R0, R0, 0);
    }
  }
}

size_t lu_tc_planes_bytes(int64_t n, int nodes) {
  return 2 * sizeof(uint16_t) * cg_planes_elems(cg_vpad(n), cg_kpad(kTcBlock), 1, nodes);
}

// A22 -= L21 U12 for the outer block of columns [k0, k0 + kb): L21 and U12
// split into bf16 planes, then the tensor-core update of every node
void lu_tc_trailing_update(c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, int64_t k0, int kb, void* planes,
                           int* status, int num_sms, cudaStream_t s) {
  const int64_t c1 = k0 + kb, rest = n - c1;
  if (rest <= 0) return;
  const int64_t vpad = cg_vpad(rest), kpad = cg_kpad(kb);
  uint16_t* Lp = (uint16_t*)planes;
  uint16_t* Up = Lp + cg_planes_elems(vpad, kpad, 1, nodes);
  // L21(i, k) = M[c1 + i, k0 + k]; U12(j, k) = M[k0 + k, c1 + j]
  cg_split(M, stride, 0, ld, c1, k0, true, false, rest, kb, (int)kpad, 1, vpad, kpad, nodes, Lp, s);
  cg_split(M, stride, 0, ld, k0, c1, false, false, rest, kb, (int)kpad, 1, vpad, kpad, nodes, Up, s);
  cg_update(cg_operand(Lp, vpad, kpad, nodes), cg_operand(Up, vpad, kpad, nodes), kb, rest, rest, M + c1 + c1 * ld,
            ld, stride, nodes, status, num_sms, s);
}

size_t solve_planes_bytes(int64_t n, int64_t m, int nodes, int entries, bool adjoint) {
  const int64_t nblk = cdiv(n, kSolveBlock);
  size_t b = sizeof(uint16_t) * cg_planes_elems(cg_vpad(n), kSolveBlock, nblk, nodes);
  b = (b + 255) & ~size_t(255);
  size_t tot = adjoint ? 2 * b : b;
  tot += sizeof(uint16_t) * cg_planes_elems(cg_vpad(m), kSolveOuter, 1, entries) + 256;
  return tot;
}

SolvePlanes solve_planes_carve(void* base, int64_t n, int64_t m, int nodes, int entries, bool adjoint) {
  SolvePlanes sp;
  sp.npad = cg_vpad(n);
  sp.nblk = cdiv(n, kSolveBlock);
  sp.mpad = cg_vpad(m);
  size_t b = sizeof(uint16_t) * cg_planes_elems(sp.npad, kSolveBlock, sp.nblk, nodes);
  b = (b + 255) & ~size_t(255);
  char* p = (char*)base;
  sp.col = (uint16_t*)p;
  p += b;
  if (adjoint) {
    sp.row = (uint16_t*)p;
    p += b;
  }
  sp.rhs = (uint16_t*)p;
  return sp;
}

void solve_planes_build(const c64* M, int64_t n, int64_t ld, int64_t stride, int nodes, const SolvePlanes& sp,
                        cudaStream_t s) {
  // column block b: element (i, k) = M[i, 64 b + k]
  cg_split(M, stride, (int64_t)kSolveBlock * ld, ld, 0, 0, true, false, n, n, kSolveBlock, sp.nblk, sp.npad,
           kSolveBlock, nodes, sp.col, s);
  // row block b, conjugated: element (j, k) = conj(M[64 b + k, j])
  if (sp.row)
    cg_split(M, stride, kSolveBlock, ld, 0, 0, false, true, n, n, kSolveBlock, sp.nblk, sp.npad, kSolveBlock, nodes,
             sp.row, s);
}

template <typename F, typename TB>
void permute_in(F* Y, int64_t ystride, const TB* B, int64_t ldb, int64_t bstride, int64_t n, int64_t m,
                const int32_t* perm, int nodes, bool adjoint, cudaStream_t s) {
  dim3 grid(grid1d(n * m), nodes);
  permute_in_kernel<F, TB><<<grid, 256, 0, s>>>(Y, ystride, B, ldb, bstride, n, m, perm, adjoint);
  FEAST_LAUNCH_CHECK();
}

template <typename F, typename TO>
void permute_out(TO* Out, int64_t ostride, const F* Y, int64_t ystride, int64_t n, int64_t m,
                 const int32_t* perm, int nodes, bool adjoint, bool accumulate, cudaStream_t s) {
  dim3 grid(grid1d(n * m), nodes);
  permute_out_kernel<F, TO><<<grid, 256, 0, s>>>(Out, ostride, Y, ystride, n, m, perm, adjoint, accumulate);
  FEAST_LAUNCH_CHECK();
}

void invert_perm(const int32_t* perm, int32_t* pinv, int64_t n, int nodes, cudaStream_t s) {
  dim3 grid(grid1d(n), nodes);
  invert_perm_kernel<<<grid, 256, 0, s>>>(perm, pinv, n);
  FEAST_LAUNCH_CHECK();
}

template <typename S, typename F>
void solve_accumulate(S* Xf, int64_t ldx, const c128* base, const F* Yn, const F* Ya, int64_t n, int64_t m, int nc,
                      const int32_t* pinv, const c128* w, cudaStream_t s) {
  solve_accumulate_kernel<S, F><<<grid1d(n * m), 256, 0, s>>>(Xf, ldx, base, Yn, Ya, n, m, nc, pinv, w);
  FEAST_LAUNCH_CHECK();
}

template void solve_accumulate<double, c64>(double*, int64_t, const c128*, const c64*, const c64*, int64_t, int64_t,
                                            int, const int32_t*, const c128*, cudaStream_t);
template void solve_accumulate<c128, c64>(c128*, int64_t, const c128*, const c64*, const c64*, int64_t, int64_t, int,
                                          const int32_t*, const c128*, cudaStream_t);
template void solve_accumulate<double, c128>(double*, int64_t, const c128*, const c128*, const c128*, int64_t,
                                             int64_t, int, const int32_t*, const c128*, cudaStream_t);
template void solve_accumulate<c128, c128>(c128*, int64_t, const c128*, const c128*, const c128*, int64_t, int64_t,
                                           int, const int32_t*, const c128*, cudaStream_t);

#define INST_F(F)                                                                                    \
  template void lu_factor_batched<F>(F*, int64_t, int64_t, int64_t, int, int32_t*, int32_t*,        \
                                     const PanelWork&, int, cudaStream_t);                          \
  template void lu_solve_batched<F>(const F*, int64_t, int64_t, int64_t, int, F*, int64_t, int64_t, \
                                    bool, cudaStream_t, const SolvePlanes*, int*, int);              \
  template void form_shifted<F, double>(F*, int64_t, int64_t, int64_t, int, const double*, int64_t, \
                                        const c128*, cudaStream_t);                                  \
  template void form_shifted<F, c128>(F*, int64_t, int64_t, int64_t, int, const c128*, int64_t,     \
                                      const c128*, cudaStream_t);                                    \
  template void permute_in<F, double>(F*, int64_t, const double*, int64_t, int64_t, int64_t, int64_t,        \
                                      const int32_t*, int, bool, cudaStream_t);                      \
  template void permute_in<F, c128>(F*, int64_t, const c128*, int64_t, int64_t, int64_t, int64_t,            \
                                    const int32_t*, int, bool, cudaStream_t);                        \
  template void permute_out<F, c128>(c128*, int64_t, const F*, int64_t, int64_t, int64_t,           \
                                     const int32_t*, int, bool, bool, cudaStream_t);

INST_F(c128)
INST_F(c64)

}  // namespace feast
