// Batched solves of many independent interval problems (Sect. I: intervals
// are independent, so they can be solved in parallel with no communication)
// and the autotuner of the complex-FP32 GEMM route.
//
// A pool of host threads, each owning a CUDA stream and a library context,
// takes problems from a shared queue ordered largest first (n^2 m0 work),
// so the small problems of an uneven batch overlap on the GPU.  Every
// problem is an ordinary feast_interval_solve on that context.
//
// Autotuner: for a mixed-precision request the GEMM updates of the shifted
// LU and solves can run on the tensor cores or on the SIMT pipes; which is
// faster depends on n (the tensor-core tiles are 128 x 128).  The first time
// a size bucket (n rounded up to 256) is met, both routes factor a probe
// matrix of that size at two nodes and solve one block of 64 right-hand
// sides, timed with CUDA events; the faster route is cached for the process.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/feast.h"
#include "common.cuh"

namespace {

std::mutex g_tune_mutex;
std::map<std::pair<int, int64_t>, int> g_route;  // (device, bucket) -> FEAST_PREC_*

__global__ void probe_matrix_kernel(double* A, int64_t n) {
  // a symmetric matrix with entries in [-1, 1] and a dominant diagonal
  const int64_t total = n * n;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t % n, j = t / n;
    const int64_t a = i < j ? i : j, b = i < j ? j : i;
    unsigned long long h = (unsigned long long)(a * 2654435761ull) ^ (unsigned long long)(b * 40503ull + 12345ull);
    h ^= h >> 33;
    h *= 0xff51afd7ed558ccdull;
    h ^= h >> 33;
    A[t] = (double)(h & 0xFFFFFF) / (double)0x800000 - 1.0 + (i == j ? 4.0 : 0.0);
  }
}

double time_route(feast_ctx* ctx, cudaStream_t st, const double* A, int64_t n, int prec, void* LU, int32_t* perm,
                  void* B, void* Y) {
  const double z[4] = {0.3, 0.5, -0.2, 0.4};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, st);
  int r = feast_shifted_lu(ctx, A, FEAST_R64, n, n, z, 2, prec, LU, perm);
  if (r == FEAST_OK) r = feast_shifted_solve(ctx, LU, perm, n, 2, prec, 0, B, 64, Y);
  cudaEventRecord(e1, st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r == FEAST_OK ? ms : 1e30;
}

// FEAST_PREC_MIXED or FEAST_PREC_MIXED_SIMT for problems of size n
int tuned_route(int device, feast_ctx* ctx, cudaStream_t st, int64_t n) {
  const int64_t bucket = ((n + 255) / 256) * 256;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_route.find({device, bucket});
    if (it != g_route.end()) return it->second;
  }
  int route = FEAST_PREC_MIXED;
  double* A = nullptr;
  void *LU = nullptr, *B = nullptr, *Y = nullptr;
  int32_t* perm = nullptr;
  const int64_t m = 64;
  bool ok = cudaMalloc(&A, sizeof(double) * bucket * bucket) == cudaSuccess &&
            cudaMalloc(&LU, 16 * (size_t)bucket * bucket * 2) == cudaSuccess &&
            cudaMalloc(&perm, sizeof(int32_t) * bucket * 2) == cudaSuccess &&
            cudaMalloc(&B, 16 * (size_t)bucket * m) == cudaSuccess &&
            cudaMalloc(&Y, 16 * (size_t)bucket * m * 2) == cudaSuccess;
  if (ok) {
    probe_matrix_kernel<<<1024, 256, 0, st>>>(A, bucket);
    feast::note_launch();
    cudaMemsetAsync(B, 0, 16 * (size_t)bucket * m, st);
    // warm both routes once, then time them
    time_route(ctx, st, A, bucket, FEAST_PREC_MIXED, LU, perm, B, Y);
    time_route(ctx, st, A, bucket, FEAST_PREC_MIXED_SIMT, LU, perm, B, Y);
    const double t_tc = time_route(ctx, st, A, bucket, FEAST_PREC_MIXED, LU, perm, B, Y);
    const double t_simt = time_route(ctx, st, A, bucket, FEAST_PREC_MIXED_SIMT, LU, perm, B, Y);
    route = t_simt < t_tc ? FEAST_PREC_MIXED_SIMT : FEAST_PREC_MIXED;
  }
  cudaGetLastError();
  cudaFree(A);
  cudaFree(LU);
  cudaFree(perm);
  cudaFree(B);
  cudaFree(Y);
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  g_route[{device, bucket}] = route;
  return route;
}

}  // namespace

extern "C" int feast_interval_solve_batch(int device, int nproblems, feast_problem* probs, const feast_opts* opts,
                                          int workers, int autotune) {
  if (nproblems < 0 || (nproblems > 0 && !probs) || workers < 1 || workers > 64) return FEAST_ERR_ARG;
  feast_opts o;
  if (opts) o = *opts;
  else feast_opts_default(&o);
  if (o.x0) return FEAST_ERR_ARG;
  if (nproblems == 0) return FEAST_OK;
  // largest first: n^2 m0 work
  std::vector<int> order(nproblems);
  for (int i = 0; i < nproblems; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (double)probs[a].n * probs[a].n * probs[a].m0 > (double)probs[b].n * probs[b].n * probs[b].m0;
  });
  std::atomic<int> next{0};
  std::atomic<int> failed{0};
  const int nw = std::min(workers, nproblems);
  auto work = [&]() {
    if (cudaSetDevice(device) != cudaSuccess) {
      cudaGetLastError();
      failed.store(FEAST_ERR_CUDA);
      return;
    }
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      failed.store(FEAST_ERR_CUDA);
      return;
    }
    feast_ctx* ctx = nullptr;
    if (feast_init(&ctx, device, st) != FEAST_OK) {
      cudaStreamDestroy(st);
      failed.store(FEAST_ERR_CUDA);
      return;
    }
    while (true) {
      const int k = next.fetch_add(1);
      if (k >= nproblems) break;
      feast_problem& p = probs[order[k]];
      feast_opts po = o;
      if (autotune && po.prec != FEAST_PREC_F64) po.prec = tuned_route(device, ctx, st, p.n);
      p.route = po.prec;
      const auto t0 = std::chrono::steady_clock::now();
      p.status = feast_interval_solve(ctx, p.A, p.dtype, p.n, p.lda, p.lmin, p.lmax, p.m0, p.n_c, p.tol, &po,
                                      p.evals, p.evecs, p.res, &p.m_found, &p.iterations, nullptr);
      p.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      if (p.status < 0) {
        int expect = 0;
        failed.compare_exchange_strong(expect, p.status);
      }
    }
    feast_finalize(ctx);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  for (int w = 0; w < nw; ++w) pool.emplace_back(work);
  for (auto& t : pool) t.join();
  return failed.load();
}
