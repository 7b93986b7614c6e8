// Allocation-free variant of the Jacobi reduced eigensolver.
//
// Some callers cannot allocate device memory when they call in: services
// that reserve their whole device memory budget up front, or frameworks whose
// caching allocator already holds the free memory, so a fresh cudaMalloc
// would fail or break the budget.  feast_jacobi_eigh_noalloc serves them: it
// takes the caller's input and output buffers and keeps every piece of
// scratch (the working copy of H, the unsorted eigenvectors, the barrier
// counter, status words and rotation parameters of the cooperative kernel,
// the sort order) in one file-scope device array of fixed size.  It calls no
// cudaMalloc, no cudaFree and no allocating library routine.
//
// The array is static: every GPU that loads this library holds it until the
// process exits, and every call shares it, so the array keeps the last
// call's contents.  The parts that must start at zero (barrier counter,
// status, sweep counters) are cleared by each call.  Calls that overlap on
// the GPU (two streams, two host threads) race on the array.
//
// The call synchronises its stream and reads the eigenvalues back to the
// host to sort them, so it cannot run on a stream that is being captured
// into a CUDA graph: on a capturing stream it returns FEAST_ERR_ARG before
// touching the stream, and the capture stays valid.  It restores the
// caller's current device on every return.
#include <algorithm>
#include <mutex>

#include "../../include/feast.h"
#include "dense.cuh"

using namespace feast;

namespace {

// 2.25 MiB: a k x k complex working copy and k x k unsorted eigenvectors for
// k <= 256, the cooperative-kernel work area and the sort buffers.
constexpr int64_t kNoAllocMaxK = 256;
constexpr size_t kScratchBytes = (size_t)9 << 18;

static __device__ __align__(256) unsigned char g_jacobi_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Once per device, with that device current: the device address of the
// static array (in host code its name is only a host-side stand-in).
int setup_device(int device, void** ptr, int* sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_ptr[device] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_jacobi_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return FEAST_ERR_CUDA;
    }
    int s = 0;
    if (cudaDeviceGetAttribute(&s, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      cudaGetLastError();
      return FEAST_ERR_CUDA;
    }
    g_scratch_ptr[device] = p;
    g_num_sms[device] = s;
  }
  *ptr = g_scratch_ptr[device];
  *sms = g_num_sms[device];
  return FEAST_OK;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

template <typename S>
int run(void* scratch, int sms, int64_t k, const S* H, double* evals, S* V, int* sweeps, cudaStream_t st) {
  // scratch layout: [cooperative work][H copy k*k][V unsorted k*k][diag k][order k]
  char* p = (char*)scratch;
  const size_t coop = align256(coop_work_bytes(kNoAllocMaxK, sms));
  CoopWork cw = coop_work_carve(p, kNoAllocMaxK, sms);
  S* Hw = (S*)(p + coop);
  S* Vu = (S*)(p + coop + align256(sizeof(S) * k * k));
  double* d_diag = (double*)(p + coop + 2 * align256(sizeof(S) * k * k));
  int* d_ord = (int*)((char*)d_diag + align256(sizeof(double) * k));
  if ((char*)(d_ord + k) > p + kScratchBytes) return FEAST_ERR_ARG;
  try {
    copy_matrix<S>(Hw, k, H, k, k, k, st);
    jacobi_eigh<S>(Hw, k, k, Vu, k, 1e-15, cw, sms, st);
    get_diag<S>(Hw, k, k, d_diag, st);
    double ev[kNoAllocMaxK];
    int ord[kNoAllocMaxK];
    int status = 0, sw = 0;
    FEAST_CUDA_TRY(cudaMemcpyAsync(ev, d_diag, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    FEAST_CUDA_TRY(cudaMemcpyAsync(&status, cw.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    FEAST_CUDA_TRY(cudaMemcpyAsync(&sw, cw.info + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
    FEAST_CUDA_TRY(cudaStreamSynchronize(st));
    if (status == DEV_BARRIER_TIMEOUT) return FEAST_ERR_TIMEOUT;
    for (int64_t i = 0; i < k; ++i) ord[i] = (int)i;
    std::stable_sort(ord, ord + k, [&](int a, int b) { return ev[a] < ev[b]; });
    FEAST_CUDA_TRY(cudaMemcpyAsync(d_ord, ord, sizeof(int) * k, cudaMemcpyHostToDevice, st));
    gather_cols<S>(V, k, Vu, k, k, d_ord, k, nullptr, st);
    FEAST_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < k; ++i) evals[i] = ev[ord[i]];
    if (sweeps) *sweeps = sw;
    return FEAST_OK;
  } catch (const CudaFailure&) {
    return FEAST_ERR_CUDA;
  }
}

// restores the calling thread's current device when it goes out of scope
struct DeviceGuard {
  int prev = -1;
  DeviceGuard() {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" int feast_jacobi_eigh_noalloc(int device, void* stream, int dtype, int64_t k, const void* H,
                                         double* evals, void* V, int* sweeps) {
  if (!H || !evals || !V || k < 1 || k > kNoAllocMaxK || device < 0 || device >= kMaxDevices)
    return FEAST_ERR_ARG;
  if (dtype != FEAST_R64 && dtype != FEAST_C128) return FEAST_ERR_ARG;
  DeviceGuard guard;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return FEAST_ERR_CUDA;
  }
  // the call synchronises and reads back: refuse a capturing stream without
  // enqueuing anything on it
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return FEAST_ERR_ARG;
  }
  if (cap != cudaStreamCaptureStatusNone) return FEAST_ERR_ARG;
  void* scratch = nullptr;
  int sms = 0;
  if (int r = setup_device(device, &scratch, &sms)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if (dtype == FEAST_R64) return run<double>(scratch, sms, k, (const double*)H, evals, (double*)V, sweeps, st);
  return run<c128>(scratch, sms, k, (const c128*)H, evals, (c128*)V, sweeps, st);
}
