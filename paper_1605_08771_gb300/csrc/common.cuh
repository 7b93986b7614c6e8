// Shared device helpers of the FEAST GB300 library: complex scalar type,
// launch/error macros, and the bounded inter-CTA barrier used by the
// cooperative kernels (panel LU, Cholesky, Jacobi).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <type_traits>

namespace feast {

// ---------------------------------------------------------------------------
// complex scalar (interleaved re, im; layout-compatible with double2/float2 and
// with C99 / numpy complex arrays)
// ---------------------------------------------------------------------------
template <typename T>
struct __align__(2 * sizeof(T)) Cx {
  T re, im;
};

using c64 = Cx<float>;
using c128 = Cx<double>;

template <typename T> struct is_cx : std::false_type {};
template <typename T> struct is_cx<Cx<T>> : std::true_type {};
template <typename T> struct real_of { using type = T; };
template <typename T> struct real_of<Cx<T>> { using type = T; };
template <typename T> using real_t = typename real_of<T>::type;

template <typename T> __host__ __device__ __forceinline__ Cx<T> cx(T re, T im) { return Cx<T>{re, im}; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator-(Cx<T> a) { return {-a.re, -a.im}; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator*(T a, Cx<T> b) { return {a * b.re, a * b.im}; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> operator*(Cx<T> a, T b) { return {a.re * b, a.im * b}; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> conj(Cx<T> a) { return {a.re, -a.im}; }
template <typename T> __host__ __device__ __forceinline__ T conj(T a) { return a; }
template <typename T> __host__ __device__ __forceinline__ T abs2(Cx<T> a) { return a.re * a.re + a.im * a.im; }
template <typename T> __host__ __device__ __forceinline__ T abs2(T a) { return a * a; }
template <typename T> __host__ __device__ __forceinline__ T real_part(Cx<T> a) { return a.re; }
template <typename T> __host__ __device__ __forceinline__ T real_part(T a) { return a; }
template <typename T> __host__ __device__ __forceinline__ Cx<T> recip(Cx<T> a) {
  // 1/a = conj(a)/|a|^2 with a power-of-two rescale against overflow
  T s = fmax(fabs(a.re), fabs(a.im));
  if (s == T(0)) return {T(0), T(0)};
  int e; frexp(s, &e);
  T ar = ldexp(a.re, -e), ai = ldexp(a.im, -e);
  T d = ar * ar + ai * ai;
  return {ldexp(ar / d, -e), ldexp(-ai / d, -e)};
}
template <typename T> __host__ __device__ __forceinline__ T recip(T a) { return T(1) / a; }

// zero / one / conversions
template <typename T> struct num {
  static __host__ __device__ __forceinline__ T zero() { return T(0); }
};
template <typename T> struct num<Cx<T>> {
  static __host__ __device__ __forceinline__ Cx<T> zero() { return {T(0), T(0)}; }
};

template <typename To, typename From> struct conv;
template <typename T, typename U> struct conv<Cx<T>, Cx<U>> {
  static __host__ __device__ __forceinline__ Cx<T> f(Cx<U> a) { return {T(a.re), T(a.im)}; }
};
template <typename T, typename U> struct conv<Cx<T>, U> {
  static __host__ __device__ __forceinline__ Cx<T> f(U a) { return {T(a), T(0)}; }
};
template <typename T, typename U> struct conv<T, Cx<U>> {  // real <- complex keeps the real part
  static __host__ __device__ __forceinline__ T f(Cx<U> a) { return T(a.re); }
};
template <typename T, typename U> struct conv {
  static __host__ __device__ __forceinline__ T f(U a) { return T(a); }
};
template <typename To, typename From> __host__ __device__ __forceinline__ To cvt(From a) { return conv<To, From>::f(a); }

// acc += a * b for every combination used (real*real, real*complex, complex*complex)
template <typename T> __device__ __forceinline__ void mac(T& acc, T a, T b) { acc = fma(a, b, acc); }
template <typename T> __device__ __forceinline__ void mac(Cx<T>& acc, Cx<T> a, Cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
template <typename T> __device__ __forceinline__ void mac(Cx<T>& acc, T a, Cx<T> b) {
  acc.re = fma(a, b.re, acc.re);
  acc.im = fma(a, b.im, acc.im);
}
template <typename T> __device__ __forceinline__ void mac(Cx<T>& acc, Cx<T> a, T b) {
  acc.re = fma(a.re, b, acc.re);
  acc.im = fma(a.im, b, acc.im);
}

template <typename T> __device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
template <typename T> __device__ __forceinline__ Cx<T> shfl(Cx<T> v, int src) {
  return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
// Device-side status words (one int each) that kernels set instead of trapping.
enum DeviceStatus : int {
  DEV_OK = 0,
  DEV_BARRIER_TIMEOUT = 1,   // a bounded inter-CTA wait gave up
  DEV_ZERO_PIVOT = 2,        // LU met an exactly zero pivot column
  DEV_CHOL_BREAKDOWN = 3,    // non-positive or non-finite Cholesky pivot
  DEV_NONFINITE = 4,
};

#define FEAST_CUDA_TRY(expr)                                                         \
  do {                                                                              \
    cudaError_t _e = (expr);                                                        \
    if (_e != cudaSuccess) {                                                        \
      if (getenv("FEAST_LOG")) fprintf(stderr, "[feast] %s:%d %s -> %s\n", __FILE__, __LINE__, #expr, cudaGetErrorString(_e)); \
      throw ::feast::CudaFailure(_e);                                               \
    }                                                                               \
  } while (0)

// every kernel launch of the library passes through here (the count is
// reported by feast_kernel_launches())
void note_launch();
unsigned long long launch_count();
#define FEAST_LAUNCH_CHECK()                \
  do {                                      \
    ::feast::note_launch();                 \
    FEAST_CUDA_TRY(cudaGetLastError());     \
  } while (0)

// CUDA-event timing of selected kernels over one solve: enable, bracket each
// launch of the kernel class, then read the summed device time, work units
// and launch count.  Classes: the FP64-accurate GEMM of the refinement
// (work = real multiply-adds), the complex-FP32 SIMT GEMM of the LU and the
// triangular solves and its tensor-core counterpart (work = real flops, 8
// per complex multiply-add).
enum TimerClass : int { TIMER_REFINE_GEMM = 0, TIMER_CGEMM = 1, TIMER_TCGEMM = 2, TIMER_CLASSES = 3 };
void kernel_timer_begin();
void kernel_timer_end(int cls, double* ms, double* work, int* launches);
void kernel_timer_launch_begin(int cls, cudaStream_t s);
void kernel_timer_launch_end(int cls, cudaStream_t s, double work);

struct CudaFailure {
  cudaError_t err;
  explicit CudaFailure(cudaError_t e) : err(e) {}
};

// ---------------------------------------------------------------------------
// bounded group barrier among the CTAs of one cooperative launch (or a subset
// of them sharing a counter).  Every wait has a wall-clock limit; on expiry the
// waiting CTA records DEV_BARRIER_TIMEOUT in *status and all CTAs leave their
// loops at the next barrier.  Returns false when the kernel must stop.
// ---------------------------------------------------------------------------
constexpr unsigned long long kBarrierLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool group_barrier(unsigned* counter, unsigned target, int* status) {
  __shared__ int s_go;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    int go = 1;
    unsigned long long t0 = globaltimer_ns();
    while (true) {
      unsigned v = ld_acquire_u32(counter);
      if ((int)(v - target) >= 0) break;
      if (*(volatile int*)status != DEV_OK) { go = 0; break; }
      if (globaltimer_ns() - t0 > kBarrierLimitNs) {
        atomicCAS(status, DEV_OK, DEV_BARRIER_TIMEOUT);
        go = 0;
        break;
      }
      __nanosleep(20);
    }
    __threadfence();
    if (*(volatile int*)status != DEV_OK) go = 0;
    s_go = go;
  }
  __syncthreads();
  return s_go != 0;
}

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

}  // namespace feast
