// Double-float ("df") scalars for FP64-accurate arithmetic on the FP32 pipes
// (FP64 runs at about 1/64 of the FP32 rate on this GPU).  A value is the
// unevaluated sum hi + lo of two floats, about 48 significant bits (Dekker,
// "A floating-point technique for extending the available precision", 1971;
// Knuth's TwoSum).  Products use the FMA form of TwoProduct; sums use the
// short ("sloppy") double-float addition, whose error is within a few units
// of 2^-48 of the larger operand, the scale the kernels that use it need.
#pragma once
#include "common.cuh"

namespace feast {

struct dfr {
  float hi, lo;
  dfr() = default;
  __host__ __device__ __forceinline__ dfr(float h, float l) : hi(h), lo(l) {}
  // from FP64 (one FP64 subtraction)
  __host__ __device__ __forceinline__ dfr(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
  __host__ __device__ __forceinline__ dfr(int x) : hi((float)x), lo(0.0f) {}
  __host__ __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
};
using dfc = Cx<dfr>;

__device__ __forceinline__ dfr df_quick_two_sum(float a, float b) {
  const float s = a + b;
  return dfr(s, b - (s - a));
}
__device__ __forceinline__ dfr df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfr(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
  dfr s = df_two_sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return df_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfr operator-(dfr a) { return dfr(-a.hi, -a.lo); }
__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}

}  // namespace feast
