// Double-single ("float-float") arithmetic: a value is the unevaluated sum hi + lo of two
// binary32 numbers with |lo| <= ulp(hi)/2, about 48 significant bits. Built from the
// error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the FMA-based
// exact product (a*b = p + e with e = fma(a, b, -p)). Used for the FP64-storage Wilson-
// clover operator when only a residual check needs it (relative accuracy ~1e-14, on the
// binary32 pipes, which on this part run about 60x faster than the FP64 ones).
//
// nvcc does not reassociate floating-point expressions; the transformations below rely on
// that, and only contract a product into an FMA where an explicit fmaf is written.
#pragma once
#include <cuda_runtime.h>

namespace dirac {

struct dsf {
  float hi, lo;
  dsf() = default;
  __device__ __forceinline__ dsf(float h, float l) : hi(h), lo(l) {}
  __device__ __forceinline__ dsf(int v) : hi((float)v), lo(0.f) {}
  // nearest double-single to a double: hi = fl32(v), lo = fl32(v - hi) (v - hi is exact)
  __device__ __forceinline__ explicit dsf(double v) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(v - (double)hi);
  }
  __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void ds_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void ds_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ dsf operator+(dsf x, dsf y) {
  float s, e;
  ds_two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  dsf r;
  ds_fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ dsf operator-(dsf x) { return dsf(-x.hi, -x.lo); }
__device__ __forceinline__ dsf operator-(dsf x, dsf y) { return x + (-y); }
__device__ __forceinline__ dsf operator*(dsf x, dsf y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);  // exact error of the leading product
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  dsf r;
  ds_fast_two_sum(p, e, r.hi, r.lo);
  return r;
}
// a * b + c for the stencils' fma on T. The standard overloads stay visible in this
// namespace, so fma on float / double arguments keeps resolving to them (exact match).
using ::fma;
__device__ __forceinline__ dsf fma(dsf a, dsf b, dsf c) { return a * b + c; }

}  // namespace dirac
