// Double-float arithmetic (internal): a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi) / 2, about 48 significant bits, computed
// on the FP32 pipes.  The operations are the error-free transformations of
// Knuth (TwoSum: the exact rounding error of a float sum) and of Dekker with a
// fused multiply-add (the exact error of a float product), combined as in
// Dekker's double-length arithmetic (1971) and the double-double routines of
// Hida, Li and Bailey (QD library), here with float parts.  Every float
// operation below goes through a round-to-nearest intrinsic so that the
// compiler does not contract it into a fused multiply-add, which would break
// the error terms.
//
// In memory a double-float is 8 bytes, (hi, lo); an array of them is an
// array of float pairs.
#pragma once

#include <cuda_runtime.h>

namespace fractal {

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h) : hi(h), lo(0.f) {}
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
};

// The double-float nearest a double (host side: kernel parameters).
inline dfloat dfloat_from_double(double x) {
  const float h = (float)x;
  return dfloat(h, (float)(x - (double)h));
}

#ifdef __CUDACC__
// s + e = a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ dfloat two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfloat(s, e);
}

// s + e = a + b exactly when |a| >= |b| (or a == 0).
__device__ __forceinline__ dfloat quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {
  dfloat s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }

// hi * hi exactly as p + e (fma(a, b, -p) is the product's rounding error),
// plus the cross terms.
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return quick_two_sum(p, e);
}

__device__ __forceinline__ dfloat fmat(dfloat a, dfloat b, dfloat c) { return a * b + c; }

// Loads and stores of double-float arrays (16 bytes = two values).
__device__ __forceinline__ void ld4(const dfloat* p, dfloat* v) {
  const float4 c0 = __ldg(reinterpret_cast<const float4*>(p));
  const float4 c1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = dfloat(c0.x, c0.y);
  v[1] = dfloat(c0.z, c0.w);
  v[2] = dfloat(c1.x, c1.y);
  v[3] = dfloat(c1.z, c1.w);
}
__device__ __forceinline__ void st4(dfloat* p, const dfloat* v) {
  reinterpret_cast<float4*>(p)[0] = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
  reinterpret_cast<float4*>(p)[1] = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
}
__device__ __forceinline__ dfloat ldg1(const dfloat* p) {
  const float2 c = __ldg(reinterpret_cast<const float2*>(p));
  return dfloat(c.x, c.y);
}
#endif

}  // namespace fractal
