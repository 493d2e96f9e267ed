// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// binary32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits
// (relative rounding ~2^-44 per operation).  Built from the error-free
// transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2) and FMA-based
// TwoProduct (the product's rounding error is fma(a, b, -a*b) exactly), as in
// the double-double / double-float libraries of Dekker (1971) and Hida, Li
// and Bailey (2001).  GB300 runs binary32 FMAs at ~64x its binary64 rate, so
// the mixed form's slice recursion runs here instead of in binary64.
#pragma once

#include <cuda_runtime.h>

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr dfl(float v) : hi(v), lo(0.f) {}
  // binary64 -> double-float: the leading 48 bits (the split is exact)
  __host__ __device__ explicit dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

// The round-to-nearest intrinsics keep the compiler from contracting these
// steps into FMAs, which would break the error-free transformations.

// s + e = a + b exactly (TwoSum, no ordering assumption)
__device__ __forceinline__ void dfl_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// p + e = a * b exactly
__device__ __forceinline__ void dfl_two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// renormalise s + e with |e| small against s (FastTwoSum)
__device__ __forceinline__ dfl dfl_fast(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfl(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  float s, e;
  dfl_two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return dfl_fast(s, e);
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }

__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  float p, e;
  dfl_two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return dfl_fast(p, e);
}

// c + a b with one renormalisation
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) {
  float p, e, s, e2;
  dfl_two_prod(a.hi, b.hi, p, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  dfl_two_sum(p, c.hi, s, e2);
  e2 = __fadd_rn(e2, __fadd_rn(c.lo, e));
  return dfl_fast(s, e2);
}

// a / b: the float quotient, corrected once by the remainder a - q b
__device__ __forceinline__ dfl operator/(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfl r = a - b * dfl(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return dfl_fast(q1, q2);
}

__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
__device__ __forceinline__ dfl& operator-=(dfl& a, dfl b) { return a = a - b; }

__device__ __forceinline__ dfl shfl_xor_any(dfl v, int off) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off));
}
__device__ __forceinline__ double shfl_xor_any(double v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
__device__ __forceinline__ float shfl_xor_any(float v, int off) { return __shfl_xor_sync(0xffffffffu, v, off); }
