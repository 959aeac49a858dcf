// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits. Built from the
// error-free transformations of Knuth (two-sum) and of Dekker with a fused
// multiply-add (two-product); the add, multiply and reciprocal follow the
// double-double algorithms of Hida, Li and Bailey (QD library, 2001), here on
// FP32 pairs. On this GPU an FP32 instruction costs ~1/64 of an FP64 one in
// pipe time, so a chain of a few hundred such operations (the post-Newtonian
// coefficients of the mixed path) is several times cheaper than in FP64.
// Every step uses explicitly rounded intrinsics, so no contraction or
// reassociation can change the error terms.
#pragma once

namespace sharpy {

struct DF {
  float hi, lo;
};

__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// |a| >= |b| (or a == 0)
__device__ __forceinline__ DF df_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

// Exact split of a double into hi + lo (the rounding error of lo, below 2^-48
// relative, is dropped). With a compile-time constant argument the
// conversions fold away.
__device__ __forceinline__ DF df_from(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ DF operator+(DF a, DF b) {
  DF s = df_two_sum(a.hi, b.hi);
  const DF t = df_two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ DF operator-(DF a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  DF p = df_two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo));
  return df_quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ DF operator+(double s, DF a) { return df_from(s) + a; }
__device__ __forceinline__ DF operator*(double s, DF a) { return df_from(s) * a; }

// 1 / a: FP32 quotient q1, remainder r = 1 - q1 a in double-float, second
// quotient q2 = r / a.hi, result q1 + q2.
__device__ __forceinline__ DF df_recip(DF a) {
  const float q1 = __fdiv_rn(1.0f, a.hi);
  const DF r = df_from(1.0) - DF{q1, 0.0f} * a;
  const float q2 = __fdiv_rn(r.hi, a.hi);
  return df_quick_two_sum(q1, q2);
}

}  // namespace sharpy
