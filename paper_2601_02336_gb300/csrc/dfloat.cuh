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

// ln(1 + j/64), j < 64, as double-float pairs (hi, lo), from a 50-digit
// evaluation of the logarithm
static __constant__ float kLnTab[64][2] = {
    {0.000000000e+00f, 0.000000000e+00f}, {1.550418697e-02f, -4.370104834e-10f}, {3.077165782e-02f, 8.422373909e-10f},
    {4.580953717e-02f, -1.141023276e-09f}, {6.062462181e-02f, 7.905942394e-12f}, {7.522342354e-02f, -2.303004676e-09f},
    {8.961215615e-02f, 2.536961974e-09f}, {1.037967950e-01f, -1.328923194e-09f}, {1.177830324e-01f, 3.298690654e-09f},
    {1.315763593e-01f, -1.483283940e-09f}, {1.451820135e-01f, -3.667159909e-09f}, {1.586050242e-01f, 5.958079363e-09f},
    {1.718502641e-01f, -7.145759096e-09f}, {1.849223375e-01f, 9.619685049e-10f}, {1.978257447e-01f, -1.418195672e-09f},
    {2.105647624e-01f, 6.753452464e-09f}, {2.231435478e-01f, 3.540848503e-09f}, {2.355660647e-01f, 6.597381308e-09f},
    {2.478361577e-01f, 6.225023608e-09f}, {2.599575222e-01f, 2.283071732e-09f}, {2.719337046e-01f, 1.086900259e-08f},
    {2.837681770e-01f, -3.901825973e-09f}, {2.954642177e-01f, -4.768975437e-09f}, {3.070250452e-01f, -9.861566674e-09f},
    {3.184537292e-01f, 1.965855256e-09f}, {3.297532797e-01f, 6.686494025e-09f}, {3.409265876e-01f, -6.110413286e-10f},
    {3.519764245e-01f, -1.298464558e-09f}, {3.629055023e-01f, -8.629967851e-09f}, {3.737164140e-01f, -4.181178070e-09f},
    {3.844116926e-01f, 6.291008159e-09f}, {3.949938118e-01f, -3.604910370e-09f}, {4.054650962e-01f, 1.187288934e-08f},
    {4.158279002e-01f, -5.027569028e-09f}, {4.260843992e-01f, -3.912427715e-09f}, {4.362367690e-01f, -2.186034687e-09f},
    {4.462870955e-01f, 7.081697007e-09f}, {4.562374353e-01f, -1.859293719e-09f}, {4.660897255e-01f, 4.430214418e-09f},
    {4.758459032e-01f, 1.711776054e-09f}, {4.855078161e-01f, -2.945778899e-10f}, {4.950772524e-01f, 1.440985109e-08f},
    {5.045560002e-01f, 1.051969889e-08f}, {5.139457583e-01f, -7.240508637e-09f}, {5.232481360e-01f, 7.720998951e-09f},
    {5.324648023e-01f, -3.395695503e-09f}, {5.415973067e-01f, -2.429561796e-08f}, {5.506471395e-01f, -2.159659296e-08f},
    {5.596157908e-01f, -2.908540964e-09f}, {5.685047507e-01f, -1.537593874e-08f}, {5.773153901e-01f, -2.507519170e-08f},
    {5.860490203e-01f, 2.471320393e-08f}, {5.947071314e-01f, -2.363911022e-08f}, {6.032908559e-01f, -4.446467639e-09f},
    {6.118015647e-01f, -2.358745732e-08f}, {6.202403903e-01f, 1.945110739e-08f}, {6.286086440e-01f, 1.541373784e-08f},
    {6.369074583e-01f, 3.931710513e-09f}, {6.451379657e-01f, -4.305583889e-09f}, {6.533012986e-01f, -2.660557108e-08f},
    {6.613984704e-01f, 1.184360077e-08f}, {6.694306731e-01f, -1.917977599e-08f}, {6.773988008e-01f, 2.274189193e-08f},
    {6.853039861e-01f, 1.702637853e-08f}};
constexpr float kLn2Hi = 6.931471825e-01f, kLn2Lo = -1.904654212e-09f;  // ln 2 = hi + lo

// ln a for a double-float with 2^-126 <= a.hi < 2^127: a = 2^e (1 + j/64)(1 + t), j
// the top six mantissa bits of a.hi and 0 <= t < 1/64 (up to the lo part);
// ln a = e ln 2 + ln(1 + j/64) + t + t^2 P(t), P(t) = -1/2 + t/3 - t^2/4 +
// t^3/5 - t^4/6 (series truncated below 4e-14; P in FP32, whose error times
// t^2 stays below 2e-11). About 60 FP32 instructions.
__device__ __forceinline__ DF df_log(DF a) {
  const unsigned b = __float_as_uint(a.hi);
  const int e = (int)((b >> 23) & 0xffu) - 127;
  const int j = (int)((b >> 17) & 63u);
  const float m = __uint_as_float((b & 0x007fffffu) | 0x3f800000u);  // a.hi 2^-e, in [1, 2)
  const float c = __uint_as_float(0x3f800000u | ((unsigned)j << 17));  // 1 + j/64 exactly
  const float sc = __uint_as_float((unsigned)(127 - e) << 23);         // 2^-e
  // t = (a 2^-e - c) / c in double-float; m - c is exact
  const DF d = df_two_sum(__fsub_rn(m, c), __fmul_rn(a.lo, sc));
  const float q1 = __fdiv_rn(d.hi, c);
  const DF r = d - df_two_prod(q1, c);
  const DF t = df_quick_two_sum(q1, __fdiv_rn(r.hi, c));
  const float th = t.hi;
  const float p = __fmaf_rn(th, __fmaf_rn(th, __fmaf_rn(th, __fmaf_rn(th, -1.0f / 6.0f, 0.2f), -0.25f), 1.0f / 3.0f), -0.5f);
  const DF l1 = t + DF{__fmul_rn(__fmul_rn(th, th), p), 0.0f};
  const DF e2 = df_two_prod((float)e, kLn2Hi) + DF{__fmul_rn((float)e, kLn2Lo), 0.0f};
  return (DF{kLnTab[j][0], kLnTab[j][1]} + l1) + e2;
}

}  // namespace sharpy
