// Device number types for the nested Krylov sign function.
//
// Three arithmetic modes share one kernel source:
//   PrecF64  - double vectors, double links, double arithmetic;
//   PrecF32  - float vectors, float links, float stencil; reductions in double-float;
//   PrecDF64 - vectors and links as unevaluated float pairs (hi + lo), error-free
//              float arithmetic. The pair arithmetic is built from the exact
//              transformations TwoSum (Knuth, TAOCP vol. 2, 4.2.2), Fast2Sum (Dekker
//              1971) and the FMA product error p = a*b, e = fma(a, b, -p) (exact in
//              IEEE arithmetic). Rounded operations inside them use the __f*_rn
//              intrinsics so the compiler never contracts them into FMAs.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ov {

// ----------------------------------------------------------------- double-float
struct df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  df64 s = df_two_sum(a.hi, b.hi);
  float lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return df_fast_two_sum(s.hi, lo);
}
__device__ __forceinline__ df64 operator-(df64 a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
// pair times a single float (links are exact floats)
__device__ __forceinline__ df64 operator*(df64 a, float u) {
  float p = __fmul_rn(a.hi, u);
  float e = __fmaf_rn(a.hi, u, -p);
  e = __fmaf_rn(a.lo, u, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 df_half(df64 a) { return {a.hi * 0.5f, a.lo * 0.5f}; }  // exact
__device__ __forceinline__ df64 df_from_double(double d) {
  float hi = __double2float_rn(d);
  float lo = __double2float_rn(d - (double)hi);
  return {hi, lo};
}
__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }
__host__ __device__ __forceinline__ df64 df_zero() { return {0.f, 0.f}; }

// ----------------------------------------------------------------- scalar helpers
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(float a) { return (double)a; }
__device__ __forceinline__ double to_double(df64 a) { return df_to_double(a); }

template <class R> __device__ __forceinline__ R from_double(double d);
template <> __device__ __forceinline__ double from_double<double>(double d) { return d; }
template <> __device__ __forceinline__ float from_double<float>(double d) { return (float)d; }
template <> __device__ __forceinline__ df64 from_double<df64>(double d) { return df_from_double(d); }

template <class R> __device__ __forceinline__ R rzero();
template <> __device__ __forceinline__ double rzero<double>() { return 0.0; }
template <> __device__ __forceinline__ float rzero<float>() { return 0.f; }
template <> __device__ __forceinline__ df64 rzero<df64>() { return df_zero(); }

__device__ __forceinline__ double rhalf(double a) { return 0.5 * a; }
__device__ __forceinline__ float rhalf(float a) { return 0.5f * a; }
__device__ __forceinline__ df64 rhalf(df64 a) { return df_half(a); }

// vector element times link element
__device__ __forceinline__ double lmul(double v, double u) { return v * u; }
__device__ __forceinline__ float lmul(float v, float u) { return v * u; }
__device__ __forceinline__ df64 lmul(df64 v, float u) { return v * u; }

// ----------------------------------------------------------------- complex
template <class R>
struct cx {
  R re, im;
};

template <class R> __device__ __forceinline__ cx<R> czero() { return {rzero<R>(), rzero<R>()}; }
template <class R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <class R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <class R> __device__ __forceinline__ cx<R> operator-(cx<R> a) { return {-a.re, -a.im}; }
// multiply by i and -i
template <class R> __device__ __forceinline__ cx<R> ci(cx<R> a) { return {-a.im, a.re}; }
template <class R> __device__ __forceinline__ cx<R> cmi(cx<R> a) { return {a.im, -a.re}; }
template <class R> __device__ __forceinline__ cx<R> chalf(cx<R> a) { return {rhalf(a.re), rhalf(a.im)}; }
template <class R> __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return {a.re * s, a.im * s}; }
// full complex product
template <class R> __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class R> __device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
// link (type L) times vector element (type R): u * v and conj(u) * v
template <class R, class L> __device__ __forceinline__ cx<R> lcmul(cx<L> u, cx<R> v) {
  return {lmul(v.re, u.re) - lmul(v.im, u.im), lmul(v.im, u.re) + lmul(v.re, u.im)};
}
template <class R, class L> __device__ __forceinline__ cx<R> lcmulc(cx<L> u, cx<R> v) {
  return {lmul(v.re, u.re) + lmul(v.im, u.im), lmul(v.im, u.re) - lmul(v.re, u.im)};
}

// ----------------------------------------------------------------- precision policies
// vec_t: storage of one complex vector element; link_t: storage of one complex link
// element; R: arithmetic of the stencil; L: link arithmetic; A: per-thread accumulator of
// dot products (converted to double at warp level).
struct PrecF64 {
  using R = double;
  using L = double;
  using A = double;
  using vec_t = double2;
  using link_t = double2;
  static constexpr int id = 0;
};
struct PrecF32 {
  using R = float;
  using L = float;
  using A = df64;
  using vec_t = float2;
  using link_t = float2;
  static constexpr int id = 1;
};
struct PrecDF64 {
  using R = df64;
  using L = float;
  using A = df64;
  using vec_t = float4;  // (re.hi, re.lo, im.hi, im.lo)
  using link_t = float2;
  static constexpr int id = 2;
};
// Relaxed steps of the double-float mode: the same storage, recurrence and reductions as
// PrecDF64, with the hopping sum in float arithmetic on the high words of the vector and
// the links (a matvec error of a few 2^-24, admitted where the step's weight in the result
// is small).
struct PrecDF64R {
  using R = df64;
  using L = float;
  using A = df64;
  using vec_t = float4;
  using link_t = float2;
  static constexpr int id = 3;
};

__device__ __forceinline__ cx<double> ld_vec(const double2* p) {
  double2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ cx<float> ld_vec(const float2* p) {
  float2 v = *p;
  return {v.x, v.y};
}
__device__ __forceinline__ cx<df64> ld_vec(const float4* p) {
  float4 v = *p;
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ void st_vec(double2* p, cx<double> a) { *p = make_double2(a.re, a.im); }
__device__ __forceinline__ void st_vec(float2* p, cx<float> a) { *p = make_float2(a.re, a.im); }
__device__ __forceinline__ void st_vec(float4* p, cx<df64> a) {
  *p = make_float4(a.re.hi, a.re.lo, a.im.hi, a.im.lo);
}
__device__ __forceinline__ cx<double> ld_link(const double2* p) {
  double2 v = __ldg(p);
  return {v.x, v.y};
}
__device__ __forceinline__ cx<float> ld_link(const float2* p) {
  float2 v = __ldg(p);
  return {v.x, v.y};
}

// accumulate conj(a) * b into a dot-product accumulator of type A
__device__ __forceinline__ void acc_dot(cx<double>& acc, cx<double> a, cx<double> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
__device__ __forceinline__ df64 df_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
// a + x1 y1 + x2 y2 in float pairs: both products exact (p = x.hi*y.hi, e = fma(x.hi, y.hi,
// -p), cross terms folded into e), the two high words added to a.hi by TwoSum, every low
// word summed once, one renormalisation
__device__ __forceinline__ df64 df_axpy2(df64 a, df64 x1, df64 y1, df64 x2, df64 y2) {
  const float p1 = __fmul_rn(x1.hi, y1.hi);
  float e1 = __fmaf_rn(x1.hi, y1.hi, -p1);
  e1 = __fmaf_rn(x1.hi, y1.lo, e1);
  e1 = __fmaf_rn(x1.lo, y1.hi, e1);
  const float p2 = __fmul_rn(x2.hi, y2.hi);
  float e2 = __fmaf_rn(x2.hi, y2.hi, -p2);
  e2 = __fmaf_rn(x2.hi, y2.lo, e2);
  e2 = __fmaf_rn(x2.lo, y2.hi, e2);
  const df64 s = df_two_sum(a.hi, p1);
  const df64 t = df_two_sum(s.hi, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(a.lo, s.lo), t.lo), __fadd_rn(e1, e2));
  return df_fast_two_sum(t.hi, lo);
}
// x1 y1 + x2 y2 + x3 y3 + x4 y4 in float pairs: every product exact as (p, e), the four
// high words summed by TwoSum, every low word once, one renormalisation
__device__ __forceinline__ df64 df_dot4(df64 x1, df64 y1, df64 x2, df64 y2, df64 x3, df64 y3, df64 x4, df64 y4) {
  const float p1 = __fmul_rn(x1.hi, y1.hi), p2 = __fmul_rn(x2.hi, y2.hi);
  const float p3 = __fmul_rn(x3.hi, y3.hi), p4 = __fmul_rn(x4.hi, y4.hi);
  float e1 = __fmaf_rn(x1.hi, y1.hi, -p1), e2 = __fmaf_rn(x2.hi, y2.hi, -p2);
  float e3 = __fmaf_rn(x3.hi, y3.hi, -p3), e4 = __fmaf_rn(x4.hi, y4.hi, -p4);
  e1 = __fmaf_rn(x1.lo, y1.hi, __fmaf_rn(x1.hi, y1.lo, e1));
  e2 = __fmaf_rn(x2.lo, y2.hi, __fmaf_rn(x2.hi, y2.lo, e2));
  e3 = __fmaf_rn(x3.lo, y3.hi, __fmaf_rn(x3.hi, y3.lo, e3));
  e4 = __fmaf_rn(x4.lo, y4.hi, __fmaf_rn(x4.hi, y4.lo, e4));
  const df64 s = df_two_sum(p1, p2);
  const df64 t = df_two_sum(s.hi, p3);
  const df64 u = df_two_sum(t.hi, p4);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(s.lo, t.lo), u.lo), __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, e4)));
  return df_fast_two_sum(u.hi, lo);
}
// a + x y
__device__ __forceinline__ df64 df_axpy1(df64 a, df64 x, df64 y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  const df64 s = df_two_sum(a.hi, p);
  return df_fast_two_sum(s.hi, __fadd_rn(__fadd_rn(a.lo, s.lo), e));
}
// the same with float factors
__device__ __forceinline__ df64 df_axpy2(df64 a, float x1, float y1, float x2, float y2) {
  const float p1 = __fmul_rn(x1, y1);
  const float e1 = __fmaf_rn(x1, y1, -p1);
  const float p2 = __fmul_rn(x2, y2);
  const float e2 = __fmaf_rn(x2, y2, -p2);
  const df64 s = df_two_sum(a.hi, p1);
  const df64 t = df_two_sum(s.hi, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(a.lo, s.lo), t.lo), __fadd_rn(e1, e2));
  return df_fast_two_sum(t.hi, lo);
}
// acc += conj(a) b
__device__ __forceinline__ void acc_dot(cx<df64>& acc, cx<float> a, cx<float> b) {
  acc.re = df_axpy2(acc.re, a.re, b.re, a.im, b.im);
  acc.im = df_axpy2(acc.im, a.re, b.im, -a.im, b.re);
}
__device__ __forceinline__ void acc_dot(cx<df64>& acc, cx<df64> a, cx<df64> b) {
  acc.re = df_axpy2(acc.re, a.re, b.re, a.im, b.im);
  acc.im = df_axpy2(acc.im, a.re, b.im, -a.im, b.re);
}
__device__ __forceinline__ cx<double> acc_to_double(cx<double> a) { return a; }
__device__ __forceinline__ cx<double> acc_to_double(cx<df64> a) {
  return {df_to_double(a.re), df_to_double(a.im)};
}

// warp-level sum of a double-float (pairs travel through two shuffles)
__device__ __forceinline__ df64 warp_sum(df64 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    df64 w;
    w.hi = __shfl_xor_sync(0xffffffffu, v.hi, o);
    w.lo = __shfl_xor_sync(0xffffffffu, v.lo, o);
    v = v + w;
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace ov
