// df32.cuh -- double-float ("df32") arithmetic: a value is hi + lo with two
// float32 words, |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 issues FP32 FMAs ~57x faster than FP64 FMAs, so every place where
// the Krylov relations must hold to ~1e-13 (basis updates, the exact
// residual of the preconditioner solves, the true residual) uses these
// error-free transformations on the FP32 pipe instead of float64.
//
// The building blocks are Knuth's TwoSum, Dekker's FastTwoSum and the FMA
// form of TwoProduct (error-free: a + b = s + e, a * b = p + e exactly).
// Every operation below goes through the __f*_rn intrinsics so that the
// compiler can neither contract nor reassociate them.
#pragma once
#include <cuda_runtime.h>

namespace lt {

struct df { float hi, lo; };
struct cdf { df re, im; };

__device__ __forceinline__ df df_make(float a) { return {a, 0.f}; }

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ df df_add(df x, df y) {
  float s, e;
  two_sum(x.hi, y.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(x.lo, y.lo));
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ df df_sub(df x, df y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ df df_add_f(df x, float y) {
  float s, e;
  two_sum(x.hi, y, s, e);
  e = __fadd_rn(e, x.lo);
  df r;
  fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_mul(df x, df y) {
  float p, e;
  two_prod(x.hi, y.hi, p, e);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df df_mul_f(df x, float y) {
  float p, e;
  two_prod(x.hi, y, p, e);
  e = __fmaf_rn(x.lo, y, e);
  df r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// x / y with y a float: q = x/y to ~2^-46 relative
__device__ __forceinline__ df df_div_f(df x, float y) {
  float q1 = __fdiv_rn(x.hi, y);
  // remainder x - q1*y, exactly: x.hi - q1*y is exact via FMA, then add x.lo
  float r = __fmaf_rn(-q1, y, x.hi);
  r = __fadd_rn(r, x.lo);
  float q2 = __fdiv_rn(r, y);
  df out;
  fast_two_sum(q1, q2, out.hi, out.lo);
  return out;
}

// host/device split of a double into a df (exact to ~2^-48 relative)
__host__ __device__ __forceinline__ df df_from_double(double v) {
  float hi = (float)v;
  float lo = (float)(v - (double)hi);
  return {hi, lo};
}

__host__ __device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

// ---- complex helpers ------------------------------------------------------
__device__ __forceinline__ cdf cdf_add(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf cdf_sub(cdf a, cdf b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// complex times real df
__device__ __forceinline__ cdf cdf_mul_r(cdf a, df r) { return {df_mul(a.re, r), df_mul(a.im, r)}; }
// full complex product
__device__ __forceinline__ cdf cdf_mul(cdf a, cdf b) {
  return {df_sub(df_mul(a.re, b.re), df_mul(a.im, b.im)), df_add(df_mul(a.re, b.im), df_mul(a.im, b.re))};
}
// acc + a x + b y (a, b df; x, y float) with one renormalisation: the two products by TwoProduct,
// their high parts summed into acc.hi by TwoSum, every rounding error and the lo-word products
// gathered in the low word
__device__ __forceinline__ df df_fma2f(df acc, df a, float x, df b, float y) {
  float p1, e1, p2, e2, s1, t1, s2, t2;
  two_prod(a.hi, x, p1, e1);
  two_prod(b.hi, y, p2, e2);
  two_sum(acc.hi, p1, s1, t1);
  two_sum(s1, p2, s2, t2);
  float lo = __fadd_rn(acc.lo, __fadd_rn(t1, t2));
  lo = __fadd_rn(lo, __fadd_rn(e1, e2));
  lo = __fmaf_rn(a.lo, x, lo);
  lo = __fmaf_rn(b.lo, y, lo);
  df r;
  fast_two_sum(s2, lo, r.hi, r.lo);
  return r;
}
// s - v (cr + i ci) for a complex float coefficient, one renormalisation per component
__device__ __forceinline__ cdf cdf_sub_mul_cf(cdf s, cdf v, float cr, float ci) {
  return {df_fma2f(s.re, v.re, -cr, v.im, ci), df_fma2f(s.im, v.re, -ci, v.im, -cr)};
}
// a * c with c a complex float (exact float components)
__device__ __forceinline__ cdf cdf_mul_cf(cdf a, float cr, float ci) {
  return {df_sub(df_mul_f(a.re, cr), df_mul_f(a.im, ci)), df_add(df_mul_f(a.re, ci), df_mul_f(a.im, cr))};
}

// acc + u * y for df32 complex values, with one renormalisation per component: the two hi x hi
// products enter the running sum through TwoSum, their rounding errors and the hi x lo cross terms
// go to the low word.
__device__ __forceinline__ df df_fma2(df acc, df a, df b, df c, df d) {   // acc + a*b - c*d
  float p1, e1, p2, e2, s1, t1, s2, t2;
  two_prod(a.hi, b.hi, p1, e1);
  two_prod(c.hi, d.hi, p2, e2);
  two_sum(acc.hi, p1, s1, t1);
  two_sum(s1, -p2, s2, t2);
  float lo = __fadd_rn(acc.lo, __fadd_rn(t1, t2));
  lo = __fadd_rn(lo, __fsub_rn(e1, e2));
  lo = __fmaf_rn(a.hi, b.lo, lo);
  lo = __fmaf_rn(a.lo, b.hi, lo);
  lo = __fmaf_rn(-c.hi, d.lo, lo);
  lo = __fmaf_rn(-c.lo, d.hi, lo);
  df r;
  fast_two_sum(s2, lo, r.hi, r.lo);
  return r;
}
// acc + u y for df32 complex u and y
__device__ __forceinline__ cdf cdf_fma(cdf acc, cdf u, cdf y) {
  return {df_fma2(acc.re, u.re, y.re, u.im, y.im), df_fma2(acc.im, u.re, y.im, df_neg(u.im), y.re)};
}

}  // namespace lt
