// Double-float arithmetic: a value is the unevaluated sum h + l of two FP32 numbers.
//
// Used by the double-float form, which computes Eq. (1)/(3) to FP64-level accuracy on the
// FP32 pipe (64x the FP64 rate on GB300). The building blocks are the classical
// error-free transformations:
//   * TwoSum (Knuth): s = fl(a + b) and t with s + t == a + b exactly, for any a, b;
//   * the FMA product error: p = fl(a * b) and e = fma(a, b, -p) with p + e == a * b exactly.
// Products keep the three leading partial products (h*h exactly, h*l and l*h rounded) and
// drop l*l (below 2^-48 relative). Accumulators are normalised lazily: the running sum is
// kept in h by TwoSum and every rounding error collects in l; df_norm restores
// |l| <= ulp(h)/2, so a caller renormalises before l has grown by more than a few ulp(h).
// Intrinsics (__fadd_rn, __fmul_rn) keep the compiler from contracting or reordering the
// sequences, which would break their exactness.
#pragma once

namespace bb {

struct dfloat {
  float h, l;
};

__device__ __forceinline__ dfloat df_zero() { return dfloat{0.f, 0.f}; }

// s + t == a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  t = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// Normalise: |l| <= ulp(h) / 2 afterwards, h + l unchanged.
__device__ __forceinline__ dfloat df_norm(dfloat a) {
  float s, t;
  two_sum(a.h, a.l, s, t);
  return dfloat{s, t};
}

// Exact conversion from a double's leading 48 bits (the rest is rounded into l).
__device__ __forceinline__ dfloat df_from_double(double x) {
  const float h = __double2float_rn(x);
  const float l = __double2float_rn(x - (double)h);
  return dfloat{h, l};
}

__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  float s, t;
  two_sum(a.h, b.h, s, t);
  return dfloat{s, __fadd_rn(t, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ dfloat df_sub(dfloat a, dfloat b) {
  float s, t;
  two_sum(a.h, -b.h, s, t);
  return dfloat{s, __fadd_rn(t, __fsub_rn(a.l, b.l))};
}

// acc += a * b (lazily normalised).
__device__ __forceinline__ void df_fma(dfloat& acc, dfloat a, dfloat b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);   // exact error of p
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  float s, t;
  two_sum(acc.h, p, s, t);
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(t, e));
}

// acc -= a * b (lazily normalised).
__device__ __forceinline__ void df_fms(dfloat& acc, dfloat a, dfloat b) {
  df_fma(acc, dfloat{-a.h, -a.l}, b);
}

// Complex double-float: (re, im).
struct dcomplex {
  dfloat re, im;
};

__device__ __forceinline__ dcomplex dc_from_double2(double2 z) {
  return dcomplex{df_from_double(z.x), df_from_double(z.y)};
}

// Product of two complex double-floats, normalised.
__device__ __forceinline__ dcomplex dc_mul(dcomplex a, dcomplex b) {
  dfloat re = df_zero(), im = df_zero();
  df_fma(re, a.re, b.re);
  df_fms(re, a.im, b.im);
  df_fma(im, a.re, b.im);
  df_fma(im, a.im, b.re);
  return dcomplex{df_norm(re), df_norm(im)};
}

__device__ __forceinline__ dcomplex dc_sub(dcomplex a, dcomplex b) {
  return dcomplex{df_norm(df_sub(a.re, b.re)), df_norm(df_sub(a.im, b.im))};
}

}  // namespace bb
