// Scalar arithmetic back-ends of the face kernels.
//
// Three arithmetic types carry the same face-flux code:
//   double : IEEE binary64 on the SM's FP64 unit;
//   df64   : "double-float", an unevaluated sum hi + lo of two binary32
//            numbers (about 48 significand bits) computed with error-free
//            transformations on the FP32 pipe (Dekker 1971; Knuth TAOCP 2;
//            Hida, Li, Bailey 2001);
//   float  : IEEE binary32.
// The state in memory is always IEEE binary64.  Conversions between binary64
// and binary32 are done with integer operations on the bit patterns so that
// they do not occupy the FP64 unit.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#define FV_HD __device__ __forceinline__

// ---------------------------------------------------------------------------
// bit-level conversions
// ---------------------------------------------------------------------------

// binary64 -> binary32, round to nearest even.  Magnitudes below 2^-126 become
// signed zero, overflow becomes infinity, NaN stays NaN.
__device__ __forceinline__ float fv_d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const unsigned ahi = hi & 0x7fffffffu;
  const unsigned e = ahi >> 20;
  unsigned f = ((ahi - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
  f = (e < 897u) ? 0u : f;
  f = (e > 1150u) ? 0x7f800000u : f;
  f = (e == 2047u) ? 0x7fc00000u : f;
  return __int_as_float((int)(f | sign));
}

// binary64 -> binary32, rounded toward zero: magnitudes below 2^-126 become
// signed zero, magnitudes from 2^128 up (and Inf, NaN) become NaN.  At most
// one unit in the last place - the binary32-flux form's face arithmetic
// carries far more - for half the instructions of fv_d2f_rn.
__device__ __forceinline__ float fv_d2f_rz(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned ahi = hi & 0x7fffffffu;
  unsigned f = ((ahi - (896u << 20)) << 3) | (lo >> 29);
  f = ahi < (897u << 20) ? 0u : f;
  f = ahi >= (1151u << 20) ? 0x7fc00000u : f;
  return __int_as_float((int)(f | (hi & 0x80000000u)));
}

// binary32 -> binary64, exact (zero and normal numbers; subnormals flush).
__device__ __forceinline__ double fv_f2d(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned a = u & 0x7fffffffu;
  unsigned hi = (((a >> 23) + 896u) << 20) | ((a >> 3) & 0xfffffu);
  unsigned lo = a << 29;
  const bool zero = a < 0x00800000u;
  const bool special = a >= 0x7f800000u;
  hi = zero ? 0u : (special ? (0x7ff00000u | ((a >> 3) & 0xfffffu)) : hi);
  lo = zero ? 0u : lo;
  return __longlong_as_double((long long)(((unsigned long long)(hi | sign) << 32) | lo));
}

// ---------------------------------------------------------------------------
// double-float
// ---------------------------------------------------------------------------
struct df64 {
  float hi, lo;
};

FV_HD df64 mk(float h, float l) { df64 r; r.hi = h; r.lo = l; return r; }

// binary32 operations that the compiler may neither contract into FMAs nor
// reorder: the error-free transformations below depend on every rounding.
#define FADD __fadd_rn
#define FSUB __fsub_rn
#define FMUL __fmul_rn
#define FFMA __fmaf_rn

// s + e = a + b exactly (any magnitudes)
FV_HD df64 two_sum(float a, float b) {
  float s = FADD(a, b);
  float bb = FSUB(s, a);
  float e = FADD(FSUB(a, FSUB(s, bb)), FSUB(b, bb));
  return mk(s, e);
}
// s + e = a + b exactly when |a| >= |b|
FV_HD df64 quick_two_sum(float a, float b) {
  float s = FADD(a, b);
  float e = FSUB(b, FSUB(s, a));
  return mk(s, e);
}
FV_HD df64 two_prod(float a, float b) {
  float p = FMUL(a, b);
  float e = FFMA(a, b, -p);
  return mk(p, e);
}

// Sum with one error-free transformation of the high parts ("sloppy" add):
// the absolute error is below ~2^-47 of the larger operand, which is the
// accuracy binary64 itself offers relative to its operands.
FV_HD df64 operator+(df64 a, df64 b) {
  df64 s = two_sum(a.hi, b.hi);
  float e = FADD(s.lo, FADD(a.lo, b.lo));
  return quick_two_sum(s.hi, e);
}
FV_HD df64 operator-(df64 a) { return mk(-a.hi, -a.lo); }
FV_HD df64 operator-(df64 a, df64 b) { return a + (-b); }
FV_HD df64 operator*(df64 a, df64 b) {
  df64 p = two_prod(a.hi, b.hi);
  float e = FFMA(a.hi, b.lo, p.lo);
  e = FFMA(a.lo, b.hi, e);
  return quick_two_sum(p.hi, e);
}
FV_HD df64 operator*(df64 a, float b) {
  df64 p = two_prod(a.hi, b);
  float e = FFMA(a.lo, b, p.lo);
  return quick_two_sum(p.hi, e);
}
FV_HD df64 operator*(float b, df64 a) { return a * b; }
FV_HD df64& operator+=(df64& a, df64 b) { a = a + b; return a; }
FV_HD df64& operator-=(df64& a, df64 b) { a = a - b; return a; }

// sum_i a_i b_i with one renormalisation at the end (a compensated dot
// product after Ogita, Rump and Oishi, "Accurate sum and dot product", SIAM
// J. Sci. Comput. 26, 2005): each product of the high parts is split exactly
// by an FMA, the high products are summed with two_sum, and every error term
// (the splits' errors, the two_sum errors, the products with the low parts)
// is gathered in binary32.  Error ~2^-47 of sum_i |a_i b_i|, as a chain of
// the operators above gives, at 12 N - 5 instead of 18 N - 11 binary32
// operations.
template <int N>
FV_HD df64 df_dot(const df64 (&a)[N], const df64 (&b)[N]) {
  float s = FMUL(a[0].hi, b[0].hi);
  float err = FFMA(a[0].hi, b[0].hi, -s);
  err = FFMA(a[0].hi, b[0].lo, err);
  err = FFMA(a[0].lo, b[0].hi, err);
#pragma unroll
  for (int i = 1; i < N; ++i) {
    const float p = FMUL(a[i].hi, b[i].hi);
    float e = FFMA(a[i].hi, b[i].hi, -p);
    e = FFMA(a[i].hi, b[i].lo, e);
    e = FFMA(a[i].lo, b[i].hi, e);
    const df64 t = two_sum(s, p);
    s = t.hi;
    err = FADD(err, FADD(t.lo, e));
  }
  return quick_two_sum(s, err);
}

__device__ __forceinline__ float fv_rcp(float x) { return __frcp_rn(x); }

// a / b: correctly rounded binary32 reciprocal of b.hi, quotient estimate and
// one correction step in double-float (relative error ~2^-47)
FV_HD df64 operator/(df64 a, df64 b) {
  float r = fv_rcp(b.hi);
  float q1 = FMUL(a.hi, r);
  df64 rem = a - b * q1;
  float q2 = FMUL(rem.hi, r);
  return quick_two_sum(q1, q2);
}
FV_HD df64 df_rcp(df64 b) { return mk(1.0f, 0.0f) / b; }

FV_HD df64 df_sqrt(df64 a) {
  if (!(a.hi > 0.0f)) return mk(a.hi == 0.0f ? 0.0f : __int_as_float(0x7fc00000), 0.0f);
  float s = __fsqrt_rn(a.hi);
  df64 e = a - two_prod(s, s);
  float corr = FMUL(e.hi, FMUL(0.5f, __fdividef(1.0f, s)));
  return quick_two_sum(s, corr);
}
FV_HD df64 df_abs(df64 a) { return a.hi < 0.0f ? -a : a; }
FV_HD bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
FV_HD bool operator>(df64 a, df64 b) { return b < a; }

// binary64 -> double-float (hi = RN(x), lo = RN(x - hi)), bit operations only
__device__ __forceinline__ df64 fv_d2df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const unsigned ahi = hi & 0x7fffffffu;
  const unsigned e = ahi >> 20;
  unsigned f = ((ahi - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
  f += up;
  // remainder x - hi = (rem - up*2^29) * 2^(e-1075), |.| <= 2^28 * 2^(e-1075)
  const int r = (int)rem - (int)(up << 29);
  float lof = __int2float_rn(r);
  // scale by 2^(e-1075): build the binary32 power of two when it is normal
  const int pe = (int)e - 1075 + 127;
  const float scale = __int_as_float(pe > 0 ? (pe << 23) : 0);
  lof = FMUL(lof, scale);
  if (sign) lof = -lof;
  f = (e < 897u) ? 0u : f;
  f = (e > 1150u) ? 0x7f800000u : f;
  f = (e == 2047u) ? 0x7fc00000u : f;
  lof = (e < 897u || e > 1150u) ? 0.0f : lof;
  return mk(__int_as_float((int)(f | sign)), lof);
}

// double-float -> binary64 (exact conversions of both halves, one FP64 add)
__device__ __forceinline__ double fv_df2d(df64 a) { return fv_f2d(a.hi) + fv_f2d(a.lo); }

// ---------------------------------------------------------------------------
// binary64 reciprocal within one unit in the last place (not always the
// correctly rounded value): the hardware's approximate reciprocal y0 of x
// (PTX rcp.approx.ftz.f64, relative error e0) refined by one third-order
// step of the geometric series 1/(x y0) = 1/(1 - e) = 1 + e + e^2 + ...,
// e = 1 - x y0:  y = y0 + y0 (e + e^2), relative error e0^3 plus the
// rounding of three fused multiply-adds.  On GB300 the compiler's IEEE
// 1.0 / x costs about 4.6 FMA issue slots of the FP64 unit, this three.
// For finite, nonzero, normal x whose reciprocal is normal (0, infinities
// and subnormals give NaN): the face code takes it of densities, squared
// sound speeds, 1 + sqrt(rho_R / rho_L), entropy-fix widths, van Albada
// denominators (>= delta^2) and van Leer sums, which it discards when they
// fall below 1e-30.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fv_rcp64(double x) {
  double y0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// ---------------------------------------------------------------------------
// binary64 square root within one unit in the last place: the hardware's
// approximate reciprocal square root y0 of x (PTX rsqrt.approx.ftz.f64),
// s = x y0 and e = 1 - s y0, so that x / s^2 = 1 / (1 - e) up to the
// rounding of s, and sqrt(x) = s (1 - e)^(-1/2) = s (1 + e/2 + 3 e^2/8 + ...)
// by the binomial series, here truncated after its e^2 term: five FP64
// instructions where the compiler's IEEE square root costs about 7.5 FMA
// issue slots on GB300.  For finite, positive, normal x (0, infinities,
// negative and subnormal x give NaN): the face code takes it of density
// ratios and squared sound speeds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double fv_sqrt64(double x) {
  double y0;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
  const double s = x * y0;
  const double e = fma(-s, y0, 1.0);
  return fma(s * e, fma(e, 0.375, 0.5), s);
}

// ---------------------------------------------------------------------------
// uniform scalar interface used by the face code
// ---------------------------------------------------------------------------
template <class T> struct Sc;

template <> struct Sc<double> {
  static __device__ __forceinline__ double from_d(double x) { return x; }
  static __device__ __forceinline__ double to_d(double x) { return x; }
  static __device__ __forceinline__ double c(double x) { return x; }     // constant
  static __device__ __forceinline__ double sqrt(double x) { return fv_sqrt64(x); }
  static __device__ __forceinline__ double abs(double x) { return ::fabs(x); }
  // reciprocal within one unit in the last place (fv_rcp64); a quotient is
  // that reciprocal times the numerator
  static __device__ __forceinline__ double rcp(double x) { return fv_rcp64(x); }
  static __device__ __forceinline__ double div(double a, double b) { return a * fv_rcp64(b); }
  static __device__ __forceinline__ double halve(double x) { return 0.5 * x; }
  static __device__ __forceinline__ double quarter(double x) { return 0.25 * x; }
  static __device__ __forceinline__ double twice(double x) { return 2.0 * x; }
  static __device__ __forceinline__ double dot2(double a, double b, double c, double d) { return a * b + c * d; }
  static __device__ __forceinline__ double dot3(double a, double b, double c, double d, double e, double f) {
    return a * b + c * d + e * f;
  }
  static __device__ __forceinline__ double dot4(double a, double b, double c, double d, double e, double f, double g,
                                                double h) {
    return a * b + c * d + e * f + g * h;
  }
  // a b + c d (+ e f) - z as a chain of fused multiply-adds from -z
  static __device__ __forceinline__ double dot2m(double a, double b, double c, double d, double z) {
    return fma(a, b, fma(c, d, -z));
  }
  static __device__ __forceinline__ double dot3m(double a, double b, double c, double d, double e, double f, double z) {
    return fma(a, b, fma(c, d, fma(e, f, -z)));
  }
  static __device__ __forceinline__ float hi(double x) { return (float)x; }
  static __device__ __forceinline__ bool lt(double a, double b) { return a < b; }
  // Sign and magnitude tests of the limiter and the entropy fix as integer
  // comparisons of the bit patterns (the FP64 unit is the binary64 kernel's
  // bottleneck; the integer units are idle).  For non-NaN binary64 values
  // the ordering of non-negative numbers is that of their bit patterns read
  // as integers, and a positive number is one whose pattern, read as a
  // signed integer, is positive.
  static __device__ __forceinline__ bool pos(double a) { return __double_as_longlong(a) > 0; }
  static __device__ __forceinline__ bool above(double a_nonneg, float t) {
    return __double_as_longlong(a_nonneg) > __double_as_longlong((double)t);
  }
  static __device__ __forceinline__ bool lt_nonneg(double a, double b) {
    return __double_as_longlong(a) < __double_as_longlong(b);
  }
  static __device__ __forceinline__ bool neg(double a) {
    const long long b = __double_as_longlong(a);
    return b < 0 && (b & 0x7fffffffffffffffLL) != 0;   // below zero (not -0)
  }
  using mask = bool;
  static __device__ __forceinline__ double sel(bool m, double a, double b) { return m ? a : b; }
  static __device__ __forceinline__ bool ge(double a, float t) { return a >= (double)t; }
  static __device__ __forceinline__ bool le(double a, float t) { return a <= (double)t; }
};

template <> struct Sc<float> {
  // integer conversion: the hardware one runs on the FP64 unit, which GB300
  // gives 1/64 of the binary32 rate (5 % slower on the 128^3 stage); toward
  // zero rather than to nearest: 4 % faster again, within the form's error
  static __device__ __forceinline__ float from_d(double x) { return fv_d2f_rz(x); }
  static __device__ __forceinline__ double to_d(float x) { return fv_f2d(x); }
  static __device__ __forceinline__ float c(double x) { return (float)x; }
  // approximate (MUFU) reciprocal and square root: the binary32 flux form
  // already carries ~1e-6 relative error, a few more ulps do not matter
  static __device__ __forceinline__ float sqrt(float x) { return x * rsqrtf(x); }
  static __device__ __forceinline__ float abs(float x) { return ::fabsf(x); }
  static __device__ __forceinline__ float rcp(float x) { return __fdividef(1.0f, x); }
  static __device__ __forceinline__ float div(float a, float b) { return a * rcp(b); }
  static __device__ __forceinline__ float halve(float x) { return 0.5f * x; }
  static __device__ __forceinline__ float quarter(float x) { return 0.25f * x; }
  static __device__ __forceinline__ float twice(float x) { return 2.0f * x; }
  static __device__ __forceinline__ float dot2(float a, float b, float c, float d) { return a * b + c * d; }
  static __device__ __forceinline__ float dot3(float a, float b, float c, float d, float e, float f) {
    return a * b + c * d + e * f;
  }
  static __device__ __forceinline__ float dot4(float a, float b, float c, float d, float e, float f, float g,
                                               float h) {
    return a * b + c * d + e * f + g * h;
  }
  static __device__ __forceinline__ float dot2m(float a, float b, float c, float d, float z) {
    return fmaf(a, b, fmaf(c, d, -z));
  }
  static __device__ __forceinline__ float dot3m(float a, float b, float c, float d, float e, float f, float z) {
    return fmaf(a, b, fmaf(c, d, fmaf(e, f, -z)));
  }
  static __device__ __forceinline__ float hi(float x) { return x; }
  static __device__ __forceinline__ bool lt(float a, float b) { return a < b; }
  static __device__ __forceinline__ bool lt_nonneg(float a, float b) { return a < b; }
  static __device__ __forceinline__ bool neg(float a) { return a < 0.0f; }
  static __device__ __forceinline__ bool pos(float a) { return a > 0.0f; }
  static __device__ __forceinline__ bool above(float a, float t) { return a > t; }
  using mask = bool;
  static __device__ __forceinline__ float sel(bool m, float a, float b) { return m ? a : b; }
  static __device__ __forceinline__ bool ge(float a, float t) { return a >= t; }
  static __device__ __forceinline__ bool le(float a, float t) { return a <= t; }
};

template <> struct Sc<df64> {
  static __device__ __forceinline__ df64 from_d(double x) { return fv_d2df(x); }
  static __device__ __forceinline__ double to_d(df64 x) { return fv_df2d(x); }
  // compile-time constants: split on the host side of the compiler
  static __device__ __forceinline__ df64 c(double x) {
    float h = (float)x;
    return mk(h, (float)(x - (double)h));
  }
  static __device__ __forceinline__ df64 sqrt(df64 x) { return df_sqrt(x); }
  static __device__ __forceinline__ df64 abs(df64 x) { return df_abs(x); }
  static __device__ __forceinline__ df64 rcp(df64 x) { return df_rcp(x); }
  static __device__ __forceinline__ df64 div(df64 a, df64 b) { return a / b; }
  // exact: both halves scale by a power of two
  static __device__ __forceinline__ df64 halve(df64 x) { return mk(0.5f * x.hi, 0.5f * x.lo); }
  static __device__ __forceinline__ df64 quarter(df64 x) { return mk(0.25f * x.hi, 0.25f * x.lo); }
  static __device__ __forceinline__ df64 twice(df64 x) { return mk(2.0f * x.hi, 2.0f * x.lo); }
  static __device__ __forceinline__ df64 dot2(df64 a, df64 b, df64 c, df64 d) {
    const df64 x[2] = {a, c}, y[2] = {b, d};
    return df_dot<2>(x, y);
  }
  static __device__ __forceinline__ df64 dot3(df64 a, df64 b, df64 c, df64 d, df64 e, df64 f) {
    const df64 x[3] = {a, c, e}, y[3] = {b, d, f};
    return df_dot<3>(x, y);
  }
  static __device__ __forceinline__ df64 dot4(df64 a, df64 b, df64 c, df64 d, df64 e, df64 f, df64 g, df64 h) {
    const df64 x[4] = {a, c, e, g}, y[4] = {b, d, f, h};
    return df_dot<4>(x, y);
  }
  // the subtracted term as one more product with -1 (exact) in the
  // compensated dot product
  static __device__ __forceinline__ df64 dot2m(df64 a, df64 b, df64 c, df64 d, df64 z) {
    const df64 x[3] = {a, c, z}, y[3] = {b, d, mk(-1.0f, 0.0f)};
    return df_dot<3>(x, y);
  }
  static __device__ __forceinline__ df64 dot3m(df64 a, df64 b, df64 c, df64 d, df64 e, df64 f, df64 z) {
    const df64 x[4] = {a, c, e, z}, y[4] = {b, d, f, mk(-1.0f, 0.0f)};
    return df_dot<4>(x, y);
  }
  static __device__ __forceinline__ float hi(df64 x) { return x.hi; }
  static __device__ __forceinline__ bool lt(df64 a, df64 b) { return a < b; }
  static __device__ __forceinline__ bool lt_nonneg(df64 a, df64 b) { return a < b; }
  static __device__ __forceinline__ bool neg(df64 a) { return a.hi < 0.0f; }
  static __device__ __forceinline__ bool pos(df64 a) { return a.hi > 0.0f; }
  static __device__ __forceinline__ bool above(df64 a, float t) { return a.hi > t; }
  using mask = bool;
  static __device__ __forceinline__ df64 sel(bool m, df64 a, df64 b) { return m ? a : b; }
  static __device__ __forceinline__ bool ge(df64 a, float t) { return a.hi > t || (a.hi == t && a.lo >= 0.0f); }
  static __device__ __forceinline__ bool le(df64 a, float t) { return a.hi < t || (a.hi == t && a.lo <= 0.0f); }
};
