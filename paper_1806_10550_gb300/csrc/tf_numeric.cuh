// tf_numeric.cuh -- arithmetic building blocks of the two precision modes.
//
// GB300 runs FP64 at about 1/62 of its FP32 rate, and its f64<->f32
// conversions run on the FP64 pipe too.  The FP32-bulk mode therefore keeps
// every per-cell operation on the FP32/INT pipes:
//   * df64: a double-float number hi + lo (two IEEE floats, |lo| <= ulp(hi)/2
//     after normalisation), carried with the error-free transformations of
//     Knuth (TwoSum), Dekker (Fast2Sum) and the FMA product error
//     (TwoProd), which give about 2^-47 relative accuracy per operation.
//   * Conversions between IEEE double bit patterns and floats / df64 pairs
//     done with integer operations only.
//   * The Newton update u + v (double + float) rounded to double with
//     integer operations only.
// Every routine here is __host__ __device__ so the host unit tests exercise
// exactly the code the kernels run.
#pragma once

#include <stdint.h>
#include <string.h>
#include <math.h>

#ifdef __CUDACC__
#define TF_HD __host__ __device__ __forceinline__
#else
#define TF_HD inline
#endif

namespace tf {

TF_HD uint64_t bits_of(double d) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(d);
#else
  uint64_t b;
  memcpy(&b, &d, 8);
  return b;
#endif
}
TF_HD double double_of(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, 8);
  return d;
#endif
}
TF_HD uint32_t bits_of(float f) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(f);
#else
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
#endif
}
TF_HD float float_of(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float f;
  memcpy(&f, &b, 4);
  return f;
#endif
}
TF_HD int clz64(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}
TF_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
  return __clz((int)x);
#else
  return x ? __builtin_clz(x) : 32;
#endif
}
TF_HD float fma_f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return fmaf(a, b, c);
#endif
}

// ---------------------------------------------------------------------------
// double bit pattern -> float (truncated to 24 significant bits).  Normal
// doubles inside the float range map exactly onto the truncated value; zero
// and doubles below the float normal range give 0; larger ones give +-inf;
// NaN stays NaN.
TF_HD float f32_trunc_of_f64(double d) {
  const uint64_t b = bits_of(d);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ff);
  if (e == 0x7ff) {
    const uint64_t man = b & 0xfffffffffffffull;
    return float_of(sign | 0x7f800000u | (man ? 0x400000u : 0u));
  }
  const int ef = e - 1023 + 127;
  if (e == 0 || ef <= 0) return float_of(sign);
  if (ef >= 255) return float_of(sign | 0x7f800000u);
  return float_of(sign | ((uint32_t)ef << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
}

// float -> exact double bit pattern (normal floats and zero; subnormal
// floats flush to signed zero; inf/NaN preserved).
TF_HD double f64_of_f32(float f) {
  const uint32_t b = bits_of(f);
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const int e = (int)((b >> 23) & 0xff);
  if (e == 0) return double_of(sign);
  if (e == 0xff)
    return double_of(sign | 0x7ff0000000000000ull | ((uint64_t)(b & 0x7fffffu) << 29));
  return double_of(sign | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)(b & 0x7fffffu) << 29));
}

// float -> double, exactly what the native conversion gives: normal floats
// and zeros with integer operations (the exponent rebiased by 1023 - 127 in
// the high word, the significand's last three bits in the low word);
// subnormal, infinite and NaN floats, which the Newton update all but never
// meets, take the native conversion.
TF_HD double f64_of_f32_exact(float f) {
  const uint32_t b = bits_of(f), a = b & 0x7fffffffu;
  if (a - 0x00800000u < 0x7f000000u)
    return double_of(((uint64_t)((b & 0x80000000u) | ((a >> 3) + 0x38000000u)) << 32) | (uint64_t)(b << 29));
  if (a == 0u) return double_of((uint64_t)b << 32);
  return (double)f;
}

// ---------------------------------------------------------------------------
// double-float numbers
struct df64 {
  float hi, lo;
};

TF_HD df64 df_make(float hi, float lo) {
  df64 r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// Knuth's TwoSum: s + e == a + b exactly.
TF_HD void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// Dekker's Fast2Sum, valid when |a| >= |b| (or a == 0).
TF_HD void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
// TwoProd with a fused multiply-add: p + e == a * b exactly.
TF_HD void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fma_f(a, b, -p);
}

// Addition with one TwoSum on the leading parts: the error is below about
// 2^-48 (|a| + |b|), enough for sums and differences of the residual, where
// the operands carry 2^-48 relative representation error already.
TF_HD df64 operator+(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  fast_two_sum(s, e, s, e);
  return df_make(s, e);
}
TF_HD df64 operator-(df64 a) { return df_make(-a.hi, -a.lo); }
TF_HD df64 operator-(df64 a, df64 b) { return a + (-b); }
TF_HD df64 operator*(df64 a, df64 b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fma_f(a.hi, b.lo, e);
  e = fma_f(a.lo, b.hi, e);
  fast_two_sum(p, e, p, e);
  return df_make(p, e);
}
// Unnormalised ("lazy") variants for chains of operations: the result pair
// (hi, lo) is exact to about 2^-47 of the operands but lo is not folded into
// hi; fold with df_norm before storing or comparing.
TF_HD df64 df_add_u(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df_make(s, e + (a.lo + b.lo));
}
TF_HD df64 df_mul_u(df64 a, df64 b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  e = fma_f(a.hi, b.lo, e);
  e = fma_f(a.lo, b.hi, e);
  return df_make(p, e);
}
TF_HD df64 df_norm(df64 a) {
  float s, e;
  fast_two_sum(a.hi, a.lo, s, e);
  return df_make(s, e);
}

// 1/a: float reciprocal refined by one Newton step in double-float.
TF_HD df64 df_rcp(df64 a) {
  float y = 1.0f / a.hi;
  df64 Y = df_make(y, 0.0f);
  df64 r = df_make(1.0f, 0.0f) - a * Y;  // residual 1 - a y, small
  return Y + Y * r;
}

// Positive normal double -> float (truncated), five integer operations.
// Valid for 2^-126 <= u < 2^128; used for film tiles of the FP32 Jacobian,
// where any height outside that range already fails the step.
TF_HD float f32_of_pos_f64_fast(double d) {
  const uint64_t b = bits_of(d);
  const uint32_t hi = (uint32_t)(b >> 32), lo = (uint32_t)b;
  return float_of((((hi - 0x38000000u) << 3) & 0x7ffffff8u) | (lo >> 29));
}

// double bit pattern -> df64 with integer operations: hi takes the leading
// 24 significant bits, lo the next 24 (rounded half up from the remaining
// 29).  Relative error below 2^-48.  Zero and values outside the float
// normal range follow f32_trunc_of_f64 with lo = 0.
TF_HD df64 df_of_f64(double d) {
  const uint64_t b = bits_of(d);
  const int e = (int)((b >> 52) & 0x7ff);
  const float hi = f32_trunc_of_f64(d);
  const int ef = e - 1023 + 127;
  if (e == 0 || e == 0x7ff || ef <= 0 || ef >= 255) return df_make(hi, 0.0f);
  uint32_t r = (uint32_t)(b & 0x1fffffffu);  // 29 bits below hi's last bit
  if (r == 0) return df_make(hi, 0.0f);
  const int L = 32 - clz32(r);  // bit length, 1..29
  uint32_t man;
  int lexp;  // exponent (unbiased) of lo's leading bit, in units of 2^(e-1075)
  if (L > 24) {
    man = (r + (1u << (L - 25))) >> (L - 24);
    lexp = L - 1;
    if (man >> 24) {  // rounding carried into a new bit
      man >>= 1;
      lexp += 1;
    }
  } else {
    man = r << (24 - L);
    lexp = L - 1;
  }
  const int lf = (e - 1075) + lexp + 127;  // biased float exponent of lo
  if (lf <= 0) return df_make(hi, 0.0f);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  return df_make(hi, float_of(sign | ((uint32_t)lf << 23) | (man & 0x7fffffu)));
}

// Positive normal double -> df64 in a few operations: hi is the
// truncated float, lo the remaining 29 significand bits rounded to float.
// Valid for 2^-74 <= u < 2^127 (lo stays a normal float); relative error
// below 2^-48.  Film heights lie far inside that range.
TF_HD df64 df_of_pos_f64_fast(double d) {
  const uint64_t b = bits_of(d);
  const float hi = f32_of_pos_f64_fast(d);
  const uint32_t r = (uint32_t)b & 0x1fffffffu;
  if (r == 0) return df_make(hi, 0.0f);
  const int e = (int)((b >> 52) & 0x7ff);
#ifdef __CUDA_ARCH__
  const float rf = __uint2float_rn(r);
#else
  const float rf = (float)r;
#endif
  return df_make(hi, float_of(bits_of(rf) - (uint32_t)((1075 - e) << 23)));
}

// u + v rounded to double (round half away from zero) with integer
// operations.  The rare cases outside the fast path (u zero, subnormal or
// non-finite; v non-finite; |v| > 256 |u|; a result outside the normal
// double range) fall back to native double arithmetic.
TF_HD double f64_add_f32(double u, float v) {
  const uint64_t ub = bits_of(u);
  const uint32_t vb = bits_of(v);
  const int ev = (int)((vb >> 23) & 0xff);
  if (ev == 0) return u;  // v zero or subnormal (|v| < 1.2e-38)
  const int eu = (int)((ub >> 52) & 0x7ff);
  const int shift = ev - eu + 925;  // (ev - 150) - (eu - 1075)
  if (eu == 0 || eu == 0x7ff || ev == 0xff || shift > 37) return u + f64_of_f32(v);
  int64_t mu = (int64_t)((ub & 0xfffffffffffffull) | 0x10000000000000ull);
  uint64_t av = (uint64_t)((vb & 0x7fffffu) | 0x800000u);
  if (shift >= 0) {
    av <<= shift;
  } else if (shift >= -25) {
    av = (av + (1ull << (-shift - 1))) >> (-shift);
  } else {
    av = 0;
  }
  const int64_t sv = (vb >> 31) ? -(int64_t)av : (int64_t)av;
  if ((ub >> 63) == 0) {
    // u > 0 and the sum stays in u's binade (the usual Newton update): the
    // significand sum is the result's significand, exactly
    const int64_t S0 = mu + sv;
    if ((S0 >> 52) == 1)
      return double_of((ub & 0xfff0000000000000ull) | ((uint64_t)S0 & 0xfffffffffffffull));
  } else {
    mu = -mu;
  }
  const int64_t S = mu + sv;
  if (S == 0) return 0.0;
  const uint64_t sgn = S < 0 ? 0x8000000000000000ull : 0ull;
  uint64_t mag = (uint64_t)(S < 0 ? -S : S);
  const int L = 64 - clz64(mag);
  int enew = eu + L - 53;
  if (L > 53) {
    const int k = L - 53;
    mag = (mag + (1ull << (k - 1))) >> k;
    if (mag >> 53) {
      mag >>= 1;
      enew += 1;
    }
  } else if (L < 53) {
    mag <<= (53 - L);
  }
  if (enew <= 0 || enew >= 0x7ff) return u + f64_of_f32(v);
  return double_of(sgn | ((uint64_t)enew << 52) | (mag & 0xfffffffffffffull));
}

// df64 -> double rounded (hi exact, lo added with f64_add_f32).
TF_HD double f64_of_df(df64 x) { return f64_add_f32(f64_of_f32(x.hi), x.lo); }

// Fixed-point image of a non-negative double for exact, order-independent
// mass sums: round(u * 2^36) for 0 <= u < 2^27, with integer operations
// (negative, zero, subnormal and non-finite inputs give 0).
TF_HD int64_t fixed36_of_f64(double u) {
  const uint64_t b = bits_of(u);
  const int e = (int)((b >> 52) & 0x7ff);
  if ((b >> 63) || e == 0 || e == 0x7ff) return 0;
  const int sh = e - 1075 + 36;  // value = man * 2^(e-1075)
  const uint64_t man = (b & 0xfffffffffffffull) | 0x10000000000000ull;
  if (sh >= 0) return sh > 10 ? (int64_t)0x7fffffffffffffffll : (int64_t)(man << sh);
  if (-sh > 54) return 0;
  return (int64_t)((man + (1ull << (-sh - 1))) >> (-sh));
}

}  // namespace tf
