// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// float32 numbers (about 47 significant bits here).  Dekker's exact product
// via fused multiply-add and Knuth's error-free two-sum; operands come from
// float64 by integer operations on the bit pattern, results go back with one
// float64 addition.  GB300 issues float32 at about 64x its float64 rate, so
// float64-accurate stencil and kernel-weight arithmetic runs faster this way.
#pragma once
#include <math.h>

#include "common.cuh"

namespace wsi {

struct dfl {
  float h, l;
};

// float64 -> (hi, lo): hi = the leading 24 significand bits (truncated), lo =
// the next 23 bits, both exact, by integer operations and one float32
// subtraction and multiplication
__device__ __forceinline__ dfl df_split(double a) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(a);
  const unsigned int hw = (unsigned int)(b >> 32), lw = (unsigned int)b;
  const unsigned int sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const int ef = e - 896;  // float32 biased exponent
  dfl r;
  if (ef <= 0) {
    r.h = 0.0f;
    r.l = 0.0f;
    return r;
  }
  if (ef >= 255) {
    r.h = __uint_as_float(sign | 0x7F800000u);
    r.l = 0.0f;
    return r;
  }
  r.h = __uint_as_float(sign | ((unsigned int)ef << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
  // bits 28..6 of the low word, weight 2^(e - 1069): as a fraction in [0, 1)
  // (exact), then scaled by the signed power of two 2^(e - 1046)
  const float frac = __uint_as_float(0x3F800000u | ((lw & 0x1FFFFFFFu) >> 6)) - 1.0f;
  const int se = e - 919;
  r.l = se > 0 ? frac * __uint_as_float(sign | ((unsigned int)se << 23)) : 0.0f;
  return r;
}

__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
  float s = a + b;
  dfl r;
  r.h = s;
  r.l = b - (s - a);
  return r;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float v = s - a;
  e = (a - (s - v)) + (b - v);
}

// error-free sum of the leading parts, trailing parts added plainly
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  float s, e;
  two_sum(x.h, y.h, s, e);
  e += x.l + y.l;
  return quick_two_sum(s, e);
}

__device__ __forceinline__ dfl df_neg(dfl x) {
  x.h = -x.h;
  x.l = -x.l;
  return x;
}

__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }

__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  return quick_two_sum(p, e);
}

// exact float32 -> float64 by integer operations (normal floats and zero)
__device__ __forceinline__ double f2d_exact(float f) {
  unsigned int u = __float_as_uint(f);
  unsigned int e = (u >> 23) & 0xFFu;
  if (e == 0) return 0.0;
  unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  unsigned long long ed = (unsigned long long)(e - 127 + 1023) << 52;
  unsigned long long m = (unsigned long long)(u & 0x7FFFFFu) << 29;
  return __longlong_as_double((long long)(sign | ed | m));
}

__device__ __forceinline__ double df_to_double(dfl x) { return f2d_exact(x.h) + f2d_exact(x.l); }

// x * c for a constant c; exact scaling of both parts when c is a power of two
__device__ __forceinline__ dfl df_mulc(dfl x, dfl c, bool pow2) {
  if (pow2) {
    x.h *= c.h;
    x.l *= c.h;
    return x;
  }
  return df_mul(x, c);
}

// exact scaling by a power of two given as a float
__device__ __forceinline__ dfl df_scale(dfl x, float p2) {
  x.h *= p2;
  x.l *= p2;
  return x;
}

__device__ __forceinline__ dfl df_from_float(float f) {
  dfl r;
  r.h = f;
  r.l = 0.0f;
  return r;
}

// square root: float32 seed s, one Newton step with the residual x - s^2
// formed exactly (s^2 = p + e by fused multiply-add); 0 for x <= 0
__device__ __forceinline__ dfl df_sqrt(dfl x) {
  if (!(x.h > 0.0f)) return df_from_float(0.0f);
  const float s = sqrtf(x.h);
  const float p = s * s;
  const float e = fmaf(s, s, -p);
  const dfl d = df_sub(x, dfl{p, e});
  return quick_two_sum(s, d.h / (2.0f * s));
}

// Unnormalised head/tail pairs: a value is h + t with the head h formed
// error-free (exact differences by Knuth's two-sum, exact products by fused
// multiply-add) and everything smaller gathered in the float32 tail t,
// which is never renormalised.  Each operation errs by about 2^-24 of the
// tail, i.e. ~2^-46 of its operands' magnitude, like a float64 operation on
// 47-bit inputs; skipping the renormalisation after every step saves three
// instructions per operation.
struct ht {
  float h, t;
};
__device__ __forceinline__ ht ht_of(float2 v) { return ht{v.x, v.y}; }
__device__ __forceinline__ ht ht_sub(ht a, ht b) {
  float s, e;
  two_sum(a.h, -b.h, s, e);
  return ht{s, e + (a.t - b.t)};
}
__device__ __forceinline__ ht ht_add(ht a, ht b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return ht{s, e + (a.t + b.t)};
}
// a * c: exact head product, the two cross terms in float32 (t * t dropped)
__device__ __forceinline__ ht ht_mul(ht a, ht c) {
  const float p = a.h * c.h;
  const float e = fmaf(a.h, c.h, -p);
  return ht{p, fmaf(a.h, c.t, fmaf(a.t, c.h, e))};
}
// a * c for a grid constant c: exact scaling when c is a power of two
__device__ __forceinline__ ht ht_k(ht a, ht c, bool pow2) {
  return pow2 ? ht{a.h * c.h, a.t * c.h} : ht_mul(a, c);
}
__device__ __forceinline__ ht ht_sgn(ht a, float s) { return ht{a.h * s, a.t * s}; }
__device__ __forceinline__ double ht_dbl(ht a) { return f2d_exact(a.h) + f2d_exact(a.t); }

// largest integer <= x (x well inside the int range)
__device__ __forceinline__ int df_floor(dfl x) {
  const float f = floorf(x.h);
  int i = (int)f;
  if (f == x.h && x.l < 0.0f) i -= 1;
  return i;
}

}  // namespace wsi
