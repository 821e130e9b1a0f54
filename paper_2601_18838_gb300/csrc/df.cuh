// Double-float arithmetic (value = hi + lo, |lo| <= ulp(hi)/2, about 44 significant bits) on
// the float32 pipe.  The float64 pipe of this GPU issues far fewer operations per clock than
// the float32 one (conversions between float and double included), so sums that need more than
// float32 precision run in pairs of floats: products split exactly with fma (Dekker / Veltkamp:
// a*b - fl(a*b) is representable), sums with the two-sum of Knuth.
#pragma once

namespace kpme {

struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);                  // exact error of the leading product
  const float t = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const float h = p + t;
  return {h, t - (h - p)};
}
__device__ __forceinline__ df df_add(df a, df b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);       // exact error of the leading sum
  const float t = e + a.lo + b.lo;
  const float h = s + t;
  return {h, t - (h - s)};
}
__device__ __forceinline__ df df_scale(df a, float c) {  // a times a float32 c
  const float p = a.hi * c;
  const float e = fmaf(a.hi, c, -p);
  const float t = fmaf(a.lo, c, e);
  const float h = p + t;
  return {h, t - (h - p)};
}

__device__ __forceinline__ df df_fma(df acc, df a, df b) { return df_add(acc, df_mul(a, b)); }   // acc + a b

// a * b rounded once to float32: the leading product plus the first-order terms, RN(p + t).
// (The normalised pair (h, l) of df_mul has h = RN(p + t) and h + l = p + t exactly, so
// RN(h + l) = h: the float32 rounding of the pair is its leading word.)
__device__ __forceinline__ float df_mul_rn(df a, df b) {
  const float p = a.hi * b.hi;
  const float e = fmaf(a.hi, b.hi, -p);
  return p + fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
}

// A float64 value as a double-float pair with integer operations only (no float64 unit):
// hi holds the leading 24 significand bits of x, lo the other 29 rounded to float32, then the
// pair is renormalised (hi + lo carries about 48 bits).  ok is false for what the split does
// not represent: |x| outside [2^-60, 2^126), NaN and infinities (x == 0 is represented).
__device__ __forceinline__ df df_bits(double x, bool& ok) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int h32 = (unsigned int)(b >> 32), l32 = (unsigned int)b;
  const unsigned int sign = h32 & 0x80000000u;
  const int E = (int)((h32 >> 20) & 0x7ffu);
  if ((b << 1) == 0ull) {
    ok = true;
    return {__uint_as_float(sign), 0.0f};
  }
  ok = E >= 1023 - 60 && E < 1023 + 126;
  if (!ok) return {0.0f, 0.0f};
  const float hi = __uint_as_float(sign | ((unsigned int)(E - 896) << 23) | ((h32 & 0xfffffu) << 3) | (l32 >> 29));
  // the remaining 29 bits are units of 2^(E - 1075); that power of two is a normal float here
  float lo = __uint2float_rn(l32 & 0x1fffffffu) * __uint_as_float((unsigned int)(E - 948) << 23);
  lo = sign ? -lo : lo;
  const float s = hi + lo;
  return {s, lo - (s - hi)};
}

// A float32 value as float64 by its bits (normal numbers and zero); others by conversion.
__device__ __forceinline__ double dbl_of(float v) {
  const unsigned int u = __float_as_uint(v);
  const unsigned int ex = (u >> 23) & 0xffu;
  if (ex == 0u || ex == 0xffu) return (u << 1) == 0u ? __longlong_as_double((long long)u << 32) : (double)v;
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

}  // namespace kpme
