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

}  // namespace kpme
