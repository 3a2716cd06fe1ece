// Double-float ("DF") arithmetic on the FP32 pipe: a value is the unevaluated sum
// h + l of two floats (|l| <= ulp(h) / 2 once normalised: 48 significand bits).
// Error-free transformations give the exact rounding error of a float sum (Knuth's
// TwoSum) and of a float product (by FMA); accumulations keep those errors as in the
// compensated dot product of Ogita, Rump and Oishi ("Accurate sum and dot product",
// SIAM J. Sci. Comput. 26, 2005).  FP32 arithmetic runs 64x faster than FP64 on this
// part, and one DF multiply-add costs about 12 FP32 operations.
#pragma once
#include "kernels.h"

namespace wcmg {

struct dfr { float h, l; };
struct dfc { dfr re, im; };

__device__ __forceinline__ dfr df_from(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ dfr df_neg(dfr a) { return {-a.h, -a.l}; }
// TwoSum: s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float v = s - a;
  e = (a - (s - v)) + (b - v);
}
// acc += x y  (low parts of the product beyond x.l y.l kept; acc left unnormalised)
__device__ __forceinline__ void df_mac(dfr& acc, dfr x, dfr y) {
  const float p = x.h * y.h;
  float pe = fmaf(x.h, y.h, -p);
  pe = fmaf(x.h, y.l, pe);
  pe = fmaf(x.l, y.h, pe);
  float s, e;
  two_sum(acc.h, p, s, e);
  acc.h = s;
  acc.l += e + pe;
}
__device__ __forceinline__ dfr df_norm(dfr a) {
  const float h = a.h + a.l;
  return {h, a.l - (h - a.h)};
}
__device__ __forceinline__ dfr df_add(dfr a, dfr b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return df_norm({s, e + (a.l + b.l)});
}
__device__ __forceinline__ dfr df_mul(dfr x, dfr y) {
  const float p = x.h * y.h;
  float pe = fmaf(x.h, y.h, -p);
  pe = fmaf(x.h, y.l, pe);
  pe = fmaf(x.l, y.h, pe);
  return df_norm({p, pe});
}
__device__ __forceinline__ dfc dfc_add(dfc a, dfc b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ dfc dfc_norm(dfc a) { return {df_norm(a.re), df_norm(a.im)}; }
// acc += conj(q) a
__device__ __forceinline__ void dfc_cjmac(dfc& acc, const dfc& q, const dfc& a) {
  df_mac(acc.re, q.re, a.re);
  df_mac(acc.re, q.im, a.im);
  df_mac(acc.im, q.re, a.im);
  df_mac(acc.im, df_neg(q.im), a.re);
}
// acc -= r q
__device__ __forceinline__ void dfc_nmac(dfc& acc, const dfc& r, const dfc& q) {
  df_mac(acc.re, df_neg(r.re), q.re);
  df_mac(acc.re, r.im, q.im);
  df_mac(acc.im, df_neg(r.re), q.im);
  df_mac(acc.im, df_neg(r.im), q.re);
}
__device__ __forceinline__ dfc dfc_load(const float4* p) {
  const float4 v = *p;
  return {{v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ dfc dfc_shfl_xor(const dfc& v, int o) {
  return {{__shfl_xor_sync(0xffffffffu, v.re.h, o), __shfl_xor_sync(0xffffffffu, v.re.l, o)},
          {__shfl_xor_sync(0xffffffffu, v.im.h, o), __shfl_xor_sync(0xffffffffu, v.im.l, o)}};
}
// Transposing warp sums of GS DF values (GS a power of two, at most 32): on return v[0] of lane l holds
// the warp sum of value dfc_sum_index<GS>(l); lanes whose low 5 - log2(GS) bits are zero
// hold each value once.
template <int GS>
__device__ __forceinline__ void dfc_warp_sum_transposed(dfc (&v)[GS], int lane) {
  int off = 16;
#pragma unroll
  for (int n = GS; n > 1; n >>= 1, off >>= 1) {
    const bool up = lane & off;
#pragma unroll
    for (int j = 0; j < n / 2; ++j) {
      const dfc send = up ? v[j] : v[j + n / 2];
      const dfc keep = up ? v[j + n / 2] : v[j];
      v[j] = dfc_add(keep, dfc_shfl_xor(send, off));
    }
  }
#pragma unroll
  for (; off > 0; off >>= 1) v[0] = dfc_add(v[0], dfc_shfl_xor(v[0], off));
}
template <int GS>
__device__ __forceinline__ int dfc_sum_index(int lane) {
  int g = 0, off = 16;
#pragma unroll
  for (int n = GS; n > 1; n >>= 1, off >>= 1) g = 2 * g + ((lane & off) ? 1 : 0);
  return g;
}
__device__ __forceinline__ dfr df_warp_sum(dfr v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
    v = df_add(v, {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
  return v;
}

// FP64 -> DF without the FP64 pipe: h = x truncated to 24 significant bits (its
// float bit pattern built from the double's sign, exponent and top mantissa bits),
// l = the remaining 29 mantissa bits as a float (rounded) scaled by the exponent.
// Exact for h; l carries x - h to float precision.  Magnitudes outside [2^-74, 2^127)
// take the FP64 conversion path.
__device__ __forceinline__ dfr df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e < 949 || e > 1149) return df_from(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned hb = sign | ((unsigned)(e - 1023 + 127) << 23) | (unsigned)((b >> 29) & 0x7FFFFFu);
  const unsigned low = (unsigned)(b & 0x1FFFFFFFull);
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);  // 2^(e - 1075)
  const float l = __uint2float_rn(low) * scale;
  return {__uint_as_float(hb), __uint_as_float(__float_as_uint(l) | sign)};
}
// DF -> FP64: both floats widened exactly by their bit patterns, one FP64 add
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xFF;
  if (e == 0 || e == 255) return (double)f;
  const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double df_to_fast(dfr a) { return f2d_exact(a.h) + f2d_exact(a.l); }
// acc += a b (complex)
__device__ __forceinline__ void dfc_mac(dfc& acc, const dfc& a, const dfc& b) {
  df_mac(acc.re, a.re, b.re);
  df_mac(acc.re, df_neg(a.im), b.im);
  df_mac(acc.im, a.re, b.im);
  df_mac(acc.im, a.im, b.re);
}
__device__ __forceinline__ dfc dfc_split(double2 v) { return {df_split(v.x), df_split(v.y)}; }
__device__ __forceinline__ double2 dfc_to_fast(const dfc& a) { return make_double2(df_to_fast(a.re), df_to_fast(a.im)); }

}  // namespace wcmg
