// Double-float arithmetic (hi + lo FP32 pairs, after Dekker and Knuth) shared by the
// split-precision kernels: B300 runs FP64 at 2 lanes per clock per SM and FP32 at 128,
// so products with their exact FMA error terms and two-sum accumulation on the FP32
// pipe (~2^-44 relative) stand in for FP64 where that precision suffices.
#pragma once
#include <cuda_runtime.h>

namespace {

// x = hi + lo with |lo| <= ulp(hi) / 2; complex values keep (re, im) pairs of each.
struct DF2 {
  float2 hi, lo;  // complex: (re, im) of the high and the low parts
};
// x = h + l from the bits on the integer pipe (B300 runs double <-> float conversions
// on its 2-lane FP64 pipe): h keeps the top 24 significant bits of x (truncated), l the
// next 29 rounded to 24, so |x - h - l| <= 2^-48 |x|.  Zero, subnormal and
// out-of-float-range inputs (not met by walkers or S^-1 of bounded condition) give
// h = l = 0 or a saturated h.
__device__ __forceinline__ void df_split(double x, float& h, float& l) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
  if (E < 897 || E > 1150) {  // outside the normal float range: zero or saturate
    h = E < 897 ? 0.f : __int_as_float((int)(sign | 0x7F7FFFFFu));
    l = 0.f;
    return;
  }
  const long long m = b & 0xFFFFFFFFFFFFFLL;
  h = __int_as_float((int)(sign | ((unsigned)(E - 896) << 23) | (unsigned)(m >> 29)));
  const int low = (int)(m & 0x1FFFFFFF);  // the 29 bits below h: low 2^(E - 1075)
  const int se = E - 1075 + 127;          // biased exponent of 2^(E - 1075)
  const float scale = se > 0 ? __int_as_float(se << 23) : 0.f;
  l = (float)low * scale;
  if (sign) l = -l;
}
// float -> double from the bits (normal floats; zero and subnormals give 0)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned e = (u >> 23) & 0xFF;
  if (e == 0) return 0.0;
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(e + 896) << 52) |
                               ((unsigned long long)(u & 0x7FFFFF) << 29);
  return __longlong_as_double((long long)b);
}
// (sh, sl) += a * b for real double-floats a = (ah, al), b = (bh, bl)
__device__ __forceinline__ void df_mac(float& sh, float& sl, float ah, float al, float bh,
                                       float bl) {
  const float p = ah * bh;
  const float e = fmaf(ah, bh, -p);             // exact error of the head product
  const float c = fmaf(ah, bl, al * bh);        // cross terms (low order)
  const float t = sh + p;                       // two-sum of the heads
  const float bv = t - sh;
  const float err = (sh - (t - bv)) + (p - bv);
  sl += err + e + c;
  sh = t;
}

// The same multiply-accumulate with every rounding spelled out (__fmul_rn / __fadd_rn
// are never contracted into an FMA, so the two-sum sees the rounded head product),
// and a renormalisation (two-sum of head and tail) for values that are stored and
// updated again: the Gauss-Jordan elimination below updates each entry up to n times.
__device__ __forceinline__ void df_mac_rn(float& sh, float& sl, float ah, float al, float bh,
                                          float bl) {
  const float p = __fmul_rn(ah, bh);
  const float e = fmaf(ah, bh, -p);
  const float c = fmaf(ah, bl, __fmul_rn(al, bh));
  const float t = __fadd_rn(sh, p);
  const float bv = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  sl = __fadd_rn(sl, __fadd_rn(err, __fadd_rn(e, c)));
  sh = t;
}
__device__ __forceinline__ void df_renorm(float& h, float& l) {
  const float s = __fadd_rn(h, l), bv = __fsub_rn(s, h);
  l = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(l, bv));
  h = s;
}
// acc - f a and a b for complex double-floats (renormalised)
__device__ __forceinline__ DF2 df_cfms(const DF2& f, const DF2& a, const DF2& acc) {
  float rh = acc.hi.x, rl = acc.lo.x, ih = acc.hi.y, il = acc.lo.y;
  df_mac_rn(rh, rl, -f.hi.x, -f.lo.x, a.hi.x, a.lo.x);
  df_mac_rn(rh, rl, f.hi.y, f.lo.y, a.hi.y, a.lo.y);
  df_mac_rn(ih, il, -f.hi.x, -f.lo.x, a.hi.y, a.lo.y);
  df_mac_rn(ih, il, -f.hi.y, -f.lo.y, a.hi.x, a.lo.x);
  df_renorm(rh, rl);
  df_renorm(ih, il);
  return DF2{make_float2(rh, ih), make_float2(rl, il)};
}
__device__ __forceinline__ DF2 df_cmul(const DF2& a, const DF2& b) {
  float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
  df_mac_rn(rh, rl, a.hi.x, a.lo.x, b.hi.x, b.lo.x);
  df_mac_rn(rh, rl, -a.hi.y, -a.lo.y, b.hi.y, b.lo.y);
  df_mac_rn(ih, il, a.hi.x, a.lo.x, b.hi.y, b.lo.y);
  df_mac_rn(ih, il, a.hi.y, a.lo.y, b.hi.x, b.lo.x);
  df_renorm(rh, rl);
  df_renorm(ih, il);
  return DF2{make_float2(rh, ih), make_float2(rl, il)};
}
__device__ __forceinline__ DF2 df_from(double2 v) {
  DF2 d;
  df_split(v.x, d.hi.x, d.lo.x);
  df_split(v.y, d.hi.y, d.lo.y);
  return d;
}
__device__ __forceinline__ double2 df_to_double(const DF2& v) {
  return make_double2(f2d_bits(v.hi.x) + f2d_bits(v.lo.x), f2d_bits(v.hi.y) + f2d_bits(v.lo.y));
}

// Complex reciprocal of a double-float: |v|^2 in double-floats, its FP32 reciprocal
// refined by one Newton step (r = r0 (1 + e), e = 1 - |v|^2 r0 to ~2^-47), times conj(v).
__device__ __forceinline__ DF2 df_crecip(const DF2& v) {
  float mh = 0.f, ml = 0.f;
  df_mac_rn(mh, ml, v.hi.x, v.lo.x, v.hi.x, v.lo.x);
  df_mac_rn(mh, ml, v.hi.y, v.lo.y, v.hi.y, v.lo.y);
  df_renorm(mh, ml);
  const float r0 = 1.0f / mh;
  const float e = __fsub_rn(fmaf(-mh, r0, 1.0f), __fmul_rn(ml, r0));
  float rh = r0, rl = __fmul_rn(r0, e);
  df_renorm(rh, rl);
  float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
  df_mac_rn(xh, xl, v.hi.x, v.lo.x, rh, rl);
  df_mac_rn(yh, yl, -v.hi.y, -v.lo.y, rh, rl);
  df_renorm(xh, xl);
  df_renorm(yh, yl);
  return DF2{make_float2(xh, yh), make_float2(xl, yl)};
}

__device__ __forceinline__ void df_add(float& h, float& l, float bh, float bl) {
  const float s = __fadd_rn(h, bh), bv = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(bh, bv));
  l = __fadd_rn(l, __fadd_rn(bl, e));
  h = s;
  df_renorm(h, l);
}
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
  for (int o = 16; o > 0; o >>= 1) {
    const float bh = __shfl_down_sync(0xffffffffu, h, o);
    const float bl = __shfl_down_sync(0xffffffffu, l, o);
    df_add(h, l, bh, bl);
  }
}

}  // namespace
