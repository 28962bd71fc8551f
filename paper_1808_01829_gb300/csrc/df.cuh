// Double-float arithmetic on the FP32 units: FP64-accurate results where
// native FP64 (1/64 of the FP32 rate on this GPU) would be the bottleneck.
// A value d is held as an unevaluated pair of floats d = hi + lo
// (|lo| <= ulp(hi)/2), one complex as float4 (re_hi, im_hi, re_lo, im_lo).
// A real product a*b is formed without rounding error in its leading part
// with an FMA (TwoProduct, Ogita, Rump and Oishi 2005):
// p = ah*bh, e = fma(ah, bh, -p) + ah*bl + al*bh; the p are summed with
// TwoSum (Knuth) and the e in an FP32 error accumulator that is folded in at
// the end.  Relative accuracy about 2^-44 per result, against 2^-24 in FP32.
#pragma once

namespace rhmc {
namespace df {


struct DF {
  float h, e;  // running sum and accumulated error
};
// The _rn intrinsics keep the compiler from contracting these steps into FMAs,
// which would break the exactness of TwoSum.
__device__ __forceinline__ void df_add_prod(DF &acc, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float err = fmaf(ah, bh, -p);
  err = fmaf(ah, bl, err);
  err = fmaf(al, bh, err);
  const float s = __fadd_rn(acc.h, p);  // TwoSum(acc.h, p)
  const float bb = __fsub_rn(s, acc.h);
  const float t = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.h = s;
  acc.e = __fadd_rn(acc.e, __fadd_rn(t, err));
}
// acc += u * v for double-float complex u, v (float4 = re_hi, im_hi, re_lo, im_lo)
__device__ __forceinline__ void df_cmac(DF &re, DF &im, const float4 &u, const float4 &v) {
  df_add_prod(re, u.x, u.z, v.x, v.z);
  df_add_prod(re, -u.y, -u.w, v.y, v.w);
  df_add_prod(im, u.x, u.z, v.y, v.w);
  df_add_prod(im, u.y, u.w, v.x, v.z);
}
__device__ __forceinline__ float4 df_pack(const DF &re, const DF &im) {
  // renormalise: (h, e) -> (hi, lo) with FastTwoSum
  const float rh = __fadd_rn(re.h, re.e), rl = __fsub_rn(re.e, __fsub_rn(rh, re.h));
  const float ih = __fadd_rn(im.h, im.e), il = __fsub_rn(im.e, __fsub_rn(ih, im.h));
  return make_float4(rh, ih, rl, il);
}


// a + b for two running sums (TwoSum of the leading parts, errors added)
__device__ __forceinline__ DF df_add(const DF &a, const DF &b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  return DF{s, __fadd_rn(__fadd_rn(a.e, b.e), t)};
}
// renormalise a running sum into a (hi, lo) pair (FastTwoSum)
__device__ __forceinline__ DF df_norm(const DF &a) {
  const float h = __fadd_rn(a.h, a.e);
  return DF{h, __fsub_rn(a.e, __fsub_rn(h, a.h))};
}

// Split x into hi = RN_float(x) and lo = RN_float(x - hi) with 32-bit integer
// operations on the two words of the IEEE-754 bit pattern (FP64 conversions run
// at 1/64 of the FP32 rate on this GPU).  x - hi is d 2^(e - 1075) exactly for
// the integer d = (mantissa remainder below the float's 24 bits, minus 2^29 if
// hi rounded up), |d| <= 2^28, so lo = RN(d) 2^(e - 1075), the scaling exact
// because 2^(e - 1075) is a normal float.  Zeros, subnormals and values whose
// hi or lo leaves the normal float range take the FP64 conversion.
__device__ __forceinline__ float2 df_split1(double x) {
  const unsigned hw = (unsigned)__double2hiint(x), lw = (unsigned)__double2loint(x);
  const int e = (int)((hw >> 20) & 0x7ffu);
  // hi normal (e - 1023 in [-126, 127]) and lo normal (e - 1075 + 28 >= -126)
  if (e < 1023 - 126 + 52 || e > 1023 + 126) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
  }
  unsigned m23 = ((hw & 0xfffffu) << 3) | (lw >> 29);  // leading 23 mantissa bits
  int rem = (int)(lw & 0x1fffffffu);                   // the 29 bits below them
  int fe = e - 1023 + 127;
  if (rem > (1 << 28) || (rem == (1 << 28) && (m23 & 1u))) {  // round to nearest even
    rem -= 1 << 29;
    if (++m23 == (1u << 23)) {
      m23 = 0;
      ++fe;
    }
  }
  const unsigned sign = hw & 0x80000000u;
  const float h = __uint_as_float(sign | ((unsigned)fe << 23) | m23);
  const float scale = __uint_as_float((unsigned)(e - 1075 + 127) << 23);  // 2^(e - 1075), e >= 949
  const float l = __int2float_rn(rem) * scale;
  return make_float2(h, sign ? -l : l);
}
// hi + lo in FP64: the floats are widened by integer operations (exact), one FP64 add
__device__ __forceinline__ double df_widen1(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xff;
  if (ex == 0 || ex == 0xff) return (double)f;  // zero, subnormal, inf/nan
  const unsigned long long b = ((unsigned long long)(u >> 31) << 63) |
                               ((unsigned long long)(ex - 127 + 1023) << 52) |
                               ((unsigned long long)(u & 0x7fffff) << 29);
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ double df_merge1(float h, float l) { return df_widen1(h) + df_widen1(l); }
}  // namespace df
}  // namespace rhmc
