// Arithmetic helpers that keep work off GB300's FP64 pipe.
//
// On this GPU the FP64 unit retires about 2 DFMA/DADD/DMUL per clock per SM, and the
// f64<->f32 conversion instructions run on that same unit.  The helpers below move
// conversions to the integer pipe and replace IEEE double division and square root
// (several FP64 instructions each) by a single-precision hardware seed refined with
// one Newton-Raphson step, evaluated without the FP64 unit (see below):
//   reciprocal:       r' = r + r (1 - x r)                (Newton on f(r) = 1/r - x)
//   reciprocal sqrt:  y' = y + y (1 - x y^2) / 2          (Newton on f(y) = 1/y^2 - x)
// A seed with relative error e becomes e^2 (reciprocal) or ~1.5 e^2 (rsqrt) after the
// step; with the ~2^-22 single-precision seeds the results carry relative errors of
// about 2^-43 or smaller, far inside the 1e-12 parity budget of the FP64 form.  The
// exponent is split off before seeding, so every finite normal double in range works
// (zero, subnormal, infinite and NaN inputs take the IEEE path).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace ak {

// ---- f64 <-> f32 on the integer pipe ----------------------------------------------
// Round-to-nearest (ties away from zero) conversion of a double to float; results
// below the smallest normal float flush to zero, finite values above the float range
// and non-finite inputs become NaN.
__device__ __forceinline__ float f64_to_f32(double d) {
  const unsigned hi = (unsigned)__double2hiint(d);
  const unsigned lo = (unsigned)__double2loint(d);
  const unsigned mag = hi & 0x7fffffffu;
  // rebias the exponent (1023 -> 127) in the high word, shift the 23 leading
  // mantissa bits into place, round on the next bit
  unsigned bits = __funnelshift_l(lo, mag - (896u << 20), 3) + ((lo >> 28) & 1u);
  bits = (mag < (897u << 20)) ? 0u : bits;            // below FLT_MIN: zero
  bits = (mag >= (1151u << 20)) ? 0x7fc00000u : bits;  // beyond the float range
  return __uint_as_float(bits | (hi & 0x80000000u));
}

// Exact conversion of a float to double (subnormal floats flush to zero).
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned mag = b & 0x7fffffffu;
  unsigned hi = (mag >> 3) + (896u << 20);
  hi = (mag < 0x00800000u) ? 0u : hi;                                   // zero
  hi = (mag >= 0x7f800000u) ? (0x7ff00000u | (mag >> 3)) : hi;          // inf / NaN
  return __hiloint2double((int)(hi | (b & 0x80000000u)), (int)(b << 29));
}

// ---- hardware seeds ----------------------------------------------------------------
__device__ __forceinline__ float rcp_approx_f32(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rsqrt_approx_f32(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// ---- Newton steps without the FP64 unit ----------------------------------------------
// For a seed r0 (a float) of 1/m or 1/sqrt(m), m = mh + ml in [1, 4) with mh its leading
// 24 bits, the residual of one Newton step is small (|e| < 2^-21), so FP32 fused
// multiply-adds on the split m give it to ~2^-46, and the correction d = c r0 e (c = 1 or
// 1/2) to ~2^-46 r0.  r0 + d then has bits from 2^-1 down to ~2^-46 only: it is exact
// in a double and is formed by adding d, in units of 2^-53 (the last place of doubles in
// [1/2, 1)), to the bit pattern of r0.  A sum that leaves [1/2, 1) lies within ~2^-44 of
// the binade edge, where the changed unit only adds an error of that size.

// d * 2^53 as a 64-bit integer, from the bits of the float d (|d| < 2^-20; bits below
// 2^-53 are dropped)
__device__ __forceinline__ long long f32_times_2p53(float d) {
  const unsigned b = __float_as_uint(d);
  const int ex = (int)((b >> 23) & 0xffu);
  const unsigned long long mant = (unsigned long long)((b & 0x7fffffu) | 0x800000u);
  const int sh = ex - 97;  // d 2^53 = mant 2^(ex - 127 - 23 + 53)
  long long v = sh >= 0 ? (long long)(mant << (sh & 63)) : (long long)(mant >> ((-sh) & 63));
  v = (ex < 40) ? 0ll : v;  // |d| < 2^-87 (or zero): nothing at or above 2^-53
  return (b >> 31) ? -v : v;
}

// bit pattern of the double nearest r0 + d for a positive normal float r0 and |d| < 2^-20 r0
__device__ __forceinline__ long long f32_plus_small_bits(float r0, float d) {
  const unsigned b = __float_as_uint(r0);
  const long long widened = ((long long)((b >> 3) + (896u << 20)) << 32) | (long long)(b << 29);
  return widened + f32_times_2p53(d);
}

// mantissa m in [1, 2) of a double (hi/lo words) split into its leading 24 bits (exact
// float) and the remaining 29 bits (rounded down to 23 bits, a float)
__device__ __forceinline__ void split_mantissa(unsigned hi, unsigned lo, float& mh, float& ml) {
  mh = __uint_as_float(0x3f800000u | ((hi & 0x000fffffu) << 3) | (lo >> 29));
  ml = (__uint_as_float(0x4b000000u | ((lo & 0x1fffffffu) >> 6)) - 8388608.0f) * 0x1p-46f;
}

// bit pattern of the double nearest (r0 + d) 2^k for a positive normal float r0 (any
// binade) and |d| < 2^-20 r0: r0 and d are first scaled by a power of two into [1/2, 1).
// When a seed lies on the other side of a power of two than the value it approximates,
// r0 + d leaves [1/2, 1) by up to the seed's error; the part beyond the edge was added in
// units of 2^-53 and is rescaled to the neighbouring binade's unit (2^-54 below 1/2,
// 2^-52 from 1 on).
__device__ __forceinline__ long long scaled_sum_bits(float r0, float d, int k) {
  const int ex = (int)((__float_as_uint(r0) >> 23) & 0xffu) - 126;  // r0 in [2^(ex-1), 2^ex)
  const float sc = __uint_as_float((unsigned)(127 - ex) << 23);
  long long s = f32_plus_small_bits(r0 * sc, d * sc);
  const long long half = 0x3fe0000000000000ll, one = 0x3ff0000000000000ll;
  s = s < half ? 2 * s - half : (s >= one ? one + ((s - one) >> 1) : s);
  return s + ((long long)(k + ex) << 52);
}

// 1/x for finite normal x.  x = +-m 2^(ex-1023), m in [1, 2): r0 = seed of 1/mh in
// (1/2, 1], e = 1 - m r0, 1/m ~ r0 + r0 e; then scaled by 2^(1023-ex) and signed.
// Relative error below 2^-43.
__device__ __forceinline__ double rcp64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex == 0u || ex >= 2045u) return 1.0 / x;  // zero, subnormal, huge, inf, NaN
  float mh, ml;
  split_mantissa(hi, lo, mh, ml);
  const float r0 = rcp_approx_f32(mh);
  const float e = fmaf(-ml, r0, fmaf(-mh, r0, 1.0f));
  long long bits = f32_plus_small_bits(r0, r0 * e);
  bits += (long long)(1023 - (int)ex) << 52;
  bits |= (long long)(hi & 0x80000000u) << 32;
  return __longlong_as_double(bits);
}

// ---- comparisons and exact scalings of doubles on the integer pipe --------------------
// Doubles order like their bit patterns once the magnitude bits of negative values are
// flipped; these tests treat -0.0 as below +0.0 and are meant for finite operands.
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffll);
}
__device__ __forceinline__ bool dgt(double a, double b) { return dkey(a) > dkey(b); }
__device__ __forceinline__ bool dpos(double x) { return __double_as_longlong(x) > 0; }   // x > 0
__device__ __forceinline__ bool dnonneg(double x) { return __double2hiint(x) >= 0; }    // x >= +0
// a > b for a, b >= 0
__device__ __forceinline__ bool dgt_pos(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}
// x * 2^n for normal x whose result stays normal (exponent arithmetic only)
__device__ __forceinline__ double dscale(double x, int n) {
  return __hiloint2double(__double2hiint(x) + (n << 20), __double2loint(x));
}
// x * 2^-n (n > 0) for finite x by exponent arithmetic; a result that would leave the
// normal range (|x| < 2^(n-1022), zero included) becomes a signed zero
__device__ __forceinline__ double dscale_down(double x, int n) {
  const int hi = __double2hiint(x);
  const bool tiny = (hi & 0x7ff00000) <= (n << 20);
  return __hiloint2double(tiny ? (hi & (int)0x80000000) : hi - (n << 20),
                          tiny ? 0 : __double2loint(x));
}

// 1/sqrt(x) for finite normal x > 0: x = m 4^k with m in [1, 4).  y0 = seed of
// 1/sqrt(mh) in (1/2, 1]; y0^2 = p + pe exactly (pe = fma(y0, y0, -p)), so
// e = 1 - m y0^2 = 1 - mh p - mh pe - ml p to ~2^-46, and 1/sqrt(m) ~ y0 + y0 e / 2.
// Relative error below 2^-42.
__device__ __forceinline__ double rsqrt64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex == 0u || ex >= 2046u || (hi & 0x80000000u)) return 1.0 / sqrt(x);
  // even part of the unbiased exponent goes into the scale, the rest stays in m
  const int e2 = (int)ex - 1023;
  const int k = e2 >> 1;  // floor(e2 / 2)
  float mh, ml;
  split_mantissa(hi, lo, mh, ml);
  if (e2 - 2 * k) {       // m in [2, 4): exact doubling of both parts
    mh *= 2.0f;
    ml *= 2.0f;
  }
  const float y0 = rsqrt_approx_f32(mh);
  const float p = y0 * y0;
  const float pe = fmaf(y0, y0, -p);
  const float e = fmaf(-mh, pe, fmaf(-ml, p, fmaf(-mh, p, 1.0f)));
  long long bits = f32_plus_small_bits(y0, 0.5f * y0 * e);
  bits -= (long long)k << 52;  // scale by 2^-k
  return __longlong_as_double(bits);
}

__device__ __forceinline__ double sqrt64(double x) {
  if ((__double_as_longlong(x) << 1) == 0) return x;  // +-0
  return x * rsqrt64(x);
}

// sqrt(a / b) for finite normal a, b > 0 without an FP64 instruction.  a = ma 2^ea,
// b = mb 2^eb with ma, mb in [1, 2) split into leading 24 bits and the rest (ma = mah +
// mal); an odd ea - eb moves a factor 2 into ma, so t = ma / mb = s^2 with the exponent
// halved exactly.  From the seed s0 ~ sqrt(mah / mbh) (rsqrt.approx, ~2^-22), one Newton
// step s = s0 + (ma - s0^2 mb) / (2 s0 mb): s0^2 = P + Pe and P mbh = Q + Qe exactly (fused
// multiply-adds), and ma - Q is exact (Sterbenz), so the residual is formed to ~2^-46 in
// FP32 and s0 + d is assembled as a double on the integer pipe (scaled_sum_bits).
// Relative error below
// 2^-42; other inputs (zero, subnormal, huge, negative, inf, NaN) take sqrt(a / b).
__device__ __forceinline__ double sqrt_ratio64(double a, double b) {
  const unsigned ah = (unsigned)__double2hiint(a), al = (unsigned)__double2loint(a);
  const unsigned bh = (unsigned)__double2hiint(b), bl = (unsigned)__double2loint(b);
  const unsigned ea = ah >> 20, eb = bh >> 20;  // sign bit included: negative -> >= 2048
  if (ea == 0u || ea >= 2045u || eb == 0u || eb >= 2045u) return sqrt(a / b);
  int e = (int)ea - (int)eb;
  float mah, mal, mbh, mbl;
  split_mantissa(ah, al, mah, mal);
  split_mantissa(bh, bl, mbh, mbl);
  if (e & 1) {  // odd exponent difference: t = 2 ma / mb, e even
    mah *= 2.0f;
    mal *= 2.0f;
    e -= 1;
  }
  int k = e / 2;  // exact: e is even
  const float s0 = mah * rsqrt_approx_f32(mah * mbh);  // about (0.7, 2)
  const float P = s0 * s0;
  const float Pe = fmaf(s0, s0, -P);
  const float Q = P * mbh;
  const float Qe = fmaf(P, mbh, -Q);
  const float r = (mah - Q) + ((mal - Qe) - fmaf(P, mbl, Pe * mbh));
  const float d = r * rcp_approx_f32(2.0f * s0 * mbh);
  return __longlong_as_double(scaled_sum_bits(s0, d, k));
}

// sqrt(g a / b) for finite normal a, b > 0 and a constant g > 0 given as a double and
// split into floats g = gh + gl (gh its nearest float): as sqrt_ratio64 with g ma in place
// of ma, so that no FP64 instruction forms the product.  gh mah = G + Ge exactly, and
// G - Q is exact (Sterbenz: both are within a few 2^-22 of g ma); the terms gh mal and
// gl mah beyond G + Ge are of order 2^-23 G, so the residual g ma - s0^2 mb is again
// formed to ~2^-46.  Relative error below 2^-42; other inputs take sqrt(g a / b).
__device__ __forceinline__ double sqrt_gratio64(double a, double b, double g, float gh,
                                                float gl) {
  const unsigned ah = (unsigned)__double2hiint(a), al = (unsigned)__double2loint(a);
  const unsigned bh = (unsigned)__double2hiint(b), bl = (unsigned)__double2loint(b);
  const unsigned ea = ah >> 20, eb = bh >> 20;  // sign bit included: negative -> >= 2048
  if (ea == 0u || ea >= 2045u || eb == 0u || eb >= 2045u) return sqrt(g * a / b);
  int e = (int)ea - (int)eb;
  float mah, mal, mbh, mbl;
  split_mantissa(ah, al, mah, mal);
  split_mantissa(bh, bl, mbh, mbl);
  if (e & 1) {  // odd exponent difference: t = 2 g ma / mb, e even
    mah *= 2.0f;
    mal *= 2.0f;
    e -= 1;
  }
  const int k = e / 2;
  const float G = gh * mah;
  const float Ge = fmaf(gh, mah, -G);
  const float s0 = G * rsqrt_approx_f32(G * mbh);
  const float P = s0 * s0;
  const float Pe = fmaf(s0, s0, -P);
  const float Q = P * mbh;
  const float Qe = fmaf(P, mbh, -Q);
  const float r = (G - Q) + ((Ge - Qe) + (fmaf(gh, mal, gl * mah) - fmaf(P, mbl, Pe * mbh)));
  const float d = r * rcp_approx_f32(2.0f * s0 * mbh);
  return __longlong_as_double(scaled_sum_bits(s0, d, k));
}

}  // namespace ak
