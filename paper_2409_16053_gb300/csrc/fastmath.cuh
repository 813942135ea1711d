// Arithmetic helpers that keep work off GB300's FP64 pipe.
//
// On this GPU the FP64 unit retires about 2 DFMA/DADD/DMUL per clock per SM, and the
// f64<->f32 conversion instructions run on that same unit.  The helpers below move
// conversions to the integer pipe and replace IEEE double division and square root
// (several FP64 instructions each) by a single-precision hardware seed refined with
// one Newton-Raphson step in FP64:
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

// ---- reciprocal, rsqrt, sqrt with one FP64 Newton step ------------------------------
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

// 1/x for finite normal x.  x = m 2^e with m in [1, 2): the seed is the float
// reciprocal of m, refined once in FP64, then scaled by 2^-e on the integer pipe.
__device__ __forceinline__ double rcp64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex == 0u || ex >= 2045u) return 1.0 / x;  // zero, subnormal, huge, inf, NaN
  const unsigned mhi = (hi & 0x800fffffu) | 0x3ff00000u;  // m in +-[1, 2)
  const double m = __hiloint2double((int)mhi, (int)lo);
  const float mf = __uint_as_float(((mhi & 0x80000000u) | 0x3f800000u) |
                                   (((mhi & 0x000fffffu) << 3) | (lo >> 29)));
  double r = f32_to_f64(rcp_approx_f32(mf));
  const double t = fma(-m, r, 1.0);
  r = fma(r, t, r);
  // scale by 2^(1023 - ex): add to the exponent field of r (|r| in (1/2, 1])
  const int rhi = __double2hiint(r) + (int)((1023u - ex) << 20);
  return __hiloint2double(rhi, __double2loint(r));
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
// x * 2^-n (n > 0) for any finite x: exponent arithmetic, or the multiply when x is
// zero or so small that the result would leave the normal range
__device__ __forceinline__ double dscale_down(double x, int n, double two_pow_minus_n) {
  const int hi = __double2hiint(x);
  if ((hi & 0x7ff00000) <= (n << 20)) return x * two_pow_minus_n;
  return __hiloint2double(hi - (n << 20), __double2loint(x));
}

// 1/sqrt(x) for finite normal x > 0: x = m 4^k with m in [1, 4).
__device__ __forceinline__ double rsqrt64(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned ex = (hi >> 20) & 0x7ffu;
  if (ex == 0u || ex >= 2046u || (hi & 0x80000000u)) return 1.0 / sqrt(x);
  // even part of the unbiased exponent goes into the scale, the rest stays in m
  const int e = (int)ex - 1023;
  const int k = e >> 1;                 // floor(e / 2)
  const unsigned mex = (unsigned)(1023 + (e - 2 * k));  // m in [1, 4)
  const unsigned mhi = (hi & 0x000fffffu) | (mex << 20);
  const double m = __hiloint2double((int)mhi, (int)lo);
  const float mf = __uint_as_float(((mex - 896u) << 23) |
                                   (((mhi & 0x000fffffu) << 3) | (lo >> 29)));
  double y = f32_to_f64(rsqrt_approx_f32(mf));
  const double t = fma(-m * y, y, 1.0);  // 1 - m y^2
  y = fma(dscale(y, -1), t, y);          // y + (y/2) t
  // scale by 2^-k
  const int yhi = __double2hiint(y) - (k << 20);
  return __hiloint2double(yhi, __double2loint(y));
}

__device__ __forceinline__ double sqrt64(double x) {
  if ((__double_as_longlong(x) << 1) == 0) return x;  // +-0
  return x * rsqrt64(x);
}

}  // namespace ak
