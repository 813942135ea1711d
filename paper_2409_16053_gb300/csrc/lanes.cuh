// Lane-generic FP32 arithmetic for the mixed form: every function below exists for a
// scalar `float` and for a `float2` that carries two independent problems in its two
// lanes (GB300's packed FP32x2 add, subtract, multiply and fused multiply-add issue one
// instruction for both).  Each lane of a float2 operation rounds exactly like the
// scalar operation, so code written once over these functions gives the same bits for a
// problem solved alone or paired with another one.  Comparisons, selects and the
// hardware reciprocal / rsqrt seeds act lane by lane.
#pragma once

#include <cuda_runtime.h>

#include "fastmath.cuh"

namespace ak {

struct bool2 {
  bool x, y;
};

// ---- arithmetic ------------------------------------------------------------------------
// scalar forms through the round-to-nearest intrinsics, which are never fused
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// The packed operations are issued as PTX so that the compiler cannot fuse a packed
// multiply into a following add (the library builds without implicit contraction, and
// the packed lanes must round exactly like the scalar code).
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
  return ((unsigned long long)__float_as_uint(a.y) << 32) | __float_as_uint(a.x);
}
__device__ __forceinline__ float2 bits_f2(unsigned long long r) {
  return make_float2(__uint_as_float((unsigned)r), __uint_as_float((unsigned)(r >> 32)));
}
__device__ __forceinline__ float2 vadd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return bits_f2(r);
}

__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

// broadcast of a scalar constant
template <typename V> __device__ __forceinline__ V vset(float c);
template <> __device__ __forceinline__ float vset<float>(float c) { return c; }
template <> __device__ __forceinline__ float2 vset<float2>(float c) { return make_float2(c, c); }

// ---- lane-wise comparisons and selects ---------------------------------------------------
__device__ __forceinline__ bool vgt(float a, float b) { return a > b; }
__device__ __forceinline__ bool vge(float a, float b) { return a >= b; }
__device__ __forceinline__ bool2 vgt(float2 a, float2 b) { return {a.x > b.x, a.y > b.y}; }
__device__ __forceinline__ bool2 vge(float2 a, float2 b) { return {a.x >= b.x, a.y >= b.y}; }

__device__ __forceinline__ bool vnot(bool a) { return !a; }
__device__ __forceinline__ bool vor(bool a, bool b) { return a || b; }
__device__ __forceinline__ bool vand(bool a, bool b) { return a && b; }
__device__ __forceinline__ bool2 vnot(bool2 a) { return {!a.x, !a.y}; }
__device__ __forceinline__ bool2 vor(bool2 a, bool2 b) { return {a.x || b.x, a.y || b.y}; }
__device__ __forceinline__ bool2 vand(bool2 a, bool2 b) { return {a.x && b.x, a.y && b.y}; }

__device__ __forceinline__ float vsel(bool c, float a, float b) { return c ? a : b; }
__device__ __forceinline__ float2 vsel(bool2 c, float2 a, float2 b) {
  return make_float2(c.x ? a.x : b.x, c.y ? a.y : b.y);
}

__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float2 vabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }

// minimum and maximum of two non-NaN values (one min / max instruction; a select on a
// comparison would also order NaNs); magnitude of a with the sign bit of b
__device__ __forceinline__ float vmin(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float2 vmin(float2 a, float2 b) {
  return make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
}
__device__ __forceinline__ float vmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float2 vmax(float2 a, float2 b) {
  return make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
}
__device__ __forceinline__ float vcopysign(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ float2 vcopysign(float2 a, float2 b) {
  return make_float2(copysignf(a.x, b.x), copysignf(a.y, b.y));
}

// ---- hardware seeds (rcp.approx / rsqrt.approx, flush-to-zero) ----------------------------
__device__ __forceinline__ float vrcp(float a) { return rcp_approx_f32(a); }
__device__ __forceinline__ float vrsqrt(float a) { return rsqrt_approx_f32(a); }
__device__ __forceinline__ float2 vrcp(float2 a) {
  return make_float2(rcp_approx_f32(a.x), rcp_approx_f32(a.y));
}
__device__ __forceinline__ float2 vrsqrt(float2 a) {
  return make_float2(rsqrt_approx_f32(a.x), rsqrt_approx_f32(a.y));
}

// lane type of a predicate
template <typename V> struct lanes_of;
template <> struct lanes_of<float> { using B = bool; };
template <> struct lanes_of<float2> { using B = bool2; };

}  // namespace ak
