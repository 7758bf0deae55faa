// Pair-of-floats arithmetic ("double-float"): a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi) / 2; the pair holds 48
// significant bits and each operation below is within ~2^-46 relative.
// Built from the error-free transformations: Knuth's two-sum (exact sum of
// two floats as a pair), the fast two-sum for |a| >= |b| (Dekker 1971) and
// the exact product by one fused multiply-add.
//
// GB300 issues FP32 lane operations at 64 times its FP64 rate, so work that
// needs more than FP32 but not the full FP64 significand (a harmonic
// recurrence whose results are within 1e-14 relative of FP64) runs here on
// the FP32 pipe.  No fast-math flags: the transformations rely on IEEE
// rounding of every operation and on no reassociation.
//
// Conversions to and from double use integer operations only (no FP64
// instruction), with an exact power-of-two scale folded into the exponent.
#pragma once
#include <cstdint>

struct f2 {
  float h, l;
};

__device__ __forceinline__ f2 f2_make(float h) { return {h, 0.0f}; }

__device__ __forceinline__ f2 f2_fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

__device__ __forceinline__ f2 f2_two_sum(float a, float b) {
  const float s = a + b;
  const float v = s - a;
  return {s, (a - (s - v)) + (b - v)};
}

__device__ __forceinline__ f2 f2_neg(f2 a) { return {-a.h, -a.l}; }

__device__ __forceinline__ f2 f2_add(f2 a, f2 b) {
  const f2 s = f2_two_sum(a.h, b.h);
  return f2_fast_two_sum(s.h, s.l + (a.l + b.l));
}

__device__ __forceinline__ f2 f2_mul(f2 a, f2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return f2_fast_two_sum(p, e);
}

// a * b - c * d (one renormalisation)
__device__ __forceinline__ f2 f2_mul_sub(f2 a, f2 b, f2 c, f2 d) {
  const float p = a.h * b.h, q = c.h * d.h;
  const float e1 = fmaf(a.h, b.h, -p);
  const float e2 = fmaf(c.h, d.h, -q);
  const f2 s = f2_two_sum(p, -q);
  float t = s.l + (e1 - e2);
  t = fmaf(a.h, b.l, t);
  t = fmaf(a.l, b.h, t);
  t = fmaf(-c.h, d.l, t);
  t = fmaf(-c.l, d.h, t);
  return f2_fast_two_sum(s.h, t);
}

// a * b + c * d
__device__ __forceinline__ f2 f2_mul_add(f2 a, f2 b, f2 c, f2 d) { return f2_mul_sub(a, b, f2_neg(c), d); }

// one Newton step for 1 / sqrt(a): y + y (1 - a y^2) / 2 (the relative
// error e goes to ~ 3 e^2 / 2)
__device__ __forceinline__ f2 f2_rsqrt_step(f2 a, f2 y) {
  const f2 r = f2_add(f2_make(1.0f), f2_neg(f2_mul(a, f2_mul(y, y))));
  const f2 c = f2_mul(y, r);
  return f2_add(y, {0.5f * c.h, 0.5f * c.l});
}

// 1 / sqrt(a) for a > 0 (normal): the FP32 estimate and two Newton steps
__device__ __forceinline__ f2 f2_rsqrt(f2 a) {
  return f2_rsqrt_step(a, f2_rsqrt_step(a, f2_make(rsqrtf(a.h))));
}

__device__ __forceinline__ f2 f2_shfl_up(f2 v, int d, int width) {
  return {__shfl_up_sync(0xffffffffu, v.h, d, width), __shfl_up_sync(0xffffffffu, v.l, d, width)};
}

__device__ __forceinline__ f2 f2_shfl(f2 v, int src, int width) {
  return {__shfl_sync(0xffffffffu, v.h, src, width), __shfl_sync(0xffffffffu, v.l, src, width)};
}

__device__ __forceinline__ f2 f2_sel(bool c, f2 a, f2 b) { return c ? a : b; }

// x * 2^e as a pair, by integer operations on the bits of x: hi takes the
// top 24 significant bits of x (rounded toward zero), lo the next 24 (the
// remaining 5 bits are dropped, 2^-48 relative).  Results below the
// smallest normal float are flushed to zero; |x 2^e| must stay below 2^127.
__device__ __forceinline__ f2 f2_from_double(double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int ex = (int)((b >> 52) & 0x7ffu) - 1023 + e;  // unbiased exponent of x 2^e
  const unsigned long long frac = b & 0xfffffffffffffull;
  f2 r = {0.0f, 0.0f};
  if (((b >> 52) & 0x7ffu) != 0u && ex >= -126) {
    const unsigned hf = (unsigned)(frac >> 29);  // 23 fraction bits
    r.h = __int_as_float((int)(sign | ((unsigned)(ex + 127) << 23) | hf));
    const unsigned rem = (unsigned)(frac & 0x1fffffffull);  // 29 bits, weight 2^(ex-52)
    if (rem != 0u) {
      // rem's top 24 bits as a float (toward zero), times 2^(ex - 52)
      const int sh = __clz(rem) - 3;  // rem < 2^29: leading bit at 28 - (clz - 3)
      const int top = 28 - sh;        // position of rem's leading bit
      const int le = ex - 52 + top;   // unbiased exponent of lo
      if (le >= -126) {
        unsigned mant;
        if (top >= 23)
          mant = (rem >> (top - 23)) & 0x7fffffu;
        else
          mant = (rem << (23 - top)) & 0x7fffffu;
        r.l = __int_as_float((int)(sign | ((unsigned)(le + 127) << 23) | mant));
      }
    }
  }
  return f2_fast_two_sum(r.h, r.l);
}

// float f times 2^e as a double, by integer operations (f normal or zero;
// the exponent of the result must stay inside the double range)
__device__ __forceinline__ double float_scaled_to_double(float f, int e) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0u) return 0.0;
  const unsigned long long sign = (unsigned long long)(u >> 31) << 63;
  const unsigned long long de = (unsigned long long)((int)ef - 127 + 1023 + e);
  const unsigned long long mant = (unsigned long long)(u & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | (de << 52) | mant));
}

// (hi + lo) 2^e as a double: the two exact conversions and one FP64 add
__device__ __forceinline__ double f2_to_double(f2 a, int e) {
  return float_scaled_to_double(a.h, e) + float_scaled_to_double(a.l, e);
}

// IEEE-754 conversions on the integer pipe (the FP64 pipe is 1/64 rate).
// float -> double is exact for normal floats; subnormal floats become 0.
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t sign = b & 0x80000000u;
  const uint32_t hi = e ? (sign | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)) : sign;
  const uint32_t lo = e ? (b << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
// double -> float rounded to nearest (ties to even), as the IEEE
// conversion; a result beyond the float range saturates to +-inf, an input
// below the smallest normal float flushes to 0 (branch-free).  The 29
// dropped significand bits decide the rounding; a carry out of the
// significand moves into the exponent, as IEEE rounding does.
__device__ __forceinline__ float d2f_int(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  uint32_t mag = ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  const uint32_t rem = lo & 0x1fffffffu, half = 0x10000000u;
  mag += (rem > half || (rem == half && (mag & 1u))) ? 1u : 0u;
  mag = (e <= 0) ? 0u : mag;
  mag = (e >= 255 || mag > 0x7f800000u) ? 0x7f800000u : mag;
  return __uint_as_float((hi & 0x80000000u) | mag);
}
