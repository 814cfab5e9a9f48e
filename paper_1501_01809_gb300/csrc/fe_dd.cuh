// Double-float ("f32x2") arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers,
// |lo| <= ulp(hi)/2 after normalisation, about 2^-46 relative precision.  Built from the
// error-free transformations TwoSum (Knuth), Fast2Sum (Dekker) and TwoProd via FMA; the
// multiply/add compositions follow the double-word algorithms of Dekker (1971) and
// Joldes-Muller-Popescu (ACM TOMS 2017).
//
// On GB300 the FP32 pipe executes 64x more operations per clock than the FP64 pipe, and
// conversions between FP32 and FP64 run at the FP64 rate, so the conversions of coordinates in
// and of results out are done here with integer bit manipulation (exact) instead.
#pragma once
#include <stdint.h>

namespace fe {

struct f2 {
  float hi, lo;
};

// All additions and products of the error-free transformations use the _rn intrinsics, which the
// compiler never contracts into FMAs (a contraction would break the exactness of the error terms).
__device__ __forceinline__ f2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, err};
}

__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// Split of an FP64 value into hi + lo with integer operations: hi = the leading 24 significand
// bits (truncated), lo = the remaining 29 bits rounded to FP32, so hi + lo carries at least 48
// significant bits.  |x| < 2^-126 gives (+-0, 0), |x| >= 2^128 gives +-inf; lo is dropped for
// |x| < 2^-74.
__device__ __forceinline__ f2 f2_from_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
  if (e < 1023 - 126) return {__uint_as_float(sign), 0.0f};
  if (e > 1023 + 127) return {__uint_as_float(sign | 0x7F800000u), 0.0f};
  const float hi = __uint_as_float(sign | ((uint32_t)(e - 1023 + 127) << 23) | (uint32_t)(m >> 29));
  const uint32_t rem = (uint32_t)(m & 0x1FFFFFFFull);  // 29 bits below hi's last bit
  float lo = 0.0f;
  const int le = e - 1023 - 52 + 127;  // FP32 exponent field of 2^(e - 1075)
  if (rem != 0 && le >= 1) {
    // rem = a*2^14 + b, both pieces converted exactly through the 2^23 mantissa trick
    const float fa = __uint_as_float(0x4B000000u | (rem >> 14)) - 8388608.0f;
    const float fb = __uint_as_float(0x4B000000u | (rem & 0x3FFFu)) - 8388608.0f;
    lo = fmaf(fa, 16384.0f, fb) * __uint_as_float((uint32_t)le << 23);
    if (sign) lo = -lo;
  }
  return {hi, lo};
}

// Nearest-or-adjacent FP64 value of hi + lo built with integer operations only (no FP64 or
// conversion-unit instructions): the FP64 significand of hi plus lo expressed in units of
// hi's FP64 ulp, renormalised when the sum crosses a binade.  Error <= 1 ulp of FP64.
// hi == 0 gives +-0; subnormal hi (|hi| < 2^-126) is flushed to zero.
// Requires a normalised pair (|lo| <= ulp(hi)/2), which every pair operation returns: a pair
// straight from f2_from_f64 (truncated hi, lo up to one ulp of hi) must pass through one first.
__device__ __forceinline__ double f2_to_f64(float hi, float lo) {
  const uint32_t hb = __float_as_uint(hi);
  const int eh = (int)((hb >> 23) & 0xFF);
  const unsigned long long sign = (unsigned long long)(hb >> 31) << 63;
  if (eh == 0) return __longlong_as_double((long long)sign);
  if (eh == 0xFF) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | ((unsigned long long)(hb & 0x7FFFFF) << 29)));
  long long S = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;  // hi = S * 2^(eh - 127 - 52)
  // t = round(lo / 2^(eh-179)) in two exact steps through the 1.5*2^23 rounding constant:
  // t1 in units of 2^(eh-173) (|t1| <= 2^22), then the remainder in units of 2^(eh-179).
  if (eh >= 52) {  // |hi| >= 2^-75; below that lo (< 2^-99 |hi| relative 2^-24) is dropped
    const float sc1 = __uint_as_float((uint32_t)(300 - eh) << 23);  // 2^(173 - eh)
    const float r1 = fmaf(lo, sc1, 12582912.0f);
    const int t1 = __float_as_int(r1) - 0x4B400000;
    const float rem = fmaf(-(float)t1, __uint_as_float((uint32_t)(eh - 46) << 23), lo);  // lo - t1*2^(eh-173), exact
    const float r2 = fmaf(rem, __uint_as_float((uint32_t)(306 - eh) << 23), 12582912.0f);  // units 2^(eh-179)
    const int t2 = __float_as_int(r2) - 0x4B400000;
    long long t = (long long)t1 * 64 + t2;
    S += (hb >> 31) ? -t : t;
  }
  int ed = eh - 127 + 1023;
  if (S < (1ll << 52)) {
    S <<= 1;
    ed -= 1;
  } else if (S >= (1ll << 53)) {
    S >>= 1;
    ed += 1;
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)ed << 52) | ((unsigned long long)S & 0xFFFFFFFFFFFFFull)));
}

// Arithmetic policy for the generated element kernels (see OpsF64 in fe_ops.cuh).  Constants c
// are FP64 literals split at compile time into (float)c + (float)(c - (float)c).
struct OpsF32x2 {
  using T = f2;
  static __device__ __forceinline__ T zero() { return {0.0f, 0.0f}; }
  static __device__ __forceinline__ T neg(T a) { return {-a.hi, -a.lo}; }
  static __device__ __forceinline__ T add(T a, T b) {
    f2 s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
  }
  static __device__ __forceinline__ T mul(T a, T b) {
    float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return fast_two_sum(p, e);
  }
  static __device__ __forceinline__ T mulc(T a, double c) {
    const float ch = (float)c, cl = (float)(c - (double)ch);
    float p = __fmul_rn(a.hi, ch);
    float e = fmaf(a.hi, ch, -p);
    e = fmaf(a.hi, cl, e);
    e = fmaf(a.lo, ch, e);
    return fast_two_sum(p, e);
  }
  static __device__ __forceinline__ T fmac(T a, double c, T acc) {
    const float ch = (float)c, cl = (float)(c - (double)ch);
    float p = __fmul_rn(a.hi, ch);
    float e = fmaf(a.hi, ch, -p);
    e = fmaf(a.hi, cl, e);
    e = fmaf(a.lo, ch, e);
    f2 s = two_sum(acc.hi, p);
    float t = __fadd_rn(s.lo, __fadd_rn(acc.lo, e));
    return fast_two_sum(s.hi, t);
  }
  static __device__ __forceinline__ T fma3(T a, T b, T c) { return add(mul(a, b), c); }
  static __device__ __forceinline__ T from_f64(double x) { return f2_from_f64(x); }
  static __device__ __forceinline__ T diff_f64(double a, double b) { return add(f2_from_f64(a), neg(f2_from_f64(b))); }
  static __device__ __forceinline__ double to_f64(T x) { return f2_to_f64(x.hi, x.lo); }
  static __device__ __forceinline__ float sign_of(T x) { return x.hi; }
  // 1/x with one Newton step in double-float (x.hi != 0)
  static __device__ __forceinline__ T recip(T x) {
    float r = __frcp_rn(x.hi);
    // e = 1 - x*r in double-float, r1 = r + r*e
    f2 xr = mul(x, {r, 0.0f});
    f2 e = add({1.0f, 0.0f}, neg(xr));
    f2 re = mul({r, 0.0f}, e);
    return add({r, 0.0f}, re);
  }
  static __device__ __forceinline__ T abs(T x) { return x.hi < 0.0f ? neg(x) : x; }
  static __device__ __forceinline__ T scale(T x, float s) { return {__fmul_rn(x.hi, s), __fmul_rn(x.lo, s)}; }  // s a power of two
  // FP32's exponent range is narrow: the geometry normalises each cell's edge vectors
  static constexpr bool kNormalise = true;
  static __device__ __forceinline__ int exponent(T x) {
    const int e = (int)((__float_as_uint(x.hi) >> 23) & 0xFF);
    return e == 0 ? -1000 : e - 127;
  }
  // x * 2^k, exact, for results inside the normal range; k split in two steps of |k| <= 126
  static __device__ __forceinline__ T ldexp2(T x, int k) {
    const int k1 = k / 2, k2 = k - k1;
    const float s1 = __uint_as_float((uint32_t)(k1 + 127) << 23), s2 = __uint_as_float((uint32_t)(k2 + 127) << 23);
    return {__fmul_rn(__fmul_rn(x.hi, s1), s2), __fmul_rn(__fmul_rn(x.lo, s1), s2)};
  }
};

// Single FP32 element tensors (the precision study of the high-order elements): inputs rounded
// to FP32 once per cell, all element arithmetic in FP32, results widened to FP64 exactly (integer
// bit construction) for the FP64 global accumulation.
__device__ __forceinline__ double f32_to_f64_exact(float x) {
  const uint32_t b = __float_as_uint(x);
  const int e = (int)((b >> 23) & 0xFF);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  if (e == 0) return __longlong_as_double((long long)sign);  // zero (subnormals flushed)
  if (e == 0xFF) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull | ((unsigned long long)(b & 0x7FFFFF) << 29)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e + 896) << 52) | ((unsigned long long)(b & 0x7FFFFF) << 29)));
}

struct OpsF32 {
  using T = float;
  static __device__ __forceinline__ T zero() { return 0.0f; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T mulc(T a, double c) { return a * (float)c; }
  static __device__ __forceinline__ T fmac(T a, double c, T acc) { return fmaf(a, (float)c, acc); }
  static __device__ __forceinline__ T fma3(T a, T b, T c) { return fmaf(a, b, c); }
  static __device__ __forceinline__ T from_f64(double x) { return f2_from_f64(x).hi + f2_from_f64(x).lo; }
  static __device__ __forceinline__ T diff_f64(double a, double b) { return from_f64(a) - from_f64(b); }
  static __device__ __forceinline__ double to_f64(T x) { return f32_to_f64_exact(x); }
  static __device__ __forceinline__ T recip(T x) { return __frcp_rn(x); }
  static __device__ __forceinline__ T abs(T x) { return fabsf(x); }
  static __device__ __forceinline__ T scale(T x, float s) { return x * s; }
  static constexpr bool kNormalise = true;
  static __device__ __forceinline__ int exponent(T x) {
    const int e = (int)((__float_as_uint(x) >> 23) & 0xFF);
    return e == 0 ? -1000 : e - 127;
  }
  static __device__ __forceinline__ T ldexp2(T x, int k) {
    const int k1 = k / 2, k2 = k - k1;
    return x * __uint_as_float((uint32_t)(k1 + 127) << 23) * __uint_as_float((uint32_t)(k2 + 127) << 23);
  }
};

}  // namespace fe
