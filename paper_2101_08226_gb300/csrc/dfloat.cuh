// Double-float numbers: an unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2, about 48
// significant bits, computed on the FP32 pipes.  On this part a warp's FP64 instruction occupies the
// SM's FP64 unit for about 19 cycles while FP32 runs 64 times faster, so a double-float operation of
// 7 to 15 FP32 instructions is several times cheaper than its FP64 counterpart.
//
// Written from the published error-free transformations:
//   TwoSum      (Knuth, TAOCP vol. 2, 4.2.2):  s + e = a + b exactly, 6 additions;
//   Fast2Sum    (Dekker 1971), |a| >= |b|:     s + e = a + b exactly, 3 additions;
//   TwoProduct  with FMA (Ogita, Rump, Oishi 2005):  p + e = a b exactly, 2 instructions.
// Sum and product are the "sloppy" double-float forms: the error of a + b is below about 2^-44
// (|a| + |b|), of a b below about 2^-44 |a b|.  Exponent range is that of float.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace octofmm {

// Conversions between float and double from the bit patterns, with integer operations only (a
// conversion instruction runs on the FP64 pipe, as slow as an FP64 multiply here).
// float -> double, exact for every float (zeros, subnormals, infinities, NaNs included).
__device__ __forceinline__ double df_f2d(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint64_t sign = uint64_t(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  // subnormal m 2^-149: leading bit at position p, exponent p - 149
  const int p = 31 - __clz(int(m | 1u));
  const uint64_t sub = (uint64_t(1023 + p - 149) << 52) | ((uint64_t(m) << (52 - p)) & ((1ull << 52) - 1));
  const uint64_t norm = (uint64_t(e == 255u ? 2047u : e + 896u) << 52) | (uint64_t(m) << 29);
  const uint64_t mag = e == 0u ? (m == 0u ? 0ull : sub) : norm;
  return __longlong_as_double(int64_t(sign | mag));
}
// double -> float by truncating the mantissa to 24 bits; magnitudes below the smallest normal
// float give a signed zero (double-float covers the float range only).
__device__ __forceinline__ float df_d2f_trunc(double d) {
  const uint64_t b = uint64_t(__double_as_longlong(d));
  const uint32_t sign = uint32_t(b >> 63) << 31;
  const int e = int((b >> 52) & 0x7ffu) - 896;
  const uint32_t m = uint32_t(b >> 29) & 0x7fffffu;
  const uint32_t mag = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : (uint32_t(e) << 23) | m);
  return __uint_as_float(sign | mag);
}

struct dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(int v) : hi(float(v)), lo(0.0f) {}  // exact for |v| < 2^24
  // the nearest float, then the nearest float of the remainder (exact for doubles of <= 48 bits)
  __host__ __device__ constexpr dfloat(double d) : hi(float(d)), lo(float(d - double(float(d)))) {}
  __host__ __device__ explicit operator double() const {
#ifdef __CUDA_ARCH__
    return df_f2d(hi) + df_f2d(lo);
#else
    return double(hi) + double(lo);
#endif
  }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

// A double as hi + lo: hi its leading 24 bits, lo the remainder's leading 24 bits (one FP64
// subtraction, exact; the rest integer operations).
__device__ __forceinline__ dfloat df_from_double(double d) {
  const float hi = df_d2f_trunc(d);
  return dfloat(hi, df_d2f_trunc(d - df_f2d(hi)));
}

__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return dfloat(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b) {
  const float s = a + b;
  return dfloat(s, b - (s - a));
}
__device__ __forceinline__ dfloat df_two_prod(float a, float b) {
  const float p = a * b;
  return dfloat(p, fmaf(a, b, -p));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  const dfloat s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  const dfloat p = df_two_prod(a.hi, b.hi);
  return df_fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
// a b + c with one renormalisation
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
  const dfloat p = df_two_prod(a.hi, b.hi);
  const float e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo));
  const dfloat s = df_two_sum(p.hi, c.hi);
  return df_fast_two_sum(s.hi, s.lo + (e + c.lo));
}
// a / b: a float quotient, corrected once by the double-float remainder a - q b
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b) {
  const float q1 = a.hi / b.hi;
  const dfloat r = a - dfloat(q1, 0.0f) * b;
  return df_fast_two_sum(q1, r.hi / b.hi);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }
__device__ __forceinline__ bool operator>(dfloat a, dfloat b) {
  return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo);
}
__device__ __forceinline__ bool operator<(dfloat a, dfloat b) { return b > a; }

// 1 / sqrt(a): the float estimate y, then two Newton steps y + y (1 - a y^2) / 2, each residual
// formed in double-float and each small correction in float (the first step leaves about 2^-43,
// the second the double-float rounding).
__device__ __forceinline__ dfloat df_rsqrt(dfloat a) {
  const float y = rsqrtf(a.hi);
  const dfloat r1 = dfloat(1) - a * df_two_prod(y, y);
  const dfloat y1 = df_fast_two_sum(y, 0.5f * y * r1.hi);
  const dfloat r2 = dfloat(1) - a * (y1 * y1);
  return y1 + dfloat(0.5f * y1.hi * r2.hi, 0.0f);
}

}  // namespace octofmm
