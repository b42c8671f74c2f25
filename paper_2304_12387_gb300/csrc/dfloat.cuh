// Double-float arithmetic: a value is the unevaluated sum hi + lo of two FP32
// numbers with |lo| < ulp(hi), about 48 significant bits. On this GPU the FP32
// pipe issues 64 lanes for every FP64 lane, so the element contractions of the
// FP64 operator run several times faster in double-float while staying within
// the FP64 parity tolerance. The error-free transformations are the classical
// ones: Knuth's TwoSum, Dekker's FastTwoSum and the FMA-based exact product
// (see Joldes, Muller, Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 2017). Conversions from
// FP64 split the bit pattern with integer operations only, because FP64<->FP32
// conversions execute on the slow FP64 pipe.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct __align__(8) dfloat {
  float hi, lo;
  dfloat() = default;
  __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ constexpr dfloat(float v) : hi(v), lo(0.f) {}
  // explicit FP64 conversions (device: the integer split below; see df_from_double)
  __device__ explicit dfloat(double v);
  __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

// s + e = a + b exactly (Knuth TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
// s + e = a + b exactly when |a| >= |b| (Dekker FastTwoSum)
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {
  float s = a + b;
  return dfloat(s, b - (s - a));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e += a.lo + b.lo;
  return fast_two_sum(s, e);
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }

// exact product of the high parts plus the cross terms (lo*lo is below the format's precision)
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// a*b + c
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) {
  float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  two_sum(c.hi, p, s, t);
  t += c.lo + e;
  return fast_two_sum(s, t);
}

// FP64 -> double-float with integer operations: hi takes the top 24 significant
// bits (truncated), lo the next 24 of the remaining 29 (truncated); values below
// 2^-126 in magnitude flush to zero. Error <= 2^-47 |x|.
__device__ __forceinline__ dfloat df_from_double(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int E = (int)((b >> 52) & 0x7FF);
  const uint64_t M = b & ((1ull << 52) - 1);
  const int eh = E - 1023 + 127;
  if (eh <= 0) return dfloat(0.f, 0.f);
  if (eh >= 255) return dfloat(__int_as_float((int)(sign | 0x7F800000u)), 0.f);
  const float hi = __uint_as_float(sign | ((uint32_t)eh << 23) | (uint32_t)(M >> 29));
  const uint32_t R = (uint32_t)(M & ((1u << 29) - 1));
  if (R == 0) return dfloat(hi, 0.f);
  const int p = 31 - __clz(R);                 // leading one of R, 0..28
  const int el = p + E - 1075 + 127;           // exponent of R * 2^(E-1075)
  if (el <= 0) return dfloat(hi, 0.f);
  const uint32_t mant = (p >= 23) ? (R >> (p - 23)) : (R << (23 - p));
  const float lo = __uint_as_float(sign | ((uint32_t)el << 23) | (mant & 0x7FFFFFu));
  return dfloat(hi, lo);
}

// double-float -> FP64: hi + lo (one FP64 add)
__device__ __forceinline__ double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ dfloat::dfloat(double v) : dfloat(df_from_double(v)) {}

// host-side split of a table entry (round-to-nearest hi, remainder in lo)
inline dfloat df_split_host(double v) {
  float h = (float)v;
  return dfloat(h, (float)(v - (double)h));
}

// FP32 -> FP64 exactly with integer operations (zero and FP32 subnormals map to 0,
// inf/NaN keep their class)
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint64_t s = (uint64_t)(b >> 31) << 63;
  const uint32_t e = (b >> 23) & 0xFF, m = b & 0x7FFFFFu;
  if (e == 0) return __longlong_as_double((long long)s);
  if (e == 255) return __longlong_as_double((long long)(s | (0x7FFull << 52) | ((uint64_t)m << 29)));
  return __longlong_as_double((long long)(s | ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)m << 29)));
}

// element-type conversions used by the templated element kernels
template <typename T, typename IO>
struct Cvt;
template <>
struct Cvt<double, double> {
  __device__ static double in(double v) { return v; }
  __device__ static double out(double v) { return v; }
};
template <>
struct Cvt<float, float> {
  __device__ static float in(float v) { return v; }
  __device__ static float out(float v) { return v; }
};
// FP32 arithmetic with FP64 vectors (the inner operator of the mixed-precision
// solve): truncation to 24 bits on the way in, exact on the way out
template <>
struct Cvt<float, double> {
  __device__ static float in(double v) { return df_from_double(v).hi; }
  __device__ static double out(float v) { return f2d_exact(v); }
};
template <>
struct Cvt<dfloat, double> {
  __device__ static dfloat in(double v) { return df_from_double(v); }
  __device__ static double out(dfloat v) { return df_to_double(v); }
};
