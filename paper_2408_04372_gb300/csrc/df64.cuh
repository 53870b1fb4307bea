// Double-float arithmetic on the FP32 pipe: a value is the unevaluated sum hi + lo of two
// floats (about 44 significand bits).  GB300 issues FP32 at 64x its FP64 rate, so the
// FP64-accuracy operator apply of the outer Krylov method runs in this arithmetic.
//
// Building blocks are the error-free transformations of Knuth (TwoSum: a + b = s + e
// exactly, six additions) and of the FMA (TwoProd: a * b = p + e exactly), with Dekker's
// Fast2Sum (|s| >= |e|) to renormalise.  A product is left unnormalised (its low part is
// at most about 2^-23 of its high part); every sum is renormalised.  Relative error per
// operation is about 2^-44 of the operands' magnitudes.  All roundings are explicit
// (__fadd_rn, __fmul_rn, __fmaf_rn): the compiler must not merge a product into a sum
// here, which would break the exactness of TwoSum and TwoProd.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace stmg {

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr df64(float h) : hi(h), lo(0.0f) {}
};

// Nearest double-float to x (host, for tables and geometry).
inline df64 df_split(double x) {
  const float h = (float)x;
  return df64(h, (float)(x - (double)h));
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return df64(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ df64 df_mul(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df64(p, e);
}

__device__ __forceinline__ df64 df_mul(df64 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df64(p, e);
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) { return df_add(a, b); }
__device__ __forceinline__ df64 operator*(df64 a, df64 b) { return df_mul(a, b); }
__device__ __forceinline__ df64 operator*(df64 a, float b) { return df_mul(a, b); }
__device__ __forceinline__ df64& operator+=(df64& a, df64 b) {
  a = df_add(a, b);
  return a;
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// Conversions between FP64 and FP32 formed from the bit fields with integer and FP32 instructions:
// on GB300 every FP64 instruction, conversions included, runs on the slow FP64 pipe (1/64 of FP32).
// Exact float -> double for zero and normal floats (others through the FP64 conversion).
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  const uint64_t sgn = (uint64_t)(u & 0x80000000u) << 32;
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sgn);
  if (e == 0u || e == 0xffu) return (double)f;
  return __longlong_as_double((long long)(sgn | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(u & 0x7fffffu) << 29)));
}
// Nearest double-float to x: hi = x rounded to 24 bits (to nearest, ties to even), lo = the remainder
// (at most 29 bits) rounded to float by one integer conversion and scaled by an exact power of two.
// Exponents for which hi or lo would leave the normal float range, zero, and non-finite values take
// the FP64 path.
__device__ __forceinline__ df64 df_split_fast(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E < 949 || E > 1149) {
    const float h = __double2float_rn(x);
    return df64(h, __double2float_rn(x - (double)h));
  }
  const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
  const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);  // 53-bit significand
  uint32_t hm = (uint32_t)(m >> 29);                           // leading 24 bits
  const uint32_t r = (uint32_t)(m & ((1u << 29) - 1));         // trailing 29 bits
  int32_t rem = (int32_t)r;
  if (r > (1u << 28) || (r == (1u << 28) && (hm & 1u))) {
    hm += 1u;
    rem -= (int32_t)(1u << 29);
  }
  int eh = E;
  if (hm == (1u << 24)) {  // rounding carried into the exponent
    hm >>= 1;
    eh += 1;
  }
  const float hi = __uint_as_float(sgn | ((uint32_t)(eh - 896) << 23) | (hm & 0x7fffffu));
  const float scale = __uint_as_float((uint32_t)(E - 1075 + 127) << 23);  // 2^(E - 1075), normal
  const float lo = __fmul_rn(__int2float_rn(rem), scale);
  return df64(hi, sgn ? -lo : lo);
}

// Accumulator of a sum of double-float terms with the renormalisation deferred to the end:
// each term costs TwoSum on the high parts (6 additions) plus 2 additions into the low part,
// instead of a renormalised double-float sum (11 additions).  The low part collects the exact
// TwoSum errors and the terms' low parts; its own rounding is of order 2^-24 of itself, i.e.
// 2^-48 of the sum, which keeps the ~44-bit accuracy of the arithmetic.
struct df_acc {
  float hi, lo;
  df_acc() = default;
  __device__ constexpr df_acc(float h) : hi(h), lo(0.0f) {}
  __device__ constexpr df_acc(df64 v) : hi(v.hi), lo(v.lo) {}
  __device__ __forceinline__ operator df64() const {
    const float h = __fadd_rn(hi, lo);
    return df64(h, __fsub_rn(lo, __fsub_rn(h, hi)));
  }
};
__device__ __forceinline__ df_acc& operator+=(df_acc& a, df64 t) {
  const float s = __fadd_rn(a.hi, t.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(t.hi, bb));
  a.hi = s;
  a.lo = __fadd_rn(a.lo, __fadd_rn(t.lo, e));
  return a;
}

// Accumulator type of a sum in arithmetic T (the type itself except for double-float).
template <typename T> struct acc_of { using type = T; };
template <> struct acc_of<df64> { using type = df_acc; };

}  // namespace stmg
