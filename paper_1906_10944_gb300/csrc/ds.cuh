// Double-single arithmetic on the FP32 pipe: every value a pair of floats
// (hi + lo), products by Dekker's exact product (fused multiply-add) plus the
// two cross terms, sums by Knuth's two-sum (Dekker 1971; Knuth, TAOCP vol.
// 2): about 46 significant bits, against the 53 of FP64.  GB300 issues FP64
// at 1/64 of the FP32 rate, and its FP64 pipe also executes the float/double
// conversions, so the splits and joins below use integer operations.  The
// explicit _rn intrinsics keep the compiler from fusing the two-sums.
#pragma once

#include <cstdint>
#include <type_traits>

namespace geneo {

struct DS {
  float h, l;
};

// acc += a * x for double-single a, x, acc
__device__ __forceinline__ void ds_fma(DS& acc, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = __fmaf_rn(ah, xh, -p);          // p + e = ah xh exactly
  e = __fmaf_rn(ah, xl, e);
  e = __fmaf_rn(al, xh, e);
  const float s = __fadd_rn(acc.h, p);      // two-sum of acc.h and p
  const float bv = __fsub_rn(s, acc.h);
  const float err = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(err, e));
}

// FP64 -> (hi, lo) floats with integer operations only (the FP64 pipe,
// which also executes conversions, is the scarce unit): hi keeps the sign,
// the exponent and the top 23 mantissa bits (truncation), lo the next 23
// of the remaining 29 bits, so hi + lo = x to 2^-46 relative.  Outside
// 2^-80 <= |x| < 2^128 the plain conversion is used and lo = 0 (below 2^-126
// both are 0).
__device__ __forceinline__ float2 split_bits(double x) {
  const uint32_t hi32 = (uint32_t)__double2hiint(x), lo32 = (uint32_t)__double2loint(x);
  const uint32_t sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  if (e < 943 || e > 1150) return make_float2(e >= 897 ? (float)x : 0.f, 0.f);
  const uint32_t mh = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const float h = __uint_as_float(sign | ((uint32_t)(e - 896) << 23) | mh);
  const uint32_t r = (lo32 & 0x1fffffffu) >> 6;                     // < 2^23
  const float f = __fsub_rn(__uint_as_float(0x4B000000u | r), 8388608.0f);  // r exactly
  const float sc = __uint_as_float(sign | ((uint32_t)(e - 942) << 23));     // +-2^(e - 1069)
  return make_float2(h, __fmul_rn(f, sc));
}

// Exact float -> double and round-to-nearest double -> float with integer
// operations for normal numbers and zero (the same results as the
// conversions, which run on the FP64 pipe); anything else converts.
__device__ __forceinline__ double f2d_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if ((u & 0x7fffffffu) == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
  if (e == 0 || e == 255) return (double)f;
  return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)), (int)(u << 29));
}
__device__ __forceinline__ float d2f_bits(double x) {
  const uint32_t hi32 = (uint32_t)__double2hiint(x), lo32 = (uint32_t)__double2loint(x);
  const uint32_t sign = hi32 & 0x80000000u;
  const int e = (int)((hi32 >> 20) & 0x7ffu);
  if (e < 897 || e > 1150) {
    if ((hi32 & 0x7fffffffu) == 0 && lo32 == 0) return __uint_as_float(sign);
    return (float)x;
  }
  uint32_t b = sign | ((uint32_t)(e - 896) << 23) | ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const uint32_t rem = lo32 & 0x1fffffffu;
  if (rem > 0x10000000u || (rem == 0x10000000u && (b & 1u))) ++b;  // nearest, ties to even
  return __uint_as_float(b);
}
template <typename D, typename S>
__device__ __forceinline__ D cv(S v) {
  if constexpr (std::is_same_v<D, S>) return v;
  else if constexpr (std::is_same_v<D, float>) return d2f_bits(v);
  else return f2d_bits(v);
}

// value of an accumulator (double-single pairs summed in FP64)
__device__ __forceinline__ double acc_value(const DS& v) { return f2d_bits(v.h) + f2d_bits(v.l); }
__device__ __forceinline__ double acc_value(double v) { return v; }
__device__ __forceinline__ double acc_value(float v) { return f2d_bits(v); }


// A double-single value with the operators of the band solves (the FP64
// factors of the FP32 mode solved on the FP32 pipe).  Sums are renormalised
// (|l| <= ulp(h) / 2), so a stored value is an accurate multiplicand;
// products keep hi*hi exactly plus the two cross terms.
struct dsv {
  float h, l;
  __device__ __forceinline__ dsv() : h(0.f), l(0.f) {}
  __device__ __forceinline__ dsv(float hh, float ll) : h(hh), l(ll) {}
  __device__ __forceinline__ explicit dsv(double x) {
    const float2 v = split_bits(x);
    h = v.x;
    l = v.y;
  }
};
__device__ __forceinline__ dsv operator+(dsv a, dsv b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bv = __fsub_rn(s, a.h);
  const float err = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bv)), __fsub_rn(b.h, bv));
  const float t = __fadd_rn(err, __fadd_rn(a.l, b.l));
  const float h = __fadd_rn(s, t);
  return dsv(h, __fsub_rn(t, __fsub_rn(h, s)));
}
__device__ __forceinline__ dsv operator-(dsv a) { return dsv(-a.h, -a.l); }
__device__ __forceinline__ dsv operator-(dsv a, dsv b) { return a + (-b); }
__device__ __forceinline__ dsv operator*(dsv a, dsv b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dsv(p, e);
}
__device__ __forceinline__ dsv& operator+=(dsv& a, dsv b) { return a = a + b; }
__device__ __forceinline__ dsv& operator-=(dsv& a, dsv b) { return a = a - b; }
__device__ __forceinline__ dsv& operator*=(dsv& a, dsv b) { return a = a * b; }
__device__ __forceinline__ double to_double(dsv a) { return f2d_bits(a.h) + f2d_bits(a.l); }
__device__ __forceinline__ double to_double(double a) { return a; }
__device__ __forceinline__ double to_double(float a) { return (double)a; }
__device__ __forceinline__ dsv shfl(dsv v, int src) {
  return dsv(__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src));
}
template <typename T>
__device__ __forceinline__ T shfl(T v, int src) { return __shfl_sync(0xffffffffu, v, src); }
// 1 / x of a storage value in arithmetic type A (FP64 division for
// double-single, once per pivot)
template <typename A, typename S>
__device__ __forceinline__ A recip_arith(S x) {
  if constexpr (std::is_same_v<A, dsv>) return dsv(1.0 / (double)x);
  else return A(1) / (A)x;
}
// value of storage type S in arithmetic type A
template <typename A, typename S>
__device__ __forceinline__ A to_arith(S x) {
  if constexpr (std::is_same_v<A, dsv>) return dsv((double)x);
  else return (A)x;
}

}  // namespace geneo
