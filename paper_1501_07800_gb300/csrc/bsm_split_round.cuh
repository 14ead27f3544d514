// Exact recombination of the split kernel's diagonal sums and their one
// rounding to FP64, for C blocks whose products fit in one narrow flush.
//
// A narrow flush leaves every diagonal sum D_d (an integer, |D_d| < 2^22) in
// the FP32 accumulator; adding 1.5 * 2^23 to it is exact and makes its bit
// pattern 0x4B400000 + D_d.  The C entry before scaling is the integer
//   V = sum_d D_d 2^(B (S-1-d)),
// which Horner's rule forms from the bit patterns in wrapping 64-bit
// arithmetic, the offsets of the S patterns removed by one subtraction of a
// constant: V mod 2^64 is exact, and it is V itself when |V| < 2^63, which
// `narrow_fits_int64` establishes from the digit bounds (otherwise the kernel
// uses its general 128-bit path).  V 2^X is then rounded once to the nearest
// double (ties to even) by normalising V's magnitude to bit 63: the top 53
// bits are the significand, the low 11 decide the rounding.
#pragma once

#include <stdint.h>

__host__ __device__ __forceinline__ int clz64_u(uint64_t x) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)x);
#else
  return x ? __builtin_clzll(x) : 64;
#endif
}

__host__ __device__ __forceinline__ double bits_to_double(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  __builtin_memcpy(&d, &b, 8);
  return d;
#endif
}

// sum_d 0x4B400000 2^(B (S-1-d)) mod 2^64: the offsets Horner's rule picks up
// from the bit patterns.
template <int S, int B>
__host__ __device__ constexpr uint64_t narrow_offset() {
  uint64_t w = 0;
  for (int d = 0; d < S; d++) w = (w << B) + 0x4B400000ull;
  return w;
}

// V = sum_d D_d 2^(B (S-1-d)) from pat[d] = bits(D_d + 1.5 * 2^23), exact
// whenever |V| < 2^63.
template <int S, int B>
__host__ __device__ __forceinline__ int64_t narrow_combine(const uint32_t (&pat)[S]) {
  uint64_t v = pat[0];
#pragma unroll
  for (int d = 1; d < S; d++) v = (v << B) + pat[d];
  return (int64_t)(v - narrow_offset<S, B>());
}

// Whether |V| < 2^63 is guaranteed for one narrow flush of at most n inner
// elements: the leading digits are at most 2^B in magnitude and the others
// 2^(B-1), so D_0 <= n 2^(2B) and D_d <= n (d+1) 2^(2B-1) for d >= 1 (one
// leading digit in each of two terms, the rest below); the check is made in
// units of n 2^(2B) 2^(B (S-1)) with a margin.
template <int S, int B>
__host__ __device__ constexpr bool narrow_fits_int64(int n) {
  // bound / (n 2^(2B + B (S-1))) = 1 + sum_{d>=1} (d+1) 2^-1 2^(-B d)
  double f = 1.0, p = 1.0;
  for (int d = 1; d < S; d++) {
    p /= (double)(1 << B);
    f += 0.5 * (d + 1) * p;
  }
  double lg = 2.0 * B + (double)B * (S - 1);  // log2 of 2^(2B + B(S-1))
  double bound = (double)n * f;
  for (int i = 0; i < (int)lg; i++) bound *= 2.0;
  return bound < 9.0e18;  // below 2^63 = 9.22e18 with margin
}

// Most inner elements of one narrow flush: the kernel's narrow flush group
// keeps n 2^(2B) (d = 0) and n (S+2) 2^(2B-2) (the largest d) below 2^22.
template <int S, int B>
__host__ __device__ constexpr int narrow_max_elems() {
  const int a = (1 << 22) >> (2 * B), b = ((1 << 22) >> (2 * B - 2)) / (S + 2);
  return a < b ? a : b;
}

// Most block products (of BS inner elements each) of one narrow flush for
// which |V| < 2^63 is guaranteed: the largest n = products * BS that passes
// narrow_fits_int64, capped by the narrow flush itself.
template <int S, int B, int BS>
__host__ __device__ constexpr int narrow_int64_products() {
  int k = 0;
  while ((k + 1) * BS <= narrow_max_elems<S, B>() && narrow_fits_int64<S, B>((k + 1) * BS)) k++;
  return k;
}

// Correctly rounded v 2^X (to nearest, ties to even) when the result is a
// normal double; false otherwise (zero is returned as +0.0 and true).
__host__ __device__ __forceinline__ bool int64_scaled_to_double(int64_t v, int X, double &out) {
  if (v == 0) {
    out = 0.0;
    return true;
  }
  const uint64_t sign = (uint64_t)v & (1ull << 63);
  const uint64_t u = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
  const int lz = clz64_u(u);
  const uint64_t nrm = u << lz;            // leading one at bit 63
  uint64_t q = nrm >> 11;                  // 53 bits, the leading one at bit 52
  const uint32_t rb = (uint32_t)nrm & 0x7FFu;
  q += (rb + (uint32_t)(q & 1u)) > 0x400u ? 1u : 0u;
  const int be = (63 - lz) + X + 1023;     // biased exponent of u 2^X
  if (be < 1 || be > 2045) return false;
  // a carry out of the significand (q = 2^53) raises the exponent by itself
  out = bits_to_double(sign | ((((uint64_t)(be - 1)) << 52) + q));
  return true;
}
