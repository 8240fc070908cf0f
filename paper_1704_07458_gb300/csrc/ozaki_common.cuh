// Integer-only conversions between the double-float accumulators of the
// tensor-core FP64 emulation and IEEE FP64 (no FP64 arithmetic).
#pragma once
#include <cstdint>

namespace lob {

// (sign, integer mantissa, exponent) of a float: f = m * 2^e exactly.
__device__ __forceinline__ void float_parts(float f, long long& m, int& e) {
  const unsigned b = __float_as_uint(f);
  const int be = (b >> 23) & 0xFF;
  long long mm = b & 0x7FFFFF;
  if (be != 0) mm |= 0x800000;
  e = (be == 0 ? 1 : be) - 150;
  m = (b >> 31) ? -mm : mm;
}

__device__ __forceinline__ void double_parts(double x, long long& m, int& e) {
  const long long b = __double_as_longlong(x);
  const int be = (int)((b >> 52) & 0x7FF);
  long long mm = b & 0x000FFFFFFFFFFFFFLL;
  if (be != 0) mm |= 0x0010000000000000LL;
  e = (be == 0 ? 1 : be) - 1075;
  m = b < 0 ? -mm : mm;
}

__device__ __forceinline__ int bitlen(long long m) {
  const unsigned long long a = m < 0 ? (unsigned long long)(-m) : (unsigned long long)m;
  return a == 0 ? 0 : 64 - __clzll(a);
}

// Round an int64 value v * 2^e to the nearest double (ties to even), integer ops only.
__device__ __forceinline__ double int_to_double(long long v, int e) {
  if (v == 0) return 0.0;
  unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const unsigned long long sign = v < 0 ? 0x8000000000000000ULL : 0ULL;
  const int lz = __clzll(a);
  const int top = 63 - lz;      // index of the leading bit
  int exp2 = e + top;           // value in [2^exp2, 2^(exp2+1))
  unsigned long long mant;
  if (top > 52) {
    const int r = top - 52;
    const unsigned long long half = 1ULL << (r - 1);
    const unsigned long long rem = a & ((1ULL << r) - 1);
    mant = a >> r;
    if (rem > half || (rem == half && (mant & 1))) {
      ++mant;
      if (mant >> 53) {
        mant >>= 1;
        ++exp2;
      }
    }
  } else {
    mant = a << (52 - top);
  }
  if (exp2 > 1023) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ULL));
  if (exp2 < -1022) {  // subnormal result: shift further (rare; truncates)
    const int r = -1022 - exp2;
    if (r > 53) return __longlong_as_double((long long)sign);
    mant >>= r;
    return __longlong_as_double((long long)(sign | mant));
  }
  const unsigned long long bits =
      sign | ((unsigned long long)(exp2 + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFULL);
  return __longlong_as_double((long long)bits);
}

// The same rounding for the common case of a normal result: one normalising
// shift, and an integer add that carries a rounded-up mantissa into the
// exponent field; zero, overflow and subnormal results take the path above.
__device__ __forceinline__ double int_to_double_fast(long long v, int e) {
  const unsigned long long a = v < 0 ? 0ULL - (unsigned long long)v : (unsigned long long)v;
  if (a == 0) return 0.0;
  const int lz = __clzll(a);
  const int exp2 = e + 63 - lz;  // value in [2^exp2, 2^(exp2+1))
  if (exp2 > 1022 || exp2 < -1022) return int_to_double(v, e);
  const unsigned long long m = a << lz;  // leading one at bit 63
  const unsigned long long mant = m >> 11;  // 53 bits, leading one at bit 52
  const unsigned long long rest = m & 0x7FFULL;
  const unsigned long long up = (rest > 0x400ULL || (rest == 0x400ULL && (mant & 1ULL))) ? 1ULL : 0ULL;
  const unsigned long long bits = ((unsigned long long)(exp2 + 1022) << 52) + mant + up;
  return __longlong_as_double((long long)(bits | (v < 0 ? 0x8000000000000000ULL : 0ULL)));
}

// (hi + lo) * 2^R + y0 (y0 may be 0), assembled in int64; error <= ~1 ulp.
__device__ __forceinline__ double assemble_df(float hi, float lo, int R, double y0) {
  long long m[3];
  int e[3];
  float_parts(hi, m[0], e[0]);
  float_parts(lo, m[1], e[1]);
  e[0] += R;
  e[1] += R;
  double_parts(y0, m[2], e[2]);
  int top = -100000;
#pragma unroll
  for (int i = 0; i < 3; ++i)
    if (m[i] != 0) top = max(top, e[i] + bitlen(m[i]));
  if (top == -100000) return 0.0;
  const int base = top - 61;
  long long acc = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (m[i] == 0) continue;
    const int sh = e[i] - base;
    if (sh >= 0)
      acc += m[i] << sh;
    else if (sh > -63)
      acc += m[i] >> (-sh);
  }
  return int_to_double(acc, base);
}

}  // namespace lob
