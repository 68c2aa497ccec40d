// FP64 <-> FP32 conversions from the IEEE-754 fields with integer operations.
// On this GPU FP64 arithmetic and conversions run on two FP64 units per SM;
// the streams of conversions of the mixed modes (FP32 copies of tensors,
// FP32 pairs of the double-float products) would be bound by them.  Here the
// 53-bit significand is cut at bit 29 with round-to-nearest-even, exactly as
// the converting instruction rounds; values outside the range where both
// parts are normal FP32 numbers take the converting instructions.
// Host- and device-callable (host tests compare them with the converting
// casts).
#pragma once
#include <cstdint>
#include <cstring>

#ifdef __CUDACC__
#define F64B_HD __host__ __device__ __forceinline__
#else
#define F64B_HD inline
#endif

namespace ttn {
namespace f64b {

F64B_HD uint64_t d_bits(double x) {
#ifdef __CUDA_ARCH__
  return static_cast<uint64_t>(__double_as_longlong(x));
#else
  uint64_t u;
  std::memcpy(&u, &x, 8);
  return u;
#endif
}
F64B_HD float f_from_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}
F64B_HD uint32_t f_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
F64B_HD double d_from_bits(uint64_t u) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double(static_cast<long long>(u));
#else
  double x;
  std::memcpy(&x, &u, 8);
  return x;
#endif
}
F64B_HD float i2f(int v) {
#ifdef __CUDA_ARCH__
  return __int2float_rn(v);
#else
  return static_cast<float>(v);
#endif
}

// Exponent fields (biased, FP64) for which the fast paths apply: the high
// part a normal FP32 number (with room for the rounding carry) and the low
// part, down to 2^-29 of it, normal too.
constexpr uint32_t kFastLo = 1075 - 126;        // |x| >= 2^-74
constexpr uint32_t kFastHi = 1023 + 126;        // |x| <  2^127

// hi = fl32(x) (round to nearest even), lo = fl32(x - hi)
F64B_HD void split(double x, float& hi, float& lo) {
  const uint64_t b = d_bits(x);
  const uint32_t e = static_cast<uint32_t>(b >> 52) & 0x7FFu;
  if (e < kFastLo || e > kFastHi) {
    hi = static_cast<float>(x);
    lo = static_cast<float>(x - static_cast<double>(hi));
    return;
  }
  const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);   // 53-bit significand
  uint32_t q = static_cast<uint32_t>(m >> 29);                   // 24 bits
  int rem = static_cast<int>(m & 0x1FFFFFFFu);                   // dropped 29 bits
  if (rem > (1 << 28) || (rem == (1 << 28) && (q & 1u))) {
    ++q;
    rem -= 1 << 29;
  }
  // (e - 896) << 23 plus the 23 stored bits; a carry of q into bit 24 moves
  // into the exponent field
  hi = f_from_bits(sign | (((e - 896u) << 23) + (q - (1u << 23))));
  // x - hi = rem * 2^(e - 1075): the integer rem (|rem| <= 2^28) rounded to
  // FP32, then scaled by a power of two (exact)
  const float scale = f_from_bits((e - 1075u + 127u) << 23);
  const float r = i2f(rem) * scale;
  lo = sign ? -r : r;
}

// fl32(x), round to nearest even
F64B_HD float to_f32(double x) {
  const uint64_t b = d_bits(x);
  const uint32_t e = static_cast<uint32_t>(b >> 52) & 0x7FFu;
  if (e < kFastLo || e > kFastHi) return static_cast<float>(x);
  const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  uint32_t q = static_cast<uint32_t>(m >> 29);
  const uint32_t rem = static_cast<uint32_t>(m & 0x1FFFFFFFu);
  if (rem > (1u << 28) || (rem == (1u << 28) && (q & 1u))) ++q;
  return f_from_bits(sign | (((e - 896u) << 23) + (q - (1u << 23))));
}

// (double) x for an FP32 x from the IEEE-754 fields (sign, exponent rebiased
// by 1023 - 127 = 896, mantissa shifted up by 29 bits) with integer
// operations.  Zeros keep their sign; subnormal, infinite and NaN inputs take
// the converting instruction.
F64B_HD double from_f32(float x) {
  const uint32_t b = f_bits(x);
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) {
    if ((b & 0x7FFFFFFFu) == 0u) return d_from_bits(static_cast<uint64_t>(b & 0x80000000u) << 32);
    return static_cast<double>(x);
  }
  const uint64_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | ((b & 0x7FFFFFu) >> 3);
  return d_from_bits((hi << 32) | static_cast<uint64_t>(b << 29));
}

}  // namespace f64b
}  // namespace ttn
