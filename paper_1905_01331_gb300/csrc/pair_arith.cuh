// Double-float ("pair") arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= 2^-24 |hi| (about
// 48 significant bits).  Error-free transformations: two-sum (Knuth) for
// additions, the FMA residual for products.  Host- and device-callable (host
// tests check the accuracy of the products built from them).
#pragma once
#include <cmath>

#include "f64_bits.cuh"

#ifdef __CUDACC__
#define PA_HD __host__ __device__ __forceinline__
#else
#define PA_HD inline
#endif

namespace ttn {

// s + e = a + b exactly
PA_HD void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (ah + al) + (bh + bl), renormalised
PA_HD void pair_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  two_sum_f(ah, bh, s, e);
  e += al + bl;
  rh = s + e;
  rl = e - (rh - s);
}

// (ah + al) (ch + cl), renormalised (al cl dropped)
PA_HD void pair_mul(float ah, float al, float ch, float cl, float& rh, float& rl) {
  const float p = ah * ch;
  float pe = std::fma(ah, ch, -p);
  pe = std::fma(ah, cl, std::fma(al, ch, pe));
  rh = p + pe;
  rl = pe - (rh - p);
}

// (sh, sl) += (ah + al)(bh + bl), without renormalising sl (callers
// renormalise every few steps with pair_renorm)
PA_HD void pair_mac(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = ah * bh;
  const float pe = std::fma(ah, bh, -p);
  const float c = std::fma(ah, bl, std::fma(al, bh, pe));
  float s, e;
  two_sum_f(sh, p, s, e);
  sl += e + c;
  sh = s;
}

PA_HD void pair_renorm(float& sh, float& sl) {
  const float s = sh + sl;
  sl = sl - (s - sh);
  sh = s;
}

// x -> (hi, lo): hi = fl32(x), lo = fl32(x - hi) (integer operations on the
// IEEE fields, f64_bits.cuh)
PA_HD void split_d(double x, float& h, float& l) { f64b::split(x, h, l); }

}  // namespace ttn
