// Double-float ("pair") arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= 2^-24 |hi| (about
// 48 significant bits).  Error-free transformations: two-sum (Knuth) for
// additions, the FMA residual for products.
#pragma once
#include <cuda_runtime.h>

#include "f64_bits.cuh"

namespace ttn {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (ah + al) + (bh + bl), renormalised
__device__ __forceinline__ void pair_add(float ah, float al, float bh, float bl, float& rh,
                                         float& rl) {
  float s, e;
  two_sum_f(ah, bh, s, e);
  e += al + bl;
  rh = s + e;
  rl = e - (rh - s);
}

// (ah + al) (ch + cl), renormalised (al cl dropped)
__device__ __forceinline__ void pair_mul(float ah, float al, float ch, float cl, float& rh,
                                         float& rl) {
  const float p = ah * ch;
  float pe = fmaf(ah, ch, -p);
  pe = fmaf(ah, cl, fmaf(al, ch, pe));
  rh = p + pe;
  rl = pe - (rh - p);
}

// (sh, sl) += (ah + al)(bh + bl), without renormalising sl (callers
// renormalise every few steps with pair_renorm)
__device__ __forceinline__ void pair_mac(float ah, float al, float bh, float bl, float& sh,
                                         float& sl) {
  const float p = ah * bh;
  const float pe = fmaf(ah, bh, -p);
  const float c = fmaf(ah, bl, fmaf(al, bh, pe));
  float s, e;
  two_sum_f(sh, p, s, e);
  sl += e + c;
  sh = s;
}

__device__ __forceinline__ void pair_renorm(float& sh, float& sl) {
  const float s = sh + sl;
  sl = sl - (s - sh);
  sh = s;
}

// x -> (hi, lo): hi = fl32(x), lo = fl32(x - hi) (integer operations on the
// IEEE fields, f64_bits.cuh)
__device__ __forceinline__ void split_d(double x, float& h, float& l) { f64b::split(x, h, l); }

}  // namespace ttn
