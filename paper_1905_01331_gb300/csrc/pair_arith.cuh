// Double-float ("pair") arithmetic on the FP32 pipes: a value is the
// unevaluated sum hi + lo of two FP32 numbers with |lo| <= 2^-24 |hi| (about
// 48 significant bits).  Error-free transformations: two-sum (Knuth) for
// additions, the FMA residual for products.  Every operation goes through
// fp_rn.cuh, so that no add or subtract is fused with a product.  Host- and
// device-callable (host tests check the accuracy of the products built from
// them).
#pragma once
#include <cmath>

#include "f64_bits.cuh"
#include "fp_rn.cuh"

#ifdef __CUDACC__
#define PA_HD __host__ __device__ __forceinline__
#else
#define PA_HD inline
#endif

namespace ttn {

// s + e = a + b exactly
PA_HD void two_sum_f(float a, float b, float& s, float& e) {
  s = rn::add(a, b);
  const float bb = rn::sub(s, a);
  e = rn::add(rn::sub(a, rn::sub(s, bb)), rn::sub(b, bb));
}

// (ah + al) + (bh + bl), renormalised
PA_HD void pair_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  two_sum_f(ah, bh, s, e);
  e = rn::add(e, rn::add(al, bl));
  rh = rn::add(s, e);
  rl = rn::sub(e, rn::sub(rh, s));
}

// (ah + al) (ch + cl), renormalised (al cl dropped)
PA_HD void pair_mul(float ah, float al, float ch, float cl, float& rh, float& rl) {
  const float p = rn::mul(ah, ch);
  float pe = rn::fma(ah, ch, -p);
  pe = rn::fma(ah, cl, rn::fma(al, ch, pe));
  rh = rn::add(p, pe);
  rl = rn::sub(pe, rn::sub(rh, p));
}

// (sh, sl) += (ah + al)(bh + bl), without renormalising sl (callers
// renormalise every few steps with pair_renorm)
PA_HD void pair_mac(float ah, float al, float bh, float bl, float& sh, float& sl) {
  const float p = rn::mul(ah, bh);
  const float pe = rn::fma(ah, bh, -p);
  const float c = rn::fma(ah, bl, rn::fma(al, bh, pe));
  float s, e;
  two_sum_f(sh, p, s, e);
  sl = rn::add(sl, rn::add(e, c));
  sh = s;
}

PA_HD void pair_renorm(float& sh, float& sl) {
  const float s = rn::add(sh, sl);
  sl = rn::sub(sl, rn::sub(s, sh));
  sh = s;
}

// x -> (hi, lo): hi = fl32(x), lo = fl32(x - hi) (integer operations on the
// IEEE fields, f64_bits.cuh)
PA_HD void split_d(double x, float& h, float& l) { f64b::split(x, h, l); }

}  // namespace ttn
