// Lowest eigenpair test of a symmetric tridiagonal matrix in double-float
// arithmetic (values as unevaluated FP32 pairs hi + lo, ~48 significant
// bits), for the convergence checks inside a Lanczos cycle.  On this GPU a
// chain of dependent FP64 operations (a Sturm sequence, a tridiagonal solve)
// runs at a small fraction of the FP32 rate; the same chains in pair
// arithmetic run on the FP32 pipes.  The functions are host- and
// device-callable so that host tests can run them.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>

#include "fp_rn.cuh"

#ifdef __CUDACC__
#define TDF_HD __host__ __device__ __forceinline__
#else
#define TDF_HD inline
#endif

namespace ttn {
namespace tdf {

struct DF {
  float h, l;
};

TDF_HD uint32_t f_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t u;
  std::memcpy(&u, &x, 4);
  return u;
#endif
}
TDF_HD float f_from_bits(uint32_t u) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float x;
  std::memcpy(&x, &u, 4);
  return x;
#endif
}

// x -> (fl32(x), fl32(x - fl32(x)))
TDF_HD DF make(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
TDF_HD double to_double(DF a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly (Knuth)
TDF_HD void two_sum(float a, float b, float& s, float& e) {
  s = rn::add(a, b);
  const float bb = rn::sub(s, a);
  e = rn::add(rn::sub(a, rn::sub(s, bb)), rn::sub(b, bb));
}
TDF_HD DF add(DF a, DF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = rn::add(e, rn::add(a.l, b.l));
  const float h = rn::add(s, e);
  return {h, rn::sub(e, rn::sub(h, s))};
}
TDF_HD DF neg(DF a) { return {-a.h, -a.l}; }
TDF_HD DF sub(DF a, DF b) { return add(a, neg(b)); }
// product with the FMA residual of the high parts (a.l b.l dropped)
TDF_HD DF mul(DF a, DF b) {
  const float p = rn::mul(a.h, b.h);
  float pe = rn::fma(a.h, b.h, -p);
  pe = rn::fma(a.h, b.l, rn::fma(a.l, b.h, pe));
  const float h = rn::add(p, pe);
  return {h, rn::sub(pe, rn::sub(h, p))};
}
// quotient: FP32 estimate, one correction from the pair remainder
TDF_HD DF div(DF a, DF b) {
  const float q1 = a.h / b.h;
  const DF r = sub(a, mul({q1, 0.f}, b));
  const float q2 = r.h / b.h;
  const float h = rn::add(q1, q2);
  return {h, rn::sub(q2, rn::sub(h, q1))};
}
TDF_HD bool is_neg(DF a) { return a.h < 0.f || (a.h == 0.f && a.l < 0.f); }
TDF_HD DF scale(DF a, float s) { return {rn::mul(a.h, s), rn::mul(a.l, s)}; }
TDF_HD float fabs_hi(DF a) { return std::fabs(a.h); }

// 2^-e for the binary exponent e of |x| (x normal), else 1
TDF_HD float pow2_inv_exp(float x) {
  const int e = (int)((f_bits(x) >> 23) & 0xFFu) - 127;
  if (e <= -126 || e >= 127) return 1.f;
  return f_from_bits((uint32_t)(127 - e) << 23);
}

// Number of eigenvalues of T (diagonal a, squared off-diagonal b2, pairs)
// below x: signs of the leading principal minors of T - x I,
// d_{i+1} = (a_i - x) d_i - b2_{i-1} d_{i-1}, rescaled by a power of two
// after every step (FP32 exponent range); a zero minor is replaced by a tiny
// one of the previous minor's sign (a tiny positive pivot).
TDF_HD int sturm_below(const DF* a, const DF* b2, int m, DF x) {
  int cnt = 0;
  DF dm = {1.f, 0.f};
  DF d = sub(a[0], x);
  if (d.h == 0.f) d = {1e-30f, 0.f};
  if (is_neg(d)) ++cnt;
  for (int i = 1; i < m; ++i) {
    DF dn = sub(mul(sub(a[i], x), d), mul(b2[i - 1], dm));
    if (dn.h == 0.f) dn = {d.h < 0.f ? -1e-30f : 1e-30f, 0.f};
    if (is_neg(dn) != is_neg(d)) ++cnt;
    dm = d;
    d = dn;
    const float sc = pow2_inv_exp(std::fmax(fabs_hi(d), fabs_hi(dm)));
    d = scale(d, sc);
    dm = scale(dm, sc);
  }
  return cnt;
}

// Solve (T - th I) x = ones by LU with partial pivoting (one round of inverse
// iteration) and return |x_{m-1}| / |x|, the last component of the
// normalised approximate eigenvector.  dd, du, du2, dl, x: scratch arrays of
// m pairs.
TDF_HD double last_component(const DF* a, const DF* b, int m, DF th, DF* dd, DF* du, DF* du2,
                             DF* dl, DF* x) {
  const DF tiny = {1e-30f, 0.f};
  for (int i = 0; i < m; ++i) {
    dd[i] = sub(a[i], th);
    du[i] = i + 1 < m ? b[i] : DF{0.f, 0.f};
    du2[i] = {0.f, 0.f};
    dl[i] = i + 1 < m ? b[i] : DF{0.f, 0.f};
    x[i] = {1.f, 0.f};
  }
  for (int i = 0; i + 1 < m; ++i) {
    if (fabs_hi(dd[i]) >= fabs_hi(dl[i])) {
      if (dd[i].h == 0.f) dd[i] = tiny;
      const DF f = div(dl[i], dd[i]);
      dd[i + 1] = sub(dd[i + 1], mul(f, du[i]));
      x[i + 1] = sub(x[i + 1], mul(f, x[i]));
    } else {
      const DF f = div(dd[i], dl[i]);
      dd[i] = dl[i];
      const DF t = du[i];
      du[i] = dd[i + 1];
      dd[i + 1] = sub(t, mul(f, dd[i + 1]));
      if (i + 2 < m) {
        du2[i] = du[i + 1];
        du[i + 1] = neg(mul(f, du[i + 1]));
      }
      const DF r = x[i];
      x[i] = x[i + 1];
      x[i + 1] = sub(r, mul(f, x[i + 1]));
    }
  }
  if (dd[m - 1].h == 0.f) dd[m - 1] = tiny;
  // back substitution, rescaled by a power of two whenever an entry passes
  // 1e18 (the solution grows like 1 / (distance to the eigenvalue))
  for (int i = m - 1; i >= 0; --i) {
    DF s = x[i];
    if (i + 1 < m) s = sub(s, mul(du[i], x[i + 1]));
    if (i + 2 < m) s = sub(s, mul(du2[i], x[i + 2]));
    x[i] = div(s, dd[i]);
    if (fabs_hi(x[i]) > 1e18f) {
      // the whole vector: solved entries and the right-hand sides above
      const float sc = pow2_inv_exp(fabs_hi(x[i]));
      for (int k = 0; k < m; ++k) x[k] = scale(x[k], sc);
    }
  }
  double n2 = 0.0;
  for (int i = 0; i < m; ++i) {
    const double v = to_double(x[i]);
    n2 += v * v;
  }
  return n2 > 0.0 ? std::fabs(to_double(x[m - 1])) / std::sqrt(n2) : 1.0;
}

}  // namespace tdf
}  // namespace ttn
