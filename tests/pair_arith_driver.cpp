// Host driver: dot products in the double-float arithmetic of the polar
// factor's products (paper_1905_01331_gb300/csrc/pair_arith.cuh), with the
// schedule of gemm_df_kernel (operands split into FP32 pairs, one pair_mac per
// term, renormalisation every 16 terms), against a long-double reference.
// Prints, per length K, the largest error relative to sum |a_i b_i| for the
// pair products and for plain FP32 accumulation of the same FP32-rounded
// operands.
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "../paper_1905_01331_gb300/csrc/pair_arith.cuh"

using namespace ttn;

int main() {
  std::mt19937_64 g(9);
  std::normal_distribution<double> nd;
  for (int K : {16, 128, 4096, 16384}) {
    double worst_df = 0.0, worst_f32 = 0.0;
    for (int t = 0; t < 200; ++t) {
      std::vector<double> a(K), b(K);
      for (int i = 0; i < K; ++i) {
        a[i] = nd(g) * std::ldexp(1.0, (int)(g() % 21) - 10);
        b[i] = nd(g);
      }
      if (t % 2) {   // heavy cancellation: b orthogonal to a up to a small part
        long double aa = 0, ab = 0;
        for (int i = 0; i < K; ++i) { aa += (long double)a[i] * a[i]; ab += (long double)a[i] * b[i]; }
        for (int i = 0; i < K; ++i) b[i] -= (double)(ab / aa) * a[i] * (1.0 - 1e-6);
      }
      long double ref = 0, mag = 0;
      for (int i = 0; i < K; ++i) {
        ref += (long double)a[i] * (long double)b[i];
        mag += std::fabs((long double)a[i] * (long double)b[i]);
      }
      float sh = 0.f, sl = 0.f, s32 = 0.f;
      for (int i = 0; i < K; ++i) {
        float ah, al, bh, bl;
        split_d(a[i], ah, al);
        split_d(b[i], bh, bl);
        pair_mac(ah, al, bh, bl, sh, sl);
        if (i % 16 == 15) pair_renorm(sh, sl);
        s32 = std::fma(ah, bh, s32);
      }
      pair_renorm(sh, sl);
      const double df = (double)sh + (double)sl;
      worst_df = std::fmax(worst_df, (double)(std::fabs((long double)df - ref) / mag));
      worst_f32 = std::fmax(worst_f32, (double)(std::fabs((long double)s32 - ref) / mag));
    }
    std::printf("%d %.3e %.3e\n", K, worst_df, worst_f32);
  }
  return 0;
}
