// Host driver for the double-float tridiagonal routines of the Lanczos
// convergence checks (paper_1905_01331_gb300/csrc/tridiag_df.cuh).
// stdin: cases "m x a_0 .. a_{m-1} b_0 .. b_{m-2}"; stdout per case:
// "count theta y_last" with count = eigenvalues below x (Sturm count),
// theta = lowest eigenvalue by pair-arithmetic bisection, y_last = last
// component of its normalised eigenvector (one inverse-iteration round).
#include <algorithm>
#include <cstdio>
#include <vector>

#include "../paper_1905_01331_gb300/csrc/tridiag_df.cuh"

using namespace ttn::tdf;

int main() {
  int m;
  double x;
  while (std::scanf("%d %lf", &m, &x) == 2) {
    std::vector<double> a(m), b(m, 0.0);
    for (int i = 0; i < m; ++i) std::scanf("%lf", &a[i]);
    for (int i = 0; i + 1 < m; ++i) std::scanf("%lf", &b[i]);
    std::vector<DF> A(m), B(m), B2(m), w(5 * m);
    double glo = a[0], ghi = a[0];
    for (int i = 0; i < m; ++i) {
      A[i] = make(a[i]);
      B[i] = make(b[i]);
      B2[i] = make(b[i] * b[i]);
      const double r = (i > 0 ? b[i - 1] : 0.0) + b[i];
      glo = std::min(glo, a[i] - r);
      ghi = std::max(ghi, a[i] + r);
    }
    const int count = sturm_below(A.data(), B2.data(), m, make(x));
    DF lo = make(glo), hi = make(ghi);
    for (int it = 0; it < 80; ++it) {
      const DF mid = add(lo, {0.5f * sub(hi, lo).h, 0.f});
      if (sturm_below(A.data(), B2.data(), m, mid) >= 1) hi = mid; else lo = mid;
    }
    const DF th = add(lo, {0.5f * sub(hi, lo).h, 0.f});
    const double y = last_component(A.data(), B.data(), m, th, w.data(), w.data() + m,
                                    w.data() + 2 * m, w.data() + 3 * m, w.data() + 4 * m);
    std::printf("%d %.17g %.17g\n", count, to_double(th), y);
  }
  return 0;
}
