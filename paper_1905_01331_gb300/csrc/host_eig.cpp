// Bond shift c = lambda_max of the two-site bond term (step a0 of the sweep):
// subtracting c from the one-site term on every site makes every bond term
// negative semidefinite, so that the update w = -polar(dE/dw) cannot raise
// the energy.  Dense symmetric eigenvalue by Householder tridiagonalisation
// (Golub & Van Loan, Alg. 8.3.1) and bisection on the Sturm sequence.
#include "host_eig.h"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ttn {

static int sturm_below(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (size_t i = 1; i < a.size(); ++i) {
    if (q == 0.0) q = 1e-300;
    q = a[i] - x - b[i - 1] * b[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

double bond_lambda_max(const double* o, const double* A, const double* B, int d0, int K) {
  const int n = d0 * d0;
  std::vector<double> H((size_t)n * n, 0.0);
  auto at = [&](int i, int j) -> double& { return H[(size_t)i * n + j]; };
  // 1/2 (o (x) I + I (x) o) + sum_k A_k (x) B_k, index (a, b) -> a * d0 + b
  for (int a = 0; a < d0; ++a)
    for (int b = 0; b < d0; ++b)
      for (int a2 = 0; a2 < d0; ++a2)
        for (int b2 = 0; b2 < d0; ++b2) {
          double v = 0.0;
          if (b == b2) v += 0.5 * o[a * d0 + a2];
          if (a == a2) v += 0.5 * o[b * d0 + b2];
          for (int k = 0; k < K; ++k)
            v += A[(size_t)k * d0 * d0 + a * d0 + a2] * B[(size_t)k * d0 * d0 + b * d0 + b2];
          at(a * d0 + b, a2 * d0 + b2) = v;
        }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      const double s = 0.5 * (at(i, j) + at(j, i));
      at(i, j) = s;
      at(j, i) = s;
    }
  // Householder tridiagonalisation
  std::vector<double> v(n), p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    double alpha = 0.0;
    for (int i = k + 1; i < n; ++i) alpha += at(i, k) * at(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0.0) continue;
    const double x0 = at(k + 1, k);
    const double sgn = x0 >= 0 ? 1.0 : -1.0;
    std::fill(v.begin(), v.end(), 0.0);
    v[k + 1] = x0 + sgn * alpha;
    for (int i = k + 2; i < n; ++i) v[i] = at(i, k);
    double vv = 0.0;
    for (int i = k + 1; i < n; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    const double beta = 2.0 / vv;
    // p = beta H v ; w = p - (beta/2)(p.v) v ; H -= v w^T + w v^T
    for (int i = k; i < n; ++i) {
      double s = 0.0;
      for (int j = k + 1; j < n; ++j) s += at(i, j) * v[j];
      p[i] = beta * s;
    }
    double pv = 0.0;
    for (int i = k + 1; i < n; ++i) pv += p[i] * v[i];
    for (int i = k; i < n; ++i) w[i] = p[i] - 0.5 * beta * pv * v[i];
    for (int i = k; i < n; ++i)
      for (int j = k; j < n; ++j) at(i, j) -= v[i] * w[j] + w[i] * v[j];
  }
  std::vector<double> a(n), b(std::max(n - 1, 1));
  for (int i = 0; i < n; ++i) a[i] = at(i, i);
  for (int i = 0; i + 1 < n; ++i) b[i] = at(i + 1, i);
  double lo = a[0], hi = a[0];
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  // largest eigenvalue: smallest x with sturm_below(x) == n
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_below(a, b, mid) >= n) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

}  // namespace ttn
