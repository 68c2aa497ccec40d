// Top-tensor update (Sec. III.B: the top tensor is "updated similarly"; read
// as the lowest eigenvector of the top Hamiltonian) as one persistent
// cooperative launch: restarted Lanczos with full reorthogonalisation,
// warm-started from the previous V.  Vectors, projections and the
// tridiagonal are FP64; in the mixed modes the matrix-vector products run in
// double-float pair arithmetic on pair copies of the operators and the basis.
//
// H_top acts on the c x c top tensor V as
//     H V = o_0 V + V o_1^T + sum_k (A_k0 V B_k1^T + B_k0 V A_k1^T),
// with (o, A_k, B_k) the identity-free operators of the two top sites (the
// two bonds of the periodic ring at the top).  One Lanczos step is
//     phase A   Y_k = A_k0 x, Y_{K+k} = B_k0 x               (2K products)
//     phase B   w = o_0 x + x o_1^T + sum_k Y_k B_k1^T + Y_{K+k} A_k1^T
//               (minus sigma x after the first step: the recurrence runs on
//               H - sigma I, sigma the Rayleigh quotient of the start vector)
//     projections on the basis and |w|^2, one classical Gram-Schmidt pass,
//     a second one ("twice is enough") when the first removed more than 3/4
//     of |w|^2, then alpha_j, beta_j and the next basis vector
// with every phase shared by all CTAs and a grid barrier between phases
// (bounded spin, error flag).  Each CTA owns the vector entries of the 8 x 8
// output tiles it computes; every reduction adds its per-CTA partial sums in
// a fixed order, so the result does not depend on timing.  Every kLCheck
// steps CTA 0 tests the tridiagonal so far for convergence in pair
// arithmetic (tridiag_df.cuh) and a passed test ends the cycle; at the end of
// a cycle CTA 0 finds the eigenpair of the tridiagonal (Sturm bisection, in
// FP32 to bracket, then in FP64, and inverse iteration).
#include <algorithm>
#include <mutex>

#include "common.h"
#include "pair_arith.cuh"
#include "tridiag_df.cuh"

namespace ttn {

namespace {

constexpr int kLT = 8;                   // output tile edge of the matrix products
constexpr int kLThreads = 256;
constexpr int kLWarps = kLThreads / 32;
constexpr int kLMaxC = 256;
constexpr int kLMaxSpin = 1 << 21;       // ~1 s of polling, then the error flag
constexpr int kLCheck = 8;               // steps between convergence checks within a cycle

struct __align__(16) LzSmem {
  double L[kLT][kLMaxC + 1];             // left-operand rows of a tile
  double R[kLT][kLMaxC + 1];             // right-operand rows (or columns) of a tile
  double red[kLWarps][kLT * kLT];
  double tri[6][kLMaxM + 2];             // inverse iteration scratch (CTA 0)
  double da[kLMaxM + 2], db2[kLMaxM + 2];  // tridiagonal: diagonal, squared off-diagonal
  float fa[kLMaxM + 2], fb2[kLMaxM + 2];
  double cf[kLMaxM + 2];                 // coefficients of the current combination
  double bcast[4];
  int ok;
};

__device__ bool lz_barrier(LzSmem& sm, unsigned* bar, unsigned& target, int* err, int max_spin) {
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    // arrive with release semantics (this CTA's writes before it), poll with
    // acquire semantics (the other CTAs' writes after it)
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int spins = 0;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (*reinterpret_cast<volatile int*>(err)) { ok = 0; break; }
      if (++spins > max_spin) { atomicOr(err, 4); ok = 0; break; }
      __nanosleep(32);
    }
    sm.ok = ok;
  }
  __syncthreads();
  return sm.ok != 0;
}

// Sum of x[0..count) in a fixed order (lane-strided partial sums, then a fixed
// butterfly), by warp 0; the result is returned to every thread of the CTA.
__device__ double cta_ordered_sum(LzSmem& sm, const double* x, int count, long long stride) {
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += 32) s += __ldcg(x + i * stride);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) sm.bcast[0] = s;
  }
  __syncthreads();
  const double v = sm.bcast[0];
  __syncthreads();
  return v;
}

// Elements staged per thread: a tile edge of 8 rows or columns of length
// c <= kLMaxC.  The staging functions issue all their loads before the first
// shared-memory store, so that a staged tile costs one load latency.
constexpr int kLStage = kLT * kLMaxC / kLThreads;

// Stage rows [r0, r0+8) of the row-major c x c matrix M (times scale) into dst.
__device__ void stage_rows(double (*dst)[kLMaxC + 1], const double* M, int c, int r0, double scale) {
  double v[kLStage];
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, r = e / c, k = e - r * c;
    v[u] = (e < kLT * c && r0 + r < c) ? __ldcg(M + (long long)(r0 + r) * c + k) : 0.0;
  }
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, r = e / c, k = e - r * c;
    if (e < kLT * c) dst[r][k] = scale * v[u];
  }
}
// Stage columns [c0, c0+8) of M (times scale) as rows of dst: dst[j][k] = M[k][c0 + j].
__device__ void stage_cols(double (*dst)[kLMaxC + 1], const double* M, int c, int c0, double scale) {
  double v[kLStage];
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, k = e / kLT, j = e - k * kLT;
    v[u] = (e < kLT * c && c0 + j < c) ? __ldcg(M + (long long)k * c + c0 + j) : 0.0;
  }
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, k = e / kLT, j = e - k * kLT;
    if (e < kLT * c) dst[j][k] = scale * v[u];
  }
}

// acc[0..1] += sum_k L[i][k] R[j][k] over this warp's K slice (i = lane/4,
// j = 2 (lane % 4) + {0, 1}).
__device__ __forceinline__ void tile_fma(const LzSmem& sm, int c, double& a0, double& a1) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  for (int k = warp; k < c; k += kLWarps) {
    const double x = sm.L[i][k];
    a0 = fma(x, sm.R[j][k], a0);
    a1 = fma(x, sm.R[j + 1][k], a1);
  }
}

// Reduce the per-warp partial sums of a tile in warp order and store it,
// minus sigma X when sigma != 0 (the shifted operator H - sigma I).
__device__ void tile_store(LzSmem& sm, double a0, double a1, double* C, int c, int i0, int j0,
                           const double* X = nullptr, double sigma = 0.0,
                           const double* Xprev = nullptr, double beta = 0.0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  sm.red[warp][i * kLT + j] = a0;
  sm.red[warp][i * kLT + j + 1] = a1;
  __syncthreads();
  if (threadIdx.x < kLT * kLT) {
    double v = 0.0;
    for (int w = 0; w < kLWarps; ++w) v += sm.red[w][threadIdx.x];
    const int r = threadIdx.x / kLT, cc = threadIdx.x % kLT;
    if (i0 + r < c && j0 + cc < c) {
      const long long e = (long long)(i0 + r) * c + j0 + cc;
      if (sigma != 0.0) v = fma(-sigma, __ldcg(X + e), v);
      if (beta != 0.0) v = fma(-beta, __ldcg(Xprev + e), v);
      __stcg(C + e, v);
    }
  }
  __syncthreads();
}

// Number of eigenvalues of the symmetric tridiagonal below x (diagonal a,
// squared off-diagonal b2), by the signs of the LDL^T pivots.
template <typename T>
__device__ int sturm_below(const T* a, const T* b2, int m, T x) {
  int cnt = 0;
  T q = a[0] - x;
  if (q < (T)0) ++cnt;
  for (int i = 1; i < m; ++i) {
    if (q == (T)0) q = (T)1e-30;
    q = a[i] - x - b2[i - 1] / q;
    if (q < (T)0) ++cnt;
  }
  return cnt;
}

// The same count in FP64 without divisions (FP64 division is a long
// instruction sequence on this GPU's two FP64 units per SM): the signs of the
// leading principal minors d_i of T - x I, d_{i+1} = (a_i - x) d_i -
// b2_{i-1} d_{i-1}, whose ratios are the pivots above (a zero pivot is
// replaced by a tiny positive one, as above); the minors are rescaled by a
// power of two (exactly) every eight steps.
__device__ int sturm_below_f64(const double* a, const double* b2, int m, double x) {
  int cnt = 0;
  double dm = 1.0, d = a[0] - x;
  if (d == 0.0) d = 1e-30;
  if (d < 0.0) ++cnt;
  for (int i = 1; i < m; ++i) {
    double dn = fma(a[i] - x, d, -b2[i - 1] * dm);
    if (dn == 0.0) dn = 1e-30 * d;
    if ((dn < 0.0) != (d < 0.0)) ++cnt;
    dm = d;
    d = dn;
    if ((i & 7) == 0) {
      const int ex = (int)((__double_as_longlong(d) >> 52) & 0x7FF) - 1023;
      if (ex > -1000 && ex < 1000) {
        const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
        d *= sc;
        dm *= sc;
      }
    }
  }
  return cnt;
}

template <typename T>
__device__ __forceinline__ int sturm_count(const T* a, const T* b2, int m, T x) {
  if constexpr (sizeof(T) == 8) return sturm_below_f64(a, b2, m, x);
  else return sturm_below<T>(a, b2, m, x);
}

// 32-way multisection of [lo, hi] for the lowest eigenvalue, by one warp,
// until the interval is narrower than rel * max(|lo|, |hi|) or `its` rounds.
template <typename T>
__device__ void multisect(const T* a, const T* b2, int m, T& lo, T& hi, T rel, int its) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < its; ++it) {
    const T mag = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
    if (!(hi - lo > rel * mag)) break;
    constexpr T r33 = (T)1 / (T)33;
    const T pt = lo + (hi - lo) * ((T)(lane + 1) * r33);
    const unsigned below = __ballot_sync(0xffffffffu, sturm_count<T>(a, b2, m, pt) >= 1);
    const int f = below ? __ffs(below) - 1 : 32;
    const T nlo = f == 0 ? lo : lo + (hi - lo) * ((T)f * r33);
    const T nhi = f == 32 ? hi : lo + (hi - lo) * ((T)(f + 1) * r33);
    lo = nlo;
    hi = nhi;
  }
}

// Lowest eigenvalue of the m x m tridiagonal (alpha, beta) by warp 0 of the
// calling CTA (threads >= 32 return at once): bracketed by FP32 multisection,
// confirmed and refined in FP64; the tridiagonal is left in sm.da / sm.db2.
__device__ double ritz_value(LzSmem& sm, const double* alpha, const double* beta, int m) {
  const int lane = threadIdx.x;
  double glo = alpha[0], ghi = alpha[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < m ? fabs(beta[i]) : 0.0);
    glo = fmin(glo, alpha[i] - r);
    ghi = fmax(ghi, alpha[i] + r);
  }
  for (int i = lane; i < m; i += 32) {
    sm.da[i] = alpha[i];
    sm.fa[i] = (float)alpha[i];
    const double b2 = i + 1 < m ? beta[i] * beta[i] : 0.0;
    sm.db2[i] = b2;
    sm.fb2[i] = (float)b2;
  }
  __syncwarp();
  // bracket in FP32, widen by the FP32 rounding of T, confirm in FP64
  float flo = (float)glo, fhi = (float)ghi;
  multisect<float>(sm.fa, sm.fb2, m, flo, fhi, 2e-6f, 8);
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  double lo = (double)flo - 1e-5 * tnorm, hi = (double)fhi + 1e-5 * tnorm;
  const int c_lo = sturm_below_f64(sm.da, sm.db2, m, lo);
  const int c_hi = sturm_below_f64(sm.da, sm.db2, m, hi);
  if (!__all_sync(0xffffffffu, c_lo == 0 && c_hi >= 1)) { lo = glo; hi = ghi; }
  multisect<double>(sm.da, sm.db2, m, lo, hi, 4e-16, 16);
  return 0.5 * (lo + hi);
}

// Convergence test of the tridiagonal of the steps so far (alpha, beta: m
// entries, shifted by -sigma) by warp 0 of the calling CTA, for the checks
// within a cycle: the lowest eigenvalue bracketed in FP32 and refined by
// 32-way multisection in pair arithmetic, then one round of inverse
// iteration in pair arithmetic for the last component y_{m-1} of its
// eigenvector; true when |beta_{m-1} y_{m-1}| <= tol |theta + sigma|.  (The
// end of a cycle recomputes the pair in FP64; a wrong early answer costs a
// restart, not accuracy.)  Uses sm.L as scratch.  The result is valid in
// thread 0.
__device__ bool ritz_check_df(LzSmem& sm, const double* alpha, const double* beta, int m,
                              double sigma, double tol) {
  using namespace tdf;
  const int lane = threadIdx.x;
  constexpr int S = kLMaxM + 2;
  DF* A = reinterpret_cast<DF*>(&sm.L[0][0]);
  DF* B = A + S;
  DF* B2 = B + S;
  double glo = alpha[0], ghi = alpha[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < m ? fabs(beta[i]) : 0.0);
    glo = fmin(glo, alpha[i] - r);
    ghi = fmax(ghi, alpha[i] + r);
  }
  for (int i = lane; i < m; i += 32) {
    const double b2 = i + 1 < m ? beta[i] * beta[i] : 0.0;
    sm.fa[i] = (float)alpha[i];
    sm.fb2[i] = (float)b2;
    A[i] = make(alpha[i]);
    B[i] = make(i + 1 < m ? beta[i] : 0.0);
    B2[i] = make(b2);
  }
  __syncwarp();
  float flo = (float)glo, fhi = (float)ghi;
  multisect<float>(sm.fa, sm.fb2, m, flo, fhi, 2e-6f, 8);
  const double tnorm = fmax(fabs(glo), fabs(ghi));
  DF lo = make((double)flo - 1e-5 * tnorm), hi = make((double)fhi + 1e-5 * tnorm);
  const int c_lo = sturm_below(A, B2, m, lo), c_hi = sturm_below(A, B2, m, hi);
  if (!__all_sync(0xffffffffu, c_lo == 0 && c_hi >= 1)) { lo = make(glo); hi = make(ghi); }
  constexpr float r33 = 1.f / 33.f;
  for (int it = 0; it < 12; ++it) {
    const float w = sub(hi, lo).h;
    if (!(w > 1e-14f * fmaxf(fabsf(lo.h), fabsf(hi.h)))) break;
    const DF pt = add(lo, {w * ((float)(lane + 1) * r33), 0.f});
    const unsigned below = __ballot_sync(0xffffffffu, sturm_below(A, B2, m, pt) >= 1);
    const int f = below ? __ffs(below) - 1 : 32;
    const DF nlo = f == 0 ? lo : add(lo, {w * ((float)f * r33), 0.f});
    const DF nhi = f == 32 ? hi : add(lo, {w * ((float)(f + 1) * r33), 0.f});
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return false;
  const DF th = add(lo, {0.5f * sub(hi, lo).h, 0.f});
  DF* w = B2 + S;
  const double ylast = last_component(A, B, m, th, w, w + S, w + 2 * S, w + 3 * S, w + 4 * S);
  return fabs(beta[m - 1]) * ylast <= tol * fmax(fabs(to_double(th) + sigma), 1e-300);
}

// Lowest eigenpair of the m x m tridiagonal (alpha, beta) by warp 0 of the
// calling CTA: y (m entries, unit norm), theta, residual |beta_{m-1} y_{m-1}|.
__device__ void ritz_pair(LzSmem& sm, const double* alpha, const double* beta, int m, double* y,
                          double* theta, double* res) {
  if (threadIdx.x >= 32) return;
  const double th = ritz_value(sm, alpha, beta, m);
  if (threadIdx.x != 0) return;
  // inverse iteration on (T - th I) x = x_prev: LU with partial pivoting of
  // the tridiagonal, two rounds
  double* x = sm.tri[0];
  double* dd = sm.tri[1];
  double* du = sm.tri[2];
  double* du2 = sm.tri[3];
  double* rhs = sm.tri[4];
  double* dl = sm.tri[5];
  for (int i = 0; i < m; ++i) x[i] = 1.0 / sqrt((double)m);
  const double eps = fmax(fabs(th), 1.0) * 1e-15;
  for (int round = 0; round < 2; ++round) {
    for (int i = 0; i < m; ++i) {
      dd[i] = alpha[i] - th;
      du[i] = i + 1 < m ? beta[i] : 0.0;
      du2[i] = 0.0;
      rhs[i] = x[i];
      dl[i] = i + 1 < m ? beta[i] : 0.0;
    }
    for (int i = 0; i + 1 < m; ++i) {
      if (fabs(dd[i]) >= fabs(dl[i])) {
        if (dd[i] == 0.0) dd[i] = eps;
        const double f = dl[i] / dd[i];
        dl[i] = f;
        dd[i + 1] -= f * du[i];
        rhs[i + 1] -= f * rhs[i];
      } else {
        const double f = dd[i] / dl[i];
        dd[i] = dl[i];
        dl[i] = f;
        const double t = du[i];
        du[i] = dd[i + 1];
        dd[i + 1] = t - f * dd[i + 1];
        if (i + 2 < m) { du2[i] = du[i + 1]; du[i + 1] = -f * du[i + 1]; }
        const double r = rhs[i];
        rhs[i] = rhs[i + 1];
        rhs[i + 1] = r - f * rhs[i + 1];
      }
    }
    if (dd[m - 1] == 0.0) dd[m - 1] = eps;
    for (int i = m - 1; i >= 0; --i) {
      double s = rhs[i];
      if (i + 1 < m) s -= du[i] * x[i + 1];
      if (i + 2 < m) s -= du2[i] * x[i + 2];
      x[i] = s / (fabs(dd[i]) < eps ? (dd[i] < 0 ? -eps : eps) : dd[i]);
    }
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += x[i] * x[i];
    nrm = sqrt(nrm);
    for (int i = 0; i < m; ++i) x[i] /= nrm;
  }
  for (int i = 0; i < m; ++i) y[i] = x[i];
  *theta = th;
  *res = fabs(beta[m - 1] * x[m - 1]);
}

// Double-float matrix-vector products (mixed modes): matrices and vectors as
// FP32 pairs (hi block of n floats, then lo block), tiles staged into the
// shared arrays L and R reinterpreted as hi/lo float rows.
using FRow = float[kLMaxC + 1];

__device__ __forceinline__ FRow* frows(double (*d)[kLMaxC + 1], int half) {
  return reinterpret_cast<FRow*>(&d[0][0]) + half * kLT;
}

// rows [r0, r0+8) of the pair matrix M (hi at M, lo at M + n)
__device__ void stage_rows_p(double (*dst)[kLMaxC + 1], const float* M, long long n, int c,
                             int r0) {
  FRow* h = frows(dst, 0);
  FRow* l = frows(dst, 1);
  float vh[kLStage], vl[kLStage];
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, r = e / c, k = e - r * c;
    const bool ok = e < kLT * c && r0 + r < c;
    const long long i = (long long)(r0 + r) * c + k;
    vh[u] = ok ? __ldcg(M + i) : 0.f;
    vl[u] = ok ? __ldcg(M + n + i) : 0.f;
  }
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, r = e / c, k = e - r * c;
    if (e < kLT * c) { h[r][k] = vh[u]; l[r][k] = vl[u]; }
  }
}
// columns [c0, c0+8) of M as rows: dst[j][k] = M[k][c0 + j]
__device__ void stage_cols_p(double (*dst)[kLMaxC + 1], const float* M, long long n, int c,
                             int c0) {
  FRow* h = frows(dst, 0);
  FRow* l = frows(dst, 1);
  float vh[kLStage], vl[kLStage];
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, k = e / kLT, j = e - k * kLT;
    const bool ok = e < kLT * c && c0 + j < c;
    const long long i = (long long)k * c + c0 + j;
    vh[u] = ok ? __ldcg(M + i) : 0.f;
    vl[u] = ok ? __ldcg(M + n + i) : 0.f;
  }
#pragma unroll
  for (int u = 0; u < kLStage; ++u) {
    const int e = threadIdx.x + u * kLThreads, k = e / kLT, j = e - k * kLT;
    if (e < kLT * c) { h[j][k] = vh[u]; l[j][k] = vl[u]; }
  }
}

__device__ __forceinline__ void tile_fma_p(LzSmem& sm, int c, float& a0h, float& a0l, float& a1h,
                                           float& a1l) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  const FRow* Lh = frows(sm.L, 0);
  const FRow* Ll = frows(sm.L, 1);
  const FRow* Rh = frows(sm.R, 0);
  const FRow* Rl = frows(sm.R, 1);
  int cnt = 0;
  for (int k = warp; k < c; k += kLWarps) {
    const float xh = Lh[i][k], xl = Ll[i][k];
    pair_mac(xh, xl, Rh[j][k], Rl[j][k], a0h, a0l);
    pair_mac(xh, xl, Rh[j + 1][k], Rl[j + 1][k], a1h, a1l);
    if (++cnt == 8) {
      cnt = 0;
      pair_renorm(a0h, a0l);
      pair_renorm(a1h, a1l);
    }
  }
  pair_renorm(a0h, a0l);
  pair_renorm(a1h, a1l);
}

// Reduce the per-warp pair partial sums of a tile in warp order; store it as
// pairs (Cp) or as FP64 (Cd, minus sigma X when sigma != 0).
__device__ void tile_store_p(LzSmem& sm, float a0h, float a0l, float a1h, float a1l, float* Cp,
                             double* Cd, long long n, int c, int i0, int j0,
                             const double* X = nullptr, double sigma = 0.0,
                             const double* Xprev = nullptr, double beta = 0.0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  float* rh = reinterpret_cast<float*>(&sm.red[0][0]);
  float* rl = rh + kLWarps * kLT * kLT;
  rh[warp * 64 + i * kLT + j] = a0h;
  rl[warp * 64 + i * kLT + j] = a0l;
  rh[warp * 64 + i * kLT + j + 1] = a1h;
  rl[warp * 64 + i * kLT + j + 1] = a1l;
  __syncthreads();
  if (threadIdx.x < kLT * kLT) {
    float vh = 0.f, vl = 0.f;
    for (int w = 0; w < kLWarps; ++w) pair_add(vh, vl, rh[w * 64 + threadIdx.x], rl[w * 64 + threadIdx.x], vh, vl);
    const int r = threadIdx.x / kLT, cc = threadIdx.x % kLT;
    if (i0 + r < c && j0 + cc < c) {
      const long long e = (long long)(i0 + r) * c + j0 + cc;
      if (Cp) { __stcg(Cp + e, vh); __stcg(Cp + n + e, vl); }
      if (Cd) {
        double v = (double)vh + (double)vl;
        if (sigma != 0.0) v = fma(-sigma, __ldcg(X + e), v);
        if (beta != 0.0) v = fma(-beta, __ldcg(Xprev + e), v);
        __stcg(Cd + e, v);
      }
    }
  }
  __syncthreads();
}

// Wide staging (double-float mode, c <= kLWideMaxC, c a multiple of 8): every
// operand tile of a matrix-vector phase is requested at once by 16-byte
// asynchronous copies (cp.async.cg: L2 only, like the loads above) into
// kLWideSlots slots of 16 rows of ldw = c + 4 floats (slots 0 and 1 reuse
// sm.L and sm.R, the others are dynamic shared memory), so that a phase costs
// one L2 latency instead of one per term.  A row tile holds rows [r0, r0+8)
// of a pair matrix (hi rows 0-7, lo rows 8-15); a column tile holds columns
// [c0, c0+8) untransposed (hi: c rows of 8 floats, then lo).  The products
// below take the same operands in the same order as tile_fma_p, so both
// stagings give the same bits.
constexpr int kLWideMaxC = 128;
constexpr int kLWideSlots = 8;

__host__ __device__ __forceinline__ int lz_wide_ld(int c) { return c + 4; }

size_t lz_wide_dyn_bytes(int c) {
  return (size_t)(kLWideSlots - 2) * 2 * kLT * lz_wide_ld(c) * sizeof(float);
}

__device__ __forceinline__ float* wide_slot(LzSmem& sm, float* dyn, int s, int ldw) {
  if (s == 0) return reinterpret_cast<float*>(&sm.L[0][0]);
  if (s == 1) return reinterpret_cast<float*>(&sm.R[0][0]);
  return dyn + (long long)(s - 2) * 2 * kLT * ldw;
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// rows [r0, r0+8) of the pair matrix M (hi at M, lo at M + n) into a row tile
__device__ void wide_rows(float* dst, const float* M, long long n, int c, int r0, int ldw) {
  const int q4 = c >> 2, per = kLT * q4;   // 16-byte chunks per half
  for (int q = threadIdx.x; q < 2 * per; q += kLThreads) {
    const int half = q >= per ? 1 : 0, qq = q - half * per;
    const int r = qq / q4, k4 = (qq - r * q4) << 2;
    cp_async16(dst + (half * kLT + r) * ldw + k4, M + half * n + (long long)(r0 + r) * c + k4);
  }
}
// columns [c0, c0+8) of M into a column tile: dst[half][k][j] = M(half)[k][c0 + j]
__device__ void wide_cols(float* dst, const float* M, long long n, int c, int c0) {
  const int per = 2 * c;                   // two 16-byte chunks per row and half
  for (int q = threadIdx.x; q < 2 * per; q += kLThreads) {
    const int half = q >= per ? 1 : 0, qq = q - half * per;
    const int k = qq >> 1, j4 = (qq & 1) << 2;
    cp_async16(dst + half * kLT * c + k * kLT + j4, M + half * n + (long long)k * c + c0 + j4);
  }
}

// acc += sum over this warp's K slice of L(i, k) R(j, k) in pair arithmetic:
// L a row tile; R a row tile (R(j, k) = row j) or, with rcol, a column tile
// (R(j, k) = M[k][c0 + j]).  Operand order, renormalisation and the final
// renormalisation are those of tile_fma_p.
__device__ __forceinline__ void wide_fma(const float* L, const float* R, bool rcol, int c, int ldw,
                                         float& a0h, float& a0l, float& a1h, float& a1l) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  const float* Lh = L + i * ldw;
  const float* Ll = L + (kLT + i) * ldw;
  int cnt = 0;
  for (int k = warp; k < c; k += kLWarps) {
    const float xh = Lh[k], xl = Ll[k];
    float r0h, r0l, r1h, r1l;
    if (rcol) {
      const float* R0 = R + k * kLT + j;
      r0h = R0[0];
      r1h = R0[1];
      r0l = R0[kLT * c];
      r1l = R0[kLT * c + 1];
    } else {
      r0h = R[j * ldw + k];
      r1h = R[(j + 1) * ldw + k];
      r0l = R[(kLT + j) * ldw + k];
      r1l = R[(kLT + j + 1) * ldw + k];
    }
    pair_mac(xh, xl, r0h, r0l, a0h, a0l);
    pair_mac(xh, xl, r1h, r1l, a1h, a1l);
    if (++cnt == 8) {
      cnt = 0;
      pair_renorm(a0h, a0l);
      pair_renorm(a1h, a1l);
    }
  }
  pair_renorm(a0h, a0l);
  pair_renorm(a1h, a1l);
}

// FP64 value and its pair at index e of a vector (pair vector: hi at P, lo at P + n)
__device__ __forceinline__ void store_both(double* D, float* P, long long n, long long e, double v) {
  __stcg(D + e, v);
  if (P) {
    float h, l;
    split_d(v, h, l);
    __stcg(P + e, h);
    __stcg(P + n + e, l);
  }
}

// Vector entries owned by a CTA: the entries of the 8 x 8 tiles of H x that
// the CTA computes (tiles t = bid, bid + G, ...), so that the projections of a
// new w start without a grid barrier.  Local index q -> global index, or -1
// for the padding of a partial tile.
__device__ __forceinline__ long long own_index(int q, int bid, int G, int nt, int c) {
  const int t = bid + (q >> 6) * G, e = q & 63;
  const int row = (t / nt) * kLT + (e >> 3), col = (t % nt) * kLT + (e & 7);
  return (row < c && col < c) ? (long long)row * c + col : -1;
}

// Per-CTA sum of a[i] * b[i] over the owned entries, reduced in a fixed order.
__device__ double own_dot(LzSmem& sm, const double* a, const double* b, int nown, int bid, int G,
                          int nt, int c) {
  double s = 0.0;
  for (int q = threadIdx.x; q < nown; q += kLThreads) {
    const long long i = own_index(q, bid, G, nt, c);
    if (i >= 0) s = fma(__ldcg(a + i), __ldcg(b + i), s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[0][threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLWarps; ++w) t += sm.red[0][w];
    sm.bcast[1] = t;
  }
  __syncthreads();
  const double v = sm.bcast[1];
  __syncthreads();
  return v;
}

// part[bid][i] = <basis_i, w> over the owned entries for i <= j, and
// part[bid][nslot] = |w|^2 when nslot >= 0.  Warp w takes the vectors
// 4w .. 4w+3, 4w+32 .. (their loads issued together); each sum runs over the
// owned entries lane by lane, then a fixed butterfly.
__device__ void own_projections(const LanczosArgs& a, double* part, int ldp, int j, int nslot,
                                int nown, int bid, int G, int nt, int c, long long n) {
  constexpr int U = 4;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nv = j + 1 + (nslot >= 0 ? 1 : 0);
  for (int i0 = warp * U; i0 < nv; i0 += kLWarps * U) {
    double s[U];
#pragma unroll
    for (int u = 0; u < U; ++u) s[u] = 0.0;
    for (int q = lane; q < nown; q += 32) {
      const long long e = own_index(q, bid, G, nt, c);
      if (e < 0) continue;
      double bv[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int i = i0 + u;
        bv[u] = i < nv ? __ldcg((i > j ? a.w : a.basis + (long long)i * n) + e) : 0.0;
      }
      const double wv = __ldcg(a.w + e);
#pragma unroll
      for (int u = 0; u < U; ++u) s[u] = fma(bv[u], wv, s[u]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      for (int o = 16; o > 0; o >>= 1) s[u] += __shfl_xor_sync(0xffffffffu, s[u], o);
      const int i = i0 + u;
      if (lane == 0 && i < nv) __stcg(part + (long long)bid * ldp + (i > j ? nslot : i), s[u]);
    }
  }
}

// Copy cnt coefficients to shared memory (sm.cf).
__device__ __forceinline__ void load_coefs(LzSmem& sm, const double* cf, int cnt) {
  __syncthreads();
  for (int i = threadIdx.x; i < cnt; i += kLThreads) sm.cf[i] = __ldcg(cf + i);
  __syncthreads();
}

// For every owned entry e: f(e, base[e] + sgn * sum_{i < cnt} sm.cf[i] basis_i[e])
// (base may be null: 0).  S = 1, 2 or 4 threads share an entry, each summing
// the terms i = sub, sub + S, ... with eight loads in flight; the S partial
// sums are added in a fixed order.
template <typename Fn>
__device__ void owned_combine(const LanczosArgs& a, const LzSmem& sm, int cnt, const double* base,
                              double sgn, int nown, int bid, int G, int nt, int c, long long n,
                              Fn f) {
  const int S = nown >= kLThreads ? 1 : (nown > kLThreads / 4 ? 2 : 4);
  const int per = kLThreads / S, sub = threadIdx.x % S;
  for (int q0 = 0; q0 < nown; q0 += per) {
    const int q = q0 + threadIdx.x / S;
    const long long e = q < nown ? own_index(q, bid, G, nt, c) : -1;
    double s = 0.0;
    if (e >= 0) {
      int i = sub;
      for (; i + 7 * S < cnt; i += 8 * S) {
        double b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) b[u] = __ldcg(a.basis + (long long)(i + u * S) * n + e);
#pragma unroll
        for (int u = 0; u < 8; ++u) s = fma(sm.cf[i + u * S], b[u], s);
      }
      for (; i < cnt; i += S) s = fma(sm.cf[i], __ldcg(a.basis + (long long)i * n + e), s);
    }
    if (S >= 2) s += __shfl_down_sync(0xffffffffu, s, 1);
    if (S >= 4) s += __shfl_down_sync(0xffffffffu, s, 2);
    if (sub == 0 && e >= 0) f(e, (base ? __ldcg(base + e) : 0.0) + sgn * s);
  }
}

__global__ void __launch_bounds__(kLThreads, 2) lanczos_kernel(const LanczosArgs a) {
  __shared__ LzSmem sm;
  extern __shared__ __align__(16) float lz_dyn[];
  const int c = a.c, K = a.K, m = a.m;
  const long long n = (long long)c * c;
  const int G = gridDim.x, bid = blockIdx.x;
  const int nt = (c + kLT - 1) / kLT;
  const int ntiles = nt * nt;
  const int nown = (bid < ntiles ? (ntiles - bid + G - 1) / G : 0) * 64;
  const int ldp = m + 2;                     // stride of the per-CTA partial sums
  const int nslot = m + 1;                   // slot of |w|^2 in a CTA's partial sums
  double* part = a.part;
  double* wn2 = a.coef + 2 * ldp - 1;        // |w|^2 of the current step
  unsigned target = 0;

  const bool df = a.df != 0;
  const bool wide = df && a.wide != 0;
  const int ldw = lz_wide_ld(c);
  float* bp0 = df ? a.bp : nullptr;          // pairs of basis_0
  // start: the operators as pairs (double-float mode), Vprev = V, basis_0 = V / |V|
  if (df) {
    const long long nops = (long long)(1 + 2 * K) * n;
    const long long gt = (long long)blockIdx.x * kLThreads + threadIdx.x, gs = (long long)G * kLThreads;
    for (int side = 0; side < (a.s1 == a.s0 ? 1 : 2); ++side) {
      const double* src = side ? a.s1 : a.s0;
      float* dst = side ? a.s1p : a.s0p;
      for (long long e = gt; e < nops; e += gs) {
        const long long q = e / n, r = e % n;
        float h, l;
        split_d(__ldcg(src + e), h, l);
        __stcg(dst + 2 * q * n + r, h);
        __stcg(dst + 2 * q * n + n + r, l);
      }
    }
  }
  for (int q = threadIdx.x; q < nown; q += kLThreads) {
    const long long e = own_index(q, bid, G, nt, c);
    if (e >= 0) __stcg(a.Vprev + e, __ldcg(a.V + e));
  }
  {
    const double s = own_dot(sm, a.V, a.V, nown, bid, G, nt, c);
    if (threadIdx.x == 0) __stcg(part + (long long)bid * ldp, s);
  }
  if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
  double inv = 1.0 / sqrt(cta_ordered_sum(sm, part, G, ldp));
  for (int q = threadIdx.x; q < nown; q += kLThreads) {
    const long long e = own_index(q, bid, G, nt, c);
    if (e >= 0) store_both(a.basis, bp0, n, e, __ldcg(a.V + e) * inv);
  }
  if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
  const float* s0p = a.s0p;
  const float* s1p = a.s1 == a.s0 ? a.s0p : a.s1p;

  int conv = 0;
  for (int cyc = 0; cyc < a.restarts && !conv; ++cyc) {
    int tdim = 0;
    double beta_prev = 0.0;
    // Steps j >= 1 run on H - sigma I with sigma = alpha_0, the Rayleigh
    // quotient of the start vector (the same Krylov space; the tridiagonal is
    // shifted by -sigma, its first entry 0).  Without the shift |w|^2 ~ E^2
    // would dwarf beta_j^2 and every step would need the second
    // Gram-Schmidt pass.
    double sigma = 0.0;
    // Step j >= 1 also subtracts, while w is stored, the two recurrence terms
    // it knows: sigma_j x_j with sigma_j = alpha_{j-1} of H (the previous
    // step's diagonal entry, close to this one's) and beta_{j-1} x_{j-1}.  The
    // projections then only remove what is left (rounding and the small
    // alpha_j - sigma_j), so the one-pass test below passes in most steps and
    // the second Gram-Schmidt pass with its two grid barriers is skipped.  The
    // tridiagonal keeps the single shift sigma: its entry j is
    // c_j + sigma_j - sigma.
    double alpha_prev_h = 0.0;
    for (int j = 0; j < m; ++j) {
      const double* x = a.basis + (long long)j * n;
      const double sigma_j = j == 0 ? 0.0 : (j == 1 ? sigma : alpha_prev_h);
      const double* xprev = j > 0 ? x - n : nullptr;
      const double beta_j1 = j > 0 ? beta_prev : 0.0;
      // phase A: Y_b = Op_b x for the 2K operators A_k0, B_k0 (stored after o_0)
      const float* xp = df ? a.bp + 2 * (long long)j * n : nullptr;
      // wide staging: all 2K products of a tile by its CTA, the columns of x
      // staged once, the operator rows two at a time
      for (int t = bid; t < ntiles && wide; t += G) {
        const int i0 = (t / nt) * kLT, j0 = (t % nt) * kLT;
        for (int b0 = 0; b0 < 2 * K; b0 += 2) {
          const int nb = min(2, 2 * K - b0);
          if (b0 == 0) wide_cols(wide_slot(sm, lz_dyn, 0, ldw), xp, n, c, j0);
          for (int u = 0; u < nb; ++u)
            wide_rows(wide_slot(sm, lz_dyn, 1 + u, ldw), s0p + 2 * (long long)(1 + b0 + u) * n, n,
                      c, i0, ldw);
          cp_async_wait_all();
          __syncthreads();
          for (int u = 0; u < nb; ++u) {
            float a0h = 0.f, a0l = 0.f, a1h = 0.f, a1l = 0.f;
            wide_fma(wide_slot(sm, lz_dyn, 1 + u, ldw), wide_slot(sm, lz_dyn, 0, ldw), true, c, ldw,
                     a0h, a0l, a1h, a1l);
            tile_store_p(sm, a0h, a0l, a1h, a1l, a.Yp + 2 * (long long)(b0 + u) * n, nullptr, n, c,
                         i0, j0);
          }
        }
      }
      for (int it = bid; it < 2 * K * ntiles && !wide; it += G) {
        const int b = it / ntiles, t = it % ntiles;
        const int i0 = (t / nt) * kLT, j0 = (t % nt) * kLT;
        if (df) {
          stage_rows_p(sm.L, s0p + 2 * (long long)(1 + b) * n, n, c, i0);
          stage_cols_p(sm.R, xp, n, c, j0);
          __syncthreads();
          float a0h = 0.f, a0l = 0.f, a1h = 0.f, a1l = 0.f;
          tile_fma_p(sm, c, a0h, a0l, a1h, a1l);
          tile_store_p(sm, a0h, a0l, a1h, a1l, a.Yp + 2 * (long long)b * n, nullptr, n, c, i0, j0);
          continue;
        }
        stage_rows(sm.L, a.s0 + (long long)(1 + b) * n, c, i0, 1.0);
        stage_cols(sm.R, x, c, j0, 1.0);
        __syncthreads();
        double a0 = 0.0, a1 = 0.0;
        tile_fma(sm, c, a0, a1);
        tile_store(sm, a0, a1, a.Y + (long long)b * n, c, i0, j0);
      }
      if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
      // phase B: w = o_0 x + x o_1^T + sum_k Y_k B_k1^T + Y_{K+k} A_k1^T on the
      // owned tiles, then their projections on basis_0..j and |w|^2
      // wide staging: the operand tiles of up to four terms in one round
      for (int t = bid; t < ntiles && wide; t += G) {
        const int i0 = (t / nt) * kLT, j0 = (t % nt) * kLT;
        float a0h = 0.f, a0l = 0.f, a1h = 0.f, a1l = 0.f;
        const int nterms = 2 + 2 * K;
        for (int t0 = 0; t0 < nterms; t0 += kLWideSlots / 2) {
          const int tn = min(kLWideSlots / 2, nterms - t0);
          for (int u = 0; u < tn; ++u) {
            const int term = t0 + u;
            float* Ls = wide_slot(sm, lz_dyn, 2 * u, ldw);
            float* Rs = wide_slot(sm, lz_dyn, 2 * u + 1, ldw);
            if (term == 0) {
              wide_rows(Ls, s0p, n, c, i0, ldw);
              wide_cols(Rs, xp, n, c, j0);
            } else if (term == 1) {
              wide_rows(Ls, xp, n, c, i0, ldw);
              wide_rows(Rs, s1p, n, c, j0, ldw);
            } else {
              const int q = term - 2;          // Y_q with q < K: B_{q,1}; else A_{q-K,1}
              const long long rop = q < K ? (long long)(1 + K + q) : (long long)(1 + q - K);
              wide_rows(Ls, a.Yp + 2 * (long long)q * n, n, c, i0, ldw);
              wide_rows(Rs, s1p + 2 * rop * n, n, c, j0, ldw);
            }
          }
          cp_async_wait_all();
          __syncthreads();
          for (int u = 0; u < tn; ++u)
            wide_fma(wide_slot(sm, lz_dyn, 2 * u, ldw), wide_slot(sm, lz_dyn, 2 * u + 1, ldw),
                     t0 + u == 0, c, ldw, a0h, a0l, a1h, a1l);
          __syncthreads();
        }
        tile_store_p(sm, a0h, a0l, a1h, a1l, nullptr, a.w, n, c, i0, j0, x, sigma_j, xprev,
                     beta_j1);
      }
      for (int t = bid; t < ntiles && df && !wide; t += G) {
        const int i0 = (t / nt) * kLT, j0 = (t % nt) * kLT;
        float a0h = 0.f, a0l = 0.f, a1h = 0.f, a1l = 0.f;
        for (int term = 0; term < 2 + 2 * K; ++term) {
          if (term == 0) {
            stage_rows_p(sm.L, s0p, n, c, i0);
            stage_cols_p(sm.R, xp, n, c, j0);
          } else if (term == 1) {
            stage_rows_p(sm.L, xp, n, c, i0);
            stage_rows_p(sm.R, s1p, n, c, j0);
          } else {
            const int q = term - 2;            // Y_q with q < K: B_{q,1}; else A_{q-K,1}
            const long long rop = q < K ? (long long)(1 + K + q) : (long long)(1 + q - K);
            stage_rows_p(sm.L, a.Yp + 2 * (long long)q * n, n, c, i0);
            stage_rows_p(sm.R, s1p + 2 * rop * n, n, c, j0);
          }
          __syncthreads();
          tile_fma_p(sm, c, a0h, a0l, a1h, a1l);
          __syncthreads();
        }
        tile_store_p(sm, a0h, a0l, a1h, a1l, nullptr, a.w, n, c, i0, j0, x, sigma_j, xprev,
                     beta_j1);
      }
      for (int t = bid; t < ntiles && !df; t += G) {
        const int i0 = (t / nt) * kLT, j0 = (t % nt) * kLT;
        double a0 = 0.0, a1 = 0.0;
        for (int term = 0; term < 2 + 2 * K; ++term) {
          if (term == 0) {
            stage_rows(sm.L, a.s0, c, i0, 1.0);
            stage_cols(sm.R, x, c, j0, 1.0);
          } else if (term == 1) {
            stage_rows(sm.L, x, c, i0, 1.0);
            stage_rows(sm.R, a.s1, c, j0, 1.0);
          } else {
            const int q = term - 2;            // Y_q with q < K: B_{q,1}; else A_{q-K,1}
            const long long rop = q < K ? (long long)(1 + K + q) * n : (long long)(1 + q - K) * n;
            stage_rows(sm.L, a.Y + (long long)q * n, c, i0, 1.0);
            stage_rows(sm.R, a.s1 + rop, c, j0, 1.0);
          }
          __syncthreads();
          tile_fma(sm, c, a0, a1);
          __syncthreads();
        }
        tile_store(sm, a0, a1, a.w, c, i0, j0, x, sigma_j, xprev, beta_j1);
      }
      own_projections(a, part, ldp, j, nslot, nown, bid, G, nt, c, n);
      if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
      // coefficients of the first Gram-Schmidt pass and |w|^2 (one CTA each)
      for (int i = bid; i <= j + 1; i += G) {
        const double s = cta_ordered_sum(sm, part + (i > j ? nslot : i), G, ldp);
        if (threadIdx.x == 0) __stcg(i > j ? wn2 : a.coef + i, s);
      }
      if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
      // |w - sum c_i b_i|^2 = |w|^2 - sum c_i^2 for orthonormal b_i; when at
      // least a quarter of |w|^2 remains, one pass is accurate to rounding
      // (the second pass of "twice is enough" is needed only after heavy
      // cancellation), and the norm needs no further reduction
      const double w2 = __ldcg(wn2);
      load_coefs(sm, a.coef, j + 1);
      // sum of c_i^2 in a fixed order (lane-strided, then a butterfly): the
      // same value, and the same one-pass decision, in every CTA
      if (threadIdx.x < 32) {
        double t = 0.0;
        for (int i = threadIdx.x; i <= j; i += 32) t = fma(sm.cf[i], sm.cf[i], t);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) sm.bcast[2] = t;
      }
      __syncthreads();
      const double c2 = sm.bcast[2];
      const bool one_pass = w2 - c2 > 0.25 * w2;
      double alpha_j = sm.cf[j];
      double beta_j;
      if (one_pass) {
        beta_j = sqrt(w2 - c2);
      } else {
        // second pass: w1 = w - sum c_i b_i, then d_i = <b_i, w1> and |w1|^2 in
        // one reduction; |w1 - sum d_i b_i|^2 = |w1|^2 - sum d_i^2 (the d_i are
        // rounding-sized), and basis_{j+1} below subtracts sum d_i b_i
        owned_combine(a, sm, j + 1, a.w, -1.0, nown, bid, G, nt, c, n,
                      [&](long long e, double v) { __stcg(a.w + e, v); });
        __syncthreads();
        own_projections(a, part, ldp, j, nslot, nown, bid, G, nt, c, n);
        if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
        for (int i = bid; i <= j + 1; i += G) {
          const double s = cta_ordered_sum(sm, part + (i > j ? nslot : i), G, ldp);
          if (threadIdx.x == 0) __stcg(a.coef + ldp + i, s);
        }
        if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
        load_coefs(sm, a.coef + ldp, j + 2);
        if (threadIdx.x < 32) {
          double t = 0.0;
          for (int i = threadIdx.x; i <= j; i += 32) t = fma(sm.cf[i], sm.cf[i], t);
          for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
          if (threadIdx.x == 0) sm.bcast[2] = t;
        }
        __syncthreads();
        alpha_j += sm.cf[j];
        beta_j = sqrt(fmax(sm.cf[j + 1] - sm.bcast[2], 0.0));
      }
      if (j == 0) {
        sigma = alpha_j;
        alpha_j = 0.0;
      } else {
        alpha_j += sigma_j - sigma;
      }
      alpha_prev_h = alpha_j + sigma;
      tdim = j + 1;
      const bool breakdown = !(beta_j > 1e-12 * fmax(fabs(alpha_j + sigma) + beta_prev, 1e-300));
      if (bid == 0 && threadIdx.x == 0) {
        a.alpha[j] = alpha_j;
        a.beta[j] = breakdown ? 0.0 : beta_j;
      }
      if (breakdown) break;
      beta_prev = beta_j;
      // basis_{j+1} = (w - sum c_i b_i) / beta_j, or (w1 - sum d_i b_i) / beta_j
      inv = 1.0 / beta_j;
      double* nb = a.basis + (long long)(j + 1) * n;
      float* nbp = df ? a.bp + 2 * (long long)(j + 1) * n : nullptr;
      // (sm.cf holds the c_i of the one-pass path or the d_i of the second pass)
      owned_combine(a, sm, j + 1, a.w, -1.0, nown, bid, G, nt, c, n,
                    [&](long long e, double v) { store_both(nb, nbp, n, e, v * inv); });
      // every kLCheck steps CTA 0 tests the tridiagonal so far (pair
      // arithmetic); the cycle ends early once its Ritz pair passes the
      // convergence test
      const bool check = (j + 1) % kLCheck == 0 && j + 1 < m;
      if (check && bid == 0) {
        __syncthreads();
        if (threadIdx.x < 32) {
          const bool ok = ritz_check_df(sm, a.alpha, a.beta, j + 1, sigma, a.tol);
          if (threadIdx.x == 0) __stcg(a.scal + 3, ok ? 1.0 : 0.0);
        }
        __syncthreads();
      }
      if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
      if (check && __ldcg(a.scal + 3) != 0.0) break;
    }
    // Ritz pair of the tridiagonal (CTA 0), then V = sum_i y_i basis_i
    if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
    if (bid == 0) {
      ritz_pair(sm, a.alpha, a.beta, tdim, a.y, a.scal + 1, a.scal + 2);
      __syncthreads();
      if (threadIdx.x == 0) {
        // Ritz value of H: the tridiagonal's plus the shift
        const double theta = *(volatile double*)(a.scal + 1) + sigma;
        a.scal[1] = theta;
        a.flags[1] = tdim;
        a.flags[0] = *(volatile double*)(a.scal + 2) <= a.tol * fmax(fabs(theta), 1e-300);
        __threadfence();
      }
    }
    if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
    conv = __ldcg(a.flags);
    load_coefs(sm, a.y, tdim);
    owned_combine(a, sm, tdim, nullptr, 1.0, nown, bid, G, nt, c, n,
                  [&](long long e, double v) { __stcg(a.V + e, v); });
    __syncthreads();
    {
      const double s = own_dot(sm, a.V, a.V, nown, bid, G, nt, c);
      if (threadIdx.x == 0) __stcg(part + (long long)bid * ldp, s);
    }
    if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
    inv = 1.0 / sqrt(cta_ordered_sum(sm, part, G, ldp));
    for (int q = threadIdx.x; q < nown; q += kLThreads) {
      const long long e = own_index(q, bid, G, nt, c);
      if (e < 0) continue;
      const double t = __ldcg(a.V + e) * inv;
      __stcg(a.V + e, t);
      store_both(a.basis, bp0, n, e, t);
    }
    if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
  }
  // sign: <V, Vprev> >= 0
  {
    const double s = own_dot(sm, a.V, a.Vprev, nown, bid, G, nt, c);
    if (threadIdx.x == 0) __stcg(part + (long long)bid * ldp + 1, s);
  }
  if (!lz_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kLMaxSpin)) return;
  if (cta_ordered_sum(sm, part + 1, G, ldp) < 0.0)
    for (int q = threadIdx.x; q < nown; q += kLThreads) {
      const long long e = own_index(q, bid, G, nt, c);
      if (e >= 0) __stcg(a.V + e, -__ldcg(a.V + e));
    }
}

struct LzGrid {
  int sms = 0, per_sm = 0;
};
std::mutex g_lz_mutex;
LzGrid g_lz_grid[64];

int lanczos_grid_cap() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(g_lz_mutex);
  LzGrid& g = g_lz_grid[dev];
  if (!g.sms) {
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    // (with the wide staging's dynamic shared memory at its largest)
    const int dyn = (int)lz_wide_dyn_bytes(kLWideMaxC);
    if (cudaFuncSetAttribute(lanczos_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) !=
        cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lanczos_kernel, kLThreads, dyn) !=
        cudaSuccess)
      return 0;
    g.sms = sms;
    g.per_sm = std::min(occ, 2);
  }
  return g.sms * g.per_sm;
}

}  // namespace

bool lanczos_supported(int c, int m) { return c >= 1 && c <= kLMaxC && m >= 2 && m <= kLMaxM; }

int lanczos_grid(int c, int grid_share) {
  int cap = lanczos_grid_cap();
  if (cap <= 0) return 0;
  if (grid_share > 1) cap = std::max(1, cap / grid_share);
  const long long n = (long long)c * c;
  // no more CTAs than 64-entry slices of the vectors, at least one
  return (int)std::max<long long>(1, std::min<long long>(std::min(cap, kLMaxGrid), n / 64));
}

int lanczos_launch(const LanczosArgs& a0, int grid, cudaStream_t s) {
  if (!lanczos_supported(a0.c, a0.m) || grid < 1 || grid > kLMaxGrid) return -1;
  // the grid cap also sets the kernel's dynamic shared-memory limit
  if (lanczos_grid_cap() <= 0) return -1;
  LanczosArgs a = a0;
  a.wide = a.df != 0 && a.c <= kLWideMaxC && a.c % 8 == 0 ? 1 : 0;
  cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kLThreads);
  cfg.dynamicSmemBytes = a.wide ? lz_wide_dyn_bytes(a.c) : 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, lanczos_kernel, a) != cudaSuccess) return -1;
  return 1;
}

}  // namespace ttn
