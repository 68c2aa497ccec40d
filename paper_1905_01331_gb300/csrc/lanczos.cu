// Top-tensor update (Sec. III.B: the top tensor is "updated similarly"; read
// as the lowest eigenvector of the top Hamiltonian) as one persistent
// cooperative launch: restarted Lanczos in FP64 with full reorthogonalisation
// (two classical Gram-Schmidt passes), warm-started from the previous V.
//
// H_top acts on the c x c top tensor V as
//     H V = o_0 V + V o_1^T + sum_k (A_k0 V B_k1^T + B_k0 V A_k1^T),
// with (o, A_k, B_k) the identity-free operators of the two top sites (the
// two bonds of the periodic ring at the top).  One Lanczos step is
//     phase A   Y_k = A_k0 x, Y_{K+k} = B_k0 x               (2K products)
//     phase B   w = o_0 x + x o_1^T + sum_k Y_k B_k1^T + Y_{K+k} A_k1^T
//     dots/reduce/subtract twice, then |w| and alpha_j, beta_j
// with every phase shared by all CTAs and a grid barrier between phases
// (bounded spin, error flag).  Vector phases split the n = c^2 entries into
// one contiguous slice per CTA; every reduction adds its per-CTA partial
// sums in a fixed order, so the result does not depend on timing.  The
// eigenpair of the tridiagonal matrix is found by CTA 0 (bisection by Sturm
// counts, first in FP32 to bracket, then in FP64, and inverse iteration).
#include <algorithm>
#include <mutex>

#include "common.h"
#include "pair_arith.cuh"

namespace ttn {

namespace {

constexpr int kLT = 8;                   // output tile edge of the matrix products
constexpr int kLThreads = 256;
constexpr int kLWarps = kLThreads / 32;
constexpr int kLMaxC = 256;
constexpr int kLMaxSpin = 1 << 23;       // ~1 s of polling, then the error flag

struct LzSmem {
  double L[kLT][kLMaxC + 1];             // left-operand rows of a tile
  double R[kLT][kLMaxC + 1];             // right-operand rows (or columns) of a tile
  double red[kLWarps][kLT * kLT];
  double tri[6][kLMaxM + 2];             // inverse iteration scratch (CTA 0)
  double da[kLMaxM + 2], db2[kLMaxM + 2];  // tridiagonal: diagonal, squared off-diagonal
  float fa[kLMaxM + 2], fb2[kLMaxM + 2];
  double bcast[4];
  int ok;
};

__device__ bool lz_barrier(LzSmem& sm, unsigned* bar, unsigned& target, int* err) {
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    __threadfence();
    atomicAdd(bar, 1u);
    int spins = 0;
    while (*reinterpret_cast<volatile unsigned*>(bar) < target) {
      if (*reinterpret_cast<volatile int*>(err)) { ok = 0; break; }
      if (++spins > kLMaxSpin) { atomicOr(err, 4); ok = 0; break; }
      __nanosleep(128);
    }
    __threadfence();
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

// Stage rows [r0, r0+8) of the row-major c x c matrix M (times scale) into dst.
__device__ void stage_rows(double (*dst)[kLMaxC + 1], const double* M, int c, int r0, double scale) {
  for (int e = threadIdx.x; e < kLT * c; e += kLThreads) {
    const int r = e / c, k = e - r * c;
    dst[r][k] = r0 + r < c ? scale * __ldcg(M + (long long)(r0 + r) * c + k) : 0.0;
  }
}
// Stage columns [c0, c0+8) of M (times scale) as rows of dst: dst[j][k] = M[k][c0 + j].
__device__ void stage_cols(double (*dst)[kLMaxC + 1], const double* M, int c, int c0, double scale) {
  for (int e = threadIdx.x; e < kLT * c; e += kLThreads) {
    const int k = e / kLT, j = e - k * kLT;
    dst[j][k] = c0 + j < c ? scale * __ldcg(M + (long long)k * c + c0 + j) : 0.0;
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

// Reduce the per-warp partial sums of a tile in warp order and store it.
__device__ void tile_store(LzSmem& sm, double a0, double a1, double* C, int c, int i0, int j0) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  sm.red[warp][i * kLT + j] = a0;
  sm.red[warp][i * kLT + j + 1] = a1;
  __syncthreads();
  if (threadIdx.x < kLT * kLT) {
    double v = 0.0;
    for (int w = 0; w < kLWarps; ++w) v += sm.red[w][threadIdx.x];
    const int r = threadIdx.x / kLT, cc = threadIdx.x % kLT;
    if (i0 + r < c && j0 + cc < c) __stcg(C + (long long)(i0 + r) * c + j0 + cc, v);
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

// 32-way multisection of [lo, hi] for the lowest eigenvalue, by one warp,
// until the interval is narrower than rel * max(|lo|, |hi|) or `its` rounds.
template <typename T>
__device__ void multisect(const T* a, const T* b2, int m, T& lo, T& hi, T rel, int its) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < its; ++it) {
    const T mag = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
    if (!(hi - lo > rel * mag)) break;
    const T pt = lo + (hi - lo) * (T)(lane + 1) / (T)33;
    const unsigned below = __ballot_sync(0xffffffffu, sturm_below<T>(a, b2, m, pt) >= 1);
    const int f = below ? __ffs(below) - 1 : 32;
    const T nlo = f == 0 ? lo : lo + (hi - lo) * (T)f / (T)33;
    const T nhi = f == 32 ? hi : lo + (hi - lo) * (T)(f + 1) / (T)33;
    lo = nlo;
    hi = nhi;
  }
}

// Lowest eigenpair of the m x m tridiagonal (alpha, beta) by warp 0 of the
// calling CTA: y (m entries, unit norm), theta, residual |beta_{m-1} y_{m-1}|.
__device__ void ritz_pair(LzSmem& sm, const double* alpha, const double* beta, int m, double* y,
                          double* theta, double* res) {
  if (threadIdx.x >= 32) return;
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
  const int c_lo = sturm_below<double>(sm.da, sm.db2, m, lo);
  const int c_hi = sturm_below<double>(sm.da, sm.db2, m, hi);
  if (!__all_sync(0xffffffffu, c_lo == 0 && c_hi >= 1)) { lo = glo; hi = ghi; }
  multisect<double>(sm.da, sm.db2, m, lo, hi, 4e-16, 16);
  if (lane != 0) return;
  const double th = 0.5 * (lo + hi);
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
  for (int e = threadIdx.x; e < kLT * c; e += kLThreads) {
    const int r = e / c, k = e - r * c;
    const bool ok = r0 + r < c;
    const long long i = (long long)(r0 + r) * c + k;
    h[r][k] = ok ? __ldcg(M + i) : 0.f;
    l[r][k] = ok ? __ldcg(M + n + i) : 0.f;
  }
}
// columns [c0, c0+8) of M as rows: dst[j][k] = M[k][c0 + j]
__device__ void stage_cols_p(double (*dst)[kLMaxC + 1], const float* M, long long n, int c,
                             int c0) {
  FRow* h = frows(dst, 0);
  FRow* l = frows(dst, 1);
  for (int e = threadIdx.x; e < kLT * c; e += kLThreads) {
    const int k = e / kLT, j = e - k * kLT;
    const bool ok = c0 + j < c;
    const long long i = (long long)k * c + c0 + j;
    h[j][k] = ok ? __ldcg(M + i) : 0.f;
    l[j][k] = ok ? __ldcg(M + n + i) : 0.f;
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
// pairs (Cp) or as FP64 (Cd).
__device__ void tile_store_p(LzSmem& sm, float a0h, float a0l, float a1h, float a1l, float* Cp,
                             double* Cd, long long n, int c, int i0, int j0) {
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
      if (Cd) __stcg(Cd + e, (double)vh + (double)vl);
    }
  }
  __syncthreads();
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

// part[bid][i] = <basis_i, w> over the owned entries for i <= j (one warp per
// vector), and part[bid][nslot] = |w|^2 when nslot >= 0.
__device__ void own_projections(const LanczosArgs& a, double* part, int ldp, int j, int nslot,
                                int nown, int bid, int G, int nt, int c, long long n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i <= j + (nslot >= 0 ? 1 : 0); i += kLWarps) {
    const bool norm = i > j;
    const double* bi = norm ? a.w : a.basis + (long long)i * n;
    double s = 0.0;
    for (int q = lane; q < nown; q += 32) {
      const long long e = own_index(q, bid, G, nt, c);
      if (e >= 0) s = fma(__ldcg(bi + e), __ldcg(a.w + e), s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) __stcg(part + (long long)bid * ldp + (norm ? nslot : i), s);
  }
}

__global__ void __launch_bounds__(kLThreads) lanczos_kernel(const LanczosArgs a) {
  __shared__ LzSmem sm;
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
  if (!lz_barrier(sm, a.bar, target, a.err)) return;
  double inv = 1.0 / sqrt(cta_ordered_sum(sm, part, G, ldp));
  for (int q = threadIdx.x; q < nown; q += kLThreads) {
    const long long e = own_index(q, bid, G, nt, c);
    if (e >= 0) store_both(a.basis, bp0, n, e, __ldcg(a.V + e) * inv);
  }
  if (!lz_barrier(sm, a.bar, target, a.err)) return;
  const float* s0p = a.s0p;
  const float* s1p = a.s1 == a.s0 ? a.s0p : a.s1p;

  int conv = 0;
  for (int cyc = 0; cyc < a.restarts && !conv; ++cyc) {
    int tdim = 0;
    double beta_prev = 0.0;
    for (int j = 0; j < m; ++j) {
      const double* x = a.basis + (long long)j * n;
      // phase A: Y_b = Op_b x for the 2K operators A_k0, B_k0 (stored after o_0)
      const float* xp = df ? a.bp + 2 * (long long)j * n : nullptr;
      for (int it = bid; it < 2 * K * ntiles; it += G) {
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
      if (!lz_barrier(sm, a.bar, target, a.err)) return;
      // phase B: w = o_0 x + x o_1^T + sum_k Y_k B_k1^T + Y_{K+k} A_k1^T on the
      // owned tiles, then their projections on basis_0..j and |w|^2
      for (int t = bid; t < ntiles && df; t += G) {
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
        tile_store_p(sm, a0h, a0l, a1h, a1l, nullptr, a.w, n, c, i0, j0);
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
        tile_store(sm, a0, a1, a.w, c, i0, j0);
      }
      own_projections(a, part, ldp, j, nslot, nown, bid, G, nt, c, n);
      if (!lz_barrier(sm, a.bar, target, a.err)) return;
      // coefficients of the first Gram-Schmidt pass and |w|^2 (one CTA each)
      for (int i = bid; i <= j + 1; i += G) {
        const double s = cta_ordered_sum(sm, part + (i > j ? nslot : i), G, ldp);
        if (threadIdx.x == 0) __stcg(i > j ? wn2 : a.coef + i, s);
      }
      if (!lz_barrier(sm, a.bar, target, a.err)) return;
      // |w - sum c_i b_i|^2 = |w|^2 - sum c_i^2 for orthonormal b_i; when at
      // least a quarter of |w|^2 remains, one pass is accurate to rounding
      // (the second pass of "twice is enough" is needed only after heavy
      // cancellation), and the norm needs no further reduction
      const double w2 = __ldcg(wn2);
      double c2 = 0.0;
      for (int i = 0; i <= j; ++i) {
        const double ci = __ldcg(a.coef + i);
        c2 = fma(ci, ci, c2);
      }
      const bool one_pass = w2 - c2 > 0.25 * w2;
      double alpha_j = __ldcg(a.coef + j);
      double beta_j;
      if (one_pass) {
        beta_j = sqrt(w2 - c2);
      } else {
        for (int q = threadIdx.x; q < nown; q += kLThreads) {
          const long long e = own_index(q, bid, G, nt, c);
          if (e < 0) continue;
          double s = __ldcg(a.w + e);
          for (int i = 0; i <= j; ++i)
            s = fma(-__ldcg(a.coef + i), __ldcg(a.basis + (long long)i * n + e), s);
          __stcg(a.w + e, s);
        }
        __syncthreads();
        own_projections(a, part, ldp, j, -1, nown, bid, G, nt, c, n);
        if (!lz_barrier(sm, a.bar, target, a.err)) return;
        for (int i = bid; i <= j; i += G) {
          const double s = cta_ordered_sum(sm, part + i, G, ldp);
          if (threadIdx.x == 0) __stcg(a.coef + ldp + i, s);
        }
        if (!lz_barrier(sm, a.bar, target, a.err)) return;
        for (int q = threadIdx.x; q < nown; q += kLThreads) {
          const long long e = own_index(q, bid, G, nt, c);
          if (e < 0) continue;
          double s = __ldcg(a.w + e);
          for (int i = 0; i <= j; ++i)
            s = fma(-__ldcg(a.coef + ldp + i), __ldcg(a.basis + (long long)i * n + e), s);
          __stcg(a.w + e, s);
        }
        __syncthreads();
        alpha_j += __ldcg(a.coef + ldp + j);
        {
          const double s = own_dot(sm, a.w, a.w, nown, bid, G, nt, c);
          if (threadIdx.x == 0) __stcg(part + (long long)bid * ldp, s);
        }
        if (!lz_barrier(sm, a.bar, target, a.err)) return;
        beta_j = sqrt(fmax(cta_ordered_sum(sm, part, G, ldp), 0.0));
      }
      tdim = j + 1;
      const bool breakdown = !(beta_j > 1e-12 * fmax(fabs(alpha_j) + beta_prev, 1e-300));
      if (bid == 0 && threadIdx.x == 0) {
        a.alpha[j] = alpha_j;
        a.beta[j] = breakdown ? 0.0 : beta_j;
      }
      if (breakdown) break;
      beta_prev = beta_j;
      // basis_{j+1} = (w - sum c_i b_i) / beta_j (the projection is applied
      // here on the one-pass path)
      inv = 1.0 / beta_j;
      double* nb = a.basis + (long long)(j + 1) * n;
      for (int q = threadIdx.x; q < nown; q += kLThreads) {
        const long long e = own_index(q, bid, G, nt, c);
        if (e < 0) continue;
        double s = __ldcg(a.w + e);
        if (one_pass)
          for (int i = 0; i <= j; ++i)
            s = fma(-__ldcg(a.coef + i), __ldcg(a.basis + (long long)i * n + e), s);
        store_both(nb, df ? a.bp + 2 * (long long)(j + 1) * n : nullptr, n, e, s * inv);
      }
      if (!lz_barrier(sm, a.bar, target, a.err)) return;
    }
    // Ritz pair of the tridiagonal (CTA 0), then V = sum_i y_i basis_i
    if (!lz_barrier(sm, a.bar, target, a.err)) return;
    if (bid == 0) {
      ritz_pair(sm, a.alpha, a.beta, tdim, a.y, a.scal + 1, a.scal + 2);
      __syncthreads();
      if (threadIdx.x == 0) {
        a.flags[1] = tdim;
        a.flags[0] = *(volatile double*)(a.scal + 2) <=
                     a.tol * fmax(fabs(*(volatile double*)(a.scal + 1)), 1e-300);
        __threadfence();
      }
    }
    if (!lz_barrier(sm, a.bar, target, a.err)) return;
    conv = __ldcg(a.flags);
    for (int q = threadIdx.x; q < nown; q += kLThreads) {
      const long long e = own_index(q, bid, G, nt, c);
      if (e < 0) continue;
      double s = 0.0;
      for (int i = 0; i < tdim; ++i) s = fma(__ldcg(a.y + i), __ldcg(a.basis + (long long)i * n + e), s);
      __stcg(a.V + e, s);
    }
    __syncthreads();
    {
      const double s = own_dot(sm, a.V, a.V, nown, bid, G, nt, c);
      if (threadIdx.x == 0) __stcg(part + (long long)bid * ldp, s);
    }
    if (!lz_barrier(sm, a.bar, target, a.err)) return;
    inv = 1.0 / sqrt(cta_ordered_sum(sm, part, G, ldp));
    for (int q = threadIdx.x; q < nown; q += kLThreads) {
      const long long e = own_index(q, bid, G, nt, c);
      if (e < 0) continue;
      const double t = __ldcg(a.V + e) * inv;
      __stcg(a.V + e, t);
      store_both(a.basis, bp0, n, e, t);
    }
    if (!lz_barrier(sm, a.bar, target, a.err)) return;
  }
  // sign: <V, Vprev> >= 0
  {
    const double s = own_dot(sm, a.V, a.Vprev, nown, bid, G, nt, c);
    if (threadIdx.x == 0) __stcg(part + (long long)bid * ldp + 1, s);
  }
  if (!lz_barrier(sm, a.bar, target, a.err)) return;
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
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, lanczos_kernel, kLThreads, 0) !=
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

int lanczos_launch(const LanczosArgs& a, int grid, cudaStream_t s) {
  if (!lanczos_supported(a.c, a.m) || grid < 1 || grid > kLMaxGrid) return -1;
  cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kLThreads);
  cfg.dynamicSmemBytes = 0;
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
