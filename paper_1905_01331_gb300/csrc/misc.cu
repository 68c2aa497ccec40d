// Reductions, elementwise steps and the Lanczos bookkeeping of the sweep.
// Every reduction is two-pass with a fixed summation order (deterministic).
#include <cmath>

#include "common.h"
#include "f64_bits.cuh"

namespace ttn {

namespace {

__device__ double block_sum(double v) {
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  v = 0.0;
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    v = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;  // valid in thread 0
}

// partial[b * kDotBlocks + blk] = sum over this block's slice of x*y
__global__ void dot_partial_kernel(const double* x, const double* y, long long n,
                                   long long stride, double* partial, const int* skip) {
  pdl_wait();
  pdl_trigger();
  if (skip && *skip) return;
  const int b = blockIdx.y, blk = blockIdx.x;
  const double* xb = x + b * stride;
  const double* yb = y + b * stride;
  // two interleaved accumulators (FP64 latency on this GPU), added at the end
  double s0 = 0.0, s1 = 0.0;
  const long long step = (long long)gridDim.x * blockDim.x;
  long long i = blk * (long long)blockDim.x + threadIdx.x;
  for (; i + step < n; i += 2 * step) {
    s0 = fma(xb[i], yb[i], s0);
    s1 = fma(xb[i + step], yb[i + step], s1);
  }
  if (i < n) s0 = fma(xb[i], yb[i], s0);
  const double s = block_sum(s0 + s1);
  if (threadIdx.x == 0) partial[b * kDotBlocks + blk] = s;
}

// The two sums <x, x> and <x, y> of the damped polar start in one pass over x:
// partial[b * kDotBlocks + blk] as dot_partial_kernel for <x, x>, and at
// partial[(nb + b) * kDotBlocks + blk] for <x, y> (the same order of terms).
__global__ void dot2_partial_kernel(const double* x, const double* y, long long n, long long stride,
                                    int nb, double* partial) {
  pdl_wait();
  pdl_trigger();
  const int b = blockIdx.y, blk = blockIdx.x;
  const double* xb = x + b * stride;
  const double* yb = y + b * stride;
  double s0 = 0.0, s1 = 0.0, t0 = 0.0, t1 = 0.0;
  const long long step = (long long)gridDim.x * blockDim.x;
  long long i = blk * (long long)blockDim.x + threadIdx.x;
  for (; i + step < n; i += 2 * step) {
    const double a = xb[i], c = xb[i + step];
    s0 = fma(a, a, s0);
    s1 = fma(c, c, s1);
    t0 = fma(a, yb[i], t0);
    t1 = fma(c, yb[i + step], t1);
  }
  if (i < n) {
    const double a = xb[i];
    s0 = fma(a, a, s0);
    t0 = fma(a, yb[i], t0);
  }
  const double s = block_sum(s0 + s1);
  if (threadIdx.x == 0) partial[b * kDotBlocks + blk] = s;
  __syncthreads();   // block_sum's shared scratch is reused
  const double t = block_sum(t0 + t1);
  if (threadIdx.x == 0) partial[(nb + b) * kDotBlocks + blk] = t;
}

// out[b] = sum of the kDotBlocks partial sums of batch b: one warp per batch,
// lane-strided sums, then a fixed butterfly.
__global__ void dot_final_kernel(const double* partial, int nb, double* out, const int* skip) {
  pdl_wait();
  pdl_trigger();
  if (skip && *skip) return;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (b >= nb) return;
  double s = 0.0;
  for (int i = lane; i < kDotBlocks; i += 32) s += partial[b * kDotBlocks + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[b] = s;
}

__global__ void polar_start_kernel(const double* G, const double* W, double* X, long long elems,
                                   int P, double mu, const double* part, int nb, float* xh,
                                   float* xl, int* zero, const int* try_first, int* run_full,
                                   int* zero2) {
  pdl_wait();
  pdl_trigger();
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
    if (zero) *zero = 0;
    if (zero2) *zero2 = 0;
    // the full schedule runs unless the layer is predicted well conditioned
    if (run_full) *run_full = *try_first ? 0 : 1;
  }
  const int b = blockIdx.y;
  // |G|^2 and <G, W> from the partial sums of dot2_partial_kernel, summed by
  // warp 0 of every CTA exactly as dot_final_kernel sums them (lane-strided,
  // then a fixed butterfly): the same two values in every CTA
  __shared__ double sums[2];
  if (threadIdx.x < 32) {
    double a = 0.0, c = 0.0;
    for (int i = threadIdx.x; i < kDotBlocks; i += 32) {
      a += part[b * kDotBlocks + i];
      c += part[(nb + b) * kDotBlocks + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (threadIdx.x == 0) { sums[0] = a; sums[1] = c; }
  }
  __syncthreads();
  const double f2 = sums[0];
  const double s = mu * sqrt(f2);
  const double nrm2 = f2 - 2.0 * s * sums[1] + s * s * P;
  const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
  const double* g = G + b * elems;
  const double* w = W + b * elems;
  double* x = X + b * elems;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < elems;
       i += (long long)gridDim.x * blockDim.x) {
    const double v = (g[i] - s * w[i]) * inv;
    // mixed modes (one batch): only the FP32 pair of X, which is all that the
    // double-float products read (X itself is not written)
    if (xh)
      f64b::split(v, xh[i], xl[i]);
    else
      x[i] = v;
  }
}

__global__ void poly_step_kernel(const double* A, double* Pm, int P, double a, double c) {
  pdl_wait();
  pdl_trigger();
  const int b = blockIdx.y;
  const long long PP = (long long)P * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < PP;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / P), j = (int)(e % P);
    Pm[b * PP + e] = (i == j ? a : 0.0) - c * A[b * PP + e];
  }
}

__global__ void identity_kernel(double* F, int P) {
  pdl_wait();
  pdl_trigger();
  const int b = blockIdx.y;
  const long long PP = (long long)P * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < PP;
       e += (long long)gridDim.x * blockDim.x)
    F[b * PP + e] = (e / P == e % P) ? 1.0 : 0.0;
}

__global__ void axpby_kernel(const double* x, double* y, long long n, double alpha, double beta) {
  pdl_wait();
  pdl_trigger();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = alpha * x[i] + beta * y[i];
}

__global__ void scale_select_kernel(const double* x0, const double* x1, const int* sel, double* y,
                                    long long n, double alpha, float* y32, const float* corr,
                                    int* pred, int pstride, int retry, const double* x2,
                                    const int* sel2) {
  pdl_wait();
  pdl_trigger();
  if (pred && blockIdx.x == 0 && threadIdx.x == 0) {
    // next sweep's prediction: a failed first try switches the layer to the
    // full schedule, which tries the first block again after `retry` sweeps
    int& try_first = pred[0];
    int& count = pred[2 * pstride];
    if (try_first) {
      if (pred[pstride]) { try_first = 0; count = 0; }
    } else if (++count >= retry) {
      try_first = 1;
      count = 0;
    }
  }
  const bool one = *sel != 0;
  // with sel2: the sel branch is x2 when *sel2, else x1 plus the correction
  const bool two = one && sel2 && *sel2 != 0;
  const bool add = corr && (!one || (sel2 && !two));
  const double* x = two ? x2 : (one ? x1 : x0);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double xi = x[i];
    if (add) xi += f64b::from_f32(corr[i]);
    const double v = alpha * xi;
    y[i] = v;
    if (y32) y32[i] = f64b::to_f32(v);
  }
}

__global__ void symmetrize_kernel(double* A, int P) {
  pdl_wait();
  pdl_trigger();
  const int b = blockIdx.y;
  double* a = A + (long long)b * P * P;
  const long long PP = (long long)P * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < PP;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / P), j = (int)(e % P);
    if (i < j) {
      const double v = 0.5 * (a[i * (long long)P + j] + a[j * (long long)P + i]);
      a[i * (long long)P + j] = v;
      a[j * (long long)P + i] = v;
    }
  }
}

// ---- Lanczos -------------------------------------------------------------

// partial[i * kDotBlocks + blk] = <basis_i, w> over this block's slice
__global__ void lz_dots_partial(const double* basis, long long n, int count, const double* w,
                                double* partial, const int* skip) {
  pdl_wait();
  pdl_trigger();
  if (*skip) return;
  const int i = blockIdx.y;
  if (i >= count) return;
  const double* v = basis + i * n;
  double s = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    s = fma(v[e], w[e], s);
  s = block_sum(s);
  if (threadIdx.x == 0) partial[i * kDotBlocks + blockIdx.x] = s;
}

__global__ void lz_dots_final(const double* partial, int count, double* coef, const int* skip) {
  pdl_wait();
  pdl_trigger();
  if (*skip) return;
  const int i = threadIdx.x;
  if (i >= count) return;
  double s = 0.0;
  for (int b = 0; b < kDotBlocks; ++b) s += partial[i * kDotBlocks + b];
  coef[i] = s;
}

__global__ void lz_sub_kernel(const double* basis, long long n, int count, double* w,
                              const double* coef, const int* skip) {
  pdl_wait();
  pdl_trigger();
  if (*skip) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = w[e];
    for (int i = 0; i < count; ++i) s = fma(-coef[i], basis[i * n + e], s);
    w[e] = s;
  }
}

// alpha_j from the two projection passes, beta_j = |w|; breakdown stops the run.
__global__ void lz_step_scalars(const double* c1, const double* c2, int j, double* alpha,
                                double* beta, const double* nrm2, int* skip, int* tdim) {
  pdl_wait();
  pdl_trigger();
  if (*skip) return;
  const double a = c1[j] + c2[j];
  alpha[j] = a;
  const double b = sqrt(fmax(nrm2[0], 0.0));
  beta[j] = b;
  *tdim = j + 1;
  const double scale = fabs(a) + (j > 0 ? beta[j - 1] : 0.0);
  if (!(b > 1e-12 * fmax(scale, 1e-300))) { beta[j] = 0.0; *skip = 1; }
}

__global__ void lz_scale_into(double* dst, const double* w, long long n, const double* beta, int j,
                              const int* skip) {
  pdl_wait();
  pdl_trigger();
  if (*skip) return;
  const double inv = 1.0 / beta[j];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    dst[e] = w[e] * inv;
}

// Sturm count: number of eigenvalues of the tridiagonal T (size m) below x.
__device__ int sturm_count(const double* a, const double* b, int m, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < m; ++i) {
    if (q == 0.0) q = 1e-300;
    q = a[i] - x - b[i - 1] * b[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Lowest eigenpair of the Lanczos tridiagonal by bisection and inverse
// iteration (Gaussian elimination with partial pivoting on the band).
__global__ void lz_ritz_kernel(const double* alpha, const double* beta, const int* tdim, int jmax,
                               double* y, double* theta, double* res, int* conv, double tol,
                               const int* skip_before) {
  pdl_wait();
  pdl_trigger();
  // one warp: 32-way multisection of the Gershgorin interval for the lowest
  // eigenvalue (each lane counts eigenvalues below its own point), then lane 0
  // runs the inverse iteration
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  if (*conv) return;
  const int lane = threadIdx.x;
  const int m = *tdim;
  double lo = alpha[0], hi = alpha[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < m ? fabs(beta[i]) : 0.0);
    lo = fmin(lo, alpha[i] - r);
    hi = fmax(hi, alpha[i] + r);
  }
  for (int it = 0; it < 16; ++it) {
    if (!(hi - lo > 4e-16 * fmax(fabs(lo), fabs(hi)))) break;
    const double pt = lo + (hi - lo) * (lane + 1) / 33.0;
    const unsigned below = __ballot_sync(0xffffffffu, sturm_count(alpha, beta, m, pt) >= 1);
    // first lane whose point has the lowest eigenvalue below it
    const int f = below ? __ffs(below) - 1 : 32;
    const double nlo = f == 0 ? lo : lo + (hi - lo) * f / 33.0;
    const double nhi = f == 32 ? hi : lo + (hi - lo) * (f + 1) / 33.0;
    lo = nlo;
    hi = nhi;
  }
  if (lane != 0) return;
  const double th = 0.5 * (lo + hi);
  // inverse iteration on (T - th I) x = x_prev, 3 rounds
  double x[128], dd[128], du[128], du2[128], rhs[128];
  for (int i = 0; i < m; ++i) x[i] = 1.0 / sqrt((double)m);
  const double eps = fmax(fabs(th), 1.0) * 1e-15;
  for (int round = 0; round < 2; ++round) {
    for (int i = 0; i < m; ++i) { dd[i] = alpha[i] - th; du[i] = i + 1 < m ? beta[i] : 0.0; du2[i] = 0.0; rhs[i] = x[i]; }
    double dl[128];
    for (int i = 0; i + 1 < m; ++i) dl[i] = beta[i];
    // LU with partial pivoting of the tridiagonal (LAPACK gttrf-style)
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
    // back substitution
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
  for (int i = 0; i < jmax; ++i) y[i] = i < m ? x[i] : 0.0;
  *theta = th;
  const double r = fabs(beta[m - 1] * x[m - 1]);
  *res = r;
  if (r <= tol * fmax(fabs(th), 1e-300)) *conv = 1;
}

__global__ void lz_combine_kernel(const double* basis, long long n, const int* tdim, const double* y,
                                  double* v) {
  pdl_wait();
  pdl_trigger();
  const int m = *tdim;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < m; ++i) s = fma(y[i], basis[i * n + e], s);
    v[e] = s;
  }
}

__global__ void scale_by_inv_sqrt(double* v, long long n, const double* nrm2, double* dst0) {
  pdl_wait();
  pdl_trigger();
  const double inv = 1.0 / sqrt(nrm2[0]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const double t = v[e] * inv;
    v[e] = t;
    if (dst0) dst0[e] = t;
  }
}

__global__ void lz_reset_kernel(int* tdim, int* skip, const int* conv) {
  pdl_wait();
  pdl_trigger();
  *tdim = 1;
  *skip = *conv;
}

__global__ void flip_if_negative(double* v, long long n, const double* dotv) {
  pdl_wait();
  pdl_trigger();
  if (dotv[0] >= 0.0) return;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    v[e] = -v[e];
}

__global__ void ordered_sum_kernel(const double* x, int count, double* out, double scale,
                                   double add) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < count; ++i) s += x[i];
  *out = scale * s + add;
}

__global__ void finite_kernel(const double* x, long long n, int* flag) {
  pdl_wait();
  pdl_trigger();
  int bad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[e])) bad = 1;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1);
}

__global__ void split_identity_kernel(double* O, long long stride, int P, const double* e_in,
                                      int per_node, double* e_out) {
  pdl_wait();
  pdl_trigger();
  const int J = blockIdx.x;
  double* o = O + J * stride;
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < P; i += blockDim.x) s += o[(long long)i * P + i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  const double tr = sh[0] / P;
  for (int i = threadIdx.x; i < P; i += blockDim.x) o[(long long)i * P + i] -= tr;
  if (threadIdx.x == 0) {
    const double el = e_in[per_node ? 2 * J : 0], er = e_in[per_node ? 2 * J + 1 : 0];
    e_out[J] = el + er + tr;
  }
}

template <typename T>
__global__ void add_identity_kernel(T* Z, const T* W, long long elems, const double* e_in,
                                    int per_node, double coef) {
  pdl_wait();
  pdl_trigger();
  const int J = blockIdx.y;
  const double c = coef * (e_in[per_node ? 2 * J : 0] + e_in[per_node ? 2 * J + 1 : 0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < elems;
       i += (long long)gridDim.x * blockDim.x)
    Z[J * elems + i] += static_cast<T>(c) * W[J * elems + i];
}

// out = 2 (w + (e_0 + e_1) v): gradient of <v, H_top v> with the identity part
__global__ void top_grad_kernel(double* out, const double* w, const double* v, long long n,
                                const double* e, int per_node) {
  pdl_wait();
  pdl_trigger();
  const double sh = e[0] + e[per_node ? 1 : 0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = 2.0 * (w[i] + sh * v[i]);
}

__global__ void scale_normalise_kernel(const double* x, double* y, long long n, const double* nrm2,
                                       double sign) {
  pdl_wait();
  pdl_trigger();
  const double f = sign / sqrt(nrm2[0]);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    y[i] = f * x[i];
}

__global__ void top_energy_kernel(const double* dot, const double* vv, const double* e,
                                  int per_node, double add, double* out) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x == 0 && blockIdx.x == 0)
    *out = dot[0] + (e[0] + e[per_node ? 1 : 0]) * vv[0] + add;
}

__global__ void to_f32_kernel(const double* src, float* dst, long long n) {
  pdl_wait();
  pdl_trigger();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = f64b::to_f32(src[i]);
}

// Energy change per spin of the last sweep (the convergence test of Sec. IV):
// dstat[0] = energy of the previous sweep, dstat[1] = change per spin,
// dstat[2] = tolerance; istat[2] = 1 when |change| < tolerance and a previous
// energy exists, istat[3] = sweeps seen since the last reset.
__global__ void sweep_delta_kernel(const double* E, double* dstat, int* istat, double inv_spins) {
  pdl_wait();
  pdl_trigger();
  const double e = *E;
  const int seen = istat[3];
  const double d = (e - dstat[0]) * inv_spins;
  dstat[1] = seen > 0 ? d : __longlong_as_double(0x7FF8000000000000LL);
  istat[2] = (seen > 0 && fabs(d) < dstat[2]) ? 1 : 0;
  dstat[0] = e;
  istat[3] = seen + 1;
}

// flag[0] |= 1 when max |A - I| of the P x P matrix A exceeds thr (one CTA).
// For a P x P matrix A: the FP32 pair (ph, pl) of a I - c A (with a = 0,
// c = -1: of A itself), and, with flag, flag |= 1 when max |A - I| > thr
// (NaN counts as far).  Grid-stride over the elements, a warp vote per pass.
__global__ void check_split_kernel(const double* A, int P, double a, double c, float* ph, float* pl,
                                   double thr, int* flag, float* d32) {
  pdl_wait();
  pdl_trigger();
  const long long PP = (long long)P * P;
  int far = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < PP;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / P), j = (int)(e % P);
    const double x = A[e];
    if (flag && !(fabs(x - (i == j ? 1.0 : 0.0)) <= thr)) far = 1;
    const double v = c == -1.0 && a == 0.0 ? x : (i == j ? a : 0.0) - c * x;
    f64b::split(v, ph[e], pl[e]);
    if (d32) d32[e] = f64b::to_f32(0.5 * ((i == j ? 1.0 : 0.0) - x));
  }
  if (flag && __any_sync(0xffffffffu, far) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void store_ints_kernel(int* dst, const int* src, int n, int value) {
  pdl_wait();
  pdl_trigger();
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src ? src[i] : value;
}

// Statistics of nb n x n blocks (block b at M + b*stride), one CTA, fixed
// order: out[0] = sum of the traces, out[1] = max |M - I| (sub_identity) or
// max |M| , out[2] = max |M_ij - M_ji|.
__global__ void mat_stats_kernel(const double* M, int n, int nb, long long stride,
                                 int sub_identity, double* out) {
  pdl_wait();
  pdl_trigger();
  __shared__ double st[256], sd[256], sa[256];
  double tr = 0.0, dev = 0.0, asym = 0.0;
  const long long nn = (long long)n * n;
  for (int b = 0; b < nb; ++b) {
    const double* Mb = M + b * stride;
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
      const int i = (int)(e / n), j = (int)(e % n);
      const double x = Mb[e];
      if (i == j) tr += x;
      dev = fmax(dev, fabs(x - ((sub_identity && i == j) ? 1.0 : 0.0)));
      asym = fmax(asym, fabs(x - Mb[(long long)j * n + i]));
    }
  }
  st[threadIdx.x] = tr;
  sd[threadIdx.x] = dev;
  sa[threadIdx.x] = asym;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      st[threadIdx.x] += st[threadIdx.x + k];
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + k]);
      sa[threadIdx.x] = fmax(sa[threadIdx.x], sa[threadIdx.x + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = st[0]; out[1] = sd[0]; out[2] = sa[0]; }
}

int grid_for(long long n, int per = 256, int cap = 1184) {
  long long g = (n + per - 1) / per;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

}  // namespace

int batched_dot(const double* x, const double* y, long long n, long long stride, int nb,
                double* out, double* scratch, cudaStream_t s) {
  launch_k(dot_partial_kernel, dim3(kDotBlocks, nb), 256, 0, s, x, y, n, stride, scratch, nullptr);
  launch_k(dot_final_kernel, (nb + 3) / 4, 128, 0, s, scratch, nb, out, nullptr);
  return 2;
}

int dot_self_and_cross_partial(const double* x, const double* y, long long n, long long stride,
                               int nb, double* scratch, cudaStream_t s) {
  launch_k(dot2_partial_kernel, dim3(kDotBlocks, nb), 256, 0, s, x, y, n, stride, nb, scratch);
  return 1;
}

int polar_start(const double* G, const double* W, double* X, long long elems, int nb, int P,
                double mu, const double* part, cudaStream_t s, float* xh, float* xl, int* zero,
                const int* try_first, int* run_full, int* zero2) {
  if (nb != 1) xh = xl = nullptr;
  if (!try_first) run_full = nullptr;
  launch_k(polar_start_kernel, dim3(grid_for(elems, 256, 512), nb), 256, 0, s, G, W, X, elems, P,
           mu, part, nb, xh, xl, zero, try_first, run_full, zero2);
  return 1;
}

int check_split(const double* A, int P, double a, double c, float* ph, float* pl, double thr,
                int* flag, cudaStream_t s, float* d32) {
  launch_k(check_split_kernel, grid_for((long long)P * P, 256, 64), 256, 0, s, A, P, a, c, ph, pl,
           thr, flag, d32);
  return 1;
}

int poly_step_matrix(const double* A, double* Pm, int P, int nb, double a, double c,
                     cudaStream_t s) {
  launch_k(poly_step_kernel, dim3(grid_for((long long)P * P, 256, 64), nb), 256, 0, s, A, Pm, P, a, c);
  return 1;
}

int set_identity(double* F, int P, int nb, cudaStream_t s) {
  launch_k(identity_kernel, dim3(grid_for((long long)P * P, 256, 64), nb), 256, 0, s, F, P);
  return 1;
}

int axpby(const double* x, double* y, long long n, double alpha, double beta, cudaStream_t s) {
  launch_k(axpby_kernel, grid_for(n), 256, 0, s, x, y, n, alpha, beta);
  return 1;
}

int scale_select(const double* x0, const double* x1, const int* sel, double* y, long long n,
                 double alpha, cudaStream_t s, float* y32, const float* corr, int* pred,
                 int pstride, int retry, const double* x2, const int* sel2) {
  launch_k(scale_select_kernel, grid_for(n), 256, 0, s, x0, x1, sel, y, n, alpha, y32, corr, pred,
           pstride, retry, x2, sel2);
  return 1;
}

int symmetrize(double* A, int P, int nb, cudaStream_t s) {
  launch_k(symmetrize_kernel, dim3(grid_for((long long)P * P, 256, 64), nb), 256, 0, s, A, P);
  return 1;
}

int lz_dots(const double* basis, long long n, int count, const double* w, double* coef,
            double* scratch, const int* skip, cudaStream_t s) {
  launch_k(lz_dots_partial, dim3(kDotBlocks, count), 256, 0, s, basis, n, count, w, scratch, skip);
  launch_k(lz_dots_final, 1, 128, 0, s, scratch, count, coef, skip);
  return 2;
}

int lz_sub(const double* basis, long long n, int count, double* w, const double* coef,
           const int* skip, cudaStream_t s) {
  launch_k(lz_sub_kernel, grid_for(n), 256, 0, s, basis, n, count, w, coef, skip);
  return 1;
}

int lz_finish_step(double* basis, long long n, int j, double* w, const double* c1,
                   const double* c2, double* alpha, double* beta, double* scratch, double* nrm2,
                   int* skip, int* tdim, cudaStream_t s) {
  launch_k(dot_partial_kernel, dim3(kDotBlocks, 1), 256, 0, s, w, w, n, 0, scratch, skip);
  launch_k(dot_final_kernel, 1, 32, 0, s, scratch, 1, nrm2, skip);
  launch_k(lz_step_scalars, 1, 1, 0, s, c1, c2, j, alpha, beta, nrm2, skip, tdim);
  launch_k(lz_scale_into, grid_for(n), 256, 0, s, basis + (j + 1) * n, w, n, beta, j, skip);
  return 4;
}

int lz_ritz(const double* alpha, const double* beta, const int* tdim, int jmax, double* y,
            double* theta, double* res, int* conv, double tol, cudaStream_t s) {
  launch_k(lz_ritz_kernel, 1, 32, 0, s, alpha, beta, tdim, jmax, y, theta, res, conv, tol, nullptr);
  return 1;
}

int lz_combine(double* basis, long long n, const int* tdim, const double* y, double* v,
               double* scratch, double* nrm2, int* tdim_rw, int* skip, const int* conv,
               cudaStream_t s) {
  launch_k(lz_combine_kernel, grid_for(n), 256, 0, s, basis, n, tdim, y, v);
  launch_k(dot_partial_kernel, dim3(kDotBlocks, 1), 256, 0, s, v, v, n, 0, scratch, nullptr);
  launch_k(dot_final_kernel, 1, 32, 0, s, scratch, 1, nrm2, nullptr);
  launch_k(scale_by_inv_sqrt, grid_for(n), 256, 0, s, v, n, nrm2, basis);
  launch_k(lz_reset_kernel, 1, 1, 0, s, tdim_rw, skip, conv);
  return 5;
}

int lz_start(double* basis, long long n, const double* v, double* scratch, double* nrm2,
             int* tdim, int* skip, int* conv, cudaStream_t s) {
  cudaMemsetAsync(conv, 0, sizeof(int), s);
  launch_k(dot_partial_kernel, dim3(kDotBlocks, 1), 256, 0, s, v, v, n, 0, scratch, nullptr);
  launch_k(dot_final_kernel, 1, 32, 0, s, scratch, 1, nrm2, nullptr);
  cudaMemcpyAsync(basis, v, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
  launch_k(scale_by_inv_sqrt, grid_for(n), 256, 0, s, basis, n, nrm2, nullptr);
  launch_k(lz_reset_kernel, 1, 1, 0, s, tdim, skip, conv);
  return 4;
}

int align_sign(double* v, const double* vprev, long long n, double* scratch, double* dotv,
               cudaStream_t s) {
  launch_k(dot_partial_kernel, dim3(kDotBlocks, 1), 256, 0, s, v, vprev, n, 0, scratch, nullptr);
  launch_k(dot_final_kernel, 1, 32, 0, s, scratch, 1, dotv, nullptr);
  launch_k(flip_if_negative, grid_for(n), 256, 0, s, v, n, dotv);
  return 3;
}

int ordered_sum(const double* x, int count, double* out, double scale, double add,
                cudaStream_t s) {
  launch_k(ordered_sum_kernel, 1, 32, 0, s, x, count, out, scale, add);
  return 1;
}

int split_identity(double* O, long long stride, int P, int nodes, const double* e_in,
                   int per_node, double* e_out, cudaStream_t s) {
  launch_k(split_identity_kernel, nodes, 256, 0, s, O, stride, P, e_in, per_node, e_out);
  return 1;
}

int add_identity_part(void* Z, const void* W, int f32, long long elems, int nodes,
                      const double* e_in, int per_node, double coef, cudaStream_t s) {
  const dim3 grid(grid_for(elems, 256, 512), nodes);
  if (f32)
    launch_k(add_identity_kernel<float>, grid, 256, 0, s, static_cast<float*>(Z),
                                                    static_cast<const float*>(W), elems, e_in,
                                                    per_node, coef);
  else
    launch_k(add_identity_kernel<double>, grid, 256, 0, s, static_cast<double*>(Z),
                                                     static_cast<const double*>(W), elems, e_in,
                                                     per_node, coef);
  return 1;
}

int scale_normalise(const double* x, double* y, long long n, const double* nrm2, double sign,
                    cudaStream_t s) {
  launch_k(scale_normalise_kernel, grid_for(n), 256, 0, s, x, y, n, nrm2, sign);
  return 1;
}

int top_grad(double* out, const double* w, const double* v, long long n, const double* e,
             int per_node, cudaStream_t s) {
  launch_k(top_grad_kernel, grid_for(n), 256, 0, s, out, w, v, n, e, per_node);
  return 1;
}

int top_energy_sum(const double* dot, const double* vv, const double* e, int per_node, double add,
                   double* out, cudaStream_t s) {
  launch_k(top_energy_kernel, 1, 32, 0, s, dot, vv, e, per_node, add, out);
  return 1;
}

int to_f32(const double* src, float* dst, long long n, cudaStream_t s) {
  launch_k(to_f32_kernel, grid_for(n), 256, 0, s, src, dst, n);
  return 1;
}

int sweep_delta(const double* E, double* dstat, int* istat, double inv_spins, cudaStream_t s) {
  launch_k(sweep_delta_kernel, 1, 1, 0, s, E, dstat, istat, inv_spins);
  return 1;
}

int store_ints(int* dst, const int* src, int n, int value, cudaStream_t s) {
  launch_k(store_ints_kernel, 1, 32, 0, s, dst, src, n, value);
  return 1;
}

int mat_stats(const double* M, int n, int nb, long long stride, int sub_identity, double* out,
              cudaStream_t s) {
  launch_k(mat_stats_kernel, 1, 256, 0, s, M, n, nb, stride, sub_identity, out);
  return 1;
}

int finite_check(const double* x, long long n, int* flag, cudaStream_t s) {
  launch_k(finite_kernel, grid_for(n, 256, 296), 256, 0, s, x, n, flag);
  return 1;
}

}  // namespace ttn
