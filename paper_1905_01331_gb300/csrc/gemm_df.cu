// Double-float products for the polar factor of the mixed modes.
//
// Each Newton-Schulz block of the polar factor (Sec. III.B update, computed as
// in the polar.cu header) needs a Gram matrix X X^T and a product F X whose
// rounding is amplified by the block's growth (up to ~1e5): the tensor cores'
// FP32 accumulation is far too coarse for them, FP64 is exact enough but runs
// at two FMA per SM per clock on this GPU.  Here each FP64 operand is held as
// an unevaluated sum of two FP32 numbers, x = hi + lo (|lo| <= 2^-24 |hi|), and
// the products accumulate in pairs of FP32 numbers on the FP32 pipes:
//     p = a_hi b_hi exactly (p + fma(a_hi, b_hi, -p)),  cross terms a_hi b_lo +
//     a_lo b_hi rounded to FP32, a_lo b_lo dropped, error-free two-sum of the
//     running high part, renormalisation once per K tile,
// about 12 FP32 instructions per multiply-add: ~48 significant bits, five
// times the FP64 rate.  A final Newton-Schulz step in the same arithmetic
// brings the isometry defect to ~1e-14.
#include <algorithm>

#include "common.h"
#include "pair_arith.cuh"

namespace ttn {

namespace {

constexpr int kDThreads = 256;
constexpr int kDBK = 16;

// x -> (hi, lo) with hi = fl32(x), lo = fl32(x - hi)
__global__ void split_f64_kernel(const double* x, float* hi, float* lo, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    split_d(x[i], hi[i], lo[i]);
}

// C (FP64) = A B for A: M x K rows (K contiguous), B either K-major (element
// (k, n) at B[n * ldb + k], the Gram case B = A^T) or N-major (B[k * ldb + n]).
// Output tile BM x BN per CTA, TM x TN per thread; blockIdx.z is the K split,
// writing to part[z][M][N] when splits > 1.  sym: only tiles on or above the
// diagonal, counted row by row in blockIdx.x.
template <int BM, int BN, bool kBKmajor>
__global__ void __launch_bounds__(kDThreads) gemm_df_kernel(
    const float* __restrict__ Ah, const float* __restrict__ Al, long long lda,
    const float* __restrict__ Bh, const float* __restrict__ Bl, long long ldb, int M, int N, int K,
    double* C, long long ldc, double* part, int splits, int sym) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ float sAh[kDBK][BM + 4], sAl[kDBK][BM + 4], sBh[kDBK][BN + 4], sBl[kDBK][BN + 4];
  const int tiles_n = (N + BN - 1) / BN;
  int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  if (sym) {
    int u = blockIdx.x, row = tiles_n;
    tm = 0;
    while (u >= row) { u -= row; ++tm; --row; }
    tn = tm + u;
  }
  const int m0 = tm * BM, n0 = tn * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int nkt = (K + kDBK - 1) / kDBK;
  const int kt_lo = (int)((long long)nkt * blockIdx.z / splits);
  const int kt_hi = (int)((long long)nkt * (blockIdx.z + 1) / splits);

  float sh[TM][TN], sl[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }

  for (int kt = kt_lo; kt < kt_hi; ++kt) {
    const int kb = kt * kDBK;
    for (int e = threadIdx.x; e < BM * kDBK; e += kDThreads) {
      const int mi = e / kDBK, ki = e % kDBK;
      const int m = m0 + mi, k = kb + ki;
      const bool ok = m < M && k < K;
      sAh[ki][mi] = ok ? Ah[m * lda + k] : 0.f;
      sAl[ki][mi] = ok ? Al[m * lda + k] : 0.f;
    }
    for (int e = threadIdx.x; e < BN * kDBK; e += kDThreads) {
      int ni, ki;
      if (kBKmajor) { ni = e / kDBK; ki = e % kDBK; } else { ki = e / BN; ni = e % BN; }
      const int nn = n0 + ni, k = kb + ki;
      const bool ok = nn < N && k < K;
      const long long off = kBKmajor ? (long long)nn * ldb + k : (long long)k * ldb + nn;
      sBh[ki][ni] = ok ? Bh[off] : 0.f;
      sBl[ki][ni] = ok ? Bl[off] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kDBK; ++kk) {
      float ah[TM], al[TM], bh[TN], bl[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) { ah[i] = sAh[kk][ty * TM + i]; al[i] = sAl[kk][ty * TM + i]; }
#pragma unroll
      for (int j = 0; j < TN; ++j) { bh[j] = sBh[kk][tx * TN + j]; bl[j] = sBl[kk][tx * TN + j]; }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) pair_mac(ah[i], al[i], bh[j], bl[j], sh[i][j], sl[i][j]);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) pair_renorm(sh[i][j], sl[i][j]);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int m = m0 + ty * TM + i, nn = n0 + tx * TN + j;
      if (m >= M || nn >= N) continue;
      const double v = (double)sh[i][j] + (double)sl[i][j];
      if (splits > 1) {
        part[((long long)blockIdx.z * M + m) * N + nn] = v;
      } else {
        C[m * ldc + nn] = v;
        if (sym && tm < tn) C[nn * ldc + m] = v;
      }
    }
}

// C[m][n] = sum_s part[s][m][n] in split order; for a symmetric product the
// tiles below the diagonal were not computed and are read from the mirror.
__global__ void df_reduce_kernel(const double* part, int splits, int M, int N, int tile, int sym,
                                 double* C, long long ldc) {
  const long long MN = (long long)M * N;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < MN;
       e += (long long)gridDim.x * blockDim.x) {
    const int m = (int)(e / N), n = (int)(e % N);
    const long long src = (sym && m / tile > n / tile) ? (long long)n * N + m : e;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[sp * MN + src];
    C[m * ldc + n] = s;
  }
}

int grid_n(long long n) { return (int)std::min<long long>((n + 255) / 256, 2048); }

}  // namespace

int df_split(const double* x, float* hi, float* lo, long long n, cudaStream_t s) {
  split_f64_kernel<<<grid_n(n), 256, 0, s>>>(x, hi, lo, n);
  return 1;
}

int df_gram_splits(int P, int n2) {
  const int nt = (P + 31) / 32, tiles = nt * (nt + 1) / 2;
  const int kt = (n2 + kDBK - 1) / kDBK;
  const int want = (296 + tiles - 1) / tiles;
  return std::max(1, std::min(std::min(want, kt / 2), 64));
}

int df_gram(const float* Xh, const float* Xl, int P, long long n2, double* C, double* part,
            cudaStream_t s) {
  const int splits = df_gram_splits(P, (int)n2);
  const int nt = (P + 31) / 32;
  dim3 grid(nt * (nt + 1) / 2, 1, splits);
  gemm_df_kernel<32, 32, true><<<grid, kDThreads, 0, s>>>(Xh, Xl, n2, Xh, Xl, n2, P, P, (int)n2,
                                                         C, P, part, splits, 1);
  int launches = 1;
  if (splits > 1) {
    df_reduce_kernel<<<grid_n((long long)P * P), 256, 0, s>>>(part, splits, P, P, 32, 1, C, P);
    ++launches;
  }
  return launches;
}

int df_apply(const float* Fh, const float* Fl, const float* Xh, const float* Xl, int P,
             long long n2, double* C, cudaStream_t s) {
  const int tn = (int)((n2 + 63) / 64), tm = (P + 63) / 64;
  dim3 grid(tm * tn, 1, 1);
  gemm_df_kernel<64, 64, false><<<grid, kDThreads, 0, s>>>(Fh, Fl, P, Xh, Xl, n2, P, (int)n2, P,
                                                          C, n2, nullptr, 1, 0);
  return 1;
}

}  // namespace ttn
