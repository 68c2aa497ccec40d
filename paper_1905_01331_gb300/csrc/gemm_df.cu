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
// about 12 FP32 instructions per multiply-add: ~48 significant bits at about
// four times the FP64 rate here (2.1 against 0.55 T multiply-adds/s).  A final
// Newton-Schulz step in the same arithmetic brings the isometry defect to
// ~1e-14.
#include <algorithm>

#include "common.h"
#include "f64_bits.cuh"
#include "pair_arith.cuh"

namespace ttn {

namespace {

constexpr int kDBK = 16;

// x -> (hi, lo) with hi = fl32(x), lo = fl32(x - hi)
__global__ void split_f64_kernel(const double* x, float* hi, float* lo, long long n) {
  pdl_wait();
  pdl_trigger();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    split_d(x[i], hi[i], lo[i]);
}

// TM consecutive floats of shared memory into registers (vector loads; the
// row pitch of every staged tile is a multiple of four floats).
template <int TM>
__device__ __forceinline__ void lds_frag(const float* p, float (&r)[TM]) {
  if constexpr (TM % 4 == 0) {
#pragma unroll
    for (int i = 0; i < TM; i += 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + i);
      r[i] = v.x; r[i + 1] = v.y; r[i + 2] = v.z; r[i + 3] = v.w;
    }
  } else if constexpr (TM % 2 == 0) {
#pragma unroll
    for (int i = 0; i < TM; i += 2) {
      const float2 v = *reinterpret_cast<const float2*>(p + i);
      r[i] = v.x; r[i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < TM; ++i) r[i] = p[i];
  }
}

// C (FP64) = A B for A: M x K rows (K contiguous), B either K-major (element
// (k, n) at B[n * ldb + k], the Gram case B = A^T) or N-major (B[k * ldb + n]).
// Output tile BM x BN per CTA of (BM / TM) x (BN / TN) threads, TM x TN per
// thread; blockIdx.z is the K split, writing to part[z][M][N] when splits > 1.
// sym: only tiles on or above the diagonal, counted row by row in blockIdx.x.
// Two shared-memory stages: the next K tile is loaded into registers while the
// current one is multiplied, one barrier per K tile.  MB: CTAs per SM the
// register allocation must allow.
template <int BM, int BN, int TM, int TN, bool kBKmajor, int MB>
__global__ void __launch_bounds__((BM / TM) * (BN / TN), MB) gemm_df_kernel(
    const float* __restrict__ Ah, const float* __restrict__ Al, long long lda,
    const float* __restrict__ Bh, const float* __restrict__ Bl, long long ldb, int M, int N, int K,
    double* C, long long ldc, double* part, int splits, int sym, const int* run_if, float* Ch,
    float* Cl) {
  pdl_wait();
  pdl_trigger();
  if (run_if && *run_if == 0) return;
  constexpr int TX = BN / TN, NT = (BM / TM) * TX;
  constexpr int LA = BM * kDBK / NT, LB = BN * kDBK / NT;
  static_assert(BM * kDBK % NT == 0 && BN * kDBK % NT == 0, "staging split");
  static_assert((BM + 4) % 4 == 0 && (BN + 4) % 4 == 0, "row pitch");
  __shared__ __align__(16) float sAh[2][kDBK][BM + 4], sAl[2][kDBK][BM + 4];
  __shared__ __align__(16) float sBh[2][kDBK][BN + 4], sBl[2][kDBK][BN + 4];
  const int tiles_n = (N + BN - 1) / BN;
  int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  if (sym) {
    int u = blockIdx.x, row = tiles_n;
    tm = 0;
    while (u >= row) { u -= row; ++tm; --row; }
    tn = tm + u;
  }
  const int m0 = tm * BM, n0 = tn * BN;
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int nkt = (K + kDBK - 1) / kDBK;
  const int kt_lo = (int)((long long)nkt * blockIdx.z / splits);
  const int kt_hi = (int)((long long)nkt * (blockIdx.z + 1) / splits);

  float rAh[LA], rAl[LA], rBh[LB], rBl[LB];
  auto load = [&](int kt) {
    const int kb = kt * kDBK;
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const int e = threadIdx.x + i * NT;
      const int m = m0 + e / kDBK, k = kb + e % kDBK;
      const bool ok = m < M && k < K;
      rAh[i] = ok ? Ah[m * lda + k] : 0.f;
      rAl[i] = ok ? Al[m * lda + k] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      const int e = threadIdx.x + i * NT;
      int ni, ki;
      if (kBKmajor) { ni = e / kDBK; ki = e % kDBK; } else { ki = e / BN; ni = e % BN; }
      const int nn = n0 + ni, k = kb + ki;
      const bool ok = nn < N && k < K;
      const long long off = kBKmajor ? (long long)nn * ldb + k : (long long)k * ldb + nn;
      rBh[i] = ok ? Bh[off] : 0.f;
      rBl[i] = ok ? Bl[off] : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int i = 0; i < LA; ++i) {
      const int e = threadIdx.x + i * NT;
      sAh[buf][e % kDBK][e / kDBK] = rAh[i];
      sAl[buf][e % kDBK][e / kDBK] = rAl[i];
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      const int e = threadIdx.x + i * NT;
      int ni, ki;
      if (kBKmajor) { ni = e / kDBK; ki = e % kDBK; } else { ki = e / BN; ni = e % BN; }
      sBh[buf][ki][ni] = rBh[i];
      sBl[buf][ki][ni] = rBl[i];
    }
  };

  float sh[TM][TN], sl[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) { sh[i][j] = 0.f; sl[i][j] = 0.f; }

  if (kt_lo < kt_hi) {
    load(kt_lo);
    store(0);
  }
  __syncthreads();
  for (int kt = kt_lo; kt < kt_hi; ++kt) {
    const int buf = (kt - kt_lo) & 1;
    const bool more = kt + 1 < kt_hi;
    if (more) load(kt + 1);
#pragma unroll 4
    for (int kk = 0; kk < kDBK; ++kk) {
      float ah[TM], al[TM], bh[TN], bl[TN];
      lds_frag<TM>(&sAh[buf][kk][ty * TM], ah);
      lds_frag<TM>(&sAl[buf][kk][ty * TM], al);
      lds_frag<TN>(&sBh[buf][kk][tx * TN], bh);
      lds_frag<TN>(&sBl[buf][kk][tx * TN], bl);
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) pair_mac(ah[i], al[i], bh[j], bl[j], sh[i][j], sl[i][j]);
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) pair_renorm(sh[i][j], sl[i][j]);
    if (more) store(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int m = m0 + ty * TM + i, nn = n0 + tx * TN + j;
      if (m >= M || nn >= N) continue;
      // FP32 -> FP64 by integer operations (f64_bits.cuh): the two converting
      // instructions per element would run on the two FP64 units per SM
      const double v = f64b::from_f32(sh[i][j]) + f64b::from_f32(sl[i][j]);
      if (splits > 1) {
        part[((long long)blockIdx.z * M + m) * N + nn] = v;
      } else {
        C[m * ldc + nn] = v;
        if (sym && tm < tn) C[nn * ldc + m] = v;
        // the pair is normalised (renormalised after the last K tile), so it
        // is the FP32 split of v
        if (Ch) {
          Ch[m * ldc + nn] = sh[i][j];
          Cl[m * ldc + nn] = sl[i][j];
        }
      }
    }
}

// C[m][n] = sum_s part[s][m][n]; for a symmetric product the tiles below the
// diagonal were not computed and are read from the mirror.  A CTA owns 32
// consecutive outputs; its 8 warps each sum a contiguous eighth of the splits
// in order (loads in flight together), warp 0 adds the eight sums in group
// order (a fixed order of terms).
__global__ void df_reduce_kernel(const double* part, int splits, int M, int N, int tile, int sym,
                                 double* C, long long ldc, const int* run_if, GramCheck chk) {
  pdl_wait();
  pdl_trigger();
  if (run_if && *run_if == 0) return;
  __shared__ double gs[8][32];
  const long long MN = (long long)M * N;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int s_lo = (int)((long long)splits * g / 8), s_hi = (int)((long long)splits * (g + 1) / 8);
  for (long long e0 = blockIdx.x * 32LL; e0 < MN; e0 += gridDim.x * 32LL) {
    const long long e = e0 + lane;
    double acc = 0.0;
    int m = 0, n = 0;
    if (e < MN) {
      m = (int)(e / N);
      n = (int)(e % N);
      const long long src = (sym && m / tile > n / tile) ? (long long)n * N + m : e;
      for (int sp0 = s_lo; sp0 < s_hi; sp0 += 8) {
        double xs[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) xs[q] = sp0 + q < s_hi ? part[(sp0 + q) * MN + src] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += xs[q];
      }
    }
    gs[g][lane] = acc;
    __syncthreads();
    int far = 0, far2 = 0;
    if (g == 0 && e < MN) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += gs[q][lane];
      C[m * ldc + n] = t;
      if (chk.ph) {
        // the check_split pass (square C, element e = m N + n)
        const double id = m == n ? 1.0 : 0.0;
        if (chk.flag && !(fabs(t - id) <= chk.thr)) far = 1;
        if (chk.flag2 && !(fabs(t - id) <= chk.thr2)) far2 = 1;
        const double v = chk.c == -1.0 && chk.a == 0.0 ? t : (m == n ? chk.a : 0.0) - chk.c * t;
        f64b::split(v, chk.ph[e], chk.pl[e]);
        if (chk.d32) chk.d32[e] = f64b::to_f32(0.5 * (id - t));
      }
    }
    if (g == 0 && chk.flag && __any_sync(0xffffffffu, far) && lane == 0) atomicOr(chk.flag, 1);
    if (g == 0 && chk.flag2 && __any_sync(0xffffffffu, far2) && lane == 0) atomicOr(chk.flag2, 1);
    __syncthreads();
  }
}

int grid_n(long long n) { return (int)std::min<long long>((n + 255) / 256, 2048); }

// Gram tiles of GB x GB (GT x GT per thread), the K range cut so that about
// `target` CTAs run.
int gram_splits(int P, int n2, int GB, int target) {
  const int nt = (P + GB - 1) / GB, tiles = nt * (nt + 1) / 2;
  const int kt = (n2 + kDBK - 1) / kDBK;
  const int want = (target + tiles - 1) / tiles;
  return std::max(1, std::min(std::min(want, kt / 2), 128));
}

template <int GB, int GT, int MB>
int gram_launch(const float* Xh, const float* Xl, int P, long long n2, double* C, double* part,
                int splits, cudaStream_t s, const int* run_if, const GramCheck* chk) {
  const int nt = (P + GB - 1) / GB;
  dim3 grid(nt * (nt + 1) / 2, 1, splits);
  launch_k(gemm_df_kernel<GB, GB, GT, GT, true, MB>, grid, (GB / GT) * (GB / GT), 0, s,
      Xh, Xl, n2, Xh, Xl, n2, P, P, (int)n2, C, P, part, splits, 1, run_if, nullptr, nullptr);
  int launches = 1;
  if (splits > 1) {
    launch_k(df_reduce_kernel, (int)std::min<long long>(((long long)P * P + 31) / 32, 8192), 256,
             0, s, part, splits, P, P, GB, 1, C, P, run_if, chk ? *chk : GramCheck());
    ++launches;
  } else if (chk) {
    launches += check_split(C, P, chk->a, chk->c, chk->ph, chk->pl, chk->thr, chk->flag, s,
                            chk->d32);
    if (chk->flag2)
      launches += check_split(C, P, chk->a, chk->c, chk->ph, chk->pl, chk->thr2, chk->flag2, s);
  }
  return launches;
}

template <int BM, int BN, int TM, int TN, int MB>
int apply_launch(const float* Fh, const float* Fl, const float* Xh, const float* Xl, int P,
                 long long n2, double* C, cudaStream_t s, const int* run_if, float* Ch,
                 float* Cl) {
  const int tn = (int)((n2 + BN - 1) / BN), tm = (P + BM - 1) / BM;
  launch_k(gemm_df_kernel<BM, BN, TM, TN, false, MB>, tm * tn, (BM / TM) * (BN / TN), 0, s,
      Fh, Fl, P, Xh, Xl, n2, P, (int)n2, P, C, n2, nullptr, 1, 0, run_if, Ch, Cl);
  return 1;
}

constexpr int kGramB = 32, kGramT = 2, kGramTarget = 296;

}  // namespace

int df_split(const double* x, float* hi, float* lo, long long n, cudaStream_t s) {
  launch_k(split_f64_kernel, grid_n(n), 256, 0, s, x, hi, lo, n);
  return 1;
}

int df_gram_splits(int P, int n2) { return gram_splits(P, n2, kGramB, kGramTarget); }

double df_gram_flops(int P, long long n2) {
  const int nt = (P + kGramB - 1) / kGramB;
  return 2.0 * nt * (nt + 1) / 2 * kGramB * kGramB * (double)n2;
}

int df_gram(const float* Xh, const float* Xl, int P, long long n2, double* C, double* part,
            cudaStream_t s, const int* run_if, const GramCheck* chk) {
  return gram_launch<kGramB, kGramT, 2>(Xh, Xl, P, n2, C, part, df_gram_splits(P, (int)n2), s,
                                        run_if, chk);
}

int df_apply(const float* Fh, const float* Fl, const float* Xh, const float* Xl, int P,
             long long n2, double* C, cudaStream_t s, const int* run_if, float* Ch, float* Cl) {
  return apply_launch<64, 32, 4, 4, 4>(Fh, Fl, Xh, Xl, P, n2, C, s, run_if, Ch, Cl);
}

}  // namespace ttn
