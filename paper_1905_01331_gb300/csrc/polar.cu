// Polar update (Sec. III.B: w = -(polar factor of the environment)): the
// composition of one block of scaled Newton-Schulz steps on the P x P level,
// in one persistent cooperative launch.
//
// A block starts from the Gram matrix A_0 = X X^T.  Step j applies
// p_j(x) = alpha_j x - beta_j x^3 to the singular values of X, which on the
// P x P level reads
//     Pm_j = alpha_j I - beta_j A_j,   F_{j+1} = Pm_j F_j,   A_{j+1} = Pm_j A_j Pm_j,
// (F_0 = I) and the block ends with X <- F X.  Per step
//     phase 1:  F_{j+1} = Pm_j F_j,  T = A_j Pm_j        (F_1 = Pm_0 needs no product)
//     phase 2:  A_{j+1} = Pm_j T
// on full tiles.  A_j is read symmetrised, (A + A^T)/2, and Pm_j is formed from
// it while the operands are staged.  In exact arithmetic every matrix here is
// a polynomial in A_0 and symmetric; in rounding the products are not, and
// keeping only one triangle of them (half the work: the upper tiles computed
// and mirrored) cost up to 20x in the isometry defect of long FP64 blocks and
// ~1000x for a 14-step block in a float64 emulation of the double-float
// kernel (whose long blocks then left the stable interval and diverged), so
// the full products are kept.
//
// The products are small (P <= 256) and FP64, which on this GPU runs at two
// DFMA per clock per SM: a separate launch per product leaves most SMs idle and
// pays the launch gap each time.  Here all SMs share the tiles of each phase
// and meet at a grid barrier (bounded spin, error flag) between phases.
#include <algorithm>
#include <mutex>

#include "common.h"
#include "pair_arith.cuh"

namespace ttn {

namespace {

constexpr int kCT = 8;                       // output tile edge
constexpr int kCThreads = 256;               // 8 warps, one K-slice each
constexpr int kCWarps = kCThreads / 32;
constexpr int kCMaxP = 256;
constexpr int kCMaxSpin = 1 << 21;           // ~1 s of polling, then the error flag

struct ComposeSmem {
  double X[kCT][kCMaxP + 1];                 // rows i0.. of the left factor
  double Y[kCT][kCMaxP + 1];                 // rows j0.. of the (symmetric) right factor
  double red[kCWarps][kCT * kCT];            // per-warp partial sums
  int ok;
};

// Element (r, c) = (tid / 8, tid % 8) of the tile (i0, j0) of X' Y', for
// threads tid < 64 (0 elsewhere): sum_k X'[i0 + r][k] Y'[k][j0 + c] with
//     X' = dx I + sx S_x(X),   Y' = dy I + sy S_y(Y),
// S(M) = (M + M^T)/2 when the flag is set, else M, formed while rows of X and
// columns of Y are staged.  The K range is cut into 8 interleaved slices (one
// per warp) whose partial sums are added in warp order.
__device__ double tile_product(ComposeSmem& sm, const double* X, double dx, double sx, bool symx,
                               const double* Y, double dy, double sy, bool symy, int P, int i0,
                               int j0) {
  for (int e = threadIdx.x; e < kCT * P; e += kCThreads) {
    // rows of X: element (r, k), consecutive threads along k
    {
      const int r = e / P, k = e - (e / P) * P;
      const int gi = i0 + r;
      double v = 0.0;
      if (gi < P) {
        const double x = __ldcg(X + (long long)gi * P + k);
        const double m = symx ? 0.5 * (x + __ldcg(X + (long long)k * P + gi)) : x;
        v = sx * m + (gi == k ? dx : 0.0);
      }
      sm.X[r][k] = v;
    }
    // columns of Y: element (k, c), consecutive threads along c
    {
      const int k = e / kCT, c = e - (e / kCT) * kCT;
      const int gj = j0 + c;
      double v = 0.0;
      if (gj < P) {
        const double y = __ldcg(Y + (long long)k * P + gj);
        const double m = symy ? 0.5 * (y + __ldcg(Y + (long long)gj * P + k)) : y;
        v = sy * m + (gj == k ? dy : 0.0);
      }
      sm.Y[c][k] = v;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  double a0 = 0.0, a1 = 0.0;
  for (int k = warp; k < P; k += kCWarps) {
    const double x = sm.X[i][k];
    a0 = fma(x, sm.Y[j][k], a0);
    a1 = fma(x, sm.Y[j + 1][k], a1);
  }
  sm.red[warp][i * kCT + j] = a0;
  sm.red[warp][i * kCT + j + 1] = a1;
  __syncthreads();
  double v = 0.0;
  if (threadIdx.x < kCT * kCT)
    for (int w = 0; w < kCWarps; ++w) v += sm.red[w][threadIdx.x];
  __syncthreads();
  return v;
}

// Grid-wide barrier of a co-resident grid: arrive on a counter zeroed before
// the launch and poll it, at most max_spin times.  Returns false (and raises
// *err) when the wait expires or another CTA has raised *err.
__device__ bool grid_barrier(ComposeSmem& sm, unsigned* bar, unsigned target, int* err,
                             int max_spin) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // arrive with release semantics, poll with acquire semantics
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int spins = 0;
    while (true) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if (v >= target) break;
      if (*reinterpret_cast<volatile int*>(err)) { ok = 0; break; }
      if (++spins > max_spin) { atomicOr(err, 2); ok = 0; break; }
      __nanosleep(32);
    }
    sm.ok = ok;
  }
  __syncthreads();
  return sm.ok != 0;
}

__device__ __forceinline__ void store_tile(double* C, int P, int ti, int tj, double v) {
  if (threadIdx.x >= kCT * kCT) return;
  const int gi = ti * kCT + threadIdx.x / kCT, gj = tj * kCT + threadIdx.x % kCT;
  if (gi < P && gj < P) __stcg(C + (long long)gi * P + gj, v);
}

__global__ void __launch_bounds__(kCThreads) polar_compose_kernel(const ComposeArgs a) {
  __shared__ ComposeSmem sm;
  const int P = a.P, ns = a.nsteps;
  const int nt = (P + kCT - 1) / kCT, ntt = nt * nt;
  const long long PP = (long long)P * P;
  // F_j lives in F when ns - j is even, else in S, so that F_ns ends in F
  auto Fbuf = [&](int j) { return ((ns - j) & 1) ? a.S : a.F; };
  unsigned target = 0;
  for (int j = 0; j < ns; ++j) {
    const double al = a.alpha[j], be = a.beta[j];
    const bool last = j + 1 == ns;
    const double* Aj = (j & 1) ? a.A1 : a.A0;
    double* An = (j & 1) ? a.A0 : a.A1;
    double* Fn = Fbuf(j + 1);
    // phase 1: F_{j+1} = Pm_j F_j (j > 0) and T = A_j Pm_j (not on the last step)
    const int np = (j > 0 ? 1 : 0) + (last ? 0 : 1);
    const int items1 = np * ntt * a.NJ;
    for (int it = blockIdx.x; it < items1; it += gridDim.x) {
      const int b = it / (np * ntt);
      const int u = it % (np * ntt);
      const bool isF = j > 0 && u < ntt;
      const int ti = (u % ntt) / nt, tj = (u % ntt) % nt;
      const double* Ab = Aj + b * PP;
      const double v = isF
          ? tile_product(sm, Ab, al, -be, true, Fbuf(j) + b * PP, 0.0, 1.0, false, P, ti * kCT,
                         tj * kCT)
          : tile_product(sm, Ab, 0.0, 1.0, true, Ab, al, -be, true, P, ti * kCT, tj * kCT);
      store_tile((isF ? Fn : a.T) + b * PP, P, ti, tj, v);
    }
    if (j == 0) {
      // F_1 = Pm_0, elementwise
      for (long long e = blockIdx.x * (long long)kCThreads + threadIdx.x; e < a.NJ * PP;
           e += (long long)gridDim.x * kCThreads) {
        const long long b = e / PP, r = e % PP, gi = r / P, gj = r % P;
        const double m = 0.5 * (__ldcg(Aj + e) + __ldcg(Aj + b * PP + gj * P + gi));
        __stcg(Fn + e, (gi == gj ? al : 0.0) - be * m);
      }
    }
    if (last) break;
    target += gridDim.x;
    if (!grid_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kCMaxSpin)) return;
    // phase 2: A_{j+1} = Pm_j T
    const int items2 = ntt * a.NJ;
    for (int it = blockIdx.x; it < items2; it += gridDim.x) {
      const int b = it / ntt, ti = (it % ntt) / nt, tj = (it % ntt) % nt;
      const double v = tile_product(sm, Aj + b * PP, al, -be, true, a.T + b * PP, 0.0, 1.0, false,
                                    P, ti * kCT, tj * kCT);
      store_tile(An + b * PP, P, ti, tj, v);
    }
    target += gridDim.x;
    if (!grid_barrier(sm, a.bar, target, a.err, a.max_spin > 0 ? a.max_spin : kCMaxSpin)) return;
  }
}

// ---------------------------------------------------------------------------
// The same composition in double-float arithmetic (mixed modes): every matrix
// is a pair of FP32 arrays (hi at p, lo at p + P*P, block b of NJ at
// p + 2*b*P*P floats), products accumulate in FP32 pairs on the FP32 pipes
// (~48 significant bits; see gemm_df.cu), and Pm_j and the step coefficients
// are applied in pair arithmetic while operands are staged.  A_j is used as
// computed, without the symmetrisation of the FP64 kernel: the step formulas
// keep every matrix of the block a polynomial in A_j whether or not rounding
// keeps it symmetric, the block's error is set by the pairs' 48-bit rounding,
// and the polar factor's final Newton-Schulz step restores the isometry.
// Without the transposed reads the staging takes half as long.  F ends as
// pairs, the operand format of the double-float apply.
//
// Work items and their order.  One item is one 8 x 8 output tile (b, ti, tj):
//   phase 1 of step j:  F_{j+1}(ti, tj) = Pm_j(ti, :) F_j(:, tj)   (F_1 = Pm_0 elementwise)
//                       T(ti, tj)       = A_j(ti, :) Pm_j(:, tj)   (not on the last step)
//   phase 2 of step j:  A_{j+1}(ti, tj) = Pm_j(ti, :) T(:, tj)
// The two phase-1 tiles share the staged rows of A_j, so one item computes
// both.  Instead of a grid barrier between phases, items wait only for the
// tiles they read, through three arrays of counters (one per row or column
// block, shared by the NJ matrices):
//   cT[tj]  phase-1 items of column block tj done,
//   rA[ti]  phase-2 items of row block ti done,   cA[tj]  ... of column block tj.
// A phase-1 item of step j >= 1 waits for rA[ti] and cA[tj] to reach nt NJ j
// (rows ti of A_j: its own rows and those of Pm_j; columns tj of A_j; and,
// through the phase-1 items those phase-2 items waited for, columns tj of F_j
// and every earlier reader of the T and F tiles it overwrites); a phase-2 item
// of step j waits for cT[tj] to reach nt NJ (j + 1) (columns tj of T, and,
// through those items, rows ti of A_j and every reader of the A_{j-1} tile it
// overwrites).  Every CTA finishes its items of one phase before the next
// phase, and items only wait for items of earlier phases, so a co-resident
// grid always progresses; each wait is bounded (error flag, then return).
// ---------------------------------------------------------------------------

constexpr int kDFArrays = 8;   // Rh Rl Ph Pl Uh Ul Vh Vl
static_assert(kCMaxP / kCT <= kComposeMaxTiles, "one counter per row or column block");

// Row stride of the staged arrays: P + 4 rounded so that the stride is 4 mod
// 32 banks (the eight rows or columns of a tile then start in distinct banks
// for the compute reads, and a staging pass of four k by eight columns hits
// 32 distinct banks).
__host__ __device__ __forceinline__ int df_ld(int P) { return P + (36 - P % 32) % 32; }

size_t compose_df_smem(int P) {
  return ((size_t)kDFArrays * kCT * df_ld(P) + 4 * kCWarps * kCT * kCT) * sizeof(float) + 16;
}

struct DFSmem {
  float *Rh, *Rl;   // rows i0.. of A_j as stored
  float *Ph, *Pl;   // the same rows of Pm_j = alpha_j I - beta_j A_j
  float *Uh, *Ul;   // columns j0.. of the first product's right factor (as stored)
  float *Vh, *Vl;   // columns j0.. of Pm_j (the second product's right factor)
  float* red;       // [product][hi, lo][warp][64] partial sums
  int* ok;
};

__device__ __forceinline__ DFSmem df_carve(float* base, int ld) {
  DFSmem s;
  const int a = kCT * ld;
  s.Rh = base; s.Rl = base + a; s.Ph = base + 2 * a; s.Pl = base + 3 * a;
  s.Uh = base + 4 * a; s.Ul = base + 5 * a; s.Vh = base + 6 * a; s.Vl = base + 7 * a;
  s.red = base + kDFArrays * a;
  s.ok = reinterpret_cast<int*>(s.red + 4 * kCWarps * kCT * kCT);
  return s;
}

// dx I + sx M at element (i, k) for the pair (mh, ml) of M there.
__device__ __forceinline__ void xform_elem(float& mh, float& ml, int i, int k, float dxh,
                                           float dxl, float sxh, float sxl) {
  if (sxh != 1.f || sxl != 0.f) pair_mul(mh, ml, sxh, sxl, mh, ml);
  if (i == k && (dxh != 0.f || dxl != 0.f)) pair_add(mh, ml, dxh, dxl, mh, ml);
}

// One work item on tile (i0, j0) of the P x P pair matrices (A, U, V at their
// block's base; the coefficient pairs (dh, dl) = alpha_j, (sh, sl) = -beta_j):
//   stage rows i0.. of A (raw into R when wantR, as Pm into P), columns j0.. of
//   U (raw) when U, and columns j0.. of V as Pm when V -- the loads of one
//   pass issued before any of them is transformed and stored;
//   OU = P-rows x U-columns when U, OV = R-rows x V-columns when V (each K
//   range cut into 8 interleaved slices, one per warp, added in warp order);
//   OE (when given) = the tile of Pm itself (F_1 = Pm_0).
__device__ void df_item(const DFSmem& sm, int P, int ld, const float* A, bool wantR,
                        const float* U, const float* V, float dh, float dl, float sh, float sl,
                        int i0, int j0, float* OU, float* OV, float* OE) {
  constexpr int kBatch = 4;
  const long long PP = (long long)P * P;
  const int total = kCT * P;
  for (int e0 = threadIdx.x; e0 < total; e0 += kBatch * kCThreads) {
    float ah[kBatch], al[kBatch], uh[kBatch], ul[kBatch], vh[kBatch], vl[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * kCThreads;
      ah[u] = al[u] = uh[u] = ul[u] = vh[u] = vl[u] = 0.f;
      if (e < total) {
        // rows: element (r, k); columns: element (k2, c)
        const int r = e / P, k = e - r * P, gi = i0 + r;
        if (gi < P) {
          ah[u] = __ldcg(A + (long long)gi * P + k);
          al[u] = __ldcg(A + PP + (long long)gi * P + k);
        }
        const int k2 = e / kCT, c = e - k2 * kCT, gj = j0 + c;
        if (gj < P) {
          if (U) {
            uh[u] = __ldcg(U + (long long)k2 * P + gj);
            ul[u] = __ldcg(U + PP + (long long)k2 * P + gj);
          }
          if (V) {
            vh[u] = __ldcg(V + (long long)k2 * P + gj);
            vl[u] = __ldcg(V + PP + (long long)k2 * P + gj);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int e = e0 + u * kCThreads;
      if (e < total) {
        const int r = e / P, k = e - r * P, gi = i0 + r;
        if (wantR) {
          sm.Rh[r * ld + k] = ah[u];
          sm.Rl[r * ld + k] = al[u];
        }
        if (gi < P) xform_elem(ah[u], al[u], gi, k, dh, dl, sh, sl);
        sm.Ph[r * ld + k] = ah[u];
        sm.Pl[r * ld + k] = al[u];
        const int k2 = e / kCT, c = e - k2 * kCT, gj = j0 + c;
        if (U) {
          sm.Uh[c * ld + k2] = uh[u];
          sm.Ul[c * ld + k2] = ul[u];
        }
        if (V) {
          if (gj < P) xform_elem(vh[u], vl[u], k2, gj, dh, dl, sh, sl);
          sm.Vh[c * ld + k2] = vh[u];
          sm.Vl[c * ld + k2] = vl[u];
        }
      }
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = lane >> 2, j = (lane & 3) * 2;
  float u0h = 0.f, u0l = 0.f, u1h = 0.f, u1l = 0.f;
  float v0h = 0.f, v0l = 0.f, v1h = 0.f, v1l = 0.f;
  int n = 0;
  for (int k = warp; k < P; k += kCWarps) {
    if (U) {
      const float xh = sm.Ph[i * ld + k], xl = sm.Pl[i * ld + k];
      pair_mac(xh, xl, sm.Uh[j * ld + k], sm.Ul[j * ld + k], u0h, u0l);
      pair_mac(xh, xl, sm.Uh[(j + 1) * ld + k], sm.Ul[(j + 1) * ld + k], u1h, u1l);
    }
    if (V) {
      const float xh = sm.Rh[i * ld + k], xl = sm.Rl[i * ld + k];
      pair_mac(xh, xl, sm.Vh[j * ld + k], sm.Vl[j * ld + k], v0h, v0l);
      pair_mac(xh, xl, sm.Vh[(j + 1) * ld + k], sm.Vl[(j + 1) * ld + k], v1h, v1l);
    }
    if (++n == 8) {
      n = 0;
      pair_renorm(u0h, u0l);
      pair_renorm(u1h, u1l);
      pair_renorm(v0h, v0l);
      pair_renorm(v1h, v1l);
    }
  }
  constexpr int kT2 = kCT * kCT;
  float* redU = sm.red;                       // [hi, lo][warp][64]
  float* redV = sm.red + 2 * kCWarps * kT2;
  const int o = i * kCT + j;
  redU[warp * kT2 + o] = u0h;
  redU[(kCWarps + warp) * kT2 + o] = u0l;
  redU[warp * kT2 + o + 1] = u1h;
  redU[(kCWarps + warp) * kT2 + o + 1] = u1l;
  redV[warp * kT2 + o] = v0h;
  redV[(kCWarps + warp) * kT2 + o] = v0l;
  redV[warp * kT2 + o + 1] = v1h;
  redV[(kCWarps + warp) * kT2 + o + 1] = v1l;
  __syncthreads();
  // threads 0..63 finish the first product's tile, 64..127 the second's,
  // 128..191 copy the tile of Pm
  const int t = threadIdx.x, q = t / kT2, e = t % kT2;
  const int gi = i0 + e / kCT, gj = j0 + e % kCT;
  if (q < 2 && gi < P && gj < P) {
    float* out = q == 0 ? OU : OV;
    if (out) {
      const float* red = q == 0 ? redU : redV;
      float rh = 0.f, rl = 0.f;
      for (int w = 0; w < kCWarps; ++w)
        pair_add(rh, rl, red[w * kT2 + e], red[(kCWarps + w) * kT2 + e], rh, rl);
      __stcg(out + (long long)gi * P + gj, rh);
      __stcg(out + PP + (long long)gi * P + gj, rl);
    }
  } else if (q == 2 && OE && gi < P && gj < P) {
    __stcg(OE + (long long)gi * P + gj, sm.Ph[(e / kCT) * ld + gj]);
    __stcg(OE + PP + (long long)gi * P + gj, sm.Pl[(e / kCT) * ld + gj]);
  }
}

// Wait until *c0 >= t0 and (c1 null or) *c1 >= t1: thread 0 polls with
// acquire loads, at most max_spin times; the CTA then continues.  Returns false
// (and raises *err) when the wait expires or another CTA has raised *err.
__device__ bool df_wait(const DFSmem& sm, const unsigned* c0, unsigned t0, const unsigned* c1,
                        unsigned t1, int* err, int max_spin) {
  if (threadIdx.x == 0) {
    int ok = 1, spins = 0;
    while (true) {
      unsigned v0, v1 = t1;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v0) : "l"(c0) : "memory");
      if (c1) asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v1) : "l"(c1) : "memory");
      if (v0 >= t0 && v1 >= t1) break;
      if (*reinterpret_cast<volatile int*>(err)) { ok = 0; break; }
      if (++spins > max_spin) { atomicOr(err, 2); ok = 0; break; }
      __nanosleep(32);
    }
    *sm.ok = ok;
  }
  __syncthreads();
  return *sm.ok != 0;
}

// The CTA's tile is stored: count it (release, after every thread's stores).
__device__ __forceinline__ void df_signal(unsigned* c0, unsigned* c1) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c0) : "memory");
    if (c1) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c1) : "memory");
  }
}

__global__ void __launch_bounds__(kCThreads) polar_compose_df_kernel(const ComposeArgs a) {
  extern __shared__ __align__(16) float df_dyn[];
  const int P = a.P, ns = a.nsteps, NJ = a.NJ;
  const int nt = (P + kCT - 1) / kCT, ntt = nt * nt, items = ntt * NJ;
  const int ld = df_ld(P);
  const DFSmem sm = df_carve(df_dyn, ld);
  const long long P2 = 2LL * P * P;               // floats per pair matrix
  float* A0 = reinterpret_cast<float*>(a.A0);
  float* A1 = reinterpret_cast<float*>(a.A1);
  float* F = reinterpret_cast<float*>(a.F);
  float* S = reinterpret_cast<float*>(a.S);
  float* T = reinterpret_cast<float*>(a.T);
  // the previous block already left X X^T within its threshold of I: the
  // block is one Newton-Schulz step, applied by its FP32 correction instead
  // (every CTA reads the same flag, so none waits for another)
  if (a.shortcut && *a.shortcut == 0) return;
  unsigned* cT = a.cnt;
  unsigned* rA = a.cnt + kComposeMaxTiles;
  unsigned* cA = a.cnt + 2 * kComposeMaxTiles;
  const unsigned per_block = (unsigned)(nt * NJ);   // items per row or column block and phase
  const int max_spin = a.max_spin > 0 ? a.max_spin : kCMaxSpin;
  // F_j lives in F when ns - j is even, else in S, so that F_ns ends in F
  auto Fbuf = [&](int j) { return ((ns - j) & 1) ? S : F; };
  for (int j = 0; j < ns; ++j) {
    float alh, all, mbh, mbl;
    split_d(a.alpha[j], alh, all);
    split_d(-a.beta[j], mbh, mbl);
    const bool last = j + 1 == ns;
    const float* Aj = (j & 1) ? A1 : A0;
    float* An = (j & 1) ? A0 : A1;
    const float* Fj = Fbuf(j);
    float* Fn = Fbuf(j + 1);
    // phase 1: F_{j+1} (F_1 = Pm_0 elementwise) and, before the last step, T
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      const int b = it / ntt, ti = (it % ntt) / nt, tj = it % nt;
      if (j > 0 && !df_wait(sm, rA + ti, per_block * j, cA + tj, per_block * j, a.err, max_spin))
        return;
      df_item(sm, P, ld, Aj + b * P2, !last, j > 0 ? Fj + b * P2 : nullptr,
              last ? nullptr : Aj + b * P2, alh, all, mbh, mbl, ti * kCT, tj * kCT,
              j > 0 ? Fn + b * P2 : nullptr, last ? nullptr : T + b * P2,
              j == 0 ? Fn + b * P2 : nullptr);
      if (!last) df_signal(cT + tj, nullptr);
      else __syncthreads();   // the staged rows are read by the stores above
    }
    if (last) break;
    // phase 2: A_{j+1} = Pm_j T
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
      const int b = it / ntt, ti = (it % ntt) / nt, tj = it % nt;
      if (!df_wait(sm, cT + tj, per_block * (j + 1), nullptr, 0, a.err, max_spin)) return;
      df_item(sm, P, ld, Aj + b * P2, false, T + b * P2, nullptr, alh, all, mbh, mbl, ti * kCT,
              tj * kCT, An + b * P2, nullptr, nullptr);
      df_signal(rA + ti, cA + tj);
    }
  }
}

struct DeviceGrid {
  int sms = 0, per_sm = 0, per_sm_df = 0;
};
std::mutex g_grid_mutex;
DeviceGrid g_grid[64];

int compose_grid_cap(bool df) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(g_grid_mutex);
  DeviceGrid& g = g_grid[dev];
  if (!g.sms) {
    int sms = 0, occ = 0, occ_df = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, polar_compose_kernel, kCThreads, 0) !=
        cudaSuccess)
      return 0;
    // the double-float kernel's shared memory is dynamic, sized by P
    const int df_max = (int)compose_df_smem(kCMaxP);
    if (cudaFuncSetAttribute(polar_compose_df_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             df_max) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_df, polar_compose_df_kernel, kCThreads,
                                                      df_max) != cudaSuccess)
      return 0;
    g.sms = sms;
    g.per_sm = std::min(occ, 2);
    g.per_sm_df = std::min(occ_df, 2);
  }
  return g.sms * (df ? g.per_sm_df : g.per_sm);
}

constexpr int kSPThreads = 256;

// c[i][j] = sum_k x[i * xs_i + k * xs_k] y[k * ys_k + j * ys_j] over k < K in
// pair arithmetic, for the (i, j) this thread owns: even and odd k in two
// independent accumulators (half the dependent chain), each renormalised
// every 8 terms, added at the end.
__device__ __forceinline__ void sp_dot(const float* xh, const float* xl, int xs_i, int xs_k,
                                      const float* yh, const float* yl, int ys_k, int ys_j, int i,
                                      int j, int K, float& vh, float& vl) {
  float sh0 = 0.f, sl0 = 0.f, sh1 = 0.f, sl1 = 0.f;
  int k = 0;
  for (; k + 1 < K; k += 2) {
    pair_mac(xh[i * xs_i + k * xs_k], xl[i * xs_i + k * xs_k], yh[k * ys_k + j * ys_j],
             yl[k * ys_k + j * ys_j], sh0, sl0);
    pair_mac(xh[i * xs_i + (k + 1) * xs_k], xl[i * xs_i + (k + 1) * xs_k],
             yh[(k + 1) * ys_k + j * ys_j], yl[(k + 1) * ys_k + j * ys_j], sh1, sl1);
    if ((k & 15) == 14) {
      pair_renorm(sh0, sl0);
      pair_renorm(sh1, sl1);
    }
  }
  if (k < K)
    pair_mac(xh[i * xs_i + k * xs_k], xl[i * xs_i + k * xs_k], yh[k * ys_k + j * ys_j],
             yl[k * ys_k + j * ys_j], sh0, sl0);
  pair_renorm(sh0, sl0);
  pair_renorm(sh1, sl1);
  pair_add(sh0, sl0, sh1, sl1, vh, vl);
}

// One CTA (up to 256 threads); all matrices as FP32 pairs in shared memory:
// X (P x N), A, F, Pm, T, U (P x P).  Per block: A = X X^T; F = I; per step
// Pm = alpha I - beta A, F <- Pm F and (not in the last step) A <- Pm (A Pm);
// then X <- F X.
__global__ void __launch_bounds__(kSPThreads) small_polar_kernel(const SmallPolarArgs a) {
  extern __shared__ __align__(16) float spm[];
  const int P = a.P, N = a.N, PP = P * P, PN = P * N;
  float* Xh = spm;
  float* Xl = Xh + PN;
  float* Yh = Xl + PN;   // F X, before it replaces X
  float* Yl = Yh + PN;
  float* Ah = Yl + PN;
  float* Al = Ah + PP;
  float* Fh = Al + PP;
  float* Fl = Fh + PP;
  float* Mh = Fl + PP;   // Pm
  float* Ml = Mh + PP;
  float* Th = Ml + PP;   // A Pm, then the new F
  float* Tl = Th + PP;
  for (int e = threadIdx.x; e < PN; e += blockDim.x) split_d(a.X[e], Xh[e], Xl[e]);
  __syncthreads();
  int step = 0;
  for (int b = 0; b < a.nblocks; ++b) {
    for (int e = threadIdx.x; e < PP; e += blockDim.x) {
      const int i = e / P, j = e % P;
      sp_dot(Xh, Xl, N, 1, Xh, Xl, 1, N, i, j, N, Ah[e], Al[e]);
      Fh[e] = i == j ? 1.f : 0.f;
      Fl[e] = 0.f;
    }
    __syncthreads();
    const int last = a.block_end[b] - 1;
    for (; step <= last; ++step) {
      float ah, al, bh, bl;
      split_d(a.alpha[step], ah, al);
      split_d(-a.beta[step], bh, bl);
      for (int e = threadIdx.x; e < PP; e += blockDim.x) {
        float h, l;
        pair_mul(Ah[e], Al[e], bh, bl, h, l);
        if (e / P == e % P) pair_add(h, l, ah, al, h, l);
        Mh[e] = h;
        Ml[e] = l;
      }
      __syncthreads();
      // new F into T (Pm F), and, not in the last step, A Pm into ... F's old
      // slot is still read, so A Pm goes to the X-sized scratch Y
      for (int e = threadIdx.x; e < PP; e += blockDim.x) {
        const int i = e / P, j = e % P;
        sp_dot(Mh, Ml, P, 1, Fh, Fl, P, 1, i, j, P, Th[e], Tl[e]);
        if (step < last) sp_dot(Ah, Al, P, 1, Mh, Ml, P, 1, i, j, P, Yh[e], Yl[e]);
      }
      __syncthreads();
      for (int e = threadIdx.x; e < PP; e += blockDim.x) {
        Fh[e] = Th[e];
        Fl[e] = Tl[e];
        if (step < last) {
          const int i = e / P, j = e % P;
          sp_dot(Mh, Ml, P, 1, Yh, Yl, P, 1, i, j, P, Ah[e], Al[e]);
        }
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < PN; e += blockDim.x) {
      const int i = e / N, j = e % N;
      sp_dot(Fh, Fl, P, 1, Xh, Xl, N, 1, i, j, P, Yh[e], Yl[e]);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < PN; e += blockDim.x) {
      Xh[e] = Yh[e];
      Xl[e] = Yl[e];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < PN; e += blockDim.x) {
    const double w = a.sign * ((double)Xh[e] + (double)Xl[e]);
    a.W[e] = w;
    if (a.W32) a.W32[e] = (float)w;
  }
}

}  // namespace

bool small_polar_supported(int P, long long N, int nblocks, int nsteps) {
  // everything in the default 48 KB of shared memory: 4 P N + 8 P^2 floats
  return P >= 1 && P <= kSmallPolarMaxP && N >= P && (4 * P * N + 8LL * P * P) * 4 <= 48 * 1024 &&
         nblocks >= 1 && nblocks <= kSmallPolarMaxBlocks && nsteps >= 1 &&
         nsteps <= kMaxComposeSteps;
}

int small_polar(const SmallPolarArgs& a, cudaStream_t s) {
  if (!small_polar_supported(a.P, a.N, a.nblocks, a.block_end[a.nblocks - 1])) return -1;
  const size_t smem = (4 * (size_t)a.P * a.N + 8 * (size_t)a.P * a.P) * sizeof(float);
  // as many threads as the largest matrix has entries, in whole warps (one
  // warp for the 4 x 4 layer: its barriers are then cheap), at most 256
  const int elems = std::max(a.P * a.N, a.P * a.P);
  const int threads = std::min(kSPThreads, (elems + 31) / 32 * 32);
  launch_k(small_polar_kernel, 1, threads, smem, s, a);
  return 1;
}

bool compose_supported(int P, int nsteps) {
  return P >= 1 && P <= kCMaxP && nsteps >= 1 && nsteps <= kMaxComposeSteps;
}

double compose_flops(int P, int NJ, int nsteps) {
  const int nt = (P + kCT - 1) / kCT;
  const double per_product = 2.0 * nt * nt * kCT * kCT * (double)P * NJ;
  double f = 0.0;
  for (int j = 0; j < nsteps; ++j) {
    const bool last = j + 1 == nsteps;
    f += per_product * ((j > 0 ? 1 : 0) + (last ? 0 : 2));
  }
  return f;
}

int polar_compose(const ComposeArgs& a, cudaStream_t s, bool df) {
  if (!compose_supported(a.P, a.nsteps)) return -1;
  int cap = compose_grid_cap(df);
  if (cap <= 0) return -1;
  if (a.grid_share > 1) cap = std::max(1, cap / a.grid_share);
  const int nt = (a.P + kCT - 1) / kCT;
  // the FP64 kernel's first phase holds two tiles per output tile, the
  // double-float kernel's one item per output tile
  const int grid = std::max(1, std::min(cap, (df ? 1 : 2) * nt * nt * a.NJ));
  if (df) cudaMemsetAsync(a.cnt, 0, 3 * kComposeMaxTiles * sizeof(unsigned), s);
  else cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kCThreads);
  cfg.dynamicSmemBytes = df ? compose_df_smem(a.P) : 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const cudaError_t e = df ? cudaLaunchKernelEx(&cfg, polar_compose_df_kernel, a)
                           : cudaLaunchKernelEx(&cfg, polar_compose_kernel, a);
  return e == cudaSuccess ? 1 : -1;
}

}  // namespace ttn
