// Diagnostic entry point: the tensor-core engine against the FP64 engine on
// seeded random operands, over the operand layouts the sweep uses (K-major,
// M/N-major, two-level K, two-level batch, ragged edges, split K, alpha/beta).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/ttn.h"
#include "common.h"

namespace ttn {
namespace {

__global__ void fill_uniform(double* x, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[i] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;   // splitmix64 -> [-1, 1)
  }
}

// A = I + eps (F + F^T) / 2 for F (P x P) with entries in [-1, 1).
__global__ void near_identity(const double* F, double* A, int P, double eps) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < P * P; e += gridDim.x * blockDim.x) {
    const int i = e / P, j = e % P;
    A[e] = (i == j ? 1.0 : 0.0) + eps * 0.5 * (F[(long long)i * P + j] + F[(long long)j * P + i]);
  }
}

__global__ void max_abs_diff(const double* a, const double* b, long long n, double* out) {
  __shared__ double sd[256], sm[256];
  double d = 0.0, m = 0.0;
  for (long long i = threadIdx.x; i < n; i += blockDim.x) {
    d = fmax(d, fabs(a[i] - b[i]));
    m = fmax(m, fabs(b[i]));
  }
  sd[threadIdx.x] = d;
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + s]);
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { out[0] = sd[0]; out[1] = sm[0]; }
}

Operand mk(const double* p, long long mn, long long k0, long long k1 = 0, long long b0 = 0,
           long long b1 = 0) {
  Operand o;
  o.p = p; o.s_mn = mn; o.s_k0 = k0; o.s_k1 = k1; o.s_b0 = b0; o.s_b1 = b1; o.f32 = 0;
  return o;
}

Operand mk32(const float* p, long long mn, long long k0) {
  Operand o = mk(nullptr, mn, k0);
  o.p = p;
  o.f32 = 1;
  return o;
}

int lg(int x) { int r = 0; while ((1 << r) < x) ++r; return r; }

}  // namespace
}  // namespace ttn

using namespace ttn;

extern "C" int ttn_selftest_gemm(void* d_ws, size_t bytes, int prec, double* out_rel, int n_out,
                                 void* stream) {
  if (!d_ws || !out_rel || n_out < 11 || prec < 1 || prec > 4) return TTN_EINVAL;   // 16 cases
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  gemm_tc_init();
  double* base = reinterpret_cast<double*>(d_ws);
  const size_t cap = bytes / sizeof(double);
  size_t off = 0;
  auto take = [&](size_t n) -> double* {
    off = (off + 31) & ~size_t(31);
    double* p = base + off;
    off += n;
    return p;
  };
  struct Case { GemmDesc d; long long c_elems; };
  std::vector<Case> cases;
  const size_t big = 16384 * 128;
  double* A = take(4 * big);
  double* B = take(4 * big);
  double* C1 = take(big);
  double* C2 = take(big);
  double* partial = take(64 * big / 4);
  double* res = take(4);
  int* err = reinterpret_cast<int*>(take(1));
  if (off > cap) return TTN_ENOMEM;
  fill_uniform<<<592, 256, 0, s>>>(A, 4 * big, 11);
  fill_uniform<<<592, 256, 0, s>>>(B, 4 * big, 23);
  cudaMemsetAsync(err, 0, sizeof(int), s);

  auto base_desc = [&](int M, int N, int B0, int B1, long long sm, long long sn, long long sb0,
                       long long sb1) {
    GemmDesc d;
    memset(&d, 0, sizeof(d));
    d.M = M; d.N = N; d.B0 = B0; d.B1 = B1;
    d.sc_m = sm; d.sc_n = sn; d.sc_b0 = sb0; d.sc_b1 = sb1;
    d.alpha = 1.0; d.beta = 0.0; d.splits = 1; d.err = err;
    return d;
  };
  auto group = [&](Operand a, Operand b, int K0, int K1) {
    Group g; g.a = a; g.b = b; g.K = K0 * K1; g.k0_log2 = lg(K0); return g;
  };
  {  // 1: A K-major, B N-major, M=256 N=128 K=256
    GemmDesc d = base_desc(256, 128, 1, 1, 128, 1, 0, 0);
    d.g[d.ngroups++] = group(mk(A, 256, 1), mk(B, 1, 128), 256, 1);
    cases.push_back({d, 256 * 128});
  }
  {  // 2: A M-major, B K-major, ragged K = 96
    GemmDesc d = base_desc(128, 64, 1, 1, 64, 1, 0, 0);
    d.g[d.ngroups++] = group(mk(A, 1, 128), mk(B, 96, 1), 32, 3);
    cases.push_back({d, 128 * 64});
  }
  {  // 3: ragged M = 200, N = 48, K = 40 (two groups of K 32 + 8)
    GemmDesc d = base_desc(200, 48, 1, 1, 48, 1, 0, 0);
    d.g[d.ngroups++] = group(mk(A, 32, 1), mk(B, 1, 48), 32, 1);
    d.g[d.ngroups++] = group(mk(A + 8192, 1, 200), mk(B + 8192, 8, 1), 8, 1);
    cases.push_back({d, 200 * 48});
  }
  {  // 4: long K = 16384 (split K), both K-major
    GemmDesc d = base_desc(128, 128, 1, 1, 128, 1, 0, 0);
    d.g[d.ngroups++] = group(mk(A, 16384, 1), mk(B, 16384, 1), 16384, 1);
    cases.push_back({d, 128 * 128});
  }
  {  // 5: two-level K (K0=16, K1=8) and two-level batch (B0=4, B1=3), two groups
    GemmDesc d = base_desc(128, 64, 4, 3, 64, 1, 128 * 64, 4 * 128 * 64);
    d.g[d.ngroups++] = group(mk(A, 16, 1, 4096, 128 * 16 * 8, 4 * 128 * 16 * 8),
                             mk(B, 1, 64, 8 * 64 * 16 / 8 * 8, 16 * 64 * 8, 0), 16, 8);
    d.g[d.ngroups++] = group(mk(A + 65536, 1, 128, 0, 0, 128 * 64),
                             mk(B + 65536, 64, 1, 0, 4096, 0), 64, 1);
    cases.push_back({d, 12 * 128 * 64});
  }
  {  // 6: alpha / beta, N = 256 (two BN=128 tiles), batch of 128 left products
    GemmDesc d = base_desc(128, 128, 128, 1, 128, 1, 128 * 128, 0);
    d.alpha = 2.0; d.beta = 0.5;
    d.g[d.ngroups++] = group(mk(A, 1, 128, 0, 0, 0), mk(B, 1, 128, 0, 128 * 128, 0), 128, 1);
    cases.push_back({d, 128 * 128 * 128});
  }
  {  // 7: M = 64 (half tile), N = 64, K = 4096, batch 3 with A batch stride (a close)
    GemmDesc d = base_desc(64, 64, 3, 1, 64, 1, 64 * 64, 0);
    d.g[d.ngroups++] = group(mk(A, 4096, 1, 0, 262144, 0), mk(B, 4096, 1, 0, 0, 0), 4096, 1);
    cases.push_back({d, 3 * 64 * 64});
  }
  {  // 8: left products batched over p (B0 = 64), M = N = K = 64, four groups, A shared
    GemmDesc d = base_desc(64, 64, 64, 1, 64, 1, 4096, 0);
    d.g[d.ngroups++] = group(mk(A, 1, 64), mk(B, 1, 64, 0, 4096, 0), 64, 1);
    d.g[d.ngroups++] = group(mk(B, 64, 1, 0, 4096, 0), mk(A + 4096, 1, 64), 64, 1);
    d.g[d.ngroups++] = group(mk(A + 8192, 1, 64), mk(B + 262144, 1, 64, 0, 4096, 0), 64, 1);
    d.g[d.ngroups++] = group(mk(A + 12288, 64, 1), mk(B + 524288, 1, 64, 0, 4096, 0), 64, 1);
    cases.push_back({d, 64 * 64 * 64});
  }
  {  // 9: right product M = 4096, N = 64, K = 64 (B = small operator, N-major)
    GemmDesc d = base_desc(4096, 64, 1, 1, 64, 1, 0, 0);
    d.g[d.ngroups++] = group(mk(A, 64, 1), mk(B, 1, 64), 64, 1);
    cases.push_back({d, 4096 * 64});
  }
  // FP32 sources (the storage of the mixed modes): copies of A and B
  float* A32 = reinterpret_cast<float*>(partial + 48 * big / 4);
  float* B32 = reinterpret_cast<float*>(partial + 56 * big / 4);
  to_f32(A, A32, 2 * big, s);
  to_f32(B, B32, 2 * big, s);
  auto mkf = [&](const float* p, long long mn, long long k0, long long k1, long long b0,
                 long long b1) {
    Operand o = mk(nullptr, mn, k0, k1, b0, b1);
    o.p = p;
    o.f32 = 1;
    return o;
  };
  {  // 10: FP32 sources, K-major A and N-major B, batch of 64 (right products)
    GemmDesc d = base_desc(4096, 64, 1, 1, 64, 1, 0, 0);
    d.g[d.ngroups++] = group(mkf(A32, 64, 1, 0, 0, 0), mkf(B32, 1, 64, 0, 0, 0), 64, 1);
    cases.push_back({d, 4096 * 64});
  }
  {  // 11: FP32 sources, M-major A and K-major B, K = 8192 (split K)
    GemmDesc d = base_desc(128, 128, 1, 1, 128, 1, 0, 0);
    d.g[d.ngroups++] = group(mkf(A32, 1, 128, 0, 0, 0), mkf(B32, 8192, 1, 0, 0, 0), 8192, 1);
    cases.push_back({d, 128 * 128});
  }
  // layouts of the TMA-fed engine (FP32 sources, TF32 modes): ragged tiles,
  // two-level K with a broadcast batch, batched transposed products, the
  // environment's mixed K-/MN-major groups, a split-K close with FP64 output
  {  // 12: ragged M = 200, N = 96 (a partial second tile of 64), both K-major, K = 64
    GemmDesc d = base_desc(200, 96, 1, 1, 96, 1, 0, 0);
    d.g[d.ngroups++] = group(mkf(A32, 64, 1, 0, 0, 0), mkf(B32, 64, 1, 0, 0, 0), 64, 1);
    cases.push_back({d, 200 * 96});
  }
  {  // 13: K0 = 32, K1 = 4; batch B0 = 3 over A, B broadcast over the batch, B MN-major
    GemmDesc d = base_desc(128, 64, 3, 1, 64, 1, 128 * 64, 0);
    d.g[d.ngroups++] = group(mkf(A32, 32, 1, 32 * 128, 4 * 32 * 128, 0),
                             mkf(B32, 1, 64, 32 * 64, 0, 0), 32, 4);
    cases.push_back({d, 3 * 128 * 64});
  }
  {  // 14: 16 left products: A MN-major shared, B MN-major batched (stride 128^2)
    GemmDesc d = base_desc(128, 128, 16, 1, 128, 1, 128 * 128, 0);
    d.g[d.ngroups++] = group(mkf(A32, 1, 128, 0, 0, 0), mkf(B32, 1, 128, 0, 128 * 128, 0), 128, 1);
    cases.push_back({d, 16 * 128 * 128});
  }
  {  // 15: environment shape, M = 128, N = 4096, K = 128: G K-major and G^T MN-major,
     // the one-leg products MN-major
    GemmDesc d = base_desc(128, 4096, 1, 1, 4096, 1, 0, 0);
    d.g[d.ngroups++] = group(mkf(A32, 128, 1, 0, 0, 0), mkf(B32, 1, 4096, 0, 0, 0), 128, 1);
    d.g[d.ngroups++] = group(mkf(A32 + 16384, 1, 128, 0, 0, 0), mkf(B32 + 524288, 1, 4096, 0, 0, 0),
                             128, 1);
    cases.push_back({d, 128 * 4096});
  }
  {  // 16: close product, K = 16384 (split K), batch of 2 over A, FP64 output
    GemmDesc d = base_desc(128, 128, 2, 1, 128, 1, 128 * 128, 0);
    d.g[d.ngroups++] = group(mkf(A32, 16384, 1, 0, 16384 * 128, 0), mkf(B32, 16384, 1, 0, 0, 0),
                             16384, 1);
    cases.push_back({d, 2 * 128 * 128});
  }
  const int nc = std::min<int>((int)cases.size(), n_out);
  std::vector<double> host(2);
  for (int i = 0; i < nc; ++i) {
    GemmDesc d = cases[i].d;
    d.partial = partial;
    if (d.beta != 0.0) {
      fill_uniform<<<592, 256, 0, s>>>(C1, cases[i].c_elems, 77);
      fill_uniform<<<592, 256, 0, s>>>(C2, cases[i].c_elems, 77);
    }
    GemmDesc r = d;
    r.prec = 0;
    r.splits = gemm_pick_splits(r);
    r.C = C1;
    gemm_launch(r, s);
    GemmDesc t = d;
    t.prec = prec;
    t.splits = gemm_pick_splits(t);
    t.C = C2;
    gemm_launch(t, s);
    max_abs_diff<<<1, 256, 0, s>>>(C2, C1, cases[i].c_elems, res);
    cudaMemcpyAsync(host.data(), res, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return TTN_ECUDA;
    out_rel[i] = host[0] / std::max(host[1], 1e-300);
  }
  int e = 0;
  cudaMemcpy(&e, err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e) return TTN_ETIMEOUT;
  return cudaGetLastError() == cudaSuccess ? TTN_OK : TTN_ECUDA;
}

extern "C" size_t ttn_selftest_bytes(void) {
  const size_t big = 16384 * 128;
  return (4 * big * 2 + 2 * big + 64 * big / 4 + 64) * sizeof(double) + 4096;
}

// Diagnostic: the double-float Gram and apply products of the polar factor
// (gemm_df.cu) against the FP64 engine on seeded operands.  Cases: Gram X X^T
// for (P, n2) = (128, 16384) (split K) and (96, 1000) (ragged); apply F X for
// (128, 16384) and (40, 1000); with n_out >= 5, out_rel[4] the Newton-Schulz
// step near convergence as the adaptive polar schedule takes it (D = 0.5 (I - A)
// from check_split, the correction D X as a 3xTF32 tensor-core product on X's
// FP32 head, X added in FP64 by scale_select; A = I + 1e-10 (F + F^T) / 2,
// P = 128, n2 = 16384) against (1.5 I - 0.5 A) X in FP64.
// out_rel[i] = max |C_df - C_fp64| / max |C_fp64|.
extern "C" int ttn_selftest_df(void* d_ws, size_t bytes, double* out_rel, int n_out,
                               void* stream) {
  if (!d_ws || !out_rel || n_out < 4) return TTN_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  double* base = reinterpret_cast<double*>(d_ws);
  const size_t cap = bytes / sizeof(double);
  size_t off = 0;
  auto take = [&](size_t n) -> double* {
    off = (off + 31) & ~size_t(31);
    double* p = base + off;
    off += n;
    return p;
  };
  const size_t big = 16384 * 128;
  double* X = take(big);                     // P x n2, FP64
  double* F = take(128 * 128);               // P x P, FP64
  float* Xp = reinterpret_cast<float*>(take(big));        // hi then lo (P n2 floats each)
  float* Fp = reinterpret_cast<float*>(take(128 * 128));
  double* C1 = take(big);
  double* C2 = take(big);
  double* partial = take(128 * 128 * 128);
  double* res = take(4);
  double* Aq = take(128 * 128);
  double* Fm = take(128 * 128);
  int* zero = reinterpret_cast<int*>(take(1));
  float* D32 = reinterpret_cast<float*>(take(128 * 128 / 2));
  float* Corr = reinterpret_cast<float*>(take(big / 2));
  if (off > cap) return TTN_ENOMEM;
  fill_uniform<<<592, 256, 0, s>>>(X, big, 31);
  fill_uniform<<<64, 256, 0, s>>>(F, 128 * 128, 37);
  struct Case { int gram, P; long long n2; };
  const Case cases[4] = {{1, 128, 16384}, {1, 96, 1000}, {0, 128, 16384}, {0, 40, 1000}};
  std::vector<double> host(2);
  for (int i = 0; i < 4; ++i) {
    const Case& cs = cases[i];
    const int P = cs.P;
    const long long n2 = cs.n2, PN = (long long)P * n2;
    df_split(X, Xp, Xp + PN, PN, s);
    GemmDesc r;
    memset(&r, 0, sizeof(r));
    r.B0 = 1; r.B1 = 1; r.alpha = 1.0; r.prec = 0; r.C = C1; r.sc_n = 1; r.partial = partial;
    long long celems;
    if (cs.gram) {
      r.M = P; r.N = P; r.sc_m = P;
      Group g;
      g.a = mk(X, n2, 1); g.b = mk(X, n2, 1); g.K = (int)n2; g.k0_log2 = 0;
      g.a.s_k1 = 1; g.b.s_k1 = 1;   // K0 = 1: any length through the K1 stride
      r.g[r.ngroups++] = g;
      df_gram(Xp, Xp + PN, P, n2, C2, partial, s);
      celems = (long long)P * P;
    } else {
      r.M = P; r.N = (int)n2; r.sc_m = n2;
      Group g;
      g.a = mk(F, P, 1); g.b = mk(X, 1, n2); g.K = P; g.k0_log2 = 0;
      g.a.s_k1 = 1; g.b.s_k1 = n2;
      r.g[r.ngroups++] = g;
      df_split(F, Fp, Fp + (long long)P * P, (long long)P * P, s);
      df_apply(Fp, Fp + (long long)P * P, Xp, Xp + PN, P, n2, C2, s);
      celems = PN;
    }
    r.splits = gemm_pick_splits(r);
    if (gemm_partial_elems(r, r.splits) > 128 * 128 * 128) r.splits = 1;
    gemm_launch(r, s);
    max_abs_diff<<<1, 256, 0, s>>>(C2, C1, celems, res);
    cudaMemcpyAsync(host.data(), res, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return TTN_ECUDA;
    out_rel[i] = host[0] / std::max(host[1], 1e-300);
  }
  if (n_out >= 5) {
    const int P = 128;
    const long long n2 = 16384, PN = (long long)P * n2;
    near_identity<<<64, 256, 0, s>>>(F, Aq, P, 1e-10);
    poly_step_matrix(Aq, Fm, P, 1, 1.5, 0.5, s);   // 1.5 I - 0.5 A
    cudaMemsetAsync(zero, 0, sizeof(int), s);
    GemmDesc r;
    memset(&r, 0, sizeof(r));
    r.B0 = 1; r.B1 = 1; r.alpha = 1.0; r.prec = 0; r.C = C1; r.sc_n = 1; r.partial = partial;
    r.M = P; r.N = (int)n2; r.sc_m = n2;
    Group g;
    g.a = mk(Fm, P, 1); g.b = mk(X, 1, n2); g.K = P; g.k0_log2 = 0;
    g.a.s_k1 = 1; g.b.s_k1 = n2;
    r.g[r.ngroups++] = g;
    r.splits = 1;
    gemm_launch(r, s);
    df_split(X, Xp, Xp + PN, PN, s);
    check_split(Aq, P, 0.0, -1.0, Fp, Fp + (long long)P * P, 1.0, nullptr, s, D32);
    GemmDesc t;
    memset(&t, 0, sizeof(t));
    t.B0 = 1; t.B1 = 1; t.alpha = 1.0; t.prec = TTN_TF32X3; t.C = Corr; t.c_f32 = 1;
    t.sc_n = 1; t.sc_m = n2; t.M = P; t.N = (int)n2; t.partial = partial;
    Group g2;
    g2.a = mk32(D32, P, 1); g2.b = mk32(Xp, 1, n2); g2.K = P; g2.k0_log2 = lg(P);
    t.g[t.ngroups++] = g2;
    t.splits = gemm_pick_splits(t);
    if (gemm_partial_elems(t, t.splits) > 128 * 128 * 128) t.splits = 1;
    gemm_launch(t, s);
    scale_select(X, X, zero, C2, PN, 1.0, s, nullptr, Corr);
    max_abs_diff<<<1, 256, 0, s>>>(C2, C1, (long long)P * n2, res);
    cudaMemcpyAsync(host.data(), res, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return TTN_ECUDA;
    out_rel[4] = host[0] / std::max(host[1], 1e-300);
  }
  return cudaGetLastError() == cudaSuccess ? TTN_OK : TTN_ECUDA;
}
