// Grouped, batched, strided FP64 matrix products on the CUDA cores.
//
// Every O(chi^4) contraction of the sweep (Sec. III.A: "a sequence of
// tensor-tensor contractions ... matrix-matrix multiplications") is one
// GemmDesc: a sum over groups of A_g B_g with two-level K and batch indices, so
// that index permutations of the rank-3 tensors (Sec. V: "permuting indices of
// rank-3 tensors") are folded into the address arithmetic and never stored.
#include <algorithm>
#include <cstdlib>
#include <cstdio>
#include <mutex>

#include "../../include/ttn.h"
#include "common.h"

namespace ttn {

namespace {

constexpr int kBK = 16;
constexpr int kThreads = 256;

struct TileRange {
  int g_begin, t_begin;  // first group and k-tile inside it
  int tiles;             // number of k-tiles of this split
};

__device__ __forceinline__ double ld_operand(const Operand& o, int k0_log2, long long base,
                                             int i, int k) {
  const int k0 = k & ((1 << k0_log2) - 1);
  const int k1 = k >> k0_log2;
  const long long e = base + i * o.s_mn + k0 * o.s_k0 + (long long)k1 * o.s_k1;
  return o.f32 ? (double)static_cast<const float*>(o.p)[e] : static_cast<const double*>(o.p)[e];
}

__device__ __forceinline__ void st_out(const GemmDesc& d, long long e, double acc) {
  if (d.c_f32) {
    float* c = static_cast<float*>(d.C) + e;
    *c = d.beta == 0.0 ? (float)(d.alpha * acc) : (float)(d.alpha * acc + d.beta * (double)*c);
  } else {
    double* c = static_cast<double*>(d.C) + e;
    *c = d.beta == 0.0 ? d.alpha * acc : d.alpha * acc + d.beta * *c;
  }
}

// BM x BN output tile per CTA, 256 threads, each thread TM x TN outputs.
template <int BM, int BN>
__global__ void __launch_bounds__(kThreads) gemm_f64_kernel(const GemmDesc d, int total_tiles) {
  pdl_wait();
  pdl_trigger();
  constexpr int TM = BM / 16, TN = BN / 16;
  if (desc_skipped(d)) return;
  __shared__ double As[kBK][BM + 1];
  __shared__ double Bs[kBK][BN + 1];

  const int tiles_n = (d.N + BN - 1) / BN;
  int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  if (d.sym) {
    // symmetric product: only tiles on or above the diagonal are launched
    // (blockIdx.x counts them row by row); the mirror tile fills the rest
    int u = blockIdx.x, row = tiles_n;
    tm = 0;
    while (u >= row) { u -= row; ++tm; --row; }
    tn = tm + u;
  }
  const int b = blockIdx.y;
  const int b0 = b % d.B0, b1 = b / d.B0;
  const int split = blockIdx.z;
  const int m0 = tm * BM, n0 = tn * BN;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;

  // contiguous range of k-tiles for this split
  const int t_lo = (int)((long long)total_tiles * split / d.splits);
  const int t_hi = (int)((long long)total_tiles * (split + 1) / d.splits);

  double acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.0;

  int t_global = 0;
  for (int g = 0; g < d.ngroups && t_global < t_hi; ++g) {
    const Group& G = d.g[g];
    const int nt = (G.K + kBK - 1) / kBK;
    if (t_global + nt <= t_lo) { t_global += nt; continue; }
    const long long abase = b0 * G.a.s_b0 + (long long)b1 * G.a.s_b1;
    const long long bbase = b0 * G.b.s_b0 + (long long)b1 * G.b.s_b1;
    const int first = max(0, t_lo - t_global), last = min(nt, t_hi - t_global);
    const bool a_kfast = (G.a.s_k0 == 1);
    const bool b_kfast = (G.b.s_k0 == 1);
    for (int t = first; t < last; ++t) {
      const int kb = t * kBK;
      // stage A tile (BM x kBK) and B tile (kBK x BN)
      for (int e = threadIdx.x; e < BM * kBK; e += kThreads) {
        int mi, ki;
        if (a_kfast) { ki = e % kBK; mi = e / kBK; } else { mi = e % BM; ki = e / BM; }
        const int m = m0 + mi, k = kb + ki;
        As[ki][mi] = (m < d.M && k < G.K) ? ld_operand(G.a, G.k0_log2, abase, m, k) : 0.0;
      }
      for (int e = threadIdx.x; e < BN * kBK; e += kThreads) {
        int ni, ki;
        if (b_kfast) { ki = e % kBK; ni = e / kBK; } else { ni = e % BN; ki = e / BN; }
        const int n = n0 + ni, k = kb + ki;
        Bs[ki][ni] = (n < d.N && k < G.K) ? ld_operand(G.b, G.k0_log2, bbase, n, k) : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kBK; ++kk) {
        double av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
    t_global += nt;
  }

  if (d.splits == 1) {
    const long long cb = b0 * d.sc_b0 + (long long)b1 * d.sc_b1;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < d.M && n < d.N) {
          st_out(d, cb + m * d.sc_m + n * d.sc_n, acc[i][j]);
          if (d.sym && tm < tn) st_out(d, cb + n * d.sc_m + m * d.sc_n, acc[i][j]);
        }
      }
  } else {
    const long long MN = (long long)d.M * d.N;
    double* Pp = d.partial + ((long long)split * d.B0 * d.B1 + b) * MN;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
        if (m < d.M && n < d.N) Pp[(long long)m * d.N + n] = acc[i][j];
      }
  }
}

// C = alpha * sum_s partial[s] + beta * C (FP64) over the K splits.  A CTA
// owns 32 consecutive outputs; its 8 warps each sum a contiguous eighth of the
// splits in order (loads in flight together), and warp 0 adds the eight sums
// in group order (a fixed order of terms).
__global__ void splitk_reduce_kernel(const GemmDesc d) {
  pdl_wait();
  pdl_trigger();
  if (desc_skipped(d)) return;
  __shared__ double gs[8][32];
  const long long MN = (long long)d.M * d.N;
  const long long total = MN * d.B0 * d.B1;
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int s_lo = (int)((long long)d.splits * g / 8);
  const int s_hi = (int)((long long)d.splits * (g + 1) / 8);
  for (long long e0 = blockIdx.x * 32LL; e0 < total; e0 += gridDim.x * 32LL) {
    const long long e = e0 + lane;
    long long b = 0, r = 0;
    double acc = 0.0;
    if (e < total) {
      b = e / MN;
      r = e % MN;
      const int m = (int)(r / d.N), n = (int)(r % d.N);
      // symmetric product: below-diagonal tiles were not computed; read the mirror
      const long long src =
          (d.sym && m / d.sym_tile > n / d.sym_tile) ? (long long)n * d.N + m : r;
      for (int sp0 = s_lo; sp0 < s_hi; sp0 += 8) {
        double xs[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          xs[q] = sp0 + q < s_hi ? d.partial[((sp0 + q) * d.B0 * d.B1 + b) * MN + src] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q) acc += xs[q];
      }
    }
    gs[g][lane] = acc;
    __syncthreads();
    if (g == 0 && e < total) {
      double t = 0.0;
      for (int q = 0; q < 8; ++q) t += gs[q][lane];
      const int m = (int)(r / d.N), n = (int)(r % d.N);
      const int b0 = (int)(b % d.B0), b1 = (int)(b / d.B0);
      st_out(d, b0 * d.sc_b0 + (long long)b1 * d.sc_b1 + m * d.sc_m + n * d.sc_n, t);
    }
    __syncthreads();
  }
}

int total_k_tiles(const GemmDesc& d) {
  int t = 0;
  for (int g = 0; g < d.ngroups; ++g) t += (d.g[g].K + kBK - 1) / kBK;
  return t;
}

template <int BM, int BN>
int launch_tile(const GemmDesc& d, cudaStream_t s) {
  const int tn = (d.N + BN - 1) / BN;
  const int tiles = d.sym ? tn * (tn + 1) / 2 : ((d.M + BM - 1) / BM) * tn;
  dim3 grid(tiles, d.B0 * d.B1, d.splits);
  launch_k(gemm_f64_kernel<BM, BN>, grid, kThreads, 0, s, d, total_k_tiles(d));
  return 1;
}

}  // namespace

// SM count of the current device, read once per device (152 on GB300, also
// the value when no device is visible, e.g. when only sizes are planned).
bool pdl_enabled() {
  static const bool on = [] {
    const char* e = std::getenv("TTN_PDL");
    return e && e[0] && e[0] != '0';
  }();
  return on;
}

int device_sm_count() {
  static std::mutex mu;
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 152;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!cache[dev]) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      cudaGetLastError();
      sms = 152;
    }
    cache[dev] = sms;
  }
  return cache[dev];
}

// 64 x 64 tiles when they alone give two waves, else 32 x 32 or 16 x 16.
int f64_tile(const GemmDesc& d) {
  if (d.tile == 16 || d.tile == 32 || d.tile == 64) return d.tile;
  const long long b = (long long)d.B0 * d.B1;
  const long long wave2 = 2LL * device_sm_count();
  if (d.M >= 64 && d.N >= 64 && ((long long)((d.M + 63) / 64) * ((d.N + 63) / 64) * b >= wave2 ||
                                 total_k_tiles(d) < 8))
    return 64;
  if (d.M >= 32 && d.N >= 32) return 32;
  if (d.M >= 64 && d.N >= 64) return 64;
  return 16;
}

int gemm_pick_splits(const GemmDesc& d) {
  if (d.prec != 0 && gemm_tc_supported(d)) return tc_pick_splits(d);
  const int bm = f64_tile(d);
  const long long tm = (d.M + bm - 1) / bm, tn = (d.N + bm - 1) / bm;
  // a symmetric product launches only the tiles on or above the diagonal
  const long long tiles = (d.sym && d.M == d.N) ? tm * (tm + 1) / 2 : tm * tn;
  const long long base = tiles * d.B0 * d.B1;
  const int kt = total_k_tiles(d);
  const long long wave2 = 2LL * device_sm_count();   // two CTAs per SM
  if (base >= wave2 || kt < 4) return 1;
  int s = (int)std::min<long long>((wave2 + base - 1) / base, kt / 2);
  s = std::max(1, std::min(s, 64));
  return s;
}

size_t gemm_partial_elems(const GemmDesc& d, int splits) {
  return splits > 1 ? (size_t)splits * d.B0 * d.B1 * d.M * d.N : 0;
}

int gemm_launch(const GemmDesc& d0, cudaStream_t s) {
  if (d0.prec != 0 && gemm_tc_supported(d0)) return gemm_tc_launch(d0, s);
  GemmDesc d = d0;
  if (d.M <= 0 || d.N <= 0 || d.B0 * d.B1 <= 0) return 0;
  int n = 0;
  const int t = f64_tile(d);
  d.sym_tile = t;
  if (d.sym && d.M != d.N) d.sym = 0;
  if (t == 64) n += launch_tile<64, 64>(d, s);
  else if (t == 32) n += launch_tile<32, 32>(d, s);
  else n += launch_tile<16, 16>(d, s);
  if (d.splits > 1) {
    const long long total = (long long)d.M * d.N * d.B0 * d.B1;
    const int blocks = (int)std::min<long long>((total + 31) / 32, 8192);
    launch_k(splitk_reduce_kernel, blocks, 256, 0, s, d);
    ++n;
  }
  return n;
}

}  // namespace ttn

// ---------------------------------------------------------------------------
// Allocation-free variant of the split-K close product.
//
// Callers such as plug-ins of a host application that owns the CUDA allocator,
// or code running where cudaMalloc is not allowed, cannot hand the library a
// scratch buffer.  For them ttn_close_noalloc runs the same FP64 split-K
// product, but keeps its partial sums in this fixed array in device memory.
// Every GPU that loads the library holds the array (8 MiB) until the process
// exits.  In host code the array's name is only a host-side stand-in, so the
// entry point fetches its device address once per device with
// cudaGetSymbolAddress and hands that to the kernels.
// ---------------------------------------------------------------------------

namespace ttn {
namespace {

constexpr long long kNoAllocScratchDoubles = 1LL << 20;   // 8 MiB of FP64 partial sums
constexpr int kNoAllocMaxDim = 256;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

double* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

}  // namespace

}  // namespace ttn

extern "C" int ttn_close_noalloc(const double* d_Y, const double* d_W, int P, int Q, long long n2,
                                 double* d_C, void* stream) {
  using namespace ttn;
  if (!d_Y || !d_W || !d_C) return TTN_EINVAL;
  if (P < 1 || Q < 1 || P > kNoAllocMaxDim || Q > kNoAllocMaxDim) return TTN_EINVAL;
  if (n2 < 1 || n2 > (1LL << 30)) return TTN_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return TTN_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TTN_ECUDA;
      g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  GemmDesc d;
  memset(&d, 0, sizeof(d));
  d.M = P; d.N = Q; d.B0 = 1; d.B1 = 1;
  d.C = d_C; d.sc_m = Q; d.sc_n = 1;
  d.alpha = 1.0; d.beta = 0.0; d.prec = 0;
  Group g;
  // K0 = 1, K1 = n2: any length, addressed through the K1 stride
  g.a.p = d_Y; g.a.s_mn = n2; g.a.s_k0 = 1; g.a.s_k1 = 1; g.a.s_b0 = 0; g.a.s_b1 = 0; g.a.f32 = 0;
  g.b.p = d_W; g.b.s_mn = n2; g.b.s_k0 = 1; g.b.s_k1 = 1; g.b.s_b0 = 0; g.b.s_b1 = 0; g.b.f32 = 0;
  g.K = static_cast<int>(n2);
  g.k0_log2 = 0;
  d.g[0] = g;
  d.ngroups = 1;
  const long long per_split = static_cast<long long>(P) * Q;
  int splits = gemm_pick_splits(d);
  splits = static_cast<int>(std::min<long long>(splits, kNoAllocScratchDoubles / per_split));
  d.splits = std::max(1, splits);
  d.partial = scratch;
  // an error left pending by earlier work of the caller is reported, not
  // cleared, and nothing is launched; an error of this call's own launches
  // is reported and cleared
  if (cudaPeekAtLastError() != cudaSuccess) return TTN_ECUDA;
  if (gemm_launch(d, reinterpret_cast<cudaStream_t>(stream)) < 1) return TTN_ECUDA;
  return cudaGetLastError() == cudaSuccess ? TTN_OK : TTN_ECUDA;
}
