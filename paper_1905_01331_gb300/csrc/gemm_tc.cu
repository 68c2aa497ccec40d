// Tensor-core (tcgen05) engine of the grouped products, sm_103a.
//
// The O(chi^4) contractions of the sweep (Sec. III.A; Sec. V: "the cost
// scales as chi^4") run here in split precision: every FP64 operand element x
// is cut into a TF32 (or BF16) head h = round(x) and tail l = round(x - h) on
// the way into shared memory, and the product is accumulated in FP32 tensor
// memory as  A_l B_h + A_h B_l + A_h B_h  (3xTF32 / BF16x3) or A_h B_h alone.
//
// One CTA owns a 128 x BN output tile (BN <= 64).  All 256 threads stage
// operand tiles (any strides: the two-level K/batch index of GemmDesc),
// converting FP32 or FP64 to the MMA type and writing the K-major
// SWIZZLE_128B canonical layout; one thread issues tcgen05.mma into a TMEM
// accumulator and commits to an mbarrier per stage, so that staging of the
// next K tile overlaps the MMAs of the current one (two stages).  Staging is
// bound by the latency of its global loads, so the tiles are kept small enough
// (<= 96 KB of shared memory, <= 128 registers) for two CTAs per SM, whose
// loads overlap.  The epilogue reads TMEM with tcgen05.ld and writes FP32 or
// FP64 (or a split-K partial).  Every mbarrier wait is bounded; on a
// timeout the kernel raises an error flag, waits (bounded) for its own MMAs,
// frees its TMEM and returns.
#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched from the driver at run time)
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "common.h"
#include "f64_bits.cuh"

namespace ttn {

namespace {

constexpr int kThreadsTC = 256;
constexpr int kBM = 128;
constexpr int kStages = 2;
constexpr long kWaitLimit = 1L << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major, 128-byte swizzle, 8-row atoms stacked every 1024 bytes.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);        // start address
  d |= static_cast<uint64_t>(1) << 16;                      // leading byte offset (unused)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;              // stride byte offset
  d |= static_cast<uint64_t>(1) << 46;                      // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                      // SWIZZLE_128B
  return d;
}

// Instruction descriptor: D = F32, A/B format fmt (2 = TF32, 1 = BF16), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, int M, int N) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}

template <bool kBF16>
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                    uint32_t acc) {
  if constexpr (kBF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <typename T>
__device__ __forceinline__ T ld_op(const Operand& o, int k0_log2, long long base, int i, int k) {
  const int k0 = k & ((1 << k0_log2) - 1);
  const int k1 = k >> k0_log2;
  return static_cast<const T*>(o.p)[base + i * o.s_mn + k0 * o.s_k0 +
                                    static_cast<long long>(k1) * o.s_k1];
}

__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// Split x into head/tail bit patterns of the MMA type.
template <bool kBF16>
__device__ __forceinline__ void split(double x, uint32_t& hi, uint32_t& lo) {
  if constexpr (kBF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(static_cast<float>(x));
    const float hf = __bfloat162float(h);
    const __nv_bfloat16 l = __float2bfloat16_rn(static_cast<float>(x - static_cast<double>(hf)));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  } else {
    hi = tf32_bits(static_cast<float>(x));
    const float hf = __uint_as_float(hi);
    lo = tf32_bits(static_cast<float>(x - static_cast<double>(hf)));
  }
}

// The same split of an FP32 value: FP32 arithmetic only (no FP64 pipe).
template <bool kBF16>
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  if constexpr (kBF16) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
  } else {
    hi = tf32_bits(x);
    lo = tf32_bits(x - __uint_as_float(hi));
  }
}

// Byte offset of element (row r, k) in a K-major SWIZZLE_128B tile whose rows
// are 128 bytes (32 TF32 or 64 BF16 elements).
template <bool kBF16>
__device__ __forceinline__ uint32_t swz_off(int r, int k) {
  const uint32_t byte = kBF16 ? k * 2 : k * 4;
  const uint32_t chunk = (byte >> 4) ^ (r & 7);
  return r * 128 + (chunk << 4) + (byte & 15);
}

template <bool kBF16>
__device__ __forceinline__ void st_elem(uint8_t* tile, int r, int k, uint32_t bits) {
  if constexpr (kBF16)
    *reinterpret_cast<uint16_t*>(tile + swz_off<true>(r, k)) = static_cast<uint16_t>(bits);
  else
    *reinterpret_cast<uint32_t*>(tile + swz_off<false>(r, k)) = bits;
}

// Store 4 (TF32) or 8 (BF16) consecutive K values of row r, starting at a
// 16-byte chunk boundary kk, as one 16-byte swizzled chunk.
template <bool kBF16>
__device__ __forceinline__ void st_chunk(uint8_t* tile, int r, int kk, const uint32_t* v) {
  uint4 q;
  if constexpr (kBF16) {
    q.x = v[0] | (v[1] << 16); q.y = v[2] | (v[3] << 16);
    q.z = v[4] | (v[5] << 16); q.w = v[6] | (v[7] << 16);
  } else {
    q.x = v[0]; q.y = v[1]; q.z = v[2]; q.w = v[3];
  }
  *reinterpret_cast<uint4*>(tile + swz_off<kBF16>(r, kk)) = q;
}

// N consecutive values (N = 4 or 8) with 16-byte loads when aligned.
template <typename T, int N>
__device__ __forceinline__ void ldv(const T* p, T* out) {
  if constexpr (sizeof(T) == 4) {
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
      for (int i = 0; i < N; i += 4) {
        const float4 t = *reinterpret_cast<const float4*>(p + i);
        out[i] = t.x; out[i + 1] = t.y; out[i + 2] = t.z; out[i + 3] = t.w;
      }
      return;
    }
  } else {
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0) {
#pragma unroll
      for (int i = 0; i < N; i += 2) {
        const double2 t = *reinterpret_cast<const double2*>(p + i);
        out[i] = t.x; out[i + 1] = t.y;
      }
      return;
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i) out[i] = p[i];
}

// Stage rows [r0, r0 + ROWS) x K tile [kb, kb + BK) of one operand.  Fast
// paths when the tile lies inside one K0 slice and the source is K-major
// (s_k0 == 1: 16-byte loads along K) or MN-major (s_mn == 1: 16-byte loads
// along rows, transposed in registers); otherwise element by element.
template <typename T, bool kBF16, bool kSplit, int BK, int ROWS>
__device__ __forceinline__ void stage_operand_t(const Operand& o, int k0_log2, long long base,
                                                int r0, int nrows_valid, int kb, int Kg,
                                                uint8_t* hi_tile, uint8_t* lo_tile) {
  constexpr int CH = kBF16 ? 8 : 4;           // K values per 16-byte chunk
  constexpr int NCH = BK / CH;                // chunks per row (8)
  const int K0 = 1 << k0_log2;
  const int kvalid = min(BK, Kg - kb);
  const bool slice = (K0 >= BK) && (kvalid == BK);
  if (slice && o.s_k0 == 1) {
    const T* tb = static_cast<const T*>(o.p) + base +
                  static_cast<long long>(kb >> k0_log2) * o.s_k1 + (kb & (K0 - 1));
    // all loads of a group of tasks are issued before any conversion, so that
    // a thread has several 16-byte loads in flight
    constexpr int TASKS = (ROWS * NCH + kThreadsTC - 1) / kThreadsTC;
    constexpr int GRP = (sizeof(T) * CH <= 16) ? 4 : 2;
#pragma unroll
    for (int g0 = 0; g0 < TASKS; g0 += GRP) {
      T v[GRP][CH];
#pragma unroll
      for (int i = 0; i < GRP; ++i) {
        const int task = threadIdx.x + (g0 + i) * kThreadsTC;
        const int r = task / NCH, c = task % NCH;
        if (g0 + i < TASKS && task < ROWS * NCH && r < nrows_valid) {
          ldv<T, CH>(tb + static_cast<long long>(r0 + r) * o.s_mn + c * CH, v[i]);
        } else {
#pragma unroll
          for (int q = 0; q < CH; ++q) v[i][q] = T(0);
        }
      }
#pragma unroll
      for (int i = 0; i < GRP; ++i) {
        const int task = threadIdx.x + (g0 + i) * kThreadsTC;
        if (g0 + i >= TASKS || task >= ROWS * NCH) continue;
        const int r = task / NCH, c = task % NCH;
        uint32_t h[CH], l[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) split<kBF16>(v[i][q], h[q], l[q]);
        st_chunk<kBF16>(hi_tile, r, c * CH, h);
        if constexpr (kSplit) st_chunk<kBF16>(lo_tile, r, c * CH, l);
      }
    }
    return;
  }
  if (slice && o.s_mn == 1 && (nrows_valid & 3) == 0) {
    const T* tb = static_cast<const T*>(o.p) + base +
                  static_cast<long long>(kb >> k0_log2) * o.s_k1 +
                  static_cast<long long>(kb & (K0 - 1)) * o.s_k0;
    // task: 4 consecutive rows x one chunk of CH consecutive K values; the
    // eight chunks of a row go to consecutive threads, so that a warp's
    // swizzled 16-byte stores fill whole 128-byte rows (no bank conflicts)
    for (int task = threadIdx.x; task < (ROWS / 4) * NCH; task += kThreadsTC) {
      const int rq = task / NCH, c = task % NCH;
      const int r = rq * 4;
      T v[CH][4];
      if (r < nrows_valid) {
#pragma unroll
        for (int q = 0; q < CH; ++q)
          ldv<T, 4>(tb + static_cast<long long>(c * CH + q) * o.s_k0 + (r0 + r), v[q]);
      } else {
#pragma unroll
        for (int q = 0; q < CH; ++q)
#pragma unroll
          for (int i = 0; i < 4; ++i) v[q][i] = T(0);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t h[CH], l[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) split<kBF16>(v[q][i], h[q], l[q]);
        st_chunk<kBF16>(hi_tile, r + i, c * CH, h);
        if constexpr (kSplit) st_chunk<kBF16>(lo_tile, r + i, c * CH, l);
      }
    }
    return;
  }
  const bool kfast = (o.s_k0 == 1);
  constexpr int total = ROWS * BK;
#pragma unroll 4
  for (int e = threadIdx.x; e < total; e += kThreadsTC) {
    int r, kk;
    if (kfast) { kk = e % BK; r = e / BK; } else { r = e % ROWS; kk = e / ROWS; }
    const int k = kb + kk;
    T x = T(0);
    if (r < nrows_valid && k < Kg) x = ld_op<T>(o, k0_log2, base, r0 + r, k);
    uint32_t hh, ll;
    split<kBF16>(x, hh, ll);
    st_elem<kBF16>(hi_tile, r, kk, hh);
    if constexpr (kSplit) st_elem<kBF16>(lo_tile, r, kk, ll);
  }
}

template <bool kBF16, bool kSplit, int BK, int ROWS>
__device__ __forceinline__ void stage_operand(const Operand& o, int k0_log2, long long base,
                                              int r0, int nrows_valid, int kb, int Kg,
                                              uint8_t* hi_tile, uint8_t* lo_tile) {
  if (o.f32)
    stage_operand_t<float, kBF16, kSplit, BK, ROWS>(o, k0_log2, base, r0, nrows_valid, kb, Kg,
                                                    hi_tile, lo_tile);
  else
    stage_operand_t<double, kBF16, kSplit, BK, ROWS>(o, k0_log2, base, r0, nrows_valid, kb, Kg,
                                                     hi_tile, lo_tile);
}

// TF32 modes with FP32 operands: the global loads of both operand tiles are
// issued before any of them is split and stored, so that a K tile costs one
// load latency instead of two.  load_f32 fills v (16 values per thread for
// ROWS <= 128) on the two fast paths of stage_operand_t and returns the path
// (1: K-major, 2: MN-major) or 0 when neither applies (the caller then stages
// that operand with stage_operand).
template <int ROWS>
__device__ __forceinline__ int load_f32(const Operand& o, int k0_log2, long long base, int r0,
                                        int nrows_valid, int kb, int Kg, float* v) {
  constexpr int BK = 32, CH = 4, NCH = BK / CH;
  const int K0 = 1 << k0_log2;
  if (!(K0 >= BK && Kg - kb >= BK)) return 0;
  const float* tb = static_cast<const float*>(o.p) + base +
                    static_cast<long long>(kb >> k0_log2) * o.s_k1 + (kb & (K0 - 1)) * o.s_k0;
  if (o.s_k0 == 1) {
    constexpr int TASKS = (ROWS * NCH + kThreadsTC - 1) / kThreadsTC;
#pragma unroll
    for (int g = 0; g < TASKS; ++g) {
      const int task = threadIdx.x + g * kThreadsTC;
      const int r = task / NCH, c = task % NCH;
      if (task < ROWS * NCH && r < nrows_valid) {
        ldv<float, CH>(tb + static_cast<long long>(r0 + r) * o.s_mn + c * CH, v + g * CH);
      } else {
#pragma unroll
        for (int q = 0; q < CH; ++q) v[g * CH + q] = 0.f;
      }
    }
    return 1;
  }
  if (o.s_mn == 1 && (nrows_valid & 3) == 0) {
    constexpr int TASKS = ((ROWS / 4) * NCH + kThreadsTC - 1) / kThreadsTC;
#pragma unroll
    for (int g = 0; g < TASKS; ++g) {
      const int task = threadIdx.x + g * kThreadsTC;
      const int rq = task / NCH, c = task % NCH;
      const int r = rq * 4;
      if (task < (ROWS / 4) * NCH && r < nrows_valid) {
#pragma unroll
        for (int q = 0; q < CH; ++q)
          ldv<float, 4>(tb + static_cast<long long>(c * CH + q) * o.s_k0 + (r0 + r),
                        v + g * 16 + q * 4);
      } else {
#pragma unroll
        for (int q = 0; q < 16; ++q) v[g * 16 + q] = 0.f;
      }
    }
    return 2;
  }
  return 0;
}

// Split and store what load_f32 loaded (same task mapping).
template <bool kSplit, int ROWS>
__device__ __forceinline__ void store_f32(int path, const float* v, uint8_t* hi_tile,
                                          uint8_t* lo_tile) {
  constexpr int BK = 32, CH = 4, NCH = BK / CH;
  if (path == 1) {
    constexpr int TASKS = (ROWS * NCH + kThreadsTC - 1) / kThreadsTC;
#pragma unroll
    for (int g = 0; g < TASKS; ++g) {
      const int task = threadIdx.x + g * kThreadsTC;
      if (task >= ROWS * NCH) continue;
      const int r = task / NCH, c = task % NCH;
      uint32_t h[CH], l[CH];
#pragma unroll
      for (int q = 0; q < CH; ++q) split<false>(v[g * CH + q], h[q], l[q]);
      st_chunk<false>(hi_tile, r, c * CH, h);
      if constexpr (kSplit) st_chunk<false>(lo_tile, r, c * CH, l);
    }
  } else if (path == 2) {
    constexpr int TASKS = ((ROWS / 4) * NCH + kThreadsTC - 1) / kThreadsTC;
#pragma unroll
    for (int g = 0; g < TASKS; ++g) {
      const int task = threadIdx.x + g * kThreadsTC;
      if (task >= (ROWS / 4) * NCH) continue;
      const int rq = task / NCH, c = task % NCH;
      const int r = rq * 4;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        uint32_t h[CH], l[CH];
#pragma unroll
        for (int q = 0; q < CH; ++q) split<false>(v[g * 16 + q * 4 + i], h[q], l[q]);
        st_chunk<false>(hi_tile, r + i, c * CH, h);
        if constexpr (kSplit) st_chunk<false>(lo_tile, r + i, c * CH, l);
      }
    }
  }
}

// FP32 -> FP64 with integer operations (f64_bits.cuh): on this GPU the FP64
// pipe (two operations per SM per clock) would bound the epilogue of a tile.
__device__ __forceinline__ double f32_to_f64(float x) { return f64b::from_f32(x); }

// C = alpha x + beta C for one FP32 accumulator x.  With beta = 0 the scaling
// is an FP32 multiply (exact for alpha = +-1 or a power of two; otherwise one
// FP32 rounding, below that of the FP32 accumulation itself); only beta != 0
// with an FP64 C needs FP64 arithmetic.
__device__ __forceinline__ void store_out(const GemmDesc& d, long long idx, float x, float af,
                                          float bf) {
  if (d.c_f32) {
    float* c = static_cast<float*>(d.C) + idx;
    *c = d.beta == 0.0 ? af * x : fmaf(af, x, bf * *c);
  } else {
    double* c = static_cast<double*>(d.C) + idx;
    *c = d.beta == 0.0 ? f32_to_f64(af * x) : d.alpha * f32_to_f64(x) + d.beta * *c;
  }
}

struct TCParams {
  int total_tiles;
  int* err;
};

template <bool kBF16, bool kSplit, int BN>
__global__ void gemm_tc_kernel(const GemmDesc d, TCParams tp);

template <bool kBF16, bool kSplit, int BN>
constexpr int tc_smem_bytes() {
  return kStages * (kSplit ? 2 : 1) * (kBM * 128 + BN * 128) + 1024;
}

template <bool kBF16, bool kSplit, int BN>
void tc_configure() {
  cudaFuncSetAttribute(gemm_tc_kernel<kBF16, kSplit, BN>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                       tc_smem_bytes<kBF16, kSplit, BN>());
}

template <bool kBF16, bool kSplit, int BN>
__global__ void __launch_bounds__(kThreadsTC, 2) gemm_tc_kernel(const GemmDesc d, TCParams tp) {
  pdl_wait();
  pdl_trigger();
  constexpr int BK = kBF16 ? 64 : 32;            // one 128-byte swizzle row
  constexpr int KSTEP = kBF16 ? 16 : 8;          // K of one tcgen05.mma
  constexpr int kA = kBM * 128;                  // bytes of one A tile (128 rows)
  constexpr int kB = BN * 128;                   // bytes of one B tile
  constexpr int kStageBytes = (kSplit ? 2 : 1) * (kA + kB);
  constexpr uint32_t kIdesc = instr_desc(kBF16 ? 1u : 2u, kBM, BN);
  constexpr int kCols = BN < 32 ? 32 : BN;       // TMEM columns (power of two >= 32)

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t bars[kStages];
  __shared__ uint32_t tmem_slot;

  if (desc_skipped(d)) return;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (d.N + BN - 1) / BN;
  const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  const int b = blockIdx.y;
  const int b0 = b % d.B0, b1 = b / d.B0;
  const int split_id = blockIdx.z;
  const int m0 = tm * kBM, n0 = tn * BN;
  const int mvalid = min(kBM, d.M - m0), nvalid = min(BN, d.N - n0);
  const int t_lo = static_cast<int>(static_cast<long long>(tp.total_tiles) * split_id / d.splits);
  const int t_hi =
      static_cast<int>(static_cast<long long>(tp.total_tiles) * (split_id + 1) / d.splits);

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  bool ok = true;
  int issued = 0;   // K tiles whose MMAs were committed
  int t_global = 0;
  for (int g = 0; g < d.ngroups && t_global < t_hi && ok; ++g) {
    const Group& G = d.g[g];
    const int nt = (G.K + BK - 1) / BK;
    if (t_global + nt <= t_lo) { t_global += nt; continue; }
    const long long abase = b0 * G.a.s_b0 + static_cast<long long>(b1) * G.a.s_b1;
    const long long bbase = b0 * G.b.s_b0 + static_cast<long long>(b1) * G.b.s_b1;
    const int first = max(0, t_lo - t_global), last = min(nt, t_hi - t_global);
    // TF32 modes with FP32 operands: the global loads of K tile t + 1 are
    // issued as soon as tile t is in shared memory, so that they are in
    // flight during the barrier, the MMA issue and the wait for a free stage
    float va[16], vb[16];
    int pa = 0, pb = 0;
    const bool f32ops = G.a.f32 && G.b.f32;
    if constexpr (!kBF16) {
      if (f32ops && first < last) {
        pa = load_f32<kBM>(G.a, G.k0_log2, abase, m0, mvalid, first * BK, G.K, va);
        pb = load_f32<BN>(G.b, G.k0_log2, bbase, n0, nvalid, first * BK, G.K, vb);
      }
    }
    for (int t = first; t < last; ++t) {
      const int stage = issued % kStages;
      // the MMAs that read this stage (tile issued - kStages) must be done;
      // the decision to stop is taken by the whole CTA
      bool w_ok = true;
      if (issued >= kStages) w_ok = mbar_wait(&bars[stage], ((issued / kStages) - 1) & 1);
      if (!__syncthreads_and(w_ok)) { ok = false; break; }
      uint8_t* st = smem + stage * kStageBytes;
      uint8_t* a_hi = st;
      uint8_t* b_hi = st + kA;
      uint8_t* a_lo = st + kA + kB;
      uint8_t* b_lo = st + 2 * kA + kB;
      const int kb = t * BK;
      if constexpr (!kBF16) {
        if (f32ops) {
          store_f32<kSplit, kBM>(pa, va, a_hi, a_lo);
          store_f32<kSplit, BN>(pb, vb, b_hi, b_lo);
          if (!pa)
            stage_operand<kBF16, kSplit, BK, kBM>(G.a, G.k0_log2, abase, m0, mvalid, kb, G.K,
                                                  a_hi, a_lo);
          if (!pb)
            stage_operand<kBF16, kSplit, BK, BN>(G.b, G.k0_log2, bbase, n0, nvalid, kb, G.K,
                                                 b_hi, b_lo);
          if (t + 1 < last) {
            pa = load_f32<kBM>(G.a, G.k0_log2, abase, m0, mvalid, kb + BK, G.K, va);
            pb = load_f32<BN>(G.b, G.k0_log2, bbase, n0, nvalid, kb + BK, G.K, vb);
          }
        } else {
          stage_operand<kBF16, kSplit, BK, kBM>(G.a, G.k0_log2, abase, m0, mvalid, kb, G.K, a_hi,
                                                a_lo);
          stage_operand<kBF16, kSplit, BK, BN>(G.b, G.k0_log2, bbase, n0, nvalid, kb, G.K, b_hi,
                                               b_lo);
        }
      } else {
        stage_operand<kBF16, kSplit, BK, kBM>(G.a, G.k0_log2, abase, m0, mvalid, kb, G.K, a_hi,
                                              a_lo);
        stage_operand<kBF16, kSplit, BK, BN>(G.b, G.k0_log2, bbase, n0, nvalid, kb, G.K, b_hi,
                                             b_lo);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (threadIdx.x == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa_hi = smem_u32(a_hi), sb_hi = smem_u32(b_hi);
        const uint32_t sa_lo = smem_u32(a_lo), sb_lo = smem_u32(b_lo);
#pragma unroll
        for (int j = 0; j < BK / KSTEP; ++j) {
          const uint32_t off = j * 32;   // 32 bytes of K per instruction
          const uint32_t acc = (issued > 0 || j > 0) ? 1u : 0u;
          if constexpr (kSplit) {
            mma<kBF16>(tmem, smem_desc(sa_lo + off), smem_desc(sb_hi + off), kIdesc, acc);
            mma<kBF16>(tmem, smem_desc(sa_hi + off), smem_desc(sb_lo + off), kIdesc, 1u);
            mma<kBF16>(tmem, smem_desc(sa_hi + off), smem_desc(sb_hi + off), kIdesc, 1u);
          } else {
            mma<kBF16>(tmem, smem_desc(sa_hi + off), smem_desc(sb_hi + off), kIdesc, acc);
          }
        }
        mma_commit(&bars[stage]);
      }
      ++issued;
    }
    t_global += nt;
  }
  // wait for the last committed stage (MMAs complete in order)
  bool f_ok = true;
  if (issued > 0) {
    const int last = issued - 1;
    f_ok = mbar_wait(&bars[last % kStages], (last / kStages) & 1);
  }
  ok = __syncthreads_and(ok && f_ok);
  if (!ok && tp.err && threadIdx.x == 0) atomicOr(tp.err, 1);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // Epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 (rows), columns half w/4.
  // A split with no K tile contributes zeros (its accumulator was never written).
  if (ok) {
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int m = m0 + row;
    constexpr int kHalf = BN >= 32 ? BN / 2 : BN;
    const int c_begin = (warp >> 2) * kHalf;
    const bool active = (BN >= 32) || (warp < 4);
    const long long MN = static_cast<long long>(d.M) * d.N;
    const float af = static_cast<float>(d.alpha), bf = static_cast<float>(d.beta);
    for (int c0 = c_begin; active && c0 < c_begin + kHalf; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + c0;
      if (issued == 0) {
#pragma unroll
        for (int j = 0; j < 16; ++j) r[j] = 0u;
      } else {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
            "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
            "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      }
      if (m < d.M) {
        if (d.splits == 1) {
          const long long cb = b0 * d.sc_b0 + static_cast<long long>(b1) * d.sc_b1 + m * d.sc_m;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + c0 + j;
            if (n < d.N) store_out(d, cb + n * d.sc_n, __uint_as_float(r[j]), af, bf);
          }
        } else {
          // FP32 partials (the reduction adds them in FP32 pairs)
          float* P = reinterpret_cast<float*>(d.partial) +
                     (static_cast<long long>(split_id) * d.B0 * d.B1 + b) * MN +
                     static_cast<long long>(m) * d.N;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = n0 + c0 + j;
            if (n < d.N) P[n] = __uint_as_float(r[j]);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// C = alpha sum_s part[s] + beta C over the FP32 partials of the K splits,
// as an FP32 pair (error-free two-sum, low parts accumulated), then rounded
// to FP32.  A CTA owns 32 consecutive outputs; its 8 warps each sum a
// contiguous eighth of the splits in order (all of a warp's loads in flight
// together), and warp 0 adds the eight pairs in group order: a fixed order of
// terms, with 8x the parallelism of one thread per output.
__global__ void splitk_reduce_tc(const GemmDesc d) {
  pdl_wait();
  pdl_trigger();
  if (desc_skipped(d)) return;
  __shared__ float gh[8][32], gl[8][32];
  const long long MN = static_cast<long long>(d.M) * d.N;
  const long long total = MN * d.B0 * d.B1;
  const float* part = reinterpret_cast<const float*>(d.partial);
  const float af = static_cast<float>(d.alpha), bf = static_cast<float>(d.beta);
  const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
  const int s_lo = static_cast<int>(static_cast<long long>(d.splits) * g / 8);
  const int s_hi = static_cast<int>(static_cast<long long>(d.splits) * (g + 1) / 8);
  const long long step = static_cast<long long>(d.B0) * d.B1 * MN;
  for (long long e0 = blockIdx.x * 32LL; e0 < total; e0 += gridDim.x * 32LL) {
    const long long e = e0 + lane;
    float sh = 0.f, sl = 0.f;
    if (e < total) {
      const float* pe = part + e;   // partial s of element e at part + s * step + e
      for (int sp0 = s_lo; sp0 < s_hi; sp0 += 8) {
        float xs[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) xs[q] = sp0 + q < s_hi ? pe[(sp0 + q) * step] : 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float x = xs[q];
          const float s = sh + x, bb = s - sh;
          sl += (sh - (s - bb)) + (x - bb);
          sh = s;
        }
      }
    }
    gh[g][lane] = sh;
    gl[g][lane] = sl;
    __syncthreads();
    if (g == 0 && e < total) {
      float th = 0.f, tl = 0.f;
      for (int q = 0; q < 8; ++q) {
        const float x = gh[q][lane];
        const float s = th + x, bb = s - th;
        tl += (th - (s - bb)) + (x - bb);
        th = s;
        tl += gl[q][lane];
      }
      const long long b = e / MN, r = e % MN;
      const int m = static_cast<int>(r / d.N), n = static_cast<int>(r % d.N);
      const int b0 = static_cast<int>(b % d.B0), b1 = static_cast<int>(b / d.B0);
      const long long ce =
          b0 * d.sc_b0 + static_cast<long long>(b1) * d.sc_b1 + m * d.sc_m + n * d.sc_n;
      store_out(d, ce, th + tl, af, bf);
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------------------
// TMA-fed, warp-specialised variant for the TF32 modes with FP32 operands
// whose K index or MN index is contiguous (every full-layer product of the
// sweep).  Per CTA one 128 x BN output tile and a ring of S stages; a stage
// holds the raw FP32 tiles of A (128 x 32) and B (BN x 32), loaded by TMA
// (SWIZZLE_128B: the K-major canonical layout of the MMA; an MN-contiguous
// operand arrives as 32 x 32 boxes and is transposed), converted in place to
// TF32 heads by four converter warps, which also write the tails of the
// split form; one thread issues the tcgen05.mma of the stage and commits its
// completion to the stage's "empty" barrier, which frees it for the next TMA.
//   warp 0: TMA producer (one thread)       warp 1: TMEM owner, MMA issuer
//   warps 2-5: converters, then the epilogue (TMEM lanes 32 (w % 4) ..)
// Every wait is bounded; an expired wait raises the error flag and the CTA's
// abort flag, every role then stops, the producer waits (bounded) for the
// copies it issued, the MMA thread commits so that the epilogue can wait for
// its MMAs, and TMEM is freed.
// ---------------------------------------------------------------------------

int tc_total_tiles(const GemmDesc& d, int BK);

constexpr int kTThreads = 192;
constexpr int kTConv = 128;
constexpr int kTSmem = 196608;           // bytes of the stage ring, one CTA per SM
constexpr int kTSmem2 = 98304;           // two CTAs per SM

struct TmaParams {
  CUtensorMap a[kMaxGroups];
  CUtensorMap b[kMaxGroups];
  int a_mn[kMaxGroups], b_mn[kMaxGroups];     // 1: MN index contiguous (transposed boxes)
  int a_use[kMaxGroups], b_use[kMaxGroups];   // bit i: map dim i is a real index (else coordinate 0)
  int total_tiles;
  int* err;
};

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait that also gives up once another role of the CTA has aborted.
__device__ __forceinline__ bool mbar_wait_ab(uint64_t* bar, uint32_t parity,
                                             const volatile int* abort_flag) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                          int c2, int c3, int c4, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// Named barrier of the four converter warps (id 1), with an AND vote.
__device__ __forceinline__ bool conv_vote(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, 128, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(v))
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// TF32 head and tail of four FP32 values (head rounded to nearest).
template <bool kSplit>
__device__ __forceinline__ void split4(const float* x, uint4& h, uint4& l) {
  uint32_t hh[4], ll[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    hh[q] = tf32_bits(x[q]);
    ll[q] = kSplit ? tf32_bits(x[q] - __uint_as_float(hh[q])) : 0u;
  }
  h = make_uint4(hh[0], hh[1], hh[2], hh[3]);
  l = make_uint4(ll[0], ll[1], ll[2], ll[3]);
}

// A K-major raw tile of ROWS rows is already in the MMA layout: heads in
// place, tails at the same offsets of the tail tile.
template <bool kSplit, int ROWS>
__device__ __forceinline__ void convert_kmajor(uint8_t* hi, uint8_t* lo, int ct) {
  constexpr int kChunks = ROWS * 128 / 16;
#pragma unroll 4
  for (int i = ct; i < kChunks; i += kTConv) {
    const float4 v = *reinterpret_cast<const float4*>(hi + 16 * i);
    const float x[4] = {v.x, v.y, v.z, v.w};
    uint4 h, l;
    split4<kSplit>(x, h, l);
    *reinterpret_cast<uint4*>(hi + 16 * i) = h;
    if constexpr (kSplit) *reinterpret_cast<uint4*>(lo + 16 * i) = l;
  }
}

// An MN-contiguous operand arrives as ROWS / 32 boxes of 32 K rows x 32 MN
// values (box j at hi + 4096 j, row k at 128 k, 16-byte chunk c stored at
// c ^ (k & 7)).  Converter thread ct owns MN row ct: it reads its 32 values,
// all converter threads meet, and it writes the row in the K-major layout.
template <bool kSplit, int ROWS>
__device__ __forceinline__ void convert_mnmajor(uint8_t* hi, uint8_t* lo, int ct) {
  float v[32];
  const bool active = ct < ROWS;
  if (active) {
    const int j = ct >> 5, c = (ct & 31) >> 2, e = ct & 3;
    const uint8_t* box = hi + 4096 * j;
#pragma unroll
    for (int k = 0; k < 32; ++k)
      v[k] = *reinterpret_cast<const float*>(box + 128 * k + ((c ^ (k & 7)) << 4) + 4 * e);
  }
  conv_sync();
  if (active) {
#pragma unroll
    for (int kc = 0; kc < 8; ++kc) {
      uint4 h, l;
      split4<kSplit>(v + 4 * kc, h, l);
      const int off = 128 * ct + ((kc ^ (ct & 7)) << 4);
      *reinterpret_cast<uint4*>(hi + off) = h;
      if constexpr (kSplit) *reinterpret_cast<uint4*>(lo + off) = l;
    }
  }
}

// 16 accumulators of row m, columns n..n+15, to C (or the split-K partials),
// with vector stores where the row is contiguous and aligned.
__device__ __forceinline__ void store_row16(const GemmDesc& d, int b, int b0, int b1, int split_id,
                                            int m, int n, const uint32_t* r, float af, float bf) {
  const bool full = n + 16 <= d.N;
  if (d.splits > 1) {
    float* P = reinterpret_cast<float*>(d.partial) +
               (static_cast<long long>(split_id) * d.B0 * d.B1 + b) * static_cast<long long>(d.M) * d.N +
               static_cast<long long>(m) * d.N + n;
    if (full && (reinterpret_cast<uintptr_t>(P) & 15) == 0) {
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(P + j) =
            make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                        __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
    } else {
      for (int j = 0; j < 16 && n + j < d.N; ++j) P[j] = __uint_as_float(r[j]);
    }
    return;
  }
  const long long cb = b0 * d.sc_b0 + static_cast<long long>(b1) * d.sc_b1 + m * d.sc_m;
  if (full && d.sc_n == 1 && d.beta == 0.0) {
    if (d.c_f32) {
      float* C = static_cast<float*>(d.C) + cb + n;
      if ((reinterpret_cast<uintptr_t>(C) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4*>(C + j) =
              make_float4(af * __uint_as_float(r[j]), af * __uint_as_float(r[j + 1]),
                          af * __uint_as_float(r[j + 2]), af * __uint_as_float(r[j + 3]));
        return;
      }
    } else {
      double* C = static_cast<double*>(d.C) + cb + n;
      if ((reinterpret_cast<uintptr_t>(C) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < 16; j += 2)
          *reinterpret_cast<double2*>(C + j) =
              make_double2(f32_to_f64(af * __uint_as_float(r[j])),
                           f32_to_f64(af * __uint_as_float(r[j + 1])));
        return;
      }
    }
  }
  for (int j = 0; j < 16; ++j)
    if (n + j < d.N) store_out(d, cb + static_cast<long long>(n + j) * d.sc_n, __uint_as_float(r[j]), af, bf);
}

template <bool kSplit, int BN, int kRing>
__global__ void __launch_bounds__(kTThreads, kRing == kTSmem ? 1 : 2)
    gemm_tma_kernel(const GemmDesc d, const __grid_constant__ TmaParams tp) {
  pdl_wait();
  pdl_trigger();
  constexpr int kA = kBM * 128;                     // raw A tile: 128 rows x 32 FP32
  constexpr int kB = BN * 128;
  constexpr int kHi = kA + kB;                      // raw tiles, TF32 heads after conversion
  constexpr int kStageBytes = (kSplit ? 2 : 1) * kHi;
  constexpr int S = kRing / kStageBytes < 8 ? kRing / kStageBytes : 8;
  constexpr uint32_t kIdesc = instr_desc(2u, kBM, BN);
  static_assert(S >= 2, "stage ring");
  static_assert(BN == 64 || BN == 128, "tile width");

  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full_bar[S], conv_bar[S], empty_bar[S], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;

  if (desc_skipped(d)) return;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_n = (d.N + BN - 1) / BN;
  const int tm = blockIdx.x / tiles_n, tn = blockIdx.x % tiles_n;
  const int b = blockIdx.y;
  const int b0 = b % d.B0, b1 = b / d.B0;
  const int split_id = blockIdx.z;
  const int m0 = tm * kBM, n0 = tn * BN;
  const int t_lo = static_cast<int>(static_cast<long long>(tp.total_tiles) * split_id / d.splits);
  const int t_hi =
      static_cast<int>(static_cast<long long>(tp.total_tiles) * (split_id + 1) / d.splits);
  const int nk = t_hi - t_lo;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full_bar[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&conv_bar[s])),
                   "r"(kTConv));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done_bar)));
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;
  volatile int* abort_v = &abort_flag;

  if (warp == 0) {
    if (lane == 0 && nk > 0) {
      // ---- TMA producer ----
      for (int g = 0; g < d.ngroups; ++g) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tp.a[g])) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tp.b[g])) : "memory");
      }
      int kt = 0, t_global = 0;
      bool ok = true;
      for (int g = 0; g < d.ngroups && t_global < t_hi && ok; ++g) {
        const Group& G = d.g[g];
        const int nt = G.K / 32;
        if (t_global + nt <= t_lo) { t_global += nt; continue; }
        const int first = max(0, t_lo - t_global), last = min(nt, t_hi - t_global);
        const int k0m = (1 << G.k0_log2) - 1;
        const int ua = tp.a_use[g], ub = tp.b_use[g];
        for (int t = first; t < last; ++t) {
          const int s = kt % S, u = kt / S;
          if (u > 0 && !mbar_wait_ab(&empty_bar[s], (u - 1) & 1, abort_v)) { ok = false; break; }
          const uint32_t st = smem_u32(smem + s * kStageBytes);
          const uint32_t fb = smem_u32(&full_bar[s]);
          mbar_expect_tx(&full_bar[s], kHi);
          const int kb = t * 32;
          const int k0 = kb & k0m, k1 = kb >> G.k0_log2;
          const int a2 = (ua & 4) ? k1 : 0, a3 = (ua & 8) ? b0 : 0, a4 = (ua & 16) ? b1 : 0;
          const int c2 = (ub & 4) ? k1 : 0, c3 = (ub & 8) ? b0 : 0, c4 = (ub & 16) ? b1 : 0;
          if (!tp.a_mn[g]) {
            tma_load5(st, &tp.a[g], k0, m0, a2, a3, a4, fb);
          } else {
#pragma unroll
            for (int j = 0; j < kBM / 32; ++j) tma_load5(st + 4096 * j, &tp.a[g], m0 + 32 * j, k0, a2, a3, a4, fb);
          }
          if (!tp.b_mn[g]) {
            tma_load5(st + kA, &tp.b[g], k0, n0, c2, c3, c4, fb);
          } else {
#pragma unroll
            for (int j = 0; j < BN / 32; ++j) tma_load5(st + kA + 4096 * j, &tp.b[g], n0 + 32 * j, k0, c2, c3, c4, fb);
          }
          ++kt;
        }
        t_global += nt;
      }
      if (!ok) {
        *abort_v = 1;
        if (tp.err) atomicOr(tp.err, 1);
      }
      // the copies of the last use of every stage must land before the CTA exits
      for (int q = max(0, kt - S); q < kt; ++q) mbar_wait(&full_bar[q % S], (q / S) & 1);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      bool ok = true;
      for (int kt = 0; kt < nk; ++kt) {
        const int s = kt % S, u = kt / S;
        if (!mbar_wait_ab(&conv_bar[s], u & 1, abort_v)) { ok = false; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a_hi = smem_u32(smem + s * kStageBytes);
        const uint32_t b_hi = a_hi + kA;
        const uint32_t a_lo = a_hi + kHi, b_lo = a_lo + kA;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const uint32_t off = j * 32;   // 8 TF32 values of K per instruction
          const uint32_t acc = (kt > 0 || j > 0) ? 1u : 0u;
          if constexpr (kSplit) {
            mma<false>(tmem, smem_desc(a_lo + off), smem_desc(b_hi + off), kIdesc, acc);
            mma<false>(tmem, smem_desc(a_hi + off), smem_desc(b_lo + off), kIdesc, 1u);
            mma<false>(tmem, smem_desc(a_hi + off), smem_desc(b_hi + off), kIdesc, 1u);
          } else {
            mma<false>(tmem, smem_desc(a_hi + off), smem_desc(b_hi + off), kIdesc, acc);
          }
        }
        mma_commit(&empty_bar[s]);
      }
      if (!ok) {
        *abort_v = 1;
        if (tp.err) atomicOr(tp.err, 1);
      }
      mma_commit(&done_bar);   // arrives once every MMA issued above is complete
    }
  } else {
    // ---- converters ----
    const int ct = threadIdx.x - 64;
    bool ok = true;
    int kt = 0, t_global = 0;
    for (int g = 0; g < d.ngroups && t_global < t_hi && ok; ++g) {
      const Group& G = d.g[g];
      const int nt = G.K / 32;
      if (t_global + nt <= t_lo) { t_global += nt; continue; }
      const int first = max(0, t_lo - t_global), last = min(nt, t_hi - t_global);
      const bool amn = tp.a_mn[g] != 0, bmn = tp.b_mn[g] != 0;
      for (int t = first; t < last; ++t) {
        const int s = kt % S, u = kt / S;
        // all converter threads take the same decision (their named barriers follow)
        if (!conv_vote(mbar_wait_ab(&full_bar[s], u & 1, abort_v))) { ok = false; break; }
        uint8_t* st = smem + s * kStageBytes;
        if (amn) convert_mnmajor<kSplit, kBM>(st, st + kHi, ct);
        else convert_kmajor<kSplit, kBM>(st, st + kHi, ct);
        if (bmn) convert_mnmajor<kSplit, BN>(st + kA, st + kHi + kA, ct);
        else convert_kmajor<kSplit, BN>(st + kA, st + kHi + kA, ct);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv_bar[s]);
        ++kt;
      }
      t_global += nt;
    }
    if (!ok) {
      *abort_v = 1;
      if (tp.err && ct == 0) atomicOr(tp.err, 1);
    }
    // ---- epilogue: wait for the MMAs (also after an abort), then TMEM -> C ----
    const bool done = mbar_wait(&done_bar, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // one decision per warp: tcgen05.ld is a warp-collective instruction
    if (__all_sync(0xffffffffu, done && !*abort_v)) {
      const int quarter = warp & 3;
      const int row = quarter * 32 + lane;
      const int m = m0 + row;
      const float af = static_cast<float>(d.alpha), bf = static_cast<float>(d.beta);
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        if (nk == 0) {
#pragma unroll
          for (int j = 0; j < 16; ++j) r[j] = 0u;
        } else {
          const uint32_t taddr = tmem + (static_cast<uint32_t>(quarter * 32) << 16) + c0;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        }
        if (m < d.M && n0 + c0 < d.N) store_row16(d, b, b0, b1, split_id, m, n0 + c0, r, af, bf);
      }
    } else if (!done && tp.err && ct == 0) {
      atomicOr(tp.err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
}

template <bool kSplit, int BN, int kRing>
void tma_configure() {
  cudaFuncSetAttribute(gemm_tma_kernel<kSplit, BN, kRing>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, kRing + 1024);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

// Layout of one operand for the TMA kernel: FP32, K0 a multiple of 32 (a K
// tile never straddles two K1 slices), K or MN index contiguous, every other
// stride a multiple of 16 bytes, 16-byte aligned base.  Arithmetic only, so
// that the split count of a product is the same when it is planned and run.
bool tma_operand_ok(const Operand& o, int k0_log2) {
  if (!o.f32 || k0_log2 < 5) return false;
  if ((reinterpret_cast<uintptr_t>(o.p) & 15) != 0) return false;
  const bool kmaj = o.s_k0 == 1, mnmaj = o.s_mn == 1;
  if (!kmaj && !mnmaj) return false;
  const long long other = kmaj ? o.s_mn : o.s_k0;
  if (other <= 0 || (other & 3)) return false;
  const long long rest[3] = {o.s_k1, o.s_b0, o.s_b1};
  for (long long r : rest)
    if (r < 0 || (r & 3)) return false;
  return true;
}

bool tma_eligible(const GemmDesc& d) {
  if (d.prec != 1 && d.prec != 2) return false;
  for (int g = 0; g < d.ngroups; ++g)
    if (!tma_operand_ok(d.g[g].a, d.g[g].k0_log2) || !tma_operand_ok(d.g[g].b, d.g[g].k0_log2))
      return false;
  return d.ngroups > 0 && d.ngroups <= kMaxGroups;
}

int tma_bn(int N) { return N >= 128 ? 128 : 64; }

// Tensor map of one operand: dims (contiguous index, the other of K0 / MN,
// K1, B0, B1); an index of extent 1 or stride 0 (a broadcast) becomes a dummy
// dimension of extent 1 whose coordinate is 0 (bit clear in *use).
bool encode_operand(const Operand& o, int k0_log2, int K, int rows, int B0, int B1, int box_rows,
                    CUtensorMap* map, int* mn_major, int* use) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const long long K0 = 1LL << k0_log2, K1 = K >> k0_log2;
  const bool kmaj = o.s_k0 == 1;
  long long ext[5] = {kmaj ? K0 : rows, kmaj ? rows : K0, K1, B0, B1};
  long long str[5] = {1, kmaj ? o.s_mn : o.s_k0, o.s_k1, o.s_b0, o.s_b1};
  *use = 0;
  cuuint64_t gdim[5], gstride[4];
  long long prev_bytes = 4, prev_ext = ext[0];
  gdim[0] = static_cast<cuuint64_t>(ext[0]);
  for (int i = 1; i < 5; ++i) {
    long long bytes;
    if (ext[i] > 1 && str[i] > 0) {
      *use |= 1 << i;
      bytes = str[i] * 4;
    } else {
      ext[i] = 1;
      bytes = prev_bytes * prev_ext;   // dummy: nested after the previous dimension
    }
    if (bytes % 16 != 0 || bytes >= (1LL << 40)) return false;
    gdim[i] = static_cast<cuuint64_t>(ext[i]);
    gstride[i - 1] = static_cast<cuuint64_t>(bytes);
    prev_bytes = bytes;
    prev_ext = ext[i];
  }
  const cuuint32_t box[5] = {32u, kmaj ? static_cast<cuuint32_t>(box_rows) : 32u, 1u, 1u, 1u};
  const cuuint32_t estr[5] = {1u, 1u, 1u, 1u, 1u};
  *mn_major = kmaj ? 0 : 1;
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<void*>(o.p), gdim, gstride, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Returns 1 (launched) or 0 (a tensor map could not be encoded: the caller
// runs the thread-staged kernel instead).
template <bool kSplit, int BN, int kRing>
int launch_tma(const GemmDesc& d, cudaStream_t s) {
  static TmaParams tp;   // host staging of the kernel parameter (launch copies it)
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  memset(&tp, 0, sizeof(tp));
  for (int g = 0; g < d.ngroups; ++g) {
    const Group& G = d.g[g];
    if (!encode_operand(G.a, G.k0_log2, G.K, d.M, d.B0, d.B1, kBM, &tp.a[g], &tp.a_mn[g], &tp.a_use[g]))
      return 0;
    if (!encode_operand(G.b, G.k0_log2, G.K, d.N, d.B0, d.B1, BN, &tp.b[g], &tp.b_mn[g], &tp.b_use[g]))
      return 0;
  }
  tp.total_tiles = tc_total_tiles(d, 32);
  tp.err = d.err;
  const int tiles = ((d.M + kBM - 1) / kBM) * ((d.N + BN - 1) / BN);
  dim3 grid(tiles, d.B0 * d.B1, d.splits);
  launch_k(gemm_tma_kernel<kSplit, BN, kRing>, grid, kTThreads, kRing + 1024, s, d, tp);
  return 1;
}

// d.occ == 2 selects the 96 KB ring (two CTAs per SM) where a stage still
// fits twice: BN = 64 in both forms, BN = 128 without the split.
int launch_tma_bn(const GemmDesc& d, cudaStream_t s) {
  const bool split = d.prec == 2;
  const int bn = (d.tile == 64 || d.tile == 128) ? d.tile : tma_bn(d.N);
  const bool two = d.occ == 2 && !(split && bn == 128);
  if (bn == 128) {
    if (split) return launch_tma<true, 128, kTSmem>(d, s);
    return two ? launch_tma<false, 128, kTSmem2>(d, s) : launch_tma<false, 128, kTSmem>(d, s);
  }
  if (split) return two ? launch_tma<true, 64, kTSmem2>(d, s) : launch_tma<true, 64, kTSmem>(d, s);
  return two ? launch_tma<false, 64, kTSmem2>(d, s) : launch_tma<false, 64, kTSmem>(d, s);
}

int tc_bn(int N) { return N >= 64 ? 64 : 32; }

int tc_total_tiles(const GemmDesc& d, int BK) {
  int t = 0;
  for (int g = 0; g < d.ngroups; ++g) t += (d.g[g].K + BK - 1) / BK;
  return t;
}

template <bool kBF16, bool kSplit, int BN>
int launch_tc(const GemmDesc& d, cudaStream_t s, int* err) {
  constexpr int BK = kBF16 ? 64 : 32;
  const int smem = tc_smem_bytes<kBF16, kSplit, BN>();
  const int tiles = ((d.M + kBM - 1) / kBM) * ((d.N + BN - 1) / BN);
  dim3 grid(tiles, d.B0 * d.B1, d.splits);
  TCParams tp{tc_total_tiles(d, BK), err};
  launch_k(gemm_tc_kernel<kBF16, kSplit, BN>, grid, kThreadsTC, smem, s, d, tp);
  return 1;
}

template <bool kBF16, bool kSplit>
int launch_tc_bn(const GemmDesc& d, cudaStream_t s, int* err) {
  switch ((d.tile == 32 || d.tile == 64 || d.tile == 128) ? d.tile : tc_bn(d.N)) {
    case 128: return launch_tc<kBF16, kSplit, 128>(d, s, err);
    case 64: return launch_tc<kBF16, kSplit, 64>(d, s, err);
    default: return launch_tc<kBF16, kSplit, 32>(d, s, err);
  }
}

}  // namespace

void gemm_tc_init() {
  tma_configure<false, 64, kTSmem>(); tma_configure<false, 128, kTSmem>();
  tma_configure<true, 64, kTSmem>(); tma_configure<true, 128, kTSmem>();
  tma_configure<false, 64, kTSmem2>(); tma_configure<false, 128, kTSmem2>();
  tma_configure<true, 64, kTSmem2>();
  tc_configure<false, false, 32>(); tc_configure<false, false, 64>(); tc_configure<false, false, 128>();
  tc_configure<false, true, 32>(); tc_configure<false, true, 64>(); tc_configure<false, true, 128>();
  tc_configure<true, false, 32>(); tc_configure<true, false, 64>(); tc_configure<true, false, 128>();
  tc_configure<true, true, 32>(); tc_configure<true, true, 64>(); tc_configure<true, true, 128>();
}

bool gemm_tma_eligible(const GemmDesc& d) { return tma_eligible(d); }

bool gemm_tc_supported(const GemmDesc& d) {
  if (d.prec == 0) return false;
  if (d.M < 64 || d.N < 32) return false;
  long long k = 0;
  for (int g = 0; g < d.ngroups; ++g) k += d.g[g].K;
  return k >= 32;
}

int tc_pick_splits(const GemmDesc& d) {
  const int BK = (d.prec == 3 || d.prec == 4) ? 64 : 32;
  const int bn = (d.tc_engine != 1 && tma_eligible(d)) ? tma_bn(d.N) : tc_bn(d.N);
  const long long base = static_cast<long long>((d.M + kBM - 1) / kBM) *
                         ((d.N + bn - 1) / bn) * d.B0 * d.B1;
  const int kt = tc_total_tiles(d, BK);
  const long long sms = device_sm_count();
  if (base >= sms || kt < 8) return 1;
  int s = static_cast<int>(std::min<long long>((sms + base - 1) / base, kt / 4));
  return std::max(1, std::min(s, 128));
}

int gemm_tc_launch(const GemmDesc& d, cudaStream_t s) {
  int n = 0;
  if (d.tc_engine != 1 && tma_eligible(d)) n = launch_tma_bn(d, s);
  if (n == 0)
  switch (d.prec) {
    case 1: n = launch_tc_bn<false, false>(d, s, d.err); break;
    case 2: n = launch_tc_bn<false, true>(d, s, d.err); break;
    case 3: n = launch_tc_bn<true, false>(d, s, d.err); break;
    default: n = launch_tc_bn<true, true>(d, s, d.err); break;
  }
  if (d.splits > 1) {
    const long long total = static_cast<long long>(d.M) * d.N * d.B0 * d.B1;
    const int blocks = static_cast<int>(std::min<long long>((total + 31) / 32, 8192));
    launch_k(splitk_reduce_tc, blocks, 256, 0, s, d);
    ++n;
  }
  return n;
}

}  // namespace ttn
