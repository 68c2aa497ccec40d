// Shared declarations of the TTN sweep kernels (device side and host side).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace ttn {

// Programmatic dependent launch.  launch_k() launches a kernel on stream s,
// with programmatic stream serialisation allowed when TTN_PDL=1 is set in the
// environment: the kernel's CTAs may then be scheduled while its predecessor
// in the stream still runs, hiding the launch gap between dependent kernels
// (also in a captured graph).  Off by default: on the headline sweep it
// measured 89.2 against 92.4 sweeps/s without it (the waiting CTAs hold SM
// slots that the concurrent graph branches would use).  Every kernel launched this way begins with
// pdl_wait() -- griddepcontrol.wait returns once the predecessor grids have
// completed and their memory is visible, so nothing is read or written
// before it -- and then pdl_trigger(), which lets its own successor be
// scheduled.  Both are no-ops for a kernel launched without the attribute.
// The cooperative kernels (Lanczos, polar composition) keep plain launches.
bool pdl_enabled();

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}
#endif

// One operand of a grouped, batched, strided matrix product.  Element (i, k)
// of batch (b0, b1) sits at p[i*s_mn + k0*s_k0 + k1*s_k1 + b0*s_b0 + b1*s_b1]
// with k0 = k mod K0, k1 = k div K0 (K0 a power of two).  i is the row for A
// and the column for B.  Two-level K and batch indices let one descriptor
// express every contraction of the sweep on tensors w[p][l][r] without
// materialising a permutation.
struct Operand {
  const void* p;     // FP64 data, or FP32 when f32 != 0
  long long s_mn, s_k0, s_k1, s_b0, s_b1;
  int f32;
};

struct Group {
  Operand a, b;
  int K;        // K0 * K1
  int k0_log2;  // log2 K0
};

constexpr int kMaxGroups = 32;   // the environment product has 1 + 4K groups: K <= 7

// C[b] = alpha * sum_g A_g[b] B_g[b] + beta * C[b] for every batch b = (b0, b1).
// The K ranges of the groups are concatenated into one reduction; `splits`
// cuts it into contiguous tile ranges whose partial sums are added in a fixed
// order by a second kernel (deterministic).
struct GemmDesc {
  int M, N, B0, B1;
  int ngroups;
  Group g[kMaxGroups];
  void* C;           // FP64 output, or FP32 when c_f32 != 0
  int c_f32;
  long long sc_m, sc_n, sc_b0, sc_b1;
  double alpha, beta;
  int splits;
  double* partial;   // splits * B0 * B1 * M * N doubles when splits > 1
  int prec;          // ttn_precision of the products
  const int* skip;   // if non-null and *skip != 0 the launch does nothing
  int skip_when_zero;  // with skip: the launch does nothing when *skip == 0 instead
  int* err;          // device flag raised when a bounded wait of a kernel expires
  int sym;           // C = A A^T (symmetric, M == N): only tiles on or above the
                     // diagonal are computed and mirrored (FP64 engine)
  int sym_tile;      // tile size the launcher used (set by the launcher)
  int tc_engine;     // tensor-core engine: 0 the TMA-fed kernel where the operand
                     // layouts allow it, 1 always the thread-staged kernel
  int tile;          // tile width chosen by the autotuner (0: the launcher's
                     // default): BN of a tensor-core kernel, the square tile of
                     // the FP64 engine
  int occ;           // TMA-fed kernel: 2 = the 96 KB stage ring (two CTAs per
                     // SM), else the 192 KB ring (one CTA per SM)
};
// passed by value as a kernel parameter (limit 32764 bytes)
static_assert(sizeof(GemmDesc) + 64 < 32764, "GemmDesc too large for a kernel parameter");

#ifdef __CUDACC__
// The device flag of a product says that its launches do nothing.
__device__ __forceinline__ bool desc_skipped(const GemmDesc& d) {
  return d.skip && ((*d.skip != 0) != (d.skip_when_zero != 0));
}
#endif

// Launch one grouped product on `stream` (FP64 CUDA-core kernel or tcgen05
// kernel by desc.prec).  Returns the number of kernel launches.
int gemm_launch(const GemmDesc& d, cudaStream_t stream);

// SM count of the current device (cached per device; 152 without a device).
int device_sm_count();

// Split count / partial-buffer size the launcher will use for a descriptor.
int gemm_pick_splits(const GemmDesc& d);
size_t gemm_partial_elems(const GemmDesc& d, int splits);

// Tensor-core path (gemm_tc.cu).
int gemm_tc_launch(const GemmDesc& d, cudaStream_t stream);
bool gemm_tc_supported(const GemmDesc& d);
// The TMA-fed kernel can run this product (TF32 modes, FP32 operands with a
// contiguous K or MN index, aligned strides).
bool gemm_tma_eligible(const GemmDesc& d);
int tc_pick_splits(const GemmDesc& d);
void gemm_tc_init();

// ---------------------------------------------------------------------------
// Small kernels (misc.cu).  All reductions are two-pass with fixed order.
// ---------------------------------------------------------------------------

// out[b] = sum_i x[b*stride + i] * y[b*stride + i] for b < nb, i < n.
// scratch: at least nb * kDotBlocks doubles.
constexpr int kDotBlocks = 256;
int batched_dot(const double* x, const double* y, long long n, long long stride, int nb,
                double* out, double* scratch, cudaStream_t s);

// Partial sums of <x_b, x_b> and <x_b, y_b> (batch b at offset b * stride, n
// elements) in one pass over x: scratch[b * kDotBlocks + i] and
// scratch[(nb + b) * kDotBlocks + i], i < kDotBlocks, each in the order of
// batched_dot (polar_start completes the two sums).
int dot_self_and_cross_partial(const double* x, const double* y, long long n, long long stride,
                               int nb, double* scratch, cudaStream_t s);

// Polar start: per batch b (P x N rows), with fro2 = |G|^2 and gw = <G, W>
// summed from the partial sums `part` of dot_self_and_cross_partial:
//   s = mu * sqrt(fro2);  X = (G - s W) / sqrt(fro2 - 2 s gw + s^2 P).
// zero (may be null): set to 0 by the launch (a flag that later kernels OR into).
// With xh, xl (one batch only) X is written as FP32 pairs for the double-float
// products instead (xh = fl32(X), xl = fl32(X - xh); X itself is not written).
// With try_first (device, may be null): *run_full = (*try_first == 0).
// zero2 (may be null): set to 0 as well.
int polar_start(const double* G, const double* W, double* X, long long elems, int nb,
                int P, double mu, const double* part, cudaStream_t s, float* xh = nullptr,
                float* xl = nullptr, int* zero = nullptr, const int* try_first = nullptr,
                int* run_full = nullptr, int* zero2 = nullptr);

// For one P x P matrix A: (ph, pl) = FP32 pair of a I - c A (a = 0, c = -1:
// of A itself, as df_split), with flag: flag |= 1 when max |A - I| > thr, and
// with d32: d32 = fl32(0.5 (I - A)).
int check_split(const double* A, int P, double a, double c, float* ph, float* pl, double thr,
                int* flag, cudaStream_t s, float* d32 = nullptr);

// Pm[b] = a I - c A[b] (P x P), nb batches.
int poly_step_matrix(const double* A, double* Pm, int P, int nb, double a, double c,
                     cudaStream_t s);

// F[b] = I (P x P).
int set_identity(double* F, int P, int nb, cudaStream_t s);

// y = alpha * x + beta * y over n elements.
int axpby(const double* x, double* y, long long n, double alpha, double beta, cudaStream_t s);
// y = alpha * (*sel ? x1 : x0 + corr) over n elements (sel on the device; corr,
// FP32, may be null); with y32 also its FP32 copy (as to_f32).  With pred
// (device: try_first = pred[0], run_full = pred[pstride], count =
// pred[2 pstride]) also the next prediction of the polar schedule: try_first
// becomes 0 when this sweep's first try failed (run_full set), and 1 again
// after `retry` sweeps.  With sel2 (device, may be null), the *sel branch is
// itself a choice: x2 when *sel2, else x1 + corr.
int scale_select(const double* x0, const double* x1, const int* sel, double* y, long long n,
                 double alpha, cudaStream_t s, float* y32 = nullptr,
                 const float* corr = nullptr, int* pred = nullptr, int pstride = 0,
                 int retry = 0, const double* x2 = nullptr, const int* sel2 = nullptr);

// Symmetrise P x P blocks in place: A = (A + A^T) / 2.
int symmetrize(double* A, int P, int nb, cudaStream_t s);

// Sum of `count` doubles in a fixed order into *out (single block).
int ordered_sum(const double* x, int count, double* out, double scale, double add,
                cudaStream_t s);

// Identity bookkeeping of the one-site operators (exact FP64 scalars):
// for node J (P x P block at O + J*stride): tr = trace/P, O -= tr I,
// e_out[J] = e_in[left] + e_in[right] + tr, where left/right = 2J, 2J+1 when
// per_node, else both 0.
int split_identity(double* O, long long stride, int P, int nodes, const double* e_in,
                   int per_node, double* e_out, cudaStream_t s);
// Z_J += coef * (e_in[left] + e_in[right]) * W_J for each node J (elems each);
// Z and W are FP32 when f32 != 0, else FP64.
int add_identity_part(void* Z, const void* W, int f32, long long elems, int nodes,
                      const double* e_in, int per_node, double coef, cudaStream_t s);
// out = 2 (w + (e[0] + e[per_node ? 1 : 0]) v): dE/dv with w = H_top v of the
// identity-free operators.
int top_grad(double* out, const double* w, const double* v, long long n, const double* e,
             int per_node, cudaStream_t s);
// y = sign * x / sqrt(nrm2[0]).
int scale_normalise(const double* x, double* y, long long n, const double* nrm2, double sign,
                    cudaStream_t s);
// *out = dot[0] + (e[0] + e[per_node ? 1 : 0]) * vv[0] + add: the energy
// <v, H_top v> + cL with the identity part of the top operators restored.
int top_energy_sum(const double* dot, const double* vv, const double* e, int per_node, double add,
                   double* out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Polar composition (polar.cu): one block of scaled Newton-Schulz steps on the
// P x P level, F = prod_j p_j(A_j) from the Gram matrix A_0, in one
// cooperative launch.  A0 holds A_0 on entry (exactly symmetric); A0, A1, T
// and S are overwritten; F receives the composed polynomial.  Each of the five
// buffers holds NJ P x P blocks.  bar is a device counter the launcher zeroes;
// err is raised (|= 2) if a grid barrier wait expires.
// ---------------------------------------------------------------------------
constexpr int kMaxComposeSteps = 64;
// row or column blocks of 8 of a composition (P <= 256)
constexpr int kComposeMaxTiles = 32;
struct ComposeArgs {
  double* A0;
  double* A1;
  double* F;
  double* T;
  double* S;
  int P, NJ, nsteps;
  double alpha[kMaxComposeSteps], beta[kMaxComposeSteps];
  unsigned* bar;    // FP64 kernel: grid-barrier counter (zeroed by polar_compose)
  // double-float kernel: 3 * kComposeMaxTiles tile counters (zeroed by polar_compose)
  unsigned* cnt;
  int* err;
  int grid_share;   // concurrent streams sharing the GPU: the grid takes 1/grid_share of it
  int max_spin;     // polls of a grid-barrier wait before it expires (<= 0: 2^21, ~1 s)
  // double-float kernel only (may be null): when *shortcut is 0 the kernel
  // returns at once (the block is then one Newton-Schulz step, corrected on
  // the tensor cores)
  const int* shortcut = nullptr;
};
bool compose_supported(int P, int nsteps);

// The whole polar factor of a small layer in one CTA (mixed modes): every
// block of the schedule -- Gram matrix, composed steps, apply -- on FP32 pairs
// in shared memory.  X (P x N, FP64) is the damped, normalised start; W =
// sign * result (FP64) and, with W32, its FP32 copy.  block_end[b] is one past
// the last step of block b.
constexpr int kSmallPolarMaxP = 32, kSmallPolarMaxBlocks = 16;
struct SmallPolarArgs {
  const double* X;
  double* W;
  float* W32;
  int P, N, nblocks;
  int block_end[kSmallPolarMaxBlocks];
  double alpha[kMaxComposeSteps], beta[kMaxComposeSteps];
  double sign;
};
bool small_polar_supported(int P, long long N, int nblocks, int nsteps);
int small_polar(const SmallPolarArgs& a, cudaStream_t s);
// Flops the composition kernel executes (all tiles of every product).
double compose_flops(int P, int NJ, int nsteps);
// Returns the number of kernel launches (1), or -1 if the launch was refused.
// df: the five buffers hold FP32 pairs (hi at p, lo at p + P*P floats; block b
// at p + 2*b*P*P floats) and the products run in double-float arithmetic.
int polar_compose(const ComposeArgs& a, cudaStream_t s, bool df = false);

// ---------------------------------------------------------------------------
// Top solve (lanczos.cu): restarted FP64 Lanczos for the lowest eigenvector of
// the top Hamiltonian in one cooperative launch.  V (c x c) holds the start
// vector on entry and the normalised eigenvector on exit, sign-aligned with
// the start (copied to Vprev).  Scratch: basis (m+1) c^2, w c^2, Y 2K c^2,
// part grid*(m+2), coef 2(m+2), alpha, beta, y (m+2 each), scal (4),
// flags[0] = converged, flags[1] = tridiagonal size.  err |= 4 when a grid
// barrier wait expires.
// ---------------------------------------------------------------------------
constexpr int kLMaxM = 120;
constexpr int kLMaxGrid = 512;
struct LanczosArgs {
  const double* s0;   // [o, A_1..A_K, B_1..B_K] of the left top site, c x c each
  const double* s1;   // the same of the right top site
  double* V;
  double* Vprev;
  double* basis;
  double* w;
  double* Y;
  double* part;
  double* coef;
  double* alpha;
  double* beta;
  double* y;
  double* scal;
  int* flags;
  int c, K, m, restarts;
  double tol;
  unsigned* bar;      // grid-barrier counter (zeroed by lanczos_launch)
  int* err;
  int max_spin;       // polls of a grid-barrier wait before it expires (<= 0: 2^21, ~1 s)
  // double-float matrix-vector products (mixed modes): df != 0 and pair
  // buffers (each matrix or vector: n hi floats, then n lo floats) for the
  // operators of both top sites ((1+2K) matrices each; s1p unused when s1 ==
  // s0), the basis (m+1 vectors) and Y (2K matrices)
  int df;
  float* s0p;
  float* s1p;
  float* bp;
  float* Yp;
  // set by lanczos_launch: the double-float matrix-vector phases stage all
  // operand tiles of a phase at once (asynchronous copies into shared memory)
  int wide = 0;
};
bool lanczos_supported(int c, int m);
// CTAs of the launch for top dimension c when grid_share streams share the GPU.
int lanczos_grid(int c, int grid_share);
// Returns the number of kernel launches (1), or -1 if the launch was refused.
int lanczos_launch(const LanczosArgs& a, int grid, cudaStream_t s);

// ---------------------------------------------------------------------------
// Double-float products (gemm_df.cu): FP64 values held as FP32 pairs
// (hi + lo), products accumulated in FP32 pairs on the FP32 pipes (~48
// significant bits).  Used for the polar factor of the mixed modes.
// ---------------------------------------------------------------------------
// hi[i] = fl32(x[i]), lo[i] = fl32(x[i] - hi[i])
int df_split(const double* x, float* hi, float* lo, long long n, cudaStream_t s);
// Split count of df_gram (its partial buffer holds splits * P * P doubles).
int df_gram_splits(int P, int n2);
// Multiply-adds x 2 of the tiles df_gram computes (upper triangle only).
double df_gram_flops(int P, long long n2);
// The check_split pass over a Gram matrix, folded into the product's split-K
// reduction: (ph, pl) = pair of a I - c C, flag |= 1 when max |C - I| > thr
// (flag may be null), d32 = fl32(0.5 (I - C)) (may be null).
struct GramCheck {
  double a = 0.0, c = -1.0;
  float* ph = nullptr;
  float* pl = nullptr;
  double thr = 0.0;
  int* flag = nullptr;
  float* d32 = nullptr;
  double thr2 = 0.0;     // flag2 |= 1 when max |C - I| > thr2 (flag2 may be null)
  int* flag2 = nullptr;
};
// C (P x P, FP64) = X X^T for X (P x n2, row-major) given as (Xh, Xl).
// run_if (device, may be null): when it points to 0 the launches return at once.
// chk (may be null): also the check_split pass over C, with the same results
// (one launch fewer when the product is split over K).
int df_gram(const float* Xh, const float* Xl, int P, long long n2, double* C, double* part,
            cudaStream_t s, const int* run_if = nullptr, const GramCheck* chk = nullptr);
// C (P x n2, FP64) = F X for F (P x P) given as (Fh, Fl) and X as (Xh, Xl);
// with Ch, Cl also the normalised FP32 pair of C (the same as splitting C).
int df_apply(const float* Fh, const float* Fl, const float* Xh, const float* Xl, int P,
             long long n2, double* C, cudaStream_t s, const int* run_if = nullptr,
             float* Ch = nullptr, float* Cl = nullptr);
// Energy change per spin after a sweep (Sec. IV convergence test): dstat =
// [previous energy, change per spin, tolerance], istat[2] = converged,
// istat[3] = sweeps seen (the first is compared with nothing).
int sweep_delta(const double* E, double* dstat, int* istat, double inv_spins, cudaStream_t s);

// dst[i] = (float) src[i]
int to_f32(const double* src, float* dst, long long n, cudaStream_t s);
// dst[i] = src ? src[i] : value for i < n.
int store_ints(int* dst, const int* src, int n, int value, cudaStream_t s);
// One CTA: out = [sum of traces, max |M - I| (or |M|), max |M - M^T|] over nb
// n x n blocks at M + b * stride.
int mat_stats(const double* M, int n, int nb, long long stride, int sub_identity, double* out,
              cudaStream_t s);

// NaN/Inf scan: flag[0] |= 1 if any element is not finite.
int finite_check(const double* x, long long n, int* flag, cudaStream_t s);

}  // namespace ttn
