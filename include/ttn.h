/*
 * ttn.h -- C ABI of the GB300 tree-tensor-network (TTN) sweep library.
 *
 * The library optimises a regular binary TTN (arXiv 1905.01331, Sec. II.C,
 * Fig. 1d) for the ground state of a periodic chain of L effective sites, or of
 * an Lx x Ly thin torus seen as a chain of Lx columns of dimension d^Ly
 * (Sec. II.B).  The Hamiltonian is given as one-site and product terms,
 *     H = sum_m [ o_m + sum_{k<K} A_k,m B_k,m+1 ],
 * whose bond index has dimension K instead of chi (Fig. 2b), so that every
 * contraction of the sweep costs O(chi^4) (Sec. III.A, Sec. V).
 *
 * Conventions for every entry point:
 *  - Return value: a ttn_status (0 on success, negative on error).  Nothing
 *    aborts or throws across the ABI; ttn_last_error() describes the last
 *    failure of a context.
 *  - Host buffers belong to the caller; the library copies from/to them and
 *    keeps no pointer to them after the call returns.
 *  - Device memory: one caller-owned workspace (device pointer + size) given
 *    to ttn_create; the library carves all its tensors out of it and never
 *    allocates device memory itself.  The workspace must stay allocated and
 *    unused by the caller until ttn_destroy.
 *  - Stream: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  The library enqueues its kernels on non-blocking streams of its
 *    own, created by ttn_create (one per concurrent instance lane), and fences
 *    them to `stream` with events: a call's work starts after everything
 *    enqueued on `stream` before the call, and `stream` waits for that work,
 *    so it behaves as if enqueued on `stream`.  Calls that return host values
 *    synchronise the library's streams only.
 *  - Layouts are row-major C order.  An isometry of layer t is w[p][l][r]
 *    with parent p < chi_{t+1} and children l, r < chi_t (Eq. (constraint)
 *    reads sum_{l,r} w[p][l][r] w[p'][l][r] = delta_{p p'}); the top tensor is
 *    v[a][b], chi_T x chi_T (Eq. (normalization)).
 *  - Bond dimensions: chi_0 = d^Ly and chi_{t+1} = min(chi, chi_t^2) for
 *    t = 0..T-1, T = log2(Lx) - 1; Lx must be a power of two >= 4.
 */
#ifndef TTN_H
#define TTN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ttn_ctx* ttn_t;

typedef enum {
  TTN_OK = 0,
  TTN_EINVAL = -1,    /* bad argument or shape */
  TTN_ENOMEM = -2,    /* workspace too small */
  TTN_ECUDA = -3,     /* a CUDA call failed */
  TTN_ENOCONV = -4,   /* top eigensolver or polar iteration did not converge */
  TTN_ETIMEOUT = -5,  /* a bounded device wait expired */
  TTN_ENAN = -6       /* NaN or Inf met in an input or a result */
} ttn_status;

/* Arithmetic of the O(chi^4) contractions (ascend, environment, descend).
 * The polar update's final isometry condition, the top eigenproblem and all
 * energies are FP64 in every mode. */
typedef enum {
  TTN_FP64 = 0,     /* plain FP64 on the CUDA cores */
  TTN_TF32 = 1,     /* tcgen05 kind::tf32, FP32 accumulation */
  TTN_TF32X3 = 2,   /* three TF32 products (hi*hi + hi*lo + lo*hi) */
  TTN_BF16 = 3,     /* tcgen05 kind::f16 with bf16 operands */
  TTN_BF16X3 = 4    /* three bf16 products */
} ttn_precision;

/* One Hamiltonian.  onesite: d0 x d0, A and B: K x d0 x d0, d0 = d^Ly, all
 * host FP64, row-major; the library copies them in ttn_create.  Lx and d0
 * powers of two, d0 <= 4096, 1 <= K <= 7 product terms per bond. */
typedef struct {
  int Lx, Ly, d, chi, K;
  int per_node;             /* 0: one isometry per layer (translation
                               invariant, Sec. III); 1: one per node */
  const double* onesite;
  const double* A;
  const double* B;
} ttn_problem;

typedef struct {
  int prec;                 /* ttn_precision */
  int top_mode;             /* 0: lowest eigenvector of the top Hamiltonian;
                               1: v <- -H_top v / |H_top v| (minus the polar
                               factor of v's environment, the literal reading
                               of "updated similarly", Sec. III.B) */
  double lanczos_tol;       /* residual |Hv - Ev| <= tol * |E|; 0 (default): 1e-13 in
                               FP64 mode, 1e-8 in the mixed modes (whose top
                               operators carry 1e-6 to 3e-5 of tensor-core
                               rounding) */
  int lanczos_max;          /* Krylov dimension per restart (default 48) */
  int lanczos_restarts;     /* restarts per sweep (default 3) */
  double shift;             /* bond shift c; NaN = lambda_max of the bond term */
  double polar_damping;     /* proximal weight mu of the update (default 1e-7) */
  int deterministic;        /* 1: fixed-order reductions (always on) */
  int use_graph;            /* 1: capture a sweep as a CUDA graph and replay */
  int persistent;           /* bit 0: the P x P Newton-Schulz composition of each
                               polar block, bit 1: the Lanczos top solve, as one
                               persistent cooperative kernel each (all SMs, grid
                               barriers with bounded waits); a clear bit runs
                               that step as separate launches.  Default 3 */
  int streams;              /* instances run on min(streams, instances) concurrent
                               streams (graph branches), each with its own
                               scratch; default 8 */
  int polar_blocks;         /* Newton-Schulz schedule of the polar factor: 1 = a
                               fresh Gram matrix every <= 4 steps (accurate to
                               FP64 rounding), 2 = two long blocks (one Gram
                               matrix per ~1e5 of growth: half the FP64 work),
                               0 (default) = 1 in FP64 mode; in the mixed modes
                               1 for layers with chi_{t+1} < 32 and otherwise
                               an adaptive double-float schedule: block 1
                               converges every singular value above 1e-5 of
                               |X|_F; when it leaves max |X X^T - I| <= 1e-9,
                               block 2 becomes one Newton-Schulz step and the
                               final step is skipped (decided on the device),
                               else block 2 covers the worst case down to
                               min(mu / 4, 1e-10) and the final step runs;
                               before it, a layer predicted well conditioned
                               (on the device: its last try succeeded, or 16
                               sweeps passed since it failed) first tries a
                               short block for singular values above 1e-2;
                               when that leaves max |X X^T - I| <= 1e-9, one
                               Newton-Schulz step ends the factor and the
                               schedule above does not run, else it runs from
                               the same start;
                               3 = as 0 with the fixed double-float schedule
                               (two long blocks and the final step always);
                               4 = as 0 without the first try */
  int double_float;         /* mixed modes, 1 (default): the polar factor's products
                               (Gram matrices, composition, apply, plus one final
                               Newton-Schulz step: isometry to ~1e-14) and the
                               Lanczos top solve's matrix-vector products in
                               double-float arithmetic (FP32 pairs, ~48 bits) on
                               the FP32 pipes; 0: FP64 */
  int tc_engine;            /* tensor-core products: 0 (default) the TMA-fed,
                               warp-specialised kernel wherever the operand
                               layouts allow it (FP32, K or MN index contiguous;
                               TF32 modes), else the thread-staged kernel;
                               1: the thread-staged kernel for every product */
  int wait_polls;           /* polls of a grid-barrier wait in the persistent
                               kernels before it expires and the sweep reports
                               TTN_ETIMEOUT (0, the default: 2^21 polls, about
                               one second) */
  int stage_streams;        /* independent products of one sweep stage (the
                               one-leg products of an ascend or environment, the
                               products and traces of a descend) run
                               concurrently on this many sub-streams of each
                               lane (parallel branches of the captured graph),
                               each with its own split-K buffer; 1: one stream;
                               0 (default): 3 (the maximum) when the context has
                               one lane, one stream when several lanes already
                               run instances concurrently (on 64 chains, 8
                               lanes: 370 against 180 instance-sweeps/s with 3
                               sub-streams per lane) */
  int recompute_ops;        /* 1: keep the ascended operators of site layers
                               1..T-1 in two shared buffers and recompute them
                               (ascending from the bottom through the current
                               isometries) whenever the descent needs them:
                               (T-3) fewer operator buffers in the workspace for
                               O(T^2) instead of O(T) ascend steps per sweep or
                               gradient; 0 (default): store every layer's */
  const void* tiles;        /* autotuner blob from ttn_autotune (NULL: the
                               launchers' default tile widths and split counts);
                               copied by ttn_create */
  size_t tiles_bytes;
} ttn_options;

/* Fill *opt with the defaults above. */
void ttn_default_options(ttn_options* opt);

/* Bytes of device workspace that ttn_create needs for these problems. */
size_t ttn_workspace_bytes(const ttn_problem* probs, int n_problems, const ttn_options* opt);

/* Build a context for n_problems independent Hamiltonians advanced together
 * (step a0: operators uploaded, shift c computed on the host from the
 * d0^2 x d0^2 bond matrix).  Isometries start undefined: call
 * ttn_set_isometries for every instance before the first sweep. */
int ttn_create(ttn_t* out, const ttn_problem* probs, int n_problems, const ttn_options* opt,
               void* d_workspace, size_t workspace_bytes, void* stream);

/* Number of doubles of one instance's isometries (all layers, layer 0 first;
 * per node: node-major within a layer) and of its top tensor. */
int ttn_sizes(ttn_t h, int inst, size_t* n_w, size_t* n_v, int* n_layers);

/* Bond dimensions chi_0..chi_T of one instance (host array of n_layers+1). */
int ttn_chis(ttn_t h, int inst, int* chis);

/* Copy isometries (concatenated as ttn_sizes describes) and top tensor of
 * one instance into the context.  The pointers may be host or device memory
 * (unified addressing).  No check of the isometric constraint. */
int ttn_set_isometries(ttn_t h, int inst, const double* host_w_all, const double* host_v);

/* Copy one instance's current isometries and top tensor out (host or device
 * pointers; either may be NULL to skip it). */
int ttn_get_isometries(ttn_t h, int inst, double* host_w_all, double* host_v);

/* Run n_sweeps sweeps of every instance (Sec. III): ascend the Hamiltonian
 * through all layers, solve the top tensor, then for t = T-1..0 form the
 * environment of w_t, replace w_t by minus its polar factor and descend the
 * density matrices through the new w_t.  host_energy (may be NULL) receives
 * n_sweeps * n_problems doubles, sweep-major: the energy found by each top
 * solve, shift restored.
 * The call returns after the sweeps have run: it reads the device status
 * words of the context (and clears them once reported).  Status, most severe
 * first: TTN_ECUDA; TTN_ETIMEOUT (a bounded wait in a kernel expired: the
 * tensors are then unspecified, restore them with ttn_set_isometries or
 * ttn_set_state); TTN_ENAN (a non-finite energy); TTN_ENOCONV (in the last
 * sweep of some instance the top solve missed its residual tolerance within
 * lanczos_max * lanczos_restarts steps -- the tensors are a valid, updated
 * state, usual in the first sweeps from a random start -- or, in the mixed
 * modes, a polar factor was left more than 1e-5 from an isometry by its
 * Newton-Schulz blocks); TTN_OK. */
int ttn_sweep(ttn_t h, int n_sweeps, double* host_energy);

/* Sweep until the energy per spin of every instance changes by less than
 * `tol` from one sweep to the next (the convergence criterion of Sec. IV,
 * |delta e| < 1e-10), or until max_sweeps sweeps.  The change is computed on
 * the device after every sweep; the host reads the instances' flags after
 * every chunk of up to 8 sweeps, so up to 7 sweeps may follow the first one
 * that met the criterion (they can only lower the energy).  The first sweep
 * of a call is compared with nothing and never counts.  *n_done (may be NULL)
 * receives the sweeps run; host_energy (may be NULL) receives max_sweeps *
 * n_problems doubles as in ttn_sweep (the first *n_done rows written).
 * Returns TTN_OK when the criterion was met, TTN_ENOCONV when max_sweeps ran
 * out first, or an error status of ttn_sweep. */
int ttn_sweep_until(ttn_t h, double tol, int max_sweeps, int* n_done, double* host_energy);

/* Diagnostics of one instance's current tensors, computed on the device in
 * FP64 (Eqs. (constraint), (normalization); Sec. IV): out[0] = max over layers
 * and nodes of max |W W^T - I| (isometry defect); out[1] = max over site
 * layers t of |Tr R_t - N_t| / N_t (R_t: the density matrices of the N_t sites
 * of layer t, summed; each has trace one); out[2] = max over site layers of
 * max |R_t - R_t^T| / N_t; out[3] = |<v, v> - 1|; out[4] = the change of the
 * energy per spin in the last sweep (NaN before two sweeps); out[5] = 1 if
 * the last sweep's top solve met its tolerance, else 0; out[6] = the Krylov
 * dimension of its last cycle; with n_out >= 8, out[7] = 1 if a polar factor
 * of the last sweep (mixed modes) was left more than 1e-5 from an isometry by
 * its Newton-Schulz blocks, else 0; with n_out >= 9, out[8] = the number of
 * isometry layers whose polar factor took the adaptive schedule's short path
 * in the last sweep (ttn_options.polar_blocks); with n_out >= 10, out[9] = the
 * number of those layers whose short first block (polar_blocks 0: singular
 * values above 1e-2 of |X|_F) already left an isometry, so that the full
 * schedule did not run.  n_out >= 7.  Overwrites the context's
 * density matrices (a sweep recomputes them). */
int ttn_diagnostics(ttn_t h, int inst, double* out, int n_out);

/* Operators of site layer `site_layer` ascended through the current
 * isometries (Fig. 3 pushed upward: o' = W[o(x)I + I(x)o + sum_k A_k(x)B_k]W^T,
 * A'_k = W(I(x)A_k)W^T, B'_k = W(B_k(x)I)W^T), computed with the products in
 * precision `prec`, copied to host as [site][1+2K][chi_t][chi_t] (o, A_k, B_k;
 * one site when the tree is translation invariant).  The one-site term
 * includes the bond shift. */
int ttn_ascend(ttn_t h, int inst, int site_layer, int prec, double* host_out);

/* Energy <psi|H|psi> of one instance's current tensors, in FP64 (ascend and
 * top contraction, no re-optimisation). */
int ttn_energy(ttn_t h, int inst, double* E_total);

/* Energy of one instance's current tensors and, with d_grad != NULL, its
 * derivative with respect to every isometry and the top tensor (the
 * environments of Sec. III.A, laid out as ttn_env with layer -1; caller device
 * memory, FP64), in one pass: ascend, top contraction, then the environment of
 * every layer top-down while descending the density matrices (no update).  The
 * ascend, environment and descend contractions run in precision prec (0..4;
 * a mixed precision needs a context created with a mixed precision), the top
 * contraction and the energy in FP64.  This is the forward and backward of the
 * energy as a differentiable function. */
int ttn_value_and_grad(ttn_t h, int inst, int prec, double* E_total, double* d_grad);

/* Reduced density matrix on one site of site layer `site_layer` (0..T) of the
 * current tensors, chi_t x chi_t, to host (Sec. IV.B).  which = 0: average
 * over the sites of that layer (R / N_t); which = 1: the leftmost site. */
int ttn_rdm(ttn_t h, int inst, int site_layer, int which, double* host_out);

/* Environment dE/dw of isometry layer `layer` at the current tensors (Sec.
 * III.A: the sum of the contributions of all Hamiltonian terms), written to
 * caller device memory d_out (FP64, the isometry's shape; per node, all
 * nodes).  layer == T (the number of isometry layers) gives dE/dv = 2 H_top v
 * of the top tensor; layer == -1 gives every layer, concatenated as
 * ttn_set_isometries lays them out, followed by dE/dv.  This is the backward
 * of ttn_energy with respect to the tensors; ascended operators are kept and
 * the chi^3 intermediates recomputed. */
int ttn_env(ttn_t h, int inst, int layer, double* d_out);

/* Serialise / restore all isometries, top tensors and sweep counters. */
int ttn_get_state(ttn_t h, void* host_buf, size_t* bytes);
int ttn_set_state(ttn_t h, const void* host_buf, size_t bytes);

/* Kernel launches enqueued by the last ttn_sweep call (a count). */
long long ttn_launch_count(ttn_t h);

/* Run one sweep without graph capture, timing every grouped product with CUDA
 * events on the library's stream.  out[0..8] = FP64-engine milliseconds,
 * useful flops (2*M*N*K summed over groups and batches), launches; the same
 * three for the tensor-core engine; milliseconds and launches of all other
 * kernels (including event gaps); total milliseconds of the sweep.  With
 * n_out >= 15, out[9..11] = the same three for the double-float Gram and
 * apply products and out[12..14] for the double-float polar composition;
 * with 12 <= n_out < 15, out[9..11] = both together; with fewer they count as
 * "other"; with n_out >= 17, out[15] and out[16] = the algorithmic bytes of
 * the FP64-engine and tensor-core products (every group's operands read once,
 * a batch index of stride 0 read once, the output written once); with n_out
 * >= 19, out[17] and out[18] = milliseconds and launches of the persistent
 * top solve (else counted as "other").  The sweep updates the tensors like
 * ttn_sweep.  n_out >= 9. */
int ttn_profile_sweep(ttn_t h, double* out, int n_out);

/* Diagnostic: the tensor-core engine against the FP64 engine on seeded random
 * operands over sixteen cases: FP64 sources (K-major / M-major, two-level K
 * and batch, ragged edges, split K, alpha/beta), then FP32 sources (cases
 * 10-16, the layouts of the TMA-fed kernel in the TF32 modes: ragged tiles,
 * two-level K with a broadcast batch, batched transposed products, mixed K- /
 * MN-major groups, a split-K close with FP64 output).  d_ws: caller device
 * memory of at least ttn_selftest_bytes(); prec: 1..4 (ttn_precision);
 * out_rel[i] receives max|C_tc - C_fp64| / max|C_fp64| of case i for
 * i < min(n_out, 16) (n_out >= 11). */
size_t ttn_selftest_bytes(void);
int ttn_selftest_gemm(void* d_ws, size_t bytes, int prec, double* out_rel, int n_out, void* stream);

/* Diagnostic: the double-float (FP32 pair) Gram and apply products that the
 * mixed modes use for the polar factor, against the FP64 engine on seeded
 * operands: Gram X X^T for (P, n2) = (128, 16384) and (96, 1000), apply F X
 * for (128, 16384) and (40, 1000).  d_ws: caller device memory of at least
 * ttn_selftest_bytes(); out_rel[i] = max |C_df - C_fp64| / max |C_fp64|
 * (n_out >= 4); with n_out >= 5, out_rel[4] the Newton-Schulz step near
 * convergence that the adaptive polar schedule uses, (1.5 I - 0.5 A) X for A
 * within 1e-10 of I (P = 128, n2 = 16384), against the same product in
 * FP64. */
int ttn_selftest_df(void* d_ws, size_t bytes, double* out_rel, int n_out, void* stream);

/* Allocation-free close product, for callers that cannot allocate device
 * memory (plug-ins inside an application that owns the CUDA allocator, or code
 * where cudaMalloc is not permitted); the paper has no counterpart.
 *   C[p][q] = sum_{j < n2} Y[p][j] W[q][j]      (FP64, row-major, all device)
 * the product over both child legs that ends every ascend step.  It runs the
 * library's FP64 split-K kernel with its partial sums in a fixed 8 MiB device
 * array inside the library instead of caller scratch; every GPU that loads the
 * library holds that array until the process exits.  The first call on a
 * device looks the array up (cudaGetSymbolAddress), so make that first call
 * before any stream capture.  Calls share the array: two calls that overlap on
 * the GPU race (use one stream, or order them).  Nothing needs clearing: each
 * call overwrites every partial sum it reads.  Limits: 1 <= P, Q <= 256 and
 * 1 <= n2 <= 2^30, else TTN_EINVAL.  Work is enqueued on `stream` (cudaStream_t
 * as void*); the call allocates nothing. */
int ttn_close_noalloc(const double* d_Y, const double* d_W, int P, int Q, long long n2,
                      double* d_C, void* stream);

/* Autotuner of the grouped products (tile shapes and split counts): with
 * reps > 0, one sweep of every instance runs eagerly on one stream and, at
 * the first occurrence of each product shape (its sizes, groups and operand
 * layouts; not its addresses), every candidate configuration is timed with
 * CUDA events over `reps` launches after one warm-up launch: for tensor-core
 * products the engine (TMA-fed where eligible, thread-staged), its tile width
 * BN, the TMA-fed kernel's stage ring (192 KB, one CTA per SM, or 96 KB, two)
 * and the split count of K (powers of two up to 128); for FP64 products the
 * tile (16, 32, 64) and the split count; the split counts are limited to the
 * context's split-K buffer.  The fastest becomes the product's configuration (the next
 * ttn_sweep captures its graph again).  The sweep updates the tensors like
 * ttn_sweep.  With blob_bytes != NULL the table is exported: blob == NULL
 * returns the size in *blob_bytes, else the table is written to blob (at
 * least *blob_bytes bytes) for ttn_options.tiles of a later ttn_create.
 * reps == 0 only exports. */
int ttn_autotune(ttn_t h, int reps, void* blob, size_t* blob_bytes);

const char* ttn_last_error(ttn_t h);
void ttn_destroy(ttn_t h);

#ifdef __cplusplus
}
#endif

#endif /* TTN_H */
