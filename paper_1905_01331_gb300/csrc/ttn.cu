// Host orchestration of the TTN sweep and the C ABI declared in include/ttn.h.
//
// One sweep (Sec. III, "standard energy minimisation"):
//   ascend the Hamiltonian through every isometry layer (Fig. 3 pushed up),
//   solve the top tensor (Sec. III.B: "the top tensor v is updated similarly"
//   -- read as its lowest eigenvector, Lanczos in FP64),
//   then for t = T-1 .. 0: environment of w_t as a sum of contractions
//   (Sec. III.A, Figs. 2b, 3), w_t <- minus its polar factor (Sec. III.B,
//   Fig. 4c-d, in the Gram form of the appendix, Fig. 9b, iterated), and
//   descend the density matrices through the new w_t.
// Every contraction is one grouped product (GemmDesc); nothing else touches
// the O(chi^4) data.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/ttn.h"
#include "common.h"
#include "host_eig.h"

namespace ttn {

// Lanczos helpers defined in misc.cu
int lz_dots(const double* basis, long long n, int count, const double* w, double* coef,
            double* scratch, const int* skip, cudaStream_t s);
int lz_sub(const double* basis, long long n, int count, double* w, const double* coef,
           const int* skip, cudaStream_t s);
int lz_finish_step(double* basis, long long n, int j, double* w, const double* c1,
                   const double* c2, double* alpha, double* beta, double* scratch, double* nrm2,
                   int* skip, int* tdim, cudaStream_t s);
int lz_ritz(const double* alpha, const double* beta, const int* tdim, int jmax, double* y,
            double* theta, double* res, int* conv, double tol, cudaStream_t s);
int lz_combine(double* basis, long long n, const int* tdim, const double* y, double* v,
               double* scratch, double* nrm2, int* tdim_rw, int* skip, const int* conv,
               cudaStream_t s);
int lz_start(double* basis, long long n, const double* v, double* scratch, double* nrm2,
             int* tdim, int* skip, int* conv, cudaStream_t s);
int align_sign(double* v, const double* vprev, long long n, double* scratch, double* dotv,
               cudaStream_t s);

typedef long long ll;

// Bump allocator over the caller's workspace; with base == nullptr it only
// measures.
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  std::vector<std::pair<size_t, size_t>>* registry = nullptr;  // (start, bytes)
  double* take(size_t n_doubles) {
    off = (off + 255) & ~size_t(255);
    double* p = base ? reinterpret_cast<double*>(base + off) : nullptr;
    if (registry && base) registry->push_back({(size_t)(base + off), n_doubles * sizeof(double)});
    off += n_doubles * sizeof(double);
    return p;
  }
  int* take_int(size_t n) {
    off = (off + 255) & ~size_t(255);
    int* p = base ? reinterpret_cast<int*>(base + off) : nullptr;
    if (registry && base) registry->push_back({(size_t)(base + off), n * sizeof(int)});
    off += n * sizeof(int);
    return p;
  }
};

struct Instance {
  int L = 0, Ly = 0, d0 = 0, K = 0, T = 0, per_node = 0, chi = 0, n_spins = 0;
  double c = 0.0;
  std::vector<int> chis;
  std::vector<double> o, A, B;       // host copies of the terms
  std::vector<double*> W, ops, adj;  // device tensors per layer / site layer
  double* V = nullptr;
  double* Vprev = nullptr;
  double* E = nullptr;               // energy of the last top solve
  // device status of the instance: dstat = [energy of the previous sweep,
  // change per spin in the last sweep, convergence tolerance]; istat = [top
  // solve of the last sweep converged, its Krylov dimension, |change| <
  // tolerance, sweeps seen since the last reset, a polar factor of the last
  // sweep missed an isometry, 3 unused]
  double* dstat = nullptr;
  int* istat = nullptr;
  // per isometry layer (mixed modes, adaptive polar schedule): 1 = the second
  // block ran in full and the final step ran, 0 = both were cut short
  int* pfull = nullptr;
  // prediction of the adaptive polar schedule, per isometry layer t (stride
  // max(T, 1)): [t] try the well-conditioned first block, [T + t] the full
  // schedule runs in this sweep, [2T + t] sweeps since a failed first try
  int* ppred = nullptr;
  // per isometry layer: the long path's block 2 left X X^T more than
  // kPolarNear from I (the final Newton-Schulz step then runs in full)
  int* pfar = nullptr;
  // Identity part of the one-site operators, kept exactly in FP64: the true
  // one-site term of site j at layer t is  ops[t][j][0] + eoff[t][j] * I.
  std::vector<double*> eoff;
  // FP32 copies used by the tensor-core products (mixed modes)
  std::vector<float*> w32, ops32, adj32;
  // ttn_options.recompute_ops: the operators of site layers 1..T-1 live in two
  // ping-pong buffers (layer t in buffer t & 1); pp_holds[b] is the layer whose
  // operators buffer b holds (-1: none)
  int pp_holds[2] = {-1, -1};
  int sites(int t) const { return per_node ? (L >> t) : 1; }
  int nodes(int t) const { return per_node ? (L >> (t + 1)) : 1; }
  size_t w_elems(int t) const {
    return (size_t)nodes(t) * chis[t + 1] * chis[t] * chis[t];
  }
  size_t op_elems(int t) const { return (size_t)sites(t) * (1 + 2 * K) * chis[t] * chis[t]; }
};

struct PolarBlock {
  std::vector<std::pair<double, double>> steps;  // p(A) = a I - c A
};

// Sub-streams of a lane: independent products of one sweep stage run on them
// concurrently (parallel branches of the captured graph), each with its own
// split-K buffer.
constexpr int kSubStreams = 3;
struct SubStreams {
  int n = 0;                              // 0: stages run on the lane's stream
  cudaStream_t s[kSubStreams] = {};
  double* partial[kSubStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kSubStreams] = {};
};

// An autotuned launch configuration of one grouped product.
struct Tuned {
  int engine, tile, splits, occ;
  float ms;
};

// Serialised form of the autotuner's table (the ttn_options.tiles blob).
struct TuneBlobHeader {
  char magic[4];       // "TTNT"
  uint32_t version;    // 2
  uint32_t count;
  uint32_t reserved;
};
struct TuneBlobEntry {
  uint64_t key;
  int32_t engine, tile, splits, occ;
  float ms;
  int32_t reserved;
};

}  // namespace ttn

using namespace ttn;

// Scratch and stream of one concurrent instance stream ("lane").  The sweep
// code works on the ttn_ctx fields of the same names; enqueueing an instance
// on lane k first loads lane k's pointers into them.
struct Lane {
  cudaStream_t stream = nullptr;
  double *Y = nullptr, *Gam = nullptr, *X = nullptr, *X2 = nullptr, *Yt = nullptr, *M1 = nullptr;
  double *pA = nullptr, *pF = nullptr, *pP = nullptr, *pT = nullptr, *pS = nullptr;
  double *partial = nullptr, *red = nullptr, *scal = nullptr;
  double *lz_basis = nullptr, *lz_w = nullptr, *lz_c1 = nullptr, *lz_c2 = nullptr,
         *lz_alpha = nullptr, *lz_beta = nullptr, *lz_y = nullptr, *lz_tmp = nullptr,
         *top_stack0 = nullptr, *top_stack1 = nullptr, *lz_part = nullptr;
  double *lz_opsp = nullptr, *lz_bp = nullptr, *lz_Yp = nullptr;
  int* iflags = nullptr;
  SubStreams sub;
};

struct ttn_ctx {
  ttn_options opt;
  std::vector<Lane> lanes;            // lanes[0].stream == stream
  std::vector<int> lane_of;           // lane of each instance
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  std::vector<Instance> inst;
  cudaStream_t user = nullptr, stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::string err;
  long long launches = 0;
  long long launches_per_sweep = 0;
  int sweeps_done = 0;
  // shared scratch
  double *Y = nullptr, *Gam = nullptr, *X = nullptr, *X2 = nullptr, *Yt = nullptr, *M1 = nullptr;
  double *pA = nullptr, *pF = nullptr, *pP = nullptr, *pT = nullptr, *pS = nullptr;
  bool compose_refused = false;   // a cooperative launch was refused
  double* partial = nullptr;
  size_t partial_cap = 0;
  double* red = nullptr;       // dot scratch
  double* scal = nullptr;      // small scalars
  double *lz_basis = nullptr, *lz_w = nullptr, *lz_c1 = nullptr, *lz_c2 = nullptr, *lz_alpha = nullptr,
         *lz_beta = nullptr, *lz_y = nullptr, *lz_tmp = nullptr, *top_stack0 = nullptr,
         *top_stack1 = nullptr;
  double* lz_part = nullptr;   // persistent Lanczos: per-CTA partial sums, then 2 (m + 2) coefficients
  // double-float Lanczos: pairs of the top operators (both sites), basis, Y
  double *lz_opsp = nullptr, *lz_bp = nullptr, *lz_Yp = nullptr;
  int* iflags = nullptr;       // [0]=skip [1]=tdim [2]=conv [3]=nan [4]=wait expired
                               // [5]=grid-barrier counter of the polar composition
                               // [6], [7]=top-solve flags; [8..]=composition tile counters
  SubStreams sub;              // of the current lane
  int lz_m = 48;
  double* E_hist = nullptr;    // device energies of the current ttn_sweep call
  std::vector<PolarBlock> polar_f64, polar_tc;
  // mixed modes, adaptive: a first block that converges every singular value
  // above kPolarTry, then either one Newton-Schulz step (when the first block
  // left an isometry) or a block for the worst case; empty if not applicable
  std::vector<PolarBlock> polar_adapt;
  // adaptive schedule, layers predicted well conditioned: a first block that
  // converges every singular value above kPolarFirst (empty if not applicable)
  std::vector<PolarBlock> polar_first;
  bool measuring = false;      // plan pass: only size the partial buffer
  // plan pass over a fake base address: every operand's address range is
  // checked against the buffer it points into (no launch happens)
  std::vector<std::pair<size_t, size_t>> registry;
  std::string bounds_error;
  // autotuner: launch configuration per product shape (key: tune_key)
  std::map<uint64_t, Tuned> tuned;
  bool tuning = false;
  int tune_reps = 3;
  // profiling sweep: events around every product, by engine (0 FP64, 1 TC)
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, double>> ev_flops;   // (engine, flops) per event pair
  std::vector<const int*> ev_cond;   // per event pair: flops count only if *cond != 0
  std::vector<double> ev_bytes;                   // algorithmic bytes per event pair
};

namespace {

#define TTN_LANE_FIELDS(X_) X_(stream) X_(Y) X_(Gam) X_(X) X_(X2) X_(Yt) X_(M1) X_(pA) X_(pF) \
  X_(pP) X_(pT) X_(pS) X_(partial) X_(red) X_(scal) X_(lz_basis) X_(lz_w) X_(lz_c1) X_(lz_c2) \
  X_(lz_alpha) X_(lz_beta) X_(lz_y) X_(lz_tmp) X_(top_stack0) X_(top_stack1) X_(lz_part) \
  X_(lz_opsp) X_(lz_bp) X_(lz_Yp) X_(iflags) X_(sub)

void load_lane(ttn_ctx* h, const Lane& l) {
#define TTN_LOAD(f) h->f = l.f;
  TTN_LANE_FIELDS(TTN_LOAD)
#undef TTN_LOAD
}

void save_lane(const ttn_ctx* h, Lane& l) {
#define TTN_SAVE(f) l.f = h->f;
  TTN_LANE_FIELDS(TTN_SAVE)
#undef TTN_SAVE
}

}  // namespace

namespace {

bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
int ilog2(int x) { int r = 0; while ((1 << r) < x) ++r; return r; }

// A typed device pointer: FP64, or FP32 (the mixed modes keep the chi^3
// intermediates and copies of w and of the operators in FP32).
struct TP {
  void* p;
  int f32;
  TP operator+(ll e) const {
    return TP{static_cast<char*>(p) + e * (f32 ? 4 : 8), f32};
  }
};
TP tp(double* p) { return TP{p, 0}; }
TP tp(const double* p) { return TP{const_cast<double*>(p), 0}; }

Operand op(TP p, ll s_mn, ll s_k0, ll s_k1 = 0, ll s_b0 = 0, ll s_b1 = 0) {
  Operand o;
  o.p = p.p; o.s_mn = s_mn; o.s_k0 = s_k0; o.s_k1 = s_k1; o.s_b0 = s_b0; o.s_b1 = s_b1;
  o.f32 = p.f32;
  return o;
}
Operand op(const double* p, ll s_mn, ll s_k0, ll s_k1 = 0, ll s_b0 = 0, ll s_b1 = 0) {
  return op(tp(p), s_mn, s_k0, s_k1, s_b0, s_b1);
}

Group grp(Operand a, Operand b, int K0, int K1 = 1) {
  Group g;
  g.a = a; g.b = b; g.K = K0 * K1; g.k0_log2 = ilog2(K0);
  return g;
}

GemmDesc desc(int M, int N, int B0, int B1, TP C, ll sc_m, ll sc_n, ll sc_b0, ll sc_b1,
              double alpha = 1.0, double beta = 0.0) {
  GemmDesc d;
  memset(&d, 0, sizeof(d));
  d.M = M; d.N = N; d.B0 = B0; d.B1 = B1; d.C = C.p; d.c_f32 = C.f32;
  d.sc_m = sc_m; d.sc_n = sc_n; d.sc_b0 = sc_b0; d.sc_b1 = sc_b1;
  d.alpha = alpha; d.beta = beta; d.splits = 1;
  return d;
}
GemmDesc desc(int M, int N, int B0, int B1, double* C, ll sc_m, ll sc_n, ll sc_b0, ll sc_b1,
              double alpha = 1.0, double beta = 0.0) {
  return desc(M, N, B0, B1, tp(C), sc_m, sc_n, sc_b0, sc_b1, alpha, beta);
}

void add(GemmDesc& d, const Group& g) {
  if (d.ngroups < kMaxGroups) d.g[d.ngroups] = g;
  d.ngroups++;   // an overflow is reported by the plan pass and never launched
}

// Highest element offset an operand reaches for extents (mn, K0, K1, B0, B1).
ll max_offset(const Operand& o, int mn, int K0, int K1, int B0, int B1) {
  return (mn - 1) * o.s_mn + (K0 - 1) * o.s_k0 + (ll)(K1 - 1) * o.s_k1 + (ll)(B0 - 1) * o.s_b0 +
         (ll)(B1 - 1) * o.s_b1;
}

void check_range(ttn_ctx* h, const void* p, ll max_off, int f32, const char* what) {
  if (h->registry.empty() || !h->bounds_error.empty()) return;
  const size_t a = (size_t)p, e = a + (size_t)(max_off + 1) * (f32 ? 4 : 8);
  for (auto& r : h->registry)
    if (a >= r.first && a < r.first + r.second) {
      if (e > r.first + r.second)
        h->bounds_error = std::string(what) + " exceeds its buffer by " +
                          std::to_string(e - r.first - r.second) + " bytes";
      return;
    }
  h->bounds_error = std::string(what) + " points outside the workspace";
}

void check_desc(ttn_ctx* h, const GemmDesc& d) {
  for (int g = 0; g < d.ngroups; ++g) {
    const Group& G = d.g[g];
    const int K0 = 1 << G.k0_log2, K1 = G.K >> G.k0_log2;
    if (K0 * K1 != G.K || G.K <= 0) { h->bounds_error = "bad K split"; return; }
    check_range(h, G.a.p, max_offset(G.a, d.M, K0, K1, d.B0, d.B1), G.a.f32, "A operand");
    check_range(h, G.b.p, max_offset(G.b, d.N, K0, K1, d.B0, d.B1), G.b.f32, "B operand");
  }
  Operand c;
  c.p = d.C; c.s_mn = d.sc_m; c.s_k0 = d.sc_n; c.s_k1 = 0; c.s_b0 = d.sc_b0; c.s_b1 = d.sc_b1;
  check_range(h, d.C, max_offset(c, d.M, d.N, 1, d.B0, d.B1), d.c_f32, "C output");
}

// Key of a product for the autotuner: its shape, groups and operand layouts
// (strides, element type, 16-byte alignment), not its addresses.  FNV-1a.
uint64_t tune_key(const GemmDesc& d) {
  uint64_t h = 1469598103934665603ULL;
  auto mix = [&](long long v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (uint64_t)((v >> (8 * i)) & 0xFF);
      h *= 1099511628211ULL;
    }
  };
  auto mix_op = [&](const Operand& o) {
    mix(o.s_mn); mix(o.s_k0); mix(o.s_k1); mix(o.s_b0); mix(o.s_b1); mix(o.f32);
    mix((long long)((uintptr_t)o.p & 15));
  };
  mix(d.prec); mix(d.M); mix(d.N); mix(d.B0); mix(d.B1); mix(d.c_f32); mix(d.sym);
  mix(d.sc_m); mix(d.sc_n); mix(d.ngroups);
  for (int g = 0; g < d.ngroups && g < kMaxGroups; ++g) {
    mix(d.g[g].K); mix(d.g[g].k0_log2);
    mix_op(d.g[g].a);
    mix_op(d.g[g].b);
  }
  return h;
}

// Time every candidate configuration of one product on the library stream
// (one warm-up launch, then h->tune_reps launches between events) and keep
// the fastest.  Products are C = sum A B without accumulation into C, so the
// repeated launches leave the sweep's data as one launch would.
Tuned tune_product(ttn_ctx* h, const GemmDesc& d0) {
  struct Cand { int engine, tile, splits, occ; };
  std::vector<Cand> cands;
  long long ksum = 0;
  for (int g = 0; g < d0.ngroups; ++g) ksum += d0.g[g].K;
  std::vector<int> splits;
  for (int s = 1; s <= 128; s *= 2)
    if (s == 1 || (s <= ksum / 64 && gemm_partial_elems(d0, s) <= h->partial_cap)) splits.push_back(s);
  const bool tc = d0.prec != 0 && gemm_tc_supported(d0);
  GemmDesc dd = d0;
  dd.tile = 0;
  const int def_splits = std::max(1, std::min(gemm_pick_splits(dd), (int)splits.back()));
  cands.push_back({d0.tc_engine, 0, def_splits, 0});   // the default configuration
  for (int s : splits) {
    if (tc) {
      if (gemm_tma_eligible(d0)) {
        for (int bn : {64, 128})
          for (int occ : {1, 2})
            if (!(occ == 2 && bn == 128 && d0.prec == 2)) cands.push_back({0, bn, s, occ});
      }
      for (int bn : {32, 64, 128})
        if (bn <= std::max(32, d0.N)) cands.push_back({1, bn, s, 0});
    } else {
      for (int t : {16, 32, 64})
        if (t == 16 || t <= std::min(d0.M, d0.N)) cands.push_back({d0.tc_engine, t, s, 0});
    }
  }
  Tuned best{cands[0].engine, cands[0].tile, cands[0].splits, cands[0].occ, 1e30f};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  for (const Cand& c : cands) {
    GemmDesc e = d0;
    e.tc_engine = c.engine;
    e.tile = c.tile;
    e.splits = c.splits;
    e.occ = c.occ;
    e.partial = h->partial;
    e.err = h->iflags + 4;
    gemm_launch(e, h->stream);
    cudaEventRecord(a, h->stream);
    for (int r = 0; r < h->tune_reps; ++r) gemm_launch(e, h->stream);
    cudaEventRecord(b, h->stream);
    if (cudaEventSynchronize(b) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    ms /= (float)std::max(1, h->tune_reps);
    if (ms < best.ms) best = Tuned{c.engine, c.tile, c.splits, c.occ, ms};
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

// Run (or, in the plan pass, size and bounds-check) one product.
void run(ttn_ctx* h, GemmDesc d, int prec) {
  d.prec = prec;
  d.tc_engine = h->opt.tc_engine;
  int s;
  const uint64_t key = h->tuned.empty() && !h->tuning ? 0 : tune_key(d);
  auto it = key ? h->tuned.find(key) : h->tuned.end();
  if (h->tuning && !h->measuring && it == h->tuned.end() && !d.skip && d.ngroups <= kMaxGroups &&
      d.M > 0 && d.N > 0) {
    it = h->tuned.emplace(key, tune_product(h, d)).first;
  }
  if (it != h->tuned.end()) {
    d.tc_engine = it->second.engine;
    d.tile = it->second.tile;
    d.occ = it->second.occ;
    s = it->second.splits;
  } else {
    s = gemm_pick_splits(d);
  }
  size_t need = gemm_partial_elems(d, s);
  if (h->measuring) {
    if (need > h->partial_cap) h->partial_cap = need;
    if (d.ngroups > kMaxGroups) h->bounds_error = "too many groups";
    check_desc(h, d);
    return;
  }
  if (need > h->partial_cap) s = 1;   // cannot happen after planning
  if (d.ngroups > kMaxGroups) return;
  d.splits = s;
  d.partial = h->partial;
  d.err = h->iflags + 4;
  if (h->profiling) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, h->stream);
    h->launches += gemm_launch(d, h->stream);
    cudaEventRecord(b, h->stream);
    h->ev_pool.push_back(a);
    h->ev_pool.push_back(b);
    double kk = 0.0;
    for (int g = 0; g < d.ngroups; ++g) kk += d.g[g].K;
    const int engine = (d.prec != 0 && gemm_tc_supported(d)) ? 1 : 0;
    h->ev_flops.push_back({engine, 2.0 * d.M * d.N * kk * d.B0 * d.B1});
    // algorithmic bytes: every group's operands read once (a batch index of
    // stride 0 is a broadcast: read once), the output written once
    double bytes = (double)d.M * d.N * d.B0 * d.B1 * (d.c_f32 ? 4 : 8);
    for (int g = 0; g < d.ngroups; ++g) {
      const Group& G = d.g[g];
      const double ba = (G.a.s_b0 ? d.B0 : 1) * (double)(G.a.s_b1 ? d.B1 : 1);
      const double bb = (G.b.s_b0 ? d.B0 : 1) * (double)(G.b.s_b1 ? d.B1 : 1);
      bytes += (double)d.M * G.K * ba * (G.a.f32 ? 4 : 8) + (double)d.N * G.K * bb * (G.b.f32 ? 4 : 8);
    }
    h->ev_bytes.push_back(bytes);
    h->ev_cond.push_back(nullptr);
    return;
  }
  h->launches += gemm_launch(d, h->stream);
}

// Independent products of one stage: fork() makes the sub-streams wait for
// the work enqueued so far, branch(i) directs the following launches to
// sub-stream i (with its own split-K buffer), join() makes the lane's stream
// wait for every sub-stream and restores it.  Without sub-streams (or in a
// profiling or tuning sweep, which time one product at a time) all three are
// no-ops and everything stays on the lane's stream.
struct StageFork {
  ttn_ctx* h;
  cudaStream_t main;
  double* partial;
  bool on;
  explicit StageFork(ttn_ctx* hh)
      : h(hh), main(hh->stream), partial(hh->partial),
        on(hh->sub.n > 0 && !hh->measuring && !hh->profiling && !hh->tuning) {
    if (!on) return;
    cudaEventRecord(h->sub.fork, main);
    for (int i = 0; i < h->sub.n; ++i) cudaStreamWaitEvent(h->sub.s[i], h->sub.fork, 0);
  }
  void branch(int i) {
    if (!on) return;
    h->stream = h->sub.s[i % h->sub.n];
    h->partial = h->sub.partial[i % h->sub.n];
  }
  void join() {
    if (!on) return;
    for (int i = 0; i < h->sub.n; ++i) {
      cudaEventRecord(h->sub.join[i], h->sub.s[i]);
      cudaStreamWaitEvent(main, h->sub.join[i], 0);
    }
    h->stream = main;
    h->partial = partial;
    on = false;
  }
  ~StageFork() { join(); }
};

// Polar schedule: scaled Newton-Schulz steps p(x) = 1.5 c x - 0.5 c^3 x^3 with
// c = sqrt(3 / (1 + l + l^2)) for singular values in [l, 1]; steps are
// composed on the P x P level in blocks whose growth stays below gmax, with
// a fresh Gram matrix at the start of every block.
// Adaptive schedule of the mixed modes: singular values (of X scaled to unit
// Frobenius norm) above kPolarTry converge in the first block; the second is
// cut to one step when max |X X^T - I| <= kPolarNear after it (one step then
// leaves a defect of at most ~0.75 (P kPolarNear)^2, ~1e-14 for P = 128).
// With kPolarTry = 1e-5 the worst case left for the second block needs a
// growth of 1.5e4 (17 + 15 steps); with 1e-4 it needed 1.9e5 in one block,
// whose rounding (48-bit emulation: 1e-12 to 5e-12; on the GPU 2e-11) the
// final step no longer removed.
constexpr double kPolarTry = 1e-5;
constexpr double kPolarNear = 1e-9;
// Layers predicted well conditioned first try a block that converges every
// singular value above kPolarFirst (10 steps instead of 17; growth <= 740,
// so its rounding stays far below kPolarNear).  If it leaves X X^T within
// kPolarNear of I, one Newton-Schulz step ends the factor as above;
// otherwise the adaptive schedule runs in full from the same start, and the
// layer skips the first try for kPolarRetry sweeps.
constexpr double kPolarFirst = 1e-2;
constexpr int kPolarRetry = 16;

std::vector<PolarBlock> polar_schedule(double l0, double gmax, double final_tol, int max_block) {
  std::vector<PolarBlock> out;
  double l = l0;
  PolarBlock cur;
  double start = l;
  int guard = 0;
  while (1.0 - l > final_tol && guard++ < 200) {
    const double c = std::sqrt(3.0 / (1.0 + l + l * l));
    const double ln = 1.5 * c * l - 0.5 * c * c * c * l * l * l;
    if (!cur.steps.empty() && (ln / start > gmax || (int)cur.steps.size() >= max_block)) {
      out.push_back(cur);
      cur = PolarBlock();
      start = l;
    }
    cur.steps.push_back({1.5 * c, 0.5 * c * c * c});
    l = ln;
  }
  if (!cur.steps.empty()) out.push_back(cur);
  return out;
}

// --------------------------------------------------------------------------
// Sweep pieces.  Layer t: P = chi_{t+1}, n = chi_t, NJ nodes.
// ops/adj of site layer t: [site][1+2K][n][n]; op 0 = o (adjoint R),
// 1+k = A_k (P_k), 1+K+k = B_k (Q_k).  Node J's children are sites 2J, 2J+1.
// --------------------------------------------------------------------------

struct LayerView {
  int P, n, NJ, K;
  ll n2, Pn2, ss, node_ss;   // ss: site stride of ops_t; node_ss: ops_t stride per node
  ll adj_ss;                 // site stride of adj_{t+1}
  TP opsL;                   // ops_t of the left child of node 0
  TP opsR;                   // ops_t of the right child of node 0
  TP W;                      // w_t
  TP adj;                    // adjoints of site layer t+1
  int f32;                   // storage of the chi^3 intermediates
};

// Storage of one layer for a product precision: FP64 tensors for FP64
// products, their FP32 copies for tensor-core products.
LayerView view(const Instance& I, int t, int prec) {
  LayerView v;
  v.P = I.chis[t + 1]; v.n = I.chis[t]; v.NJ = I.nodes(t); v.K = I.K;
  v.n2 = (ll)v.n * v.n; v.Pn2 = (ll)v.P * v.n2;
  v.ss = (1 + 2 * I.K) * v.n2;
  v.node_ss = I.per_node ? 2 * v.ss : 0;
  v.adj_ss = I.per_node ? (ll)(1 + 2 * I.K) * v.P * v.P : 0;
  v.f32 = prec != 0;
  const TP ops = v.f32 ? TP{I.ops32[t], 1} : tp(I.ops[t]);
  v.opsL = ops;
  v.opsR = ops + (I.per_node ? v.ss : 0);
  v.W = v.f32 ? TP{I.w32[t], 1} : tp(I.W[t]);
  v.adj = v.f32 ? TP{I.adj32[t + 1], 1} : tp(I.adj[t + 1]);
  return v;
}

TP scratch(double* p, const LayerView& v) { return TP{p, v.f32}; }

// Y[b0][J] = W_J X_b0 for X = ops(side, first + b0), b0 < count:  right product.
void right_mult(ttn_ctx* h, const LayerView& v, TP W, TP side, int first, int count, bool transX,
                TP Y, ll y_b0, int prec) {
  GemmDesc d = desc(v.P * v.n, v.n, count, v.NJ, Y, v.n, 1, y_b0, v.Pn2);
  // B(i = column r', k = r) = X[r][r'] (or X[r'][r] when transposed)
  add(d, grp(op(W, v.n, 1, 0, 0, v.Pn2),
             op(side + first * v.n2, transX ? v.n : 1, transX ? 1 : v.n, 0, v.n2, v.node_ss), v.n));
  run(h, d, prec);
}

// Y[b0][J][p] = X_b0^T W_{J,p} (transX: X_b0 W_{J,p}): left product, batched over p.
void left_mult(ttn_ctx* h, const LayerView& v, TP W, TP side, int first, int count, bool transX,
               TP Y, ll y_b0, int prec) {
  for (int k = 0; k < count; ++k) {
    GemmDesc d = desc(v.n, v.n, v.P, v.NJ, Y + k * y_b0, v.n, 1, v.n2, v.Pn2);
    // A(m = l', k = l) = X[l][l'] (X^T), or X[l'][l] (X)
    const TP X = side + (first + k) * v.n2;
    add(d, grp(op(X, transX ? v.n : 1, transX ? 1 : v.n, 0, 0, v.node_ss),
               op(W, 1, v.n, 0, v.n2, v.Pn2), v.n));
    run(h, d, prec);
  }
}

void ascend_layer(ttn_ctx* h, Instance& I, int t, int prec) {
  const LayerView v = view(I, t, prec);
  const int K = I.K;
  const TP W = v.W;
  const ll slab = (ll)v.NJ * v.Pn2;    // one stacked tensor
  const TP U = scratch(h->M1, v);     // U_k = W B_k(right child), K slabs
  const TP Y = scratch(h->Y, v);
  StageFork fk(h);
  fk.branch(0);
  right_mult(h, v, W, v.opsR, 1 + K, K, false, U, slab, prec);
  // Y0 = o_L^T W_p + W_p o_R + sum_k A_{k,L}^T U_k,p
  {
    GemmDesc d = desc(v.n, v.n, v.P, v.NJ, Y, v.n, 1, v.n2, v.Pn2);
    add(d, grp(op(v.opsL, 1, v.n, 0, 0, v.node_ss), op(W, 1, v.n, 0, v.n2, v.Pn2), v.n));
    add(d, grp(op(W, v.n, 1, 0, v.n2, v.Pn2), op(v.opsR, 1, v.n, 0, 0, v.node_ss), v.n));
    for (int k = 0; k < K; ++k)
      add(d, grp(op(v.opsL + (1 + k) * v.n2, 1, v.n, 0, 0, v.node_ss),
                 op(U + k * slab, 1, v.n, 0, v.n2, v.Pn2), v.n));
    run(h, d, prec);
  }
  // Y_{1+k} = W A_{k,R};  Y_{1+K+k} = B_{k,L}^T W
  fk.branch(1);
  right_mult(h, v, W, v.opsR, 1, K, false, Y + slab, slab, prec);
  fk.branch(2);
  left_mult(h, v, W, v.opsL, 1 + K, K, false, Y + (1 + K) * slab, slab, prec);
  fk.join();
  // ops_{t+1}[J][j] = sum_{lr} Y_j[J][p][lr] W_J[q][lr]   (FP64 output)
  const ll out_site = (ll)(1 + 2 * K) * v.P * v.P;
  GemmDesc d = desc(v.P, v.P, 1 + 2 * K, v.NJ, I.ops[t + 1], v.P, 1, (ll)v.P * v.P,
                    I.per_node ? out_site : 0);
  add(d, grp(op(Y, v.n2, 1, 0, slab, v.Pn2), op(W, v.n2, 1, 0, 0, v.Pn2), (int)v.n2));
  run(h, d, prec);
  // identity part: e'_J = e_L + e_R + tr(o'_J)/P, o'_J -= tr/P I
  if (!h->measuring) {
    h->launches += split_identity(I.ops[t + 1], I.per_node ? out_site : 0, v.P, v.NJ, I.eoff[t],
                                  I.per_node ? 1 : 0, I.eoff[t + 1], h->stream);
    if (v.f32) h->launches += to_f32(I.ops[t + 1], I.ops32[t + 1], I.op_elems(t + 1), h->stream);
  }
  if (t + 1 < I.T) I.pp_holds[(t + 1) & 1] = t + 1;
}

// With recomputation (ttn_options.recompute_ops), make the operators of site
// layer t available again: re-ascend from the bottom through the current (not
// yet updated) isometries of layers 0..t-1.  A no-op when they are stored.
void ensure_ops(ttn_ctx* h, Instance& I, int t, int prec) {
  if (!h->opt.recompute_ops || t <= 0 || t >= I.T || I.pp_holds[t & 1] == t) return;
  for (int u = 0; u < t; ++u) ascend_layer(h, I, u, prec);
}

// Top Hamiltonian on x (c x c): w = o_0 x + x o_1^T + sum_k (A_k0 x B_k1^T + B_k0 x A_k1^T)
void top_matvec(ttn_ctx* h, Instance& I, const double* x, double* w, const int* skip) {
  const int T = I.T, c = I.chis[T], K = I.K;
  const ll c2 = (ll)c * c, ss = (ll)(1 + 2 * K) * c2;
  const double* s0 = I.ops[T];
  const double* s1 = I.ops[T] + (I.per_node ? ss : 0);
  double* Yk = h->lz_tmp;   // 2K stacked: A_k0 x, then B_k0 x
  {
    GemmDesc d = desc(c, c, 2 * K, 1, Yk, c, 1, c2, 0);
    add(d, grp(op(s0 + c2, c, 1, 0, c2, 0), op(x, 1, c, 0, 0, 0), c));
    d.skip = skip;
    run(h, d, 0);
  }
  GemmDesc d = desc(c, c, 1, 1, w, c, 1, 0, 0);
  d.skip = skip;
  add(d, grp(op(s0, c, 1), op(x, 1, c), c));                 // o_0 x
  add(d, grp(op(x, c, 1), op(s1, c, 1), c));                 // x o_1^T
  for (int k = 0; k < K; ++k) {
    add(d, grp(op(Yk + k * c2, c, 1), op(s1 + (1 + K + k) * c2, c, 1), c));      // (A_k0 x) B_k1^T
    add(d, grp(op(Yk + (K + k) * c2, c, 1), op(s1 + (1 + k) * c2, c, 1), c));    // (B_k0 x) A_k1^T
  }
  run(h, d, 0);
}

// Residual tolerance of the top solve: the option, or by default 1e-13 in
// FP64 mode and 1e-8 in the mixed modes, whose top operators carry the
// tensor-core rounding of the ascended layers (1e-6 to 3e-5 relative): a
// tighter solve of that operator would not move the state further (the
// residual is still two orders below the operator's own rounding; the energy
// error of the solve is quadratic in it).
double lanczos_tolerance(const ttn_ctx* h) {
  if (h->opt.lanczos_tol > 0.0) return h->opt.lanczos_tol;
  return h->opt.prec == 0 ? 1e-13 : 1e-8;
}

void top_solve(ttn_ctx* h, Instance& I, double* energy_out) {
  const int T = I.T, c = I.chis[T];
  const ll n = (ll)c * c;
  if (h->opt.top_mode == 1) {
    // v <- -H_top v / |H_top v|: minus the polar factor of the top tensor's
    // environment (one power step with the negative semidefinite H_top)
    top_matvec(h, I, I.V, h->lz_w, nullptr);
    if (h->measuring) { top_matvec(h, I, I.V, h->lz_w, nullptr); return; }
    h->launches += top_grad(h->lz_tmp, h->lz_w, I.V, n, I.eoff[T], I.per_node ? 1 : 0, h->stream);
    h->launches += batched_dot(h->lz_tmp, h->lz_tmp, n, 0, 1, h->scal, h->red, h->stream);
    h->launches += scale_normalise(h->lz_tmp, I.V, n, h->scal, -1.0, h->stream);
    top_matvec(h, I, I.V, h->lz_w, nullptr);
    h->launches += batched_dot(I.V, h->lz_w, n, 0, 1, h->scal + 4, h->red, h->stream);
    h->launches += batched_dot(I.V, I.V, n, 0, 1, h->scal + 6, h->red, h->stream);
    h->launches += top_energy_sum(h->scal + 4, h->scal + 6, I.eoff[I.T], I.per_node ? 1 : 0,
                                  I.c * I.L, energy_out, h->stream);
    h->launches += store_ints(I.istat, nullptr, 2, 1, h->stream);   // no solve to converge
    return;
  }
  const int m = (int)std::min<ll>(h->lz_m, n);
  if ((h->opt.persistent & 2) && lanczos_supported(c, m)) {
    if (!h->measuring) {
      LanczosArgs a;
      a.s0 = I.ops[T];
      a.s1 = I.ops[T] + (I.per_node ? (ll)(1 + 2 * I.K) * n : 0);
      a.V = I.V; a.Vprev = I.Vprev;
      a.basis = h->lz_basis; a.w = h->lz_w; a.Y = h->lz_tmp; a.part = h->lz_part;
      a.coef = h->lz_part + (ll)kLMaxGrid * (h->lz_m + 2);   // 2 (m + 2) doubles
      a.alpha = h->lz_alpha; a.beta = h->lz_beta; a.y = h->lz_y; a.scal = h->scal;
      a.flags = h->iflags + 6;
      a.c = c; a.K = I.K; a.m = m; a.restarts = h->opt.lanczos_restarts;
      a.tol = lanczos_tolerance(h);
      a.bar = reinterpret_cast<unsigned*>(h->iflags + 5);
      a.err = h->iflags + 4;
      a.max_spin = h->opt.wait_polls;
      a.df = h->opt.prec != 0 && h->opt.double_float;
      a.s0p = reinterpret_cast<float*>(h->lz_opsp);
      a.s1p = a.s0p + 2 * (ll)(1 + 2 * I.K) * n;
      a.bp = reinterpret_cast<float*>(h->lz_bp);
      a.Yp = reinterpret_cast<float*>(h->lz_Yp);
      const int grid = lanczos_grid(c, h->profiling ? 1 : (int)h->lanes.size());
      cudaEvent_t ev[2];
      if (h->profiling) {
        cudaEventCreate(&ev[0]);
        cudaEventCreate(&ev[1]);
        cudaEventRecord(ev[0], h->stream);
      }
      const int nl = grid > 0 ? lanczos_launch(a, grid, h->stream) : -1;
      if (nl < 0) h->compose_refused = true;
      else h->launches += nl;
      if (h->profiling) {
        // family 4: the top solve (executed matrix-vector flops are not counted)
        cudaEventRecord(ev[1], h->stream);
        h->ev_pool.push_back(ev[0]);
        h->ev_pool.push_back(ev[1]);
        h->ev_flops.push_back({4, 0.0});
        h->ev_bytes.push_back(0.0);
        h->ev_cond.push_back(nullptr);
      }
      // converged flag and Krylov dimension of this solve, kept per instance
      h->launches += store_ints(I.istat, a.flags, 2, 0, h->stream);
    }
  } else {
  int* skip = h->iflags;
  int* tdim = h->iflags + 1;
  int* conv = h->iflags + 2;
  double* nrm2 = h->scal;
  double* theta = h->scal + 1;
  double* res = h->scal + 2;
  double* dotv = h->scal + 3;
  if (!h->measuring) {
    cudaMemcpyAsync(I.Vprev, I.V, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    h->launches += lz_start(h->lz_basis, n, I.V, h->red, nrm2, tdim, skip, conv, h->stream);
  }
  for (int cyc = 0; cyc < h->opt.lanczos_restarts; ++cyc) {
    for (int j = 0; j < m; ++j) {
      top_matvec(h, I, h->lz_basis + j * n, h->lz_w, skip);
      if (h->measuring) continue;
      h->launches += lz_dots(h->lz_basis, n, j + 1, h->lz_w, h->lz_c1, h->red, skip, h->stream);
      h->launches += lz_sub(h->lz_basis, n, j + 1, h->lz_w, h->lz_c1, skip, h->stream);
      h->launches += lz_dots(h->lz_basis, n, j + 1, h->lz_w, h->lz_c2, h->red, skip, h->stream);
      h->launches += lz_sub(h->lz_basis, n, j + 1, h->lz_w, h->lz_c2, skip, h->stream);
      if (j + 1 < m || true)
        h->launches += lz_finish_step(h->lz_basis, n, j, h->lz_w, h->lz_c1, h->lz_c2,
                                      h->lz_alpha, h->lz_beta, h->red, nrm2, skip, tdim,
                                      h->stream);
    }
    if (h->measuring) continue;
    h->launches += lz_ritz(h->lz_alpha, h->lz_beta, tdim, h->lz_m, h->lz_y, theta, res, conv,
                           lanczos_tolerance(h), h->stream);
    h->launches += lz_combine(h->lz_basis, n, tdim, h->lz_y, I.V, h->red, nrm2, tdim, skip, conv,
                              h->stream);
  }
  if (!h->measuring) {
    h->launches += align_sign(I.V, I.Vprev, n, h->red, dotv, h->stream);
    h->launches += store_ints(I.istat, conv, 1, 0, h->stream);
    h->launches += store_ints(I.istat + 1, tdim, 1, 0, h->stream);
  }
  }
  if (h->measuring) { top_matvec(h, I, I.V, h->lz_w, nullptr); return; }
  // energy = <V, H V> + c L
  top_matvec(h, I, I.V, h->lz_w, nullptr);
  h->launches += batched_dot(I.V, h->lz_w, n, 0, 1, h->scal + 4, h->red, h->stream);
  h->launches += batched_dot(I.V, I.V, n, 0, 1, h->scal + 6, h->red, h->stream);
  h->launches += top_energy_sum(h->scal + 4, h->scal + 6, I.eoff[I.T], I.per_node ? 1 : 0,
                                I.c * I.L, energy_out, h->stream);
}

void energy_only(ttn_ctx* h, Instance& I, double* energy_out) {
  const ll n = (ll)I.chis[I.T] * I.chis[I.T];
  top_matvec(h, I, I.V, h->lz_w, nullptr);
  if (h->measuring) return;
  h->launches += batched_dot(I.V, h->lz_w, n, 0, 1, h->scal + 4, h->red, h->stream);
  h->launches += batched_dot(I.V, I.V, n, 0, 1, h->scal + 6, h->red, h->stream);
  h->launches += top_energy_sum(h->scal + 4, h->scal + 6, I.eoff[I.T], I.per_node ? 1 : 0,
                                I.c * I.L, energy_out, h->stream);
}

// Top adjoints: R = V V^T + V^T V, P_k = V B_k V^T + V^T B_k V, Q_k = V^T A_k V + V A_k V^T
// (per node: site 0 gets the V ... V^T terms, site 1 the V^T ... V terms).
void top_adjoints(ttn_ctx* h, Instance& I) {
  const int T = I.T, c = I.chis[T], K = I.K;
  const ll c2 = (ll)c * c, ss = (ll)(1 + 2 * K) * c2;
  const double* s0 = I.ops[T];
  const double* s1 = I.ops[T] + (I.per_node ? ss : 0);
  double* T0 = h->top_stack0;   // [V | V B_k1 | V A_k1]
  double* T1 = h->top_stack1;   // [V | B_k0 V | A_k0 V]
  if (!h->measuring) {
    cudaMemcpyAsync(T0, I.V, c2 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(T1, I.V, c2 * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  }
  {  // T0[1+j] = V X_j(site 1), X = [A..., B...] -> order B first then A
    GemmDesc d = desc(c, c, K, 1, T0 + c2, c, 1, c2, 0);
    add(d, grp(op(I.V, c, 1), op(s1 + (1 + K) * c2, 1, c, 0, c2, 0), c));   // V B_k1
    run(h, d, 0);
    GemmDesc e = desc(c, c, K, 1, T0 + (1 + K) * c2, c, 1, c2, 0);
    add(e, grp(op(I.V, c, 1), op(s1 + c2, 1, c, 0, c2, 0), c));             // V A_k1
    run(h, e, 0);
    GemmDesc f = desc(c, c, K, 1, T1 + c2, c, 1, c2, 0);
    add(f, grp(op(s0 + (1 + K) * c2, c, 1, 0, c2, 0), op(I.V, 1, c), c));   // B_k0 V
    run(h, f, 0);
    GemmDesc g = desc(c, c, K, 1, T1 + (1 + K) * c2, c, 1, c2, 0);
    add(g, grp(op(s0 + c2, c, 1, 0, c2, 0), op(I.V, 1, c), c));             // A_k0 V
    run(h, g, 0);
  }
  double* adj = I.adj[T];
  // site-0 part: T0_j V^T ; site-1 part: V^T T1_j
  Group g0 = grp(op(T0, c, 1, 0, c2, 0), op(I.V, c, 1), c);           // B(i=col, k) = V[i][k]
  Group g1 = grp(op(I.V, 1, c), op(T1, 1, c, 0, c2, 0), c);           // A(m, k) = V[k][m]
  if (I.per_node) {
    GemmDesc d0 = desc(c, c, 1 + 2 * K, 1, adj, c, 1, c2, 0);
    add(d0, g0);
    run(h, d0, 0);
    GemmDesc d1 = desc(c, c, 1 + 2 * K, 1, adj + ss, c, 1, c2, 0);
    add(d1, g1);
    run(h, d1, 0);
  } else {
    GemmDesc d = desc(c, c, 1 + 2 * K, 1, adj, c, 1, c2, 0);
    add(d, g0);
    add(d, g1);
    run(h, d, 0);
  }
}

// Gamma_J = R_J Zs + sum_k [P_k W A_k^T + P_k^T W A_k + Q_k B_k W + Q_k^T B_k^T W]
void environment(ttn_ctx* h, Instance& I, int t, int prec, double* Gam) {
  const LayerView v = view(I, t, prec);
  const int K = I.K;
  const TP W = v.W;
  const ll slab = (ll)v.NJ * v.Pn2;
  const TP E_ = scratch(h->M1, v);            // W B_k^T (K slabs)
  const TP U = E_ + K * slab;                 // W B_k   (K slabs)
  StageFork fk(h);
  fk.branch(0);
  right_mult(h, v, W, v.opsR, 1 + K, K, true, E_, slab, prec);
  right_mult(h, v, W, v.opsR, 1 + K, K, false, U, slab, prec);
  const TP Zs = scratch(h->Y, v);             // slab 0
  {
    GemmDesc d = desc(v.n, v.n, v.P, v.NJ, Zs, v.n, 1, v.n2, v.Pn2);
    Operand Wl = op(W, 1, v.n, 0, v.n2, v.Pn2);      // B operand: W_p[k][i]
    Operand Wr = op(W, v.n, 1, 0, v.n2, v.Pn2);      // A operand: W_p[m][k]
    add(d, grp(op(v.opsL, v.n, 1, 0, 0, v.node_ss), Wl, v.n));    // o_L W_p
    add(d, grp(op(v.opsL, 1, v.n, 0, 0, v.node_ss), Wl, v.n));    // o_L^T W_p
    add(d, grp(Wr, op(v.opsR, v.n, 1, 0, 0, v.node_ss), v.n));    // W_p o_R^T
    add(d, grp(Wr, op(v.opsR, 1, v.n, 0, 0, v.node_ss), v.n));    // W_p o_R
    for (int k = 0; k < K; ++k) {
      const TP Ak = v.opsL + (1 + k) * v.n2;
      add(d, grp(op(Ak, v.n, 1, 0, 0, v.node_ss), op(E_ + k * slab, 1, v.n, 0, v.n2, v.Pn2), v.n));
      add(d, grp(op(Ak, 1, v.n, 0, 0, v.node_ss), op(U + k * slab, 1, v.n, 0, v.n2, v.Pn2), v.n));
    }
    run(h, d, prec);
    // identity parts of o_L and o_R: W (e I (x) I + I (x) e I) = (e_L + e_R) W, twice (S + S^T)
    if (!h->measuring)
      h->launches += add_identity_part(Zs.p, W.p, v.f32, v.Pn2, v.NJ, I.eoff[t],
                                       I.per_node ? 1 : 0, 2.0, h->stream);
  }
  // one-leg products: slabs 1.. of Y: WAt_k, WA_k, BW_k, BtW_k
  const TP WAt = Zs + slab;
  const TP WA = WAt + K * slab;
  const TP BW = WA + K * slab;
  const TP BtW = BW + K * slab;
  fk.branch(1);
  right_mult(h, v, W, v.opsR, 1, K, true, WAt, slab, prec);
  right_mult(h, v, W, v.opsR, 1, K, false, WA, slab, prec);
  fk.branch(2);
  left_mult(h, v, W, v.opsL, 1 + K, K, true, BW, slab, prec);
  left_mult(h, v, W, v.opsL, 1 + K, K, false, BtW, slab, prec);
  fk.join();
  const TP G = v.adj;
  const ll PP = (ll)v.P * v.P;
  GemmDesc d = desc(v.P, (int)v.n2, 1, v.NJ, Gam, v.n2, 1, 0, v.Pn2);   // FP64 output
  auto Gn = [&](int j) { return op(G + j * PP, v.P, 1, 0, 0, v.adj_ss); };
  auto Gt = [&](int j) { return op(G + j * PP, 1, v.P, 0, 0, v.adj_ss); };
  auto Tn = [&](TP T) { return op(T, 1, v.n2, 0, 0, v.Pn2); };
  add(d, grp(Gn(0), Tn(Zs), v.P));
  for (int k = 0; k < K; ++k) {
    add(d, grp(Gn(1 + k), Tn(WAt + k * slab), v.P));
    add(d, grp(Gt(1 + k), Tn(WA + k * slab), v.P));
    add(d, grp(Gn(1 + K + k), Tn(BW + k * slab), v.P));
    add(d, grp(Gt(1 + K + k), Tn(BtW + k * slab), v.P));
  }
  run(h, d, prec);
}

// w_t <- -polar(Gam - mu |Gam| w_t) by scaled Newton-Schulz blocks.
// Profiling sweeps time the double-float products as engine 2: an event
// before (df_begin) and after (df_end) each of them.
void df_begin(ttn_ctx* h) {
  if (!h->profiling) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, h->stream);
  h->ev_pool.push_back(e);
}
void df_end(ttn_ctx* h, int launches, double flops, const int* cond = nullptr) {
  h->launches += launches;
  if (!h->profiling) return;
  cudaEvent_t e;
  cudaEventCreate(&e);
  cudaEventRecord(e, h->stream);
  h->ev_pool.push_back(e);
  h->ev_flops.push_back({2, flops});
  h->ev_bytes.push_back(0.0);
  h->ev_cond.push_back(cond);
}

// F = composed polynomial of one block from the Gram matrix in pA (one
// cooperative launch; pA, pP, pT, pS are overwritten).  shortcut (double-float
// only, device, may be null): when it holds 0 the block is one Newton-Schulz
// step instead.
void compose_block(ttn_ctx* h, const PolarBlock& blk, int P, int NJ, bool df,
                   const int* shortcut = nullptr) {
  ComposeArgs a;
  // double-float: A_0 arrives as pairs in pP (split from the FP64 Gram in pA)
  a.A0 = df ? h->pP : h->pA; a.A1 = df ? h->pA : h->pP;
  a.F = h->pF; a.T = h->pT; a.S = h->pS;
  a.P = P; a.NJ = NJ; a.nsteps = (int)blk.steps.size();
  for (int j = 0; j < a.nsteps; ++j) {
    a.alpha[j] = blk.steps[j].first;
    a.beta[j] = blk.steps[j].second;
  }
  a.bar = reinterpret_cast<unsigned*>(h->iflags + 5);
  a.cnt = reinterpret_cast<unsigned*>(h->iflags + 8);
  a.err = h->iflags + 4;
  a.max_spin = h->opt.wait_polls;
  a.grid_share = h->profiling ? 1 : (int)h->lanes.size();
  a.shortcut = df ? shortcut : nullptr;
  cudaEvent_t ev[2];
  if (h->profiling) {
    cudaEventCreate(&ev[0]);
    cudaEventCreate(&ev[1]);
    cudaEventRecord(ev[0], h->stream);
  }
  const int n = polar_compose(a, h->stream, df);
  if (n < 0) {
    // the launch was refused: the flag turns the sweep into an error
    h->compose_refused = true;
    return;
  }
  h->launches += n;
  if (h->profiling) {
    cudaEventRecord(ev[1], h->stream);
    h->ev_pool.push_back(ev[0]);
    h->ev_pool.push_back(ev[1]);
    h->ev_flops.push_back({df ? 3 : 0, compose_flops(P, NJ, a.nsteps)});
    h->ev_bytes.push_back(0.0);
    h->ev_cond.push_back(a.shortcut);
  }
}

void polar(ttn_ctx* h, Instance& I, int t, int prec, const double* Gam) {
  const LayerView v = view(I, t, 0);
  const int P = v.P, NJ = v.NJ;
  const ll N = v.n2, PN = v.Pn2, PP = (ll)P * P;
  double* W = I.W[t];
  double* X = h->X;
  double* X2 = h->X2;
  // The polar factor is FP64 in every mode (the small singular directions
  // must not drown in tensor-core rounding).  FP64 mode, and layers too small
  // for the double-float products (P < 32, negligible cost): short blocks (at
  // most four composed steps per Gram matrix) for full accuracy; mixed modes
  // otherwise: two Gram matrices and two long compositions, then one more
  // Newton-Schulz step (adaptive: the second composition and the final step
  // become one Newton-Schulz step when the first block already converged).
  const int pb = h->opt.polar_blocks;
  const bool short_blocks = pb == 1 || ((pb == 0 || pb == 3 || pb == 4) && (prec == 0 || P < 32));
  const std::vector<PolarBlock>* schedp = short_blocks ? &h->polar_f64 : &h->polar_tc;
  // Mixed modes: every block's Gram and apply products in double-float
  // arithmetic on the FP32 pipes (~48 bits: the rounding amplified by a
  // block's growth stays far below the tensor-core rounding of the
  // environment), then one more Newton-Schulz step X <- (1.5 I - 0.5 X X^T) X
  // that takes the isometry defect from ~1e-11 to ~1e-14.  Operands in FP32
  // pairs, in the one-leg scratch Y and Yt (both free during the polar step).
  const bool df_ok = prec != 0 && h->opt.double_float && NJ == 1 && P >= 32 && schedp->size() > 1;
  // Adaptive schedule (polar_blocks 0 and 4 in the mixed modes, double-float
  // composition kernel): block 2 and the final step are cut short on the
  // device when block 1 already left an isometry (flag pfull[t] = 0).
  const bool adaptive = df_ok && !short_blocks && (pb == 0 || pb == 4) &&
                        h->polar_adapt.size() == 2 && (h->opt.persistent & 1) &&
                        compose_supported(P, (int)h->polar_adapt[0].steps.size()) &&
                        compose_supported(P, (int)h->polar_adapt[1].steps.size());
  if (adaptive) schedp = &h->polar_adapt;
  const std::vector<PolarBlock>& sched = *schedp;
  int* full = I.pfull + t;
  // polar_blocks 0: a layer predicted well conditioned first tries the short
  // first block (kPolarFirst); the full adaptive schedule then runs only when
  // that try did not leave an isometry (run_full, set on the device)
  const bool try_first = adaptive && pb == 0 && !h->polar_first.empty() &&
                         compose_supported(P, (int)h->polar_first[0].steps.size());
  const int nT = std::max(I.T, 1);
  int* try_flag = I.ppred + t;
  int* run_full = try_first ? I.ppred + nT + t : nullptr;
  if (df_ok && !h->measuring && !adaptive)
    h->launches += store_ints(full, nullptr, 1, 1, h->stream);
  // X as FP32 pairs for the double-float products (hi at Xp, lo at Xp + PN),
  // written by the kernel that produces X (the damped start, then every
  // apply), in two buffers that alternate like X and X2; F as pairs in Yt.
  // (Splitting X while the products load it was measured slower: the
  // products are issue-bound and the Gram product would split every element
  // four to five times.)
  float* Xp = reinterpret_cast<float*>(h->Y);
  float* Xp2 = reinterpret_cast<float*>(h->Y + PN);
  float* Fh = reinterpret_cast<float*>(h->Yt);
  float* Fl = Fh + PP;
  // the adaptive short path: D = 0.5 (I - X X^T) (FP32, in the composition's
  // scratch pT) and its correction D X (FP32, after F in Yt); X_short is the
  // last block's input
  float* Dc = reinterpret_cast<float*>(h->pT);
  float* Corr = Fh + 2 * PP;
  const double* X_short = X;
  const double* X_block = X;   // the long path's block-2 result
  if (!h->measuring) {
    // |Gamma|^2 and <Gamma, W> from one pass over Gamma (partial sums, completed
    // inside the polar start)
    h->launches += dot_self_and_cross_partial(Gam, W, PN, PN, NJ, h->red, h->stream);
    // (the adaptive schedule's flag starts at 0: the check before the last
    // block ORs 1 into it when that block and the final step must run)
    h->launches += polar_start(Gam, W, X, PN, NJ, P, h->opt.polar_damping, h->red, h->stream,
                               df_ok ? Xp : nullptr, df_ok ? Xp + PN : nullptr,
                               adaptive ? full : nullptr, try_first ? try_flag : nullptr,
                               run_full, adaptive ? I.pfar + t : nullptr);
  }
  // Mixed modes, layers with P < 32 (short blocks): the whole factor in one
  // CTA in pair arithmetic (small_polar) instead of a Gram, a composition and
  // an apply launch per block, then the update and its FP32 copy.
  int nsteps = 0;
  for (const auto& b : sched) nsteps += (int)b.steps.size();
  if (prec != 0 && short_blocks && NJ == 1 && (h->opt.persistent & 1) &&
      small_polar_supported(P, N, (int)sched.size(), nsteps)) {
    if (h->measuring) return;
    SmallPolarArgs sa;
    sa.X = X; sa.W = W; sa.W32 = I.w32[t];
    sa.P = P; sa.N = (int)N; sa.nblocks = (int)sched.size(); sa.sign = -1.0;
    int k = 0;
    for (size_t b = 0; b < sched.size(); ++b) {
      for (const auto& st : sched[b].steps) {
        sa.alpha[k] = st.first;
        sa.beta[k] = st.second;
        ++k;
      }
      sa.block_end[b] = k;
    }
    const int n = small_polar(sa, h->stream);
    if (n < 0) h->compose_refused = true;
    else h->launches += n;
    return;
  }
  if (df_ok && h->measuring)
    h->partial_cap = std::max<size_t>(h->partial_cap, (size_t)df_gram_splits(P, (int)N) * PP);
  if (try_first && !h->measuring) {
    // The first try (every launch returns at once unless *try_flag): Gram
    // matrix of X_0 (its pairs for the composition), the short block's
    // composition, X_A = F X_0 into X2 and Xp2 (X_0 stays in Xp for the full
    // schedule), and the Gram matrix of X_A with the test max |X_A X_A^T -
    // I| > kPolarNear (far: 1 into run_full) and D = 0.5 (I - X_A X_A^T) for
    // the correction.  When the try succeeds, every launch of the full
    // schedule below returns at once, block 1's swap leaves X_A where block
    // 1's result would be, and the short path's correction and the final
    // selection proceed as for a short path after block 1.
    GramCheck g0;
    g0.ph = reinterpret_cast<float*>(h->pP);
    g0.pl = g0.ph + PP;
    df_begin(h);
    df_end(h, df_gram(Xp, Xp + PN, P, N, h->pA, h->partial, h->stream, try_flag, &g0),
           df_gram_flops(P, N), try_flag);
    compose_block(h, h->polar_first[0], P, NJ, true, try_flag);
    const float* Fah = reinterpret_cast<const float*>(h->pF);
    df_begin(h);
    df_end(h, df_apply(Fah, Fah + PP, Xp, Xp + PN, P, N, X2, h->stream, try_flag, Xp2, Xp2 + PN),
           2.0 * P * P * (double)N, try_flag);
    GramCheck g1 = g0;
    g1.thr = kPolarNear;
    g1.flag = run_full;
    g1.d32 = Dc;
    df_begin(h);
    df_end(h, df_gram(Xp2, Xp2 + PN, P, N, h->pA, h->partial, h->stream, try_flag, &g1),
           df_gram_flops(P, N), try_flag);
  }
  for (size_t bi = 0; bi < sched.size(); ++bi) {
    const PolarBlock& blk = sched[bi];
    const bool df = df_ok && !h->measuring;
    const bool kernel = (h->opt.persistent & 1) && compose_supported(P, (int)blk.steps.size());
    if (df) {
      // with the composition kernel, the Gram product's reduction also writes
      // A_0 as pairs for it; before the adaptive schedule's last block also
      // the test max |X X^T - I| > kPolarNear (far: 1 into the flag, the
      // block and the final step run in full) and D = 0.5 (I - X X^T) in FP32
      // for the short path's correction
      GramCheck chk;
      chk.ph = reinterpret_cast<float*>(h->pP);
      chk.pl = chk.ph + PP;
      chk.thr = kPolarNear;
      if (adaptive && bi + 1 == sched.size()) {
        chk.flag = full;
        chk.d32 = Dc;
      }
      df_begin(h);
      df_end(h, df_gram(Xp, Xp + PN, P, N, h->pA, h->partial, h->stream, run_full,
                        kernel ? &chk : nullptr),
             df_gram_flops(P, N), run_full);
    } else {
    // A = X X^T (symmetric product: upper tiles computed, mirrored)
    GemmDesc g = desc(P, P, 1, NJ, h->pA, P, 1, 0, PP);
    add(g, grp(op(X, N, 1, 0, 0, PN), op(X, N, 1, 0, 0, PN), (int)N));
    g.sym = 1;
    run(h, g, 0);
    }
    // the flag that lets this block's launches run: run_full for block 1
    // after a first try, full for the adaptive schedule's last block
    const int* gate = adaptive && bi + 1 == sched.size() ? full : (bi == 0 ? run_full : nullptr);
    if (kernel) {
      if (!h->measuring) compose_block(h, blk, P, NJ, df, gate);
    } else {
    if (!h->measuring) h->launches += set_identity(h->pF, P, NJ, h->stream);
    for (size_t j = 0; j < blk.steps.size(); ++j) {
      if (!h->measuring)
        h->launches += poly_step_matrix(h->pA, h->pP, P, NJ, blk.steps[j].first,
                                        blk.steps[j].second, h->stream);
      // F <- Pm F ; T <- A Pm ; A <- Pm T
      GemmDesc a = desc(P, P, 1, NJ, h->pT, P, 1, 0, PP);
      add(a, grp(op(h->pP, P, 1, 0, 0, PP), op(h->pF, 1, P, 0, 0, PP), P));
      run(h, a, 0);
      if (!h->measuring) {
        cudaMemcpyAsync(h->pF, h->pT, NJ * PP * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
      }
      if (j + 1 < blk.steps.size()) {
        GemmDesc b = desc(P, P, 1, NJ, h->pT, P, 1, 0, PP);
        add(b, grp(op(h->pA, P, 1, 0, 0, PP), op(h->pP, 1, P, 0, 0, PP), P));
        run(h, b, 0);
        GemmDesc c = desc(P, P, 1, NJ, h->pA, P, 1, 0, PP);
        add(c, grp(op(h->pP, P, 1, 0, 0, PP), op(h->pT, 1, P, 0, 0, PP), P));
        run(h, c, 0);
        if (!h->measuring) h->launches += symmetrize(h->pA, P, NJ, h->stream);
      }
    }
    }
    // X2 = F X ; swap.  F amplifies the small singular directions by up to
    // 1/damping, so this product is FP64 (or double-float) in every mode (a
    // tensor-core product of it would lose those directions to cancellation).
    if (df) {
      // F as pairs: straight from the double-float composition, else split
      const float* Fah = reinterpret_cast<const float*>(h->pF);
      const float* Fal = Fah + PP;
      if (!kernel) {
        h->launches += df_split(h->pF, Fh, Fl, PP, h->stream);
        Fah = Fh;
        Fal = Fl;
      }
      // the adaptive schedule's last block: the composed F (full == 1) or one
      // Newton-Schulz step from the Gram matrix still in pA (full == 0)
      const int* cut = gate;
      df_begin(h);
      df_end(h, df_apply(Fah, Fal, Xp, Xp + PN, P, N, X2, h->stream, cut, Xp2, Xp2 + PN),
             2.0 * P * P * (double)N, cut);
    } else {
    GemmDesc f = desc(P, (int)N, 1, NJ, X2, N, 1, 0, PN);
    add(f, grp(op(h->pF, P, 1, 0, 0, PP), op(X, 1, N, 0, 0, PN), P));
    run(h, f, 0);
    }
    if (adaptive && bi + 1 == sched.size()) {
      // short path (full == 0): the block is one Newton-Schulz step,
      // X + 0.5 (I - X X^T) X; its correction D X (entries <= 5e-10 of X)
      // needs FP32 accuracy only: a 3xTF32 tensor-core product on X's FP32
      // head, added to X in FP64 when W is written (skipped when full == 1)
      GemmDesc c = desc(P, (int)N, 1, 1, TP{Corr, 1}, N, 1, 0, 0);
      add(c, grp(op(TP{Dc, 1}, P, 1), op(TP{Xp, 1}, 1, N), P));
      c.skip = full;
      run(h, c, TTN_TF32X3);
      X_short = X;
    }
    std::swap(X, X2);
    std::swap(Xp, Xp2);
  }
  if (df_ok && !h->measuring) {
    // (cut short: these products return at once; the defect flag below then
    // reads the last block's Gram matrix, within kPolarNear of I)
    // F = 1.5 I - 0.5 X X^T as pairs, from the Gram product's reduction; the
    // final step converges quadratically only from |X X^T - I| << 1, so the
    // same pass flags the instance when the blocks left it above 1e-5 (the
    // isometry would then miss 1e-10).  Cut short, the pass is skipped with
    // the product: the last block's Gram matrix is then within kPolarNear of I.
    GramCheck fin;
    fin.a = 1.5;
    fin.c = 0.5;
    fin.ph = Fh;
    fin.pl = Fl;
    fin.thr = 1e-5;
    fin.flag = I.istat + 4;
    // adaptive schedule: when block 2 left X X^T within kPolarNear of I (far
    // stays 0), the final step is the same FP32 correction as the short
    // path's, D X on the tensor cores with D = 0.5 (I - X X^T) from this pass;
    // otherwise the double-float step runs
    int* far = adaptive ? I.pfar + t : nullptr;
    if (adaptive) {
      fin.thr2 = kPolarNear;
      fin.flag2 = far;
      fin.d32 = Dc;
    }
    df_begin(h);
    df_end(h, df_gram(Xp, Xp + PN, P, N, h->pA, h->partial, h->stream, full, &fin),
           df_gram_flops(P, N), full);
    X_block = X;
    if (adaptive) {
      // (runs whenever the long path runs; unused when far is set)
      GemmDesc c = desc(P, (int)N, 1, 1, TP{Corr, 1}, N, 1, 0, 0);
      add(c, grp(op(TP{Dc, 1}, P, 1), op(TP{Xp, 1}, 1, N), P));
      c.skip = full;
      c.skip_when_zero = 1;
      run(h, c, TTN_TF32X3);
    }
    const int* run_final = adaptive ? far : full;
    df_begin(h);
    df_end(h, df_apply(Fh, Fl, Xp, Xp + PN, P, N, X2, h->stream, run_final),
           2.0 * P * P * (double)N, run_final);
    std::swap(X, X2);
  }
  if (!h->measuring) {
    if (df_ok) {
      // W and its FP32 copy for the tensor-core products in one pass: from the
      // final step's result (full == 1), or from the last block's input plus
      // the short path's correction (full == 0)
      // (adaptive, long path: block 2's result plus the correction, or the
      // double-float final step's result when block 2 was left far)
      h->launches += scale_select(adaptive ? X_short : X, adaptive ? X_block : X, full, W,
                                  NJ * PN, -1.0, h->stream, I.w32[t], adaptive ? Corr : nullptr,
                                  try_first ? try_flag : nullptr, nT, kPolarRetry,
                                  adaptive ? X : nullptr, adaptive ? I.pfar + t : nullptr);
    } else {
      h->launches += axpby(X, W, NJ * PN, -1.0, 0.0, h->stream);
      if (prec != 0) h->launches += to_f32(W, I.w32[t], NJ * PN, h->stream);
    }
  }
}

// Adjoints of site layer t from those of t+1 through (new) w_t.
void descend(ttn_ctx* h, Instance& I, int t, int prec) {
  const LayerView v = view(I, t, prec);
  const int K = I.K;
  const TP W = v.W;
  const ll slab = (ll)v.NJ * v.Pn2;
  const ll PP = (ll)v.P * v.P;
  const TP Yt = scratch(h->Yt, v);     // [j][J] G_j W
  StageFork fk(h);
  fk.branch(0);
  {
    GemmDesc d = desc(v.P, (int)v.n2, 1 + 2 * K, v.NJ, Yt, v.n2, 1, slab, v.Pn2);
    add(d, grp(op(v.adj, v.P, 1, 0, PP, v.adj_ss), op(W, 1, v.n2, 0, 0, v.Pn2), v.P));
    run(h, d, prec);
  }
  const TP WB = scratch(h->M1, v);     // W B_{k,R}
  const TP AW = WB + K * slab;         // A_{k,L}^T W
  fk.branch(1);
  right_mult(h, v, W, v.opsR, 1 + K, K, false, WB, slab, prec);
  fk.branch(2);
  left_mult(h, v, W, v.opsL, 1, K, false, AW, slab, prec);
  fk.join();
  // trace_r(T, Y)[l,l'] = sum_{p,r} T[p,l,r] Y[p,l',r];  trace_l(T, Y)[r,r'] = sum_{p,l} T[p,l,r] Y[p,l,r']
  auto tr_r = [&](TP Tt, ll tb0, TP Y, ll yb0) {
    return grp(op(Tt, v.n, 1, v.n2, tb0, v.Pn2), op(Y, v.n, 1, v.n2, yb0, v.Pn2), v.n, v.P);
  };
  auto tr_l = [&](TP Tt, ll tb0, TP Y, ll yb0) {
    return grp(op(Tt, 1, v.n, v.n2, tb0, v.Pn2), op(Y, 1, v.n, v.n2, yb0, v.Pn2), v.n, v.P);
  };
  double* out = I.adj[t];    // FP64 output
  const ll n2 = v.n2;
  if (!I.per_node) {
    StageFork fk2(h);          // the three traces are independent
    fk2.branch(0);
    GemmDesc r = desc(v.n, v.n, 1, 1, out, v.n, 1, 0, 0);
    add(r, tr_r(W, 0, Yt, 0));
    add(r, tr_l(W, 0, Yt, 0));
    run(h, r, prec);
    fk2.branch(1);
    GemmDesc p = desc(v.n, v.n, K, 1, out + n2, v.n, 1, n2, 0);
    add(p, tr_r(WB, slab, Yt, 0));
    add(p, tr_l(W, 0, Yt + slab, slab));
    run(h, p, prec);
    fk2.branch(2);
    GemmDesc q = desc(v.n, v.n, K, 1, out + (1 + K) * n2, v.n, 1, n2, 0);
    add(q, tr_l(AW, slab, Yt, 0));
    add(q, tr_r(W, 0, Yt + (1 + K) * slab, slab));
    run(h, q, prec);
    fk2.join();
  } else {
    const ll ss = v.ss;
    double* outL = out;          // site 2J
    double* outR = out + ss;     // site 2J+1
    const ll so = 2 * ss;        // per node
    GemmDesc r1 = desc(v.n, v.n, 1, v.NJ, outL, v.n, 1, 0, so);
    add(r1, tr_r(W, 0, Yt, 0));
    run(h, r1, prec);
    GemmDesc r2 = desc(v.n, v.n, 1, v.NJ, outR, v.n, 1, 0, so);
    add(r2, tr_l(W, 0, Yt, 0));
    run(h, r2, prec);
    GemmDesc p1 = desc(v.n, v.n, K, v.NJ, outL + n2, v.n, 1, n2, so);
    add(p1, tr_r(WB, slab, Yt, 0));
    run(h, p1, prec);
    GemmDesc p2 = desc(v.n, v.n, K, v.NJ, outR + n2, v.n, 1, n2, so);
    add(p2, tr_l(W, 0, Yt + slab, slab));
    run(h, p2, prec);
    GemmDesc q1 = desc(v.n, v.n, K, v.NJ, outR + (1 + K) * n2, v.n, 1, n2, so);
    add(q1, tr_l(AW, slab, Yt, 0));
    run(h, q1, prec);
    GemmDesc q2 = desc(v.n, v.n, K, v.NJ, outL + (1 + K) * n2, v.n, 1, n2, so);
    add(q2, tr_r(W, 0, Yt + (1 + K) * slab, slab));
    run(h, q2, prec);
  }
  if (v.f32 && !h->measuring) h->launches += to_f32(I.adj[t], I.adj32[t], I.op_elems(t), h->stream);
}

void forward(ttn_ctx* h, Instance& I, int prec) {
  if (prec != 0 && !h->measuring) {
    // FP32 copies of the layer-0 operators and of every isometry
    h->launches += to_f32(I.ops[0], I.ops32[0], I.op_elems(0), h->stream);
    for (int t = 0; t < I.T; ++t) h->launches += to_f32(I.W[t], I.w32[t], I.w_elems(t), h->stream);
  }
  for (int t = 0; t < I.T; ++t) ascend_layer(h, I, t, prec);
}

void sweep_instance(ttn_ctx* h, Instance& I) {
  const int prec = h->opt.prec;
  if (!h->measuring) h->launches += store_ints(I.istat + 4, nullptr, 1, 0, h->stream);
  forward(h, I, prec);
  top_solve(h, I, I.E);
  top_adjoints(h, I);
  if (prec != 0 && !h->measuring)
    h->launches += to_f32(I.adj[I.T], I.adj32[I.T], I.op_elems(I.T), h->stream);
  for (int t = I.T - 1; t >= 0; --t) {
    ensure_ops(h, I, t, prec);
    environment(h, I, t, prec, h->Gam);
    polar(h, I, t, prec, h->Gam);
    descend(h, I, t, prec);
  }
  // energy change per spin of this sweep (Sec. IV convergence test)
  if (!h->measuring)
    h->launches += sweep_delta(I.E, I.dstat, I.istat, 1.0 / I.n_spins, h->stream);
}

// Gram matrices W W^T of every isometry layer (FP64), each followed by its
// statistics (trace, max |W W^T - I|, asymmetry) at res + 3 t.
void isometry_grams(ttn_ctx* h, Instance& I, double* res) {
  for (int t = 0; t < I.T; ++t) {
    const LayerView v = view(I, t, 0);
    const ll PP = (ll)v.P * v.P;
    GemmDesc g = desc(v.P, v.P, 1, v.NJ, h->pA, v.P, 1, 0, PP);
    add(g, grp(op(I.W[t], v.n2, 1, 0, 0, v.Pn2), op(I.W[t], v.n2, 1, 0, 0, v.Pn2), (int)v.n2));
    g.sym = 1;
    run(h, g, 0);
    if (!h->measuring) h->launches += mat_stats(h->pA, v.P, v.NJ, PP, 1, res + 3 * t, h->stream);
  }
}

// Adjoints of every site layer at the stored tensors (no update).
void adjoints_only(ttn_ctx* h, Instance& I, int down_to) {
  forward(h, I, 0);
  top_adjoints(h, I);
  for (int t = I.T - 1; t >= down_to; --t) {
    ensure_ops(h, I, t, 0);
    descend(h, I, t, 0);
  }
}

// Energy of the stored tensors and, with grad != nullptr, its derivative with
// respect to every tensor (laid out as ttn_env with layer -1), with the
// contractions of the ascend, environment and descend in precision prec (the
// top contraction, the top adjoints and the energy FP64).
void value_and_grad(ttn_ctx* h, Instance& I, int prec, double* energy_out, double* grad) {
  forward(h, I, prec);
  energy_only(h, I, energy_out);
  if (!grad) return;
  const ll c2 = (ll)I.chis[I.T] * I.chis[I.T];
  size_t off = 0;
  for (int t = 0; t < I.T; ++t) off += I.w_elems(t);
  if (!h->measuring) {
    top_matvec(h, I, I.V, h->lz_w, nullptr);
    h->launches += top_grad(grad + off, h->lz_w, I.V, c2, I.eoff[I.T], I.per_node ? 1 : 0,
                            h->stream);
  } else {
    top_matvec(h, I, I.V, h->lz_w, nullptr);
  }
  top_adjoints(h, I);
  if (prec != 0 && !h->measuring)
    h->launches += to_f32(I.adj[I.T], I.adj32[I.T], I.op_elems(I.T), h->stream);
  for (int t = I.T - 1; t >= 0; --t) {
    off -= I.w_elems(t);
    ensure_ops(h, I, t, prec);
    environment(h, I, t, prec, h->Gam);
    if (!h->measuring)
      cudaMemcpyAsync(grad + off, h->Gam, I.w_elems(t) * sizeof(double), cudaMemcpyDeviceToDevice,
                      h->stream);
    if (t > 0) descend(h, I, t, prec);
  }
}

// Plan all scratch sizes (pass with base == nullptr) or carve them.
void layout(ttn_ctx* h, Arena& ar) {
  size_t slab_max = 0, pp_max = 0, c2_max = 0, nj_max = 1;
  int K_max = 1;
  for (Instance& I : h->inst) {
    I.W.assign(I.T, nullptr);
    I.ops.assign(I.T + 1, nullptr);
    I.adj.assign(I.T + 1, nullptr);
    I.w32.assign(I.T, nullptr);
    I.ops32.assign(I.T + 1, nullptr);
    I.adj32.assign(I.T + 1, nullptr);
    for (int t = 0; t < I.T; ++t) {
      I.W[t] = ar.take(I.w_elems(t));
      if (h->opt.prec != 0) I.w32[t] = reinterpret_cast<float*>(ar.take((I.w_elems(t) + 1) / 2));
      slab_max = std::max(slab_max, I.w_elems(t));
      pp_max = std::max(pp_max, (size_t)I.nodes(t) * I.chis[t + 1] * I.chis[t + 1]);
      nj_max = std::max(nj_max, (size_t)I.nodes(t));
    }
    I.eoff.assign(I.T + 1, nullptr);
    const bool rec = h->opt.recompute_ops != 0;
    size_t pp_elems = 0;
    for (int t = 1; t < I.T; ++t) pp_elems = std::max(pp_elems, I.op_elems(t));
    double* pp[2] = {nullptr, nullptr};
    float* pp32[2] = {nullptr, nullptr};
    if (rec && pp_elems) {
      for (int b = 0; b < 2; ++b) {
        pp[b] = ar.take(pp_elems);
        if (h->opt.prec != 0) pp32[b] = reinterpret_cast<float*>(ar.take((pp_elems + 1) / 2));
      }
    }
    I.pp_holds[0] = I.pp_holds[1] = -1;
    for (int t = 0; t <= I.T; ++t) {
      const bool shared = rec && t > 0 && t < I.T;
      I.ops[t] = shared ? pp[t & 1] : ar.take(I.op_elems(t));
      I.adj[t] = ar.take(I.op_elems(t));
      I.eoff[t] = ar.take(I.sites(t));
      if (h->opt.prec != 0) {
        I.ops32[t] = shared ? pp32[t & 1] : reinterpret_cast<float*>(ar.take((I.op_elems(t) + 1) / 2));
        I.adj32[t] = reinterpret_cast<float*>(ar.take((I.op_elems(t) + 1) / 2));
      }
    }
    const int c = I.chis[I.T];
    I.V = ar.take((size_t)c * c);
    I.Vprev = ar.take((size_t)c * c);
    I.E = ar.take(4);
    I.dstat = ar.take(4);
    I.istat = ar.take_int(8);
    I.pfull = ar.take_int(std::max(I.T, 1));
    I.ppred = ar.take_int(3 * std::max(I.T, 1));
    I.pfar = ar.take_int(std::max(I.T, 1));
    c2_max = std::max(c2_max, (size_t)c * c);
    K_max = std::max(K_max, I.K);
  }
  // scratch of every lane (a full copy each: lanes run concurrently)
  for (size_t k = 0; k < h->lanes.size(); ++k) {
    h->Y = ar.take((1 + 4 * K_max) * slab_max);
    h->Yt = ar.take((1 + 2 * K_max) * slab_max);
    h->M1 = ar.take(2 * K_max * slab_max);
    h->Gam = ar.take(slab_max);
    h->X = ar.take(slab_max);
    h->X2 = ar.take(slab_max);
    h->pA = ar.take(pp_max);
    h->pF = ar.take(pp_max);
    h->pP = ar.take(pp_max);
    h->pT = ar.take(pp_max);
    h->pS = ar.take(pp_max);
    h->red = ar.take(std::max<size_t>(kDotBlocks * (h->lz_m + 2), kDotBlocks * nj_max * 2));
    h->scal = ar.take(16 + 2 * nj_max);
    h->lz_basis = ar.take((h->lz_m + 1) * c2_max);
    h->lz_w = ar.take(c2_max);
    h->lz_tmp = ar.take(2 * K_max * c2_max);
    h->lz_c1 = ar.take(h->lz_m + 2);
    h->lz_c2 = ar.take(h->lz_m + 2);
    h->lz_alpha = ar.take(h->lz_m + 2);
    h->lz_beta = ar.take(h->lz_m + 2);
    h->lz_y = ar.take(h->lz_m + 2);
    h->top_stack0 = ar.take((1 + 2 * K_max) * c2_max);
    h->top_stack1 = ar.take((1 + 2 * K_max) * c2_max);
    h->lz_part = ar.take((size_t)(kLMaxGrid + 2) * (h->lz_m + 2));
    if (h->opt.prec != 0) {
      h->lz_opsp = ar.take(2 * (1 + 2 * K_max) * c2_max);
      h->lz_bp = ar.take((h->lz_m + 1) * c2_max);
      h->lz_Yp = ar.take(2 * K_max * c2_max);
    }
    h->iflags = ar.take_int(8 + 3 * kComposeMaxTiles);
    h->partial = ar.take(h->partial_cap);
    const int ss = h->opt.stage_streams == 0 ? (h->lanes.size() == 1 ? kSubStreams : 1)
                                             : h->opt.stage_streams;
    h->sub.n = ss > 1 ? std::min(ss, kSubStreams) : 0;
    for (int i = 0; i < h->sub.n; ++i) h->sub.partial[i] = ar.take(h->partial_cap);
    save_lane(h, h->lanes[k]);
  }
  h->E_hist = ar.take(4096 * h->inst.size() + 16);
  load_lane(h, h->lanes[0]);
}

int fail(ttn_ctx* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

int check_cuda(ttn_ctx* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TTN_OK;
  return fail(h, TTN_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int build_instances(ttn_ctx* h, const ttn_problem* probs, int n) {
  for (int i = 0; i < n; ++i) {
    const ttn_problem& p = probs[i];
    if (p.Lx < 4 || !is_pow2(p.Lx) || p.Ly < 1 || p.d < 2 || p.chi < 1 || p.K < 1 || p.K > 7 ||
        !p.onesite || !p.A || !p.B)
      return fail(h, TTN_EINVAL, "problem " + std::to_string(i) + ": bad shape or null terms");
    Instance I;
    I.L = p.Lx; I.Ly = p.Ly; I.K = p.K; I.per_node = p.per_node ? 1 : 0; I.chi = p.chi;
    double d0f = std::pow((double)p.d, p.Ly);
    if (d0f > 4096) return fail(h, TTN_EINVAL, "d^Ly too large");
    I.d0 = (int)d0f;
    if (!is_pow2(I.d0)) return fail(h, TTN_EINVAL, "d^Ly must be a power of two");
    I.n_spins = p.Lx * p.Ly;
    I.T = ilog2(p.Lx) - 1;
    I.chis.push_back(I.d0);
    for (int t = 0; t < I.T; ++t) {
      long long sq = (long long)I.chis.back() * I.chis.back();
      I.chis.push_back((int)std::min<long long>(p.chi, sq));
    }
    for (int c : I.chis)
      if (!is_pow2(c)) return fail(h, TTN_EINVAL, "bond dimensions must be powers of two");
    if (I.chis.back() * (long long)I.chis.back() > (1 << 20))
      return fail(h, TTN_EINVAL, "top tensor too large");
    const size_t d2 = (size_t)I.d0 * I.d0;
    I.o.assign(p.onesite, p.onesite + d2);
    I.A.assign(p.A, p.A + d2 * p.K);
    I.B.assign(p.B, p.B + d2 * p.K);
    for (double x : I.o) if (!std::isfinite(x)) return fail(h, TTN_ENAN, "non-finite one-site term");
    for (double x : I.A) if (!std::isfinite(x)) return fail(h, TTN_ENAN, "non-finite product term");
    for (double x : I.B) if (!std::isfinite(x)) return fail(h, TTN_ENAN, "non-finite product term");
    const double sh = h->opt.shift;
    I.c = std::isnan(sh) ? bond_lambda_max(I.o.data(), I.A.data(), I.B.data(), I.d0, I.K) : sh;
    h->inst.push_back(I);
  }
  return TTN_OK;
}

void plan(ttn_ctx* h) {
  h->measuring = true;
  h->partial_cap = 0;
  for (Instance& I : h->inst) {
    sweep_instance(h, I);
    adjoints_only(h, I, 0);
    energy_only(h, I, nullptr);
    isometry_grams(h, I, nullptr);
    value_and_grad(h, I, h->opt.prec, nullptr, h->Gam);
  }
  h->measuring = false;
}

void setup_schedules(ttn_ctx* h) {
  const double l0 = std::max(h->opt.polar_damping * 0.25, 1e-300);
  // At most four composed steps (growth <= 30) per fresh Gram matrix: longer
  // compositions lose accuracy on the small singular directions.
  h->polar_f64 = polar_schedule(l0, 30.0, 1e-15, 4);
  // mixed modes: two blocks -- one long composition for the growth of the
  // small singular values (its ~1e-8 loss of accuracy on those directions is
  // below the rounding of the tensor-core contractions around it), then a
  // fresh Gram matrix for the well-conditioned convergence to an exact
  // isometry.  The tensor-core rounding of the environment (up to 1e-4 in
  // TF32) can take singular values of the damped environment below mu |Gamma|
  // (measured: the top isometry layer of the 64 x 4 torus in TF32, by small
  // factors), so the schedule starts at min(mu / 4, 1e-10): six more steps,
  // the same two Gram matrices (growth up to 1e6 per block, ~3e-9 relative
  // in double-float arithmetic)
  h->polar_tc = polar_schedule(std::min(l0, 1e-10), 1e6, 1e-15, 1000);
  // Adaptive variant (mixed modes): block 1 is the full schedule from
  // kPolarTry (it converges every singular value above it); block 2 assumes
  // the worst case again -- the image of the same lower bound under block 1's
  // polynomials -- and, when it fits one block, is replaced on the device by a
  // single Newton-Schulz step whenever block 1 already left X X^T within
  // kPolarNear of I (then the final step is not needed either).
  h->polar_adapt.clear();
  const std::vector<PolarBlock> first = polar_schedule(kPolarTry, 1e300, 1e-15, 1000);
  if (first.size() == 1) {
    double l = std::min(l0, 1e-10);
    for (const auto& st : first[0].steps) l = st.first * l - st.second * l * l * l;
    const std::vector<PolarBlock> second = polar_schedule(l, 1e6, 1e-15, 1000);
    if (second.size() == 1 && (int)first[0].steps.size() <= kMaxComposeSteps &&
        (int)second[0].steps.size() <= kMaxComposeSteps)
      h->polar_adapt = {first[0], second[0]};
  }
  h->polar_first.clear();
  const std::vector<PolarBlock> well = polar_schedule(kPolarFirst, 1e300, 1e-15, 1000);
  if (well.size() == 1 && (int)well[0].steps.size() <= kMaxComposeSteps) h->polar_first = well;
}

}  // namespace

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------

extern "C" {

void ttn_default_options(ttn_options* o) {
  if (!o) return;
  o->prec = TTN_FP64;
  o->top_mode = 0;
  o->lanczos_tol = 0.0;
  o->lanczos_max = 48;
  o->lanczos_restarts = 3;
  o->shift = NAN;
  o->polar_damping = 1e-7;
  o->deterministic = 1;
  o->use_graph = 1;
  o->persistent = 3;
  o->streams = 8;
  o->polar_blocks = 0;
  o->double_float = 1;
  o->tc_engine = 0;
  o->wait_polls = 0;
  o->tiles = nullptr;
  o->tiles_bytes = 0;
  o->recompute_ops = 0;
  o->stage_streams = 0;
}

// Parse an autotuner blob (ttn_options.tiles) into the table.
static int load_tiles(ttn_ctx* h, const void* blob, size_t bytes) {
  if (!blob || bytes == 0) return TTN_OK;
  if (bytes < sizeof(TuneBlobHeader)) return fail(h, TTN_EINVAL, "tiles blob too short");
  TuneBlobHeader hd;
  std::memcpy(&hd, blob, sizeof(hd));
  if (std::memcmp(hd.magic, "TTNT", 4) != 0 || hd.version != 2 ||
      bytes < sizeof(hd) + (size_t)hd.count * sizeof(TuneBlobEntry))
    return fail(h, TTN_EINVAL, "not a tiles blob of this library");
  const char* p = static_cast<const char*>(blob) + sizeof(hd);
  for (uint32_t i = 0; i < hd.count; ++i) {
    TuneBlobEntry e;
    std::memcpy(&e, p + i * sizeof(e), sizeof(e));
    if (e.engine < 0 || e.engine > 1 || e.splits < 1 || e.splits > 128 || e.occ < 0 ||
        e.occ > 2 || !(e.tile == 0 || e.tile == 16 || e.tile == 32 || e.tile == 64 || e.tile == 128))
      return fail(h, TTN_EINVAL, "tiles blob entry out of range");
    h->tuned[e.key] = Tuned{e.engine, e.tile, e.splits, e.occ, e.ms};
  }
  return TTN_OK;
}

// Instances go to min(streams, instances) lanes, longest first onto the least
// loaded lane (cost ~ the chi^4 contractions of a sweep plus its Lanczos).
static void assign_lanes(ttn_ctx* h) {
  const int ni = (int)h->inst.size();
  const int nl = std::max(1, std::min(h->opt.streams, ni));
  h->lanes.assign(nl, Lane());
  h->lane_of.assign(ni, 0);
  std::vector<std::pair<double, int>> cost;
  for (int i = 0; i < ni; ++i) {
    const Instance& I = h->inst[i];
    double c = 0.0;
    for (int t = 0; t < I.T; ++t)
      c += (double)I.nodes(t) * I.chis[t + 1] * std::pow((double)I.chis[t], 3) * (1 + 2 * I.K);
    c += 150.0 * std::pow((double)I.chis[I.T], 3) * (1 + 2 * I.K);
    cost.push_back({c, i});
  }
  std::stable_sort(cost.begin(), cost.end(),
                   [](const std::pair<double, int>& a, const std::pair<double, int>& b) {
                     return a.first > b.first;
                   });
  std::vector<double> load(nl, 0.0);
  for (const auto& ci : cost) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    h->lane_of[ci.second] = k;
    load[k] += ci.first;
  }
}

static int prepare(ttn_ctx* h, const ttn_problem* probs, int n, const ttn_options* opt) {
  if (!probs || n <= 0) return fail(h, TTN_EINVAL, "no problems");
  if (opt) h->opt = *opt; else ttn_default_options(&h->opt);
  if (h->opt.prec < 0 || h->opt.prec > 4) return fail(h, TTN_EINVAL, "bad precision");
  if (h->opt.top_mode != 0 && h->opt.top_mode != 1) return fail(h, TTN_EINVAL, "top_mode is 0 or 1");
  if (h->opt.lanczos_max < 2 || h->opt.lanczos_max > 120) return fail(h, TTN_EINVAL, "lanczos_max in [2,120]");
  if (h->opt.lanczos_restarts < 1) h->opt.lanczos_restarts = 1;
  if (!(h->opt.polar_damping >= 0.0)) return fail(h, TTN_EINVAL, "polar_damping < 0");
  if (h->opt.wait_polls < 0) return fail(h, TTN_EINVAL, "wait_polls < 0");
  if (h->opt.tc_engine != 0 && h->opt.tc_engine != 1) return fail(h, TTN_EINVAL, "tc_engine is 0 or 1");
  if (h->opt.stage_streams < 0 || h->opt.stage_streams > kSubStreams)
    return fail(h, TTN_EINVAL, "stage_streams in [0, 3]");
  h->lz_m = h->opt.lanczos_max;
  int rc = load_tiles(h, h->opt.tiles, h->opt.tiles_bytes);
  if (rc) return rc;
  h->opt.tiles = nullptr;   // copied: the caller's blob is not kept
  h->opt.tiles_bytes = 0;
  rc = build_instances(h, probs, n);
  if (rc) return rc;
  if (h->opt.streams < 1 || h->opt.streams > 64) return fail(h, TTN_EINVAL, "streams in [1,64]");
  if (h->opt.polar_blocks < 0 || h->opt.polar_blocks > 4)
    return fail(h, TTN_EINVAL, "polar_blocks is 0, 1, 2, 3 or 4");
  assign_lanes(h);
  setup_schedules(h);
  Arena a0;
  a0.base = reinterpret_cast<char*>((size_t)1 << 40);   // fake address, never dereferenced
  a0.registry = &h->registry;
  layout(h, a0);          // sizes of everything but the partial buffer
  plan(h);                // partial buffer size; bounds of every product
  h->registry.clear();
  if (!h->bounds_error.empty()) return fail(h, TTN_EINVAL, "internal bounds check: " + h->bounds_error);
  return TTN_OK;
}

size_t ttn_workspace_bytes(const ttn_problem* probs, int n, const ttn_options* opt) {
  ttn_ctx tmp;
  if (prepare(&tmp, probs, n, opt)) return 0;
  Arena a;
  layout(&tmp, a);
  return a.off + 256;
}

int ttn_create(ttn_t* out, const ttn_problem* probs, int n, const ttn_options* opt, void* d_ws,
               size_t bytes, void* stream) {
  if (!out) return TTN_EINVAL;
  *out = nullptr;
  ttn_ctx* h = new ttn_ctx();
  int rc = prepare(h, probs, n, opt);
  if (rc) { *out = h; return rc; }
  Arena a;
  layout(h, a);
  if (!d_ws || bytes < a.off) { *out = h; return fail(h, TTN_ENOMEM, "workspace too small: need " + std::to_string(a.off)); }
  Arena real;
  real.base = reinterpret_cast<char*>(d_ws);
  layout(h, real);
  h->user = reinterpret_cast<cudaStream_t>(stream);
  gemm_tc_init();
  rc = check_cuda(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "stream");
  h->lanes[0].stream = h->stream;
  h->ev_join.assign(h->lanes.size(), nullptr);
  if (!rc && h->lanes.size() > 1)
    rc = check_cuda(h, cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "event");
  for (size_t k = 1; k < h->lanes.size() && !rc; ++k) {
    rc = check_cuda(h, cudaStreamCreateWithFlags(&h->lanes[k].stream, cudaStreamNonBlocking),
                    "stream");
    if (!rc)
      rc = check_cuda(h, cudaEventCreateWithFlags(&h->ev_join[k], cudaEventDisableTiming), "event");
  }
  // sub-streams of every lane for the independent products of a stage
  for (size_t k = 0; k < h->lanes.size() && !rc; ++k) {
    SubStreams& sb = h->lanes[k].sub;
    if (!sb.n) continue;
    rc = check_cuda(h, cudaEventCreateWithFlags(&sb.fork, cudaEventDisableTiming), "event");
    for (int i = 0; i < sb.n && !rc; ++i) {
      rc = check_cuda(h, cudaStreamCreateWithFlags(&sb.s[i], cudaStreamNonBlocking), "stream");
      if (!rc) rc = check_cuda(h, cudaEventCreateWithFlags(&sb.join[i], cudaEventDisableTiming), "event");
    }
  }
  if (!rc) load_lane(h, h->lanes[0]);
  for (size_t k = 0; k < h->lanes.size() && !rc; ++k)
    rc = check_cuda(h, cudaMemsetAsync(h->lanes[k].iflags, 0, 8 * sizeof(int), h->stream), "flags");
  for (size_t i = 0; i < h->inst.size() && !rc; ++i) {
    rc = check_cuda(h, cudaMemsetAsync(h->inst[i].istat, 0, 8 * sizeof(int), h->stream), "status");
    if (!rc)
      rc = check_cuda(h, cudaMemsetAsync(h->inst[i].dstat, 0, 4 * sizeof(double), h->stream), "status");
    if (!rc) {
      // no polar block cut short yet; every layer first tries the
      // well-conditioned first block
      const int nT = std::max(h->inst[i].T, 1);
      h->launches += store_ints(h->inst[i].pfull, nullptr, nT, 1, h->stream);
      h->launches += store_ints(h->inst[i].ppred, nullptr, 2 * nT, 1, h->stream);
      h->launches += store_ints(h->inst[i].ppred + 2 * nT, nullptr, nT, 0, h->stream);
      rc = check_cuda(h, cudaPeekAtLastError(), "status");
    }
  }
  if (rc) { *out = h; return rc; }
  // upload operators of site layer 0 (shifted one-site term)
  for (Instance& I : h->inst) {
    const size_t d2 = (size_t)I.d0 * I.d0;
    std::vector<double> host((size_t)(1 + 2 * I.K) * d2);
    for (size_t e = 0; e < d2; ++e) host[e] = I.o[e];
    double tr = 0.0;
    for (int i = 0; i < I.d0; ++i) tr += I.o[(size_t)i * I.d0 + i];
    const double e0 = tr / I.d0 - I.c;   // o - c I = (o - tr/d0 I) + e0 I
    for (int i = 0; i < I.d0; ++i) host[(size_t)i * I.d0 + i] -= tr / I.d0;
    std::vector<double> e0s(I.sites(0), e0);
    rc = check_cuda(h, cudaMemcpyAsync(I.eoff[0], e0s.data(), e0s.size() * sizeof(double),
                                       cudaMemcpyHostToDevice, h->stream), "upload");
    if (rc) { *out = h; return rc; }
    std::memcpy(host.data() + d2, I.A.data(), I.K * d2 * sizeof(double));
    std::memcpy(host.data() + (1 + I.K) * d2, I.B.data(), I.K * d2 * sizeof(double));
    for (int s = 0; s < I.sites(0); ++s) {
      rc = check_cuda(h, cudaMemcpyAsync(I.ops[0] + s * host.size(), host.data(),
                                         host.size() * sizeof(double), cudaMemcpyHostToDevice,
                                         h->stream), "upload");
      if (rc) { *out = h; return rc; }
    }
  }
  rc = check_cuda(h, cudaStreamSynchronize(h->stream), "create sync");
  *out = h;
  return rc;
}

int ttn_sizes(ttn_t h, int inst, size_t* n_w, size_t* n_v, int* n_layers) {
  if (!h || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  const Instance& I = h->inst[inst];
  size_t s = 0;
  for (int t = 0; t < I.T; ++t) s += I.w_elems(t);
  if (n_w) *n_w = s;
  if (n_v) *n_v = (size_t)I.chis[I.T] * I.chis[I.T];
  if (n_layers) *n_layers = I.T;
  return TTN_OK;
}

int ttn_chis(ttn_t h, int inst, int* chis) {
  if (!h || !chis || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  const Instance& I = h->inst[inst];
  for (int t = 0; t <= I.T; ++t) chis[t] = I.chis[t];
  return TTN_OK;
}

static int sync_user(ttn_ctx* h) {
  // order: work on the library stream starts after what the user enqueued
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, h->user);
  cudaStreamWaitEvent(h->stream, ev, 0);
  cudaEventDestroy(ev);
  return TTN_OK;
}

int ttn_set_isometries(ttn_t h, int inst, const double* w, const double* v) {
  if (!h || !w || !v || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  Instance& I = h->inst[inst];
  sync_user(h);
  size_t off = 0;
  for (int t = 0; t < I.T; ++t) {
    int rc = check_cuda(h, cudaMemcpyAsync(I.W[t], w + off, I.w_elems(t) * sizeof(double),
                                           cudaMemcpyDefault, h->stream), "set w");
    if (rc) return rc;
    off += I.w_elems(t);
  }
  const size_t c2 = (size_t)I.chis[I.T] * I.chis[I.T];
  int rc = check_cuda(h, cudaMemcpyAsync(I.V, v, c2 * sizeof(double), cudaMemcpyDefault,
                                         h->stream), "set v");
  if (rc) return rc;
  // a new state: no previous energy to compare the next sweep with
  rc = check_cuda(h, cudaMemsetAsync(I.istat, 0, 4 * sizeof(int), h->stream), "set status");
  if (rc) return rc;
  return check_cuda(h, cudaStreamSynchronize(h->stream), "set sync");
}

int ttn_get_isometries(ttn_t h, int inst, double* w, double* v) {
  if (!h || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  Instance& I = h->inst[inst];
  size_t off = 0;
  for (int t = 0; t < I.T && w; ++t) {
    int rc = check_cuda(h, cudaMemcpyAsync(w + off, I.W[t], I.w_elems(t) * sizeof(double),
                                           cudaMemcpyDefault, h->stream), "get w");
    if (rc) return rc;
    off += I.w_elems(t);
  }
  if (v) {
    const size_t c2 = (size_t)I.chis[I.T] * I.chis[I.T];
    int rc = check_cuda(h, cudaMemcpyAsync(v, I.V, c2 * sizeof(double), cudaMemcpyDefault,
                                           h->stream), "get v");
    if (rc) return rc;
  }
  return check_cuda(h, cudaStreamSynchronize(h->stream), "get sync");
}

// One sweep of every instance.  With several lanes the instances of each lane
// follow one another on the lane's stream and the lanes fork from and join
// the library stream (in a captured graph: parallel branches).  A profiling
// sweep keeps everything on one stream so that its events time one product
// at a time.
static void enqueue_sweep(ttn_ctx* h) {
  const int nl = (int)h->lanes.size();
  if (nl == 1 || h->profiling) {
    for (Instance& I : h->inst) sweep_instance(h, I);
    return;
  }
  cudaStream_t main = h->lanes[0].stream;
  cudaEventRecord(h->ev_fork, main);
  for (int k = 1; k < nl; ++k) cudaStreamWaitEvent(h->lanes[k].stream, h->ev_fork, 0);
  for (size_t i = 0; i < h->inst.size(); ++i) {
    load_lane(h, h->lanes[h->lane_of[i]]);
    sweep_instance(h, h->inst[i]);
  }
  load_lane(h, h->lanes[0]);
  for (int k = 1; k < nl; ++k) {
    cudaEventRecord(h->ev_join[k], h->lanes[k].stream);
    cudaStreamWaitEvent(main, h->ev_join[k], 0);
  }
}

// Device status after work on the library's streams: a raised "bounded wait
// expired" flag of any lane (cleared once read, so that the context stays
// usable) and, with conv, whether every instance's last top solve converged.
static int read_status(ttn_ctx* h, bool conv) {
  const size_t nl = h->lanes.size(), ni = h->inst.size();
  std::vector<int> flag(nl, 0), top(ni, 1), pol(ni, 0);
  int rc = TTN_OK;
  for (size_t k = 0; k < nl && !rc; ++k)
    rc = check_cuda(h, cudaMemcpyAsync(&flag[k], h->lanes[k].iflags + 4, sizeof(int),
                                       cudaMemcpyDeviceToHost, h->stream), "status");
  for (size_t i = 0; i < ni && conv && !rc; ++i) {
    rc = check_cuda(h, cudaMemcpyAsync(&top[i], h->inst[i].istat, sizeof(int),
                                       cudaMemcpyDeviceToHost, h->stream), "status");
    if (!rc)
      rc = check_cuda(h, cudaMemcpyAsync(&pol[i], h->inst[i].istat + 4, sizeof(int),
                                         cudaMemcpyDeviceToHost, h->stream), "status");
  }
  if (!rc) rc = check_cuda(h, cudaStreamSynchronize(h->stream), "status sync");
  if (rc) return rc;
  bool expired = false;
  for (int f : flag) expired = expired || f != 0;
  if (expired) {
    for (size_t k = 0; k < nl; ++k) cudaMemsetAsync(h->lanes[k].iflags + 4, 0, sizeof(int), h->stream);
    rc = check_cuda(h, cudaStreamSynchronize(h->stream), "status clear");
    if (rc) return rc;
    return fail(h, TTN_ETIMEOUT, "a bounded wait in a kernel expired (flag cleared)");
  }
  for (size_t i = 0; i < ni && conv; ++i) {
    if (!top[i])
      return fail(h, TTN_ENOCONV, "instance " + std::to_string(i) +
                                      ": the last top solve missed its residual tolerance");
    if (pol[i])
      return fail(h, TTN_ENOCONV, "instance " + std::to_string(i) +
                                      ": a polar factor of the last sweep missed an isometry");
  }
  return TTN_OK;
}

// Enqueue n_sweeps sweeps (graph replays, captured on first use) and, with
// host_energy, copy every sweep's energies out (synchronising per chunk).
static int launch_sweeps(ttn_ctx* h, int n_sweeps, double* host_energy) {
  const int ni = (int)h->inst.size();
  int rc = TTN_OK;
  const bool graph = h->opt.use_graph != 0;
  if (graph && !h->exec) {
    h->launches = 0;
    rc = check_cuda(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal), "capture");
    if (rc) return rc;
    enqueue_sweep(h);
    rc = check_cuda(h, cudaStreamEndCapture(h->stream, &h->graph), "end capture");
    if (rc) return rc;
    if (h->compose_refused) return fail(h, TTN_ECUDA, "cooperative launch refused");
    rc = check_cuda(h, cudaGraphInstantiate(&h->exec, h->graph, 0), "instantiate");
    if (rc) return rc;
    h->launches_per_sweep = h->launches;
  }
  int done = 0;
  while (done < n_sweeps) {
    const int chunk = std::min(n_sweeps - done, 4096);
    for (int s = 0; s < chunk; ++s) {
      if (graph) {
        rc = check_cuda(h, cudaGraphLaunch(h->exec, h->stream), "graph launch");
        if (rc) return rc;
        h->launches += h->launches_per_sweep;
      } else {
        enqueue_sweep(h);
        if (h->compose_refused) return fail(h, TTN_ECUDA, "cooperative launch refused");
      }
      if (host_energy)
        for (int i = 0; i < ni; ++i)
          cudaMemcpyAsync(h->E_hist + (size_t)s * ni + i, h->inst[i].E, sizeof(double),
                          cudaMemcpyDeviceToDevice, h->stream);
    }
    if (host_energy) {
      rc = check_cuda(h, cudaMemcpyAsync(host_energy + (size_t)done * ni, h->E_hist,
                                         (size_t)chunk * ni * sizeof(double),
                                         cudaMemcpyDeviceToHost, h->stream), "energies");
      if (rc) return rc;
      rc = check_cuda(h, cudaStreamSynchronize(h->stream), "sweep sync");
      if (rc) return rc;
    }
    done += chunk;
  }
  h->sweeps_done += n_sweeps;
  return check_cuda(h, cudaGetLastError(), "sweep");
}

// The user's stream waits for the library's work.
static void fence_user(ttn_ctx* h) {
  cudaEvent_t ev;
  cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  cudaEventRecord(ev, h->stream);
  cudaStreamWaitEvent(h->user, ev, 0);
  cudaEventDestroy(ev);
}

int ttn_sweep(ttn_t h, int n_sweeps, double* host_energy) {
  if (!h || n_sweeps < 0) return TTN_EINVAL;
  if (n_sweeps == 0) return TTN_OK;
  sync_user(h);
  h->launches = 0;
  int rc = launch_sweeps(h, n_sweeps, host_energy);
  fence_user(h);
  if (rc) return rc;
  // expired waits first (the state is then unspecified), then the energies,
  // then the convergence of the last top solves
  rc = read_status(h, false);
  if (rc) return rc;
  if (host_energy)
    for (int i = 0; i < n_sweeps * (int)h->inst.size(); ++i)
      if (!std::isfinite(host_energy[i])) return fail(h, TTN_ENAN, "non-finite energy");
  return read_status(h, true);
}

int ttn_sweep_until(ttn_t h, double tol, int max_sweeps, int* n_done, double* host_energy) {
  if (n_done) *n_done = 0;
  if (!h || !(tol > 0.0) || max_sweeps < 1) return TTN_EINVAL;
  sync_user(h);
  h->launches = 0;
  const int ni = (int)h->inst.size();
  int rc = TTN_OK;
  // the tolerance, and no previous energy: the first sweep of the call never counts
  for (int i = 0; i < ni && !rc; ++i) {
    rc = check_cuda(h, cudaMemcpyAsync(h->inst[i].dstat + 2, &tol, sizeof(double),
                                       cudaMemcpyHostToDevice, h->stream), "tolerance");
    if (!rc)
      rc = check_cuda(h, cudaMemsetAsync(h->inst[i].istat + 2, 0, 2 * sizeof(int), h->stream),
                      "status");
  }
  if (!rc) rc = check_cuda(h, cudaStreamSynchronize(h->stream), "tolerance sync");
  if (rc) return rc;
  std::vector<int> conv(ni, 0);
  int done = 0;
  bool all = false;
  while (done < max_sweeps && !all) {
    const int chunk = std::min(8, max_sweeps - done);
    rc = launch_sweeps(h, chunk, host_energy ? host_energy + (size_t)done * ni : nullptr);
    if (rc) break;
    for (int i = 0; i < ni && !rc; ++i)
      rc = check_cuda(h, cudaMemcpyAsync(&conv[i], h->inst[i].istat + 2, sizeof(int),
                                         cudaMemcpyDeviceToHost, h->stream), "convergence");
    if (!rc) rc = check_cuda(h, cudaStreamSynchronize(h->stream), "convergence sync");
    if (rc) break;
    done += chunk;
    all = true;
    for (int c : conv) all = all && c != 0;
  }
  fence_user(h);
  if (n_done) *n_done = done;
  if (rc) return rc;
  rc = read_status(h, false);
  if (rc) return rc;
  if (host_energy)
    for (int i = 0; i < done * ni; ++i)
      if (!std::isfinite(host_energy[i])) return fail(h, TTN_ENAN, "non-finite energy");
  if (!all)
    return fail(h, TTN_ENOCONV, "the energy change per spin stayed above the tolerance for " +
                                    std::to_string(max_sweeps) + " sweeps");
  return TTN_OK;
}

int ttn_diagnostics(ttn_t h, int inst, double* out, int n_out) {
  if (!h || !out || n_out < 7 || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  sync_user(h);
  Instance& I = h->inst[inst];
  const int T = I.T;
  // results in the (idle) Lanczos basis: 3 per site layer (traces of R,
  // max |R|, asymmetry), 3 per isometry layer, then <v, v>
  double* res = h->lz_basis;
  adjoints_only(h, I, 0);
  for (int t = 0; t <= T; ++t) {
    const int n = I.chis[t];
    h->launches += mat_stats(I.adj[t], n, I.sites(t), (ll)(1 + 2 * I.K) * n * n, 0,
                             res + 3 * t, h->stream);
  }
  isometry_grams(h, I, res + 3 * (T + 1));
  const ll c2 = (ll)I.chis[T] * I.chis[T];
  h->launches += batched_dot(I.V, I.V, c2, 0, 1, res + 3 * (2 * T + 1), h->red, h->stream);
  std::vector<double> r(3 * (2 * T + 1) + 1);
  double dst[4];
  int ist[8];
  std::vector<int> pf(std::max(T, 1)), pr(std::max(T, 1));
  int rc = check_cuda(h, cudaMemcpyAsync(r.data(), res, r.size() * sizeof(double),
                                         cudaMemcpyDeviceToHost, h->stream), "diagnostics");
  if (!rc) rc = check_cuda(h, cudaMemcpyAsync(dst, I.dstat, sizeof(dst), cudaMemcpyDeviceToHost,
                                              h->stream), "diagnostics");
  if (!rc) rc = check_cuda(h, cudaMemcpyAsync(ist, I.istat, sizeof(ist), cudaMemcpyDeviceToHost,
                                              h->stream), "diagnostics");
  if (!rc) rc = check_cuda(h, cudaMemcpyAsync(pf.data(), I.pfull, pf.size() * sizeof(int),
                                              cudaMemcpyDeviceToHost, h->stream), "diagnostics");
  // (run_full flags of the last sweep: 0 where the first try succeeded)
  if (!rc) rc = check_cuda(h, cudaMemcpyAsync(pr.data(), I.ppred + pr.size(), pr.size() * sizeof(int),
                                              cudaMemcpyDeviceToHost, h->stream), "diagnostics");
  if (!rc) rc = check_cuda(h, cudaStreamSynchronize(h->stream), "diagnostics sync");
  if (rc) return rc;
  rc = read_status(h, false);
  if (rc) return rc;
  double defect = 0.0, trace_err = 0.0, asym = 0.0;
  for (int t = 0; t <= T; ++t) {
    const double N = (double)(I.L >> t);
    trace_err = std::max(trace_err, std::fabs(r[3 * t] - N) / N);
    asym = std::max(asym, r[3 * t + 2] / N);
  }
  for (int t = 0; t < T; ++t) defect = std::max(defect, r[3 * (T + 1) + 3 * t + 1]);
  out[0] = defect;
  out[1] = trace_err;
  out[2] = asym;
  out[3] = std::fabs(r[3 * (2 * T + 1)] - 1.0);
  out[4] = ist[3] >= 2 ? dst[1] : NAN;
  out[5] = ist[0] ? 1.0 : 0.0;
  out[6] = ist[1];
  if (n_out >= 8) out[7] = ist[4] ? 1.0 : 0.0;
  if (n_out >= 9) {
    int cut = 0;
    for (int t = 0; t < T; ++t) cut += pf[t] == 0;
    out[8] = cut;
  }
  if (n_out >= 10) {
    int first = 0;
    for (int t = 0; t < T; ++t) first += pr[t] == 0;
    out[9] = first;
  }
  return TTN_OK;
}

int ttn_ascend(ttn_t h, int inst, int site_layer, int prec, double* host_out) {
  if (!h || !host_out || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  Instance& I = h->inst[inst];
  if (site_layer < 0 || site_layer > I.T || prec < 0 || prec > 4) return fail(h, TTN_EINVAL, "bad layer");
  sync_user(h);
  if (prec != 0) {
    if (I.w32.empty() || !I.w32[0]) return fail(h, TTN_EINVAL, "context was created for FP64 only");
    h->launches += to_f32(I.ops[0], I.ops32[0], I.op_elems(0), h->stream);
    for (int t = 0; t < site_layer; ++t) h->launches += to_f32(I.W[t], I.w32[t], I.w_elems(t), h->stream);
  }
  for (int t = 0; t < site_layer; ++t) ascend_layer(h, I, t, prec);
  std::vector<double> e(I.sites(site_layer));
  int rc = check_cuda(h, cudaMemcpyAsync(host_out, I.ops[site_layer], I.op_elems(site_layer) * sizeof(double),
                                         cudaMemcpyDeviceToHost, h->stream), "ascend");
  if (rc) return rc;
  rc = check_cuda(h, cudaMemcpyAsync(e.data(), I.eoff[site_layer], e.size() * sizeof(double),
                                     cudaMemcpyDeviceToHost, h->stream), "ascend");
  if (rc) return rc;
  rc = check_cuda(h, cudaStreamSynchronize(h->stream), "ascend sync");
  if (rc) return rc;
  rc = read_status(h, false);
  if (rc) return rc;
  const int n = I.chis[site_layer];
  const size_t ss = (size_t)(1 + 2 * I.K) * n * n;
  for (size_t j = 0; j < e.size(); ++j)
    for (int i = 0; i < n; ++i) host_out[j * ss + (size_t)i * n + i] += e[j];
  return TTN_OK;
}

int ttn_energy(ttn_t h, int inst, double* E) {
  if (!h || !E || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  sync_user(h);
  Instance& I = h->inst[inst];
  forward(h, I, 0);
  energy_only(h, I, h->scal + 5);
  int rc = check_cuda(h, cudaMemcpyAsync(E, h->scal + 5, sizeof(double), cudaMemcpyDeviceToHost,
                                         h->stream), "energy");
  if (rc) return rc;
  rc = check_cuda(h, cudaStreamSynchronize(h->stream), "energy sync");
  return rc ? rc : read_status(h, false);
}

int ttn_value_and_grad(ttn_t h, int inst, int prec, double* E, double* d_grad) {
  if (!h || !E || inst < 0 || inst >= (int)h->inst.size() || prec < 0 || prec > 4)
    return TTN_EINVAL;
  if (prec != 0 && prec != h->opt.prec && h->opt.prec == 0)
    return fail(h, TTN_EINVAL, "context was created for FP64 only");
  sync_user(h);
  Instance& I = h->inst[inst];
  value_and_grad(h, I, prec, h->scal + 5, d_grad);
  int rc = check_cuda(h, cudaMemcpyAsync(E, h->scal + 5, sizeof(double), cudaMemcpyDeviceToHost,
                                         h->stream), "value_and_grad");
  if (rc) return rc;
  rc = check_cuda(h, cudaStreamSynchronize(h->stream), "value_and_grad sync");
  fence_user(h);
  return rc ? rc : read_status(h, false);
}

int ttn_rdm(ttn_t h, int inst, int site_layer, int which, double* out) {
  if (!h || !out || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  Instance& I = h->inst[inst];
  if (site_layer < 0 || site_layer > I.T || (which != 0 && which != 1)) return fail(h, TTN_EINVAL, "bad layer");
  sync_user(h);
  const int n = I.chis[site_layer];
  const size_t n2 = (size_t)n * n;
  std::vector<double> host;
  if (which == 0 || I.per_node) {
    adjoints_only(h, I, site_layer);
    const int S = I.sites(site_layer);
    host.resize((size_t)S * (1 + 2 * I.K) * n2);
    int rc = check_cuda(h, cudaMemcpyAsync(host.data(), I.adj[site_layer], host.size() * sizeof(double),
                                           cudaMemcpyDeviceToHost, h->stream), "rdm");
    if (rc) return rc;
    rc = check_cuda(h, cudaStreamSynchronize(h->stream), "rdm sync");
    if (rc) return rc;
    rc = read_status(h, false);
    if (rc) return rc;
    const size_t ss = (1 + 2 * I.K) * n2;
    if (which == 1) {
      for (size_t e = 0; e < n2; ++e) out[e] = host[e];
    } else {
      for (size_t e = 0; e < n2; ++e) {
        double s = 0;
        for (int j = 0; j < S; ++j) s += host[j * ss + e];
        out[e] = s / (double)(I.L >> site_layer);
      }
    }
    return TTN_OK;
  }
  // translation-invariant tree, leftmost site: rho = V V^T, then Tr_r(W^T rho W) downwards
  const int c = I.chis[I.T];
  double* rho = h->pA;
  {
    GemmDesc d = desc(c, c, 1, 1, rho, c, 1, 0, 0);
    add(d, grp(op(I.V, c, 1), op(I.V, c, 1), c));
    run(h, d, 0);
  }
  for (int t = I.T - 1; t >= site_layer; --t) {
    const LayerView v = view(I, t, 0);
    GemmDesc g = desc(v.P, (int)v.n2, 1, 1, h->Yt, v.n2, 1, 0, 0);
    add(g, grp(op(rho, v.P, 1), op(I.W[t], 1, v.n2), v.P));
    run(h, g, 0);
    GemmDesc r = desc(v.n, v.n, 1, 1, rho, v.n, 1, 0, 0);
    add(r, grp(op(I.W[t], v.n, 1, v.n2), op(h->Yt, v.n, 1, v.n2), v.n, v.P));
    run(h, r, 0);
  }
  int rc = check_cuda(h, cudaMemcpyAsync(out, rho, n2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream), "rdm");
  if (rc) return rc;
  rc = check_cuda(h, cudaStreamSynchronize(h->stream), "rdm sync");
  return rc ? rc : read_status(h, false);
}

int ttn_env(ttn_t h, int inst, int layer, double* d_out) {
  if (!h || !d_out || inst < 0 || inst >= (int)h->inst.size()) return TTN_EINVAL;
  Instance& I = h->inst[inst];
  if (layer < -1 || layer > I.T) return fail(h, TTN_EINVAL, "bad layer");
  sync_user(h);
  const int c = I.chis[I.T];
  const ll c2 = (ll)c * c;
  if (layer == I.T) {
    // top: dE/dV = 2 H_top V (H_top symmetric)
    forward(h, I, 0);
    top_matvec(h, I, I.V, h->lz_w, nullptr);
    h->launches += top_grad(d_out, h->lz_w, I.V, c2, I.eoff[I.T], I.per_node ? 1 : 0, h->stream);
    const int rc_sync = check_cuda(h, cudaStreamSynchronize(h->stream), "env sync");
    return rc_sync ? rc_sync : read_status(h, false);
  }
  adjoints_only(h, I, layer < 0 ? 0 : layer + 1);
  if (layer >= 0) {
    ensure_ops(h, I, layer, 0);
    environment(h, I, layer, 0, h->Gam);
    int rc = check_cuda(h, cudaMemcpyAsync(d_out, h->Gam, I.w_elems(layer) * sizeof(double),
                                           cudaMemcpyDeviceToDevice, h->stream), "env");
    if (rc) return rc;
    const int rc_sync = check_cuda(h, cudaStreamSynchronize(h->stream), "env sync");
    return rc_sync ? rc_sync : read_status(h, false);
  }
  // all layers, concatenated as ttn_set_isometries lays them out, then the top
  size_t off = 0;
  for (int t = 0; t < I.T; ++t) {
    ensure_ops(h, I, t, 0);
    environment(h, I, t, 0, h->Gam);
    int rc = check_cuda(h, cudaMemcpyAsync(d_out + off, h->Gam, I.w_elems(t) * sizeof(double),
                                           cudaMemcpyDeviceToDevice, h->stream), "env");
    if (rc) return rc;
    off += I.w_elems(t);
  }
  top_matvec(h, I, I.V, h->lz_w, nullptr);
  h->launches += top_grad(d_out + off, h->lz_w, I.V, c2, I.eoff[I.T], I.per_node ? 1 : 0,
                          h->stream);
  const int rc_end = check_cuda(h, cudaStreamSynchronize(h->stream), "env sync");
  return rc_end ? rc_end : read_status(h, false);
}

int ttn_get_state(ttn_t h, void* buf, size_t* bytes) {
  if (!h || !bytes) return TTN_EINVAL;
  size_t need = 2 * sizeof(long long);
  for (size_t i = 0; i < h->inst.size(); ++i) {
    size_t nw, nv;
    ttn_sizes(h, (int)i, &nw, &nv, nullptr);
    need += (nw + nv + 1) * sizeof(double);
  }
  if (!buf) { *bytes = need; return TTN_OK; }
  if (*bytes < need) return fail(h, TTN_EINVAL, "state buffer too small");
  char* p = reinterpret_cast<char*>(buf);
  long long hdr[2] = {(long long)h->inst.size(), (long long)h->sweeps_done};
  std::memcpy(p, hdr, sizeof(hdr));
  p += sizeof(hdr);
  for (size_t i = 0; i < h->inst.size(); ++i) {
    size_t nw, nv;
    ttn_sizes(h, (int)i, &nw, &nv, nullptr);
    double* d = reinterpret_cast<double*>(p);
    d[0] = h->inst[i].c;
    int rc = ttn_get_isometries(h, (int)i, d + 1, d + 1 + nw);
    if (rc) return rc;
    p += (nw + nv + 1) * sizeof(double);
  }
  *bytes = need;
  return TTN_OK;
}

int ttn_set_state(ttn_t h, const void* buf, size_t bytes) {
  if (!h || !buf) return TTN_EINVAL;
  const char* p = reinterpret_cast<const char*>(buf);
  long long hdr[2];
  if (bytes < sizeof(hdr)) return fail(h, TTN_EINVAL, "state too short");
  std::memcpy(hdr, p, sizeof(hdr));
  if (hdr[0] != (long long)h->inst.size()) return fail(h, TTN_EINVAL, "state instance count");
  p += sizeof(hdr);
  for (size_t i = 0; i < h->inst.size(); ++i) {
    size_t nw, nv;
    ttn_sizes(h, (int)i, &nw, &nv, nullptr);
    const double* d = reinterpret_cast<const double*>(p);
    if (d[0] != h->inst[i].c) return fail(h, TTN_EINVAL, "state was made with another shift");
    int rc = ttn_set_isometries(h, (int)i, d + 1, d + 1 + nw);
    if (rc) return rc;
    p += (nw + nv + 1) * sizeof(double);
  }
  h->sweeps_done = (int)hdr[1];
  return TTN_OK;
}

long long ttn_launch_count(ttn_t h) { return h ? h->launches : 0; }

int ttn_profile_sweep(ttn_t h, double* out, int n_out) {
  if (!h || !out || n_out < 9) return TTN_EINVAL;
  sync_user(h);
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  h->profiling = true;
  h->launches = 0;
  cudaEventRecord(t0, h->stream);
  enqueue_sweep(h);
  cudaEventRecord(t1, h->stream);
  h->profiling = false;
  int rc = check_cuda(h, cudaStreamSynchronize(h->stream), "profile sync");
  if (!rc && h->compose_refused) rc = fail(h, TTN_ECUDA, "cooperative launch refused");
  double ms[5] = {0, 0, 0, 0, 0}, fl[5] = {0, 0, 0, 0, 0}, cnt[5] = {0, 0, 0, 0, 0},
         by[5] = {0, 0, 0, 0, 0};
  for (size_t i = 0; i < h->ev_flops.size(); ++i) {
    float e = 0.f;
    cudaEventElapsedTime(&e, h->ev_pool[2 * i], h->ev_pool[2 * i + 1]);
    const int g = h->ev_flops[i].first;
    ms[g] += e;
    // products cut short on the device (adaptive polar schedule) count no flops
    int run = 1;
    if (i < h->ev_cond.size() && h->ev_cond[i] && !rc)
      rc = check_cuda(h, cudaMemcpy(&run, h->ev_cond[i], sizeof(int), cudaMemcpyDeviceToHost),
                      "profile flags");
    if (run) fl[g] += h->ev_flops[i].second;
    cnt[g] += 1;
    if (i < h->ev_bytes.size()) by[g] += h->ev_bytes[i];
  }
  float tot = 0.f;
  cudaEventElapsedTime(&tot, t0, t1);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  h->ev_pool.clear();
  h->ev_flops.clear();
  h->ev_bytes.clear();
  h->ev_cond.clear();
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  out[0] = ms[0]; out[1] = fl[0]; out[2] = cnt[0];
  out[3] = ms[1]; out[4] = fl[1]; out[5] = cnt[1];
  out[6] = tot - ms[0] - ms[1] - ms[2] - ms[3] - ms[4];
  out[7] = (double)h->launches - cnt[0] - cnt[1] - cnt[2] - cnt[3] - cnt[4];
  out[8] = tot;
  if (n_out >= 17) {
    out[15] = by[0];
    out[16] = by[1];
  }
  if (n_out >= 19) {
    out[17] = ms[4];
    out[18] = cnt[4];
  } else {
    out[6] += ms[4];
    out[7] += cnt[4];
  }
  if (n_out >= 15) {
    out[9] = ms[2]; out[10] = fl[2]; out[11] = cnt[2];
    out[12] = ms[3]; out[13] = fl[3]; out[14] = cnt[3];
  } else if (n_out >= 12) {
    out[9] = ms[2] + ms[3]; out[10] = fl[2] + fl[3]; out[11] = cnt[2] + cnt[3];
  } else {
    out[6] += ms[2] + ms[3];
    out[7] += cnt[2] + cnt[3];
  }
  h->sweeps_done += 1;
  return rc ? rc : read_status(h, false);
}

int ttn_autotune(ttn_t h, int reps, void* blob, size_t* blob_bytes) {
  if (!h || reps < 0) return TTN_EINVAL;
  int rc = TTN_OK;
  if (reps > 0) {
    sync_user(h);
    h->tuned.clear();
    h->tuning = true;
    h->tune_reps = reps;
    h->profiling = true;   // one stream, no capture, like the profiling sweep
    h->launches = 0;
    enqueue_sweep(h);
    h->profiling = false;
    h->tuning = false;
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    h->ev_pool.clear();
    h->ev_flops.clear();
    h->ev_bytes.clear();
    h->ev_cond.clear();
    rc = check_cuda(h, cudaStreamSynchronize(h->stream), "autotune sync");
    if (!rc && h->compose_refused) rc = fail(h, TTN_ECUDA, "cooperative launch refused");
    if (!rc) rc = read_status(h, false);
    h->sweeps_done += 1;
    fence_user(h);
    // the captured sweep used the previous configurations: capture again
    if (h->exec) { cudaGraphExecDestroy(h->exec); h->exec = nullptr; }
    if (h->graph) { cudaGraphDestroy(h->graph); h->graph = nullptr; }
    if (rc) return rc;
  }
  if (blob_bytes) {
    const size_t need = sizeof(TuneBlobHeader) + h->tuned.size() * sizeof(TuneBlobEntry);
    if (!blob) {
      *blob_bytes = need;
      return TTN_OK;
    }
    if (*blob_bytes < need) return fail(h, TTN_EINVAL, "tiles buffer too small");
    TuneBlobHeader hd;
    std::memcpy(hd.magic, "TTNT", 4);
    hd.version = 2;
    hd.count = (uint32_t)h->tuned.size();
    hd.reserved = 0;
    char* p = static_cast<char*>(blob);
    std::memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    for (const auto& kv : h->tuned) {
      TuneBlobEntry e{kv.first, kv.second.engine, kv.second.tile, kv.second.splits,
                      kv.second.occ, kv.second.ms, 0};
      std::memcpy(p, &e, sizeof(e));
      p += sizeof(e);
    }
    *blob_bytes = need;
  }
  return TTN_OK;
}

const char* ttn_last_error(ttn_t h) { return h ? h->err.c_str() : "null handle"; }

void ttn_destroy(ttn_t h) {
  if (!h) return;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (size_t k = 1; k < h->lanes.size(); ++k)
    if (h->lanes[k].stream) {
      cudaStreamSynchronize(h->lanes[k].stream);
      cudaStreamDestroy(h->lanes[k].stream);
    }
  for (cudaEvent_t e : h->ev_join)
    if (e) cudaEventDestroy(e);
  for (Lane& l : h->lanes) {
    for (int i = 0; i < kSubStreams; ++i) {
      if (l.sub.s[i]) {
        cudaStreamSynchronize(l.sub.s[i]);
        cudaStreamDestroy(l.sub.s[i]);
      }
      if (l.sub.join[i]) cudaEventDestroy(l.sub.join[i]);
    }
    if (l.sub.fork) cudaEventDestroy(l.sub.fork);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (!h->lanes.empty()) h->stream = h->lanes[0].stream;
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

}  // extern "C"
