// C ABI entry points and the host-side solver driver.
//
// rhmc_block_multishift_cg runs SBCGrQ (Algorithm 1) for all right-hand sides
// and shifts at once.  Per iteration k (device work only, no host round trip):
//   AP = (A + sigma_0) P^(0)                      two hops, axpy fused   (alpha_k step)
//   Gram1 = P^(0)dagger AP -> alpha_k            gram + n x n kernel     (alpha_k step)
//   W = Q_{k-1} - AP alpha_k                      block axpy             (block QR)
//   Gram2 = W^dagger W -> rho_k (Cholesky QR), base and shifted
//   coefficients                                  gram + n x n kernels   (block QR, delta_k,
//                                                                         beta^(s)_k, alpha^(s)_k)
//   Q_k = W rho_k^-1; for every live shift
//   X^(s) += P^(s) M1^(s), P^(s) = Q_k + P^(s) M2^(s)   one fused pass   (base and shifted
//                                                                         updates)
// The host reads the residual estimates every few iterations to decide on
// convergence (and, in mixed precision, on reliable updates).
//
// Mixed precision (RHMC_MIXED_FP32): the fields P, Q, W, AP and the solution
// increments are FP32; the n x n algebra is FP64.  When the base residual
// has dropped by kReliableDelta since the last reliable update, the FP32
// solution increments are added into the FP64 solutions, the base residual
// B - (A + sigma_0) X^(0) is recomputed with the FP64 operator and its thin
// QR replaces (Q_k, delta_k).  After the loop every shift's true residual is
// evaluated in FP64; a shift above tol gets a defect-correction solve
// (A + sigma_s) E = R^(s) with the same machinery, X^(s) += E.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "scg.h"

namespace rhmc {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};
// launches by the calling host thread (stream capture counts its own kernels with it:
// refinement lanes on other threads launch concurrently)
static thread_local long long t_launches = 0;

void count_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
}

// ------------------------------------------------------------ profiler
struct ProfRec {
  int cat;
  cudaEvent_t a, b;
  double bytes;
  double flops;  // tensor-core flops issued (tensor kernels), else 0
};
static bool g_prof = false;
static std::vector<ProfRec> g_recs;
static std::vector<cudaEvent_t> g_pool;
static size_t g_pool_next = 0;

static cudaEvent_t pool_event() {
  if (g_pool_next == g_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g_pool.push_back(e);
  }
  return g_pool[g_pool_next++];
}

bool prof_on() { return g_prof; }

static int g_tune[TUNE_NKEYS] = {0};
// per-context settings (rhmc_ctx_tune_set) of the context the calling host
// thread works for; nonzero entries override the process-wide ones
static thread_local const int *t_tune_override = nullptr;
int tune_get(int key) {
  if (key < 0 || key >= TUNE_NKEYS) return 0;
  if (t_tune_override && t_tune_override[key] > 0) return t_tune_override[key];
  return g_tune[key];
}

void prof_begin(int cat, cudaStream_t s) {
  if (!g_prof) return;
  ProfRec r{cat, pool_event(), pool_event(), 0.0, 0.0};
  cudaEventRecord(r.a, s);
  g_recs.push_back(r);
}

void prof_end(cudaStream_t s, double bytes) {
  if (!g_prof || g_recs.empty()) return;
  cudaEventRecord(g_recs.back().b, s);
  g_recs.back().bytes = bytes;
}

void prof_flops(double flops) {
  if (g_prof && !g_recs.empty()) g_recs.back().flops = flops;
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

constexpr int kParts = 304;           // partial sums of the simple reductions (2 CTAs per SM)
constexpr int kGramParts = 1;         // the Gram kernels deliver the summed n x n matrix
constexpr double kReliableDelta = 0.1;
constexpr int kCheckEvery = 6;        // iterations between host checks (a multiple of 6 keeps the
                                      // k % 2 and k % 3 slot pattern of a captured chunk fixed)
constexpr int kGraphCacheMax = 48;
constexpr int kMaxRefine = 4;
constexpr double kShiftFreezeMixed = 0.0;  // built-in freeze level of the shifted systems (mixed)
constexpr int kRefineLanes = 4;       // concurrent defect corrections (built-in and most; 8 measured 2 % faster)
// host checks of a defect-correction solve (divides kCheckEvery); measured at 24^4 with the
// 0.9 margin: every 1, 2, 3 iterations took 223, 230, 240 correction iterations (95, 97, 100 ms)
constexpr int kCorrectionCheckEvery = 1;
// A defect correction stops when its recursive residual is kCorrectionMargin x tol / r of the
// residual r it started from.  Its own FP32 drift is about 1e-6 of r (1e-3 of its target),
// so the true residual after it lands within that margin of tol; a second round
// follows only when it does not.  Measured at 24^4 (15 corrections): margin 0.5 took 342
// iterations, 0.7 266, 0.8 246, 0.9 232 (largest true residual 0.88 tol), 0.95 226.
constexpr double kCorrectionMargin = 0.9;
// The multishift phase runs to kPhase1Margin x tol (0.5, 0.7 and 0.9 measured within
// noise of each other at 24^4: the shifted systems leave it drift-bound either way).
constexpr double kPhase1Margin = 0.5;

// Bump allocator over a device buffer; with base == nullptr it only measures.
struct Arena {
  char *base;
  size_t off = 0;
  explicit Arena(void *b) : base((char *)b) {}
  template <typename T> T *take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

}  // namespace rhmc

using namespace rhmc;

// Host-side state of one stream of solver work: its capture stream, pinned
// readback buffer and captured graphs.  The caller's solve runs on the main
// lane; the defect corrections of different shifts run on lanes of their own,
// one host thread each.
struct SolverLane {
  cudaStream_t s = nullptr;    // the lane's stream (null for the main lane: the caller's)
  cudaStream_t cap = nullptr;  // graph capture (the caller's stream may be the legacy default stream)
  double *h_pin = nullptr;     // pinned host staging (readbacks)
  size_t h_pin_bytes = 0;
  struct GraphEntry {
    std::vector<double> key;   // what the captured chunk depends on
    cudaGraphExec_t exec;
    long long launches;        // kernels in one replay
    unsigned long long last_use;
  };
  std::vector<GraphEntry> graphs;  // captured SBCGrQ chunks (CUDA graphs)
  unsigned long long graph_clock = 0;
  void release() {
    for (auto &e : graphs) cudaGraphExecDestroy(e.exec);
    graphs.clear();
    if (h_pin) cudaFreeHost(h_pin);
    h_pin = nullptr;
    h_pin_bytes = 0;
    if (cap) cudaStreamDestroy(cap);
    cap = nullptr;
    if (s) cudaStreamDestroy(s);
    s = nullptr;
  }
};

struct rhmc_ctx {
  int device = 0;
  Geom g{};
  double mass = 0;
  int bc_t = -1;
  double2 *l64[2] = {nullptr, nullptr};
  float2 *l32[2] = {nullptr, nullptr};
  float4 *ldf[2] = {nullptr, nullptr};  // double-float copy of the FP64 link records
  float2 *l12[2] = {nullptr, nullptr};  // first two rows of the FP32 records (used when every link is SU(3))
  bool rec12 = false;
  bool have_gauge = false;
  void *pool = nullptr;
  size_t pool_bytes = 0;
  cudaStream_t side = nullptr;     // shifted coefficient steps and updates
  cudaStream_t own = nullptr;      // the context's stream in batched solves
  cudaEvent_t ev_base[3] = {};     // base update of iteration k done (slot k % 3)
  cudaEvent_t ev_side[3] = {};     // shifted updates of iteration k done
  SolverLane main;                 // the caller's stream
  int tune[TUNE_NKEYS] = {};       // per-context launch settings (0: the process-wide value)
  std::vector<std::unique_ptr<SolverLane>> lanes;  // concurrent defect corrections
  double *d_parts = nullptr;       // partial sums of rhmc_force_lie's norm (kParts)
  void *md_buf = nullptr;          // molecular-dynamics fields (momenta, force, trial links)
  size_t md_bytes = 0;
};

namespace rhmc {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// The calling thread uses ctx's launch settings for the duration of a call.
struct TuneScope {
  const int *prev;
  explicit TuneScope(const rhmc_ctx *c) : prev(t_tune_override) { t_tune_override = c ? c->tune : nullptr; }
  ~TuneScope() { t_tune_override = prev; }
};

CtxTuneScope::CtxTuneScope(const rhmc_ctx_t *c) : prev(t_tune_override) { t_tune_override = c ? c->tune : nullptr; }
CtxTuneScope::~CtxTuneScope() { t_tune_override = prev; }

static rhmc_status_t ensure_pool(rhmc_ctx *c, size_t bytes) {
  if (c->pool_bytes >= bytes) return RHMC_OK;
  if (c->pool) {
    RHMC_CUDA_TRY(cudaDeviceSynchronize());
    RHMC_CUDA_TRY(cudaFree(c->pool));
    c->pool = nullptr;
    c->pool_bytes = 0;
  }
  RHMC_CUDA_TRY(cudaMalloc(&c->pool, bytes));
  c->pool_bytes = bytes;
  return RHMC_OK;
}

// The lane the calling host thread works on (the main lane unless a
// defect-correction worker set its own).
static thread_local SolverLane *t_lane = nullptr;
static SolverLane &lane(rhmc_ctx *c) { return t_lane ? *t_lane : c->main; }

static rhmc_status_t ensure_pinned(rhmc_ctx *c, size_t bytes) {
  SolverLane &L = lane(c);
  if (L.h_pin_bytes >= bytes) return RHMC_OK;
  if (L.h_pin) cudaFreeHost(L.h_pin);
  L.h_pin = nullptr;
  RHMC_CUDA_TRY(cudaMallocHost(&L.h_pin, bytes));
  L.h_pin_bytes = bytes;
  return RHMC_OK;
}

// ------------------------------------------------------------ operator helpers
template <typename T> struct LinksOf;
template <> struct LinksOf<float> {
  static const float2 *get(const rhmc_ctx *c, int p) { return c->l32[p]; }
};
template <> struct LinksOf<double> {
  static const double2 *get(const rhmc_ctx *c, int p) { return c->l64[p]; }
};
template <typename T> struct Links12Of;
template <> struct Links12Of<float> {
  static const float2 *get(const rhmc_ctx *c, int p) {
    // opt-in: at 24^4, n = 16 the rebuild costs what the 128 fewer bytes per site save
    return (c->rec12 && tune_get(TUNE_LINKS12) == 1) ? c->l12[p] : nullptr;
  }
};
template <> struct Links12Of<double> {
  static const double2 *get(const rhmc_ctx *, int) { return nullptr; }
};

// Y = (A + sigma) X, tmp: odd-parity field of the same width.
template <typename T>
static rhmc_status_t apply_A(const rhmc_ctx *c, const C<T> *X, C<T> *Y, C<T> *tmp, int n, double sigma,
                             cudaStream_t s) {
  RHMC_TRY(hop<T>(c->g, 1, LinksOf<T>::get(c, 1), X, tmp, nullptr, 0.0, n, 1, 0, s, Links12Of<T>::get(c, 1),
                  c->bc_t));
  RHMC_TRY(hop<T>(c->g, 0, LinksOf<T>::get(c, 0), tmp, Y, X, 4.0 * c->mass * c->mass + sigma, n, 1, 0, s,
                  Links12Of<T>::get(c, 0), c->bc_t));
  return RHMC_OK;
}

// Y = (A + sigma) X with FP64 accuracy on the FP32 units (double-float):
// split writes X as (hi, lo) into `split`, tmp holds the odd intermediate;
// Y is written in FP64.  split, tmp, Y: FP64-field-sized buffers.
static rhmc_status_t apply_A_df(const rhmc_ctx *c, const double2 *X, double2 *Y, double2 *tmp, double2 *split, int n,
                                double sigma, cudaStream_t s) {
  const long len = c->g.Vh * 3 * n;
  RHMC_TRY(df_split(X, (float4 *)split, len, s));
  RHMC_TRY(hop_df(c->g, 1, c->ldf[1], (const float4 *)split, (float4 *)tmp, nullptr, 0.0, n, s));
  RHMC_TRY(hop_df(c->g, 0, c->ldf[0], (const float4 *)tmp, (float4 *)Y, (const float4 *)split,
                  4.0 * c->mass * c->mass + sigma, n, s));
  RHMC_TRY(df_merge((float4 *)Y, len, s));
  return RHMC_OK;
}

// R = B - (A + sigma) X with FP64 accuracy for the mixed path; Rf (optional)
// receives the FP32 rounding of R and npart (optional) the kParts x n column
// partials of |R|^2.  Y, tmp, split: FP64-field-sized scratch; R may be split.
// The double-float form subtracts the operator's (hi, lo) result directly.
static rhmc_status_t residual_accurate(const rhmc_ctx *c, const double2 *B, const double2 *X, double2 *R,
                                       float2 *Rf, double2 *Y, double2 *tmp, double2 *split, int n, double sigma,
                                       double *npart, cudaStream_t s) {
  const long rows = c->g.Vh * 3, len = rows * n;
  if (tune_get(TUNE_NATIVE_FP64_RESIDUALS)) {
    RHMC_TRY(apply_A<double>(c, X, Y, tmp, n, sigma, s));
    RHMC_TRY(sub(B, Y, R, len, s));
    if (Rf) RHMC_TRY((convert<double, float>(R, Rf, len, s)));
    if (npart) RHMC_TRY(colnorm2<double>(R, rows, n, npart, kParts, s));
    return RHMC_OK;
  }
  RHMC_TRY(df_split(X, (float4 *)split, len, s));
  RHMC_TRY(hop_df(c->g, 1, c->ldf[1], (const float4 *)split, (float4 *)tmp, nullptr, 0.0, n, s));
  RHMC_TRY(hop_df(c->g, 0, c->ldf[0], (const float4 *)tmp, (float4 *)Y, (const float4 *)split,
                  4.0 * c->mass * c->mass + sigma, n, s));
  return resid_df(B, (const float4 *)Y, R, Rf, rows, n, npart, kParts, s);
}

// ------------------------------------------------------------ solver workspace
struct SolveBufs {
  // precision-specific fields (T = float or double)
  void *P, *Qb[2], *W, *AP, *Todd, *Xinc;  // Qb: Q_k in Qb[k & 1]; Xinc: FP32 increments (mixed only)
  void *coef, *mw;
  // FP64 helpers
  double2 *R64, *T64, *AP64, *rinv64;
  float *btiles;      // tensor-core B tiles of the shifted updates
  double2 *partial;   // the summed Gram matrix (n x n)
  double2 *gscratch;  // per-CTA Gram partials
  double *npart;
  SolverState *st;
  int accumulate = 0;  // shifts s >= 1 add w_s X^(s) into one field after X^(0) (FP64)
  // stored-basis mode (mixed, several shifts): the block basis Q_0 .. Q_{cap-1}
  // (rows x cap*n, row-major), the per-iteration shift coefficients and the
  // assembly's operands; basis == nullptr: shifted updates in HBM
  float2 *basis = nullptr;
  double2 *hist = nullptr;
  BasisBufs asmb;
  int cap = 0;
};

// Stored-basis capacity.  RHMC_TUNE_BASIS_ITERS: 0 = built-in, 1 = off, >= 2 = that
// many iterations.  Built-in: up to kBasisCapMax blocks within a quarter of the
// device's memory, off when fewer than kBasisCapMin would fit.  The base update of
// the column-owner path stores the blocks, so the lane-slice kernel turns it off.
constexpr int kBasisCapMax = 384, kBasisCapMin = 24;
static size_t device_total_memory() {
  static std::mutex mu;
  static std::map<int, size_t> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  cudaDeviceProp p{};
  const size_t total = cudaGetDeviceProperties(&p, dev) == cudaSuccess ? p.totalGlobalMem : 0;
  cache[dev] = total;
  return total;
}
static int basis_cap(const Geom &g, int n, int ns, bool mixed) {
  if (!mixed || ns < 2 || tune_get(TUNE_UPDATE_TENSOR) == 2) return 0;
  const int v = tune_get(TUNE_BASIS_ITERS);
  if (v == 1) return 0;
  // even, so that every basis row (cap * 2n floats) starts on a 16-byte boundary
  if (v >= 2) return v & ~1;
  const size_t block = (size_t)g.Vh * 3 * n * sizeof(float2);
  const size_t fit = (device_total_memory() / 4) / std::max<size_t>(block, 1);
  const int cap = (int)std::min<size_t>(fit, kBasisCapMax) & ~1;
  return cap >= kBasisCapMin ? cap : 0;
}

static void layout_solve(Arena &a, const Geom &g, int n, int ns, bool mixed, SolveBufs &b) {
  const size_t len = (size_t)g.Vh * 3 * n;
  const size_t esz = mixed ? sizeof(float2) : sizeof(double2);
  auto field = [&](size_t count) { return (void *)a.take<char>(count * len * esz); };
  b.P = field(ns);
  b.Qb[0] = field(1);
  b.Qb[1] = field(1);
  b.W = field(1);
  b.AP = field(1);
  b.Todd = field(1);
  b.Xinc = mixed ? field(ns) : nullptr;
  b.coef = a.take<char>((size_t)(1 + 2 * ns) * n * n * esz);
  b.mw = a.take<char>((size_t)n * n * esz);
  b.R64 = a.take<double2>(len);
  b.T64 = a.take<double2>(len);
  b.AP64 = a.take<double2>(len);
  b.rinv64 = a.take<double2>((size_t)n * n);
  b.btiles = a.take<float>((size_t)ns * 3 * 64 * 32);
  b.partial = a.take<double2>((size_t)n * n);
  b.gscratch = a.take<double2>((size_t)kGramCtas * n * n);
  b.npart = a.take<double>((size_t)kParts * kMaxN);
  b.st = a.take<SolverState>(1);
  const int cap = basis_cap(g, n, ns, mixed);
  if (cap > 0) {
    b.cap = cap;
    b.basis = a.take<float2>((size_t)g.Vh * 3 * cap * n);
    b.hist = a.take<double2>((size_t)cap * ns * 2 * n * n);
    b.asmb.basis = b.basis;
    b.asmb.hist = b.hist;
    b.asmb.cap = cap;
    b.asmb.cf = a.take<double2>((size_t)(ns - 1) * (cap + 1) * n * n);
    b.asmb.bpack = a.take<unsigned char>(basis_pack_bytes(n, ns, cap));
    b.asmb.bscale = a.take<double>((size_t)ns);
    b.asmb.tile_nkt = a.take<int>((size_t)ns);
  }
}

// Phase-2 buffers live above the (dead) phase-1 buffers of the top-level solve.
struct RefineBufs {
  double2 *Bref, *E;
};

// Lanes of the defect-correction phase: workspace is laid out for the
// built-in count, the tuning key can only lower it.
static int refine_lanes(int ns) { return std::max(1, std::min(kRefineLanes, ns)); }

static size_t solve_bytes(const Geom &g, int n, int ns, bool mixed, bool own_X) {
  Arena a(nullptr);
  if (own_X) a.take<double2>((size_t)ns * g.Vh * 3 * n);
  SolveBufs b;
  layout_solve(a, g, n, ns, mixed, b);
  // refinement: per lane Bref, E, plus a single-shift solve
  Arena r(nullptr);
  if (own_X) r.take<double2>((size_t)ns * g.Vh * 3 * n);
  for (int l = 0; l < refine_lanes(ns); ++l) {
    r.take<double2>((size_t)g.Vh * 3 * n);
    r.take<double2>((size_t)g.Vh * 3 * n);
    SolveBufs b1;
    layout_solve(r, g, n, 1, mixed, b1);
  }
  return std::max(a.off, r.off) + 256;
}

struct SolveParams {
  double tol;
  int max_iter;
  bool mixed;
  int fixed_iters;  // > 0: exactly this many iterations, no freezing, no checks
  bool verify_at_convergence = true;  // mixed: reliable update before declaring convergence
  const double *acc_w = nullptr;       // accumulating solve: weights of the shifts' solutions
  bool reliable = true;                // mixed: reliable updates when the residual has dropped
  int check_every = 0;                 // iterations between host checks (0: RHMC_TUNE_CHECK_EVERY / 6)
};

struct SolveStats {
  int iters = 0, dirac = 0, reliable = 0;
};

// Host sums (fixed order) of the kParts x n column partials written on stream s.
static rhmc_status_t read_colnorms(rhmc_ctx *c, const double *npart, int n, double *out, cudaStream_t s) {
  RHMC_TRY(ensure_pinned(c, sizeof(double) * kParts * kMaxN));
  RHMC_CUDA_TRY(cudaMemcpyAsync(lane(c).h_pin, npart, sizeof(double) * kParts * n, cudaMemcpyDeviceToHost, s));
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  for (int j = 0; j < n; ++j) {
    double t = 0;
    for (int p = 0; p < kParts; ++p) t += lane(c).h_pin[p * n + j];
    out[j] = t;
  }
  return RHMC_OK;
}

// Column norms squared of an FP64 block (host result, n entries).
static rhmc_status_t colnorms(rhmc_ctx *c, const double2 *A, int n, double *out, double *npart, cudaStream_t s) {
  RHMC_TRY(colnorm2<double>(A, c->g.Vh * 3, n, npart, kParts, s));
  return read_colnorms(c, npart, n, out, s);
}

struct StateView {
  double res[kMaxS][kMaxN];
  int active[kMaxS];
  int breakdown;
  int device_timeout;
};

static rhmc_status_t read_state(rhmc_ctx *c, SolverState *st, StateView &v, cudaStream_t s) {
  RHMC_TRY(ensure_pinned(c, sizeof(StateView) + 64));
  StateView *h = reinterpret_cast<StateView *>(lane(c).h_pin);
  RHMC_CUDA_TRY(cudaMemcpyAsync(h->res, st->res, sizeof(v.res), cudaMemcpyDeviceToHost, s));
  RHMC_CUDA_TRY(cudaMemcpyAsync(h->active, st->active, sizeof(v.active), cudaMemcpyDeviceToHost, s));
  RHMC_CUDA_TRY(cudaMemcpyAsync(&h->breakdown, &st->breakdown, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(&v, h, sizeof(StateView));
  return RHMC_OK;
}

// Captured CUDA graphs for the solver chunks (not while profiling).
static bool use_graphs() { return !prof_on() && tune_get(TUNE_GRAPHS) != 2; }

// Tensor-core shifted updates: FP32 fields, 16 right-hand sides.
template <typename T> static bool use_tensor_update(int n) {
  if (sizeof(T) != 4 || n != 16) return false;
  // Built-in choice: CUDA cores.  Measured at 24^4: the tcgen05 kernel (one
  // CTA per row tile, three-piece TF32 split) moves 2.1 TB/s against 4.5 for
  // the packed CUDA-core kernel and its drift costs more defect correction
  // (510 against 324 iterations).
  return tune_get(TUNE_UPDATE_TENSOR) == 1;
}
// Column-owner shifted updates (FP32): the built-in choice; RHMC_TUNE_UPDATE_TENSOR = 2
// selects the lane-slice kernel.
template <typename T> static bool use_column_update() {
  return sizeof(T) == 4 && tune_get(TUNE_UPDATE_TENSOR) != 2;
}

// One SBCGrQ iteration (device work only).  The base recursion runs on the
// caller's stream s; with more than one shift the shifted coefficient step and
// the shifted updates of iteration k run on the context's side stream, where
// they overlap iteration k+1 of the base.  Ordering:
//   side(k)   waits for the base update of k (Q_k, rho_k, alpha_k in place);
//   base(k)   waits for side(k-2) before it overwrites the state slot k % 3 and
//             the buffer Q_k = Qb[k & 1] that side(k-2) was reading.
template <typename T, typename TX>
static rhmc_status_t sbcgrq_iteration(rhmc_ctx *c, const SolveBufs &b, TX *Xacc, int n, int ns, double sigma0, int k,
                                      int chunk_start, double tol_shift, int freeze, cudaStream_t s) {
  const long rows = c->g.Vh * 3;
  const long len = rows * n;
  C<T> *P = (C<T> *)b.P, *W = (C<T> *)b.W, *AP = (C<T> *)b.AP, *Todd = (C<T> *)b.Todd;
  C<T> *Qprev = (C<T> *)b.Qb[(k - 1) & 1], *Qcur = (C<T> *)b.Qb[k & 1];
  // With the profiler on, the shifted steps run on s as well (same kernels,
  // serialised) so that per-kernel event times are not inflated by overlap.
  const bool split = ns > 1 && !prof_on();
  cudaStream_t ss = split ? c->side : s;
  // (chunk boundaries are joined on the host, so only waits inside a chunk are needed)
  if (split && k - 2 > chunk_start) RHMC_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_side[(k - 2) % 3], 0));
  RHMC_TRY(apply_A<T>(c, P, AP, Todd, n, sigma0, s));
  RHMC_TRY(gram<T>(P, AP, rows, n, b.gscratch, b.partial, s));
  RHMC_TRY(nxn_alpha<T>(b.partial, kGramParts, n, b.st, k, (C<T> *)b.mw, s));
  const bool cols = use_column_update<T>();
  if (cols) {
    // W = Q - (AP) alpha and its Gram W^dagger W in one pass
    RHMC_TRY(axpy_gram_cols((const float2 *)AP, (const float2 *)Qprev, (const float2 *)b.mw, (float2 *)W, rows, n,
                            b.gscratch, b.partial, s));
  } else {
    RHMC_TRY(block_axpy<T, T>(AP, Qprev, (const C<T> *)b.mw, W, rows, n, s));
    RHMC_TRY(gram<T>(W, W, rows, n, b.gscratch, b.partial, s));
  }
  RHMC_TRY(nxn_rho<T>(b.partial, kGramParts, n, b.st, k, (C<T> *)b.coef, s));
  // base: Q_k = W rho_k^-1, X^(0), P^(0)
  if (cols && tune_get(TUNE_AXPY_SCALAR) != 1) {
    // one pass: Q_k = W rho^-1, X^(0), P^(0), and block k of the stored basis (k from the
    // device counter: graph replays)
    RHMC_TRY(base_step((const float2 *)W, (float2 *)Qcur, (float2 *)P, (float2 *)Xacc, (const float2 *)b.coef,
                       b.basis, b.cap, b.basis ? &b.st->kabs[k % kSlots] : nullptr, rows, n, s));
  } else if (cols) {
    RHMC_TRY(axpy_cols((const float2 *)W, nullptr, (const float2 *)b.coef, (float2 *)Qcur, rows, n, s));
    if (b.basis)  // block k of the stored basis (k from the device counter: graph replays)
      RHMC_TRY(basis_store_dev((const float2 *)Qcur, b.basis, rows, n, b.cap, &b.st->kabs[k % kSlots], s));
    RHMC_TRY(update_shifts_cols((const float2 *)Qcur, (float2 *)P, (float2 *)Xacc, (const float2 *)b.coef,
                                b.st->upd, 0, 1, rows, n, len, s));
  } else {
    RHMC_TRY(update_all<T, TX>(W, Qcur, P, (C<TX> *)Xacc, (const C<T> *)b.coef, b.st->upd, 0, 1, 1, rows, n, len, s));
  }
  if (ns > 1) {
    if (split) {
      RHMC_CUDA_TRY(cudaEventRecord(c->ev_base[k % 3], s));
      RHMC_CUDA_TRY(cudaStreamWaitEvent(ss, c->ev_base[k % 3], 0));
    }
    RHMC_TRY(nxn_shifts<T>(n, ns, b.st, k, (C<T> *)b.coef, tol_shift, freeze, b.hist, b.cap, ss));
    if (b.basis) {
      // stored-basis mode: the shifted solutions are assembled at the end
    } else if (use_tensor_update<T>(n))
      RHMC_TRY(update_shifts_tc((const float2 *)Qcur, (float2 *)P, (float2 *)Xacc, (const float2 *)b.coef,
                                b.st->upd, 1, ns, rows, len, b.btiles, &b.st->device_timeout, ss));
    else if (cols)
      RHMC_TRY(update_shifts_cols((const float2 *)Qcur, (float2 *)P, (float2 *)Xacc, (const float2 *)b.coef,
                                  b.st->upd, 1, ns, rows, n, len, ss));
    else if (b.accumulate)
      RHMC_TRY(update_all<T, TX>(W, Qcur, P, (C<TX> *)Xacc + len, (const C<T> *)b.coef, b.st->upd, 1, ns, 0, rows,
                                 n, len, ss, 1));
    else
      RHMC_TRY(update_all<T, TX>(W, Qcur, P, (C<TX> *)Xacc, (const C<T> *)b.coef, b.st->upd, 1, ns, 0, rows, n, len,
                                 ss));
    if (split) RHMC_CUDA_TRY(cudaEventRecord(c->ev_side[k % 3], ss));
  }
  return RHMC_OK;
}

// Make stream s wait for everything enqueued so far on the side stream.
static rhmc_status_t join_side(rhmc_ctx *c, int k, int ns, cudaStream_t s) {
  if (ns > 1 && k >= 1 && !prof_on()) RHMC_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_side[k % 3], 0));
  return RHMC_OK;
}

// Run iterations chunk_start+1 .. chunk_start+len, joined back to stream s.
template <typename T>
static rhmc_status_t run_chunk(rhmc_ctx *c, const SolveBufs &b, double2 *X, int n, int ns, double sigma0,
                               int chunk_start, int len, double target, int freeze, cudaStream_t s) {
  for (int q = 1; q <= len; ++q) {
    const int k = chunk_start + q;
    if (std::is_same<T, float>::value)
      RHMC_TRY((sbcgrq_iteration<float, float>(c, b, (float *)b.Xinc, n, ns, sigma0, k, chunk_start, target, freeze,
                                                s)));
    else
      RHMC_TRY((sbcgrq_iteration<double, double>(c, b, (double *)X, n, ns, sigma0, k, chunk_start, target, freeze,
                                                  s)));
  }
  return join_side(c, chunk_start + len, ns, s);
}

// The same chunk as a CUDA graph, captured once per (workspace, sizes, shift,
// tolerance, tuning) and replayed for every later chunk that starts at a
// multiple of kCheckEvery.  Capture runs on the context's capture stream (the
// legacy default stream cannot be captured); the graph is launched on s.
template <typename T>
static rhmc_status_t run_chunk_graph(rhmc_ctx *c, const SolveBufs &b, double2 *X, int n, int ns, double sigma0,
                                     int chunk_start, int len, double target, int freeze, cudaStream_t s) {
  // (b.basis: chunks with and without the stored basis record different kernels)
  std::vector<double> key = {(double)(uintptr_t)b.P, (double)(uintptr_t)X, (double)(uintptr_t)b.basis,
                             (double)b.accumulate, (double)n,
                             (double)ns, sigma0, target, (double)freeze, (double)sizeof(T), (double)len,
                             (double)(chunk_start % kCheckEvery)};
  for (int t = 0; t < TUNE_NKEYS; ++t) key.push_back((double)tune_get(t));
  SolverLane &L = lane(c);
  SolverLane::GraphEntry *hit = nullptr;
  for (auto &e : L.graphs)
    if (e.key == key) hit = &e;
  if (!hit) {
    if ((int)L.graphs.size() >= kGraphCacheMax) {  // evict the least recently used
      auto lru = std::min_element(L.graphs.begin(), L.graphs.end(),
                                  [](const SolverLane::GraphEntry &a, const SolverLane::GraphEntry &b2) {
                                    return a.last_use < b2.last_use;
                                  });
      cudaGraphExecDestroy(lru->exec);
      L.graphs.erase(lru);
    }
    const long long before = t_launches;
    RHMC_CUDA_TRY(cudaStreamBeginCapture(L.cap, cudaStreamCaptureModeThreadLocal));
    const rhmc_status_t rc = run_chunk<T>(c, b, X, n, ns, sigma0, chunk_start, len, target, freeze, L.cap);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(L.cap, &g);
    const long long captured = t_launches - before;
    g_launches.fetch_sub(captured);  // recorded, not run: counted at every replay instead
    if (rc != RHMC_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ec != cudaSuccess) {
      set_error("stream capture of a solver chunk failed: %s", cudaGetErrorString(ec));
      return RHMC_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      set_error("graph instantiation failed: %s", cudaGetErrorString(ei));
      return RHMC_ERR_CUDA;
    }
    L.graphs.push_back({key, exec, captured, 0});
    hit = &L.graphs.back();
  }
  hit->last_use = ++L.graph_clock;
  RHMC_CUDA_TRY(cudaGraphLaunch(hit->exec, s));
  g_launches.fetch_add(hit->launches);
  return RHMC_OK;
}

// Device time between marks on one stream (events; read after the stream has
// been synchronised).
struct PhaseTimer {
  cudaStream_t s;
  cudaEvent_t ev[3] = {};
  int n = 0;
  explicit PhaseTimer(cudaStream_t s_) : s(s_) {
    for (auto &e : ev) cudaEventCreate(&e);
    cudaEventRecord(ev[n++], s);
  }
  void mark() {
    if (n < 3) cudaEventRecord(ev[n++], s);
  }
  double ms(int phase) {
    float t = 0.f;
    if (phase + 1 >= n || cudaEventSynchronize(ev[phase + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, ev[phase], ev[phase + 1]) != cudaSuccess)
      return 0.0;
    return t;
  }
  ~PhaseTimer() {
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
  }
};

// Core solve of (A + sigma_s) X^(s) = B, shifts ascending, X FP64 [ns][len].
// Returns OK when the recursive residuals reached the target (phase 1 only).
template <typename T>
static rhmc_status_t solve_phase1(rhmc_ctx *c, const double2 *B, int n, int ns, const double *shifts, double2 *X,
                                  const SolveParams &prm, const SolveBufs &b0, SolveStats &stats, cudaStream_t s) {
  const bool mixed = std::is_same<T, float>::value;
  const long rows = c->g.Vh * 3;
  const long len = rows * n;
  const double sigma0 = shifts[0];
  // stored-basis mode (mixed, several shifts, not accumulating): b.basis set
  SolveBufs b = b0;
  if (!mixed || ns < 2 || b.accumulate) b.basis = nullptr, b.hist = nullptr, b.cap = 0;
  // X^(s) = sum_i Q_i C_i (want_p = 0), or P^(s) = sum_{i <= K} Q_i D_i (want_p = 1),
  // for s >= 1 from the stored basis (tcgen05 kernel whose epilogue writes the FP64
  // solutions; RHMC_TUNE_BASIS_CHUNK: FP32 partial sums over that many blocks).  X^(s),
  // s >= 1, is zero until then: the shifted increments are not updated in this mode.
  auto assemble = [&](int K, int want_p) -> rhmc_status_t {
    if (K <= 0 && !want_p) return RHMC_OK;
    return basis_assemble(b.asmb, n, ns, b.st, rows, K, want_p, X, (float2 *)b.P, len, tune_get(TUNE_BASIS_CHUNK),
                          tune_get(TUNE_BASIS_GEMM) == 1, tune_get(TUNE_BASIS_ACC_KT), &b.st->device_timeout, s);
  };
  // end of the stored-basis mode at iteration K: the shifted solutions so far into X
  auto finish_basis = [&](int K) -> rhmc_status_t {
    if (!b.basis) return RHMC_OK;
    RHMC_TRY(assemble(K, 0));
    b.basis = nullptr, b.hist = nullptr, b.cap = 0;
    StateView vf;
    RHMC_TRY(read_state(c, b.st, vf, s));
    if (vf.device_timeout) {
      set_error("a bounded device-side wait expired in the stored-basis assembly");
      return RHMC_ERR_DEVICE_TIMEOUT;
    }
    return RHMC_OK;
  };
  // FP32 increments to flush into X: in the stored-basis mode those of the shifts s >= 1
  // stay zero (their solutions come from the assembly), so only the base system's
  auto nflush = [&]() { return b.basis ? 1 : ns; };
  RHMC_CUDA_TRY(cudaMemcpyAsync(b.st->sigma, shifts, sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  // accumulating solve: X^(0) and one field for sum_{s>=1} w_s X^(s)
  RHMC_CUDA_TRY(cudaMemsetAsync(X, 0, sizeof(double2) * len * (b.accumulate ? std::min(ns, 2) : ns), s));
  // initialisation: {Q_0, delta_0} = qr(B) (FP64 Gram), P^(s) = Q_0
  if (mixed) {
    // the FP32 basis only needs FP32 orthonormality: QR of the rounded block
    RHMC_TRY((convert<double, float>(B, (float2 *)b.W, len, s)));
    RHMC_TRY(gram<float>((float2 *)b.W, (float2 *)b.W, rows, n, b.gscratch, b.partial, s));
    RHMC_TRY(nxn_qr_init<float>(b.partial, kGramParts, n, ns, b.st, (float2 *)b.mw, s));
    RHMC_TRY((block_axpy<float, float>((float2 *)b.W, nullptr, (float2 *)b.mw, (float2 *)b.Qb[0], rows, n, s)));
  } else {
    RHMC_TRY(gram<double>(B, B, rows, n, b.gscratch, b.partial, s));
    RHMC_TRY(nxn_qr_init<double>(b.partial, kGramParts, n, ns, b.st, b.rinv64, s));
    RHMC_TRY(block_axpy<double, T>(B, nullptr, b.rinv64, (C<T> *)b.Qb[0], rows, n, s));
  }
  for (int q = 0; q < ns; ++q)
    RHMC_CUDA_TRY(cudaMemcpyAsync((C<T> *)b.P + q * len, b.Qb[0], sizeof(C<T>) * len, cudaMemcpyDeviceToDevice, s));
  if (mixed) RHMC_CUDA_TRY(cudaMemsetAsync(b.Xinc, 0, sizeof(float2) * len * ns, s));
  if (b.basis) RHMC_TRY(basis_store((const float2 *)b.Qb[0], b.basis, rows, n, b.cap, 0, s));
  if (prm.acc_w) RHMC_CUDA_TRY(cudaMemcpyAsync(b.st->w1, prm.acc_w, sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  StateView v;
  RHMC_TRY(read_state(c, b.st, v, s));
  if (v.breakdown) {
    set_error("breakdown: right-hand-side block is rank deficient");
    return RHMC_ERR_BREAKDOWN;
  }
  const double target = prm.tol;
  // Shifted systems freeze once their recursive residuals are below
  // max(tol, RHMC_TUNE_SHIFT_FREEZE_NANO x 1e-9) in mixed precision.  Built-in:
  // tol.  Freezing earlier (their true residuals stop near the FP32 drift level)
  // shortens phase 1 but costs more in the corrections: at 24^4, n = 16, 1e-6
  // gave 211 + 256 ms against 235 + 158 ms (the large shifts drift little when
  // run to tol and then need almost no correction).
  const int fz = tune_get(TUNE_SHIFT_FREEZE_NANO);
  const double tol_shift = mixed ? std::max(target, fz > 0 ? 1e-9 * fz : kShiftFreezeMixed) : target;
  double res_at_reliable = 1.0;
  const int check_every = prm.check_every > 0                ? prm.check_every
                          : tune_get(TUNE_CHECK_EVERY) > 0 ? tune_get(TUNE_CHECK_EVERY)
                                                           : kCheckEvery;
  const int flush_every = tune_get(TUNE_FLUSH_EVERY);
  const double rel_delta = tune_get(TUNE_RELIABLE_DELTA_MILLI) > 0 ? 1e-3 * tune_get(TUNE_RELIABLE_DELTA_MILLI)
                                                                     : kReliableDelta;
  int k = 0, last_flush = 0;
  const int kmax = prm.fixed_iters > 0 ? prm.fixed_iters : prm.max_iter;
  while (k < kmax) {
    const int chunk = prm.fixed_iters > 0 ? kmax : std::min(check_every, kmax - k);
    const int freeze = prm.fixed_iters > 0 ? 0 : 1;
    if (b.basis && k + chunk > b.cap - 1) {
      // the basis is full: X^(s) and P^(s) from it, then the shifted updates in HBM
      RHMC_TRY(assemble(k, 0));
      RHMC_TRY(assemble(k, 1));
      b.basis = nullptr, b.hist = nullptr, b.cap = 0;
    }
    // a captured chunk replays for every later chunk with the same start modulo kCheckEvery
    // (the k % 2 buffer and k % 3 state-slot patterns), so its length must divide kCheckEvery
    const bool graph = use_graphs() && chunk == check_every && kCheckEvery % check_every == 0 && k > 0 &&
                       k % check_every == 0;
    if (graph)
      RHMC_TRY(run_chunk_graph<T>(c, b, X, n, ns, sigma0, k, chunk, tol_shift, freeze, s));
    else
      RHMC_TRY(run_chunk<T>(c, b, X, n, ns, sigma0, k, chunk, tol_shift, freeze, s));
    k += chunk;
    stats.dirac += chunk;
    RHMC_TRY(read_state(c, b.st, v, s));
    if (v.device_timeout) {
      set_error("a bounded device-side wait expired in the tensor-core update (iteration %d)", k);
      stats.iters = k;
      return RHMC_ERR_DEVICE_TIMEOUT;
    }
    if (v.breakdown) {
      set_error("breakdown in coefficient step %d at iteration %d", v.breakdown, k);
      stats.iters = k;
      return RHMC_ERR_BREAKDOWN;
    }
    if (prm.fixed_iters > 0) break;
    double base = 0.0;
    for (int j = 0; j < n; ++j) base = std::max(base, v.res[0][j]);
    if (!std::isfinite(base)) {
      set_error("non-finite residual at iteration %d", k);
      stats.iters = k;
      return RHMC_ERR_BREAKDOWN;
    }
    bool shifts_done = true;
    for (int q = 1; q < ns; ++q) shifts_done = shifts_done && !v.active[q];
    const bool converged = base < target && shifts_done;
    if (mixed && flush_every > 0 && k - last_flush >= flush_every) {
      for (int q = 0; q < nflush(); ++q) RHMC_TRY(flush(X + q * len, (float2 *)b.Xinc + q * len, len, s));
      last_flush = k;
    }
    if (mixed && converged && !prm.verify_at_convergence) {
      for (int q = 0; q < nflush(); ++q) RHMC_TRY(flush(X + q * len, (float2 *)b.Xinc + q * len, len, s));
      RHMC_TRY(finish_basis(k));
      stats.iters = k;
      return RHMC_OK;
    }
    if (mixed && prm.reliable && (base < rel_delta * res_at_reliable || converged)) {
      // reliable update: flush FP32 increments, FP64 true base residual, re-QR
      for (int q = 0; q < nflush(); ++q) RHMC_TRY(flush(X + q * len, (float2 *)b.Xinc + q * len, len, s));
      // thin QR of the FP32-rounded true residual (Q is an FP32 basis)
      RHMC_TRY(residual_accurate(c, B, X, b.R64, (float2 *)b.W, b.AP64, b.T64, b.R64, n, sigma0, nullptr, s));
      RHMC_TRY(gram<float>((float2 *)b.W, (float2 *)b.W, rows, n, b.gscratch, b.partial, s));
      RHMC_TRY(nxn_reliable<float>(b.partial, kGramParts, n, b.st, k, (float2 *)b.mw, s));
      // (the stored basis keeps the replaced block: P^(s)_k was formed from it, and the
      // new Q_k enters the shifted systems only through the base recursion from k + 1 on)
      RHMC_TRY((block_axpy<float, float>((float2 *)b.W, nullptr, (float2 *)b.mw, (float2 *)b.Qb[k & 1], rows, n, s)));
      stats.dirac++;
      stats.reliable++;
      RHMC_TRY(read_state(c, b.st, v, s));
      if (v.breakdown) {
        // the true residual is numerically zero: every column has converged
        RHMC_TRY(finish_basis(k));
        stats.iters = k;
        return RHMC_OK;
      }
      base = 0.0;
      for (int j = 0; j < n; ++j) base = std::max(base, v.res[0][j]);
      res_at_reliable = base;
      if (base < target && shifts_done) {
        RHMC_TRY(finish_basis(k));
        stats.iters = k;
        return RHMC_OK;
      }
      continue;
    }
    if (converged) {
      RHMC_TRY(finish_basis(k));
      stats.iters = k;
      return RHMC_OK;
    }
  }
  if (mixed)
    for (int q = 0; q < nflush(); ++q) RHMC_TRY(flush(X + q * len, (float2 *)b.Xinc + q * len, len, s));
  RHMC_TRY(finish_basis(k));
  stats.iters = k;
  if (prm.fixed_iters > 0) return RHMC_OK;
  set_error("not converged after %d iterations", k);
  return RHMC_ERR_NOT_CONVERGED;
}

// Full solve with FP64 true residuals and per-shift defect correction.
static rhmc_status_t solve_all(rhmc_ctx *c, const double2 *B, int n, int ns, const double *shifts, double2 *X,
                               const SolveParams &prm, void *ws, rhmc_info_t *info, cudaStream_t s) {
  const long rows = c->g.Vh * 3;
  const long len = rows * n;
  Arena a(ws);
  SolveBufs b;
  layout_solve(a, c->g, n, ns, prm.mixed, b);
  SolveStats st;
  SolveParams p1 = prm;
  if (prm.fixed_iters <= 0) {
    // the multishift phase runs to kPhase1Margin x tol (recursive residuals; the base system's
    // is verified by a reliable update at convergence, every shift's by the FP64 check below)
    const int pm = tune_get(TUNE_PHASE1_MARGIN_MILLI);
    p1.tol = (pm > 0 && pm < 1000 ? 1e-3 * pm : kPhase1Margin) * prm.tol;
  }
  PhaseTimer timer(s);
  rhmc_status_t rc = prm.mixed ? solve_phase1<float>(c, B, n, ns, shifts, X, p1, b, st, s)
                               : solve_phase1<double>(c, B, n, ns, shifts, X, p1, b, st, s);
  timer.mark();
  if (rc != RHMC_OK && rc != RHMC_ERR_NOT_CONVERGED) return rc;
  const rhmc_status_t rc1 = rc;

  // phase 2: FP64 true residual per shift, defect correction where needed.
  // The shifts are independent here: they are spread over up to `nl` lanes
  // (stream + host thread each, hardest shifts first), so that the
  // latency-bound parts of one correction overlap the bulk kernels of another.
  const int tl = tune_get(TUNE_REFINE_LANES);
  // one lane (no worker threads) under the library's profiler, and when a CUDA injection
  // library is loaded (a kernel profiler such as Nsight Compute: its replay of kernels
  // captured concurrently on several host threads ended the process with SIGSEGV)
  const bool injected = std::getenv("CUDA_INJECTION64_PATH") != nullptr;
  const int nl = (prof_on() || injected) ? 1 : std::min(refine_lanes(ns), tl > 0 ? tl : kRefineLanes);
  struct LaneWork {
    RefineBufs rb;
    SolveBufs b1;
    int refinements = 0, refine_iters = 0, dirac = 0;
    double worst = 0.0, worst1 = 0.0;
    rhmc_status_t rc = RHMC_OK;
    std::string err;
  };
  std::vector<LaneWork> work(nl);
  Arena ra(ws);
  for (auto &w : work) {
    w.rb.Bref = ra.take<double2>(len);
    w.rb.E = ra.take<double2>(len);
    layout_solve(ra, c->g, n, 1, prm.mixed, w.b1);
  }
  // work[*] overlaps b: phase-1 buffers are dead from here on (colnorms syncs s)
  double bn[kMaxN];
  RHMC_TRY(colnorms(c, B, n, bn, work[0].b1.npart, s));
  for (int j = 0; j < n; ++j) bn[j] = std::sqrt(bn[j]);
  std::vector<double> resid((size_t)ns * n, 0.0);

  auto refine_shift = [&](int q, LaneWork &w, cudaStream_t ls) -> rhmc_status_t {
    double2 *Xq = X + q * len;
    SolveBufs &b1 = w.b1;
    for (int round = 0;; ++round) {
      double rn[kMaxN];
      if (prm.mixed) {
        RHMC_TRY(residual_accurate(c, B, Xq, w.rb.Bref, nullptr, b1.AP64, b1.T64, b1.R64, n, shifts[q], b1.npart,
                                   ls));
        RHMC_TRY(read_colnorms(c, b1.npart, n, rn, ls));
      } else {
        RHMC_TRY(apply_A<double>(c, Xq, b1.AP64, b1.T64, n, shifts[q], ls));
        RHMC_TRY(sub(B, b1.AP64, w.rb.Bref, len, ls));
        RHMC_TRY(colnorms(c, w.rb.Bref, n, rn, b1.npart, ls));
      }
      w.dirac++;
      double mx = 0.0, ratio_min = 1e300;
      for (int j = 0; j < n; ++j) {
        const double r = std::sqrt(rn[j]) / bn[j];
        resid[(size_t)q * n + j] = r;
        mx = std::max(mx, r);
        if (r > 0) ratio_min = std::min(ratio_min, prm.tol / r);
      }
      if (round == 0) w.worst1 = std::max(w.worst1, mx);
      if (mx <= prm.tol || prm.fixed_iters > 0 || round >= kMaxRefine || tune_get(TUNE_NO_DEFECT_CORRECTION) == 1) {
        w.worst = std::max(w.worst, mx);
        return RHMC_OK;
      }
      // defect correction: (A + sigma_q) E = R, X_q += E
      SolveParams pr = prm;
      const int cm = tune_get(TUNE_CORRECTION_MARGIN_MILLI);
      pr.tol = std::min(0.1, (cm > 0 && cm < 1000 ? 1e-3 * cm : kCorrectionMargin) * ratio_min);
      pr.fixed_iters = 0;
      pr.verify_at_convergence = false;  // the FP64 true residual is checked right after
      // A correction needs only tol / r (about 1e-3) relative accuracy: far above the
      // FP32 recursion's own drift (about 1e-6 relative), so it runs without reliable
      // updates, and it is checked every kCorrectionCheckEvery iterations to stop closer
      // to its target
      pr.reliable = false;
      pr.check_every = tune_get(TUNE_CORRECTION_CHECK_EVERY) > 0 ? tune_get(TUNE_CORRECTION_CHECK_EVERY)
                                                                 : kCorrectionCheckEvery;
      SolveStats st1;
      rhmc_status_t rr = prm.mixed ? solve_phase1<float>(c, w.rb.Bref, n, 1, &shifts[q], w.rb.E, pr, b1, st1, ls)
                                   : solve_phase1<double>(c, w.rb.Bref, n, 1, &shifts[q], w.rb.E, pr, b1, st1, ls);
      if (rr != RHMC_OK && rr != RHMC_ERR_NOT_CONVERGED && rr != RHMC_ERR_BREAKDOWN) return rr;
      w.refinements++;
      w.refine_iters += st1.iters;
      w.dirac += st1.dirac;
      RHMC_TRY(add_inplace(Xq, w.rb.E, len, ls));  // X_q += E
    }
  };

  if (nl == 1) {
    for (int q = 0; q < ns && work[0].rc == RHMC_OK; ++q) work[0].rc = refine_shift(q, work[0], s);
    if (work[0].rc != RHMC_OK) return work[0].rc;
  } else {
    while ((int)c->lanes.size() < nl) {
      auto l = std::make_unique<SolverLane>();
      if (cudaStreamCreateWithFlags(&l->s, cudaStreamNonBlocking) != cudaSuccess ||
          cudaStreamCreateWithFlags(&l->cap, cudaStreamNonBlocking) != cudaSuccess) {
        l->release();
        set_error("cannot create a refinement stream");
        return RHMC_ERR_CUDA;
      }
      c->lanes.push_back(std::move(l));
    }
    std::atomic<int> next{0};
    std::vector<std::thread> pool;
    for (int l = 0; l < nl; ++l)
      pool.emplace_back([&, l] {
        DeviceGuard dg(c->device);
        TuneScope tscope(c);
        SolverLane *L = c->lanes[l].get();
        t_lane = L;
        LaneWork &w = work[l];
        for (int q = next++; q < ns && w.rc == RHMC_OK; q = next++) w.rc = refine_shift(q, w, L->s);
        if (cudaStreamSynchronize(L->s) != cudaSuccess && w.rc == RHMC_OK) {
          set_error("refinement stream: %s", cudaGetErrorString(cudaGetLastError()));
          w.rc = RHMC_ERR_CUDA;
        }
        if (w.rc != RHMC_OK) w.err = rhmc_last_error();
        t_lane = nullptr;
      });
    for (auto &t : pool) t.join();
    for (auto &w : work)
      if (w.rc != RHMC_OK) {
        set_error("%s", w.err.c_str());
        return w.rc;
      }
  }
  int refinements = 0, refine_iters = 0;
  double worst = 0.0, worst1 = 0.0;
  for (auto &w : work) {
    refinements += w.refinements;
    refine_iters += w.refine_iters;
    st.dirac += w.dirac;
    worst = std::max(worst, w.worst);
    worst1 = std::max(worst1, w.worst1);
  }
  timer.mark();
  if (info) {
    info->phase1_ms = timer.ms(0);
    info->refine_ms = timer.ms(1);
    info->iters = st.iters;
    info->dirac_calls = st.dirac;
    info->reliable_updates = st.reliable;
    info->refinements = refinements;
    info->refine_iters = refine_iters;
    info->true_rel_resid_max = worst;
    info->phase1_rel_resid_max = worst1;
    if (info->per_shift_resid) std::memcpy(info->per_shift_resid, resid.data(), sizeof(double) * resid.size());
  }
  if (prm.fixed_iters > 0) return RHMC_OK;
  if (worst > prm.tol) {
    set_error("true residual %.3e above tol %.3e after refinement (phase 1: %d)", worst, prm.tol, (int)rc1);
    return RHMC_ERR_NOT_CONVERGED;
  }
  return RHMC_OK;
}

rhmc_status_t ctx_geometry(const rhmc_ctx_t *c, int *device, Geom *g, double *mass, const double2 **l64_even,
                           const double2 **l64_odd) {
  if (!c->have_gauge) {
    set_error("gauge field not set");
    return RHMC_ERR_NO_GAUGE;
  }
  *device = c->device;
  *g = c->g;
  *mass = c->mass;
  *l64_even = c->l64[0];
  *l64_odd = c->l64[1];
  return RHMC_OK;
}

rhmc_status_t ctx_lattice(const rhmc_ctx_t *c, int *device, Geom *g) {
  if (!c) {
    set_error("null context");
    return RHMC_ERR_INVALID_ARG;
  }
  *device = c->device;
  *g = c->g;
  return RHMC_OK;
}

rhmc_status_t ctx_partials(rhmc_ctx_t *c, double **parts, int *nparts) {
  if (!c->d_parts) RHMC_CUDA_TRY(cudaMalloc(&c->d_parts, sizeof(double) * kParts));
  *parts = c->d_parts;
  *nparts = kParts;
  return RHMC_OK;
}

rhmc_status_t ctx_md_buffer(rhmc_ctx_t *c, size_t bytes, void **buf) {
  if (c->md_bytes < bytes) {
    if (c->md_buf) {
      RHMC_CUDA_TRY(cudaDeviceSynchronize());
      RHMC_CUDA_TRY(cudaFree(c->md_buf));
    }
    c->md_buf = nullptr;
    c->md_bytes = 0;
    RHMC_CUDA_TRY(cudaMalloc(&c->md_buf, bytes));
    c->md_bytes = bytes;
  }
  *buf = c->md_buf;
  return RHMC_OK;
}

// ------------------------------------------------------------ per-vector SCG baseline
static size_t scg_bytes(const Geom &g, int ns) {
  Arena a(nullptr);
  const size_t len = (size_t)g.Vh * 3;
  a.take<double2>(len);           // b
  a.take<double2>(len);           // r
  a.take<double2>(len);           // Ap
  a.take<double2>(len);           // tmp (odd)
  a.take<double2>(len * ns);      // p
  a.take<double2>(len * ns);      // x
  a.take<double>(kParts);
  a.take<double>(kMaxS);
  a.take<ScgScalars>(1);
  return a.off + 256;
}

}  // namespace rhmc

// =================================================================== C ABI
extern "C" {

const char *rhmc_last_error(void) { return rhmc::g_err; }

long long rhmc_kernel_launches(void) { return rhmc::g_launches.load(); }

rhmc_status_t rhmc_tune_set(int key, int value) {
  if (key < 0 || key >= rhmc::TUNE_NKEYS || value < 0) {
    set_error("rhmc_tune_set: bad key %d or value %d", key, value);
    return RHMC_ERR_INVALID_ARG;
  }
  rhmc::g_tune[key] = value;
  return RHMC_OK;
}

int rhmc_tune_get(int key) { return (key >= 0 && key < rhmc::TUNE_NKEYS) ? rhmc::g_tune[key] : 0; }

rhmc_status_t rhmc_ctx_tune_set(rhmc_ctx_t *c, int key, int value) {
  if (!c || key < 0 || key >= rhmc::TUNE_NKEYS || value < 0) {
    set_error("rhmc_ctx_tune_set: bad context, key %d or value %d", key, value);
    return RHMC_ERR_INVALID_ARG;
  }
  c->tune[key] = value;
  return RHMC_OK;
}

int rhmc_ctx_tune_get(const rhmc_ctx_t *c, int key) {
  if (!c || key < 0 || key >= rhmc::TUNE_NKEYS) return 0;
  return c->tune[key] > 0 ? c->tune[key] : rhmc::g_tune[key];
}

rhmc_status_t rhmc_profile_enable(int on) {
  rhmc::g_recs.clear();
  rhmc::g_pool_next = 0;
  rhmc::g_prof = on != 0;
  return RHMC_OK;
}

rhmc_status_t rhmc_profile_read(int cat, long long *launches, double *ms, double *bytes) {
  if (cat < 0 || cat >= rhmc::PROF_NCAT || !launches || !ms || !bytes) {
    set_error("rhmc_profile_read: bad argument");
    return RHMC_ERR_INVALID_ARG;
  }
  *launches = 0;
  *ms = 0.0;
  *bytes = 0.0;
  for (auto &r : rhmc::g_recs) {
    if (r.cat != cat) continue;
    RHMC_CUDA_TRY(cudaEventSynchronize(r.b));
    float t = 0.f;
    RHMC_CUDA_TRY(cudaEventElapsedTime(&t, r.a, r.b));
    *launches += 1;
    *ms += t;
    *bytes += r.bytes;
  }
  return RHMC_OK;
}

rhmc_status_t rhmc_profile_read_flops(int cat, double *flops) {
  if (cat < 0 || cat >= rhmc::PROF_NCAT || !flops) {
    set_error("rhmc_profile_read_flops: bad argument");
    return RHMC_ERR_INVALID_ARG;
  }
  *flops = 0.0;
  for (auto &r : rhmc::g_recs)
    if (r.cat == cat) *flops += r.flops;
  return RHMC_OK;
}

rhmc_status_t rhmc_create(rhmc_ctx_t **out, const rhmc_lattice_t *lat, int device) {
  if (!out || !lat) {
    set_error("rhmc_create: null argument");
    return RHMC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  for (int mu = 0; mu < 4; ++mu)
    if (lat->dims[mu] < 2 || lat->dims[mu] % 2) {
      set_error("rhmc_create: extent %d of direction %d must be even and >= 2", lat->dims[mu], mu);
      return RHMC_ERR_INVALID_ARG;
    }
  if (!(lat->mass >= 0.0)) {
    set_error("rhmc_create: mass must be >= 0");
    return RHMC_ERR_INVALID_ARG;
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    set_error("rhmc_create: no CUDA device %d", device);
    return RHMC_ERR_CUDA;
  }
  DeviceGuard dg(device);
  rhmc_ctx *c = new rhmc_ctx();
  c->device = device;
  for (int mu = 0; mu < 4; ++mu) c->g.L[mu] = lat->dims[mu];
  c->g.Lxh = lat->dims[0] / 2;
  c->g.V = (long)lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3];
  c->g.Vh = c->g.V / 2;
  c->mass = lat->mass;
  c->bc_t = lat->bc_t == 1 ? 1 : -1;
  for (int p = 0; p < 2; ++p) {
    if (cudaMalloc(&c->l64[p], sizeof(double2) * 72 * c->g.Vh) != cudaSuccess ||
        cudaMalloc(&c->l32[p], sizeof(float2) * 72 * c->g.Vh) != cudaSuccess ||
        cudaMalloc(&c->ldf[p], sizeof(float4) * 72 * c->g.Vh) != cudaSuccess ||
        cudaMalloc(&c->l12[p], sizeof(float2) * 48 * c->g.Vh) != cudaSuccess) {
      set_error("rhmc_create: out of device memory for links");
      rhmc_destroy(c);
      return RHMC_ERR_CUDA;
    }
  }
  // the side stream (shifted steps) yields to the base recursion: lowest
  // priority; captured chunks of the base recursion run at the highest
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->main.cap, cudaStreamNonBlocking, prio_hi) != cudaSuccess) {
    set_error("rhmc_create: cannot create the side stream");
    rhmc_destroy(c);
    return RHMC_ERR_CUDA;
  }
  for (int q = 0; q < 3; ++q)
    if (cudaEventCreateWithFlags(&c->ev_base[q], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_side[q], cudaEventDisableTiming) != cudaSuccess) {
      set_error("rhmc_create: cannot create events");
      rhmc_destroy(c);
      return RHMC_ERR_CUDA;
    }
  *out = c;
  return RHMC_OK;
}

rhmc_status_t rhmc_destroy(rhmc_ctx_t *c) {
  if (!c) return RHMC_OK;
  DeviceGuard dg(c->device);
  for (int p = 0; p < 2; ++p) {
    if (c->l64[p]) cudaFree(c->l64[p]);
    if (c->l32[p]) cudaFree(c->l32[p]);
    if (c->ldf[p]) cudaFree(c->ldf[p]);
    if (c->l12[p]) cudaFree(c->l12[p]);
  }
  if (c->side) cudaStreamSynchronize(c->side);
  for (auto &l : c->lanes) {
    if (l->s) cudaStreamSynchronize(l->s);
    l->release();
  }
  c->lanes.clear();
  c->main.release();
  if (c->pool) cudaFree(c->pool);
  if (c->d_parts) cudaFree(c->d_parts);
  if (c->md_buf) cudaFree(c->md_buf);
  for (int q = 0; q < 3; ++q) {
    if (c->ev_base[q]) cudaEventDestroy(c->ev_base[q]);
    if (c->ev_side[q]) cudaEventDestroy(c->ev_side[q]);
  }
  if (c->side) cudaStreamDestroy(c->side);
  if (c->own) cudaStreamDestroy(c->own);
  delete c;
  return RHMC_OK;
}

rhmc_status_t rhmc_set_gauge(rhmc_ctx_t *c, const void *U, rhmc_stream_t sv) {
  if (!c || !U) {
    set_error("rhmc_set_gauge: null argument");
    return RHMC_ERR_INVALID_ARG;
  }
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  RHMC_TRY(stage_links(c->g, (const double2 *)U, c->bc_t, c->l64, c->l32, s));
  for (int p = 0; p < 2; ++p) RHMC_TRY(stage_links_df(c->g, c->l64[p], c->ldf[p], s));
  RHMC_TRY(stage_links12(c->g, c->bc_t, c->l32, c->l12, &c->rec12, s));
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  c->have_gauge = true;
  return RHMC_OK;
}

size_t rhmc_workspace_bytes(const rhmc_ctx_t *c, int n, int ns, rhmc_precision_t p) {
  if (!c || n < 1 || n > RHMC_MAX_NRHS || ns < 1 || ns > RHMC_MAX_SHIFTS) return 0;
  // sized under the context's own settings and device, as its solves lay it out
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  const bool mixed = p == RHMC_MIXED_FP32;
  // solve with an internal X (unsorted shifts or force) + force's Y fields
  const size_t len = (size_t)c->g.Vh * 3 * n;
  size_t solve = solve_bytes(c->g, n, ns, mixed, true);
  size_t force = sizeof(double2) * len * ns * 2 + sizeof(double) * (kMaxS + kParts) + 4096;
  return std::max(solve, force) + sizeof(double2) * len * ns + 4096;
}

static rhmc_status_t check_common(rhmc_ctx_t *c, const void *a, const void *b, int n) {
  if (!c || !a || !b) {
    set_error("null argument");
    return RHMC_ERR_INVALID_ARG;
  }
  if (n < 1 || n > RHMC_MAX_NRHS) {
    set_error("n_rhs = %d out of range [1, %d]", n, RHMC_MAX_NRHS);
    return RHMC_ERR_INVALID_ARG;
  }
  if (!c->have_gauge) {
    set_error("gauge field not set");
    return RHMC_ERR_NO_GAUGE;
  }
  return RHMC_OK;
}

rhmc_status_t rhmc_apply_mdagm_mrhs(rhmc_ctx_t *c, const void *X, void *Y, int n, double sigma, rhmc_precision_t p,
                                    rhmc_stream_t sv) {
  RHMC_TRY(check_common(c, X, Y, n));
  if (X == Y) {
    set_error("X and Y may not alias");
    return RHMC_ERR_INVALID_ARG;
  }
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  const long len = c->g.Vh * 3 * n;
  if (p == RHMC_FP64) {
    RHMC_TRY(ensure_pool(c, sizeof(double2) * len + 256));
    return apply_A<double>(c, (const double2 *)X, (double2 *)Y, (double2 *)c->pool, n, sigma, s);
  }
  if (p == RHMC_DF64) {
    RHMC_TRY(ensure_pool(c, 2 * (sizeof(double2) * len + 256)));
    Arena a(c->pool);
    double2 *tmp = a.take<double2>(len), *split = a.take<double2>(len);
    return apply_A_df(c, (const double2 *)X, (double2 *)Y, tmp, split, n, sigma, s);
  }
  RHMC_TRY(ensure_pool(c, 3 * (sizeof(float2) * len + 256)));
  Arena a(c->pool);
  float2 *x32 = a.take<float2>(len), *y32 = a.take<float2>(len), *t32 = a.take<float2>(len);
  RHMC_TRY((convert<double, float>((const double2 *)X, x32, len, s)));
  RHMC_TRY(apply_A<float>(c, x32, y32, t32, n, sigma, s));
  RHMC_TRY((convert<float, double>(y32, (double2 *)Y, len, s)));
  return RHMC_OK;
}

rhmc_status_t rhmc_hop(rhmc_ctx_t *c, const void *X, void *Y, int n, int out_par, rhmc_precision_t p,
                       rhmc_stream_t sv) {
  RHMC_TRY(check_common(c, X, Y, n));
  if (X == Y || (out_par != 0 && out_par != 1)) {
    set_error("rhmc_hop: aliasing or bad parity");
    return RHMC_ERR_INVALID_ARG;
  }
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  const long len = c->g.Vh * 3 * n;
  if (p == RHMC_FP64) return hop<double>(c->g, out_par, c->l64[out_par], (const double2 *)X, (double2 *)Y, nullptr, 0, n, 1, 0, s);
  if (p == RHMC_DF64) {
    RHMC_TRY(ensure_pool(c, sizeof(double2) * len + 256));
    RHMC_TRY(df_split((const double2 *)X, (float4 *)c->pool, len, s));
    RHMC_TRY(hop_df(c->g, out_par, c->ldf[out_par], (const float4 *)c->pool, (float4 *)Y, nullptr, 0.0, n, s));
    return df_merge((float4 *)Y, len, s);
  }
  RHMC_TRY(ensure_pool(c, 2 * (sizeof(float2) * len + 256)));
  Arena a(c->pool);
  float2 *x32 = a.take<float2>(len), *y32 = a.take<float2>(len);
  RHMC_TRY((convert<double, float>((const double2 *)X, x32, len, s)));
  RHMC_TRY(hop<float>(c->g, out_par, c->l32[out_par], x32, y32, nullptr, 0, n, 1, 0, s,
                      Links12Of<float>::get(c, out_par), c->bc_t));
  RHMC_TRY((convert<float, double>(y32, (double2 *)Y, len, s)));
  return RHMC_OK;
}

static rhmc_status_t check_shifts(int ns, const double *shifts, double tol) {
  if (ns < 1 || ns > RHMC_MAX_SHIFTS || !shifts) {
    set_error("n_shifts = %d out of range [1, %d] or null shifts", ns, RHMC_MAX_SHIFTS);
    return RHMC_ERR_INVALID_ARG;
  }
  for (int q = 0; q < ns; ++q)
    if (!(shifts[q] >= 0.0) || !std::isfinite(shifts[q])) {
      set_error("shift %d = %g must be finite and >= 0", q, shifts[q]);
      return RHMC_ERR_INVALID_ARG;
    }
  if (!(tol > 0.0) || !(tol < 1.0)) {
    set_error("tol = %g must be in (0, 1)", tol);
    return RHMC_ERR_INVALID_ARG;
  }
  return RHMC_OK;
}

static int default_max_iter(const rhmc_ctx *c, double sigma0, double tol) {
  const double lo = 4.0 * c->mass * c->mass + sigma0;
  const double kappa = (lo > 0) ? (64.0 + lo) / lo : 1e12;
  const double it = 10.0 * std::sqrt(kappa) * std::log(1.0 / tol) + 100.0;
  return (int)std::min(it, 1e6);
}

// Solve into caller X (any shift order) using workspace ws.
static rhmc_status_t block_solve_entry(rhmc_ctx_t *c, const double2 *B, int n, int ns, const double *shifts,
                                       double2 *X, double tol, int max_iter, bool mixed, int fixed_iters, void *ws,
                                       rhmc_info_t *info, cudaStream_t s) {
  const long len = c->g.Vh * 3 * n;
  std::vector<int> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return shifts[a] < shifts[b]; });
  bool sorted = true;
  for (int q = 0; q < ns; ++q) sorted = sorted && order[q] == q;
  std::vector<double> sh(ns);
  for (int q = 0; q < ns; ++q) sh[q] = shifts[order[q]];
  SolveParams prm{tol, max_iter > 0 ? max_iter : default_max_iter(c, sh[0], tol), mixed, fixed_iters};
  std::vector<double> resid((size_t)ns * n);
  rhmc_info_t local{};
  local.per_shift_resid = resid.data();
  rhmc_status_t rc;
  if (sorted) {
    rc = solve_all(c, B, n, ns, sh.data(), X, prm, ws, &local, s);
  } else {
    Arena a(ws);
    double2 *Xs = a.take<double2>((size_t)ns * len);
    rc = solve_all(c, B, n, ns, sh.data(), Xs, prm, (char *)ws + a.off, &local, s);
    if (rc == RHMC_OK || rc == RHMC_ERR_NOT_CONVERGED)
      for (int q = 0; q < ns; ++q)
        RHMC_CUDA_TRY(cudaMemcpyAsync(X + (size_t)order[q] * len, Xs + (size_t)q * len, sizeof(double2) * len,
                                      cudaMemcpyDeviceToDevice, s));
  }
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    double *user = info->per_shift_resid;
    *info = local;
    info->per_shift_resid = user;
    if (user)
      for (int q = 0; q < ns; ++q)
        for (int j = 0; j < n; ++j) user[(size_t)order[q] * n + j] = resid[(size_t)q * n + j];
  }
  return rc;
}

rhmc_status_t rhmc_block_multishift_cg(rhmc_ctx_t *c, const void *B, int n, int ns, const double *shifts, void *X,
                                       double tol, int max_iter, rhmc_precision_t p, void *ws, rhmc_info_t *info,
                                       rhmc_stream_t sv) {
  RHMC_TRY(check_common(c, B, X, n));
  RHMC_TRY(check_shifts(ns, shifts, tol));
  if (p != RHMC_FP64 && p != RHMC_MIXED_FP32) {
    set_error("precision %d not supported by the solver", (int)p);
    return RHMC_ERR_INVALID_ARG;
  }
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  if (!ws) {
    RHMC_TRY(ensure_pool(c, rhmc_workspace_bytes(c, n, ns, p)));
    ws = c->pool;
  }
  return block_solve_entry(c, (const double2 *)B, n, ns, shifts, (double2 *)X, tol, max_iter, p == RHMC_MIXED_FP32,
                           0, ws, info, s);
}

rhmc_status_t rhmc_block_multishift_cg_batch(rhmc_batch_item_t *items, int count, double tol, int max_iter,
                                             rhmc_precision_t p, rhmc_stream_t sv) {
  if (!items || count < 1 || count > 64) {
    set_error("rhmc_block_multishift_cg_batch: bad item list (count %d)", count);
    return RHMC_ERR_INVALID_ARG;
  }
  for (int i = 0; i < count; ++i) {
    rhmc_batch_item_t &it = items[i];
    it.status = check_common(it.ctx, it.B, it.X, it.n_rhs);
    if (it.status == RHMC_OK) it.status = check_shifts(it.n_shifts, it.shifts, tol);
    if (it.status != RHMC_OK) return it.status;
    for (int j = 0; j < i; ++j)
      if (items[j].ctx == it.ctx) {
        set_error("rhmc_block_multishift_cg_batch: items %d and %d share a context", j, i);
        return RHMC_ERR_INVALID_ARG;
      }
  }
  cudaStream_t s = (cudaStream_t)sv;
  cudaEvent_t start;
  RHMC_CUDA_TRY(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
  RHMC_CUDA_TRY(cudaEventRecord(start, s));
  std::vector<std::string> msg(count);
  std::vector<std::thread> pool;
  for (int i = 0; i < count; ++i)
    pool.emplace_back([&, i] {
      rhmc_batch_item_t &it = items[i];
      rhmc_ctx *c = it.ctx;
      DeviceGuard dg(c->device);
      TuneScope tscope(c);
      cudaStreamWaitEvent(c->own, start, 0);
      void *ws = it.workspace;
      if (!ws) {
        it.status = ensure_pool(c, rhmc_workspace_bytes(c, it.n_rhs, it.n_shifts, p));
        ws = c->pool;
      }
      if (it.status == RHMC_OK)
        it.status = block_solve_entry(c, (const double2 *)it.B, it.n_rhs, it.n_shifts, it.shifts, (double2 *)it.X,
                                      tol, max_iter, p == RHMC_MIXED_FP32, 0, ws, it.info, c->own);
      if (it.status != RHMC_OK) msg[i] = rhmc_last_error();
    });
  for (auto &t : pool) t.join();
  cudaEventDestroy(start);
  rhmc_status_t worst = RHMC_OK;
  for (int i = 0; i < count; ++i) {
    // the caller's stream continues after every item's work
    cudaEvent_t done;
    RHMC_CUDA_TRY(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    RHMC_CUDA_TRY(cudaEventRecord(done, items[i].ctx->own));
    RHMC_CUDA_TRY(cudaStreamWaitEvent(s, done, 0));
    cudaEventDestroy(done);
    if (items[i].status != RHMC_OK && worst == RHMC_OK) {
      worst = items[i].status;
      set_error("batch item %d: %s", i, msg[i].c_str());
    }
  }
  return worst;
}

rhmc_status_t rhmc_multishift_cg_pervector(rhmc_ctx_t *c, const void *Bv, int n, int ns, const double *shifts,
                                           void *Xv, double tol, int max_iter, void *ws, rhmc_info_t *info,
                                           rhmc_stream_t sv) {
  RHMC_TRY(check_common(c, Bv, Xv, n));
  RHMC_TRY(check_shifts(ns, shifts, tol));
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  const size_t need = scg_bytes(c->g, ns);
  if (!ws) {
    RHMC_TRY(ensure_pool(c, need));
    ws = c->pool;
  }
  std::vector<int> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return shifts[a] < shifts[b]; });
  std::vector<double> sh(ns);
  for (int q = 0; q < ns; ++q) sh[q] = shifts[order[q]];
  const long len1 = c->g.Vh * 3;
  const long lenb = len1 * n;
  Arena a(ws);
  double2 *b = a.take<double2>(len1), *r = a.take<double2>(len1), *Ap = a.take<double2>(len1),
          *tmp = a.take<double2>(len1), *p = a.take<double2>(len1 * ns), *x = a.take<double2>(len1 * ns);
  double *parts = a.take<double>(kParts), *sig = a.take<double>(kMaxS);
  ScgScalars *sc = a.take<ScgScalars>(1);
  RHMC_CUDA_TRY(cudaMemcpyAsync(sig, sh.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  const int kmax = max_iter > 0 ? max_iter : default_max_iter(c, sh[0], tol);
  const double a0 = 4.0 * c->mass * c->mass + sh[0];
  int total_iters = 0, dirac = 0;
  bool all_ok = true;
  RHMC_TRY(ensure_pinned(c, sizeof(ScgScalars)));
  for (int j = 0; j < n; ++j) {
    RHMC_TRY(column((const double2 *)Bv, b, len1, n, j, 1, s));
    RHMC_CUDA_TRY(cudaMemcpyAsync(r, b, sizeof(double2) * len1, cudaMemcpyDeviceToDevice, s));
    for (int q = 0; q < ns; ++q)
      RHMC_CUDA_TRY(cudaMemcpyAsync(p + q * len1, b, sizeof(double2) * len1, cudaMemcpyDeviceToDevice, s));
    RHMC_CUDA_TRY(cudaMemsetAsync(x, 0, sizeof(double2) * len1 * ns, s));
    RHMC_TRY(redot(r, r, len1, parts, kParts, s));
    RHMC_TRY(scg_init(sc, parts, kParts, ns, sig, s));
    int k = 0;
    bool done = false;
    while (k < kmax && !done) {
      const int chunk = std::min(kCheckEvery, kmax - k);
      for (int q = 0; q < chunk; ++q) {
        ++k;
        RHMC_TRY(hop<double>(c->g, 1, c->l64[1], p, tmp, nullptr, 0.0, 1, 1, 0, s));
        RHMC_TRY(hop<double>(c->g, 0, c->l64[0], tmp, Ap, p, a0, 1, 1, 0, s));
        RHMC_TRY(redot(p, Ap, len1, parts, kParts, s));
        RHMC_TRY(scg_alpha(sc, parts, kParts, ns, s));
        RHMC_TRY(scg_update1(sc, r, Ap, x, p, ns, len1, parts, kParts, s));
        RHMC_TRY(scg_beta(sc, parts, kParts, ns, tol, s));
        RHMC_TRY(scg_update2(sc, r, p, ns, len1, s));
        dirac++;
      }
      ScgScalars *h = reinterpret_cast<ScgScalars *>(lane(c).h_pin);
      RHMC_CUDA_TRY(cudaMemcpyAsync(h, sc, sizeof(ScgScalars), cudaMemcpyDeviceToHost, s));
      RHMC_CUDA_TRY(cudaStreamSynchronize(s));
      if (h->breakdown) {
        set_error("scg breakdown (p^dagger A p <= 0)");
        return RHMC_ERR_BREAKDOWN;
      }
      bool act = false;
      for (int q = 1; q < ns; ++q) act = act || h->active[q];
      done = h->rel < tol && !act;
    }
    all_ok = all_ok && done;
    total_iters += k;
    for (int q = 0; q < ns; ++q) RHMC_TRY(column(x + q * len1, (double2 *)Xv + (size_t)order[q] * lenb, len1, n, j, 0, s));
  }
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  if (info) {
    info->iters = total_iters;
    info->dirac_calls = dirac;
    info->reliable_updates = 0;
    info->refinements = 0;
    info->refine_iters = 0;
    info->true_rel_resid_max = -1.0;
    info->phase1_rel_resid_max = -1.0;
  }
  if (!all_ok) {
    set_error("per-vector multishift CG not converged");
    return RHMC_ERR_NOT_CONVERGED;
  }
  return RHMC_OK;
}

rhmc_status_t rhmc_rational_apply(rhmc_ctx_t *c, const void *Phi, int n, double alpha0, const double *alpha,
                                  int ns, const void *X, void *Y, rhmc_stream_t sv) {
  RHMC_TRY(check_common(c, Phi, Y, n));
  if (!X || !alpha || ns < 1 || ns > RHMC_MAX_SHIFTS) {
    set_error("rhmc_rational_apply: null X/alpha or n_shifts out of range");
    return RHMC_ERR_INVALID_ARG;
  }
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  const long len = c->g.Vh * 3 * n;
  return rational_combine((const double2 *)Phi, alpha0, alpha, (const double2 *)X, ns, len, (double2 *)Y, s);
}

// R(A) Phi by the block multishift solve without per-shift solutions: FP64,
// shifts sorted ascending, X^(0) kept (its true residual is checked), the
// other shifts' solutions summed with their residues in the update kernel.
rhmc_status_t rhmc_rational_solve(rhmc_ctx_t *c, const void *Phi, int n, double alpha0, const double *alpha,
                                  const double *beta, int ns, double tol, int max_iter, void *Y, void *ws,
                                  rhmc_info_t *info, rhmc_stream_t sv) {
  RHMC_TRY(check_common(c, Phi, Y, n));
  if (!alpha || !beta || Phi == Y) {
    set_error("rhmc_rational_solve: null alpha/beta or aliased Phi and Y");
    return RHMC_ERR_INVALID_ARG;
  }
  RHMC_TRY(check_shifts(ns, beta, tol));
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  if (!ws) {
    RHMC_TRY(ensure_pool(c, rhmc_rational_solve_bytes(c, n, ns)));
    ws = c->pool;
  }
  const long len = c->g.Vh * 3 * n;
  std::vector<int> order(ns);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return beta[a] < beta[b]; });
  std::vector<double> sh(ns), w(ns);
  for (int q = 0; q < ns; ++q) {
    sh[q] = beta[order[q]];
    w[q] = alpha[order[q]];
  }
  Arena a(ws);
  double2 *X2 = a.take<double2>((size_t)2 * len);  // X^(0), sum_{s>=1} w_s X^(s)
  SolveBufs b;
  layout_solve(a, c->g, n, ns, false, b);
  b.accumulate = 1;
  SolveParams prm{tol, max_iter > 0 ? max_iter : default_max_iter(c, sh[0], tol), false, 0};
  prm.acc_w = w.data();
  SolveStats st;
  PhaseTimer timer(s);
  const rhmc_status_t rc = solve_phase1<double>(c, (const double2 *)Phi, n, ns, sh.data(), X2, prm, b, st, s);
  timer.mark();
  if (rc != RHMC_OK && rc != RHMC_ERR_NOT_CONVERGED) return rc;
  // recursive residuals of every shift, true FP64 residual of the base system
  StateView v;
  RHMC_TRY(read_state(c, b.st, v, s));
  double rec = 0.0;
  for (int q = 0; q < ns; ++q)
    for (int j = 0; j < n; ++j) rec = std::max(rec, v.res[q][j]);
  RHMC_TRY(apply_A<double>(c, X2, b.AP64, b.T64, n, sh[0], s));
  RHMC_TRY(sub((const double2 *)Phi, b.AP64, b.R64, len, s));
  double bn[kMaxN], rn[kMaxN];
  RHMC_TRY(colnorms(c, (const double2 *)Phi, n, bn, b.npart, s));
  RHMC_TRY(colnorms(c, b.R64, n, rn, b.npart, s));
  double tr = 0.0;
  for (int j = 0; j < n; ++j) tr = std::max(tr, std::sqrt(rn[j] / bn[j]));
  // Y = alpha0 Phi + w_0 X^(0) + sum_{s>=1} w_s X^(s)
  const double wts[2] = {w[0], 1.0};
  RHMC_TRY(rational_combine((const double2 *)Phi, alpha0, wts, X2, ns > 1 ? 2 : 1, len, (double2 *)Y, s));
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  timer.mark();
  if (info) {
    double *user = info->per_shift_resid;
    std::memset(info, 0, sizeof(*info));
    info->per_shift_resid = user;
    info->iters = st.iters;
    info->dirac_calls = st.dirac + 1;
    info->true_rel_resid_max = tr;
    info->phase1_rel_resid_max = rec;
    info->phase1_ms = timer.ms(0);
    info->refine_ms = timer.ms(1);
    if (user)
      for (int q = 0; q < ns; ++q)
        for (int j = 0; j < n; ++j) user[(size_t)order[q] * n + j] = v.res[q][j];
  }
  if (rc == RHMC_ERR_NOT_CONVERGED || rec > tol) {
    set_error("rational solve: recursive residual %.3e above tol %.3e", rec, tol);
    return RHMC_ERR_NOT_CONVERGED;
  }
  return RHMC_OK;
}

size_t rhmc_rational_solve_bytes(const rhmc_ctx_t *c, int n, int ns) {
  if (!c || n < 1 || n > RHMC_MAX_NRHS || ns < 1 || ns > RHMC_MAX_SHIFTS) return 0;
  Arena a(nullptr);
  a.take<double2>((size_t)2 * c->g.Vh * 3 * n);
  SolveBufs b;
  layout_solve(a, c->g, n, ns, false, b);
  return a.off + 256;
}

rhmc_status_t rhmc_force(rhmc_ctx_t *c, const void *Phi, int n, double alpha0, const double *alpha,
                         const double *beta, int ns, double tol, int max_iter, rhmc_precision_t p, const void *X_in,
                         void *G, double *S_out, void *ws, rhmc_info_t *info, rhmc_stream_t sv) {
  RHMC_TRY(check_common(c, Phi, G ? G : (void *)S_out, n));
  if (!alpha || !beta) {
    set_error("rhmc_force: null alpha/beta");
    return RHMC_ERR_INVALID_ARG;
  }
  RHMC_TRY(check_shifts(ns, beta, X_in ? 0.5 : tol));
  DeviceGuard dg(c->device);
  TuneScope tscope(c);
  cudaStream_t s = (cudaStream_t)sv;
  if (!ws) {
    RHMC_TRY(ensure_pool(c, rhmc_workspace_bytes(c, n, ns, p)));
    ws = c->pool;
  }
  const long len = c->g.Vh * 3 * n;
  Arena a(ws);
  double2 *X = (double2 *)X_in;
  if (!X) X = a.take<double2>((size_t)ns * len);
  void *rest = (char *)ws + a.off;
  if (!X_in) {
    const rhmc_status_t rc = block_solve_entry(c, (const double2 *)Phi, n, ns, beta, X, tol, max_iter,
                                               p == RHMC_MIXED_FP32, 0, rest, info, s);
    if (rc != RHMC_OK) return rc;
  } else if (info) {  // no solve: every field zero except the caller's array pointer
    double *user = info->per_shift_resid;
    std::memset(info, 0, sizeof(*info));
    info->per_shift_resid = user;
  }
  // Y^(s) = D_oe X^(s), then the outer-product sum; FP64-accurate in
  // double-float arithmetic on the FP32 units (native FP64 with
  // RHMC_TUNE_NATIVE_FP64_RESIDUALS)
  Arena fa(rest);
  void *Xf = fa.take<double2>((size_t)ns * len);  // double-float copy of X (float4 = double2 bytes)
  void *Yf = fa.take<double2>((size_t)ns * len);
  double *alpha_d = fa.take<double>(kMaxS);
  double *parts = fa.take<double>(kParts);
  if (G) {
    RHMC_CUDA_TRY(cudaMemcpyAsync(alpha_d, alpha, sizeof(double) * ns, cudaMemcpyHostToDevice, s));
    if (tune_get(TUNE_NATIVE_FP64_RESIDUALS)) {
      double2 *Y = (double2 *)Yf;
      RHMC_TRY(hop<double>(c->g, 1, c->l64[1], X, Y, nullptr, 0.0, n, ns, len, s));
      RHMC_TRY(force_links(c->g, X, Y, n, ns, len, alpha_d, c->bc_t, (double2 *)G, s));
    } else {
      float4 *Xd = (float4 *)Xf, *Yd = (float4 *)Yf;
      RHMC_TRY(df_split(X, Xd, (long)ns * len, s));
      for (int q = 0; q < ns; ++q)
        RHMC_TRY(hop_df(c->g, 1, c->ldf[1], Xd + (size_t)q * len, Yd + (size_t)q * len, nullptr, 0.0, n, s));
      RHMC_TRY(force_links_df(c->g, Xd, Yd, n, ns, len, alpha_d, c->bc_t, (double2 *)G, s));
    }
  }
  if (S_out) {
    RHMC_TRY(ensure_pinned(c, sizeof(double) * kParts));
    double S = 0.0;
    RHMC_TRY(redot((const double2 *)Phi, (const double2 *)Phi, len, parts, kParts, s));
    RHMC_CUDA_TRY(cudaMemcpyAsync(lane(c).h_pin, parts, sizeof(double) * kParts, cudaMemcpyDeviceToHost, s));
    RHMC_CUDA_TRY(cudaStreamSynchronize(s));
    for (int q = 0; q < kParts; ++q) S += alpha0 * lane(c).h_pin[q];
    for (int q = 0; q < ns; ++q) {
      RHMC_TRY(redot((const double2 *)Phi, X + (size_t)q * len, len, parts, kParts, s));
      RHMC_CUDA_TRY(cudaMemcpyAsync(lane(c).h_pin, parts, sizeof(double) * kParts, cudaMemcpyDeviceToHost, s));
      RHMC_CUDA_TRY(cudaStreamSynchronize(s));
      double t = 0.0;
      for (int k = 0; k < kParts; ++k) t += lane(c).h_pin[k];
      S += alpha[q] * t;
    }
    *S_out = S;
  }
  return RHMC_OK;
}

rhmc_status_t rhmc_force_lie(rhmc_ctx_t *c, const void *U, const void *G, void *F, double *norm2_out,
                             rhmc_stream_t sv) {
  if (!c || !U || !G || (!F && !norm2_out)) {
    set_error("rhmc_force_lie: null context, U or G, or neither F nor norm2_out requested");
    return RHMC_ERR_INVALID_ARG;
  }
  DeviceGuard dg(c->device);
  cudaStream_t s = (cudaStream_t)sv;
  if (!c->d_parts) RHMC_CUDA_TRY(cudaMalloc(&c->d_parts, sizeof(double) * kParts));
  RHMC_TRY(force_lie(c->g, (const double2 *)U, (const double2 *)G, (double2 *)F, c->d_parts, kParts, s));
  if (norm2_out) {
    RHMC_TRY(ensure_pinned(c, sizeof(double) * kParts));
    RHMC_CUDA_TRY(cudaMemcpyAsync(lane(c).h_pin, c->d_parts, sizeof(double) * kParts, cudaMemcpyDeviceToHost, s));
    RHMC_CUDA_TRY(cudaStreamSynchronize(s));
    double sum = 0.0;
    for (int q = 0; q < kParts; ++q) sum += lane(c).h_pin[q];
    *norm2_out = sum;
  }
  return RHMC_OK;
}

}  // extern "C"
