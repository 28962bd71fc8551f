// Internal launch wrappers (host functions enqueueing kernels on a stream).
#pragma once

#include "common.cuh"

namespace rhmc {

constexpr int kMaxN = RHMC_MAX_NRHS;
constexpr int kMaxS = RHMC_MAX_SHIFTS;

// Device-resident state of the SBCGrQ coefficient recursion (FP64).  Matrices
// are n x n row-major in the first n*n entries.  Slot k % kSlots holds
// iteration k's alpha, Gram1 (= alpha^-1), rho and delta: the shifted
// coefficient step of iteration k reads slots k and k-1 while the base step of
// iteration k+1 already writes slot k+1 on another stream.
constexpr int kSlots = 3;
struct SolverState {
  double2 alpha[kSlots][kMaxN * kMaxN];
  double2 G1[kSlots][kMaxN * kMaxN];
  double2 rho[kSlots][kMaxN * kMaxN];
  double2 delta[kSlots][kMaxN * kMaxN];
  double2 m2_s[kMaxS][kMaxN * kMaxN];   // beta^(s)_k rho_k^dagger of the last update of shift s
  double2 alpha_s[kMaxS][kMaxN * kMaxN];
  double sigma[kMaxS];        // shifts, ascending
  double d0[kMaxN];           // ||B e_j||
  double inv_d0[kMaxN];       // 1 / ||B e_j||
  double w1[kMaxS];           // weight of shift s's solution update (accumulating solves), 1 otherwise
  double res[kMaxS][kMaxN];   // recursive relative residual per shift and column (s = 0: base)
  int active[kMaxS];          // shift still being updated
  int upd[kMaxS];             // shift updated in the current iteration
  int last_k[kMaxS];          // last iteration that updated shift s (stored-basis mode)
  int kabs[kSlots];           // absolute iteration number of slot k % kSlots (graph replays reuse k's slot)
  int breakdown;              // nonzero: which coefficient step failed
  int device_timeout;         // a bounded device-side wait expired
};

// dslash.cu
rhmc_status_t stage_links(const Geom &g, const double2 *U, int bc_t, double2 *l64[2], float2 *l32[2],
                          cudaStream_t s);
// links12: optional 12-real copy of `links` (FP32 single-field hops use it), bc_t
// its boundary condition (signs of the rebuilt third rows)
template <typename T>
rhmc_status_t hop(const Geom &g, int par, const C<T> *links, const C<T> *in, C<T> *out, const C<T> *self, double a,
                  int n, int nbatch, long bstride, cudaStream_t s, const C<T> *links12 = nullptr, int bc_t = -1);
rhmc_status_t stage_links12(const Geom &g, int bc_t, float2 *const l32[2], float2 *l12[2], bool *ok, cudaStream_t s);

// double-float (FP64-accurate, FP32 units) operator pieces
rhmc_status_t stage_links_df(const Geom &g, const double2 *l64, float4 *ldf, cudaStream_t s);
rhmc_status_t df_split(const double2 *in, float4 *out, long len, cudaStream_t s);
rhmc_status_t df_merge(float4 *io, long len, cudaStream_t s);
// R = B - Y (Y in double-float, FP64 R), with the optional FP32 copy Rf and per-CTA
// column sums of |R|^2 (partial: nparts x n; launched with nparts CTAs)
rhmc_status_t resid_df(const double2 *B, const float4 *Y, double2 *R, float2 *Rf, long rows, int n,
                       double *partial, int nparts, cudaStream_t s);
rhmc_status_t hop_df(const Geom &g, int par, const float4 *links, const float4 *in, float4 *out, const float4 *self,
                     double a, int n, cudaStream_t s);

// blas.cu
constexpr int kGramCtas = 4 * 152;  // CTAs of the Gram kernel (its scratch holds kGramCtas * n * n partials)
template <typename T>
rhmc_status_t gram(const C<T> *A, const C<T> *B, long rows, int n, double2 *scratch, double2 *out, cudaStream_t s);
template <typename TA, typename TY>
rhmc_status_t block_axpy(const C<TA> *A, const C<TY> *Cin, const C<TA> *M, C<TY> *Y, long rows, int n,
                         cudaStream_t s);
// Shifts [s_begin, s_end): X^(s) += P^(s) M1^(s), P^(s) = Q + P^(s) M2^(s).
// compute_q: first form Q = W rho^-1 (and store it); otherwise read Q.
template <typename T, typename TX>
rhmc_status_t update_all(const C<T> *W, C<T> *Q, C<T> *P, C<TX> *X, const C<T> *coef, const int *upd, int s_begin,
                         int s_end, int compute_q, long rows, int n, long fstride, cudaStream_t s, int acc = 0);
rhmc_status_t flush(double2 *X64, float2 *X32, long len, cudaStream_t s);

// update_tc.cu: shifted updates on the tensor cores (mixed path, n = 16)
// Y = C + A M (FP32, C may be null) with column-owner lanes and cp.async-staged row tiles
rhmc_status_t axpy_cols(const float2 *A, const float2 *C, const float2 *M, float2 *Y, long rows, int n,
                        cudaStream_t s);
// Y = C + A M fused with out = Y^dagger Y (n x n FP64, scratch: kGramCtas * n * n partials)
rhmc_status_t axpy_gram_cols(const float2 *A, const float2 *C, const float2 *M, float2 *Y, long rows, int n,
                             double2 *scratch, double2 *out, cudaStream_t s);
// The base step after rho_k in one pass: Q = W rho^-1, X^(0) += P^(0) M1, P^(0) = Q + P^(0) M2
// (coef: rho^-1, M1, M2), and Q into basis block *kdev when basis is given (capacity cap)
rhmc_status_t base_step(const float2 *W, float2 *Q, float2 *P, float2 *X, const float2 *coef, float2 *basis, int cap,
                        const int *kdev, long rows, int n, cudaStream_t s);
// FP32 shifted updates (Algorithm 1) with column-owner lanes and cp.async-staged row tiles
rhmc_status_t update_shifts_cols(const float2 *Q, float2 *P, float2 *X, const float2 *coef, const int *upd,
                                 int s_begin, int s_end, long rows, int n, long fstride, cudaStream_t s);
rhmc_status_t update_shifts_tc(const float2 *Q, float2 *P, float2 *X, const float2 *coef, const int *upd,
                               int s_begin, int s_end, long rows, long fstride, float *btiles, int *err,
                               cudaStream_t s);
template <typename TI, typename TO>
rhmc_status_t convert(const C<TI> *in, C<TO> *out, long len, cudaStream_t s);
rhmc_status_t sub(const double2 *a, const double2 *b, double2 *out, long len, cudaStream_t s);
rhmc_status_t add_inplace(double2 *a, const double2 *b, long len, cudaStream_t s);
template <typename T>
rhmc_status_t colnorm2(const C<T> *A, long rows, int n, double *partial, int nparts, cudaStream_t s);
rhmc_status_t redot(const double2 *A, const double2 *B, long len, double *partial, int nparts, cudaStream_t s);

// small.cu
template <typename T>
rhmc_status_t nxn_qr_init(const double2 *partial, int nparts, int n, int nshift, SolverState *st, C<T> *rinv,
                          cudaStream_t s);
template <typename T>
rhmc_status_t nxn_alpha(const double2 *partial, int nparts, int n, SolverState *st, int k, C<T> *mw, cudaStream_t s);
// small_df.cu: double-float forms of nxn_alpha / nxn_rho for the mixed solve (summed Gram input)
rhmc_status_t nxn_alpha_dd(const double2 *gram, int n, SolverState *st, int k, float2 *mw, cudaStream_t s);
rhmc_status_t nxn_rho_dd(const double2 *gram, int n, SolverState *st, int k, float2 *coef, cudaStream_t s);
rhmc_status_t nxn_shifts_dd(int n, int nshift, SolverState *st, int k, float2 *coef, double tol_shift, int freeze,
                            double2 *hist, int cap, cudaStream_t s);
template <typename T>
rhmc_status_t nxn_rho(const double2 *partial, int nparts, int n, SolverState *st, int k, C<T> *coef, cudaStream_t s);
// hist (nullable, stored-basis mode): [cap][nshift][2][n*n] FP64, alpha^(s)_k and
// beta^(s)_k rho_k^dagger recorded at iteration k < cap
template <typename T>
rhmc_status_t nxn_shifts(int n, int nshift, SolverState *st, int k, C<T> *coef, double tol_shift, int freeze,
                         double2 *hist, int cap, cudaStream_t s);
// Stored-basis mode (basis.cu).  Buffers of the assembly: the block basis
// (rows x cap*n FP32 complex, row-major), the recorded per-iteration shift
// coefficients hist [cap][nshift][2][n*n] (alpha^(s)_k, beta^(s)_k rho_k^dagger),
// FP64 expansion coefficients cf [nshift-1][cap+1][n*n], the packed FP16 operand
// tiles of the tensor-core kernel (basis_pack_bytes), per-shift scales and per-tile
// K extents.
struct BasisBufs {
  float2 *basis = nullptr;
  double2 *hist = nullptr;
  double2 *cf = nullptr;
  unsigned char *bpack = nullptr;
  double *bscale = nullptr;  // [nshift]
  int *tile_nkt = nullptr;   // [nshift]
  int cap = 0;
};
size_t basis_pack_bytes(int n, int nshift, int cap);
// want_p = 0: X^(s) = sum_{i < last_s} Q_i C_i for s = 1 .. nshift-1 (FP64, C_i = alpha_{i+1}
// + M2_{i+1} C_{i+1}; X^(s), s >= 1, is overwritten: it is zero before the one assembly of a
// solve); want_p = 1: P^(s) = sum_{i <= K} Q_i D_i (FP32, D_K = 1, D_i = M2_{i+1} D_{i+1}),
// active shifts only.  chunk_blocks > 0 (X only): FP32 partial sums over about that many
// blocks, added in FP64.  simt: CUDA-core kernel instead of tcgen05.  acc_kt: K tiles (of 64
// reals) per tensor-memory accumulation chunk (0: built-in).  err: device flag set when a
// bounded wait of the tensor-core kernel gave up.
rhmc_status_t basis_assemble(const BasisBufs &bb, int n, int nshift, const SolverState *st, long rows, int K,
                             int want_p, double2 *X, float2 *P, long fstride, int chunk_blocks, int simt, int acc_kt,
                             int *err, cudaStream_t s);
// Q (rows x n) into column block k of the basis (rows x cap*n, row-major)
rhmc_status_t basis_store(const float2 *Q, float2 *basis, long rows, int n, int cap, int k, cudaStream_t s);
// the same with the block index read from *kdev (an iteration counter in device memory)
rhmc_status_t basis_store_dev(const float2 *Q, float2 *basis, long rows, int n, int cap, const int *kdev,
                              cudaStream_t s);
template <typename T>
rhmc_status_t nxn_reliable(const double2 *partial, int nparts, int n, SolverState *st, int k, C<T> *rinv,
                           cudaStream_t s);

// force.cu
rhmc_status_t rational_combine(const double2 *Phi, double alpha0, const double *alpha_host, const double2 *X, int ns,
                               long len, double2 *Y, cudaStream_t s);
// the same from double-float fields (float4 per complex)
rhmc_status_t force_links_df(const Geom &g, const float4 *X, const float4 *Y, int n, int nshift, long fstride,
                             const double *alpha_dev, int bc_t, double2 *G, cudaStream_t s);
rhmc_status_t force_links(const Geom &g, const double2 *X, const double2 *Y, int n, int nshift, long fstride,
                          const double *alpha_dev, int bc_t, double2 *G, cudaStream_t s);
// F = TA(U G^dagger) per link (F may be null or alias G); partial[nparts]: per-CTA sums of |F|_F^2 / 4
rhmc_status_t force_lie(const Geom &g, const double2 *U, const double2 *G, double2 *F, double *partial, int nparts,
                        cudaStream_t s);

// api.cu: the calling thread uses ctx's launch settings (rhmc_ctx_tune_set) while
// an object of this type lives, as every entry point of api.cu does.
struct CtxTuneScope {
  const int *prev;
  explicit CtxTuneScope(const rhmc_ctx_t *c);
  ~CtxTuneScope();
};

// api.cu: read-only view of a context (device, geometry, mass, staged FP64
// links of the two output parities); NO_GAUGE before rhmc_set_gauge.
rhmc_status_t ctx_geometry(const rhmc_ctx_t *ctx, int *device, Geom *g, double *mass, const double2 **l64_even,
                           const double2 **l64_odd);

// api.cu: device and geometry of a context (no gauge field needed), and its
// scratch array of per-CTA partial sums (allocated on first use)
rhmc_status_t ctx_lattice(const rhmc_ctx_t *ctx, int *device, Geom *g);
rhmc_status_t ctx_partials(rhmc_ctx_t *ctx, double **parts, int *nparts);
// api.cu: the context's molecular-dynamics buffer, at least `bytes` long (kept
// across calls, reallocated when too small)
rhmc_status_t ctx_md_buffer(rhmc_ctx_t *ctx, size_t bytes, void **buf);

// scg.cu (per-vector FP64 multishift CG baseline)
struct ScgState;

}  // namespace rhmc
