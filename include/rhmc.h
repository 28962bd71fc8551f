/*
 * rhmc.h -- C ABI of the GB300 block multishift RHMC library (librhmc.so).
 *
 * The library implements the hot path of de Forcrand & Keegan, "Rational
 * Hybrid Monte Carlo with Block Solvers and Multiple Pseudofermions"
 * (arXiv:1808.01829):
 *   - the even-odd preconditioned unimproved staggered operator
 *     A = M^dagger M on even sites (Sec. IV), applied to a block of
 *     right-hand sides that shares each gauge-link load ("pencil", Sec. III
 *     and the conclusions);
 *   - the block multishift solver SBCGrQ (Algorithm 1) for
 *     (A + sigma_s) X^(s) = B, all right-hand sides and all shifts at once;
 *   - the pseudofermion action and force of Eqs. (RA) and (force).
 *
 * Conventions (all calls):
 *   Lattice    dims = {Lx, Ly, Lz, Lt}, all even and >= 2; site lex index
 *              x + Lx*(y + Ly*(z + Lz*t)).  Even sites have x+y+z+t even;
 *              a site's rank among its parity is lex/2.
 *   Operator   M = 2m + D,
 *              (D psi)(x) = sum_mu eta_mu(x) [b_mu(x) U_mu(x) psi(x+mu)
 *                                   - b_mu(x-mu) U_mu(x-mu)^dagger psi(x-mu)],
 *              eta_mu(x) = (-1)^(x_0+...+x_{mu-1}), b = -1 on t-links that
 *              wrap Lt-1 -> 0 when bc_t = -1 (antiperiodic), else +1.
 *              A = 4 m^2 - D_eo D_oe; its spectrum lies in [4m^2, 4m^2+64].
 *   Gauge U    device, complex128 (interleaved re,im doubles),
 *              [Lt][Lz][Ly][Lx][mu=0..3][3][3].
 *   Fields     device, complex128 [V/2][3][n]: one parity, the n right-hand
 *              sides fastest.  Shifted solutions are [n_shifts][V/2][3][n].
 *   Force G    device, complex128 [V][4][3][3], G = dS/dRe U + i dS/dIm U.
 *   Streams    rhmc_stream_t is a cudaStream_t (NULL = legacy default).
 *              Work is enqueued on that stream; calls that return solver
 *              information (info, S_out) synchronise the stream first.
 *   Ownership  the caller owns every buffer it passes.  The context owns its
 *              staged copy of the gauge field and an internal scratch pool
 *              (used when a call's `workspace` is NULL).  No call retains a
 *              caller pointer after it returns.
 *   Errors     every call returns an rhmc_status_t; no exception crosses the
 *              ABI.  rhmc_last_error() gives a thread-local message for the
 *              last failing call of the thread.
 *   Threads    a context may be used by one host thread at a time.
 */
#ifndef RHMC_H
#define RHMC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rhmc_ctx rhmc_ctx_t;
typedef void *rhmc_stream_t; /* cudaStream_t */

typedef enum {
  RHMC_OK = 0,
  RHMC_ERR_INVALID_ARG = 1,    /* null pointer, odd extent, n out of range, bad shifts/tol */
  RHMC_ERR_NOT_CONVERGED = 2,  /* max_iter reached; results and info are still written */
  RHMC_ERR_BREAKDOWN = 3,      /* non-positive-definite Gram matrix / non-finite coefficients */
  RHMC_ERR_CUDA = 4,           /* a CUDA runtime call failed */
  RHMC_ERR_DEVICE_TIMEOUT = 5, /* a bounded device-side wait expired */
  RHMC_ERR_NO_GAUGE = 6        /* rhmc_set_gauge has not been called */
} rhmc_status_t;

typedef struct {
  int dims[4];  /* Lx, Ly, Lz, Lt: even, >= 2 */
  double mass;  /* m in M = 2m + D */
  int bc_t;     /* -1 antiperiodic in t (default), +1 periodic */
} rhmc_lattice_t;

typedef enum {
  RHMC_FP64 = 0,       /* everything in FP64 */
  RHMC_MIXED_FP32 = 1, /* FP32 operator and block updates inside an FP64-accurate
                          reliable-update / defect-correction loop; FP64 n x n
                          coefficient algebra, FP64 force.  The residuals of the
                          loop use the double-float operator (RHMC_DF64) */
  RHMC_DF64 = 2        /* operator only (apply / hop): FP64-accurate double-float
                          arithmetic (pairs of FP32, about 2^-44 relative) on the
                          FP32 units, which on this GPU are 74x faster than FP64 */
} rhmc_precision_t;

/* Largest number of right-hand sides per block (n_pf). */
#define RHMC_MAX_NRHS 16
/* Largest number of shifts per solve. */
#define RHMC_MAX_SHIFTS 64

typedef struct {
  int iters;                 /* SBCGrQ iterations of the main solve */
  int dirac_calls;           /* applications of A to an n-wide block, all phases */
  int reliable_updates;      /* FP64 residual replacements (mixed precision) */
  int refinements;           /* per-shift defect-correction solves */
  int refine_iters;          /* iterations spent in them */
  double true_rel_resid_max; /* max_{s,j} ||B e_j - (A+sigma_s) X^(s) e_j|| / ||B e_j||, FP64 */
  double phase1_rel_resid_max; /* the same before any defect correction */
  double *per_shift_resid;   /* optional caller array [n_shifts*n_rhs] (shift-major), or NULL */
  double phase1_ms;          /* device time of the multishift solve (events on the call's stream) */
  double refine_ms;          /* device time of the true-residual checks and defect corrections */
} rhmc_info_t;

/* Create a context on CUDA device `device` for lattice `lat`.
 * INVALID_ARG if an extent is odd or < 2, or lat/ctx is NULL. */
rhmc_status_t rhmc_create(rhmc_ctx_t **ctx, const rhmc_lattice_t *lat, int device);

/* Release the context and everything it allocated. NULL is accepted. */
rhmc_status_t rhmc_destroy(rhmc_ctx_t *ctx);

/* Stage the gauge field (Sec. IV's links U_mu(x)) into the context's internal
 * FP64 and FP32 link arrays, phases and boundary signs folded in.  U is read
 * on stream s and not retained; the call returns after staging completes. */
rhmc_status_t rhmc_set_gauge(rhmc_ctx_t *ctx, const void *U_dev, rhmc_stream_t s);

/* Bytes of device workspace that rhmc_block_multishift_cg / rhmc_force need
 * for this problem size, under the context's launch settings; 0 on invalid
 * arguments.  In mixed precision with several shifts this includes the stored
 * block basis (RHMC_TUNE_BASIS_ITERS: built in, up to 384 blocks of
 * V/2 * 3 * n_rhs * 8 bytes within a quarter of the device memory, e.g.
 * 24.5 GB at 24^4, n_rhs = 16); RHMC_TUNE_BASIS_ITERS = 1 sizes without it. */
size_t rhmc_workspace_bytes(const rhmc_ctx_t *ctx, int n_rhs, int n_shifts, rhmc_precision_t p);

/* Y = (A + sigma) X for an n_rhs-wide block (multi-RHS operator, each link
 * loaded once for all right-hand sides; Sec. IV, Fig. 8 top).  X, Y complex128
 * [V/2][3][n_rhs], may not alias.  p = RHMC_MIXED_FP32 evaluates the FP32
 * kernel (input rounded to FP32, result widened).  1 <= n_rhs <= RHMC_MAX_NRHS. */
rhmc_status_t rhmc_apply_mdagm_mrhs(rhmc_ctx_t *ctx, const void *X_dev, void *Y_dev, int n_rhs, double sigma,
                                    rhmc_precision_t p, rhmc_stream_t s);

/* The same operator application as rhmc_apply_mdagm_mrhs with p = RHMC_FP64,
 * for callers that must not allocate device memory (inside a stream capture,
 * under a fixed memory budget, or under a framework that owns all
 * allocation).  The paper has no counterpart; this is a deployment variant.
 * It allocates nothing: the odd-parity intermediate lives in a file-scope
 * device array of fixed size (32 MiB, i.e. V/2 * 3 * n_rhs * 16 bytes at most,
 * e.g. a 16^4 lattice with 16 right-hand sides), which every GPU that loads
 * the library holds until the process exits.  Larger problems are rejected
 * with INVALID_ARG.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the array: calls that overlap on the GPU (other
 * streams, other threads) race on it and must be serialised by the caller.
 * The looked-up address belongs to the device's primary context: after a
 * cudaDeviceReset of that device, do not call this entry point there again.
 * The context's launch settings (rhmc_ctx_tune_set) apply as in
 * rhmc_apply_mdagm_mrhs.  Requires rhmc_set_gauge (NO_GAUGE otherwise). */
rhmc_status_t rhmc_apply_mdagm_mrhs_noalloc(rhmc_ctx_t *ctx, const void *X_dev, void *Y_dev, int n_rhs, double sigma,
                                            rhmc_stream_t s);

/* One staggered hop Y = D X onto parity out_parity (0: D_eo, input odd;
 * 1: D_oe, input even).  Same layouts and precision rule as above. */
rhmc_status_t rhmc_hop(rhmc_ctx_t *ctx, const void *X_dev, void *Y_dev, int n_rhs, int out_parity,
                       rhmc_precision_t p, rhmc_stream_t s);

/* SBCGrQ (Algorithm 1): solve (A + sigma_s) X^(s) = B for every shift.
 *   B         complex128 [V/2][3][n_rhs], columns linearly independent
 *   shifts    host array [n_shifts], each >= 0; solved in ascending order,
 *             the smallest drives the Krylov space (sigma_0)
 *   X         complex128 [n_shifts][V/2][3][n_rhs], in the caller's shift order
 *   tol       relative residual target per column and shift (> 0)
 *   max_iter  iteration cap of the main solve (<= 0: 10 sqrt(64/4m^2) ln(1/tol))
 *   workspace device buffer of rhmc_workspace_bytes() bytes, or NULL to use
 *             the context's pool
 *   info      optional; filled after a stream synchronise
 * Returns OK once every (shift, column) true FP64 residual is <= tol,
 * NOT_CONVERGED otherwise (X still written), BREAKDOWN on a singular block. */
rhmc_status_t rhmc_block_multishift_cg(rhmc_ctx_t *ctx, const void *B_dev, int n_rhs, int n_shifts,
                                       const double *shifts, void *X_dev, double tol, int max_iter,
                                       rhmc_precision_t p, void *workspace, rhmc_info_t *info, rhmc_stream_t s);

/* One member of a batched solve: its own context (lattice, gauge field),
 * right-hand sides, shifts, output and (optional) workspace, as in
 * rhmc_block_multishift_cg.  status is written by the call. */
typedef struct {
  rhmc_ctx_t *ctx;
  const void *B;
  int n_rhs;
  int n_shifts;
  const double *shifts;
  void *X;
  void *workspace;    /* NULL: the context's pool */
  rhmc_info_t *info;  /* optional */
  rhmc_status_t status;
} rhmc_batch_item_t;

/* Several independent SBCGrQ solves at once (ensembles of different lattice
 * sizes, widths and shifts): every item runs on its context's own stream from
 * a worker thread, with its iterations in captured CUDA graphs, so the small
 * lattices' kernels overlap the large ones' on the GPU.  Work starts after what
 * is already queued on stream s, and s waits for all of it.  Each context may
 * appear once.  Returns the first failing item's status (all items run). */
rhmc_status_t rhmc_block_multishift_cg_batch(rhmc_batch_item_t *items, int count, double tol, int max_iter,
                                             rhmc_precision_t p, rhmc_stream_t s);

/* Baseline: plain per-vector FP64 multishift CG (SCG, Sec. III), one
 * right-hand side at a time with a width-1 operator.  Same arguments and
 * output as rhmc_block_multishift_cg with p = RHMC_FP64. */
rhmc_status_t rhmc_multishift_cg_pervector(rhmc_ctx_t *ctx, const void *B_dev, int n_rhs, int n_shifts,
                                           const double *shifts, void *X_dev, double tol, int max_iter,
                                           void *workspace, rhmc_info_t *info, rhmc_stream_t s);

/* Pseudofermion action and force for n_pf pseudofermions Phi (Eqs. (RA),
 * (force)):  S = sum_i [alpha0 |phi_i|^2 + sum_s alpha_s phi_i^dagger X^(s) e_i],
 *   G_mu(x) = dS/dRe U_mu(x) + i dS/dIm U_mu(x)
 *           = 2 eps(x) eta_mu(x) b_mu(x) sum_{s,i} alpha_s W_si(x) W_si(x+mu)^dagger,
 * W = X^(s) on even sites, D_oe X^(s) on odd sites, eps = +1 even / -1 odd.
 *   Phi       complex128 [V/2][3][n_pf]
 *   alpha, beta  host [n_shifts]: residues and poles of Eq. (RA), beta > 0
 *   X_in      optional complex128 [n_shifts][V/2][3][n_pf] solutions of
 *             (A + beta_s) X = Phi; NULL = solve them (block solver, tol, p)
 *   G         complex128 [V][4][3][3] output, or NULL for the action only
 *   S_out     optional host double, the action (G and S_out may not both be NULL)
 * The force is FP64-accurate in both precision modes: double-float arithmetic
 * (pairs of FP32, TwoProduct/TwoSum) on the FP32 units, or native FP64 with
 * RHMC_TUNE_NATIVE_FP64_RESIDUALS. */
rhmc_status_t rhmc_force(rhmc_ctx_t *ctx, const void *Phi_dev, int n_pf, double alpha0, const double *alpha,
                         const double *beta, int n_shifts, double tol, int max_iter, rhmc_precision_t p,
                         const void *X_in_dev, void *G_dev, double *S_out, void *workspace, rhmc_info_t *info,
                         rhmc_stream_t s);

/* Lie-algebra force and its norm (Sec. II, Eqs. (force), (force_norm)).
 * Per link, F_mu(x) = TA(U_mu(x) G_mu(x)^dagger) with
 * TA(M) = (M - M^dagger)/2 - tr(M - M^dagger)/6 (traceless anti-Hermitian);
 * with generators T^a = i lambda^a / 2 (Gell-Mann lambda^a) the derivative of
 * S along U -> exp(w T^a) U is F^a = Re tr(G^dagger T^a U) = tr(F T^a), i.e.
 * F = -2 sum_a F^a T^a.
 *   U         complex128 [V][4][3][3], the links given to rhmc_set_gauge
 *   G         complex128 [V][4][3][3], rhmc_force's output
 *   F         complex128 [V][4][3][3] output, or NULL; may alias G
 *   norm2_out optional host double: sum over links of sum_a (F^a)^2 / 2
 *             (= |F|_F^2 / 4), summed in a fixed order (deterministic)
 * FP64.  With norm2_out the call synchronises stream s; otherwise it is
 * asynchronous.  INVALID_ARG for null U or G, or when neither F nor norm2_out
 * is given. */
rhmc_status_t rhmc_force_lie(rhmc_ctx_t *ctx, const void *U_dev, const void *G_dev, void *F_dev, double *norm2_out,
                             rhmc_stream_t s);

/* R(A) Phi of Eq. (RA) by the block multishift solve, without storing the
 * shifted solutions (pseudofermion heatbath and action evaluation, where only
 * the rational sum is needed):
 *   Y = alpha0 Phi + sum_s alpha_s (A + beta_s)^-1 Phi.
 * FP64 throughout.  The solve keeps X^(0) (smallest shift) and one field for
 * sum_{s>=1} alpha_s X^(s), added in the fused shifted update (the per-shift
 * X^(s) are never written), so it needs about n_shifts - 2 fewer fields than
 * rhmc_block_multishift_cg and moves less data per iteration.
 *   Phi, Y   complex128 [V/2][3][n_pf] on the device (no aliasing)
 *   alpha, beta  host [n_shifts], beta >= 0 (any sign of alpha: x^(+r) works)
 *   workspace  rhmc_rational_solve_bytes(ctx, n_pf, n_shifts) bytes, or NULL (pool)
 *   info     optional: iters; true_rel_resid_max = FP64 true residual of the
 *            smallest-shift system; phase1_rel_resid_max = largest recursive
 *            residual over all (shift, column); per_shift_resid = those
 *            recursive residuals (caller's shift order)
 * Returns OK once every recursive residual is <= tol, NOT_CONVERGED otherwise
 * (Y still written).  In FP64 the recursive residuals track the true ones
 * closely; the smallest-shift true residual is reported as a check. */
rhmc_status_t rhmc_rational_solve(rhmc_ctx_t *ctx, const void *Phi_dev, int n_pf, double alpha0, const double *alpha,
                                  const double *beta, int n_shifts, double tol, int max_iter, void *Y_dev,
                                  void *workspace, rhmc_info_t *info, rhmc_stream_t s);
size_t rhmc_rational_solve_bytes(const rhmc_ctx_t *ctx, int n_pf, int n_shifts);

/* R(A) Phi of Eq. (RA) from given shifted solutions:
 *   Y = alpha0 Phi + sum_s alpha_s X^(s),   X^(s) = (A + beta_s)^-1 Phi,
 * Phi, Y complex128 [V/2][3][n_pf]; X complex128 [n_shifts][V/2][3][n_pf];
 * alpha host [n_shifts].  Y may not alias X.  (The gradient of the action
 * with respect to Phi is 2 R(A) Phi.)  Asynchronous on stream s. */
rhmc_status_t rhmc_rational_apply(rhmc_ctx_t *ctx, const void *Phi_dev, int n_pf, double alpha0, const double *alpha,
                                  int n_shifts, const void *X_dev, void *Y_dev, rhmc_stream_t s);

/* ------------------------------------------------------------------------
 * The RHMC trajectory around the pseudofermion force (Sec. II set-up; Sec. IV
 * run parameters: Wilson gauge action, two-level OMF2 integrator, heatbath and
 * accept/reject solves at 1e-14).  FP64 throughout.  Fields:
 *   U   complex128 [V][4][3][3] links, lexicographic sites x + Lx (y + Ly (z + Lz t)),
 *       periodic in every direction (the antiperiodic temporal boundary
 *       belongs to the fermion operator only);
 *   P   complex128 [V][4][3][3] momenta, traceless anti-Hermitian,
 *       P = sum_a p^a T^a with T^a = i lambda^a / 2 (Gell-Mann lambda^a);
 *   G   complex128 [V][4][3][3] action derivative dS/dRe U + i dS/dIm U
 *       (rhmc_force's output for the pseudofermion action).
 * The molecular dynamics is dU/dtau = P U, dP/dtau = TA(U G^dagger) / 2 with
 * TA(M) = (M - M^dagger)/2 - tr(M - M^dagger)/6, and conserves
 * H = K + S_g + S_f, K = -sum tr(P^2) = sum_a (p^a)^2 / 2.
 * These calls do not need rhmc_set_gauge (the context gives the lattice);
 * those that return a host scalar synchronise stream s, the others are
 * asynchronous.  INVALID_ARG for null pointers. */

/* Wilson gauge action S_g = beta sum_{x, mu<nu} (1 - Re tr Pi_{mu nu}(x) / 3),
 * Pi_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger (Sec. IV).
 * Summed per CTA, then on the host in a fixed order (deterministic). */
rhmc_status_t rhmc_gauge_action(rhmc_ctx_t *ctx, const void *U_dev, double beta, double *S_out, rhmc_stream_t s);

/* Kinetic energy K = -sum_{x,mu} Re tr(P_mu(x)^2), deterministic like the action. */
rhmc_status_t rhmc_kinetic_energy(rhmc_ctx_t *ctx, const void *P_dev, double *K_out, rhmc_stream_t s);

/* Momentum heatbath from caller-drawn normals: P_mu(x) = sum_a p[x][mu][a] T^a,
 * p float64 [V][4][8], p^a ~ N(0, 1) for the distribution exp(-K). */
rhmc_status_t rhmc_momenta_from_normals(rhmc_ctx_t *ctx, const double *p_dev, void *P_dev, rhmc_stream_t s);

/* Gauge-force kick P += eps TA(U G_g^dagger) / 2 with G_g = -(beta / 3) V^dagger,
 * V_mu(x) the sum of the six staples around U_mu(x):
 *   V_mu(x) = sum_{nu != mu} [U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger
 *                             + U_nu(x+mu-nu)^dagger U_mu(x-nu)^dagger U_nu(x-nu)]. */
rhmc_status_t rhmc_gauge_momentum(rhmc_ctx_t *ctx, const void *U_dev, void *P_dev, double beta, double eps,
                                  rhmc_stream_t s);

/* Kick by a given derivative: P += eps TA(U G^dagger) / 2 (G from rhmc_force). */
rhmc_status_t rhmc_momentum_update(rhmc_ctx_t *ctx, const void *U_dev, const void *G_dev, void *P_dev, double eps,
                                   rhmc_stream_t s);

/* Drift U <- exp(eps P) U per link.  The exponential is a degree-16 Taylor
 * polynomial of eps P / 2^k, k the smallest with |eps P|_F / 2^k <= 1/2, squared
 * k times (truncation below 1e-19 relative). */
rhmc_status_t rhmc_link_update(rhmc_ctx_t *ctx, void *U_dev, const void *P_dev, double eps, rhmc_stream_t s);

/* Rational function of Eq. (RA): R(x) = alpha0 + sum_s alpha_s / (x + beta_s). */
typedef struct {
  int n_shifts;        /* 1 .. RHMC_MAX_SHIFTS */
  double alpha0;
  const double *alpha; /* host [n_shifts] */
  const double *beta;  /* host [n_shifts], > 0 */
} rhmc_rational_t;

/* Molecular-dynamics parameters of the two-level OMF2 integrator (Sec. IV). */
typedef struct {
  double beta;      /* Wilson gauge coupling */
  double tau;       /* trajectory length */
  int n_steps;      /* outer steps, step size dtau = tau / n_steps (pseudofermion force) */
  int n_gauge;      /* inner steps per outer drift of length dtau / 2 (gauge force) */
  double lambda;    /* OMF2 parameter (1/6 in the paper's acceptance study) */
  double tol_md;    /* stopping criterion of the force solves (1e-7 in the paper) */
  int max_iter;     /* of the force solves; 0 = built-in */
  rhmc_precision_t precision_md; /* RHMC_FP64 or RHMC_MIXED_FP32 force solves */
} rhmc_md_params_t;

typedef struct {
  int force_evals;        /* pseudofermion force evaluations (block multishift solves) */
  int gauge_force_evals;  /* gauge-force kicks */
  long long solver_iters; /* SBCGrQ iterations summed over the force solves (incl. corrections) */
  long long dirac_calls;  /* block operator applications summed over the force solves */
  double max_rel_resid;   /* largest true relative residual of any force solve */
} rhmc_md_info_t;

/* Molecular dynamics over one trajectory, (U, P) updated in place.  Per outer
 * step of length e = tau / n_steps (OMF2, Omelyan's second-order scheme):
 *   P += lambda e F_f; D(e/2); P += (1 - 2 lambda) e F_f; D(e/2); P += lambda e F_f,
 * where F_f = TA(U G_f^dagger)/2 is the pseudofermion force of
 * S_f = sum_i phi_i^dagger R_md(A) phi_i (rhmc_force with `md`) and each drift
 * D(h) is the same scheme with the gauge force and the link update in n_gauge
 * steps of length h / n_gauge.  Consecutive kicks at the same links are
 * merged (one force evaluation for the lambda e kicks that end one step and
 * start the next), so a trajectory takes 2 n_steps + 1 pseudofermion forces.
 *   Phi   complex128 [V/2][3][n_pf] pseudofermions, or NULL (n_pf = 0: gauge only)
 * The context's staged links are replaced (rhmc_set_gauge) at every force
 * evaluation and hold the final U on return.  Uses the context's buffers (one
 * G field) and pool.  Status of the first failing solve (NOT_CONVERGED
 * included) is returned at once, with (U, P) part-way. */
rhmc_status_t rhmc_md_evolve(rhmc_ctx_t *ctx, void *U_dev, void *P_dev, const void *Phi_dev, int n_pf,
                             const rhmc_rational_t *md, const rhmc_md_params_t *p, rhmc_md_info_t *info,
                             rhmc_stream_t s);

typedef struct {
  double H_old, H_new, dH;  /* H = K + S_g + S_f at the start and end */
  double K[2], S_g[2], S_f[2];
  int accepted;             /* 1: U holds the new links */
  rhmc_md_info_t md;
} rhmc_hmc_info_t;

/* One RHMC trajectory with accept/reject (Sec. II set-up, Sec. IV):
 *   1. momenta P = sum_a p^a T^a from the caller's normals p (float64 [V][4][8]);
 *   2. pseudofermion heatbath Phi = R_hb(A) eta with R_hb ~ x^(+n_f/(8 n_pf)),
 *      eta complex128 [V/2][3][n_pf] drawn by the caller with density
 *      exp(-|eta|^2) (real and imaginary parts N(0, 1/2)); FP64 solve at tol_action;
 *   3. H_old = K + S_g + S_f with S_f = sum_i phi_i^dagger R_act(A) phi_i
 *      (R_act ~ x^(-n_f/(4 n_pf)), FP64 block solve at tol_action);
 *   4. rhmc_md_evolve on a copy of U with the MD rational `md`;
 *   5. H_new as in 3; accept when u_accept < exp(-(H_new - H_old)), with
 *      u_accept in [0, 1) drawn by the caller.
 * On accept U is overwritten with the new links; the context's staged links
 * are those of U on return.  Phi_out optional complex128 [V/2][3][n_pf] (the
 * heatbath field).  n_pf = 0 (eta NULL) is pure-gauge HMC. */
rhmc_status_t rhmc_hmc_trajectory(rhmc_ctx_t *ctx, void *U_dev, const double *p_dev, const void *eta_dev, int n_pf,
                                  const rhmc_rational_t *heatbath, const rhmc_rational_t *md,
                                  const rhmc_rational_t *action, const rhmc_md_params_t *p, double tol_action,
                                  double u_accept, void *Phi_out_dev, rhmc_hmc_info_t *info, rhmc_stream_t s);

/* Thread-local message describing the last failing call ("" if none). */
const char *rhmc_last_error(void);

/* Running count of kernels this library has launched in the process (all
 * contexts and threads); differences around a call count its launches. */
long long rhmc_kernel_launches(void);

/* Per-kernel timing for measurement runs.  rhmc_profile_enable(1) clears the
 * record and starts recording, for every kernel launch of the library, a pair
 * of CUDA events on the launching stream plus the launch's algorithmic bytes
 * (each input read once, each output written once); (0) stops recording.
 * While enabled the fused update kernel reads its shift flags back to the host
 * first (a synchronisation), so use it outside timed regions.
 * rhmc_profile_read(category, ...) synchronises on the recorded events and
 * returns the number of launches, their summed duration (ms) and summed bytes
 * of one category (RHMC_PROF_*). */
enum {
  RHMC_PROF_HOP_FP32 = 0, RHMC_PROF_HOP_FP64, RHMC_PROF_GRAM_FP32, RHMC_PROF_GRAM_FP64, RHMC_PROF_BLOCK_AXPY,
  RHMC_PROF_UPDATE_FP32, RHMC_PROF_UPDATE_FP64, RHMC_PROF_NXN, RHMC_PROF_FORCE, RHMC_PROF_OTHER,
  RHMC_PROF_HOP_DF, RHMC_PROF_NXN_SHIFTS, RHMC_PROF_UPDATE_TC, RHMC_PROF_UPDATE_SHIFTS32,
  RHMC_PROF_BASIS_TC, RHMC_PROF_NCAT
};
rhmc_status_t rhmc_profile_enable(int on);

/* Launch-parameter tuning, process-wide (used by the autotuner).  Keys:
 *   RHMC_TUNE_HOP_RHS_PER_THREAD  right-hand sides per thread in the hop
 *                                 kernel: 1, 2 or 4 (must divide n_rhs)
 *   RHMC_TUNE_UPDATE_THREADS      threads per CTA of the fused shift update: a
 *                                 multiple of 32 up to 256 (other values: 256)
 *   RHMC_TUNE_FLUSH_EVERY         mixed precision: add the FP32 solution increments
 *                                 into the FP64 solutions every k iterations as
 *                                 well as at reliable updates (0: only there)
 *   RHMC_TUNE_RELIABLE_DELTA_MILLI  mixed precision: reliable update when the
 *                                 base residual fell by value/1000 (0: 0.1)
 *   RHMC_TUNE_CHECK_EVERY         iterations between host convergence checks (0: 6)
 *   RHMC_TUNE_NATIVE_FP64_RESIDUALS  mixed precision: compute the reliable-update and
 *                                 true residuals with native FP64 instead of RHMC_DF64
 *   RHMC_TUNE_UPDATE_TENSOR       mixed precision, shifted updates: on the tensor cores
 *                                 (tcgen05, three-piece TF32 split, n_rhs = 16 only) = 1; CUDA-core kernel with
 *                                 lane-owned row slices = 2; CUDA-core kernel with column-owner
 *                                 lanes and cp.async-staged row tiles = 0 (built-in: packed
 *                                 FP32x2 FMAs) or 3..11 (tile shape and FMA variants, see the
 *                                 autotuner)
 *   RHMC_TUNE_GRAPHS              solver iterations in captured CUDA graphs (0, 1: built-in)
 *                                 or as eager launches (2)
 *   RHMC_TUNE_HOP_STAGED          FP32 hop kernel: all 8 neighbours' loads issued at once,
 *                                 links by cp.async (0: built-in; 3: one right-hand side per
 *                                 thread; 4: two, even n); tiles staged in shared memory by
 *                                 cp.async, even n (1); register staged with one direction of
 *                                 prefetch (2)
 *   RHMC_TUNE_LINKS12             1: the FP32 hop reads the first two rows of each link and
 *                                 rebuilds the third (only when rhmc_set_gauge found every link
 *                                 in SU(3) to FP32 accuracy); 0, 2: full records (built-in;
 *                                 measured no faster at 24^4, n = 16)
 *   RHMC_TUNE_SHIFT_FREEZE_NANO   mixed precision: shifted systems stop being updated once their
 *                                 recursive residuals are below max(tol, value x 1e-9)
 *                                 (0: tol, built-in)
 *   RHMC_TUNE_REFINE_LANES        defect corrections of different shifts run concurrently on
 *                                 up to this many streams, one host thread each (0: 4, the
 *                                 most; 1: in turn on the caller's stream)
 *   RHMC_TUNE_AXPY_SCALAR         mixed precision, tall-skinny updates Y = C + A M (with or
 *                                 without the fused Gram): 1 = scalar FP32 FMAs; 0 = packed
 *                                 FP32x2 FMAs (built-in)
 *   RHMC_TUNE_NO_DEFECT_CORRECTION  1: no defect corrections after the multishift phase; the
 *                                 FP64 true residuals it left are reported (info) and shifts
 *                                 above tol give NOT_CONVERGED (for convergence studies)
 *   RHMC_TUNE_BASIS_ITERS         mixed precision, several shifts: the block basis Q_k is kept for
 *                                 up to this many iterations (V/2 * 3 * n_rhs * 8 bytes each,
 *                                 counted by rhmc_workspace_bytes) and the shifted solutions are
 *                                 assembled from it at the end of the multishift phase instead of
 *                                 updating P^(s), X^(s) every iteration; a solve that runs longer
 *                                 switches to the updates at that point.  0 = built-in (up to 384
 *                                 iterations within a quarter of the device memory, off below
 *                                 24), 1 = off, >= 2 = that capacity
 *   RHMC_TUNE_BASIS_GEMM          the assembly's contraction: 0 = tcgen05 tensor-core kernel (FP16
 *                                 pieces of the scaled FP32 operands, three products, FP32
 *                                 accumulation moved to a correctly rounded running sum every 48
 *                                 MMAs, written into the FP64 solutions), 1 = CUDA-core kernel
 *                                 (FP32 products, FP64 sum over blocks)
 *   RHMC_TUNE_BASIS_CHUNK         the assembly sums FP32 partial products over this many basis
 *                                 blocks and adds them in FP64 (0: one GEMM)
 *   RHMC_TUNE_BASIS_ACC_KT        the tensor-core assembly moves its accumulator into the correctly
 *                                 rounded running sum every this many K tiles of 64 reals (12 MMAs
 *                                 each; 0: built-in)
 *   RHMC_TUNE_NXN_FP64            mixed precision: the base n x n steps (alpha_k; rho_k, delta_k)
 *                                 in native FP64 (1) instead of double-float on the FP32 units (0)
 *   RHMC_TUNE_BASE_TILE           fused base step at n = 16: rows per warp tile x warps per CTA,
 *                                 0 = 8 x 16, 1 = 16 x 12, 2 = 16 x 8, 3 = 8 x 12
 *   RHMC_TUNE_GRAM_TILE           packed Gram at n = 16: rows per warp tile x warps per CTA,
 *                                 0 = 16 x 4, 1 = 32 x 8, 2 = 16 x 8, 3 = 8 x 8
 *   RHMC_TUNE_AXPY_ROWS           fused axpy + Gram at n = 16: 0 = 8-row, 1 = 16-row warp tiles
 *   RHMC_TUNE_CORRECTION_MARGIN_MILLI  a defect correction of a shift whose true residual is r
 *                                 stops when its recursive residual is value/1000 x tol / r
 *                                 (1 .. 999; 0: built-in)
 *   RHMC_TUNE_PHASE1_MARGIN_MILLI the multishift phase runs to value/1000 x tol before the
 *                                 true-residual checks (1 .. 999; 0: built-in)
 *   RHMC_TUNE_CORRECTION_CHECK_EVERY  iterations between the host checks of a defect
 *                                 correction (a divisor of 6 uses captured graphs; 0: built-in 1)
 * Value 0 restores the built-in choice.  INVALID_ARG for an unknown key. */
enum {
  RHMC_TUNE_HOP_RHS_PER_THREAD = 0,
  RHMC_TUNE_UPDATE_THREADS = 1,
  RHMC_TUNE_FLUSH_EVERY = 2,
  RHMC_TUNE_RELIABLE_DELTA_MILLI = 3,
  RHMC_TUNE_CHECK_EVERY = 4,
  RHMC_TUNE_NATIVE_FP64_RESIDUALS = 5,
  RHMC_TUNE_UPDATE_TENSOR = 6,
  RHMC_TUNE_GRAPHS = 7,
  RHMC_TUNE_HOP_STAGED = 8,
  RHMC_TUNE_REFINE_LANES = 9,
  RHMC_TUNE_LINKS12 = 10,
  RHMC_TUNE_SHIFT_FREEZE_NANO = 11,
  RHMC_TUNE_AXPY_SCALAR = 12,
  RHMC_TUNE_NO_DEFECT_CORRECTION = 13,
  RHMC_TUNE_BASIS_ITERS = 14,
  RHMC_TUNE_BASIS_GEMM = 15,
  RHMC_TUNE_BASIS_CHUNK = 16,
  RHMC_TUNE_BASIS_ACC_KT = 17,
  RHMC_TUNE_NXN_FP64 = 18,
  RHMC_TUNE_BASE_TILE = 19,
  RHMC_TUNE_GRAM_TILE = 20,
  RHMC_TUNE_AXPY_ROWS = 21,
  RHMC_TUNE_CORRECTION_MARGIN_MILLI = 22,
  RHMC_TUNE_PHASE1_MARGIN_MILLI = 23,
  RHMC_TUNE_CORRECTION_CHECK_EVERY = 24
};

/* Self-test of the device-side timeout path used by kernels that wait on
 * mbarriers (the tensor-core update): one warp on `device` waits for an
 * mbarrier phase that nothing completes; the wait gives up after about
 * `seconds` (0 < seconds <= 2) and the call returns RHMC_ERR_DEVICE_TIMEOUT
 * with the context usable afterwards.  Any other status means the timeout
 * path is broken. */
rhmc_status_t rhmc_selftest_bounded_wait(int device, double seconds, rhmc_stream_t s);

/* Measurement helper (no counterpart in the paper): the arithmetic peaks of
 * the CUDA cores of `device`, in TFLOP/s, for scalar FP32 FMA, packed FP32x2
 * FMA (fma.rn.f32x2, two lanes per instruction) and FP64 FMA.  Each is the
 * best of five launches of independent FMA chains filling every SM (2 flops
 * per FMA lane), timed with CUDA events on stream s after one warm-up launch;
 * about 50 ms in all.  They are the denominators of the FP32 and FP64 roofline
 * fractions (double-float operator, n x n coefficient chain, FP64 baseline).
 * The call synchronises s.  INVALID_ARG for a null output pointer. */
rhmc_status_t rhmc_probe_alu_peaks(int device, double *fp32_tflops, double *fp32x2_tflops, double *fp64_tflops,
                                   rhmc_stream_t s);

/* Self-test of internal arithmetic (no counterpart in the paper): for each of
 * the `count` doubles x_dev[k] > 0 (device), writes out_dev[q * count + k]
 * (device, 6 * count doubles) = q = 0: the library's Newton-Raphson FP64
 * reciprocal of the n x n coefficient step, 1: its square root, 2: its fast
 * reciprocal, 3: its reciprocal square root, 4: CUDA's IEEE 1.0 / x, 5: CUDA's
 * IEEE sqrt(x).  Asynchronous on stream s.  INVALID_ARG for null pointers or
 * count < 1. */
rhmc_status_t rhmc_selftest_fp64_helpers(const double *x_dev, int count, double *out_dev, rhmc_stream_t s);

/* Self-test of the double-float arithmetic (no counterpart in the paper): a
 * value is an unevaluated pair of floats hi + lo; products by an FMA-based
 * TwoProduct (Ogita, Rump and Oishi 2005), sums by TwoSum (Knuth).  The mixed
 * solve's FP64-accurate residuals and force, and its base n x n steps, run on
 * it.  For the `count` pairs a = x_dev[k], b = y_dev[k] (device doubles; the
 * stated accuracy holds for magnitudes within 2^-30 .. 2^30, where the low parts
 * and the products' rounding errors stay normal floats), writes
 * out_dev[q * count + k] (device, 8 * count doubles) = q = 0: hi of
 * a's split (RN_float(a)), 1: lo (RN_float(a - hi)), 2: hi + lo, 3: a + b,
 * 4: a b, 5: 1 / a, 6: 1 / sqrt(a) for a > 0 (else 0), 7: a b + b b as a
 * running sum of two products; 2-7 in double-float, returned in FP64.
 * Asynchronous on stream s.  INVALID_ARG for null pointers or count < 1. */
rhmc_status_t rhmc_selftest_df_helpers(const double *x_dev, const double *y_dev, int count, double *out_dev,
                                       rhmc_stream_t s);

/* The same settings for one context only (they take precedence over the
 * process-wide ones in every call on ctx, including the concurrent solves of
 * rhmc_block_multishift_cg_batch, so each ensemble can run its own tuned
 * kernels).  Value 0 falls back to the process-wide setting.  get returns the
 * value in effect for ctx. */
rhmc_status_t rhmc_ctx_tune_set(rhmc_ctx_t *ctx, int key, int value);
int rhmc_ctx_tune_get(const rhmc_ctx_t *ctx, int key);
rhmc_status_t rhmc_tune_set(int key, int value);
int rhmc_tune_get(int key);
rhmc_status_t rhmc_profile_read(int category, long long *launches, double *ms, double *bytes);
/* Tensor-core flops (multiply and add counted separately) issued by the
 * recorded launches of one category: nonzero for the tensor-core kernels only
 * (RHMC_PROF_BASIS_TC: three FP16 products per tile).  Same recording as
 * rhmc_profile_read. */
rhmc_status_t rhmc_profile_read_flops(int category, double *flops);

#ifdef __cplusplus
}
#endif

#endif /* RHMC_H */
