// The RHMC trajectory around the pseudofermion force (Sec. II set-up; Sec. IV
// run parameters: Wilson gauge action, two-level OMF2 integrator, heatbath and
// accept/reject with 1e-14 solves).  FP64 throughout: next to the force solves
// these kernels are a few percent of a trajectory.
//
// Conventions (the force's):
//   * U[site][mu][3][3], site = x + Lx (y + Ly (z + Lz t)), periodic links;
//   * S_g = beta sum_{x, mu<nu} (1 - Re tr Pi_{mu nu}(x) / 3),
//     Pi_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger;
//   * G = dS/dRe U + i dS/dIm U; the plaquettes through U_mu(x) add up to
//     Re tr(U_mu(x) V_mu(x)) with the staple sum
//     V_mu(x) = sum_{nu != mu} [U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger
//                              + U_nu(x+mu-nu)^dagger U_mu(x-nu)^dagger U_nu(x-nu)],
//     so G_g = -(beta / 3) V^dagger;
//   * P = sum_a p^a T^a (T^a = i lambda^a / 2), dU/dtau = P U,
//     K = -sum tr(P^2) = sum_a (p^a)^2 / 2, dP/dtau = TA(U G^dagger) / 2,
//     TA(M) = (M - M^dagger)/2 - tr(M - M^dagger)/6.
// One thread per link (or site, for the plaquettes); the reductions write one
// partial sum per CTA, added on the host in a fixed order.
#include <cmath>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

namespace {
constexpr int kTaylor = 16;  // degree of the exponential's Taylor polynomial (argument norm <= 1/2)

struct M3 {
  double2 e[9];
};

__device__ __forceinline__ M3 ld3(const double2 *p) {
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = p[k];
  return m;
}
__device__ __forceinline__ M3 zero3() {
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = make_double2(0.0, 0.0);
  return m;
}
// a b
__device__ __forceinline__ M3 mul(const M3 &a, const M3 &b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 x = a.e[i * 3 + k], y = b.e[k * 3 + j];
        re = fma(x.x, y.x, fma(-x.y, y.y, re));
        im = fma(x.x, y.y, fma(x.y, y.x, im));
      }
      c.e[i * 3 + j] = make_double2(re, im);
    }
  return c;
}
// a b^dagger
__device__ __forceinline__ M3 mul_nd(const M3 &a, const M3 &b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 x = a.e[i * 3 + k], y = b.e[j * 3 + k];  // x conj(y)
        re = fma(x.x, y.x, fma(x.y, y.y, re));
        im = fma(x.y, y.x, fma(-x.x, y.y, im));
      }
      c.e[i * 3 + j] = make_double2(re, im);
    }
  return c;
}
// a^dagger b
__device__ __forceinline__ M3 mul_dn(const M3 &a, const M3 &b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double re = 0.0, im = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double2 x = a.e[k * 3 + i], y = b.e[k * 3 + j];  // conj(x) y
        re = fma(x.x, y.x, fma(x.y, y.y, re));
        im = fma(x.x, y.y, fma(-x.y, y.x, im));
      }
      c.e[i * 3 + j] = make_double2(re, im);
    }
  return c;
}
__device__ __forceinline__ void addto(M3 &a, const M3 &b) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    a.e[k].x += b.e[k].x;
    a.e[k].y += b.e[k].y;
  }
}
// p += c TA(m)
__device__ __forceinline__ void add_ta(double2 *p, const M3 &m, double c) {
  const double t = (m.e[0].y + m.e[4].y + m.e[8].y) / 3.0;  // Im tr(M) / 3: (M - M^dagger)/2 has an imaginary diagonal
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const double2 a = m.e[i * 3 + j], b = m.e[j * 3 + i];
      double2 f = make_double2(0.5 * (a.x - b.x), 0.5 * (a.y + b.y));
      if (i == j) f.y -= t;
      double2 q = p[i * 3 + j];
      q.x = fma(c, f.x, q.x);
      q.y = fma(c, f.y, q.y);
      p[i * 3 + j] = q;
    }
}

__device__ __forceinline__ void lex_coords(const Geom &g, long lex, int x[4]) {
  long r = lex;
  x[0] = (int)(r % g.L[0]);
  r /= g.L[0];
  x[1] = (int)(r % g.L[1]);
  r /= g.L[1];
  x[2] = (int)(r % g.L[2]);
  x[3] = (int)(r / g.L[2]);
}
// x + d mu (periodic), d = +1 / -1, as coordinates
__device__ __forceinline__ void step(const Geom &g, const int x[4], int mu, int d, int y[4]) {
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    int v = x[nu];
    if (nu == mu) {
      v += d;
      if (v < 0) v += g.L[nu];
      if (v >= g.L[nu]) v -= g.L[nu];
    }
    y[nu] = v;
  }
}
__device__ __forceinline__ M3 link(const double2 *U, const Geom &g, const int x[4], int mu) {
  return ld3(U + (lex_of(g, x) * 4 + mu) * 9);
}

// sum of the partial sums of a CTA (blockDim.x == 256) into partial[blockIdx.x]
__device__ __forceinline__ void cta_sum(double v, double *partial) {
  __shared__ double red[256];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}
}  // namespace

// partial[b] = sum over the CTA's sites and planes mu < nu of (1 - Re tr Pi / 3).
// Re tr(A B^dagger) = sum_ij Re(A_ij conj(B_ij)) with A = U_mu(x) U_nu(x+mu),
// B = U_nu(x) U_mu(x+nu).
__global__ void __launch_bounds__(256) k_plaquette(Geom g, const double2 *__restrict__ U, double *__restrict__ partial) {
  double acc = 0.0;
  for (long site = (long)blockIdx.x * blockDim.x + threadIdx.x; site < g.V; site += (long)gridDim.x * blockDim.x) {
    int x[4];
    lex_coords(g, site, x);
    for (int mu = 0; mu < 3; ++mu) {
      int xm[4];
      step(g, x, mu, 1, xm);
      const M3 Um = ld3(U + (site * 4 + mu) * 9);
      for (int nu = mu + 1; nu < 4; ++nu) {
        int xn[4];
        step(g, x, nu, 1, xn);
        const M3 A = mul(Um, link(U, g, xm, nu));
        const M3 B = mul(ld3(U + (site * 4 + nu) * 9), link(U, g, xn, mu));
        double rt = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) rt = fma(A.e[k].x, B.e[k].x, fma(A.e[k].y, B.e[k].y, rt));
        acc += 1.0 - rt / 3.0;
      }
    }
  }
  cta_sum(acc, partial);
}

// partial[b] = -sum over the CTA's links of Re tr(P P)
__global__ void __launch_bounds__(256) k_kinetic(const double2 *__restrict__ P, long nlinks, double *__restrict__ partial) {
  double acc = 0.0;
  for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (long)gridDim.x * blockDim.x) {
    const M3 p = ld3(P + l * 9);
    double rt = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double2 a = p.e[i * 3 + j], b = p.e[j * 3 + i];
        rt = fma(a.x, b.x, fma(-a.y, b.y, rt));
      }
    acc -= rt;
  }
  cta_sum(acc, partial);
}

// P = sum_a p^a T^a, T^a = i lambda^a / 2 in the standard Gell-Mann basis
__global__ void __launch_bounds__(256) k_momenta(const double *__restrict__ p, double2 *__restrict__ P, long nlinks) {
  const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlinks) return;
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = 0.5 * p[l * 8 + k];
  const double r3 = 0.57735026918962576451;  // 1 / sqrt(3)
  double2 *o = P + l * 9;
  o[0] = make_double2(0.0, a[2] + r3 * a[7]);
  o[4] = make_double2(0.0, -a[2] + r3 * a[7]);
  o[8] = make_double2(0.0, -2.0 * r3 * a[7]);
  o[1] = make_double2(a[1], a[0]);   // i (lambda1 p1 + lambda2 p2) / 2, entry (0, 1)
  o[3] = make_double2(-a[1], a[0]);  // entry (1, 0)
  o[2] = make_double2(a[4], a[3]);
  o[6] = make_double2(-a[4], a[3]);
  o[5] = make_double2(a[6], a[5]);
  o[7] = make_double2(-a[6], a[5]);
}

// P_mu(x) += coef TA(U_mu(x) V_mu(x)); the kick P += eps TA(U G_g^dagger)/2 with
// G_g = -(beta/3) V^dagger has coef = -eps beta / 6
__global__ void __launch_bounds__(128) k_gauge_momentum(Geom g, const double2 *__restrict__ U, double2 *__restrict__ P,
                                                        double coef) {
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * g.V) return;
  const long site = e >> 2;
  const int mu = (int)(e & 3);
  int x[4], xp[4];
  lex_coords(g, site, x);
  step(g, x, mu, 1, xp);
  M3 V = zero3();
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    int xn[4], xd[4], xpd[4];
    step(g, x, nu, 1, xn);   // x + nu
    step(g, x, nu, -1, xd);  // x - nu
    step(g, xd, mu, 1, xpd); // x + mu - nu
    // U_nu(x+mu) U_mu(x+nu)^dagger U_nu(x)^dagger
    addto(V, mul_nd(mul_nd(link(U, g, xp, nu), link(U, g, xn, mu)), ld3(U + (site * 4 + nu) * 9)));
    // (U_mu(x-nu) U_nu(x+mu-nu))^dagger U_nu(x-nu)
    addto(V, mul_dn(mul(link(U, g, xd, mu), link(U, g, xpd, nu)), link(U, g, xd, nu)));
  }
  add_ta(P + e * 9, mul(ld3(U + e * 9), V), coef);
}

// P += coef TA(U G^dagger)
__global__ void __launch_bounds__(128) k_momentum_update(const double2 *__restrict__ U, const double2 *__restrict__ G,
                                                         double2 *__restrict__ P, long nlinks, double coef) {
  const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlinks) return;
  add_ta(P + l * 9, mul_nd(ld3(U + l * 9), ld3(G + l * 9)), coef);
}

// U <- exp(eps P) U.  exp(Y) for |Y|_F <= 1/2 by the Taylor polynomial of degree
// kTaylor in Horner form, E = I + Y (I + Y/2 (I + ... (I + Y/kTaylor))), whose
// remainder is below |Y|^(kTaylor+1) / (kTaylor+1)! e^|Y| < 4e-20; larger
// arguments are scaled by 2^-k first and the result squared k times.
__global__ void __launch_bounds__(128) k_link_update(double2 *__restrict__ U, const double2 *__restrict__ P, long nlinks,
                                                     double eps) {
  const long l = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nlinks) return;
  M3 Y = ld3(P + l * 9);
  double n2 = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Y.e[k].x *= eps;
    Y.e[k].y *= eps;
    n2 = fma(Y.e[k].x, Y.e[k].x, fma(Y.e[k].y, Y.e[k].y, n2));
  }
  int sq = 0;
  double sc = 1.0;
  while (n2 * sc * sc > 0.25 && sq < 64) {  // bounded: a non-finite norm stops at 64
    sc *= 0.5;
    ++sq;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    Y.e[k].x *= sc;
    Y.e[k].y *= sc;
  }
  M3 E = zero3();
  E.e[0].x = E.e[4].x = E.e[8].x = 1.0;
#pragma unroll
  for (int k = kTaylor; k >= 1; --k) {
    E = mul(Y, E);
    const double r = 1.0 / k;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      E.e[q].x *= r;
      E.e[q].y *= r;
    }
    E.e[0].x += 1.0;
    E.e[4].x += 1.0;
    E.e[8].x += 1.0;
  }
  for (int i = 0; i < sq; ++i) E = mul(E, E);
  const M3 u = mul(E, ld3(U + l * 9));
#pragma unroll
  for (int k = 0; k < 9; ++k) U[l * 9 + k] = u.e[k];
}

// ------------------------------------------------------------ launch wrappers
namespace {
constexpr size_t kLinkBytes = 9 * sizeof(double2);

rhmc_status_t reduce_parts(double *parts, int nparts, cudaStream_t s, double *out) {
  std::vector<double> h(nparts);
  RHMC_CUDA_TRY(cudaMemcpyAsync(h.data(), parts, sizeof(double) * nparts, cudaMemcpyDeviceToHost, s));
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  double sum = 0.0;
  for (int q = 0; q < nparts; ++q) sum += h[q];
  *out = sum;
  return RHMC_OK;
}

struct Lat {
  int device = 0;
  Geom g{};
};
rhmc_status_t lattice(rhmc_ctx_t *c, Lat *l) { return ctx_lattice(c, &l->device, &l->g); }
}  // namespace

rhmc_status_t gauge_action(rhmc_ctx_t *c, const Geom &g, const double2 *U, double beta, double *S, cudaStream_t s) {
  double *parts;
  int nparts;
  RHMC_TRY(ctx_partials(c, &parts, &nparts));
  prof_begin(PROF_OTHER, s);
  k_plaquette<<<nparts, 256, 0, s>>>(g, U, parts);
  prof_end(s, (double)g.V * 4 * kLinkBytes);
  RHMC_LAUNCH_CHECK();
  double sum = 0.0;
  RHMC_TRY(reduce_parts(parts, nparts, s, &sum));
  *S = beta * sum;
  return RHMC_OK;
}

rhmc_status_t kinetic_energy(rhmc_ctx_t *c, const Geom &g, const double2 *P, double *K, cudaStream_t s) {
  double *parts;
  int nparts;
  RHMC_TRY(ctx_partials(c, &parts, &nparts));
  prof_begin(PROF_OTHER, s);
  k_kinetic<<<nparts, 256, 0, s>>>(P, g.V * 4, parts);
  prof_end(s, (double)g.V * 4 * kLinkBytes);
  RHMC_LAUNCH_CHECK();
  return reduce_parts(parts, nparts, s, K);
}

rhmc_status_t momenta_from_normals(const Geom &g, const double *p, double2 *P, cudaStream_t s) {
  const long nl = g.V * 4;
  prof_begin(PROF_OTHER, s);
  k_momenta<<<(unsigned)((nl + 255) / 256), 256, 0, s>>>(p, P, nl);
  prof_end(s, (double)nl * (8 * sizeof(double) + kLinkBytes));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t gauge_momentum(const Geom &g, const double2 *U, double2 *P, double beta, double eps, cudaStream_t s) {
  const long nl = g.V * 4;
  prof_begin(PROF_OTHER, s);
  k_gauge_momentum<<<(unsigned)((nl + 127) / 128), 128, 0, s>>>(g, U, P, -eps * beta / 6.0);
  prof_end(s, (double)nl * 3 * kLinkBytes);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t momentum_update(const Geom &g, const double2 *U, const double2 *G, double2 *P, double eps,
                              cudaStream_t s) {
  const long nl = g.V * 4;
  prof_begin(PROF_OTHER, s);
  k_momentum_update<<<(unsigned)((nl + 127) / 128), 128, 0, s>>>(U, G, P, nl, 0.5 * eps);
  prof_end(s, (double)nl * 4 * kLinkBytes);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t link_update(const Geom &g, double2 *U, const double2 *P, double eps, cudaStream_t s) {
  const long nl = g.V * 4;
  prof_begin(PROF_OTHER, s);
  k_link_update<<<(unsigned)((nl + 127) / 128), 128, 0, s>>>(U, P, nl, eps);
  prof_end(s, (double)nl * 3 * kLinkBytes);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// ------------------------------------------------------------ integrator
namespace {
struct Md {
  rhmc_ctx_t *c;
  Geom g;
  double2 *U, *P, *G;
  const void *Phi;
  int n_pf;
  const rhmc_rational_t *md;
  const rhmc_md_params_t *p;
  rhmc_md_info_t *info;
  cudaStream_t s;

  rhmc_status_t fermion_kick(double eps) {
    if (!Phi || n_pf == 0 || eps == 0.0) return RHMC_OK;
    RHMC_TRY(rhmc_set_gauge(c, U, s));
    rhmc_info_t fi{};
    const rhmc_status_t st = rhmc_force(c, Phi, n_pf, md->alpha0, md->alpha, md->beta, md->n_shifts, p->tol_md,
                                        p->max_iter, p->precision_md, nullptr, G, nullptr, nullptr, &fi, s);
    info->force_evals += 1;
    info->solver_iters += fi.iters + fi.refine_iters;
    info->dirac_calls += fi.dirac_calls;
    if (fi.true_rel_resid_max > info->max_rel_resid) info->max_rel_resid = fi.true_rel_resid_max;
    if (st != RHMC_OK) return st;
    return momentum_update(g, U, G, P, eps, s);
  }
  rhmc_status_t gauge_kick(double eps) {
    info->gauge_force_evals += 1;
    return gauge_momentum(g, U, P, p->beta, eps, s);
  }
  // D(h): n_gauge OMF2 steps of the gauge force, the kicks at the same links merged
  rhmc_status_t drift(double h) {
    const double e = h / p->n_gauge, lam = p->lambda;
    RHMC_TRY(gauge_kick(lam * e));
    for (int i = 0; i < p->n_gauge; ++i) {
      RHMC_TRY(link_update(g, U, P, 0.5 * e, s));
      RHMC_TRY(gauge_kick((1.0 - 2.0 * lam) * e));
      RHMC_TRY(link_update(g, U, P, 0.5 * e, s));
      RHMC_TRY(gauge_kick(i + 1 < p->n_gauge ? 2.0 * lam * e : lam * e));
    }
    return RHMC_OK;
  }
  rhmc_status_t run() {
    const double e = p->tau / p->n_steps, lam = p->lambda;
    RHMC_TRY(fermion_kick(lam * e));
    for (int k = 0; k < p->n_steps; ++k) {
      RHMC_TRY(drift(0.5 * e));
      RHMC_TRY(fermion_kick((1.0 - 2.0 * lam) * e));
      RHMC_TRY(drift(0.5 * e));
      RHMC_TRY(fermion_kick(k + 1 < p->n_steps ? 2.0 * lam * e : lam * e));
    }
    return RHMC_OK;
  }
};

rhmc_status_t check_md(const rhmc_rational_t *md, const rhmc_md_params_t *p, const void *Phi, int n_pf) {
  if (!p || p->n_steps < 1 || p->n_gauge < 1 || !(p->tau >= 0.0) || !std::isfinite(p->lambda) ||
      !std::isfinite(p->beta)) {
    set_error("md parameters: need n_steps >= 1, n_gauge >= 1, finite tau >= 0, lambda and beta");
    return RHMC_ERR_INVALID_ARG;
  }
  if (Phi && n_pf > 0) {
    if (n_pf > RHMC_MAX_NRHS || !md || !md->alpha || !md->beta || md->n_shifts < 1 ||
        md->n_shifts > RHMC_MAX_SHIFTS) {
      set_error("md rational: need 1 <= n_shifts <= %d, alpha and beta, and n_pf <= %d", RHMC_MAX_SHIFTS,
                RHMC_MAX_NRHS);
      return RHMC_ERR_INVALID_ARG;
    }
    if (p->precision_md != RHMC_FP64 && p->precision_md != RHMC_MIXED_FP32) {
      set_error("md precision must be RHMC_FP64 or RHMC_MIXED_FP32");
      return RHMC_ERR_INVALID_ARG;
    }
  }
  return RHMC_OK;
}
}  // namespace

}  // namespace rhmc

using namespace rhmc;

namespace {
struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~Guard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};
}  // namespace

#define RHMC_LATTICE(c, L)                                                    \
  Lat L;                                                                       \
  if (!(c)) {                                                                  \
    set_error("null context");                                                 \
    return RHMC_ERR_INVALID_ARG;                                               \
  }                                                                            \
  RHMC_TRY(lattice(c, &L));                                                    \
  Guard dg_(L.device);                                                         \
  CtxTuneScope ts_(c)

extern "C" {

rhmc_status_t rhmc_gauge_action(rhmc_ctx_t *c, const void *U, double beta, double *S_out, rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  if (!U || !S_out) {
    set_error("rhmc_gauge_action: null U or S_out");
    return RHMC_ERR_INVALID_ARG;
  }
  return gauge_action(c, L.g, (const double2 *)U, beta, S_out, (cudaStream_t)sv);
}

rhmc_status_t rhmc_kinetic_energy(rhmc_ctx_t *c, const void *P, double *K_out, rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  if (!P || !K_out) {
    set_error("rhmc_kinetic_energy: null P or K_out");
    return RHMC_ERR_INVALID_ARG;
  }
  return kinetic_energy(c, L.g, (const double2 *)P, K_out, (cudaStream_t)sv);
}

rhmc_status_t rhmc_momenta_from_normals(rhmc_ctx_t *c, const double *p, void *P, rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  if (!p || !P) {
    set_error("rhmc_momenta_from_normals: null p or P");
    return RHMC_ERR_INVALID_ARG;
  }
  return momenta_from_normals(L.g, p, (double2 *)P, (cudaStream_t)sv);
}

rhmc_status_t rhmc_gauge_momentum(rhmc_ctx_t *c, const void *U, void *P, double beta, double eps, rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  if (!U || !P) {
    set_error("rhmc_gauge_momentum: null U or P");
    return RHMC_ERR_INVALID_ARG;
  }
  return gauge_momentum(L.g, (const double2 *)U, (double2 *)P, beta, eps, (cudaStream_t)sv);
}

rhmc_status_t rhmc_momentum_update(rhmc_ctx_t *c, const void *U, const void *G, void *P, double eps,
                                   rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  if (!U || !G || !P) {
    set_error("rhmc_momentum_update: null U, G or P");
    return RHMC_ERR_INVALID_ARG;
  }
  return momentum_update(L.g, (const double2 *)U, (const double2 *)G, (double2 *)P, eps, (cudaStream_t)sv);
}

rhmc_status_t rhmc_link_update(rhmc_ctx_t *c, void *U, const void *P, double eps, rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  if (!U || !P) {
    set_error("rhmc_link_update: null U or P");
    return RHMC_ERR_INVALID_ARG;
  }
  return link_update(L.g, (double2 *)U, (const double2 *)P, eps, (cudaStream_t)sv);
}

rhmc_status_t rhmc_md_evolve(rhmc_ctx_t *c, void *U, void *P, const void *Phi, int n_pf, const rhmc_rational_t *md,
                             const rhmc_md_params_t *p, rhmc_md_info_t *info, rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  if (!U || !P || (Phi && n_pf < 1)) {
    set_error("rhmc_md_evolve: null U or P, or pseudofermions with n_pf < 1");
    return RHMC_ERR_INVALID_ARG;
  }
  RHMC_TRY(check_md(md, p, Phi, n_pf));
  rhmc_md_info_t local{};
  if (!info) info = &local;
  *info = rhmc_md_info_t{};
  void *buf = nullptr;
  if (Phi) RHMC_TRY(ctx_md_buffer(c, (size_t)L.g.V * 4 * kLinkBytes, &buf));
  Md m{c, L.g, (double2 *)U, (double2 *)P, (double2 *)buf, Phi, Phi ? n_pf : 0, md, p, info, (cudaStream_t)sv};
  RHMC_TRY(m.run());
  // the context's staged links follow U
  return rhmc_set_gauge(c, U, sv);
}

rhmc_status_t rhmc_hmc_trajectory(rhmc_ctx_t *c, void *U, const double *pn, const void *eta, int n_pf,
                                  const rhmc_rational_t *hb, const rhmc_rational_t *md, const rhmc_rational_t *act,
                                  const rhmc_md_params_t *p, double tol_action, double u_accept, void *Phi_out,
                                  rhmc_hmc_info_t *info, rhmc_stream_t sv) {
  RHMC_LATTICE(c, L);
  const bool ferm = eta != nullptr;
  if (!U || !pn || (ferm && (n_pf < 1 || n_pf > RHMC_MAX_NRHS)) || !(tol_action > 0.0)) {
    set_error("rhmc_hmc_trajectory: null U or p, n_pf out of [1, %d] with eta, or tol_action <= 0", RHMC_MAX_NRHS);
    return RHMC_ERR_INVALID_ARG;
  }
  for (const rhmc_rational_t *r : {hb, act})
    if (ferm && (!r || !r->alpha || !r->beta || r->n_shifts < 1 || r->n_shifts > RHMC_MAX_SHIFTS)) {
      set_error("rhmc_hmc_trajectory: heatbath and action rationals need 1 <= n_shifts <= %d", RHMC_MAX_SHIFTS);
      return RHMC_ERR_INVALID_ARG;
    }
  RHMC_TRY(check_md(md, p, ferm ? eta : nullptr, n_pf));
  cudaStream_t s = (cudaStream_t)sv;
  rhmc_hmc_info_t local{};
  if (!info) info = &local;
  *info = rhmc_hmc_info_t{};

  // buffer: momenta | trial links | force | pseudofermions
  const size_t fld = (size_t)L.g.V * 4 * kLinkBytes;
  const size_t pf = ferm ? (size_t)L.g.Vh * 3 * n_pf * sizeof(double2) : 0;
  void *buf = nullptr;
  RHMC_TRY(ctx_md_buffer(c, 3 * fld + pf, &buf));
  double2 *P = (double2 *)buf;
  double2 *U1 = (double2 *)((char *)buf + fld);
  double2 *G = (double2 *)((char *)buf + 2 * fld);
  double2 *Phi = ferm ? (double2 *)((char *)buf + 3 * fld) : nullptr;

  RHMC_TRY(momenta_from_normals(L.g, pn, P, s));
  RHMC_TRY(rhmc_set_gauge(c, U, sv));
  auto fermion_action = [&](double *Sf) -> rhmc_status_t {
    *Sf = 0.0;
    if (!ferm) return RHMC_OK;
    return rhmc_force(c, Phi, n_pf, act->alpha0, act->alpha, act->beta, act->n_shifts, tol_action, 0, RHMC_FP64,
                      nullptr, nullptr, Sf, nullptr, nullptr, sv);
  };
  if (ferm) {
    RHMC_TRY(rhmc_rational_solve(c, eta, n_pf, hb->alpha0, hb->alpha, hb->beta, hb->n_shifts, tol_action, 0, Phi,
                                 nullptr, nullptr, sv));
    if (Phi_out) RHMC_CUDA_TRY(cudaMemcpyAsync(Phi_out, Phi, pf, cudaMemcpyDeviceToDevice, s));
  }
  RHMC_TRY(kinetic_energy(c, L.g, P, &info->K[0], s));
  RHMC_TRY(gauge_action(c, L.g, (const double2 *)U, p->beta, &info->S_g[0], s));
  RHMC_TRY(fermion_action(&info->S_f[0]));
  info->H_old = info->K[0] + info->S_g[0] + info->S_f[0];

  RHMC_CUDA_TRY(cudaMemcpyAsync(U1, U, fld, cudaMemcpyDeviceToDevice, s));
  Md m{c, L.g, U1, P, G, Phi, ferm ? n_pf : 0, md, p, &info->md, s};
  RHMC_TRY(m.run());

  RHMC_TRY(rhmc_set_gauge(c, U1, sv));
  RHMC_TRY(kinetic_energy(c, L.g, P, &info->K[1], s));
  RHMC_TRY(gauge_action(c, L.g, U1, p->beta, &info->S_g[1], s));
  RHMC_TRY(fermion_action(&info->S_f[1]));
  info->H_new = info->K[1] + info->S_g[1] + info->S_f[1];
  info->dH = info->H_new - info->H_old;
  info->accepted = (info->dH <= 0.0 || u_accept < std::exp(-info->dH)) ? 1 : 0;
  if (info->accepted) {
    RHMC_CUDA_TRY(cudaMemcpyAsync(U, U1, fld, cudaMemcpyDeviceToDevice, s));
    RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    RHMC_TRY(rhmc_set_gauge(c, U, sv));
  }
  return RHMC_OK;
}

}  // extern "C"
