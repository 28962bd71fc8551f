// Pseudofermion force, Eq. (force) with the rational approximation of Eq. (RA):
//
//   G_mu(x) = dS/dRe U_mu(x) + i dS/dIm U_mu(x)
//           = 2 eps(x) eta_mu(x) b_mu(x) sum_s alpha_s sum_i W_si(x) W_si(x+mu)^dagger,
//
// with W = X^(s) on even sites and W = Y^(s) = D_oe X^(s) on odd sites (the
// derivative of S = sum_s alpha_s phi^dagger (A + beta_s)^-1 phi through
// A = 4m^2 - D_eo D_oe and D_oe = -D_eo^dagger).  Per link this is a
// (3 x R)(R x 3) contraction over R = n * n_shifts columns.  FP64 throughout.
//
// One group of 16 lanes per link: lane i accumulates the columns i, i+16, ...
// of every shift (coalesced loads across the lanes), the 9 complex partial
// sums are then reduced across the group with shuffles.
#include "common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace rhmc {

__global__ void __launch_bounds__(256) k_force(Geom g, const double2 *__restrict__ X, const double2 *__restrict__ Y,
                                               int n, int ns, long fstride, const double *__restrict__ alpha,
                                               int bc_t, double2 *__restrict__ G) {
  const long pair = (long)blockIdx.x * 16 + threadIdx.x / 16;
  const int lane = threadIdx.x & 15;
  const bool valid = pair < 4 * g.V;
  const long lex = valid ? (pair >> 2) : 0;
  const int mu = (int)(pair & 3);
  int x[4];
  {
    long r = lex;
    x[0] = (int)(r % g.L[0]);
    r /= g.L[0];
    x[1] = (int)(r % g.L[1]);
    r /= g.L[1];
    x[2] = (int)(r % g.L[2]);
    x[3] = (int)(r / g.L[2]);
  }
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long hx = lex >> 1;
  const long hy = nb_rank(g, x, mu, +1);
  const double2 *Wx = par ? Y : X;
  const double2 *Wy = par ? X : Y;
  double2 acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = make_double2(0.0, 0.0);
  if (valid) {
    for (int s = 0; s < ns; ++s) {
      const double a = alpha[s];
      const double2 *px = Wx + s * fstride + hx * 3 * n;
      const double2 *py = Wy + s * fstride + hy * 3 * n;
      for (int i = lane; i < n; i += 16) {
        double2 u[3], v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          u[c] = px[c * n + i];
          const double2 w = py[c * n + i];
          v[c] = make_double2(a * w.x, a * w.y);
        }
#pragma unroll
        for (int ca = 0; ca < 3; ++ca)
#pragma unroll
          for (int cb = 0; cb < 3; ++cb) cmac_bcj<double>(acc[ca * 3 + cb], u[ca], v[cb]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q)
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      acc[q].x += __shfl_xor_sync(0xffffffffu, acc[q].x, off);
      acc[q].y += __shfl_xor_sync(0xffffffffu, acc[q].y, off);
    }
  if (valid && lane == 0) {
    int sum = 0;
#pragma unroll
    for (int nu = 0; nu < 4; ++nu)
      if (nu < mu) sum += x[nu];
    double pre = 2.0 * (par ? -1.0 : 1.0) * ((sum & 1) ? -1.0 : 1.0);
    if (mu == 3 && bc_t == -1 && x[3] == g.L[3] - 1) pre = -pre;
    double2 *o = G + pair * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) o[q] = make_double2(pre * acc[q].x, pre * acc[q].y);
  }
}

// Y = alpha0 Phi + sum_s alpha_s X^(s): the rational approximation R(A) Phi of
// Eq. (RA) from the shifted solutions (FP64).
struct Coeffs {
  double a[kMaxS];
};

__global__ void k_rational_combine(const double2 *__restrict__ Phi, double alpha0, const Coeffs alpha,
                                   const double2 *__restrict__ X, int ns, long len, double2 *__restrict__ Y) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const double2 p = Phi[i];
  double2 y = make_double2(alpha0 * p.x, alpha0 * p.y);
  for (int s = 0; s < ns; ++s) {
    const double2 x = X[s * len + i];
    y.x = fma(alpha.a[s], x.x, y.x);
    y.y = fma(alpha.a[s], x.y, y.y);
  }
  Y[i] = y;
}

rhmc_status_t rational_combine(const double2 *Phi, double alpha0, const double *alpha_host, const double2 *X, int ns,
                               long len, double2 *Y, cudaStream_t s) {
  if (ns < 1 || ns > kMaxS) return RHMC_ERR_INVALID_ARG;
  Coeffs c{};
  for (int q = 0; q < ns; ++q) c.a[q] = alpha_host[q];
  k_rational_combine<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(Phi, alpha0, c, X, ns, len, Y);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// The same contraction in double-float arithmetic on the FP32 units (FP64
// accuracy, 2^-44 relative per product): X and Y arrive as double-float fields
// (float4 per complex), alpha_s is split into a float pair once per shift and
// folded into the W(x+mu) factor, the products u conj(v') are formed with
// TwoProduct and summed with TwoSum; G is assembled in FP64.
namespace {
// (ah + al) (bh + bl) as a normalised pair
__device__ __forceinline__ float2 df_mul(float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}
}  // namespace

__global__ void __launch_bounds__(256) k_force_df(Geom g, const float4 *__restrict__ X, const float4 *__restrict__ Y,
                                                  int n, int ns, long fstride, const double *__restrict__ alpha,
                                                  int bc_t, double2 *__restrict__ G) {
  using namespace df;
  const long pair = (long)blockIdx.x * 16 + threadIdx.x / 16;
  const int lane = threadIdx.x & 15;
  const bool valid = pair < 4 * g.V;
  const long lex = valid ? (pair >> 2) : 0;
  const int mu = (int)(pair & 3);
  int x[4];
  {
    long r = lex;
    x[0] = (int)(r % g.L[0]);
    r /= g.L[0];
    x[1] = (int)(r % g.L[1]);
    r /= g.L[1];
    x[2] = (int)(r % g.L[2]);
    x[3] = (int)(r / g.L[2]);
  }
  const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long hx = lex >> 1;
  const long hy = nb_rank(g, x, mu, +1);
  const float4 *Wx = par ? Y : X;
  const float4 *Wy = par ? X : Y;
  DF re[9], im[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) re[q] = im[q] = DF{0.f, 0.f};
  if (valid) {
    for (int s = 0; s < ns; ++s) {
      const double a = alpha[s];
      const float ah = (float)a, al = (float)(a - (double)ah);
      const float4 *px = Wx + s * fstride + hx * 3 * n;
      const float4 *py = Wy + s * fstride + hy * 3 * n;
      for (int i = lane; i < n; i += 16) {
        float4 u[3], v[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          u[c] = px[c * n + i];
          const float4 w = py[c * n + i];
          const float2 vr = df_mul(ah, al, w.x, w.z), vi = df_mul(ah, al, w.y, w.w);
          v[c] = make_float4(vr.x, vi.x, vr.y, vi.y);
        }
#pragma unroll
        for (int ca = 0; ca < 3; ++ca)
#pragma unroll
          for (int cb = 0; cb < 3; ++cb) {
            // u conj(v): re = u.re v.re + u.im v.im, im = u.im v.re - u.re v.im
            const int q = ca * 3 + cb;
            df_add_prod(re[q], u[ca].x, u[ca].z, v[cb].x, v[cb].z);
            df_add_prod(re[q], u[ca].y, u[ca].w, v[cb].y, v[cb].w);
            df_add_prod(im[q], u[ca].y, u[ca].w, v[cb].x, v[cb].z);
            df_add_prod(im[q], -u[ca].x, -u[ca].z, v[cb].y, v[cb].w);
          }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q)
#pragma unroll
    for (int off = 8; off > 0; off >>= 1) {
      DF ro{__shfl_xor_sync(0xffffffffu, re[q].h, off), __shfl_xor_sync(0xffffffffu, re[q].e, off)};
      DF io{__shfl_xor_sync(0xffffffffu, im[q].h, off), __shfl_xor_sync(0xffffffffu, im[q].e, off)};
      re[q] = df_add(re[q], ro);
      im[q] = df_add(im[q], io);
    }
  if (valid && lane == 0) {
    int sum = 0;
#pragma unroll
    for (int nu = 0; nu < 4; ++nu)
      if (nu < mu) sum += x[nu];
    double pre = 2.0 * (par ? -1.0 : 1.0) * ((sum & 1) ? -1.0 : 1.0);
    if (mu == 3 && bc_t == -1 && x[3] == g.L[3] - 1) pre = -pre;
    double2 *o = G + pair * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q)
      o[q] = make_double2(pre * ((double)re[q].h + (double)re[q].e), pre * ((double)im[q].h + (double)im[q].e));
  }
}

rhmc_status_t force_links_df(const Geom &g, const float4 *X, const float4 *Y, int n, int nshift, long fstride,
                             const double *alpha_dev, int bc_t, double2 *G, cudaStream_t s) {
  const long pairs = 4 * g.V;
  const long grid = (pairs + 15) / 16;
  prof_begin(PROF_FORCE, s);
  k_force_df<<<(unsigned)grid, 256, 0, s>>>(g, X, Y, n, nshift, fstride, alpha_dev, bc_t, G);
  prof_end(s, 2.0 * nshift * g.Vh * 3.0 * n * sizeof(float4) + 4.0 * g.V * 9 * sizeof(double2));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t force_links(const Geom &g, const double2 *X, const double2 *Y, int n, int nshift, long fstride,
                          const double *alpha_dev, int bc_t, double2 *G, cudaStream_t s) {
  const long pairs = 4 * g.V;
  const long grid = (pairs + 15) / 16;
  prof_begin(PROF_FORCE, s);
  k_force<<<(unsigned)grid, 256, 0, s>>>(g, X, Y, n, nshift, fstride, alpha_dev, bc_t, G);
  // algorithmic bytes: X and Y of every shift once, G written once
  prof_end(s, 2.0 * nshift * g.Vh * 3.0 * n * sizeof(double2) + 4.0 * g.V * 9 * sizeof(double2));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// ------------------------------------------------------------ Lie-algebra force
// F_mu(x) = TA(U_mu(x) G_mu(x)^dagger), TA(M) = (M - M^dagger)/2 - tr(M - M^dagger)/6,
// the traceless anti-Hermitian projection: with generators T^a = i lambda^a / 2,
// the derivative of S along U -> exp(w T^a) U is F^a = Re tr(G^dagger T^a U)
// = tr(F T^a), so F = -2 sum_a F^a T^a and sum_a (F^a)^2 / 2 = |F|_F^2 / 4, the
// summand of the force norm F^2 (Sec. II).  FP64, one thread per link; each
// CTA writes the sum of its links' |F|_F^2 / 4 to partial[blockIdx.x].
__global__ void __launch_bounds__(256) k_force_lie(const double2 *__restrict__ U, const double2 *G,
                                                   double2 *F, long nlinks, double *__restrict__ partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long l = (long)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (long)gridDim.x * blockDim.x) {
    double2 u[9], g[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      u[e] = U[l * 9 + e];
      g[e] = G[l * 9 + e];
    }
    double2 m[9];  // M = U G^dagger
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        double re = 0.0, im = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const double2 a = u[i * 3 + k], b = g[j * 3 + k];  // a conj(b)
          re = fma(a.x, b.x, fma(a.y, b.y, re));
          im = fma(a.y, b.x, fma(-a.x, b.y, im));
        }
        m[i * 3 + j] = make_double2(re, im);
      }
    // (M - M^dagger)/2 has a purely imaginary diagonal; its trace / 3 is removed
    const double t = (m[0].y + m[4].y + m[8].y) / 3.0;
    double nrm = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const double2 a = m[i * 3 + j], b = m[j * 3 + i];
        double2 f = make_double2(0.5 * (a.x - b.x), 0.5 * (a.y + b.y));
        if (i == j) f.y -= t;
        nrm += f.x * f.x + f.y * f.y;
        if (F) F[l * 9 + i * 3 + j] = f;
      }
    acc += 0.25 * nrm;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

rhmc_status_t force_lie(const Geom &g, const double2 *U, const double2 *G, double2 *F, double *partial, int nparts,
                        cudaStream_t s) {
  prof_begin(PROF_FORCE, s);
  const long nlinks = g.V * 4;
  k_force_lie<<<nparts, 256, 0, s>>>(U, G, F, nlinks, partial);
  prof_end(s, (double)nlinks * 9 * sizeof(double2) * (F ? 3 : 2));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

}  // namespace rhmc
