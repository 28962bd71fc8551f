// Baseline: plain per-vector multishift CG (SCG, Sec. III) in FP64 for one
// right-hand side at a time, with the width-1 operator.  CG runs on
// (A + sigma_0); every shifted residual stays collinear with the base one,
// r^(s) = zeta^(s) r, and the shifted coefficients follow from the CG
// three-term recurrence:
//   zeta_{k+1} = zeta_k zeta_{k-1} a_{k-1} /
//                (a_{k-1} zeta_{k-1} (1 + (sigma_s - sigma_0) a_k) + a_k b_{k-1} (zeta_{k-1} - zeta_k)),
//   a^(s)_k = a_k zeta_{k+1} / zeta_k,   b^(s)_k = b_k (zeta_{k+1} / zeta_k)^2.
// Scalars live on the device; a shift is frozen once |zeta| |r| / |b| < tol.
#include "common.cuh"
#include "kernels.h"
#include "scg.h"

namespace rhmc {

// Sum of nparts partials by the whole CTA (256 threads); valid in every thread.
static __device__ double reduce_parts(const double *p, int nparts) {
  __shared__ double red[256];
  double s = 0.0;
  for (int q = threadIdx.x; q < nparts; q += blockDim.x) s += p[q];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void k_scg_init(ScgScalars *sc, const double *parts, int nparts, int ns, const double *sigma) {
  const double rr = reduce_parts(parts, nparts);
  if (threadIdx.x != 0) return;
  sc->rr = rr;
  sc->bb = rr;
  sc->alpha_prev = 1.0;
  sc->beta_prev = 0.0;
  for (int s = 0; s < ns; ++s) {
    sc->zeta[s] = 1.0;
    sc->zeta_prev[s] = 1.0;
    sc->zeta_next[s] = 1.0;
    sc->active[s] = 1;
    sc->sigma[s] = sigma[s];
  }
  sc->breakdown = 0;
}

// alpha_k and the shifted alphas
__global__ void k_scg_alpha(ScgScalars *sc, const double *parts, int nparts, int ns) {
  const double pAp = reduce_parts(parts, nparts);
  if (threadIdx.x != 0) return;
  if (!(pAp > 0.0)) sc->breakdown = 1;
  const double a = sc->rr / pAp;
  sc->alpha = a;
  sc->alpha_s[0] = a;
  sc->upd[0] = 1;
  for (int s = 1; s < ns; ++s) {
    if (!sc->active[s]) {
      sc->upd[s] = 0;
      continue;
    }
    const double ds = sc->sigma[s] - sc->sigma[0];
    const double z = sc->zeta[s], zp = sc->zeta_prev[s];
    const double zn = z * zp * sc->alpha_prev / (sc->alpha_prev * zp * (1.0 + ds * a) + a * sc->beta_prev * (zp - z));
    sc->zeta_next[s] = zn;
    sc->alpha_s[s] = a * zn / z;
    sc->upd[s] = 1;
  }
}

// r -= alpha Ap; x_s += alpha_s p_s; partial |r|^2
__global__ void __launch_bounds__(256) k_scg_update1(const ScgScalars *__restrict__ sc, double2 *__restrict__ r,
                                                     const double2 *__restrict__ Ap, double2 *__restrict__ x,
                                                     const double2 *__restrict__ p, int ns, long len,
                                                     double *__restrict__ parts) {
  __shared__ double red[256];
  const double a = sc->alpha;
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x) {
    double2 ri = r[i];
    const double2 api = Ap[i];
    ri.x -= a * api.x;
    ri.y -= a * api.y;
    r[i] = ri;
    acc += ri.x * ri.x + ri.y * ri.y;
    for (int s = 0; s < ns; ++s) {
      if (!sc->upd[s]) continue;
      const double as = sc->alpha_s[s];
      const double2 ps = p[s * len + i];
      double2 xs = x[s * len + i];
      xs.x += as * ps.x;
      xs.y += as * ps.y;
      x[s * len + i] = xs;
    }
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) parts[blockIdx.x] = red[0];
}

// beta_k, shifted betas, freezing, roll the recurrence
__global__ void k_scg_beta(ScgScalars *sc, const double *parts, int nparts, int ns, double tol) {
  const double rr_new = reduce_parts(parts, nparts);
  if (threadIdx.x != 0) return;
  const double b = rr_new / sc->rr;
  sc->beta = b;
  sc->beta_s[0] = b;
  sc->pz[0] = 1.0;
  const double rel = sqrt(rr_new / sc->bb);
  for (int s = 1; s < ns; ++s) {
    if (!sc->active[s]) continue;
    const double q = sc->zeta_next[s] / sc->zeta[s];
    sc->beta_s[s] = b * q * q;
    sc->pz[s] = sc->zeta_next[s];
    sc->zeta_prev[s] = sc->zeta[s];
    sc->zeta[s] = sc->zeta_next[s];
    if (fabs(sc->zeta[s]) * rel < tol) sc->active[s] = 0;
  }
  sc->alpha_prev = sc->alpha;
  sc->beta_prev = b;
  sc->rr = rr_new;
  sc->rel = rel;
}

// p_s = zeta_s r + beta_s p_s  for the shifts updated this iteration
__global__ void __launch_bounds__(256) k_scg_update2(const ScgScalars *__restrict__ sc, const double2 *__restrict__ r,
                                                     double2 *__restrict__ p, int ns, long len) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const double2 ri = r[i];
  for (int s = 0; s < ns; ++s) {
    if (!sc->upd[s]) continue;
    const double z = sc->pz[s], b = sc->beta_s[s];
    double2 ps = p[s * len + i];
    ps.x = z * ri.x + b * ps.x;
    ps.y = z * ri.y + b * ps.y;
    p[s * len + i] = ps;
  }
}

// strided column gather / scatter between an n-wide block and a single field
__global__ void k_column(const double2 *__restrict__ in, double2 *__restrict__ out, long rows, int n, int j,
                         int gather) {
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  if (gather)
    out[r] = in[r * n + j];
  else
    out[r * n + j] = in[r];
}

rhmc_status_t scg_init(ScgScalars *sc, const double *parts, int nparts, int ns, const double *sigma_dev,
                       cudaStream_t s) {
  k_scg_init<<<1, 256, 0, s>>>(sc, parts, nparts, ns, sigma_dev);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
rhmc_status_t scg_alpha(ScgScalars *sc, const double *parts, int nparts, int ns, cudaStream_t s) {
  k_scg_alpha<<<1, 256, 0, s>>>(sc, parts, nparts, ns);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
rhmc_status_t scg_update1(const ScgScalars *sc, double2 *r, const double2 *Ap, double2 *x, const double2 *p, int ns,
                          long len, double *parts, int nparts, cudaStream_t s) {
  k_scg_update1<<<nparts, 256, 0, s>>>(sc, r, Ap, x, p, ns, len, parts);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
rhmc_status_t scg_beta(ScgScalars *sc, const double *parts, int nparts, int ns, double tol, cudaStream_t s) {
  k_scg_beta<<<1, 256, 0, s>>>(sc, parts, nparts, ns, tol);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
rhmc_status_t scg_update2(const ScgScalars *sc, const double2 *r, double2 *p, int ns, long len, cudaStream_t s) {
  k_scg_update2<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(sc, r, p, ns, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
rhmc_status_t column(const double2 *in, double2 *out, long rows, int n, int j, int gather, cudaStream_t s) {
  k_column<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(in, out, rows, n, j, gather);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

}  // namespace rhmc
