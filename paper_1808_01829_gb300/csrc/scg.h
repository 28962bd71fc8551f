// Per-vector FP64 multishift CG baseline: device scalars and launchers.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

struct ScgScalars {
  double rr, bb, rel;
  double alpha, alpha_prev, beta, beta_prev;
  double zeta[kMaxS], zeta_prev[kMaxS], zeta_next[kMaxS];
  double alpha_s[kMaxS], beta_s[kMaxS], pz[kMaxS], sigma[kMaxS];
  int active[kMaxS], upd[kMaxS];
  int breakdown;
};

rhmc_status_t scg_init(ScgScalars *sc, const double *parts, int nparts, int ns, const double *sigma_dev,
                       cudaStream_t s);
rhmc_status_t scg_alpha(ScgScalars *sc, const double *parts, int nparts, int ns, cudaStream_t s);
rhmc_status_t scg_update1(const ScgScalars *sc, double2 *r, const double2 *Ap, double2 *x, const double2 *p, int ns,
                          long len, double *parts, int nparts, cudaStream_t s);
rhmc_status_t scg_beta(ScgScalars *sc, const double *parts, int nparts, int ns, double tol, cudaStream_t s);
rhmc_status_t scg_update2(const ScgScalars *sc, const double2 *r, double2 *p, int ns, long len, cudaStream_t s);
rhmc_status_t column(const double2 *in, double2 *out, long rows, int n, int j, int gather, cudaStream_t s);

}  // namespace rhmc
