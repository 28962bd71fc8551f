// Stored-basis assembly of the shifted solutions (mixed precision).
//
// Algorithm 1, lines 11-12, for a shift s: X^(s) += P^(s) alpha^(s)_k and
// P^(s) = Q_k + P^(s) M2_k, M2_k = beta^(s)_k rho_k^dagger, starting from
// P^(s)_0 = Q_0, X^(s) = 0.  Unrolled, P^(s)_k = sum_{i <= k} Q_i D_{i,k}
// with D_{k,k} = 1, D_{i,k} = M2_{i+1} ... M2_k, and after the shift's last
// update L:
//   X^(s) = sum_{i < L} Q_i C_i,   C_{L-1} = alpha_L,  C_i = alpha_{i+1} + M2_{i+1} C_{i+1}.
// So instead of updating P^(s) and X^(s) in HBM at every iteration, the solve
// keeps the block basis Q_0, Q_1, ... (FP32) and the n x n coefficients of
// every iteration (FP64), and forms all X^(s) at the end in one contraction
//   [rows x K 2n] . [K 2n x (nshift - 1) 2n]
// of real-embedded blocks (a plain GEMM, done by cuBLAS with FP32-accurate
// BF16x9 tensor-core emulation).  Only the base system keeps its recursion.
#include <cublas_v2.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

namespace {

// write z = C[q][j] of shift column block `colblk` into the real embedding
__device__ __forceinline__ void put_embedded(float *Ccat, long cols, long rowbase, int colbase, int q, int j,
                                             double2 z) {
  float *r0 = Ccat + (rowbase + 2 * q) * cols + colbase + 2 * j;
  float *r1 = r0 + cols;
  r0[0] = (float)z.x;   // (re, re) -> Re
  r0[1] = (float)z.y;   // (re, im) -> Im
  r1[0] = (float)-z.y;  // (im, re) -> -Im
  r1[1] = (float)z.x;   // (im, im) -> Re
}

}  // namespace

__global__ void __launch_bounds__(256) k_basis_coef(int n, int nshift, const SolverState *__restrict__ st,
                                                    const double2 *__restrict__ hist, int K, int want_p,
                                                    float *__restrict__ Ccat) {
  __shared__ double2 Cm[kMaxN * kMaxN], Tm[kMaxN * kMaxN];
  const int s = blockIdx.x + 1;
  if (s >= nshift) return;
  const int nn = n * n, t = threadIdx.x;
  const bool own = t < nn;
  const int qi = own ? t / n : 0, qj = own ? t % n : 0;
  const long cols = (long)(nshift - 1) * 2 * n;
  const int colbase = (s - 1) * 2 * n;
  const int nblk = want_p ? K + 1 : K;  // row blocks of Ccat
  // X: blocks i < last carry C_i; P: blocks i <= K carry D_i (active shifts only)
  int last = want_p ? (st->active[s] ? K : -1) : min(st->last_k[s], K);
  // blocks without a coefficient are zero
  for (int i = (want_p ? max(last + 1, 0) : max(last, 0)); i < nblk; ++i)
    if (own) put_embedded(Ccat, cols, (long)i * 2 * n, colbase, qi, qj, make_double2(0.0, 0.0));
  if (last < 0 || (!want_p && last == 0)) return;
  int i;
  if (want_p) {
    if (own) Cm[t] = make_double2(qi == qj ? 1.0 : 0.0, 0.0);  // D_K = 1
    i = K;
  } else {
    if (own) Cm[t] = hist[((size_t)last * nshift + s) * 2 * nn + t];  // C_{L-1} = alpha_L
    i = last - 1;
  }
  __syncthreads();
  for (;; --i) {
    if (own) put_embedded(Ccat, cols, (long)i * 2 * n, colbase, qi, qj, Cm[t]);
    if (i == 0) break;
    // step to block i - 1: C_{i-1} = alpha_i + M2_i C_i  /  D_{i-1} = M2_i D_i
    const double2 *h = hist + ((size_t)i * nshift + s) * 2 * nn;
    if (own) {
      double2 acc = want_p ? make_double2(0.0, 0.0) : h[t];
      const double2 *M2 = h + nn;
      for (int q = 0; q < n; ++q) {
        const double2 a = M2[qi * n + q], b = Cm[q * n + qj];
        acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
        acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
      }
      Tm[t] = acc;
    }
    __syncthreads();
    if (own) Cm[t] = Tm[t];
    __syncthreads();
  }
}

rhmc_status_t basis_coefficients(int n, int nshift, const SolverState *st, const double2 *hist, int K, int want_p,
                                 float *Ccat, cudaStream_t s) {
  if (nshift < 2) return RHMC_OK;
  prof_begin(PROF_NXN_SHIFTS, s);
  k_basis_coef<<<nshift - 1, 256, 0, s>>>(n, nshift, st, hist, K, want_p, Ccat);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// Q (rows x n) into column block k of the basis; k from kdev[slot] when kdev is given
// (graph replays), else the argument
__global__ void __launch_bounds__(256) k_basis_store(const float2 *__restrict__ Q, float2 *__restrict__ basis,
                                                     long rows, int n, int cap, int k, const int *kdev) {
  const int kb = kdev ? *kdev : k;
  if (kb < 0 || kb >= cap) return;
  const long len = rows * n;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (long)gridDim.x * blockDim.x) {
    const long r = e / n;
    const int j = (int)(e - r * n);
    basis[r * (long)cap * n + (long)kb * n + j] = Q[e];
  }
}

rhmc_status_t basis_store_dev(const float2 *Q, float2 *basis, long rows, int n, int cap, const int *kdev,
                              cudaStream_t s) {
  prof_begin(PROF_OTHER, s);
  k_basis_store<<<4 * 152, 256, 0, s>>>(Q, basis, rows, n, cap, 0, kdev);
  prof_end(s, (double)rows * n * sizeof(float2) * 2);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t basis_store(const float2 *Q, float2 *basis, long rows, int n, int cap, int k, cudaStream_t s) {
  prof_begin(PROF_OTHER, s);
  k_basis_store<<<4 * 152, 256, 0, s>>>(Q, basis, rows, n, cap, k, nullptr);
  prof_end(s, (double)rows * n * sizeof(float2) * 2);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// X^(s) += tmp block (FP64) or P^(s) = tmp block (FP32), shifts 1 .. nshift - 1
__global__ void __launch_bounds__(256) k_basis_scatter(const float2 *__restrict__ tmp, double2 *X, float2 *P,
                                                       long rows, int n, int nshift, long fstride) {
  const int m = (nshift - 1) * n;
  const long total = rows * m;
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const long r = e / m;
    const int c = (int)(e - r * m);
    const int s = 1 + c / n, j = c - (c / n) * n;
    const float2 v = tmp[e];
    const long o = s * fstride + r * n + j;
    if (X) {
      double2 x = X[o];
      x.x += (double)v.x;
      x.y += (double)v.y;
      X[o] = x;
    } else {
      P[o] = v;
    }
  }
}

rhmc_status_t basis_scatter(const float2 *tmp, double2 *X, float2 *P, long rows, int n, int nshift, long fstride,
                            cudaStream_t s) {
  if (nshift < 2) return RHMC_OK;
  prof_begin(PROF_OTHER, s);
  k_basis_scatter<<<4 * 152, 256, 0, s>>>(tmp, X, P, rows, n, nshift, fstride);
  prof_end(s, (double)rows * (nshift - 1) * n * (sizeof(float2) + (X ? 2 * sizeof(double2) : sizeof(float2))));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// tmp (rows x m, row-major, m = (nshift - 1) 2n reals) = basis (rows x nblk 2n, row stride
// cap 2n) . Ccat (nblk 2n x m, row-major).  Column-major view for cuBLAS:
// tmp^T (m x rows) = Ccat^T (m x nblk 2n) . basis^T (nblk 2n x rows).
rhmc_status_t basis_gemm(void *handle, const float2 *basis, const float *Ccat, float2 *tmp, long rows, int n,
                         int cap, int nblk, int nshift, int emulated, cudaStream_t s) {
  cublasHandle_t h = (cublasHandle_t)handle;
  const int m = (nshift - 1) * 2 * n, kk = nblk * 2 * n;
  if (rows > INT32_MAX || m <= 0 || kk <= 0) return RHMC_ERR_INVALID_ARG;
  if (cublasSetStream(h, s) != CUBLAS_STATUS_SUCCESS) {
    set_error("cublasSetStream failed");
    return RHMC_ERR_CUDA;
  }
  const float one = 1.0f, zero = 0.0f;
  prof_begin(PROF_OTHER, s);
  const cublasStatus_t st = cublasGemmEx(
      h, CUBLAS_OP_N, CUBLAS_OP_N, m, (int)rows, kk, &one, Ccat, CUDA_R_32F, m, basis, CUDA_R_32F, cap * 2 * n, &zero,
      tmp, CUDA_R_32F, m, emulated ? CUBLAS_COMPUTE_32F_EMULATED_16BFX9 : CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
  prof_end(s, (double)rows * (kk + m) * sizeof(float));
  if (st != CUBLAS_STATUS_SUCCESS) {
    set_error("cublasGemmEx (basis assembly) failed: status %d", (int)st);
    return RHMC_ERR_CUDA;
  }
  return RHMC_OK;
}

rhmc_status_t basis_handle_create(void **handle) {
  cublasHandle_t h = nullptr;
  if (cublasCreate(&h) != CUBLAS_STATUS_SUCCESS) {
    set_error("cublasCreate failed");
    return RHMC_ERR_CUDA;
  }
  *handle = h;
  return RHMC_OK;
}

void basis_handle_destroy(void *handle) {
  if (handle) cublasDestroy((cublasHandle_t)handle);
}

}  // namespace rhmc
