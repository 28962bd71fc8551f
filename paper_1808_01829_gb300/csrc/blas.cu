// Tall-skinny block kernels of SBCGrQ (Algorithm 1).  A block is a field
// [rows = 3 V/2][n] of complex numbers; every kernel here is a streaming pass
// over rows with an n x n coefficient matrix held in shared memory.
//
//   gram        G = A^dagger B (n x n), per-CTA partial sums in FP64
//               (lines 4-5: P^dagger (A + sigma_0) P and the Cholesky-QR Gram W^dagger W)
//   block_axpy  Y = C + A M (line 5: W = Q - (A + sigma_0) P alpha; also Q = R rho^-1)
//   update_all  Q = W rho^-1, then for every shift still being updated
//               X^(s) += P^(s) M1^(s),  P^(s) = Q + P^(s) M2^(s)
//               (lines 6-7 for s = 0 with M1 = alpha_k delta_{k-1}, M2 = rho_k^dagger;
//                lines 11-12 with M1 = alpha^(s)_k, M2 = beta^(s)_k rho_k^dagger)
//   flush       X64 += X32, X32 = 0 (mixed precision reliable-update flush)
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

// ------------------------------------------------------------ Gram partials
// G = A^dagger B.  Thread layout: BS x BS blocks of the n x n result (register
// blocking); the threads of one row group read each row's BS-wide chunks
// straight from global memory (the lanes that share a chunk are served by one
// L1 access), two rows in flight per thread.  FP32 products accumulate in FP32
// per thread; each CTA reduces its row groups in FP64, and the CTAs of a
// cluster of kGramCluster sum their partials through distributed shared memory
// in a fixed order, so one FP64 partial per cluster reaches global memory
// (deterministic).
constexpr int kGramCluster = 8;


template <typename T, int N, int BS>
__global__ void __launch_bounds__(256) k_gram(const C<T> *__restrict__ A, const C<T> *__restrict__ B, long rows,
                                              double2 *__restrict__ partial) {
  constexpr int NB = N / BS;
  constexpr int NBLK = NB * NB;   // threads per row group
  constexpr int RG = 256 / NBLK;  // row groups per CTA
  __shared__ double2 red[N * N];
  const int t = threadIdx.x;
  const int blk = t % NBLK, grp = t / NBLK;
  const int i0 = BS * (blk / NB), j0 = BS * (blk % NB);
  C<T> acc[BS][BS];
#pragma unroll
  for (int u = 0; u < BS; ++u)
#pragma unroll
    for (int v = 0; v < BS; ++v) acc[u][v] = czero<T>();
  if (grp < RG) {
    // rows of this row group: grp + RG * (blockIdx + gridDim * k), two at a time
    const long stride = (long)RG * gridDim.x;
    long r = (long)blockIdx.x * RG + grp;
    for (; r + stride < rows; r += 2 * stride) {
      C<T> a0[BS], b0[BS], a1[BS], b1[BS];
#pragma unroll
      for (int u = 0; u < BS; ++u) {
        a0[u] = A[r * N + i0 + u];
        b0[u] = B[r * N + j0 + u];
        a1[u] = A[(r + stride) * N + i0 + u];
        b1[u] = B[(r + stride) * N + j0 + u];
      }
#pragma unroll
      for (int u = 0; u < BS; ++u)
#pragma unroll
        for (int v = 0; v < BS; ++v) {
          cmac_cj<T>(acc[u][v], a0[u], b0[v]);
          cmac_cj<T>(acc[u][v], a1[u], b1[v]);
        }
    }
    if (r < rows) {
      C<T> a0[BS], b0[BS];
#pragma unroll
      for (int u = 0; u < BS; ++u) {
        a0[u] = A[r * N + i0 + u];
        b0[u] = B[r * N + j0 + u];
      }
#pragma unroll
      for (int u = 0; u < BS; ++u)
#pragma unroll
        for (int v = 0; v < BS; ++v) cmac_cj<T>(acc[u][v], a0[u], b0[v]);
    }
  }
  // reduce the row groups in FP64 into red[N*N]
  for (int k = t; k < N * N; k += 256) red[k] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int g = 0; g < RG; ++g) {
    if (grp == g) {
#pragma unroll
      for (int u = 0; u < BS; ++u)
#pragma unroll
        for (int v = 0; v < BS; ++v) {
          double2 &d = red[(i0 + u) * N + j0 + v];
          d.x += (double)acc[u][v].x;
          d.y += (double)acc[u][v].y;
        }
    }
    __syncthreads();
  }
  // cluster reduction through distributed shared memory, fixed order
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  cl.sync();
  if (cl.block_rank() == 0) {
    for (int k = t; k < N * N; k += 256) {
      double2 sum = red[k];
      for (unsigned q = 1; q < cl.num_blocks(); ++q) {
        const double2 *rem = cl.map_shared_rank(red, q);
        sum.x += rem[k].x;
        sum.y += rem[k].y;
      }
      partial[(long)(blockIdx.x / cl.num_blocks()) * N * N + k] = sum;
    }
  }
  cl.sync();
}

// ------------------------------------------------------------ Y = C + A M
// One thread per row; M (n x n) in shared memory.  TA: type of A, TC: type
// of C, TY: type of Y (conversion between precisions happens here).
template <typename TA, typename TY, int N>
__global__ void __launch_bounds__(256) k_block_axpy(const C<TA> *__restrict__ Ain, const C<TY> *__restrict__ Cin,
                                                    const C<TA> *__restrict__ M, C<TY> *__restrict__ Y, long rows) {
  __shared__ C<TA> sm[N * N];
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) sm[k] = M[k];
  __syncthreads();
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  C<TA> a[N];
#pragma unroll
  for (int k = 0; k < N; ++k) a[k] = Ain[r * N + k];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    C<TA> acc = czero<TA>();
#pragma unroll
    for (int k = 0; k < N; ++k) cmac<TA>(acc, a[k], sm[k * N + j]);
    if (Cin) {
      const C<TY> c = Cin[r * N + j];
      Y[r * N + j] = mk<TY>((TY)(c.x + acc.x), (TY)(c.y + acc.y));
    } else {
      Y[r * N + j] = mk<TY>((TY)acc.x, (TY)acc.y);
    }
  }
}

// ------------------------------------------------------------ fused all-shift update
// Whole-row loads: 16-byte vector loads when the row is 16-byte aligned.
template <typename T, int N> struct Row {
  __device__ static void load(const C<T> *src, C<T> *dst) {
    constexpr int PER16 = 16 / (int)sizeof(C<T>);  // complex numbers per 16 bytes
    if (N % PER16 == 0) {
      const float4 *v = reinterpret_cast<const float4 *>(src);
#pragma unroll
      for (int q = 0; q < N / PER16; ++q) {
        const float4 w = v[q];
        if (PER16 == 2) {
          reinterpret_cast<float2 *>(dst)[2 * q] = make_float2(w.x, w.y);
          reinterpret_cast<float2 *>(dst)[2 * q + 1] = make_float2(w.z, w.w);
        } else {
          reinterpret_cast<float4 *>(dst)[q] = w;
        }
      }
    } else {
#pragma unroll
      for (int k = 0; k < N; ++k) dst[k] = src[k];
    }
  }
};

// coef layout (type C<T>): [0, N*N) rho^-1; then for s: M1^(s) at (1+2s)*N*N,
// M2^(s) at (2+2s)*N*N.  upd[s] != 0 selects the shifts updated this iteration.
// X^(s) is of type TX (FP64 in the FP64 solver, FP32 partial sums in the mixed
// one).
//
// Layout: CG output columns per thread, N / CG threads per row (consecutive
// lanes of one warp; a row never straddles two warps), persistent grid-stride
// loop over rows.  All coefficient
// matrices stay in shared memory for the whole launch.  A thread keeps the
// full P^(s) row in registers; the lanes of a row finish reading it
// (__syncwarp) before any of them overwrites its columns.
template <typename T, typename TX, int N, int CG>
__global__ void __launch_bounds__(256) k_update_all(const C<T> *__restrict__ W, C<T> *__restrict__ Q,
                                                    C<T> *__restrict__ P, TX *__restrict__ Xv,
                                                    const C<T> *__restrict__ coef, const int *__restrict__ upd,
                                                    int s_begin, int s_end, int compute_q, long rows, long fstride) {
  constexpr int TPR = N / CG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T> *sc = reinterpret_cast<C<T> *>(smem_raw);  // rho^-1 (if compute_q), then the pairs of [s_begin, s_end)
  __shared__ int supd[kMaxS];
  const int c0 = compute_q ? 0 : (1 + 2 * s_begin) * N * N;  // first coefficient staged
  const int ncoef = (1 + 2 * s_end) * N * N - c0;
  for (int k = threadIdx.x; k < ncoef; k += blockDim.x) sc[k] = coef[c0 + k];
  for (int k = threadIdx.x; k < s_end; k += blockDim.x) supd[k] = upd[k];
  __syncthreads();
  using CX = C<TX>;
  CX *X = reinterpret_cast<CX *>(Xv);
  // rows never straddle a warp: 32 / TPR rows per warp, remaining lanes idle
  constexpr int RPW = 32 / TPR;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / TPR;
  const int j0 = (lane - slot * TPR) * CG;
  const long rows_per_cta = (long)(blockDim.x >> 5) * RPW;
  for (long rbase = (long)blockIdx.x * rows_per_cta; rbase < rows; rbase += (long)gridDim.x * rows_per_cta) {
    const long r = rbase + (long)warp * RPW + slot;
    const bool live = slot < RPW && r < rows;
    // Q row slice = W row rho^-1  (rho^-1 is upper triangular), or read it
    C<T> q[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) q[c] = czero<T>();
    if (live) {
      if (compute_q) {
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const C<T> w = W[r * N + k];
#pragma unroll
          for (int c = 0; c < CG; ++c)
            if (k <= j0 + c) cmac<T>(q[c], w, sc[k * N + j0 + c]);
        }
#pragma unroll
        for (int c = 0; c < CG; ++c) Q[r * N + j0 + c] = q[c];
      } else {
#pragma unroll
        for (int c = 0; c < CG; ++c) q[c] = Q[r * N + j0 + c];
      }
    }
    for (int s = s_begin; s < s_end; ++s) {
      if (!supd[s]) continue;
      const C<T> *m1 = sc + (1 + 2 * s) * N * N - c0;
      const C<T> *m2 = m1 + N * N;
      C<T> *Ps = P + s * fstride;
      C<T> p[N];
      if (live) Row<T, N>::load(Ps + r * N, p);
      __syncwarp();
      if (live) {
        C<T> a1[CG], a2[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) {
          a1[c] = czero<T>();
          a2[c] = czero<T>();
        }
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
          for (int c = 0; c < CG; ++c) {
            cmac<T>(a1[c], p[k], m1[k * N + j0 + c]);
            cmac<T>(a2[c], p[k], m2[k * N + j0 + c]);
          }
        CX *Xs = X + s * fstride + r * N + j0;
#pragma unroll
        for (int c = 0; c < CG; ++c) {
          CX x = Xs[c];
          x.x += a1[c].x;
          x.y += a1[c].y;
          Xs[c] = x;
          Ps[r * N + j0 + c] = mk<T>(q[c].x + a2[c].x, q[c].y + a2[c].y);
        }
      }
      __syncwarp();
    }
  }
}

// ------------------------------------------------------------ flush
__global__ void k_flush(double2 *__restrict__ X64, float2 *__restrict__ X32, long len) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const float2 a = X32[i];
  double2 b = X64[i];
  b.x += (double)a.x;
  b.y += (double)a.y;
  X64[i] = b;
  X32[i] = make_float2(0.f, 0.f);
}

// ------------------------------------------------------------ misc elementwise
template <typename TI, typename TO>
__global__ void k_convert(const C<TI> *__restrict__ in, C<TO> *__restrict__ out, long len) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const C<TI> z = in[i];
  out[i] = mk<TO>((TO)z.x, (TO)z.y);
}

// out = a - b (FP64)
__global__ void k_sub(const double2 *__restrict__ a, const double2 *__restrict__ b, double2 *__restrict__ out,
                      long len) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  out[i] = make_double2(a[i].x - b[i].x, a[i].y - b[i].y);
}

// a += b (FP64)
__global__ void k_add(double2 *__restrict__ a, const double2 *__restrict__ b, long len) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  a[i] = make_double2(a[i].x + b[i].x, a[i].y + b[i].y);
}

// Per-column sums of |A|^2 (n columns) and Re sum conj(A) B, partials per CTA.
template <typename T>
__global__ void __launch_bounds__(256) k_colnorm2(const C<T> *__restrict__ A, long rows, int n,
                                                  double *__restrict__ partial) {
  __shared__ double red[256];
  const int t = threadIdx.x;
  // thread t handles column t % n of rows (t / n) + k * (256 / n)
  const int per = 256 / n;
  const int c = t % n, g = t / n;
  double acc = 0.0;
  if (g < per)
    for (long r = (long)blockIdx.x * per + g; r < rows; r += (long)gridDim.x * per) {
      const C<T> z = A[r * n + c];
      acc += (double)z.x * z.x + (double)z.y * z.y;
    }
  red[t] = (g < per) ? acc : 0.0;
  __syncthreads();
  if (t < n) {
    double s = 0.0;
    for (int q = 0; q < per; ++q) s += red[q * n + t];
    partial[(long)blockIdx.x * n + t] = s;
  }
}

__global__ void __launch_bounds__(256) k_redot(const double2 *__restrict__ A, const double2 *__restrict__ B, long len,
                                               double *__restrict__ partial) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (long)gridDim.x * blockDim.x)
    acc += A[i].x * B[i].x + A[i].y * B[i].y;
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

// ------------------------------------------------------------ launchers
#define RHMC_DISPATCH_N(n, MACRO) \
  switch (n) {                    \
    case 1: MACRO(1); break;      \
    case 2: MACRO(2); break;      \
    case 3: MACRO(3); break;      \
    case 4: MACRO(4); break;      \
    case 5: MACRO(5); break;      \
    case 6: MACRO(6); break;      \
    case 7: MACRO(7); break;      \
    case 8: MACRO(8); break;      \
    case 9: MACRO(9); break;      \
    case 10: MACRO(10); break;    \
    case 11: MACRO(11); break;    \
    case 12: MACRO(12); break;    \
    case 13: MACRO(13); break;    \
    case 14: MACRO(14); break;    \
    case 15: MACRO(15); break;    \
    case 16: MACRO(16); break;    \
    default: return RHMC_ERR_INVALID_ARG; \
  }

template <typename T, int N>
static cudaError_t launch_gram(const C<T> *A, const C<T> *B, long rows, double2 *partial, int nparts,
                               cudaStream_t s) {
  constexpr int BS = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nparts * kGramCluster);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = kGramCluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_gram<T, N, BS>, A, B, rows, partial);
}

// nparts: number of FP64 partial n x n sums written (one per cluster of CTAs).
template <typename T>
rhmc_status_t gram(const C<T> *A, const C<T> *B, long rows, int n, double2 *partial, int nparts, cudaStream_t s) {
  prof_begin(sizeof(T) == 4 ? PROF_GRAM32 : PROF_GRAM64, s);
  cudaError_t e = cudaSuccess;
#define L_GRAM(NN) e = launch_gram<T, NN>(A, B, rows, partial, nparts, s)
  RHMC_DISPATCH_N(n, L_GRAM)
#undef L_GRAM
  if (e != cudaSuccess) {
    set_error("gram launch: %s", cudaGetErrorString(e));
    return RHMC_ERR_CUDA;
  }
  prof_end(s, (double)rows * n * sizeof(C<T>) * (A == B ? 1 : 2));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t gram<float>(const float2 *, const float2 *, long, int, double2 *, int, cudaStream_t);
template rhmc_status_t gram<double>(const double2 *, const double2 *, long, int, double2 *, int, cudaStream_t);

template <typename TA, typename TY>
rhmc_status_t block_axpy(const C<TA> *A, const C<TY> *Cin, const C<TA> *M, C<TY> *Y, long rows, int n,
                         cudaStream_t s) {
  const int bs = 128;
  const long grid = (rows + bs - 1) / bs;
  prof_begin(PROF_AXPY, s);
#define L_AXPY(NN) k_block_axpy<TA, TY, NN><<<grid, bs, 0, s>>>(A, Cin, M, Y, rows)
  RHMC_DISPATCH_N(n, L_AXPY)
#undef L_AXPY
  prof_end(s, (double)rows * n * (sizeof(C<TA>) + sizeof(C<TY>) * (Cin ? 2 : 1)));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t block_axpy<float, float>(const float2 *, const float2 *, const float2 *, float2 *, long, int,
                                                cudaStream_t);
template rhmc_status_t block_axpy<double, double>(const double2 *, const double2 *, const double2 *, double2 *, long,
                                                  int, cudaStream_t);
template rhmc_status_t block_axpy<double, float>(const double2 *, const float2 *, const double2 *, float2 *, long,
                                                 int, cudaStream_t);

template <typename T, typename TX, int N>
static void launch_update(const C<T> *W, C<T> *Q, C<T> *P, C<TX> *X, const C<T> *coef, const int *upd, int s_begin,
                          int s_end, int compute_q, long rows, long fstride, cudaStream_t s) {
  constexpr int CG = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 1);
  const size_t smem = (size_t)((1 + 2 * s_end) - (compute_q ? 0 : 1 + 2 * s_begin)) * N * N * sizeof(C<T>);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_update_all<T, TX, N, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    attr = true;
  }
  int threads = tune_get(TUNE_UPDATE_THREADS);
  if (threads <= 0 || threads > 1024 || threads % 32) threads = 256;
  const long rows_per_cta = (long)(threads / 32) * (32 / (N / CG));
  long grid = (rows + rows_per_cta - 1) / rows_per_cta;
  grid = std::min(grid, (long)(8 * 152));
  k_update_all<T, TX, N, CG><<<(unsigned)grid, threads, smem, s>>>(W, Q, P, reinterpret_cast<TX *>(X), coef, upd,
                                                                   s_begin, s_end, compute_q, rows, fstride);
}

template <typename T, typename TX>
rhmc_status_t update_all(const C<T> *W, C<T> *Q, C<T> *P, C<TX> *X, const C<T> *coef, const int *upd, int s_begin,
                         int s_end, int compute_q, long rows, int n, long fstride, cudaStream_t s) {
  if ((size_t)(1 + 2 * s_end) * n * n * sizeof(C<T>) > 220 * 1024) {
    set_error("update_all: %d shifts at n = %d exceed the shared-memory coefficient store", s_end, n);
    return RHMC_ERR_INVALID_ARG;
  }
  int nupd = s_end - s_begin;
  if (prof_on()) {  // profiling only: count the shifts this launch updates (host sync)
    int h[kMaxS];
    cudaStreamSynchronize(s);
    cudaMemcpy(h, upd, sizeof(int) * s_end, cudaMemcpyDeviceToHost);
    nupd = 0;
    for (int q = s_begin; q < s_end; ++q) nupd += h[q] != 0;
  }
  prof_begin(sizeof(T) == 4 ? PROF_UPDATE32 : PROF_UPDATE64, s);
#define L_UPD(NN) launch_update<T, TX, NN>(W, Q, P, X, coef, upd, s_begin, s_end, compute_q, rows, fstride, s)
  RHMC_DISPATCH_N(n, L_UPD)
#undef L_UPD
  prof_end(s, (double)rows * n * ((compute_q ? 2.0 : 1.0) * sizeof(C<T>) + nupd * 2.0 * (sizeof(C<T>) + sizeof(C<TX>))));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t update_all<float, float>(const float2 *, float2 *, float2 *, float2 *, const float2 *,
                                                const int *, int, int, int, long, int, long, cudaStream_t);
template rhmc_status_t update_all<double, double>(const double2 *, double2 *, double2 *, double2 *, const double2 *,
                                                  const int *, int, int, int, long, int, long, cudaStream_t);

rhmc_status_t flush(double2 *X64, float2 *X32, long len, cudaStream_t s) {
  const int bs = 256;
  k_flush<<<(unsigned)((len + bs - 1) / bs), bs, 0, s>>>(X64, X32, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

template <typename TI, typename TO>
rhmc_status_t convert(const C<TI> *in, C<TO> *out, long len, cudaStream_t s) {
  const int bs = 256;
  k_convert<TI, TO><<<(unsigned)((len + bs - 1) / bs), bs, 0, s>>>(in, out, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t convert<double, float>(const double2 *, float2 *, long, cudaStream_t);
template rhmc_status_t convert<float, double>(const float2 *, double2 *, long, cudaStream_t);

rhmc_status_t sub(const double2 *a, const double2 *b, double2 *out, long len, cudaStream_t s) {
  const int bs = 256;
  k_sub<<<(unsigned)((len + bs - 1) / bs), bs, 0, s>>>(a, b, out, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t add_inplace(double2 *a, const double2 *b, long len, cudaStream_t s) {
  const int bs = 256;
  k_add<<<(unsigned)((len + bs - 1) / bs), bs, 0, s>>>(a, b, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

template <typename T>
rhmc_status_t colnorm2(const C<T> *A, long rows, int n, double *partial, int nparts, cudaStream_t s) {
  k_colnorm2<T><<<nparts, 256, 0, s>>>(A, rows, n, partial);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t colnorm2<double>(const double2 *, long, int, double *, int, cudaStream_t);
template rhmc_status_t colnorm2<float>(const float2 *, long, int, double *, int, cudaStream_t);

rhmc_status_t redot(const double2 *A, const double2 *B, long len, double *partial, int nparts, cudaStream_t s) {
  k_redot<<<nparts, 256, 0, s>>>(A, B, len, partial);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

}  // namespace rhmc
