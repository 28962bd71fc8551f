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
#include "common.cuh"
#include "kernels.h"

namespace rhmc {

// ------------------------------------------------------------ Gram partials
// Thread layout: (ib, jb) 2x2 blocks of the n x n result, `rg` row groups.
// Rows are staged through shared memory in tiles of TR rows.
template <typename T, int N>
__global__ void __launch_bounds__(256) k_gram(const C<T> *__restrict__ A, const C<T> *__restrict__ B, long rows,
                                              double2 *__restrict__ partial) {
  constexpr int NB = (N + 1) / 2;
  constexpr int NBLK = NB * NB;
  constexpr int RG = 256 / NBLK;
  constexpr int TR = 64;
  __shared__ C<T> sa[TR][N + 1], sb[TR][N + 1];
  __shared__ double2 red[256];
  const int t = threadIdx.x;
  const int blk = t % NBLK, grp = t / NBLK;
  const int i0 = 2 * (blk / NB), j0 = 2 * (blk % NB);
  C<T> acc[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) acc[u][v] = czero<T>();
  const long per = (rows + gridDim.x - 1) / gridDim.x;
  const long r0 = (long)blockIdx.x * per;
  const long r1 = min(rows, r0 + per);
  for (long rt = r0; rt < r1; rt += TR) {
    const int nr = (int)min((long)TR, r1 - rt);
    __syncthreads();
    for (int k = t; k < nr * N; k += 256) {
      const int r = k / N, c = k - r * N;
      sa[r][c] = A[(rt + r) * N + c];
      sb[r][c] = B[(rt + r) * N + c];
    }
    __syncthreads();
    if (grp < RG) {
      for (int r = grp; r < nr; r += RG) {
        const C<T> a0 = sa[r][i0], b0 = sb[r][j0];
        const C<T> a1 = (i0 + 1 < N) ? sa[r][i0 + 1] : czero<T>();
        const C<T> b1 = (j0 + 1 < N) ? sb[r][j0 + 1] : czero<T>();
        cmac_cj<T>(acc[0][0], a0, b0);
        cmac_cj<T>(acc[0][1], a0, b1);
        cmac_cj<T>(acc[1][0], a1, b0);
        cmac_cj<T>(acc[1][1], a1, b1);
      }
    }
  }
  // reduce over row groups in FP64
  double2 *out = partial + (long)blockIdx.x * N * N;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      __syncthreads();
      red[t] = make_double2((double)acc[u][v].x, (double)acc[u][v].y);
      __syncthreads();
      if (t < NBLK) {
        double2 s = red[t];
        for (int q = 1; q < RG; ++q) {
          s.x += red[t + q * NBLK].x;
          s.y += red[t + q * NBLK].y;
        }
        const int i = i0 + u, j = j0 + v;
        if (i < N && j < N) out[i * N + j] = s;
      }
    }
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
// coef layout (type C<T>): [0, N*N) rho^-1; then for s: M1^(s) at (1+2s)*N*N,
// M2^(s) at (2+2s)*N*N.  upd[s] != 0 selects the shifts updated this iteration.
// X^(s) is of type TX (FP64 in the FP64 solver, FP32 partial sums in the mixed
// one).  The coefficient pair of one shift at a time sits in shared memory.
template <typename T, typename TX, int N>
__global__ void __launch_bounds__(128) k_update_all(const C<T> *__restrict__ W, C<T> *__restrict__ Q,
                                                    C<T> *__restrict__ P, TX *__restrict__ Xv,
                                                    const C<T> *__restrict__ coef, const int *__restrict__ upd,
                                                    int nshift, long rows, long fstride) {
  __shared__ C<T> sr[N * N], s1[N * N], s2[N * N];
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) sr[k] = coef[k];
  __syncthreads();
  const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = r < rows;
  using CX = C<TX>;
  CX *X = reinterpret_cast<CX *>(Xv);
  // Q row = W row rho^-1  (rho^-1 is upper triangular)
  C<T> q[N];
  if (live) {
    C<T> w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = W[r * N + k];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      C<T> acc = czero<T>();
#pragma unroll
      for (int k = 0; k <= j; ++k) cmac<T>(acc, w[k], sr[k * N + j]);
      q[j] = acc;
      Q[r * N + j] = acc;
    }
  }
  for (int s = 0; s < nshift; ++s) {
    if (!upd[s]) continue;  // uniform across the CTA
    __syncthreads();
    for (int k = threadIdx.x; k < N * N; k += blockDim.x) {
      s1[k] = coef[(1 + 2 * s) * N * N + k];
      s2[k] = coef[(2 + 2 * s) * N * N + k];
    }
    __syncthreads();
    if (!live) continue;
    C<T> p[N];
    C<T> *Ps = P + s * fstride + r * N;
    CX *Xs = X + s * fstride + r * N;
#pragma unroll
    for (int k = 0; k < N; ++k) p[k] = Ps[k];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      C<T> a1 = czero<T>(), a2 = czero<T>();
#pragma unroll
      for (int k = 0; k < N; ++k) {
        cmac<T>(a1, p[k], s1[k * N + j]);
        cmac<T>(a2, p[k], s2[k * N + j]);
      }
      CX x = Xs[j];
      x.x += a1.x;
      x.y += a1.y;
      Xs[j] = x;
      Ps[j] = mk<T>(q[j].x + a2.x, q[j].y + a2.y);
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

template <typename T>
rhmc_status_t gram(const C<T> *A, const C<T> *B, long rows, int n, double2 *partial, int nparts, cudaStream_t s) {
  prof_begin(sizeof(T) == 4 ? PROF_GRAM32 : PROF_GRAM64, s);
#define L_GRAM(NN) k_gram<T, NN><<<nparts, 256, 0, s>>>(A, B, rows, partial)
  RHMC_DISPATCH_N(n, L_GRAM)
#undef L_GRAM
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

template <typename T, typename TX>
rhmc_status_t update_all(const C<T> *W, C<T> *Q, C<T> *P, C<TX> *X, const C<T> *coef, const int *upd, int nshift,
                         long rows, int n, long fstride, cudaStream_t s) {
  const int bs = 128;
  const long grid = (rows + bs - 1) / bs;
#define L_UPD(NN)                                                                                     \
  k_update_all<T, TX, NN><<<grid, bs, 0, s>>>(W, Q, P, reinterpret_cast<TX *>(X), coef, upd, nshift, rows, \
                                              fstride)
  int nupd = nshift;
  if (prof_on()) {  // profiling only: count the shifts this launch updates (host sync)
    int h[kMaxS];
    cudaMemcpy(h, upd, sizeof(int) * nshift, cudaMemcpyDeviceToHost);
    nupd = 0;
    for (int q = 0; q < nshift; ++q) nupd += h[q] != 0;
  }
  prof_begin(sizeof(T) == 4 ? PROF_UPDATE32 : PROF_UPDATE64, s);
  RHMC_DISPATCH_N(n, L_UPD)
#undef L_UPD
  prof_end(s, (double)rows * n * (2.0 * sizeof(C<T>) + nupd * 2.0 * (sizeof(C<T>) + sizeof(C<TX>))));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t update_all<float, float>(const float2 *, float2 *, float2 *, float2 *, const float2 *,
                                                const int *, int, long, int, long, cudaStream_t);
template rhmc_status_t update_all<double, double>(const double2 *, double2 *, double2 *, double2 *, const double2 *,
                                                  const int *, int, long, int, long, cudaStream_t);

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
