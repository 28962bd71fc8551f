// Tall-skinny block kernels of SBCGrQ (Algorithm 1).  A block is a field
// [rows = 3 V/2][n] of complex numbers; every kernel here is a streaming pass
// over rows with an n x n coefficient matrix held in shared memory.
//
//   gram        G = A^dagger B (n x n), per-CTA partial sums in FP64
//               (P^dagger (A + sigma_0) P of the alpha_k step, the Cholesky-QR Gram W^dagger W)
//   block_axpy  Y = C + A M (block QR: W = Q - (A + sigma_0) P alpha; also Q = R rho^-1)
//   update_all  Q = W rho^-1, then for every shift still being updated
//               X^(s) += P^(s) M1^(s),  P^(s) = Q + P^(s) M2^(s)
//               (base updates for s = 0 with M1 = alpha_k delta_{k-1}, M2 = rho_k^dagger;
//                shifted updates with M1 = alpha^(s)_k, M2 = beta^(s)_k rho_k^dagger)
//   flush       X64 += X32, X32 = 0 (mixed precision reliable-update flush)
#include <algorithm>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

// Instantiate a launch for the runtime width n = 1..16.
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


// ------------------------------------------------------------ packed FP32x2 helpers
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long v) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
  return make_float2(lo, hi);
}
// d = a * b + c on two FP32 lanes at once (one rounding per lane)
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// ------------------------------------------------------------ Gram
// G = A^dagger B (n x n), summed over all rows, in two launches:
//   k_gram      every warp streams its own 16-row tiles of A and B through a
//               private double buffer in shared memory (cp.async, only warp
//               synchronisation); each lane owns n*n/32 entries of G and
//               accumulates them in FP32; the CTA sums its warps in FP64 and
//               writes one partial per entry, transposed ([entry][CTA]);
//   k_gram_sum  one CTA per entry sums the partials in a fixed order (FP64),
//               so the result is deterministic.
// For n = 16 lane L owns row i = L/2 of G and 8 consecutive columns, so a row
// of the tile costs one 8-byte and four 16-byte shared loads per 8 complex MACs.
constexpr int kGramTileRows = 16;
constexpr int kGramWarps = 8;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// PK (FP32, n = 16): packed FP32x2 FMAs, conj(a) b from the duplicated pairs
// (a.re, a.re), (a.im, a.im) times the (re, im) pair of b as loaded.  Every use
// of the Gram matrix here is Hermitian (P^dagger (A + sigma) P, W^dagger W,
// B^dagger B), so the packed form computes one circulant half: lane pair i
// forms G[i][(i + o) mod 16] for o = 0 .. 8 (5 entries per lane instead of 8)
// and the CTA reduction writes the rest as conjugates.
template <typename T, int N, bool SAME, bool PK, int TR = kGramTileRows, int WG = kGramWarps>
__global__ void __launch_bounds__(WG * 32) k_gram(const C<T> *__restrict__ A, const C<T> *__restrict__ B, long rows,
                                                  double2 *__restrict__ partial) {
  constexpr int TE = TR * N;  // complex per tile and operand
  constexpr int E = (N * N + 31) / 32;   // entries per lane
  constexpr bool STRUCT = (N == 16);
  constexpr bool PACKED = PK && STRUCT && sizeof(T) == 4;
  constexpr int NQ = 5;  // circulant entries per lane (packed form)
  unsigned long long p1[PACKED ? NQ : 1], p2[PACKED ? NQ : 1];  // (sum a.re b.re, a.re b.im), (a.im b.re, a.im b.im)
#pragma unroll
  for (int q = 0; q < (PACKED ? NQ : 1); ++q) p1[q] = p2[q] = 0ull;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int STAGE = (SAME ? 1 : 2) * TE;  // complex per pipeline stage
  C<T> *ws = reinterpret_cast<C<T> *>(smem_raw) + (size_t)warp * 2 * STAGE;
  auto sa = [&](int st) { return ws + st * STAGE; };
  auto sb = [&](int st) { return SAME ? ws + st * STAGE : ws + st * STAGE + TE; };
  C<T> acc[E];
#pragma unroll
  for (int q = 0; q < E; ++q) acc[q] = czero<T>();
  const long ntiles = (rows + TR - 1) / TR;
  const long wstride = (long)gridDim.x * WG;
  long tile = (long)blockIdx.x * WG + warp;
  auto issue = [&](long tl, int st) {
    const long r0 = tl * TR;
    const int nr = (int)min((long)TR, rows - r0);
    if (nr == TR) {
      constexpr int NV = (int)(TE * sizeof(C<T>) / 16);
      const char *ga = reinterpret_cast<const char *>(A + r0 * N);
      const char *gb = reinterpret_cast<const char *>(B + r0 * N);
      for (int k = lane; k < NV; k += 32) {
        cp_async16(reinterpret_cast<char *>(sa(st)) + 16 * k, ga + 16 * k);
        if (!SAME) cp_async16(reinterpret_cast<char *>(sb(st)) + 16 * k, gb + 16 * k);
      }
    } else {  // ragged last tile: plain loads, zero fill
      for (int k = lane; k < TE; k += 32) {
        const bool in = k < nr * N;
        sa(st)[k] = in ? A[r0 * N + k] : czero<T>();
        if (!SAME) sb(st)[k] = in ? B[r0 * N + k] : czero<T>();
      }
    }
    cp_async_commit();
  };
  int st = 0;
  if (tile < ntiles) issue(tile, 0);
  for (; tile < ntiles; tile += wstride) {
    if (tile + wstride < ntiles)
      issue(tile + wstride, st ^ 1);
    else
      cp_async_commit();
    cp_async_wait1();
    __syncwarp();
    const C<T> *ta = sa(st), *tb = sb(st);
    if constexpr (PACKED) {
      // lane pair i: offsets o = 5 h + q (h = lane & 1; o = 9 is computed and dropped)
      const int i = lane >> 1, o0 = (lane & 1) * NQ;
#pragma unroll 4
      for (int r = 0; r < TR; ++r) {
        const float2 a = *reinterpret_cast<const float2 *>(ta + r * N + i);
        const unsigned long long axx = pack2(a.x, a.x), ayy = pack2(a.y, a.y);
        const unsigned long long *br = reinterpret_cast<const unsigned long long *>(tb + r * N);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const unsigned long long bv = br[(i + o0 + q) & (N - 1)];
          p1[q] = fma2(axx, bv, p1[q]);
          p2[q] = fma2(ayy, bv, p2[q]);
        }
      }
    } else if (STRUCT) {
      const int i = lane >> 1, j0 = (lane & 1) * 8;
#pragma unroll 4
      for (int r = 0; r < TR; ++r) {
        const C<T> a = ta[r * N + i];
        C<T> b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = tb[r * N + j0 + q];
#pragma unroll
        for (int q = 0; q < 8; ++q) cmac_cj<T>(acc[q], a, b[q]);
      }
    } else {
#pragma unroll 4
      for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int q = 0; q < E; ++q) {
          const int e = lane + 32 * q;
          if (e < N * N) cmac_cj<T>(acc[q], ta[r * N + e / N], tb[r * N + e % N]);
        }
    }
    __syncwarp();
    st ^= 1;
  }
  cp_async_wait0();
  __syncthreads();
  // CTA reduction in FP64 (reuses the tile buffers), then one partial per entry
  double2 *red = reinterpret_cast<double2 *>(smem_raw);  // [WG][N*N]
  if constexpr (PACKED) {
    const int i = lane >> 1, o0 = (lane & 1) * NQ;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int o = o0 + q;
      if (o > N / 2) continue;
      const float2 u = unpack2(p1[q]), v = unpack2(p2[q]);
      const double gx = (double)(u.x + v.y), gy = (double)(u.y - v.x);
      const int j = (i + o) & (N - 1);
      red[warp * N * N + i * N + j] = make_double2(gx, gy);
      if (o > 0 && 2 * o != N) red[warp * N * N + j * N + i] = make_double2(gx, -gy);
    }
  } else {
#pragma unroll
    for (int q = 0; q < E; ++q) {
      const int e = STRUCT ? (lane >> 1) * N + (lane & 1) * 8 + q : lane + 32 * q;
      if (e < N * N) red[warp * N * N + e] = make_double2((double)acc[q].x, (double)acc[q].y);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    double2 sum = red[e];
    for (int w = 1; w < WG; ++w) {
      sum.x += red[w * N * N + e].x;
      sum.y += red[w * N * N + e].y;
    }
    partial[(long)e * gridDim.x + blockIdx.x] = sum;
  }
}

// out[e] = sum over the nparts partials of entry e, fixed order.
__global__ void __launch_bounds__(128) k_gram_sum(const double2 *__restrict__ partial, int nparts,
                                                  double2 *__restrict__ out) {
  __shared__ double2 red[128];
  const int e = blockIdx.x;
  double2 s = make_double2(0.0, 0.0);
  for (int p = threadIdx.x; p < nparts; p += blockDim.x) {
    const double2 v = partial[(long)e * nparts + p];
    s.x += v.x;
    s.y += v.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      red[threadIdx.x].x += red[threadIdx.x + w].x;
      red[threadIdx.x].y += red[threadIdx.x + w].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[e] = red[0];
}

// Whole-row loads: 16-byte vector loads when the row is 16-byte aligned.
// A lane's slice of CG consecutive complex numbers (32-byte aligned for FP32
// complex with CG = 4): 16-byte vector accesses where the type allows.
template <typename T, int CG> __device__ __forceinline__ void ld_slice(const C<T> *p, C<T> *v) {
  if constexpr (sizeof(C<T>) == 8 && CG % 2 == 0) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int i = 0; i < CG / 2; ++i) {
      const float4 w = q[i];
      v[2 * i] = mk<T>(w.x, w.y);
      v[2 * i + 1] = mk<T>(w.z, w.w);
    }
  } else {
#pragma unroll
    for (int c = 0; c < CG; ++c) v[c] = p[c];
  }
}
template <typename T, int CG> __device__ __forceinline__ void st_slice(C<T> *p, const C<T> *v) {
  if constexpr (sizeof(C<T>) == 8 && CG % 2 == 0) {
    float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int i = 0; i < CG / 2; ++i) q[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
  } else {
#pragma unroll
    for (int c = 0; c < CG; ++c) p[c] = v[c];
  }
}

template <typename T, int N> struct Row {
  __device__ static void load(const C<T> *src, C<T> *dst) {
    if (sizeof(C<T>) == 8 && N % 2 == 0) {  // FP32 complex: two per 16-byte load
      const float4 *v = reinterpret_cast<const float4 *>(src);
#pragma unroll
      for (int q = 0; q < N / 2; ++q) {
        const float4 w = v[q];
        dst[2 * q] = mk<T>((T)w.x, (T)w.y);
        dst[2 * q + 1] = mk<T>((T)w.z, (T)w.w);
      }
    } else {  // FP64 complex is one 16-byte load each
#pragma unroll
      for (int k = 0; k < N; ++k) dst[k] = src[k];
    }
  }
};

// ------------------------------------------------------------ Y = C + A M
// CG output columns per lane, N / CG lanes per row (a row never straddles a
// warp); each lane loads only its slice of the A row, the row is assembled in
// a padded per-warp buffer and read back whole.  M (n x n) sits in shared
// memory.  TA: type of A and M, TY: type of C and Y (precision conversion here).
template <typename TA, typename TY, int N, int CG>
__global__ void __launch_bounds__(256) k_block_axpy(const C<TA> *__restrict__ Ain, const C<TY> *__restrict__ Cin,
                                                    const C<TA> *__restrict__ M, C<TY> *__restrict__ Y, long rows) {
  constexpr int TPR = N / CG;
  constexpr int RPW = 32 / TPR;
  constexpr int RS = N + (16 / (int)sizeof(C<TA>) > 0 ? 16 / (int)sizeof(C<TA>) : 1);
  __shared__ C<TA> sm[N * N];
  __shared__ __align__(16) C<TA> rowbuf[8][RPW * RS];
  for (int k = threadIdx.x; k < N * N; k += blockDim.x) sm[k] = M[k];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int slot = lane / TPR;
  const int j0 = (lane - slot * TPR) * CG;
  C<TA> *wrow = rowbuf[warp];
  const long rows_per_cta = (long)(blockDim.x >> 5) * RPW;
  for (long rbase = (long)blockIdx.x * rows_per_cta; rbase < rows; rbase += (long)gridDim.x * rows_per_cta) {
    const long r = rbase + (long)warp * RPW + slot;
    const bool live = slot < RPW && r < rows;
    if (live) {
#pragma unroll
      for (int c = 0; c < CG; ++c) wrow[slot * RS + j0 + c] = Ain[r * N + j0 + c];
    }
    __syncwarp();
    if (live) {
      C<TA> a[N];
      Row<TA, N>::load(wrow + slot * RS, a);
#pragma unroll
      for (int c = 0; c < CG; ++c) {
        C<TA> acc = czero<TA>();
#pragma unroll
        for (int k = 0; k < N; ++k) cmac<TA>(acc, a[k], sm[k * N + j0 + c]);
        if (Cin) {
          const C<TY> cv = Cin[r * N + j0 + c];
          Y[r * N + j0 + c] = mk<TY>((TY)(cv.x + acc.x), (TY)(cv.y + acc.y));
        } else {
          Y[r * N + j0 + c] = mk<TY>((TY)acc.x, (TY)acc.y);
        }
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------ fused all-shift update

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
                                                    int s_begin, int s_end, int compute_q, long rows, long fstride,
                                                    int acc) {
  constexpr int TPR = N / CG;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T> *sc = reinterpret_cast<C<T> *>(smem_raw);  // rho^-1 (if compute_q), then the pairs of [s_begin, s_end)
  __shared__ int supd[kMaxS];
  const int c0 = compute_q ? 0 : (1 + 2 * s_begin) * N * N;  // first coefficient staged
  const int ncoef = (1 + 2 * s_end) * N * N - c0;
  // per-warp row buffer after the coefficients: [warps][32 / TPR][RS], rows
  // padded by 16 bytes so that the rows of a warp start in different banks
  constexpr int RS = N + 16 / (int)sizeof(C<T>);
  C<T> *wrow_all = sc + ncoef;
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
  C<T> *wrow = wrow_all + warp * RPW * RS;
  const long rows_per_cta = (long)(blockDim.x >> 5) * RPW;
  for (long rbase = (long)blockIdx.x * rows_per_cta; rbase < rows; rbase += (long)gridDim.x * rows_per_cta) {
    const long r = rbase + (long)warp * RPW + slot;
    const bool live = slot < RPW && r < rows;
    // Q row slice = W row rho^-1  (rho^-1 is upper triangular), or read it
    C<T> q[CG];
#pragma unroll
    for (int c = 0; c < CG; ++c) q[c] = czero<T>();
    if (compute_q) {
      // the W row is assembled in the warp's row buffer from the lanes' slices
      if (live) {
#pragma unroll
        for (int c = 0; c < CG; ++c) wrow[slot * RS + j0 + c] = W[r * N + j0 + c];
      }
      __syncwarp();
      if (live) {
        C<T> w[N];
        Row<T, N>::load(wrow + slot * RS, w);
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
          for (int c = 0; c < CG; ++c)
            if (k <= j0 + c) cmac<T>(q[c], w[k], sc[k * N + j0 + c]);
#pragma unroll
        for (int c = 0; c < CG; ++c) Q[r * N + j0 + c] = q[c];
      }
      __syncwarp();
    } else if (live) {
#pragma unroll
      for (int c = 0; c < CG; ++c) q[c] = Q[r * N + j0 + c];
    }
    // software pipeline over the live shifts: the P^(s) and X^(s) slices of the
    // next live shift are loaded while the current one is combined, so that a
    // warp keeps two shifts' rows in flight
    auto next_live = [&](int from) {
      while (from < s_end && !supd[from]) ++from;
      return from;
    };
    // acc: X is one accumulator for all shifts (sum_s X^(s), the M1 already
    // weighted), read once per row, summed in registers, written once
    const long xs = acc ? 0 : fstride;
    int s = next_live(s_begin);
    const bool touched = live && s < s_end;
    C<T> own[CG];
    CX ox[CG];
    if (touched) {
      ld_slice<T, CG>(P + s * fstride + r * N + j0, own);
      ld_slice<TX, CG>(X + s * xs + r * N + j0, ox);
    }
    while (s < s_end) {
      const int sn = next_live(s + 1);
      C<T> nown[CG];
      CX nox[CG];
      if (live && sn < s_end) {
        ld_slice<T, CG>(P + sn * fstride + r * N + j0, nown);
        if (!acc) ld_slice<TX, CG>(X + sn * xs + r * N + j0, nox);
      }
      const C<T> *m1 = sc + (1 + 2 * s) * N * N - c0;
      const C<T> *m2 = m1 + N * N;
      // each lane holds only its own CG columns; the row is assembled in the
      // warp's shared row buffer and read back whole (no redundant global loads)
      if (live) {
#pragma unroll
        for (int c = 0; c < CG; ++c) wrow[slot * RS + j0 + c] = own[c];
      }
      __syncwarp();
      if (live) {
        C<T> p[N];
        Row<T, N>::load(wrow + slot * RS, p);
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
        C<T> pn[CG];
#pragma unroll
        for (int c = 0; c < CG; ++c) {
          ox[c].x += a1[c].x;
          ox[c].y += a1[c].y;
          pn[c] = mk<T>(q[c].x + a2[c].x, q[c].y + a2[c].y);
        }
        if (!acc) st_slice<TX, CG>(X + s * xs + r * N + j0, ox);
        st_slice<T, CG>(P + s * fstride + r * N + j0, pn);
      }
      __syncwarp();
      if (sn < s_end) {
#pragma unroll
        for (int c = 0; c < CG; ++c) {
          own[c] = nown[c];
          if (!acc) ox[c] = nox[c];
        }
      }
      s = sn;
    }
    if (acc && touched) st_slice<TX, CG>(X + r * N + j0, ox);
  }
}

// ------------------------------------------------------------ shifted updates, column owners
// FP32 shifted updates of Algorithm 1 for every live shift:
//   X^(s) += P^(s) M1^(s),   P^(s) = Q + P^(s) M2^(s)
// (M1 = alpha^(s)_k, M2 = beta^(s)_k rho_k^dagger).  Each warp owns tiles of
// R rows; lane l < 2N owns output column j = l mod N of M1 (l < N) or M2
// (N <= l < 2N) and keeps that coefficient column in registers for the shift.
// The tile's Q rows and, NB - 1 shifts ahead, its P^(s) and X^(s) rows are
// staged in the warp's shared memory by cp.async; every lane reads the P^(s)
// rows as broadcasts.
__device__ __forceinline__ void cpa16(unsigned dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
template <int NW> __device__ __forceinline__ void cpa_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(NW) : "memory");
}

// X^(s) rows r, r+1 (lanes of M1) or P^(s) rows (lanes of M2) of a column-owner tile
__device__ __forceinline__ void col_store(int mat, int j, int r, int N, long off, const float2 *xt, const float2 *qs,
                                          float2 *X, float2 *P, float2 s0, float2 s1) {
  if (mat == 0) {
    const float2 x0 = xt[r * N + j], x1 = xt[(r + 1) * N + j];
    X[off + r * N + j] = make_float2(x0.x + s0.x, x0.y + s0.y);
    X[off + (r + 1) * N + j] = make_float2(x1.x + s1.x, x1.y + s1.y);
  } else {
    const float2 q0 = qs[r * N + j], q1 = qs[(r + 1) * N + j];
    P[off + r * N + j] = make_float2(q0.x + s0.x, q0.y + s0.y);
    P[off + (r + 1) * N + j] = make_float2(q1.x + s1.x, q1.y + s1.y);
  }
}

// tiles of R x N complex per warp: Q, NB x (P, X)
template <int NB> constexpr int col_tiles_per_warp() { return 1 + 2 * NB; }

// R rows per warp tile, W warps per CTA, NB shifts in flight per warp;
// PACKED: FP32x2 FMAs.  A complex product u c is formed from the (re, im) pair
// of u as loaded, times the duplicated pairs (c.re, c.re) and (c.im, c.im)
// held in registers: A = sum (u.re c.re, u.im c.re), B = sum (u.re c.im,
// u.im c.im), u c = (A.x - B.y, A.y + B.x): two packed FMAs per complex
// multiply-add instead of four scalar ones.
template <int N, int R, int W, int NB, bool PACKED>
__global__ void __launch_bounds__(W * 32, 1) k_update_cols(const float2 *__restrict__ Q, float2 *__restrict__ P,
                                                        float2 *__restrict__ X, const float2 *__restrict__ coef,
                                                        const int *__restrict__ upd, int s_begin, int s_end, long rows,
                                                        long fstride) {
  constexpr int TILE = R * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int live[kMaxS];
  __shared__ int nlive;
  const int nsh = s_end - s_begin;
  float2 *cs = reinterpret_cast<float2 *>(smem_raw);  // [nsh][2][N * N]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 *qs = cs + (size_t)nsh * 2 * N * N + (size_t)warp * col_tiles_per_warp<NB>() * TILE;
  auto ptile = [&](int b) { return qs + TILE * (1 + 2 * b); };
  auto xtile = [&](int b) { return qs + TILE * (2 + 2 * b); };
  for (int k = threadIdx.x; k < nsh * 2 * N * N; k += blockDim.x) cs[k] = coef[(1 + 2 * s_begin) * N * N + k];
  if (threadIdx.x == 0) {
    int m = 0;
    for (int q = s_begin; q < s_end; ++q)
      if (upd[q]) live[m++] = q;
    nlive = m;
  }
  __syncthreads();
  const int nl = nlive;
  if (nl == 0) return;
  const int mat = lane / N, j = lane - (lane / N) * N;
  const bool act = lane < 2 * N;
  const long ntiles = (rows + R - 1) / R;
  for (long tile = (long)blockIdx.x * W + warp; tile < ntiles; tile += (long)gridDim.x * W) {
    const long r0 = tile * R;
    const int nr = (int)min((long)R, rows - r0);  // rows is a multiple of 8: nr is even
    const int chunks = nr * N / 2;                 // 16-byte chunks of one tile
    auto copy_tile = [&](float2 *dst, const float2 *src) {
      const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
      const char *s8 = reinterpret_cast<const char *>(src);
      for (int c = lane; c < chunks; c += 32) cpa16(d + 16u * c, s8 + 16L * c);
    };
    copy_tile(qs, Q + r0 * N);
#pragma unroll
    for (int b = 0; b < NB - 1; ++b) {
      if (b < nl) {
        const long off = live[b] * fstride + r0 * N;
        copy_tile(ptile(b), P + off);
        copy_tile(xtile(b), X + off);
      }
      cp_async_commit();
    }
    for (int i = 0; i < nl; ++i) {
      const int b = i % NB;
      const int inext = i + NB - 1;
      if (inext < nl) {
        const long off = live[inext] * fstride + r0 * N;
        copy_tile(ptile(inext % NB), P + off);
        copy_tile(xtile(inext % NB), X + off);
      }
      cp_async_commit();
      cpa_wait<NB - 1>();  // shift i's tiles (and the Q tile) have landed for this lane
      __syncwarp();        // ... and for the whole warp
      const int sh = live[i];
      const float2 *xt = xtile(b);
      const long off = sh * fstride + r0 * N;
      if constexpr (PACKED) {
        unsigned long long cr[N], ci[N];
        if (act) {
          const float2 *m = cs + ((sh - s_begin) * 2 + mat) * N * N + j;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const float2 c = m[k * N];
            cr[k] = pack2(c.x, c.x);
            ci[k] = pack2(c.y, c.y);
          }
        }
        const float2 *pt = ptile(b);
        if (act) {
#pragma unroll 1
          for (int r = 0; r < nr; r += 2) {
            unsigned long long a0 = 0ull, a1 = 0ull, b0 = 0ull, b1 = 0ull;  // row r: A, B (even, odd k)
            unsigned long long c0 = 0ull, c1 = 0ull, d0 = 0ull, d1 = 0ull;  // row r + 1
            const float2 *p0 = pt + r * N, *p1 = p0 + N;
            if constexpr (N % 2 == 0) {
#pragma unroll
              for (int k = 0; k < N; k += 2) {
                const ulonglong2 u = *reinterpret_cast<const ulonglong2 *>(p0 + k);
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p1 + k);
                a0 = fma2(u.x, cr[k], a0);
                b0 = fma2(u.x, ci[k], b0);
                a1 = fma2(u.y, cr[k + 1], a1);
                b1 = fma2(u.y, ci[k + 1], b1);
                c0 = fma2(v.x, cr[k], c0);
                d0 = fma2(v.x, ci[k], d0);
                c1 = fma2(v.y, cr[k + 1], c1);
                d1 = fma2(v.y, ci[k + 1], d1);
              }
            } else {
#pragma unroll
              for (int k = 0; k < N; ++k) {
                const unsigned long long u = *reinterpret_cast<const unsigned long long *>(p0 + k);
                const unsigned long long v = *reinterpret_cast<const unsigned long long *>(p1 + k);
                a0 = fma2(u, cr[k], a0);
                b0 = fma2(u, ci[k], b0);
                c0 = fma2(v, cr[k], c0);
                d0 = fma2(v, ci[k], d0);
              }
            }
            const float2 A0 = unpack2(add2(a0, a1)), B0 = unpack2(add2(b0, b1));
            const float2 A1 = unpack2(add2(c0, c1)), B1 = unpack2(add2(d0, d1));
            col_store(mat, j, r, N, off, xt, qs, X, P, make_float2(A0.x - B0.y, A0.y + B0.x),
                      make_float2(A1.x - B1.y, A1.y + B1.x));
          }
        }
      } else {
        float2 cf[N];
        if (act) {
          const float2 *m = cs + ((sh - s_begin) * 2 + mat) * N * N + j;
#pragma unroll
          for (int k = 0; k < N; ++k) cf[k] = m[k * N];
        }
        const float2 *pt = ptile(b);
        if (act) {
#pragma unroll 1
          for (int r = 0; r < nr; r += 2) {
            float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f, bx0 = 0.f, by0 = 0.f, bx1 = 0.f, by1 = 0.f;
            const float2 *p0 = pt + r * N, *p1 = p0 + N;
            if constexpr (N % 2 == 0) {
#pragma unroll
              for (int k = 0; k < N; k += 2) {
                const float4 u = *reinterpret_cast<const float4 *>(p0 + k);
                const float4 v = *reinterpret_cast<const float4 *>(p1 + k);
                const float2 c0 = cf[k], c1 = cf[k + 1];
                ax0 = fmaf(u.x, c0.x, ax0); ax0 = fmaf(-u.y, c0.y, ax0);
                ay0 = fmaf(u.x, c0.y, ay0); ay0 = fmaf(u.y, c0.x, ay0);
                ax1 = fmaf(u.z, c1.x, ax1); ax1 = fmaf(-u.w, c1.y, ax1);
                ay1 = fmaf(u.z, c1.y, ay1); ay1 = fmaf(u.w, c1.x, ay1);
                bx0 = fmaf(v.x, c0.x, bx0); bx0 = fmaf(-v.y, c0.y, bx0);
                by0 = fmaf(v.x, c0.y, by0); by0 = fmaf(v.y, c0.x, by0);
                bx1 = fmaf(v.z, c1.x, bx1); bx1 = fmaf(-v.w, c1.y, bx1);
                by1 = fmaf(v.z, c1.y, by1); by1 = fmaf(v.w, c1.x, by1);
              }
            } else {
#pragma unroll
              for (int k = 0; k < N; ++k) {
                const float2 u = p0[k], v = p1[k], c0 = cf[k];
                ax0 = fmaf(u.x, c0.x, ax0); ax0 = fmaf(-u.y, c0.y, ax0);
                ay0 = fmaf(u.x, c0.y, ay0); ay0 = fmaf(u.y, c0.x, ay0);
                bx0 = fmaf(v.x, c0.x, bx0); bx0 = fmaf(-v.y, c0.y, bx0);
                by0 = fmaf(v.x, c0.y, by0); by0 = fmaf(v.y, c0.x, by0);
              }
            }
            col_store(mat, j, r, N, off, xt, qs, X, P, make_float2(ax0 + ax1, ay0 + ay1),
                      make_float2(bx0 + bx1, by0 + by1));
          }
        }
      }
      __syncwarp();  // buffer b is refilled at the next step
    }
    cpa_wait<0>();
    __syncwarp();  // the Q tile and buffers are reused by the next tile
  }
}

template <int N, int R, int W, int NB, bool PACKED>
static size_t col_smem(int nsh) {
  return (size_t)nsh * 2 * N * N * sizeof(float2) + (size_t)W * col_tiles_per_warp<NB>() * R * N * sizeof(float2);
}

template <int N, int R, int W, int NB, bool PACKED>
static rhmc_status_t launch_update_cols(const float2 *Q, float2 *P, float2 *X, const float2 *coef, const int *upd,
                                        int s_begin, int s_end, long rows, long fstride, cudaStream_t s) {
  const int threads = W * 32;
  const size_t smem = col_smem<N, R, W, NB, PACKED>(s_end - s_begin);
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_update_cols<N, R, W, NB, PACKED>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  if (smem > 220 * 1024) return RHMC_ERR_INVALID_ARG;
  const long ntiles = (rows + R - 1) / R;
  long grid = (ntiles + W - 1) / W;
  grid = std::min(grid, (long)resident_ctas(k_update_cols<N, R, W, NB, PACKED>, threads, smem));
  k_update_cols<N, R, W, NB, PACKED><<<(unsigned)grid, threads, smem, s>>>(Q, P, X, coef, upd, s_begin, s_end, rows,
                                                                             fstride);
  return RHMC_OK;
}

// Variants of the column-owner kernel (RHMC_TUNE_UPDATE_TENSOR), rows per warp
// tile / warps per CTA / shifts in flight (p: FP32x2 FMAs): 3 = 16/8/3;
// 4 = 8/16/3; 5 = 8/16/2p (built-in, 0); 6 = 4/32/3; 7 = 8/24/2; 8 = 8/28/2;
// 9 = 4/32/2; 10 = 8/16/3p; 11 = 8/20/2p.  Measured at 24^4, n = 16, 15 live
// shifts, one launch alone: 1116, 830, -, 1042, 792, 720, 694, 789 us for 3,
// 4, 6 ... 9 (scalar FMAs); in the whole force evaluation 5 takes the update
// from 4.35 to 4.54 TB/s: with packed FMAs the kernel is bound by the FMA pipe
// (60 % busy, issue 56 %) rather than by instruction issue (80 %).
#define RHMC_COL_VARIANTS(X_)                   \
  switch (col_variant()) {                      \
    case 3: X_(16, 8, 3, false); break;         \
    case 4: X_(8, 16, 3, false); break;         \
    case 6: X_(4, 32, 3, false); break;         \
    case 7: X_(8, 24, 2, false); break;         \
    case 8: X_(8, 28, 2, false); break;         \
    case 9: X_(4, 32, 2, false); break;         \
    case 10: X_(8, 16, 3, true); break;         \
    case 11: X_(8, 20, 2, true); break;         \
    default: X_(8, 16, 2, true); break;         \
  }
static int col_variant() { return tune_get(TUNE_UPDATE_TENSOR); }
template <int N> static size_t col_tiles_bytes() {
  size_t b = 0;
#define L_(R_, W_, NB_, P_) b = col_smem<N, R_, W_, NB_, P_>(0)
  RHMC_COL_VARIANTS(L_)
#undef L_
  return b;
}
template <int N>
static rhmc_status_t launch_update_cols_variant(const float2 *Q, float2 *P, float2 *X, const float2 *coef,
                                                const int *upd, int s_begin, int s_end, long rows, long fstride,
                                                cudaStream_t s) {
  rhmc_status_t rc = RHMC_OK;
#define L_(R_, W_, NB_, P_) \
  rc = launch_update_cols<N, R_, W_, NB_, P_>(Q, P, X, coef, upd, s_begin, s_end, rows, fstride, s)
  RHMC_COL_VARIANTS(L_)
#undef L_
  return rc;
}

// ------------------------------------------------------------ fused base step
// The base system's updates of Algorithm 1 after rho_k, in one pass over the
// rows (FP32, column-owner lanes, packed FP32x2 FMAs):
//   Q_k = W rho_k^-1                                  (block QR)
//   X^(0) += P^(0) M1,  M1 = alpha_k delta_{k-1}       (base solution)
//   P^(0) = Q_k + P^(0) M2,  M2 = rho_k^dagger         (base search block)
// and, in the stored-basis mode, Q_k into block kb of the basis.  coef holds
// rho^-1, M1, M2 (n x n each).  Each warp stages a tile of R rows of W, P^(0)
// and X^(0) by cp.async; pass 1: lane j < n forms column j of Q (stored to Q
// and the basis) while lane n + j forms column j of X; pass 2: lane n + j
// (with lane j) forms column j of P, each lane of the pair half of the sum.  It
// replaces three passes (Q = W rho^-1, the basis copy, the base update):
// W, P, X read once, Q, P, X (and the basis block) written once.  The tiles
// are double-buffered: a warp's next row tile is in flight while the current
// one is multiplied.
template <int N, int R, int WW>
__global__ void __launch_bounds__(WW * 32, 1) k_base_step(const float2 *__restrict__ Wf, float2 *__restrict__ Q,
                                                        float2 *__restrict__ P, float2 *__restrict__ X,
                                                        const float2 *__restrict__ coef, float2 *__restrict__ basis,
                                                        int cap, const int *__restrict__ kdev, long rows) {
  constexpr int TILE = R * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int CS = (3 * N * N + 1) & ~1;  // coefficient area, padded: the tiles start on 16-byte boundaries
  float2 *cs = reinterpret_cast<float2 *>(smem_raw);  // rho^-1, M1, M2
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 *wbuf = cs + CS + (size_t)warp * 6 * TILE;  // [2][W, P, X] tiles
  for (int k = threadIdx.x; k < 3 * N * N; k += blockDim.x) cs[k] = coef[k];
  const int kb = (basis && kdev) ? *kdev : -1;
  const bool store_basis = kb >= 0 && kb < cap;
  __syncthreads();
  const bool lo = lane < N, hi = lane >= N && lane < 2 * N;
  const int j = lo ? lane : (hi ? lane - N : 0);
  const long ntiles = (rows + R - 1) / R;
  const long t0 = (long)blockIdx.x * WW + warp, dt = (long)gridDim.x * WW;
  auto issue = [&](long tile, int b) {
    const long r0 = tile * R;
    const int chunks = (int)min((long)R, rows - r0) * N / 2;
    const unsigned d = (unsigned)__cvta_generic_to_shared(wbuf + (size_t)b * 3 * TILE);
    const char *sw = reinterpret_cast<const char *>(Wf + r0 * N);
    const char *sp = reinterpret_cast<const char *>(P + r0 * N);
    const char *sx = reinterpret_cast<const char *>(X + r0 * N);
    for (int c = lane; c < chunks; c += 32) {
      cpa16(d + 16u * c, sw + 16L * c);
      cpa16(d + 16u * (TILE / 2 + c), sp + 16L * c);
      cpa16(d + 16u * (TILE + c), sx + 16L * c);
    }
  };
  if (t0 < ntiles) issue(t0, 0);
  cp_async_commit();
  int buf = 0;
  for (long tile = t0; tile < ntiles; tile += dt, buf ^= 1) {
    if (tile + dt < ntiles) issue(tile + dt, buf ^ 1);
    cp_async_commit();
    const long r0 = tile * R;
    const int nr = (int)min((long)R, rows - r0);  // rows is a multiple of 8: nr is even
    const float2 *wt = wbuf + (size_t)buf * 3 * TILE, *pt = wt + TILE, *xt = pt + TILE;
    unsigned long long cr[N], ci[N];
    {  // pass-1 coefficient column: rho^-1 (lanes < N) or M1 (lanes N .. 2N-1)
      const float2 *m = cs + (hi ? N * N : 0) + j;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const float2 c = m[k * N];
        cr[k] = pack2(c.x, c.x);
        ci[k] = pack2(c.y, c.y);
      }
    }
    cpa_wait<1>();
    __syncwarp();
    // pass 1: row r of W (lanes < N) or of P (lanes N .. 2N-1) times the lane's column
    float2 qv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      qv[r] = make_float2(0.f, 0.f);
      if (r < nr && (lo || hi)) {
        const float2 *u = (lo ? wt : pt) + r * N;
        unsigned long long a = 0ull, b = 0ull;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const unsigned long long v = *reinterpret_cast<const unsigned long long *>(u + k);
          a = fma2(v, cr[k], a);
          b = fma2(v, ci[k], b);
        }
        const float2 A = unpack2(a), B = unpack2(b);
        const float2 prod = make_float2(A.x - B.y, A.y + B.x);
        const long row = r0 + r;
        if (lo) {
          qv[r] = prod;
          Q[row * N + j] = prod;
          if (store_basis) basis[row * (long)cap * N + (long)kb * N + j] = prod;
        } else {
          const float2 x = xt[r * N + j];
          X[row * N + j] = make_float2(x.x + prod.x, x.y + prod.y);
        }
      }
    }
    // pass 2: P = Q + P M2 with the sum over k split between the lane pair (j, N + j):
    // lane j takes k < N/2, lane N + j the rest; lane j adds Q's column j and stores
    constexpr int KH = (N + 1) / 2;
    const int k0 = hi ? N / 2 : 0, k1 = hi ? N : N / 2;
    {  // pass-2 coefficient half-column of M2 (zero past the lane's range)
      const float2 *m = cs + 2 * N * N + j;
#pragma unroll
      for (int kk = 0; kk < KH; ++kk) {
        const int k = k0 + kk;
        const float2 c = k < k1 ? m[k * N] : make_float2(0.f, 0.f);
        cr[kk] = pack2(c.x, c.x);
        ci[kk] = pack2(c.y, c.y);
      }
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 part = make_float2(0.f, 0.f);
      if (r < nr && (lo || hi)) {
        const float2 *u = pt + r * N + k0;
        unsigned long long a = 0ull, b = 0ull;
#pragma unroll
        for (int kk = 0; kk < KH; ++kk) {
          const unsigned long long v = (k0 + kk < N) ? *reinterpret_cast<const unsigned long long *>(u + kk) : 0ull;
          a = fma2(v, cr[kk], a);
          b = fma2(v, ci[kk], b);
        }
        const float2 A = unpack2(a), B = unpack2(b);
        part = make_float2(A.x - B.y, A.y + B.x);
      }
      const float ox = __shfl_down_sync(0xffffffffu, part.x, N);
      const float oy = __shfl_down_sync(0xffffffffu, part.y, N);
      if (r < nr && lo) P[(r0 + r) * N + j] = make_float2(qv[r].x + part.x + ox, qv[r].y + part.y + oy);
    }
    __syncwarp();  // buffer buf is refilled for the tile after next
  }
  cpa_wait<0>();
}

constexpr int kBaseRows = 8, kBaseWarps = 16;

template <int N, int R, int WW>
static void launch_base(const float2 *W, float2 *Q, float2 *P, float2 *X, const float2 *coef, float2 *basis, int cap,
                        const int *kdev, long rows, cudaStream_t s) {
  const int threads = WW * 32;
  const size_t smem = (((3 * N * N + 1) & ~1) + (size_t)WW * 6 * R * N) * sizeof(float2);
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_base_step<N, R, WW>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const long ntiles = (rows + R - 1) / R;
  long grid = (ntiles + WW - 1) / WW;
  grid = std::min(grid, (long)resident_ctas(k_base_step<N, R, WW>, threads, smem));
  k_base_step<N, R, WW><<<(unsigned)grid, threads, smem, s>>>(W, Q, P, X, coef, basis, cap, kdev, rows);
}

rhmc_status_t base_step(const float2 *W, float2 *Q, float2 *P, float2 *X, const float2 *coef, float2 *basis, int cap,
                        const int *kdev, long rows, int n, cudaStream_t s) {
  if (rows % 8) return RHMC_ERR_INVALID_ARG;
  prof_begin(PROF_UPDATE_SHIFTS32, s);
  rhmc_status_t rc = RHMC_OK;
  // n = 16: row tile and warps per CTA from RHMC_TUNE_BASE_TILE (0: 8 rows, 16 warps)
  const int tile = tune_get(TUNE_BASE_TILE);
#define L_BASE(NN)                                                                               \
  {                                                                                              \
    if constexpr (NN == 16) {                                                                    \
      if (tile == 1)                                                                             \
        launch_base<NN, 16, 12>(W, Q, P, X, coef, basis, cap, kdev, rows, s);                    \
      else if (tile == 2)                                                                        \
        launch_base<NN, 16, 8>(W, Q, P, X, coef, basis, cap, kdev, rows, s);                     \
      else if (tile == 3)                                                                        \
        launch_base<NN, 8, 12>(W, Q, P, X, coef, basis, cap, kdev, rows, s);                     \
      else                                                                                       \
        launch_base<NN, kBaseRows, kBaseWarps>(W, Q, P, X, coef, basis, cap, kdev, rows, s);     \
    } else {                                                                                     \
      launch_base<NN, kBaseRows, kBaseWarps>(W, Q, P, X, coef, basis, cap, kdev, rows, s);       \
    }                                                                                            \
  }
  RHMC_DISPATCH_N(n, L_BASE)
#undef L_BASE
  prof_end(s, (double)rows * n * sizeof(float2) * (6.0 + (basis ? 1.0 : 0.0)));
  RHMC_LAUNCH_CHECK();
  return rc;
}

static rhmc_status_t update_shifts_cols_range(const float2 *Q, float2 *P, float2 *X, const float2 *coef,
                                              const int *upd, int s_begin, int s_end, long rows, int n, long fstride,
                                              cudaStream_t s);

// Shifted updates (no base) for the FP32 mixed path with the column-owner kernel,
// in as many launches as the shared-memory coefficient store needs.
rhmc_status_t update_shifts_cols(const float2 *Q, float2 *P, float2 *X, const float2 *coef, const int *upd,
                                 int s_begin, int s_end, long rows, int n, long fstride, cudaStream_t s) {
  if (rows % 8) return RHMC_ERR_INVALID_ARG;
  // shifts per launch that fit the shared-memory coefficient store
  size_t tiles = 0;
#define L_TB(NN) tiles = col_tiles_bytes<NN>()
  RHMC_DISPATCH_N(n, L_TB)
#undef L_TB
  const int per_launch = (int)((220 * 1024 - tiles) / (2 * n * n * sizeof(float2)));
  if (per_launch < 1) return RHMC_ERR_INVALID_ARG;
  for (int b = s_begin; b < s_end; b += per_launch) {
    const int e = std::min(s_end, b + per_launch);
    const rhmc_status_t rc = update_shifts_cols_range(Q, P, X, coef, upd, b, e, rows, n, fstride, s);
    if (rc != RHMC_OK) return rc;
  }
  return RHMC_OK;
}

static rhmc_status_t update_shifts_cols_range(const float2 *Q, float2 *P, float2 *X, const float2 *coef,
                                              const int *upd, int s_begin, int s_end, long rows, int n, long fstride,
                                              cudaStream_t s) {
  int nupd = s_end - s_begin;
  if (prof_on()) {  // profiling only: count the shifts this launch updates (host sync)
    int h[kMaxS];
    cudaStreamSynchronize(s);
    cudaMemcpy(h, upd, sizeof(int) * s_end, cudaMemcpyDeviceToHost);
    nupd = 0;
    for (int q = s_begin; q < s_end; ++q) nupd += h[q] != 0;
  }
  prof_begin(PROF_UPDATE_SHIFTS32, s);
  rhmc_status_t rc = RHMC_OK;
#define L_COLS(NN) rc = launch_update_cols_variant<NN>(Q, P, X, coef, upd, s_begin, s_end, rows, fstride, s)
  RHMC_DISPATCH_N(n, L_COLS)
#undef L_COLS
  prof_end(s, (double)rows * n * (sizeof(float2) + nupd * 4.0 * sizeof(float2)));
  if (rc != RHMC_OK) {
    set_error("update_shifts_cols: %d shifts at n = %d do not fit", s_end - s_begin, n);
    return rc;
  }
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// ------------------------------------------------------------ Y = C + A M, column owners
// FP32 tall-skinny update (Algorithm 1's block QR step, W = Q - (AP) alpha, and
// Q = W rho^-1): lane l < 2N owns column j = l mod N of M (kept in registers)
// for rows of parity l / N of each row pair; the warp's tiles of R rows of A
// and C are staged by cp.async two tiles deep; every lane reads the A row as
// a broadcast.  PK: packed FP32x2 FMAs on the (re, im) pair of each A element
// times the duplicated coefficient pairs (c.re, c.re), (c.im, c.im), as in
// the shifted updates.

// y = sum_k a[k] M[k][j], packed: cr[k] = (c.re, c.re), ci[k] = (c.im, c.im)
template <int N>
__device__ __forceinline__ float2 row_times_col_packed(const float2 *ar, const unsigned long long *cr,
                                                       const unsigned long long *ci) {
  unsigned long long a0 = 0ull, a1 = 0ull, b0 = 0ull, b1 = 0ull;
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int k = 0; k < N; k += 2) {
      const ulonglong2 u = *reinterpret_cast<const ulonglong2 *>(ar + k);
      a0 = fma2(u.x, cr[k], a0);
      b0 = fma2(u.x, ci[k], b0);
      a1 = fma2(u.y, cr[k + 1], a1);
      b1 = fma2(u.y, ci[k + 1], b1);
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const unsigned long long u = *reinterpret_cast<const unsigned long long *>(ar + k);
      a0 = fma2(u, cr[k], a0);
      b0 = fma2(u, ci[k], b0);
    }
  }
  const float2 A = unpack2(add2(a0, a1)), B = unpack2(add2(b0, b1));
  return make_float2(A.x - B.y, A.y + B.x);
}

// the same with scalar FMAs and cf[k] = M[k][j]
template <int N> __device__ __forceinline__ float2 row_times_col(const float2 *ar, const float2 *cf) {
  float ax0 = 0.f, ay0 = 0.f, ax1 = 0.f, ay1 = 0.f;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const float2 u = ar[k], c0 = cf[k];
    if (k & 1) {
      ax1 = fmaf(u.x, c0.x, ax1); ax1 = fmaf(-u.y, c0.y, ax1);
      ay1 = fmaf(u.x, c0.y, ay1); ay1 = fmaf(u.y, c0.x, ay1);
    } else {
      ax0 = fmaf(u.x, c0.x, ax0); ax0 = fmaf(-u.y, c0.y, ax0);
      ay0 = fmaf(u.x, c0.y, ay0); ay0 = fmaf(u.y, c0.x, ay0);
    }
  }
  return make_float2(ax0 + ax1, ay0 + ay1);
}

// the lane's coefficient column j of M, scalar (cf) or as duplicated pairs (cr, ci)
template <int N, bool PK>
__device__ __forceinline__ void load_col(const float2 *__restrict__ M, int j, float2 *cf, unsigned long long *cr,
                                         unsigned long long *ci) {
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const float2 c = M[k * N + j];
    if constexpr (PK) {
      cr[k] = pack2(c.x, c.x);
      ci[k] = pack2(c.y, c.y);
    } else {
      cf[k] = c;
    }
  }
}

template <int N, int R, int W, bool PK>
__global__ void __launch_bounds__(W * 32, PK ? 1 : 2) k_axpy_cols(const float2 *__restrict__ A,
                                                                  const float2 *__restrict__ Cin,
                                                                  const float2 *__restrict__ M,
                                                                  float2 *__restrict__ Y, long rows) {
  constexpr int TILE = R * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 *wb = reinterpret_cast<float2 *>(smem_raw) + (size_t)warp * 4 * TILE;  // [2 buffers][A, C]
  const int h = lane / N, j = lane - (lane / N) * N;
  const bool act = lane < 2 * N;
  float2 cf[PK ? 1 : N];
  unsigned long long cr[PK ? N : 1], ci[PK ? N : 1];
  if (act) load_col<N, PK>(M, j, cf, cr, ci);
  const long ntiles = (rows + R - 1) / R;
  const long t0 = (long)blockIdx.x * W + warp, dt = (long)gridDim.x * W;
  auto issue = [&](long tile, int b) {
    const long r0 = tile * R;
    const int chunks = (int)min((long)R, rows - r0) * N / 2;
    const unsigned da = (unsigned)__cvta_generic_to_shared(wb + (2 * b) * TILE);
    const unsigned dc = (unsigned)__cvta_generic_to_shared(wb + (2 * b + 1) * TILE);
    const char *sa = reinterpret_cast<const char *>(A + r0 * N);
    const char *sc = reinterpret_cast<const char *>(Cin ? Cin + r0 * N : nullptr);
    for (int c = lane; c < chunks; c += 32) {
      cpa16(da + 16u * c, sa + 16L * c);
      if (Cin) cpa16(dc + 16u * c, sc + 16L * c);
    }
  };
  if (t0 < ntiles) issue(t0, 0);
  cp_async_commit();
  int b = 0;
  for (long tile = t0; tile < ntiles; tile += dt, b ^= 1) {
    if (tile + dt < ntiles) issue(tile + dt, b ^ 1);
    cp_async_commit();
    cpa_wait<1>();
    __syncwarp();
    const long r0 = tile * R;
    const int nr = (int)min((long)R, rows - r0);
    const float2 *at = wb + (2 * b) * TILE, *ct = wb + (2 * b + 1) * TILE;
    if (act) {
#pragma unroll 1
      for (int r = h; r < nr; r += 2) {
        float2 y;
        if constexpr (PK)
          y = row_times_col_packed<N>(at + r * N, cr, ci);
        else
          y = row_times_col<N>(at + r * N, cf);
        if (Cin) {
          const float2 cv = ct[r * N + j];
          y.x += cv.x;
          y.y += cv.y;
        }
        Y[(r0 + r) * N + j] = y;
      }
    }
    __syncwarp();  // buffer b is refilled for the tile after next
  }
  cpa_wait<0>();
}

// Y = C + A M fused with the Gram G = Y^dagger Y (the thin-QR Gram of the block QR step):
// after a row pair of Y is formed, it is written to the warp's row buffer and
// lane (h, j) adds conj(Y[r][i]) Y[r][j] for all i to its FP32 column of G;
// the columns are combined across the row parities, the warps (FP64, shared
// memory) and the CTAs (partials summed in fixed order by k_gram_sum).
template <int N, int R, int W, bool PK>
__global__ void __launch_bounds__(W * 32, 1) k_axpy_gram_cols(const float2 *__restrict__ A,
                                                           const float2 *__restrict__ Cin,
                                                           const float2 *__restrict__ M, float2 *__restrict__ Y,
                                                           long rows, double2 *__restrict__ partial) {
  constexpr int TILE = R * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float2 *wb = reinterpret_cast<float2 *>(smem_raw) + (size_t)warp * (4 * TILE + 2 * N);  // [2][A, C], row pair
  float2 *wrow = wb + 4 * TILE;
  const int h = lane / N, j = lane - (lane / N) * N;
  const bool act = lane < 2 * N;
  // W^dagger W is Hermitian: lane j accumulates the circulant half G[(j + o) mod N][j],
  // o = 0 .. N/2; the reduction writes the other entries as conjugates
  constexpr int NO = N / 2 + 1;
  float2 g[NO];
#pragma unroll
  for (int k = 0; k < NO; ++k) g[k] = make_float2(0.f, 0.f);
  float2 cf[PK ? 1 : N];
  unsigned long long cr[PK ? N : 1], ci[PK ? N : 1];
  if (act) load_col<N, PK>(M, j, cf, cr, ci);
  const long ntiles = (rows + R - 1) / R;
  const long t0 = (long)blockIdx.x * W + warp, dt = (long)gridDim.x * W;
  auto issue = [&](long tile, int b) {
    const long r0 = tile * R;
    const int chunks = (int)min((long)R, rows - r0) * N / 2;
    const unsigned da = (unsigned)__cvta_generic_to_shared(wb + (2 * b) * TILE);
    const unsigned dc = (unsigned)__cvta_generic_to_shared(wb + (2 * b + 1) * TILE);
    const char *sa = reinterpret_cast<const char *>(A + r0 * N);
    const char *sc = reinterpret_cast<const char *>(Cin + r0 * N);
    for (int c = lane; c < chunks; c += 32) {
      cpa16(da + 16u * c, sa + 16L * c);
      cpa16(dc + 16u * c, sc + 16L * c);
    }
  };
  if (t0 < ntiles) issue(t0, 0);
  cp_async_commit();
  int b = 0;
  for (long tile = t0; tile < ntiles; tile += dt, b ^= 1) {
    if (tile + dt < ntiles) issue(tile + dt, b ^ 1);
    cp_async_commit();
    cpa_wait<1>();
    __syncwarp();
    const long r0 = tile * R;
    const int nr = (int)min((long)R, rows - r0);
    const float2 *at = wb + (2 * b) * TILE, *ct = wb + (2 * b + 1) * TILE;
#pragma unroll 1
    for (int r = 0; r < nr; r += 2) {
      float2 y = make_float2(0.f, 0.f);
      if (act) {
        const float2 *ar = at + (r + h) * N;
        float2 p;
        if constexpr (PK)
          p = row_times_col_packed<N>(ar, cr, ci);
        else
          p = row_times_col<N>(ar, cf);
        const float2 cv = ct[(r + h) * N + j];
        y = make_float2(p.x + cv.x, p.y + cv.y);
        Y[(r0 + r + h) * N + j] = y;
        wrow[h * N + j] = y;
      }
      __syncwarp();
      if (act) {
        const float2 *wr = wrow + h * N;
#pragma unroll
        for (int o = 0; o < NO; ++o) {  // g[o] += conj(Y[r][i]) Y[r][j], i = (j + o) mod N
          const float2 w = wr[j + o < N ? j + o : j + o - N];
          g[o].x = fmaf(w.x, y.x, fmaf(w.y, y.y, g[o].x));
          g[o].y = fmaf(w.x, y.y, fmaf(-w.y, y.x, g[o].y));
        }
      }
      __syncwarp();
    }
    __syncwarp();  // buffer b is refilled for the tile after next
  }
  cpa_wait<0>();
  // row parities: lane j += lane N + j
#pragma unroll
  for (int o = 0; o < NO; ++o) {
    g[o].x += __shfl_down_sync(0xffffffffu, g[o].x, N);
    g[o].y += __shfl_down_sync(0xffffffffu, g[o].y, N);
  }
  __syncthreads();
  double2 *red = reinterpret_cast<double2 *>(smem_raw);  // [W][N * N], reuses the tile buffers
  if (lane < N) {
#pragma unroll
    for (int o = 0; o < NO; ++o) {
      const int i = lane + o < N ? lane + o : lane + o - N;
      const double gx = (double)g[o].x, gy = (double)g[o].y;
      red[warp * N * N + i * N + lane] = make_double2(gx, gy);
      if (o > 0 && 2 * o != N) red[warp * N * N + lane * N + i] = make_double2(gx, -gy);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
    double2 sum = red[e];
    for (int w = 1; w < W; ++w) {
      sum.x += red[w * N * N + e].x;
      sum.y += red[w * N * N + e].y;
    }
    partial[(long)e * gridDim.x + blockIdx.x] = sum;
  }
}

constexpr int kAxpyRows = 8, kAxpyWarps = 16;
// warps per CTA of the fused axpy + Gram kernel (the packed form holds 64 more
// registers of coefficients per lane)
template <bool PK> constexpr int axpy_gram_warps() { return PK ? 12 : 16; }
static bool axpy_packed() { return tune_get(TUNE_AXPY_SCALAR) != 1; }

template <int N, bool PK>
static void launch_axpy_cols(const float2 *A, const float2 *C, const float2 *M, float2 *Y, long rows,
                             cudaStream_t s) {
  const int threads = kAxpyWarps * 32;
  const size_t smem = (size_t)kAxpyWarps * 4 * kAxpyRows * N * sizeof(float2);
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_axpy_cols<N, kAxpyRows, kAxpyWarps, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         220 * 1024);
  });
  const long ntiles = (rows + kAxpyRows - 1) / kAxpyRows;
  long grid = (ntiles + kAxpyWarps - 1) / kAxpyWarps;
  grid = std::min(grid, (long)resident_ctas(k_axpy_cols<N, kAxpyRows, kAxpyWarps, PK>, threads, smem));
  k_axpy_cols<N, kAxpyRows, kAxpyWarps, PK><<<(unsigned)grid, threads, smem, s>>>(A, C, M, Y, rows);
}

template <int N, bool PK>
static void launch_axpy_gram_cols(const float2 *A, const float2 *C, const float2 *M, float2 *Y, long rows,
                                  double2 *scratch, double2 *out, cudaStream_t s) {
  constexpr int W = axpy_gram_warps<PK>();
  // rows per warp tile: 8, or 16 at n = 16 with RHMC_TUNE_AXPY_ROWS = 1
  constexpr int R = (PK && N == 16) ? 16 : kAxpyRows;
  const bool big = (PK && N == 16) && tune_get(TUNE_AXPY_ROWS) == 1;
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(k_axpy_gram_cols<N, R, W, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    cudaFuncSetAttribute(k_axpy_gram_cols<N, kAxpyRows, W, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         220 * 1024);
  });
  auto run = [&](auto kern, int rr) {
    const int threads = W * 32;
    const size_t smem = std::max((size_t)W * (4 * rr * N + 2 * N) * sizeof(float2), (size_t)W * N * N * sizeof(double2));
    const long ntiles = (rows + rr - 1) / rr;
    long grid = (ntiles + W - 1) / W;
    grid = std::min(grid, (long)std::min(kGramCtas, resident_ctas(kern, threads, smem)));
    kern<<<(unsigned)grid, threads, smem, s>>>(A, C, M, Y, rows, scratch);
    return grid;
  };
  const long grid = big ? run(k_axpy_gram_cols<N, R, W, PK>, R) : run(k_axpy_gram_cols<N, kAxpyRows, W, PK>, kAxpyRows);
  k_gram_sum<<<N * N, 128, 0, s>>>(scratch, (int)grid, out);
  count_launch();  // the second kernel of this launcher (the caller counts the first)
}

// Y = C + A M and out = Y^dagger Y (FP64 sums of FP32 products) in one pass over
// the rows; scratch holds kGramCtas * n * n partials.
rhmc_status_t axpy_gram_cols(const float2 *A, const float2 *C, const float2 *M, float2 *Y, long rows, int n,
                             double2 *scratch, double2 *out, cudaStream_t s) {
  if (rows % 8 || !C) return RHMC_ERR_INVALID_ARG;
  prof_begin(PROF_AXPY, s);
#define L_AG(NN)                                                        \
  if (axpy_packed())                                                    \
    launch_axpy_gram_cols<NN, true>(A, C, M, Y, rows, scratch, out, s); \
  else                                                                  \
    launch_axpy_gram_cols<NN, false>(A, C, M, Y, rows, scratch, out, s)
  RHMC_DISPATCH_N(n, L_AG)
#undef L_AG
  prof_end(s, (double)rows * n * sizeof(float2) * 3);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// Y = C + A M for FP32 fields of width n (C may be null), column-owner kernel.
rhmc_status_t axpy_cols(const float2 *A, const float2 *C, const float2 *M, float2 *Y, long rows, int n,
                        cudaStream_t s) {
  if (rows % 8) return RHMC_ERR_INVALID_ARG;
  prof_begin(PROF_AXPY, s);
#define L_AX(NN)                                   \
  if (axpy_packed())                               \
    launch_axpy_cols<NN, true>(A, C, M, Y, rows, s); \
  else                                             \
    launch_axpy_cols<NN, false>(A, C, M, Y, rows, s)
  RHMC_DISPATCH_N(n, L_AX)
#undef L_AX
  prof_end(s, (double)rows * n * sizeof(float2) * (C ? 3 : 2));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
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

template <typename T, int N, bool PK, int TR, int WG>
static void launch_gram_tw(const C<T> *A, const C<T> *B, long rows, double2 *scratch, double2 *out, cudaStream_t s) {
  const bool same = (A == B);
  const size_t smem = (size_t)WG * 2 * (same ? 1 : 2) * TR * N * sizeof(C<T>);
  const size_t smem_red = (size_t)WG * N * N * sizeof(double2);
  const size_t bytes = std::max(smem, smem_red);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_gram<T, N, true, PK, TR, WG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_gram<T, N, false, PK, TR, WG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const long ntiles = (rows + TR - 1) / TR;
  // one wave: as many CTAs as are resident at once (at most the partials' capacity)
  const int threads = WG * 32;
  const int resident = same ? resident_ctas(k_gram<T, N, true, PK, TR, WG>, threads, bytes)
                            : resident_ctas(k_gram<T, N, false, PK, TR, WG>, threads, bytes);
  const int grid = (int)std::min<long>((ntiles + WG - 1) / WG, std::min(kGramCtas, resident));
  if (same)
    k_gram<T, N, true, PK, TR, WG><<<grid, threads, bytes, s>>>(A, B, rows, scratch);
  else
    k_gram<T, N, false, PK, TR, WG><<<grid, threads, bytes, s>>>(A, B, rows, scratch);
  k_gram_sum<<<N * N, 128, 0, s>>>(scratch, grid, out);
  count_launch();  // the second kernel of this launcher (the caller counts the first)
}
template <typename T, int N, bool PK>
static void launch_gram(const C<T> *A, const C<T> *B, long rows, double2 *scratch, double2 *out, cudaStream_t s) {
  // packed n = 16: tile rows x warps from RHMC_TUNE_GRAM_TILE (0: 16 x 4, measured at 24^4:
  // 37.6 us against 41.8 for 16 x 8, 38.2 for 32 x 8, 41.5 for 8 x 8)
  if constexpr (PK && N == 16) {
    switch (tune_get(TUNE_GRAM_TILE)) {
      case 1: launch_gram_tw<T, N, PK, 32, 8>(A, B, rows, scratch, out, s); return;
      case 2: launch_gram_tw<T, N, PK, 16, 8>(A, B, rows, scratch, out, s); return;
      case 3: launch_gram_tw<T, N, PK, 8, 8>(A, B, rows, scratch, out, s); return;
      default: launch_gram_tw<T, N, PK, 16, 4>(A, B, rows, scratch, out, s); return;
    }
  }
  launch_gram_tw<T, N, PK, kGramTileRows, kGramWarps>(A, B, rows, scratch, out, s);
}

// packed FMAs for FP32 at n = 16 unless RHMC_TUNE_AXPY_SCALAR = 1
template <typename T, int N>
static void launch_gram_any(const C<T> *A, const C<T> *B, long rows, double2 *scratch, double2 *out, cudaStream_t s) {
  if constexpr (N == 16 && sizeof(T) == 4) {
    if (tune_get(TUNE_AXPY_SCALAR) != 1) {
      launch_gram<T, N, true>(A, B, rows, scratch, out, s);
      return;
    }
  }
  launch_gram<T, N, false>(A, B, rows, scratch, out, s);
}

// G = A^dagger B into out (n x n, FP64); scratch holds kGramCtas * n * n partials.
template <typename T>
rhmc_status_t gram(const C<T> *A, const C<T> *B, long rows, int n, double2 *scratch, double2 *out, cudaStream_t s) {
  prof_begin(sizeof(T) == 4 ? PROF_GRAM32 : PROF_GRAM64, s);
#define L_GRAM(NN) launch_gram_any<T, NN>(A, B, rows, scratch, out, s)
  RHMC_DISPATCH_N(n, L_GRAM)
#undef L_GRAM
  prof_end(s, (double)rows * n * sizeof(C<T>) * (A == B ? 1 : 2));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t gram<float>(const float2 *, const float2 *, long, int, double2 *, double2 *, cudaStream_t);
template rhmc_status_t gram<double>(const double2 *, const double2 *, long, int, double2 *, double2 *, cudaStream_t);

template <typename TA, typename TY>
rhmc_status_t block_axpy(const C<TA> *A, const C<TY> *Cin, const C<TA> *M, C<TY> *Y, long rows, int n,
                         cudaStream_t s) {
  const int bs = 256;
  prof_begin(PROF_AXPY, s);
#define L_AXPY(NN)                                                                           \
  do {                                                                                       \
    constexpr int CG = (NN % 4 == 0) ? 4 : ((NN % 2 == 0) ? 2 : 1);                          \
    const long rpc = (long)(bs / 32) * (32 / (NN / CG));                                     \
    const long grid = std::min<long>((rows + rpc - 1) / rpc, 8 * 152);                      \
    k_block_axpy<TA, TY, NN, CG><<<(unsigned)grid, bs, 0, s>>>(A, Cin, M, Y, rows);          \
  } while (0)
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
                          int s_end, int compute_q, long rows, long fstride, int acc, cudaStream_t s) {
  constexpr int CG = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 1);
  int threads = tune_get(TUNE_UPDATE_THREADS);
  if (threads <= 0 || threads > 256 || threads % 32) threads = 256;  // __launch_bounds__(256)
  const size_t smem = (size_t)((1 + 2 * s_end) - (compute_q ? 0 : 1 + 2 * s_begin)) * N * N * sizeof(C<T>) +
                      (size_t)(threads / 32) * (32 / (N / CG)) * (N + 16 / sizeof(C<T>)) * sizeof(C<T>);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_update_all<T, TX, N, CG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  const long rows_per_cta = (long)(threads / 32) * (32 / (N / CG));
  long grid = (rows + rows_per_cta - 1) / rows_per_cta;
  // persistent grid: as many CTAs as are resident at once (shared memory bound)
  grid = std::min(grid, (long)resident_ctas(k_update_all<T, TX, N, CG>, threads, smem));
  k_update_all<T, TX, N, CG><<<(unsigned)grid, threads, smem, s>>>(W, Q, P, reinterpret_cast<TX *>(X), coef, upd,
                                                                   s_begin, s_end, compute_q, rows, fstride, acc);
}

template <typename T, typename TX>
rhmc_status_t update_all(const C<T> *W, C<T> *Q, C<T> *P, C<TX> *X, const C<T> *coef, const int *upd, int s_begin,
                         int s_end, int compute_q, long rows, int n, long fstride, cudaStream_t s, int acc) {
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
#define L_UPD(NN) launch_update<T, TX, NN>(W, Q, P, X, coef, upd, s_begin, s_end, compute_q, rows, fstride, acc, s)
  RHMC_DISPATCH_N(n, L_UPD)
#undef L_UPD
  prof_end(s, (double)rows * n * ((compute_q ? 2.0 : 1.0) * sizeof(C<T>) + nupd * 2.0 * (sizeof(C<T>) + sizeof(C<TX>))));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template rhmc_status_t update_all<float, float>(const float2 *, float2 *, float2 *, float2 *, const float2 *,
                                                const int *, int, int, int, long, int, long, cudaStream_t, int);
template rhmc_status_t update_all<double, double>(const double2 *, double2 *, double2 *, double2 *, const double2 *,
                                                  const int *, int, int, int, long, int, long, cudaStream_t, int);

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
