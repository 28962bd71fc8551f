// Base-system n x n coefficient steps of SBCGrQ (Algorithm 1: the alpha_k step,
// the block QR, the base updates and delta_k) in double-float arithmetic for the
// mixed-precision solve, and its shifted coefficient step.
//
// The FP64 kernels of small.cu are bound by the FP64 unit: on this GPU a warp
// FP64 instruction holds its sub-partition's FP64 pipe for about 64 cycles, so
// each LDL^dagger step costs a few hundred cycles however few its items.  Here
// every value is an unevaluated pair of floats h + l (|l| <= ulp(h)/2) and the
// arithmetic runs on the FP32 units: products by TwoProduct (an FMA gives the
// rounding error of h_a h_b exactly, Ogita, Rump and Oishi 2005), sums by
// TwoSum (Knuth), about 2^-44 relative per operation.  The mixed solve's Gram
// matrices are sums of FP32 products, so this is far below their own error;
// the FP64 solve keeps the FP64 kernels.  The outputs are those of small.cu:
// the FP64 recursion state (alpha_k, Gram1_k, rho_k, delta_k, the base
// residuals) for the shifted step and the FP32 coefficients of the bulk kernels.
#include "common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace rhmc {
namespace {

struct dd {
  float h, l;
};
struct cd {
  dd r, i;
};

// The _rn intrinsics keep the compiler from contracting the error-free
// transformations into FMAs.
__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return dd{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {  // |a| >= |b| or a = 0
  const float s = __fadd_rn(a, b);
  return dd{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dd dadd(dd a, dd b) {
  const dd s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dd dneg(dd a) { return dd{-a.h, -a.l}; }
__device__ __forceinline__ dd dsub(dd a, dd b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ dd dmul(dd a, dd b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dd dhalf(dd a) { return dd{0.5f * a.h, 0.5f * a.l}; }
// 1/x: r = RN(1/h), then r + r (1 - x r) with 1 - x r formed exactly to first order
__device__ __forceinline__ dd drcp(dd x) {
  const float r = __frcp_rn(x.h);
  const float p = __fmul_rn(x.h, r);
  const float pe = fmaf(x.h, r, -p);
  float e = __fsub_rn(1.0f, p);  // p is within 2^-23 of 1: exact
  e = __fsub_rn(e, pe);
  e = fmaf(-x.l, r, e);
  return fast_two_sum(r, __fmul_rn(r, e));
}
// 1/sqrt(x): y = rsqrt(h), then one Newton step y + y (1 - x y^2) / 2 with the
// residual 1 - x y^2 formed from the exact square of y
__device__ __forceinline__ dd drsqrt(dd x) {
  const float y = rsqrtf(x.h);
  const float y2 = __fmul_rn(y, y);
  const float y2e = fmaf(y, y, -y2);
  const float t = __fmul_rn(x.h, y2);
  float te = fmaf(x.h, y2, -t);
  te = fmaf(x.h, y2e, te);
  te = fmaf(x.l, y2, te);
  float r = __fsub_rn(1.0f, t);
  r = __fsub_rn(r, te);
  return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), r));
}
__device__ __forceinline__ bool dpos(dd a) { return a.h > 0.0f && isfinite(a.h); }

__device__ __forceinline__ cd cconj(cd a) { return cd{a.r, dneg(a.i)}; }
__device__ __forceinline__ cd cscale(cd a, dd s) { return cd{dmul(a.r, s), dmul(a.i, s)}; }
__device__ __forceinline__ cd czero_dd() { return cd{dd{0.f, 0.f}, dd{0.f, 0.f}}; }

// running sums of products (TwoProduct errors and TwoSum errors accumulated in
// one float, folded in at the end)
struct acc_t {
  df::DF r, i;
};
__device__ __forceinline__ acc_t acc_zero() { return acc_t{df::DF{0.f, 0.f}, df::DF{0.f, 0.f}}; }
__device__ __forceinline__ acc_t acc_from(cd v) { return acc_t{df::DF{v.r.h, v.r.l}, df::DF{v.i.h, v.i.l}}; }
// acc += a b
__device__ __forceinline__ void acc_mac(acc_t &acc, cd a, cd b) {
  df::df_add_prod(acc.r, a.r.h, a.r.l, b.r.h, b.r.l);
  df::df_add_prod(acc.r, -a.i.h, -a.i.l, b.i.h, b.i.l);
  df::df_add_prod(acc.i, a.r.h, a.r.l, b.i.h, b.i.l);
  df::df_add_prod(acc.i, a.i.h, a.i.l, b.r.h, b.r.l);
}
// acc += conj(a) b
__device__ __forceinline__ void acc_mac_cj(acc_t &acc, cd a, cd b) {
  df::df_add_prod(acc.r, a.r.h, a.r.l, b.r.h, b.r.l);
  df::df_add_prod(acc.r, a.i.h, a.i.l, b.i.h, b.i.l);
  df::df_add_prod(acc.i, a.r.h, a.r.l, b.i.h, b.i.l);
  df::df_add_prod(acc.i, -a.i.h, -a.i.l, b.r.h, b.r.l);
}
__device__ __forceinline__ cd acc_get(const acc_t &a) {
  const df::DF r = df::df_norm(a.r), i = df::df_norm(a.i);
  return cd{dd{r.h, r.e}, dd{i.h, i.e}};
}

__device__ __forceinline__ dd from_d(double x) {
  const float2 p = df::df_split1(x);
  return dd{p.x, p.y};
}
__device__ __forceinline__ cd from_z(double2 z) { return cd{from_d(z.x), from_d(z.y)}; }
__device__ __forceinline__ double to_d(dd a) { return df::df_merge1(a.h, a.l); }
__device__ __forceinline__ double2 to_z(cd a) { return make_double2(to_d(a.r), to_d(a.i)); }
__device__ __forceinline__ float2 to_f(cd a) { return make_float2(a.r.h, a.i.h); }

constexpr int kNN = 256;  // shared matrix capacity (n <= 16)
constexpr int kS = 16;    // row stride of the shared matrices of the base steps

// LDL^dagger of the Hermitian part of the Gram matrix G (FP64, n x n, row-major)
// in the stride-16 shared matrices, thread t owning entry (i, j) = (t / 16, t % 16)
// (256 threads).  On return the strictly lower part of A holds L (unit lower),
// A[k][k].r the pivot D_k, Li = L^-1 (unit lower) and rd[k] = 1 / D_k; h0 is the
// thread's entry of the Hermitian part.  Step k updates the trailing lower triangle
// (i >= j > k) and rows i > k of L^-1 (j <= k), one entry per thread on one code
// path; the thread on the next diagonal entry forms the next pivot's reciprocal, so
// each step takes one barrier.  Returns false (in all threads) if a pivot is not
// positive and finite.
__device__ bool ldl16(int n, const double2 *G, cd *A, cd *Li, dd *rd, int *flag, cd &h0) {
  const int t = threadIdx.x, i = t >> 4, j = t & 15;
  const bool in = i < n && j < n;
  h0 = czero_dd();
  if (in) {
    const cd a = from_z(G[i * n + j]), b = from_z(G[j * n + i]);
    h0 = (i == j) ? cd{a.r, dd{0.f, 0.f}} : cd{dhalf(dadd(a.r, b.r)), dhalf(dsub(a.i, b.i))};
    A[t] = h0;
    Li[t] = cd{dd{i == j ? 1.f : 0.f, 0.f}, dd{0.f, 0.f}};
  }
  __syncthreads();
  if (t == 0) {
    const dd d = A[0].r;
    *flag = !dpos(d);
    rd[0] = drcp(dpos(d) ? d : dd{1.f, 0.f});
  }
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    if (*flag) return false;
    // A[i][j] -= (A[i][k] / D_k) conj(A[j][k])  (i >= j > k)
    // Li[i][j] -= (A[i][k] / D_k) Li[k][j]      (i > k >= j)
    const bool upd_a = j > k && i >= j;
    if (in && i > k && (upd_a || j <= k)) {
      const cd lik = cscale(A[i * kS + k], dneg(rd[k]));
      cd *X = upd_a ? A : Li;
      const cd y = upd_a ? cconj(A[j * kS + k]) : Li[k * kS + j];
      acc_t v = acc_from(X[t]);
      acc_mac(v, lik, y);
      const cd w = acc_get(v);
      X[t] = w;
      if (i == k + 1 && j == k + 1) {
        *flag = !dpos(w.r);
        rd[k + 1] = drcp(dpos(w.r) ? w.r : dd{1.f, 0.f});
      }
    }
    __syncthreads();
  }
  if (*flag) return false;
  if (in && i > j) A[t] = cscale(A[t], rd[j]);
  __syncthreads();
  return true;
}

// the value of the sum of two running sums (kept apart as independent dependency chains)
__device__ __forceinline__ cd acc_join(const acc_t &a, const acc_t &b) {
  return acc_get(acc_t{df::df_add(a.r, b.r), df::df_add(a.i, b.i)});
}

// ||M e_j|| * scale[j] of an upper-triangular M (stride ld; 16 lanes per column)
__device__ void colnorms_upper_dd(int n, const cd *M, int ld, double *out, const double *scale) {
  const int t = threadIdx.x;
  const int j = t >> 4, i = t & 15;
  df::DF s{0.f, 0.f};
  if (j < n && i <= j) {
    const cd z = M[i * ld + j];
    df::df_add_prod(s, z.r.h, z.r.l, z.r.h, z.r.l);
    df::df_add_prod(s, z.i.h, z.i.l, z.i.h, z.i.l);
  }
  const df::DF sn = df::df_norm(s);
  dd v = dd{sn.h, sn.e};
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    const dd u = dd{__shfl_xor_sync(0xffffffffu, v.h, o, 16), __shfl_xor_sync(0xffffffffu, v.l, o, 16)};
    v = dadd(v, u);
  }
  if (j < n && i == 0) {
    const dd nv = v.h > 0.f ? dmul(v, drsqrt(v)) : dd{0.f, 0.f};
    out[j] = to_d(nv) * scale[j];
  }
}


// Out = op(A) op(B), one element per thread (t < n^2); ca / cb: adjoint of A / B.
// Out may not alias A or B.  Ends with a barrier.
__device__ void mm_dd(int n, cd *Out, const cd *A, const cd *B, bool ca = false, bool cb = false) {
  const int t = threadIdx.x;
  if (t < n * n) {
    const int i = t / n, j = t - (t / n) * n;
    acc_t acc = acc_zero();
    for (int k = 0; k < n; ++k) {
      const cd a = ca ? cconj(A[k * n + i]) : A[i * n + k];
      const cd b = cb ? cconj(B[j * n + k]) : B[k * n + j];
      acc_mac(acc, a, b);
    }
    Out[t] = acc_get(acc);
  }
  __syncthreads();
}

// dst = an FP64 n x n matrix of the state (one element per thread).  Ends with a barrier.
__device__ void stage(int n, cd *dst, const double2 *src) {
  if (threadIdx.x < n * n) dst[threadIdx.x] = from_z(src[threadIdx.x]);
  __syncthreads();
}

// Ai = A^-1 by Gauss-Jordan elimination with partial pivoting (A is destroyed).
// Per pivot step: warp 0 finds the pivot row (largest |a|^2 by the leading floats,
// ties to the lower index), forms the pivot's reciprocal and the elimination
// factors; the rows are swapped and the pivot row scaled; every other row is then
// updated.  Returns false (in all threads) for a zero or non-finite pivot.
__device__ bool inv_general_dd(int n, cd *Ai, cd *A, int *piv, int *flag) {
  const int t = threadIdx.x, nn = n * n;
  __shared__ cd fcol[kMaxN];
  __shared__ cd dinv;
  if (t < nn) Ai[t] = cd{dd{(t / n) == (t % n) ? 1.f : 0.f, 0.f}, dd{0.f, 0.f}};
  if (t == 0) *flag = 0;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (t < 32) {
      const int r = t;
      const cd a = (r < n) ? A[r * n + k] : czero_dd();
      float v = (r >= k && r < n) ? fmaf(a.r.h, a.r.h, a.i.h * a.i.h) : -1.f;
      int idx = r;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const float ov = __shfl_down_sync(0xffffffffu, v, off);
        const int oi = __shfl_down_sync(0xffffffffu, idx, off);
        if (ov > v || (ov == v && oi < idx)) {
          v = ov;
          idx = oi;
        }
      }
      const int p = __shfl_sync(0xffffffffu, idx, 0);
      const float best = __shfl_sync(0xffffffffu, v, 0);
      if (r < n) {  // elimination factor of row r after the swap (row p holds the old row k)
        const int src = (r == p) ? k : r;
        fcol[r] = (r == k) ? czero_dd() : A[src * n + k];
      }
      if (r == 0) {
        *piv = p;
        if (!(best > 0.f) || !isfinite(best)) {
          *flag = 1;
        } else {
          const cd d = A[p * n + k];  // conj(d) / |d|^2
          acc_t m = acc_zero();
          acc_mac_cj(m, d, d);
          const dd rr = drcp(acc_get(m).r);
          dinv = cd{dmul(d.r, rr), dneg(dmul(d.i, rr))};
        }
      }
    }
    __syncthreads();
    if (*flag) return false;
    const int p = *piv;
    if (t < 2 * n) {  // swap rows k and p, scale the new row k
      const int col = t % n;
      cd *M = (t < n) ? A : Ai;
      const cd rk = M[k * n + col], rp = M[p * n + col];
      if (p != k) M[p * n + col] = rk;
      acc_t m = acc_zero();
      acc_mac(m, rp, dinv);
      M[k * n + col] = acc_get(m);
    }
    __syncthreads();
    if (t < nn) {
      const int i = t / n, j = t - (t / n) * n;
      if (i != k) {
        const cd f = fcol[i];
        const cd nf = cd{dneg(f.r), dneg(f.i)};
        acc_t a1 = acc_from(A[t]), a2 = acc_from(Ai[t]);
        acc_mac(a1, nf, A[k * n + j]);
        acc_mac(a2, nf, Ai[k * n + j]);
        A[t] = acc_get(a1);
        Ai[t] = acc_get(a2);
      }
    }
    __syncthreads();
  }
  return true;
}
}  // namespace

// alpha_k step: alpha_k = Gram1^-1 (Hermitian part of Gram1 = P^dagger (A + sigma_0) P)
// = L^-dagger D^-1 L^-1; FP64 alpha_k and Gram1_k into the state, -alpha_k (FP32)
// for the block QR step.  Thread t owns entry (t / 16, t % 16) throughout.
__global__ void __launch_bounds__(256) k_nxn_alpha_dd(const double2 *G, int n, SolverState *st, int k,
                                                      float2 *mw_out) {
  __shared__ cd A[kNN], Li[kNN], S[kNN];
  __shared__ dd rd[kMaxN];
  __shared__ int flag;
  const int cur = k % kSlots;
  const int t = threadIdx.x, i = t >> 4, j = t & 15;
  const bool in = i < n && j < n;
  if (t == 0) st->kabs[cur] = st->kabs[(k - 1) % kSlots] + 1;
  cd h0;
  if (!ldl16(n, G, A, Li, rd, &flag, h0)) {
    if (t == 0) st->breakdown = 2;
    return;
  }
  if (in) S[t] = cscale(Li[t], rd[i]);  // S[q][j] = Li[q][j] / D_q
  __syncthreads();
  // alpha[i][j] = sum_{q >= j} conj(Li[q][i]) S[q][j], i <= j (two running sums)
  if (in && i <= j) {
    acc_t a0 = acc_zero(), a1 = acc_zero();
    int q = j;
    for (; q + 1 < n; q += 2) {
      acc_mac_cj(a0, Li[q * kS + i], S[q * kS + j]);
      acc_mac_cj(a1, Li[(q + 1) * kS + i], S[(q + 1) * kS + j]);
    }
    if (q < n) acc_mac_cj(a0, Li[q * kS + i], S[q * kS + j]);
    const cd v = acc_join(a0, a1);
    const double2 vz = to_z(v);
    const float2 vf = to_f(v);
    st->alpha[cur][i * n + j] = vz;
    mw_out[i * n + j] = make_float2(-vf.x, -vf.y);
    if (i != j) {
      st->alpha[cur][j * n + i] = make_double2(vz.x, -vz.y);
      mw_out[j * n + i] = make_float2(-vf.x, vf.y);
    }
  }
  if (in) st->G1[cur][i * n + j] = to_z(h0);  // Gram1_k (Hermitian part) for the shifted step
}

// block QR and base updates: rho_k = R = D^1/2 L^dagger of the LDL^dagger of W^dagger W (thin QR);
// coef = [rho_k^-1, M1 = alpha_k delta_{k-1}, rho_k^dagger] (FP32); FP64 rho_k,
// delta_k = rho_k delta_{k-1} and the base column residuals into the state.
// Thread t owns entry (t / 16, t % 16) throughout.
__global__ void __launch_bounds__(256) k_nxn_rho_dd(const double2 *G, int n, SolverState *st, int k, float2 *coef) {
  __shared__ cd A[kNN], Li[kNN], Al[kNN], Dp[kNN];
  __shared__ dd rd[kMaxN], sd[kMaxN], rsd[kMaxN];
  __shared__ int flag;
  const int cur = k % kSlots, prev = (k - 1) % kSlots;
  const int t = threadIdx.x, i = t >> 4, j = t & 15, nn = n * n;
  const bool in = i < n && j < n;
  // alpha_k and delta_{k-1} do not depend on the factorisation (ldl16's barriers publish them)
  if (in) {
    Al[t] = from_z(st->alpha[cur][i * n + j]);
    Dp[t] = from_z(st->delta[prev][i * n + j]);
  }
  cd h0;
  if (!ldl16(n, G, A, Li, rd, &flag, h0)) {
    if (t == 0) st->breakdown = 3;
    return;
  }
  if (t < n) {
    const dd d = A[t * kS + t].r;
    const dd y = drsqrt(d);
    rsd[t] = y;
    sd[t] = dmul(d, y);
  }
  __syncthreads();
  cd dk = czero_dd();
  if (in) {
    // R = D^1/2 L^dagger (upper) and R^-1 = L^-dagger D^-1/2 (upper)
    cd r = czero_dd(), ri = czero_dd();
    if (i == j) {
      r.r = sd[i];
      ri.r = rsd[i];
    } else if (i < j) {
      r = cscale(cconj(A[j * kS + i]), sd[i]);
      ri = cscale(cconj(Li[j * kS + i]), rsd[j]);
    }
    st->rho[cur][i * n + j] = to_z(r);
    coef[i * n + j] = to_f(ri);
    coef[2 * nn + j * n + i] = to_f(cconj(r));  // rho^dagger
    // M1[i][j] = sum_{q <= j} alpha[i][q] delta_{k-1}[q][j] (delta_{k-1} upper)
    acc_t m0 = acc_zero(), m1 = acc_zero();
    int q = 0;
    for (; q + 1 <= j; q += 2) {
      acc_mac(m0, Al[i * kS + q], Dp[q * kS + j]);
      acc_mac(m1, Al[i * kS + q + 1], Dp[(q + 1) * kS + j]);
    }
    if (q <= j) acc_mac(m0, Al[i * kS + q], Dp[q * kS + j]);
    coef[nn + i * n + j] = to_f(acc_join(m0, m1));
    // delta_k[i][j] = sum_{i <= q <= j} R[i][q] delta_{k-1}[q][j]
    //              = sd[i] (delta_{k-1}[i][j] + sum_{i < q <= j} conj(L[q][i]) delta_{k-1}[q][j])
    if (i <= j) {
      acc_t d0 = acc_from(Dp[i * kS + j]), d1 = acc_zero();
      q = i + 1;
      for (; q + 1 <= j; q += 2) {
        acc_mac_cj(d0, A[q * kS + i], Dp[q * kS + j]);
        acc_mac_cj(d1, A[(q + 1) * kS + i], Dp[(q + 1) * kS + j]);
      }
      if (q <= j) acc_mac_cj(d0, A[q * kS + i], Dp[q * kS + j]);
      dk = cscale(acc_join(d0, d1), sd[i]);
    }
    st->delta[cur][i * n + j] = to_z(dk);
  }
  __syncthreads();  // A, Li, Al are read above: reuse Li for delta_k
  Li[t] = dk;
  __syncthreads();
  colnorms_upper_dd(n, Li, kS, st->res[0], st->inv_d0);
  if (t == 0) st->upd[0] = 1;
}

// shifted coefficients and updates for shift s = blockIdx.x + 1 (the FP64 k_nxn_shifts of small.cu in
// double-float).  With C = alpha_k rho_{k-1} alpha_{k-1}^-1 (alpha_{k-1}^-1 = Gram1_{k-1})
// and M2_prev = beta^(s)_{k-1} rho_{k-1}^dagger:
//   T = 1 + dsig alpha_k + C rho_{k-1}^dagger - C M2_prev,   beta^(s)_k = T^-1
//   alpha^(s)_k = beta^(s)_k C alpha^(s)_{k-1}
//   M1 = w_s alpha^(s)_k (shifted solution), M2 = beta^(s)_k rho_k^dagger (shifted search block),
//   delta^(s)_k = rho_k alpha_k^-1 alpha^(s)_k (the shifted residual), freezing.
// The recursion state (alpha^(s), M2_prev, the basis history) stays FP64 in memory.
__global__ void __launch_bounds__(256) k_nxn_shifts_dd(int n, int nshift, SolverState *st, int k, float2 *coef,
                                                       double tol_shift, int freeze, double2 *hist, int cap) {
  __shared__ cd Cs[kNN], A1[kNN], A2[kNN], B[kNN], Bi[kNN], S1[kNN], S2[kNN], S3[kNN];
  __shared__ int flag, piv;
  __shared__ float colres[kMaxN];
  const int s = blockIdx.x + 1;
  if (s >= nshift) return;
  const int t = threadIdx.x;
  const int cur = k % kSlots, prev = (k - 1) % kSlots;
  const int nn = n * n;
  if (!st->active[s]) {
    if (t == 0) st->upd[s] = 0;
    return;
  }
  const int kabs = st->kabs[cur];
  const dd dsig = from_d(st->sigma[s] - st->sigma[0]);
  if (t < nn) {
    S1[t] = from_z(st->alpha[cur][t]);
    S2[t] = from_z(st->rho[prev][t]);
    S3[t] = from_z(st->G1[prev][t]);
  }
  __syncthreads();
  mm_dd(n, A1, S1, S2);
  mm_dd(n, Cs, A1, S3);               // C
  mm_dd(n, A2, Cs, S2, false, true);  // C rho_{k-1}^dagger
  stage(n, S3, st->m2_s[s]);
  mm_dd(n, A1, Cs, S3);  // C M2_prev
  if (t < nn) {
    const int i = t / n, j = t - (t / n) * n;
    cd b = cd{dadd(dmul(dsig, S1[t].r), dsub(A2[t].r, A1[t].r)), dadd(dmul(dsig, S1[t].i), dsub(A2[t].i, A1[t].i))};
    if (i == j) b.r = dadd(b.r, dd{1.f, 0.f});
    B[t] = b;
  }
  __syncthreads();
  if (!inv_general_dd(n, Bi, B, &piv, &flag)) {
    if (t == 0) st->breakdown = 4;
    return;
  }
  stage(n, S3, st->alpha_s[s]);
  mm_dd(n, A2, Cs, S3);
  mm_dd(n, A1, Bi, A2);  // alpha^(s)_k
  stage(n, S2, st->rho[cur]);
  mm_dd(n, A2, Bi, S2, false, true);  // beta^(s)_k rho_k^dagger
  const dd w = from_d(st->w1[s]);
  if (t < nn) {
    coef[(1 + 2 * s) * nn + t] = to_f(cscale(A1[t], w));
    coef[(2 + 2 * s) * nn + t] = to_f(A2[t]);
    const double2 a1 = to_z(A1[t]), a2 = to_z(A2[t]);
    st->m2_s[s][t] = a2;
    st->alpha_s[s][t] = a1;
    if (hist && kabs < cap) {
      double2 *h = hist + ((size_t)kabs * nshift + s) * 2 * nn;
      h[t] = a1;
      h[nn + t] = a2;
    }
  }
  if (t == 0) st->last_k[s] = kabs;
  stage(n, S3, st->G1[cur]);
  mm_dd(n, Cs, S2, S3);
  mm_dd(n, B, Cs, A1);  // delta^(s)_k
  if (t < n) {
    df::DF q{0.f, 0.f};
    for (int i = 0; i < n; ++i) {
      const cd z = B[i * n + t];
      df::df_add_prod(q, z.r.h, z.r.l, z.r.h, z.r.l);
      df::df_add_prod(q, z.i.h, z.i.l, z.i.h, z.i.l);
    }
    const df::DF qn = df::df_norm(q);
    const dd v{qn.h, qn.e};
    const dd nv = v.h > 0.f ? dmul(v, drsqrt(v)) : dd{0.f, 0.f};
    const double r = to_d(nv) * st->inv_d0[t];
    colres[t] = (float)r;
    st->res[s][t] = r;
  }
  __syncthreads();
  if (t == 0) {
    float mx = 0.f;
    for (int j = 0; j < n; ++j) mx = fmaxf(mx, colres[j]);
    st->upd[s] = 1;
    if (freeze && (double)mx < tol_shift) st->active[s] = 0;
  }
}

rhmc_status_t nxn_shifts_dd(int n, int nshift, SolverState *st, int k, float2 *coef, double tol_shift, int freeze,
                            double2 *hist, int cap, cudaStream_t s) {
  prof_begin(PROF_NXN_SHIFTS, s);
  k_nxn_shifts_dd<<<nshift - 1, 256, 0, s>>>(n, nshift, st, k, coef, tol_shift, freeze, hist, cap);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t nxn_alpha_dd(const double2 *gram, int n, SolverState *st, int k, float2 *mw, cudaStream_t s) {
  prof_begin(PROF_NXN, s);
  k_nxn_alpha_dd<<<1, 256, 0, s>>>(gram, n, st, k, mw);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t nxn_rho_dd(const double2 *gram, int n, SolverState *st, int k, float2 *coef, cudaStream_t s) {
  prof_begin(PROF_NXN, s);
  k_nxn_rho_dd<<<1, 256, 0, s>>>(gram, n, st, k, coef);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// ------------------------------------------------------------ self-test of the double-float helpers
__global__ void k_df_helpers(const double *__restrict__ x, const double *__restrict__ y, int count,
                             double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const double a = x[k], b = y[k];
  const dd da = from_d(a), db = from_d(b);
  const size_t c = (size_t)count;
  out[0 * c + k] = (double)da.h;  // the split: hi = RN_float(a)
  out[1 * c + k] = (double)da.l;  //            lo = RN_float(a - hi)
  out[2 * c + k] = to_d(da);      // hi + lo in FP64
  out[3 * c + k] = to_d(dadd(da, db));
  out[4 * c + k] = to_d(dmul(da, db));
  out[5 * c + k] = to_d(drcp(da));
  out[6 * c + k] = a > 0.0 ? to_d(drsqrt(da)) : 0.0;
  df::DF acc{0.f, 0.f};  // running sum of products, as the double-float hop and force form them
  df::df_add_prod(acc, da.h, da.l, db.h, db.l);
  df::df_add_prod(acc, db.h, db.l, db.h, db.l);
  const df::DF an = df::df_norm(acc);
  out[7 * c + k] = to_d(dd{an.h, an.e});
}

}  // namespace rhmc

extern "C" rhmc_status_t rhmc_selftest_df_helpers(const double *x_dev, const double *y_dev, int count,
                                                  double *out_dev, rhmc_stream_t sv) {
  using namespace rhmc;
  if (!x_dev || !y_dev || !out_dev || count < 1) {
    set_error("rhmc_selftest_df_helpers: null pointer or count < 1");
    return RHMC_ERR_INVALID_ARG;
  }
  k_df_helpers<<<(count + 255) / 256, 256, 0, (cudaStream_t)sv>>>(x_dev, y_dev, count, out_dev);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
