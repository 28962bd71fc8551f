// n x n coefficient algebra of SBCGrQ (Algorithm 1), FP64, on the device.
//
// A CTA of 256 threads works on n x n complex matrices (n <= 16) held in
// shared memory.  On this GPU an FP64 warp instruction occupies its SM
// sub-partition's FP64 unit for about 64 cycles however many lanes are active,
// and a dependent FP64 operation waits as long; the base-system kernels
// therefore hand each step's work items to the fewest warps (items are packed
// by index, not owned by element), exploit every triangular and Hermitian
// structure, and keep one barrier per factorisation step.  The shifted step
// (one CTA per shift) keeps the simpler element-per-thread form.  The state of the
// recursion lives in a SolverState in device memory; quantities of iteration
// k are written to slot k % 3 and those of k-1 read from slot (k-1) % 3, so a
// launch never overwrites what a launch still running on the other stream reads.
//
//   qr_init   {Q_0, delta_0} = qr(B) by Cholesky of B^dagger B   (initialisation)
//   alpha     alpha_k = (P^dagger (A + sigma_0) P)^-1            (alpha_k step)
//   rho       rho_k from the Cholesky of W^dagger W (thin QR),     (block QR, base updates,
//             base coefficients alpha_k delta_{k-1}, rho_k^dagger,  delta_k)
//             delta_k
//   shifts    beta^(s)_k, alpha^(s)_k and the coefficients of      (shifted coefficients
//             the shifted updates, one CTA per shift; shifted       and updates)
//             residual
//             delta^(s)_k = rho_k alpha_k^-1 alpha^(s)_k (Sec. III), freezing
//   reliable  delta_k replaced by the R factor of the true residual
#include "common.cuh"
#include "kernels.h"

namespace rhmc {

namespace {

struct Cta {
  int n, t, i, j;
  bool own;
  __device__ Cta(int n_) : n(n_), t(threadIdx.x), i(threadIdx.x / n_), j(threadIdx.x % n_), own(threadIdx.x < n_ * n_) {}
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmulz(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 conjz(double2 a) { return make_double2(a.x, -a.y); }
// FP64 reciprocal and square root without the long IEEE sequences (FP64 is
// latency-bound here): an FP32 estimate of the scaled mantissa refined by
// Newton-Raphson in FP64, r <- r + r (1 - x r) for 1/x, and
// y <- y (3 - x y^2) / 2 for 1/sqrt(x) followed by s <- s + y (x - s^2) / 2.
// Two (three) steps take the 2^-23 estimate to full double precision.
__device__ __forceinline__ double frcp(double x) {
  int e;
  const double m = frexp(x, &e);
  double r = ldexp((double)__frcp_rn((float)m), -e);
  double err = fma(-x, r, 1.0);
  r = fma(r, err, r);
  err = fma(-x, r, 1.0);
  return fma(r, err, r);
}
__device__ __forceinline__ double fsqrt(double x) {
  if (!(x > 0.0)) return 0.0;
  int e;
  double m = frexp(x, &e);  // x = m 2^e, m in [0.5, 1)
  if (e & 1) {
    m *= 2.0;
    e -= 1;
  }
  double y = (double)rsqrtf((float)m);
  y = y * fma(-0.5 * m * y, y, 1.5);
  y = y * fma(-0.5 * m * y, y, 1.5);
  double sq = m * y;
  sq = fma(0.5 * y, fma(-sq, sq, m), sq);
  return ldexp(sq, e / 2);
}
// a / b = a conj(b) / |b|^2
__device__ __forceinline__ double2 cdivz(double2 a, double2 b) {
  const double r = frcp(b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * r, (a.y * b.x - a.x * b.y) * r);
}
__device__ __forceinline__ double2 cscale(double2 a, double r) { return make_double2(a.x * r, a.y * r); }

// C = op(A) op(B); ca / cb: use the adjoint of A / B.  C may not alias A or B.
__device__ void mm(const Cta &c, double2 *Cm, const double2 *A, const double2 *B, bool ca = false, bool cb = false) {
  if (c.own) {
    double2 acc = make_double2(0, 0);
    for (int k = 0; k < c.n; ++k) {
      const double2 a = ca ? conjz(A[k * c.n + c.i]) : A[c.i * c.n + k];
      const double2 b = cb ? conjz(B[c.j * c.n + k]) : B[k * c.n + c.j];
      acc = cadd(acc, cmulz(a, b));
    }
    Cm[c.t] = acc;
  }
  __syncthreads();
}

__device__ void copy(const Cta &c, double2 *D, const double2 *S) {
  if (c.own) D[c.t] = S[c.t];
  __syncthreads();
}

__device__ void set_eye(const Cta &c, double2 *D) {
  if (c.own) D[c.t] = make_double2(c.i == c.j ? 1.0 : 0.0, 0.0);
  __syncthreads();
}

// Sum the per-cluster partials of a Gram matrix into G (8 loads in flight per thread).
__device__ void reduce_partials(const Cta &c, double2 *G, const double2 *partial, int nparts) {
  if (c.own) {
    const int nn = c.n * c.n;
    double2 acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = make_double2(0, 0);
    int p = 0;
    for (; p + 8 <= nparts; p += 8) {
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = cadd(acc[q], partial[(long)(p + q) * nn + c.t]);
    }
    for (; p < nparts; ++p) acc[0] = cadd(acc[0], partial[(long)p * nn + c.t]);
    double2 sum = acc[0];
#pragma unroll
    for (int q = 1; q < 8; ++q) sum = cadd(sum, acc[q]);
    G[c.t] = sum;
  }
  __syncthreads();
}

// In-place Cholesky A = L L^dagger (lower, positive real diagonal).  The Gram
// matrix is symmetrised first.  Returns false (for all threads) if A is not
// numerically positive definite.
__device__ bool cholesky(const Cta &c, double2 *A, int *flag) {
  const int n = c.n;
  double2 h = make_double2(0, 0);
  if (c.own) h = (c.i == c.j) ? make_double2(A[c.t].x, 0.0)
                              : make_double2(0.5 * (A[c.t].x + A[c.j * n + c.i].x),
                                             0.5 * (A[c.t].y - A[c.j * n + c.i].y));
  __syncthreads();
  if (c.own) A[c.t] = h;
  if (c.t == 0) *flag = 0;
  __syncthreads();
  __shared__ double rpiv;
  for (int k = 0; k < n; ++k) {
    if (c.t == 0) {
      const double d = A[k * n + k].x;
      if (!(d > 0.0) || !isfinite(d)) *flag = 1;
      const double sd = fsqrt(fmax(d, 0.0));
      A[k * n + k] = make_double2(sd, 0.0);
      rpiv = frcp(sd);
    }
    __syncthreads();
    if (*flag) return false;
    if (c.t > k && c.t < n) A[c.t * n + k] = cscale(A[c.t * n + k], rpiv);
    __syncthreads();
    if (c.own && c.i > k && c.j > k && c.j <= c.i)
      A[c.t] = csub(A[c.t], cmulz(A[c.i * n + k], conjz(A[c.j * n + k])));
    __syncthreads();
  }
  if (c.own && c.j > c.i) A[c.t] = make_double2(0, 0);
  __syncthreads();
  return true;
}

// Inverse of an upper-triangular R (R^-1 upper).  Thread j < n owns column j.
// The diagonal of R is real and positive (Cholesky factors).
__device__ void inv_upper(const Cta &c, double2 *Ri, const double2 *R) {
  const int n = c.n;
  __shared__ double rd[kMaxN];
  if (c.own) Ri[c.t] = make_double2(0, 0);
  if (c.t < n) rd[c.t] = frcp(R[c.t * n + c.t].x);
  __syncthreads();
  if (c.t < n) {
    const int j = c.t;
    for (int i = j; i >= 0; --i) {
      double2 s = make_double2(i == j ? 1.0 : 0.0, 0.0);
      for (int k = i + 1; k <= j; ++k) s = csub(s, cmulz(R[i * n + k], Ri[k * n + j]));
      Ri[i * n + j] = cscale(s, rd[i]);
    }
  }
  __syncthreads();
}

// General inverse by Gauss-Jordan with partial pivoting.  A is destroyed.
// Ai = A^-1 by Gauss-Jordan elimination with partial pivoting (A is destroyed).
// Per pivot step: warp 0 finds the pivot row by a shuffle reduction, forms the
// pivot reciprocal and the column of elimination factors; the rows are swapped
// and the pivot row scaled; every other row is then updated from the factor
// column and the pivot row.  Three barriers per step.
__device__ bool inv_general(const Cta &c, double2 *Ai, double2 *A, int *piv, int *flag) {
  const int n = c.n;
  __shared__ double2 fcol[kMaxN];
  __shared__ double2 dinv;
  set_eye(c, Ai);
  for (int k = 0; k < n; ++k) {
    if (c.t < 32) {
      const int r = c.t;
      const double2 a = (r < n) ? A[r * n + k] : make_double2(0.0, 0.0);
      double v = (r >= k && r < n) ? a.x * a.x + a.y * a.y : -1.0;
      int idx = r;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, v, off);
        const int oi = __shfl_down_sync(0xffffffffu, idx, off);
        if (ov > v || (ov == v && oi < idx)) {
          v = ov;
          idx = oi;
        }
      }
      const int p = __shfl_sync(0xffffffffu, idx, 0);
      const double best = __shfl_sync(0xffffffffu, v, 0);
      // elimination factor of row r after the swap: row p holds the old row k
      const double2 akk = make_double2(__shfl_sync(0xffffffffu, a.x, k), __shfl_sync(0xffffffffu, a.y, k));
      if (r < n) fcol[r] = (r == k) ? make_double2(0.0, 0.0) : (r == p ? akk : a);
      if (r == 0) {
        *piv = p;
        if (!(best > 0.0) || !isfinite(best)) {
          *flag = 1;
        } else {
          const double2 d = (p == k) ? akk : A[p * n + k];
          const double rr = frcp(best);
          dinv = make_double2(d.x * rr, -d.y * rr);
        }
      }
    }
    __syncthreads();
    if (*flag) return false;
    const int p = *piv;
    if (c.t < 2 * n) {  // swap rows k and p, scale the new row k
      const int col = c.t % n;
      double2 *M = (c.t < n) ? A : Ai;
      const double2 rk = M[k * n + col], rp = M[p * n + col];
      if (p != k) M[p * n + col] = rk;
      M[k * n + col] = cmulz(rp, dinv);
    }
    __syncthreads();
    if (c.own && c.i != k) {
      const double2 f = fcol[c.i];
      A[c.t] = csub(A[c.t], cmulz(f, A[k * n + c.j]));
      Ai[c.t] = csub(Ai[c.t], cmulz(f, Ai[k * n + c.j]));
    }
    __syncthreads();
  }
  return true;
}

__device__ double colnorm(const Cta &c, const double2 *A, int j) {
  double s0 = 0.0, s1 = 0.0;
  for (int i = 0; i < c.n; ++i) {
    s0 = fma(A[i * c.n + j].x, A[i * c.n + j].x, s0);
    s1 = fma(A[i * c.n + j].y, A[i * c.n + j].y, s1);
  }
  return fsqrt(s0 + s1);
}

template <typename T>
__device__ void store_coef(const Cta &c, C<T> *dst, const double2 *M, double scale = 1.0) {
  if (c.own) dst[c.t] = mk<T>((T)(scale * M[c.t].x), (T)(scale * M[c.t].y));
}

// 1/x for x > 0: FP32 estimate refined by two Newton-Raphson steps
// r <- r + r (1 - x r) in FP64 (the estimate's 2^-23 error squares twice);
// the exponent is split off only when x is outside the FP32 range.
__device__ __forceinline__ double frcp_fast(double x) {
  if (!(x > 1e-30 && x < 1e30)) return frcp(x);
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}
// 1/sqrt(x) for x > 0: Newton-Raphson y <- y (3 - x y^2) / 2 from an FP32 estimate.
__device__ __forceinline__ double frsqrt(double x) {
  int e = 0;
  double m = x;
  if (!(x > 1e-30 && x < 1e30)) {
    m = frexp(x, &e);
    if (e & 1) {
      m *= 2.0;
      e -= 1;
    }
  }
  const double h = 0.5 * m;
  double y = (double)rsqrtf((float)m);
  y = y * fma(-h * y, y, 1.5);
  y = y * fma(-h * y, y, 1.5);
  return e ? ldexp(y, -e / 2) : y;
}

// Index of row a of a packed lower triangle (a (a+1)/2 <= e < (a+1)(a+2)/2).
__device__ __forceinline__ int tri_row(int e) {
  int a = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
  while ((a + 1) * (a + 2) / 2 <= e) ++a;
  while (a * (a + 1) / 2 > e) --a;
  return a;
}

// LDL^dagger factorisation of the Hermitian positive definite A (n x n, full
// storage in shared memory, its Hermitian part is used).  On return the
// strictly lower part of A holds L (unit lower), A[k][k].x holds D_k,
// Li = L^-1 (unit lower, full storage) and rd[k] = 1 / D_k.  Step k updates
// the trailing lower triangle and rows k+1.. of L^-1 as one list of work
// items; the item on the next diagonal entry also forms the next pivot's
// reciprocal, so each step needs one barrier.  Returns false (in all threads)
// if a pivot is not positive and finite.
__device__ bool ldl(int n, double2 *A, double2 *Li, double *rd, int *flag) {
  const int t = threadIdx.x, nt = blockDim.x, nn = n * n;
  double2 h = make_double2(0, 0);
  if (t < nn) {
    const int i = t / n, j = t - (t / n) * n;
    const double2 a = A[t], b = A[j * n + i];
    h = (i == j) ? make_double2(a.x, 0.0) : make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
  __syncthreads();
  if (t < nn) {
    const int i = t / n, j = t - (t / n) * n;
    A[t] = h;
    Li[t] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (t == 0) {
    const double d = h.x;
    *flag = !(d > 0.0) || !isfinite(d);
    rd[0] = frcp_fast(d > 0.0 ? d : 1.0);
  }
  __syncthreads();
  for (int k = 0; k + 1 < n; ++k) {
    if (*flag) return false;
    const double r = rd[k];
    const int m = n - 1 - k;
    const int ntri = m * (m + 1) / 2, nli = m * (k + 1);
    for (int e = t; e < ntri + nli; e += nt) {
      if (e < ntri) {
        // A[i][j] -= A[i][k] conj(A[j][k]) / D_k,  i >= j > k
        const int a = tri_row(e), b = e - a * (a + 1) / 2;
        const int i = k + 1 + a, j = k + 1 + b;
        const double2 aik = A[i * n + k], ajk = A[j * n + k];
        double2 v = A[i * n + j];
        const double px = fma(aik.x, ajk.x, aik.y * ajk.y), py = fma(aik.y, ajk.x, -aik.x * ajk.y);
        v.x = fma(-px, r, v.x);
        v.y = fma(-py, r, v.y);
        A[i * n + j] = v;
        if (i == k + 1 && j == k + 1) {
          *flag = !(v.x > 0.0) || !isfinite(v.x);
          rd[k + 1] = frcp_fast(v.x > 0.0 ? v.x : 1.0);
        }
      } else {
        // Li[i][j] -= L[i][k] Li[k][j],  i > k >= j,  L[i][k] = A[i][k] / D_k
        const int e2 = e - ntri;
        const int a = e2 / (k + 1), j = e2 - a * (k + 1);
        const int i = k + 1 + a;
        const double2 aik = A[i * n + k], lkj = Li[k * n + j];
        const double lx = aik.x * r, ly = aik.y * r;
        double2 v = Li[i * n + j];
        v.x -= fma(lx, lkj.x, -ly * lkj.y);
        v.y -= fma(lx, lkj.y, ly * lkj.x);
        Li[i * n + j] = v;
      }
    }
    __syncthreads();
  }
  if (*flag) return false;
  for (int e = t; e < nn; e += nt) {
    const int i = e / n, j = e - (e / n) * n;
    if (i > j) A[e] = cscale(A[e], rd[j]);
  }
  __syncthreads();
  return true;
}

// From an LDL^dagger factorisation: the thin-QR factor R = D^1/2 L^dagger
// (upper, positive real diagonal) and R^-1 = L^-dagger D^-1/2 (upper), full
// storage with zero lower parts.  sd, rsd: scratch for D^1/2 and D^-1/2.
__device__ void qr_factors(int n, const double2 *A, const double2 *Li, double2 *R, double2 *Ri, double *sd,
                           double *rsd) {
  const int t = threadIdx.x, nt = blockDim.x, nn = n * n;
  if (t < n) {
    const double d = A[t * n + t].x;
    const double y = frsqrt(d);
    rsd[t] = y;
    sd[t] = d * y;
  }
  __syncthreads();
  for (int e = t; e < nn; e += nt) {
    const int i = e / n, j = e - (e / n) * n;
    double2 r = make_double2(0, 0), ri = make_double2(0, 0);
    if (i == j) {
      r = make_double2(sd[i], 0.0);
      ri = make_double2(rsd[i], 0.0);
    } else if (i < j) {
      const double2 l = A[j * n + i], li = Li[j * n + i];  // conj(L[j][i]), conj(Li[j][i])
      r = make_double2(sd[i] * l.x, -sd[i] * l.y);
      ri = make_double2(li.x * rsd[j], -li.y * rsd[j]);
    }
    R[e] = r;
    Ri[e] = ri;
  }
  __syncthreads();
}

// Column norms of an upper-triangular n x n matrix M: 16 lanes per column,
// shuffle reduction; writes out[j] = ||M e_j|| * scale[j] (scale may be null).
__device__ void colnorms_upper(int n, const double2 *M, double *out, const double *scale, double *norm_out) {
  const int t = threadIdx.x;
  const int j = t >> 4, i = t & 15;
  double v = 0.0;
  if (j < n && i <= j) {
    const double2 z = M[i * n + j];
    v = fma(z.x, z.x, z.y * z.y);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, 16);
  if (j < n && i == 0) {
    const double nv = v > 0.0 ? v * frsqrt(v) : 0.0;
    if (norm_out) norm_out[j] = nv;
    if (out) out[j] = scale ? nv * scale[j] : nv;
  }
}

#define NN 256  // shared matrix capacity (n <= 16)

}  // namespace

// ------------------------------------------------------------ kernels

// initialisation: {Q_0, delta_0} = qr(B): delta_0 = R of the Cholesky QR of B^dagger B;
// writes delta_0^-1 (for Q_0 = B delta_0^-1) and initialises the state.
template <typename T>
__global__ void __launch_bounds__(256) k_qr_init(const double2 *partial, int nparts, int n, int nshift,
                                                 SolverState *st, C<T> *rinv_out) {
  __shared__ double2 A[NN], Li[NN], R[NN], Ri[NN];
  __shared__ double rd[kMaxN], sd[kMaxN], rsd[kMaxN], nrm[kMaxN];
  __shared__ int flag;
  Cta c(n);
  reduce_partials(c, A, partial, nparts);
  if (!ldl(n, A, Li, rd, &flag)) {
    if (c.t == 0) st->breakdown = 1;
    return;
  }
  qr_factors(n, A, Li, R, Ri, sd, rsd);
  store_coef<T>(c, rinv_out, Ri);
  colnorms_upper(n, R, nullptr, nullptr, nrm);
  __syncthreads();
  if (c.own) {
    st->delta[0][c.t] = R[c.t];
    st->rho[0][c.t] = R[c.t];
    const double2 e = make_double2(c.i == c.j ? 1.0 : 0.0, 0.0);
    st->alpha[0][c.t] = e;
    st->G1[0][c.t] = e;
    const double2 rh = R[c.j * n + c.i];  // beta^(s)_0 rho_0^dagger = delta_0^dagger (beta^(s)_0 = 1)
    for (int s = 0; s < nshift; ++s) {
      st->m2_s[s][c.t] = make_double2(rh.x, -rh.y);
      st->alpha_s[s][c.t] = e;
    }
  }
  if (c.t < n) {
    st->d0[c.t] = nrm[c.t];
    st->inv_d0[c.t] = frcp_fast(nrm[c.t] > 0.0 ? nrm[c.t] : 1.0);
  }
  if (c.t < kSlots) st->kabs[c.t] = 0;
  if (c.t < nshift) {
    st->last_k[c.t] = 0;
    st->active[c.t] = 1;
    st->upd[c.t] = 0;
    st->w1[c.t] = 1.0;
    for (int j = 0; j < n; ++j) st->res[c.t][j] = 1.0;
  }
  if (c.t == 0) {
    st->breakdown = 0;
    st->device_timeout = 0;
  }
}

// alpha_k step: alpha_k = Gram1^-1, Gram1 = P^dagger (A + sigma_0) P (Hermitian part),
// from Gram1 = L D L^dagger: alpha = L^-dagger D^-1 L^-1, only i <= j formed;
// also -alpha for the block QR step.
template <typename T>
__global__ void __launch_bounds__(256) k_nxn_alpha(const double2 *partial, int nparts, int n, SolverState *st, int k,
                                                   C<T> *mw_out) {
  __shared__ double2 A[NN], Li[NN], S[NN];
  __shared__ double rd[kMaxN];
  __shared__ int flag;
  Cta c(n);
  const int cur = k % kSlots;
  const int t = c.t, nt = blockDim.x, nn = n * n;
  reduce_partials(c, A, partial, nparts);
  if (t == 0) st->kabs[cur] = st->kabs[(k - 1) % kSlots] + 1;
  // Gram1_k (Hermitian part) for the shifted step
  if (c.own) {
    const double2 a = A[t], b = A[c.j * n + c.i];
    st->G1[cur][t] = (c.i == c.j) ? make_double2(a.x, 0.0) : make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  }
  if (!ldl(n, A, Li, rd, &flag)) {
    if (t == 0) st->breakdown = 2;
    return;
  }
  // S[k][j] = Li[k][j] / D_k
  for (int e = t; e < nn; e += nt) {
    const int kk = e / n;
    S[e] = cscale(Li[e], rd[kk]);
  }
  __syncthreads();
  // alpha[i][j] = sum_{q >= j} conj(Li[q][i]) S[q][j], i <= j (column-major packing)
  for (int e = t; e < n * (n + 1) / 2; e += nt) {
    const int j = tri_row(e), i = e - j * (j + 1) / 2;
    double ax = 0.0, ay = 0.0;
    for (int q = j; q < n; ++q) {
      const double2 l = Li[q * n + i], sv = S[q * n + j];
      ax = fma(l.x, sv.x, fma(l.y, sv.y, ax));
      ay = fma(l.x, sv.y, fma(-l.y, sv.x, ay));
    }
    const double2 v = make_double2(ax, ay), vc = make_double2(ax, -ay);
    st->alpha[cur][i * n + j] = v;
    mw_out[i * n + j] = mk<T>((T)(-ax), (T)(-ay));
    if (i != j) {
      st->alpha[cur][j * n + i] = vc;
      mw_out[j * n + i] = mk<T>((T)(-ax), (T)(ay));
    }
  }
}

// block QR and base updates: rho_k = R factor of the Cholesky QR of W^dagger W; base
// coefficients rho_k^-1 (Q_k = W rho_k^-1), M1 = alpha_k delta_{k-1} (base solution),
// M2 = rho_k^dagger (base search block); delta_k = rho_k delta_{k-1} and the base column
// residuals.
template <typename T>
__global__ void __launch_bounds__(256) k_nxn_rho(const double2 *partial, int nparts, int n, SolverState *st, int k,
                                                 C<T> *coef) {
  __shared__ double2 A[NN], Li[NN], R[NN], Ri[NN];
  __shared__ double rd[kMaxN], sd[kMaxN], rsd[kMaxN];
  __shared__ int flag;
  Cta c(n);
  const int cur = k % kSlots, prev = (k - 1) % kSlots;
  const int t = c.t, nt = blockDim.x, nn = n * n;
  reduce_partials(c, A, partial, nparts);
  if (!ldl(n, A, Li, rd, &flag)) {
    if (t == 0) st->breakdown = 3;
    return;
  }
  qr_factors(n, A, Li, R, Ri, sd, rsd);
  // A, Li are free now: alpha_k and delta_{k-1} into shared memory
  double2 *Al = A, *Dp = Li;
  if (c.own) {
    Al[t] = st->alpha[cur][t];
    Dp[t] = st->delta[prev][t];
    st->rho[cur][t] = R[t];
  }
  store_coef<T>(c, coef, Ri);
  if (c.own) coef[2 * nn + t] = mk<T>((T)R[c.j * n + c.i].x, (T)(-R[c.j * n + c.i].y));  // rho^dagger
  __syncthreads();
  // M1[i][j] = sum_{q <= j} alpha[i][q] delta[q][j] (n^2 items, column-major so a
  // warp's items share their length); delta_k[i][j] = sum_{i <= q <= j} rho[i][q] delta[q][j]
  double2 *Dk = Ri;  // Ri was stored above
  for (int e = t; e < nn + n * (n + 1) / 2; e += nt) {
    if (e < nn) {
      const int j = e / n, i = e - (e / n) * n;
      double ax = 0.0, ay = 0.0;
      for (int q = 0; q <= j; ++q) {
        const double2 a = Al[i * n + q], d = Dp[q * n + j];
        ax = fma(a.x, d.x, fma(-a.y, d.y, ax));
        ay = fma(a.x, d.y, fma(a.y, d.x, ay));
      }
      coef[nn + i * n + j] = mk<T>((T)ax, (T)ay);
    } else {
      const int e2 = e - nn;
      const int j = tri_row(e2), i = e2 - j * (j + 1) / 2;
      double ax = 0.0, ay = 0.0;
      for (int q = i; q <= j; ++q) {
        const double2 a = R[i * n + q], d = Dp[q * n + j];
        ax = fma(a.x, d.x, fma(-a.y, d.y, ax));
        ay = fma(a.x, d.y, fma(a.y, d.x, ay));
      }
      Dk[i * n + j] = make_double2(ax, ay);
      if (i != j) Dk[j * n + i] = make_double2(0.0, 0.0);
    }
  }
  __syncthreads();
  if (c.own) st->delta[cur][t] = Dk[t];
  colnorms_upper(n, Dk, st->res[0], st->inv_d0, nullptr);
  if (t == 0) st->upd[0] = 1;
}
// shifted coefficients and updates for shift s = blockIdx.x + 1.  With
// C = alpha_k rho_{k-1} alpha_{k-1}^-1 and M2_prev = beta^(s)_{k-1} rho_{k-1}^dagger (kept in FP64 from the last update):
//   T = 1 + dsig alpha_k + C (1 - beta^(s)_{k-1}) rho_{k-1}^dagger
//     = 1 + dsig alpha_k + C rho_{k-1}^dagger - C M2_prev,      beta^(s)_k = T^-1
//   alpha^(s)_k = beta^(s)_k C alpha^(s)_{k-1}
//   M1 = alpha^(s)_k (shifted solution), M2 = beta^(s)_k rho_k^dagger (shifted search block),
//   delta^(s)_k = rho_k alpha_k^-1 alpha^(s)_k (the shifted residual).
// Nine n x n products and one inverse per shift.
template <typename T>
__global__ void __launch_bounds__(256) k_nxn_shifts(int n, int nshift, SolverState *st, int k, C<T> *coef,
                                                    double tol_shift, int freeze, double2 *hist, int cap) {
  __shared__ double2 Cs[NN], A1[NN], A2[NN], B[NN], Bi[NN];
  __shared__ int flag, piv;
  Cta c(n);
  const int s = blockIdx.x + 1;
  if (s >= nshift) return;
  const int cur = k % kSlots, prev = (k - 1) % kSlots;
  const int nn = n * n;
  if (!st->active[s]) {
    if (c.t == 0) st->upd[s] = 0;
    return;
  }
  if (c.t == 0) flag = 0;
  const int kabs = st->kabs[cur];
  const double dsig = st->sigma[s] - st->sigma[0];
  mm(c, A1, st->alpha[cur], st->rho[prev]);
  mm(c, Cs, A1, st->G1[prev]);                        // C
  mm(c, A2, Cs, st->rho[prev], false, true);          // C rho_{k-1}^dagger
  mm(c, A1, Cs, st->m2_s[s]);                         // C M2_prev
  if (c.own) {
    const double2 a = st->alpha[cur][c.t];
    B[c.t] = make_double2((c.i == c.j ? 1.0 : 0.0) + dsig * a.x + A2[c.t].x - A1[c.t].x,
                          dsig * a.y + A2[c.t].y - A1[c.t].y);
  }
  __syncthreads();
  if (!inv_general(c, Bi, B, &piv, &flag)) {
    if (c.t == 0) st->breakdown = 4;
    return;
  }
  mm(c, A2, Cs, st->alpha_s[s]);
  mm(c, A1, Bi, A2);  // alpha^(s)_k
  store_coef<T>(c, coef + (1 + 2 * s) * nn, A1, st->w1[s]);
  mm(c, A2, Bi, st->rho[cur], false, true);  // beta^(s)_k rho_k^dagger
  store_coef<T>(c, coef + (2 + 2 * s) * nn, A2);
  if (c.own) {
    st->m2_s[s][c.t] = A2[c.t];
    st->alpha_s[s][c.t] = A1[c.t];
    if (hist && kabs < cap) {
      double2 *h = hist + ((size_t)kabs * nshift + s) * 2 * nn;
      h[c.t] = A1[c.t];
      h[nn + c.t] = A2[c.t];
    }
  }
  if (c.t == 0) st->last_k[s] = kabs;
  mm(c, Cs, st->rho[cur], st->G1[cur]);
  mm(c, B, Cs, A1);  // delta^(s)_k
  __shared__ double colres[kMaxN];
  if (c.t < n) {
    const double r = colnorm(c, B, c.t) * st->inv_d0[c.t];
    colres[c.t] = r;
    st->res[s][c.t] = r;
  }
  __syncthreads();
  if (c.t == 0) {
    double mx = 0.0;
    for (int j = 0; j < n; ++j) mx = fmax(mx, colres[j]);
    st->upd[s] = 1;
    if (freeze && mx < tol_shift) st->active[s] = 0;
  }
}

// Reliable update: delta_k <- R factor of the true residual (Gram of R^dagger R);
// writes (delta')^-1 for Q = R (delta')^-1.
template <typename T>
__global__ void __launch_bounds__(256) k_nxn_reliable(const double2 *partial, int nparts, int n, SolverState *st,
                                                      int k, C<T> *rinv_out) {
  __shared__ double2 A[NN], Li[NN], R[NN], Ri[NN];
  __shared__ double rd[kMaxN], sd[kMaxN], rsd[kMaxN];
  __shared__ int flag;
  Cta c(n);
  const int cur = k % kSlots;
  reduce_partials(c, A, partial, nparts);
  if (!ldl(n, A, Li, rd, &flag)) {
    if (c.t == 0) st->breakdown = 5;
    return;
  }
  qr_factors(n, A, Li, R, Ri, sd, rsd);
  if (c.own) st->delta[cur][c.t] = R[c.t];
  store_coef<T>(c, rinv_out, Ri);
  colnorms_upper(n, R, st->res[0], st->inv_d0, nullptr);
}

// ------------------------------------------------------------ launchers
template <typename T>
rhmc_status_t nxn_qr_init(const double2 *partial, int nparts, int n, int nshift, SolverState *st, C<T> *rinv,
                          cudaStream_t s) {
  prof_begin(PROF_NXN, s);
  k_qr_init<T><<<1, 256, 0, s>>>(partial, nparts, n, nshift, st, rinv);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
// The mixed solve (FP32 fields) takes the double-float kernels of small_df.cu for
// the base steps unless RHMC_TUNE_NXN_FP64 = 1.
template <typename T> static bool use_dd(int nparts) {
  return sizeof(T) == 4 && nparts == 1 && tune_get(TUNE_NXN_FP64) != 1;
}
template <typename T>
rhmc_status_t nxn_alpha(const double2 *partial, int nparts, int n, SolverState *st, int k, C<T> *mw, cudaStream_t s) {
  if constexpr (sizeof(T) == 4)
    if (use_dd<T>(nparts)) return nxn_alpha_dd(partial, n, st, k, mw, s);
  prof_begin(PROF_NXN, s);
  k_nxn_alpha<T><<<1, 256, 0, s>>>(partial, nparts, n, st, k, mw);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template <typename T>
rhmc_status_t nxn_rho(const double2 *partial, int nparts, int n, SolverState *st, int k, C<T> *coef,
                      cudaStream_t s) {
  if constexpr (sizeof(T) == 4)
    if (use_dd<T>(nparts)) return nxn_rho_dd(partial, n, st, k, coef, s);
  prof_begin(PROF_NXN, s);
  k_nxn_rho<T><<<1, 256, 0, s>>>(partial, nparts, n, st, k, coef);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
template <typename T>
rhmc_status_t nxn_shifts(int n, int nshift, SolverState *st, int k, C<T> *coef, double tol_shift, int freeze,
                         double2 *hist, int cap, cudaStream_t s) {
  if constexpr (sizeof(T) == 4)
    if (nshift > 1 && tune_get(TUNE_NXN_FP64) != 1)
      return nxn_shifts_dd(n, nshift, st, k, coef, tol_shift, freeze, hist, cap, s);
  if (nshift > 1) {
    prof_begin(PROF_NXN_SHIFTS, s);
    k_nxn_shifts<T><<<nshift - 1, 256, 0, s>>>(n, nshift, st, k, coef, tol_shift, freeze, hist, cap);
    prof_end(s, 0.0);
    RHMC_LAUNCH_CHECK();
  }
  return RHMC_OK;
}
template <typename T>
rhmc_status_t nxn_reliable(const double2 *partial, int nparts, int n, SolverState *st, int k, C<T> *rinv,
                           cudaStream_t s) {
  prof_begin(PROF_NXN, s);
  k_nxn_reliable<T><<<1, 256, 0, s>>>(partial, nparts, n, st, k, rinv);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

#define RHMC_INST_NXN(T)                                                                                     \
  template rhmc_status_t nxn_qr_init<T>(const double2 *, int, int, int, SolverState *, C<T> *, cudaStream_t); \
  template rhmc_status_t nxn_alpha<T>(const double2 *, int, int, SolverState *, int, C<T> *, cudaStream_t);   \
  template rhmc_status_t nxn_rho<T>(const double2 *, int, int, SolverState *, int, C<T> *, cudaStream_t);     \
  template rhmc_status_t nxn_shifts<T>(int, int, SolverState *, int, C<T> *, double, int, double2 *, int,     \
                                       cudaStream_t);                                                            \
  template rhmc_status_t nxn_reliable<T>(const double2 *, int, int, SolverState *, int, C<T> *, cudaStream_t);
RHMC_INST_NXN(float)
RHMC_INST_NXN(double)

}  // namespace rhmc

// ------------------------------------------------------------ self-test of the FP64 helpers
namespace rhmc {
__global__ void k_fp64_helpers(const double *__restrict__ x, int count, double *__restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= count) return;
  const double v = x[k];
  out[0 * (size_t)count + k] = frcp(v);
  out[1 * (size_t)count + k] = fsqrt(v);
  out[2 * (size_t)count + k] = frcp_fast(v);
  out[3 * (size_t)count + k] = frsqrt(v);
  out[4 * (size_t)count + k] = 1.0 / v;  // IEEE division
  out[5 * (size_t)count + k] = sqrt(v);  // IEEE square root
}
}  // namespace rhmc

extern "C" rhmc_status_t rhmc_selftest_fp64_helpers(const double *x_dev, int count, double *out_dev,
                                                    rhmc_stream_t sv) {
  using namespace rhmc;
  if (!x_dev || !out_dev || count < 1) {
    set_error("rhmc_selftest_fp64_helpers: null pointer or count < 1");
    return RHMC_ERR_INVALID_ARG;
  }
  k_fp64_helpers<<<(count + 255) / 256, 256, 0, (cudaStream_t)sv>>>(x_dev, count, out_dev);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}
