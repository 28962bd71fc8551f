// Multi-RHS even-odd staggered hop (Sec. IV operator; block "pencil"
// application of Sec. III / conclusions: each gauge link is loaded once for
// all n right-hand sides).
//
// Internal link layout, one array per output parity p:
//   L_p[h][d][3][3], h = rank of the output site x among parity p,
//   d = mu       : eta_mu(x) b_mu(x) U_mu(x)                (forward, x+mu)
//   d = 4 + mu   : -eta_mu(x) b_mu(x-mu) U_mu(x-mu)^dagger   (backward, x-mu)
// so that (D psi)(x) = sum_d L_p[h][d] psi(nb_d(x)).  The 72 complex numbers a
// site needs are contiguous: a CTA stages the records of its site tile into
// shared memory with coalesced 16-byte loads and every thread of the tile (one
// per (site, right-hand side)) reads them from there.
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "df.cuh"
#include "kernels.h"

namespace rhmc {

// ------------------------------------------------------------ link staging
template <typename T>
__global__ void k_stage_links(Geom g, int par, const double2 *__restrict__ U, int bc_t, C<T> *__restrict__ out) {
  const long h = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= g.Vh) return;
  int x[4];
  site_coords(g, par, h, x);
  const long lex = lex_of(g, x);
  C<T> *o = out + h * 72;
  int sum = 0;
  for (int mu = 0; mu < 4; ++mu) {
    const double eta = (sum & 1) ? -1.0 : 1.0;
    sum += x[mu];
    // forward link U_mu(x)
    const double bf = (mu == 3 && bc_t == -1 && x[3] == g.L[3] - 1) ? -1.0 : 1.0;
    const double2 *u = U + (lex * 4 + mu) * 9;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double2 z = u[a * 3 + b];
        o[mu * 9 + a * 3 + b] = mk<T>((T)(eta * bf * z.x), (T)(eta * bf * z.y));
      }
    // backward link U_mu(x-mu)^dagger
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[mu] = (x[mu] == 0) ? g.L[mu] - 1 : x[mu] - 1;
    const double bb = (mu == 3 && bc_t == -1 && y[3] == g.L[3] - 1) ? -1.0 : 1.0;
    const double2 *v = U + (lex_of(g, y) * 4 + mu) * 9;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const double2 z = v[b * 3 + a];  // dagger: transpose + conjugate
        o[(4 + mu) * 9 + a * 3 + b] = mk<T>((T)(-eta * bb * z.x), (T)(eta * bb * z.y));
      }
  }
}

rhmc_status_t stage_links(const Geom &g, const double2 *U, int bc_t, double2 *l64[2], float2 *l32[2],
                          cudaStream_t s) {
  const int bs = 128;
  const int grid = (int)((g.Vh + bs - 1) / bs);
  for (int p = 0; p < 2; ++p) {
    k_stage_links<double><<<grid, bs, 0, s>>>(g, p, U, bc_t, l64[p]);
    RHMC_LAUNCH_CHECK();
    k_stage_links<float><<<grid, bs, 0, s>>>(g, p, U, bc_t, l32[p]);
    RHMC_LAUNCH_CHECK();
  }
  return RHMC_OK;
}

// Coordinates of the site with parity `par` and parity rank h, 32-bit
// arithmetic (V/2 < 2^31): x = 2 xh + (parity of y + z + t xor par).
__device__ __forceinline__ void site_coords32(const Geom &g, int par, int h, int &x0, int &x1, int &x2, int &x3) {
  const int r = h / g.Lxh;
  const int xh = h - r * g.Lxh;
  const int r2 = r / g.L[1];
  x1 = r - r2 * g.L[1];
  x3 = r2 / g.L[2];
  x2 = r2 - x3 * g.L[2];
  x0 = 2 * xh + (((x1 + x2 + x3) & 1) ^ par);
}

// ------------------------------------------------------------ 12-real links
// A link record L = f V with V in SU(3) and f = +-1 (f = eta b for the forward
// links, f = -eta b for the daggered backward ones) is determined by its first
// two rows: row 3 = f conj(row 1 x row 2).  The FP32 hop can therefore read 6
// of the 9 complex entries (384 instead of 576 bytes per site) and rebuild the
// third rows in shared memory.  The sign of record d of the site with parity
// `par` and coordinates x:
__device__ __forceinline__ float link_sign(const Geom &g, int bc_t, int d, int x0, int x1, int x2, int x3) {
  const int mu = d & 3;
  const int ps = mu == 0 ? 0 : mu == 1 ? x0 : mu == 2 ? x0 + x1 : x0 + x1 + x2;
  float f = (ps & 1) ? -1.f : 1.f;  // eta_mu(x)
  if (d < 4) {
    if (mu == 3 && bc_t == -1 && x3 == g.L[3] - 1) f = -f;  // b_mu(x)
  } else {
    if (mu == 3 && bc_t == -1 && x3 == 0) f = -f;  // b_mu(x - mu)
    f = -f;
  }
  return f;
}

__device__ __forceinline__ float2 cross_conj(float2 a1, float2 a2, float2 b1, float2 b2) {
  // conj(a1 b2 - a2 b1)
  const float re = a1.x * b2.x - a1.y * b2.y - (a2.x * b1.x - a2.y * b1.y);
  const float im = a1.x * b2.y + a1.y * b2.x - (a2.x * b1.y + a2.y * b1.x);
  return make_float2(re, -im);
}

// first two rows of every FP32 record; *dev_max = largest |row 3 - rebuilt row 3|
__global__ void k_links12(Geom g, int par, int bc_t, const float2 *__restrict__ l32, float2 *__restrict__ l12,
                          unsigned *dev_max) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;  // (site, d)
  if (k >= g.Vh * 8) return;
  const int h = (int)(k >> 3), d = (int)(k & 7);
  const float2 *L = l32 + k * 9;
  float2 r[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    r[e] = L[e];
    l12[k * 6 + e] = r[e];
  }
  int x0, x1, x2, x3;
  site_coords32(g, par, h, x0, x1, x2, x3);
  const float f = link_sign(g, bc_t, d, x0, x1, x2, x3);
  float dev = 0.f;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
    const float2 t = cross_conj(r[c1], r[c2], r[3 + c1], r[3 + c2]);
    const float2 w = L[6 + c];
    dev = fmaxf(dev, fmaxf(fabsf(w.x - f * t.x), fabsf(w.y - f * t.y)));
  }
  atomicMax(dev_max, __float_as_uint(dev));  // non-negative floats order as their bit patterns
}

// ------------------------------------------------------------ hop
// out[b] = D in[b]                 (self == nullptr)
// out[b] = a self[b] - D in[b]     (the fused 4m^2 + sigma axpy of A)
// on parity `par`, for nbatch independent fields b (stride bstride) that
// share the staged links.
//
// Thread layout: R right-hand sides per thread (register blocking), n / R
// threads per site, `tile` sites per CTA.  The CTA stages the 72-complex link
// records of its sites into shared memory once, together with the 8 neighbour
// offsets of each site.  The loop over the 8 directions keeps the next
// direction's neighbour block in flight while the current one is multiplied.
namespace {


template <typename T> __device__ __forceinline__ void lmac(C<T> &acc, const C<T> &e, const C<T> &v) {
  cmac<T>(acc, e, v);
}

template <typename T> struct LinkSlot { using t = C<T>; };

template <typename T> __device__ __forceinline__ void expand(C<T> &dst, C<T> z) { dst = z; }

// Vector load / store of R consecutive complex numbers.
template <typename T, int R> struct Vec;
template <> struct Vec<float, 4> {
  __device__ static void ld(const float2 *p, float2 *v) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p)), b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w); v[2] = make_float2(b.x, b.y); v[3] = make_float2(b.z, b.w);
  }
  __device__ static void st(float2 *p, const float2 *v) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
    reinterpret_cast<float4 *>(p)[1] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
  }
};
template <> struct Vec<float, 2> {
  __device__ static void ld(const float2 *p, float2 *v) {
    const float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = make_float2(a.x, a.y); v[1] = make_float2(a.z, a.w);
  }
  __device__ static void st(float2 *p, const float2 *v) {
    reinterpret_cast<float4 *>(p)[0] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
  }
};
template <typename T> struct Vec1 {
  __device__ static void ld(const C<T> *p, C<T> *v) { v[0] = p[0]; }
  __device__ static void st(C<T> *p, const C<T> *v) { p[0] = v[0]; }
};
template <> struct Vec<float, 1> : Vec1<float> {};
template <> struct Vec<double, 1> : Vec1<double> {};
template <int R> struct VecD {
  __device__ static void ld(const double2 *p, double2 *v) {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = __ldg(p + r);
  }
  __device__ static void st(double2 *p, const double2 *v) {
#pragma unroll
    for (int r = 0; r < R; ++r) p[r] = v[r];
  }
};
template <> struct Vec<double, 2> : VecD<2> {};
template <> struct Vec<double, 4> : VecD<4> {};

}  // namespace

template <typename T, int R, bool SELF, bool STAGE>
__global__ void __launch_bounds__(128) k_hop(Geom g, int par, const C<T> *__restrict__ links,
                                             const C<T> *__restrict__ in, C<T> *__restrict__ out,
                                             const C<T> *__restrict__ self, T a, int n, int tile, int nbatch,
                                             long bstride) {
  using LS = typename LinkSlot<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  LS *sl = reinterpret_cast<LS *>(smem_raw);
  const int tps = n / R;
  const int h0 = blockIdx.x * tile;
  const int nsites = min(tile, (int)g.Vh - h0);
  if (STAGE) {
    const C<T> *src = links + (long)h0 * 72;
    for (int k = threadIdx.x; k < nsites * 72; k += blockDim.x) expand<T>(sl[k], __ldg(src + k));
    __syncthreads();
  }
  // neighbour ranks of every site of the tile, shared by the site's threads
  int *snb = reinterpret_cast<int *>(smem_raw + (STAGE ? (size_t)tile * 72 * sizeof(LS) : 0));
  for (int k = threadIdx.x; k < nsites * 8; k += blockDim.x) {
    const int site = k >> 3, d = k & 7;
    int x[4];
    site_coords(g, par, h0 + site, x);
    const int mu = d & 3, st = d < 4 ? 1 : -1;
    // neighbour coordinates without dynamic indexing of x[]
    int y0 = x[0], y1 = x[1], y2 = x[2], y3 = x[3];
    if (mu == 0) y0 = (y0 + st + g.L[0]) % g.L[0];
    else if (mu == 1) y1 = (y1 + st + g.L[1]) % g.L[1];
    else if (mu == 2) y2 = (y2 + st + g.L[2]) % g.L[2];
    else y3 = (y3 + st + g.L[3]) % g.L[3];
    const int lex = y0 + g.L[0] * (y1 + g.L[1] * (y2 + g.L[2] * y3));
    snb[k] = (lex >> 1) * 3 * n;
  }
  __syncthreads();
  const int ls = threadIdx.x / tps;
  const int j0 = (threadIdx.x - ls * tps) * R;
  if (ls >= nsites) return;
  const int h = h0 + ls;
  const int o = h * 3 * n + j0;
  for (int b = 0; b < nbatch; ++b) {
    const C<T> *inb = in + b * bstride;
    C<T> acc[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < R; ++r) acc[c][r] = czero<T>();
    C<T> v[3][R], vn[3][R];
#pragma unroll
    for (int c = 0; c < 3; ++c) Vec<T, R>::ld(inb + snb[ls * 8] + j0 + c * n, v[c]);
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
      // prefetch the next direction's neighbour block while this one is used
      const int dn = d < 7 ? d + 1 : d;
#pragma unroll
      for (int c = 0; c < 3; ++c) Vec<T, R>::ld(inb + snb[ls * 8 + dn] + j0 + c * n, vn[c]);
#pragma unroll
      for (int ca = 0; ca < 3; ++ca)
#pragma unroll
        for (int cb = 0; cb < 3; ++cb) {
          LS e;
          if (STAGE)
            e = sl[ls * 72 + d * 9 + ca * 3 + cb];
          else
            expand<T>(e, __ldg(links + (long)h * 72 + d * 9 + ca * 3 + cb));
#pragma unroll
          for (int r = 0; r < R; ++r) lmac<T>(acc[ca][r], e, v[cb][r]);
        }
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < R; ++r) v[c][r] = vn[c][r];
    }
    C<T> *ob = out + b * bstride + o;
    if (SELF) {
      const C<T> *sb = self + b * bstride + o;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        C<T> sv[R];
        Vec<T, R>::ld(sb + c * n, sv);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[c][r] = mk<T>(a * sv[r].x - acc[c][r].x, a * sv[r].y - acc[c][r].y);
      }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) Vec<T, R>::st(ob + c * n, acc[c]);
  }
}

template <typename T, int R>
static void launch_hop(const Geom &g, int par, const C<T> *links, const C<T> *in, C<T> *out, const C<T> *self,
                       double a, int n, int nbatch, long bstride, cudaStream_t s) {
  using LS = typename LinkSlot<T>::t;
  const int tps = n / R;
  const bool stage = tps >= 2;  // links are reused only when several threads share a site
  const int tile = max(1, 128 / tps);
  const int threads = ((tile * tps + 31) / 32) * 32;
  const size_t smem = (stage ? (size_t)tile * 72 * sizeof(LS) : 0) + (size_t)tile * 8 * sizeof(int);
  const unsigned grid = (unsigned)((g.Vh + tile - 1) / tile);
  static std::once_flag attr_done;
  std::call_once(attr_done, [&] {
    cudaFuncSetAttribute(k_hop<T, R, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    cudaFuncSetAttribute(k_hop<T, R, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    cudaFuncSetAttribute(k_hop<T, R, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    cudaFuncSetAttribute(k_hop<T, R, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  });
  if (self) {
    if (stage)
      k_hop<T, R, true, true><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
    else
      k_hop<T, R, true, false><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
  } else {
    if (stage)
      k_hop<T, R, false, true><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
    else
      k_hop<T, R, false, false><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
  }
}

// ------------------------------------------------------------ hop, all directions in flight
// FP32, one right-hand side per thread, n threads per site, TS = 128 / n sites
// per CTA.  The CTA's link records go to shared memory by cp.async while the
// neighbour table is built; then every thread issues the loads of all 8
// neighbours' 3 colour components at once (24 independent 8-byte loads, about
// 200 bytes per thread in flight) before it multiplies anything, so the
// latency of the gathered reads is paid once per site instead of once per
// direction.
template <int N, int R, bool SELF, bool REC>
__global__ void __launch_bounds__(128) k_hop_pf(Geom g, int par, const float2 *__restrict__ links,
                                                const float2 *__restrict__ in, float2 *__restrict__ out,
                                                const float2 *__restrict__ self, float a, int bc_t) {
  constexpr int TPS = N / R;                                 // threads per site
  constexpr int TILE = (128 / TPS) < 32 ? (128 / TPS) : 32;  // sites per CTA (static shared memory <= 20 KB)
  constexpr int LR = REC ? 48 : 72;  // complex per site record as stored
  __shared__ __align__(16) float2 sl[TILE * 72];
  __shared__ __align__(16) float2 sl12[REC ? TILE * 48 : 1];
  __shared__ float sgn[REC ? TILE * 8 : 1];
  __shared__ int snb[TILE * 8];
  const int tid = threadIdx.x;
  const int h0 = blockIdx.x * TILE;
  const int nsites = min(TILE, (int)g.Vh - h0);
  {
    const unsigned base = (unsigned)__cvta_generic_to_shared(REC ? sl12 : sl);
    const char *src = reinterpret_cast<const char *>(links + (long)h0 * LR);
    for (int c = tid; c < nsites * (LR / 2); c += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(base + 16u * c), "l"(src + 16L * c) : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int k = tid; k < nsites * 8; k += blockDim.x) {
    const int site = k >> 3, d = k & 7;
    int y0, y1, y2, y3;
    site_coords32(g, par, h0 + site, y0, y1, y2, y3);
    if (REC) sgn[k] = link_sign(g, bc_t, d, y0, y1, y2, y3);
    const int mu = d & 3;
    const bool fwd = d < 4;
    if (mu == 0) y0 = fwd ? (y0 + 1 == g.L[0] ? 0 : y0 + 1) : (y0 == 0 ? g.L[0] - 1 : y0 - 1);
    else if (mu == 1) y1 = fwd ? (y1 + 1 == g.L[1] ? 0 : y1 + 1) : (y1 == 0 ? g.L[1] - 1 : y1 - 1);
    else if (mu == 2) y2 = fwd ? (y2 + 1 == g.L[2] ? 0 : y2 + 1) : (y2 == 0 ? g.L[2] - 1 : y2 - 1);
    else y3 = fwd ? (y3 + 1 == g.L[3] ? 0 : y3 + 1) : (y3 == 0 ? g.L[3] - 1 : y3 - 1);
    const int lex = y0 + g.L[0] * (y1 + g.L[1] * (y2 + g.L[2] * y3));
    snb[k] = (lex >> 1) * 3 * N;
  }
  __syncthreads();
  const int ls = tid / TPS, j = (tid - (tid / TPS) * TPS) * R;
  const bool live = ls < nsites;
  float2 v[8][3][R];
  if (live) {
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const float2 *nb = in + snb[ls * 8 + d] + j;
#pragma unroll
      for (int c = 0; c < 3; ++c) Vec<float, R>::ld(nb + c * N, v[d][c]);
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  if (REC) {  // full records from the first two rows: row 3 = f conj(row 1 x row 2)
    for (int e = tid; e < nsites * 8; e += blockDim.x) {
      const float2 *r = sl12 + e * 6;
      float2 *o = sl + (e >> 3) * 72 + (e & 7) * 9;
      const float f = sgn[e];
#pragma unroll
      for (int c = 0; c < 6; ++c) o[c] = r[c];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        const float2 t = cross_conj(r[c1], r[c2], r[3 + c1], r[3 + c2]);
        o[6 + c] = make_float2(f * t.x, f * t.y);
      }
    }
    __syncthreads();
  }
  if (!live) return;
  float2 acc[3][R];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < R; ++r) acc[c][r] = make_float2(0.f, 0.f);
  const float2 *lk = sl + ls * 72;
#pragma unroll
  for (int d = 0; d < 8; ++d)
#pragma unroll
    for (int ca = 0; ca < 3; ++ca)
#pragma unroll
      for (int cb = 0; cb < 3; ++cb) {
        const float2 e = lk[d * 9 + ca * 3 + cb];
#pragma unroll
        for (int r = 0; r < R; ++r) cmac<float>(acc[ca][r], e, v[d][cb][r]);
      }
  float2 *op = out + (long)(h0 + ls) * 3 * N + j;
  if (SELF) {
    const float2 *sp = self + (long)(h0 + ls) * 3 * N + j;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      float2 sv[R];
      Vec<float, R>::ld(sp + c * N, sv);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[c][r] = make_float2(a * sv[r].x - acc[c][r].x, a * sv[r].y - acc[c][r].y);
    }
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) Vec<float, R>::st(op + c * N, acc[c]);
}

template <int N, int R>
static void launch_hop_pf_n(const Geom &g, int par, const float2 *links, const float2 *in, float2 *out,
                            const float2 *self, double a, const float2 *links12, int bc_t, cudaStream_t s) {
  constexpr int TPS = N / R;
  constexpr int TILE = (128 / TPS) < 32 ? (128 / TPS) : 32;
  const int threads = ((TILE * TPS + 31) / 32) * 32;
  const unsigned grid = (unsigned)((g.Vh + TILE - 1) / TILE);
  if (links12) {
    if (self)
      k_hop_pf<N, R, true, true><<<grid, threads, 0, s>>>(g, par, links12, in, out, self, (float)a, bc_t);
    else
      k_hop_pf<N, R, false, true><<<grid, threads, 0, s>>>(g, par, links12, in, out, self, (float)a, bc_t);
  } else if (self) {
    k_hop_pf<N, R, true, false><<<grid, threads, 0, s>>>(g, par, links, in, out, self, (float)a, bc_t);
  } else {
    k_hop_pf<N, R, false, false><<<grid, threads, 0, s>>>(g, par, links, in, out, self, (float)a, bc_t);
  }
}

static bool launch_hop_pf(const Geom &g, int par, const float2 *links, const float2 *in, float2 *out,
                          const float2 *self, double a, int n, const float2 *links12, int bc_t, cudaStream_t s) {
  // two right-hand sides per thread (16-byte loads, half the load instructions): built-in
  // for even n >= 12 (measured at 24^4: n = 16 65 us against 71 us; n = 8 no gain)
  const int mode = tune_get(TUNE_HOP_STAGED);
  const bool r2 = n % 2 == 0 && (mode == 4 || (mode == 0 && n >= 12));
  switch (n) {
#define L_PF(NN)                                                                   \
  case NN:                                                                         \
    if constexpr (NN % 2 == 0) {                                                   \
      if (r2) {                                                                    \
        launch_hop_pf_n<NN, 2>(g, par, links, in, out, self, a, links12, bc_t, s); \
        return true;                                                               \
      }                                                                            \
    }                                                                              \
    launch_hop_pf_n<NN, 1>(g, par, links, in, out, self, a, links12, bc_t, s);     \
    return true;
    L_PF(1) L_PF(2) L_PF(3) L_PF(4) L_PF(5) L_PF(6) L_PF(7) L_PF(8)
    L_PF(9) L_PF(10) L_PF(11) L_PF(12) L_PF(13) L_PF(14) L_PF(15) L_PF(16)
#undef L_PF
    default: return false;
  }
}

// ------------------------------------------------------------ hop, cp.async staged
// FP32, one field, even n: persistent CTAs walk over tiles of TS output sites.
// All threads stage the next tile into shared memory with 16-byte cp.async
// copies (L2 only) while the current tile is multiplied:
//   the TS link records (TS * 72 complex, contiguous),
//   the 8 neighbour rows of every site (3n complex each, gathered),
//   the TS rows of `self` for the fused axpy (contiguous).
// Two buffers, one cp.async group per tile, so every thread keeps a whole
// tile's share of loads in flight without holding them in registers.  Every
// thread owns R right-hand sides of one site.
namespace {
template <int R> struct SVec;  // shared-memory vector loads
template <> struct SVec<1> {
  __device__ static void ld(const float2 *p, float2 *v) { v[0] = p[0]; }
};
template <> struct SVec<2> {
  __device__ static void ld(const float2 *p, float2 *v) {
    const float4 a = *reinterpret_cast<const float4 *>(p);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
  }
};
template <> struct SVec<4> {
  __device__ static void ld(const float2 *p, float2 *v) {
    SVec<2>::ld(p, v);
    SVec<2>::ld(p + 2, v + 2);
  }
};
__device__ __forceinline__ void cp_async16(unsigned dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
}  // namespace

template <int R, bool SELF>
__global__ void __launch_bounds__(128) k_hop_staged(Geom g, int par, const float2 *__restrict__ links,
                                                    const float2 *__restrict__ in, float2 *__restrict__ out,
                                                    const float2 *__restrict__ self, float a, int n, int TS,
                                                    int ntiles) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tps = n / R;
  const int row = 3 * n;      // complex numbers of one site row
  const int cpr = 3 * n / 2;  // 16-byte chunks of one site row
  const unsigned link_b = (unsigned)TS * 72 * 8, nb_b = (unsigned)TS * 8 * row * 8;
  const unsigned stage_b = link_b + nb_b + (SELF ? (unsigned)TS * row * 8 : 0u);
  int *snb = reinterpret_cast<int *>(smem_raw + 2 * stage_b);  // [2][TS * 8] neighbour ranks
  const int nthr = blockDim.x, tid = threadIdx.x;
  // per-thread walk over (row, chunk) pairs: start and stride without divisions in the loop
  const int q0 = tid % cpr, r0 = tid / cpr, dq = nthr % cpr, dr = nthr / cpr;

  auto fill_nb = [&](int tile, int buf) {
    const int h0 = tile * TS;
    const int ns = min(TS, (int)g.Vh - h0);
    for (int k = tid; k < ns * 8; k += nthr) {
      const int site = k >> 3, d = k & 7;
      int x[4];
      site_coords(g, par, h0 + site, x);
      const int mu = d & 3, st = d < 4 ? 1 : -1;
      int y0 = x[0], y1 = x[1], y2 = x[2], y3 = x[3];
      if (mu == 0) y0 = (y0 + st + g.L[0]) % g.L[0];
      else if (mu == 1) y1 = (y1 + st + g.L[1]) % g.L[1];
      else if (mu == 2) y2 = (y2 + st + g.L[2]) % g.L[2];
      else y3 = (y3 + st + g.L[3]) % g.L[3];
      const int lex = y0 + g.L[0] * (y1 + g.L[1] * (y2 + g.L[2] * y3));
      snb[buf * TS * 8 + k] = lex >> 1;
    }
  };
  auto issue = [&](int tile, int buf) {
    const int h0 = tile * TS;
    const int ns = min(TS, (int)g.Vh - h0);
    const unsigned base = (unsigned)__cvta_generic_to_shared(smem_raw + buf * stage_b);
    const char *lsrc = reinterpret_cast<const char *>(links + (long)h0 * 72);
    for (int c = tid; c < ns * 36; c += nthr) cp_async16(base + 16u * c, lsrc + 16L * c);
    const int *nb = snb + buf * TS * 8;
    int q = q0, r = r0;
    while (r < ns * 8) {
      cp_async16(base + link_b + (unsigned)(r * row * 8 + q * 16),
                 reinterpret_cast<const char *>(in + (long)nb[r] * row) + 16 * q);
      q += dq;
      r += dr;
      if (q >= cpr) {
        q -= cpr;
        ++r;
      }
    }
    if (SELF) {
      const char *ssrc = reinterpret_cast<const char *>(self + (long)h0 * row);
      for (int c = tid; c < ns * cpr; c += nthr) cp_async16(base + link_b + nb_b + 16u * c, ssrc + 16L * c);
    }
  };
  const int ls = tid / tps;
  const int j0 = (tid - ls * tps) * R;
  int tile = blockIdx.x;
  if (tile < ntiles) {
    fill_nb(tile, 0);
    __syncthreads();
    issue(tile, 0);
  }
  cp_async_commit();
  for (int i = 0; tile < ntiles; tile += gridDim.x, ++i) {
    const int buf = i & 1;
    const int next = tile + gridDim.x;
    if (next < ntiles) fill_nb(next, buf ^ 1);
    __syncthreads();  // neighbour table ready; buffer buf ^ 1 no longer read
    if (next < ntiles) issue(next, buf ^ 1);
    cp_async_commit();
    cp_async_wait<1>();  // this thread's copies of the current tile landed
    __syncthreads();     // ... and everyone else's
    const int h0 = tile * TS;
    const int ns = min(TS, (int)g.Vh - h0);
    if (ls < ns) {
      const unsigned char *sb = smem_raw + buf * stage_b;
      const float2 *sl = reinterpret_cast<const float2 *>(sb) + ls * 72;
      const float2 *sn = reinterpret_cast<const float2 *>(sb + link_b) + ls * 8 * row + j0;
      float2 acc[3][R];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[c][r] = make_float2(0.f, 0.f);
#pragma unroll 2
      for (int d = 0; d < 8; ++d) {
        float2 v[3][R];
#pragma unroll
        for (int c = 0; c < 3; ++c) SVec<R>::ld(sn + d * row + c * n, v[c]);
#pragma unroll
        for (int ca = 0; ca < 3; ++ca)
#pragma unroll
          for (int cb = 0; cb < 3; ++cb) {
            const float2 e = sl[d * 9 + ca * 3 + cb];
#pragma unroll
            for (int r = 0; r < R; ++r) cmac<float>(acc[ca][r], e, v[cb][r]);
          }
      }
      const long o = (long)(h0 + ls) * row + j0;
      if (SELF) {
        const float2 *ss = reinterpret_cast<const float2 *>(sb + link_b + nb_b) + ls * row + j0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          float2 sv[R];
          SVec<R>::ld(ss + c * n, sv);
#pragma unroll
          for (int r = 0; r < R; ++r) acc[c][r] = make_float2(a * sv[r].x - acc[c][r].x, a * sv[r].y - acc[c][r].y);
        }
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) Vec<float, R>::st(out + o + c * n, acc[c]);
    }
  }
  cp_async_wait<0>();
}

template <int R>
static bool launch_hop_staged(const Geom &g, int par, const float2 *links, const float2 *in, float2 *out,
                              const float2 *self, double a, int n, cudaStream_t s) {
  const int tps = n / R;
  const long per_site = 576 + 8L * 24 * n + (self ? 24L * n : 0);
  const int TS = (int)std::min<long>(128 / tps, (96 * 1024) / per_site);
  if (TS < 1) return false;
  const int threads = ((TS * tps + 31) / 32) * 32;
  const size_t smem = 2 * (size_t)TS * per_site + 2 * (size_t)TS * 8 * sizeof(int);
  const int ntiles = (int)((g.Vh + TS - 1) / TS);
  static std::once_flag attr_done;
  std::call_once(attr_done, [] {
    cudaFuncSetAttribute(k_hop_staged<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
    cudaFuncSetAttribute(k_hop_staged<R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 210 * 1024);
  });
  const int resident = self ? resident_ctas(k_hop_staged<R, true>, threads, smem)
                            : resident_ctas(k_hop_staged<R, false>, threads, smem);
  const int grid = std::min(ntiles, resident);
  if (self)
    k_hop_staged<R, true><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (float)a, n, TS, ntiles);
  else
    k_hop_staged<R, false><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (float)a, n, TS, ntiles);
  return true;
}

// The all-directions-in-flight kernel: FP32 single fields, the built-in choice
// (RHMC_TUNE_HOP_STAGED 0 or 3; 2 selects the register-staged kernel).
template <typename T> static bool use_hop_pf(const void *links, const void *in, int nbatch) {
  if (sizeof(C<T>) != 8 || nbatch != 1 || ((uintptr_t)links & 15)) return false;
  const int mode = tune_get(TUNE_HOP_STAGED);
  return mode == 0 || mode == 3 || mode == 4;  // 3: one right-hand side per thread, 4: two
}

// The staged kernel applies to FP32 single fields with 16-byte aligned rows.
template <typename T>
static bool try_hop_staged(const Geom &g, int par, const C<T> *links, const C<T> *in, C<T> *out,
                           const C<T> *self, double a, int n, int nbatch, int R, cudaStream_t s) {
  if constexpr (sizeof(C<T>) != 8) {
    return false;
  } else {
    const int mode = tune_get(TUNE_HOP_STAGED);
    // built-in: the register-staged kernel (measured faster at 24^4, n = 8 and 16)
    if (mode != 1 || nbatch != 1 || n % 2) return false;
    auto al16 = [](const void *p) { return ((uintptr_t)p & 15) == 0; };
    if (!al16(links) || !al16(in) || !al16(out) || (self && !al16(self))) return false;
    const float2 *L = reinterpret_cast<const float2 *>(links), *X = reinterpret_cast<const float2 *>(in),
                 *S = reinterpret_cast<const float2 *>(self);
    float2 *Y = reinterpret_cast<float2 *>(out);
    if (R == 4) return launch_hop_staged<4>(g, par, L, X, Y, S, a, n, s);
    if (R == 2) return launch_hop_staged<2>(g, par, L, X, Y, S, a, n, s);
    return launch_hop_staged<1>(g, par, L, X, Y, S, a, n, s);
  }
}

template <typename T>
rhmc_status_t hop(const Geom &g, int par, const C<T> *links, const C<T> *in, C<T> *out, const C<T> *self, double a,
                  int n, int nbatch, long bstride, cudaStream_t s, const C<T> *links12, int bc_t) {
  if (n < 1 || n > RHMC_MAX_NRHS || g.Vh * 3L * n > 0x7fffffffL) return RHMC_ERR_INVALID_ARG;
  prof_begin(sizeof(T) == 4 ? PROF_HOP32 : PROF_HOP64, s);
  int R = tune_get(TUNE_HOP_RHS_PER_THREAD);
  // measured at 24^4 (FP32): 2 per thread best for n >= 12, 1 otherwise; FP64 is ALU bound
  if (R <= 0 || n % R != 0) R = (sizeof(T) == 4 && n >= 12 && n % 2 == 0) ? 2 : 1;
  if (try_hop_staged<T>(g, par, links, in, out, self, a, n, nbatch, R, s)) {
  } else if (use_hop_pf<T>(links, in, nbatch)) {
    launch_hop_pf(g, par, reinterpret_cast<const float2 *>(links), reinterpret_cast<const float2 *>(in),
                  reinterpret_cast<float2 *>(out), reinterpret_cast<const float2 *>(self), a, n,
                  reinterpret_cast<const float2 *>(links12), bc_t, s);
  } else if (R == 4)
    launch_hop<T, 4>(g, par, links, in, out, self, a, n, nbatch, bstride, s);
  else if (R == 2)
    launch_hop<T, 2>(g, par, links, in, out, self, a, n, nbatch, bstride, s);
  else
    launch_hop<T, 1>(g, par, links, in, out, self, a, n, nbatch, bstride, s);
  // algorithmic bytes: every link once, every input field once, the output once (+ self)
  prof_end(s, (double)g.Vh * sizeof(C<T>) * (72.0 + nbatch * 3.0 * n * (self ? 3 : 2)));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

// ------------------------------------------------------------ double-float hop
// FP64-accurate hop on the FP32 units (double-float arithmetic of df.cuh).
using namespace df;


template <bool SELF>
__global__ void __launch_bounds__(128) k_hop_df(Geom g, int par, const float4 *__restrict__ links,
                                                const float4 *__restrict__ in, float4 *__restrict__ out,
                                                const float4 *__restrict__ self, float ah, float al, int n, int tile) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4 *sl = reinterpret_cast<float4 *>(smem_raw);
  int *snb = reinterpret_cast<int *>(smem_raw + (size_t)tile * 72 * sizeof(float4));
  const int h0 = blockIdx.x * tile;
  const int nsites = min(tile, (int)g.Vh - h0);
  for (int k = threadIdx.x; k < nsites * 72; k += blockDim.x) sl[k] = links[(long)h0 * 72 + k];
  for (int k = threadIdx.x; k < nsites * 8; k += blockDim.x) {
    const int site = k >> 3, d = k & 7;
    int x[4];
    site_coords(g, par, h0 + site, x);
    const int mu = d & 3, st = d < 4 ? 1 : -1;
    int y0 = x[0], y1 = x[1], y2 = x[2], y3 = x[3];
    if (mu == 0) y0 = (y0 + st + g.L[0]) % g.L[0];
    else if (mu == 1) y1 = (y1 + st + g.L[1]) % g.L[1];
    else if (mu == 2) y2 = (y2 + st + g.L[2]) % g.L[2];
    else y3 = (y3 + st + g.L[3]) % g.L[3];
    const int lex = y0 + g.L[0] * (y1 + g.L[1] * (y2 + g.L[2] * y3));
    snb[k] = (lex >> 1) * 3 * n;
  }
  __syncthreads();
  const int ls = threadIdx.x / n, j = threadIdx.x - ls * n;
  if (ls >= nsites) return;
  const int h = h0 + ls;
  DF re[3], im[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) re[c] = im[c] = DF{0.f, 0.f};
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    const float4 *v = in + snb[ls * 8 + d] + j;
    const float4 v0 = v[0], v1 = v[n], v2 = v[2 * n];
    const float4 *l = sl + ls * 72 + d * 9;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      df_cmac(re[a], im[a], l[a * 3 + 0], v0);
      df_cmac(re[a], im[a], l[a * 3 + 1], v1);
      df_cmac(re[a], im[a], l[a * 3 + 2], v2);
    }
  }
  const int o = h * 3 * n + j;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    if (SELF) {
      // result = a * self - D in: negate the hop sum, add the scaled self term
      DF r2{-re[c].h, -re[c].e}, i2{-im[c].h, -im[c].e};
      const float4 sv = self[o + c * n];
      df_add_prod(r2, ah, al, sv.x, sv.z);
      df_add_prod(i2, ah, al, sv.y, sv.w);
      out[o + c * n] = df_pack(r2, i2);
    } else {
      out[o + c * n] = df_pack(re[c], im[c]);
    }
  }
}

// FP64 <-> double-float conversion of complex fields (to_df: d -> (hi, lo)).
__global__ void k_df_convert(const double2 *__restrict__ in64, float4 *__restrict__ outdf, long len) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const double2 z = in64[i];
  const float2 a = df_split1(z.x), b = df_split1(z.y);
  outdf[i] = make_float4(a.x, b.x, a.y, b.y);
}
__global__ void k_df_merge(float4 *__restrict__ io, long len) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= len) return;
  const float4 v = io[i];
  reinterpret_cast<double2 *>(io)[i] = make_double2(df_merge1(v.x, v.z), df_merge1(v.y, v.w));
}

// R = B - Y in FP64 for Y in double-float as the second hop writes it:
// (B - hi) - lo, which needs no FP64 copy of Y.  Optionally Rf, the FP32
// rounding of R, and per-CTA sums of |R|^2 per column (n interleaved
// columns; partial[cta * n + column], CTA order fixed, so the host's sum of
// the partials is deterministic).  Thread t owns column t % n of every
// (256 / n)-th row; four rows are loaded before any is used.
__global__ void __launch_bounds__(256) k_resid_df(const double2 *__restrict__ B, const float4 *__restrict__ Y,
                                                  double2 *__restrict__ R, float2 *__restrict__ Rf, long rows,
                                                  int n, double *__restrict__ partial) {
  __shared__ double red[256];
  const int t = threadIdx.x;
  const int per = 256 / n;
  const int c = t % n, g = t / n;
  const long step = (long)gridDim.x * per;
  double acc = 0.0;
  if (g < per) {
    long r = (long)blockIdx.x * per + g;
    for (; r + 3 * step < rows; r += 4 * step) {
      double2 b[4];
      float4 y[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        b[u] = B[(r + u * step) * n + c];
        y[u] = Y[(r + u * step) * n + c];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double x = (b[u].x - df_widen1(y[u].x)) - df_widen1(y[u].z);
        const double z = (b[u].y - df_widen1(y[u].y)) - df_widen1(y[u].w);
        const long i = (r + u * step) * n + c;
        R[i] = make_double2(x, z);
        if (Rf) Rf[i] = make_float2((float)x, (float)z);
        acc += x * x + z * z;
      }
    }
    for (; r < rows; r += step) {
      const long i = r * n + c;
      const double2 bv = B[i];
      const float4 yv = Y[i];
      const double x = (bv.x - df_widen1(yv.x)) - df_widen1(yv.z);
      const double z = (bv.y - df_widen1(yv.y)) - df_widen1(yv.w);
      R[i] = make_double2(x, z);
      if (Rf) Rf[i] = make_float2((float)x, (float)z);
      acc += x * x + z * z;
    }
  }
  if (!partial) return;
  red[t] = acc;
  __syncthreads();
  if (t < n) {
    double sum = 0.0;
    for (int q = 0; q < per; ++q) sum += red[q * n + t];
    partial[(long)blockIdx.x * n + t] = sum;
  }
}

rhmc_status_t resid_df(const double2 *B, const float4 *Y, double2 *R, float2 *Rf, long rows, int n,
                       double *partial, int nparts, cudaStream_t s) {
  if (n < 1 || n > RHMC_MAX_NRHS || nparts < 1) return RHMC_ERR_INVALID_ARG;
  k_resid_df<<<nparts, 256, 0, s>>>(B, Y, R, Rf, rows, n, partial);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t stage_links_df(const Geom &g, const double2 *l64, float4 *ldf, cudaStream_t s) {
  const long len = g.Vh * 72;
  k_df_convert<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(l64, ldf, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t df_split(const double2 *in, float4 *out, long len, cudaStream_t s) {
  k_df_convert<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(in, out, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t df_merge(float4 *io, long len, cudaStream_t s) {
  k_df_merge<<<(unsigned)((len + 255) / 256), 256, 0, s>>>(io, len);
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

rhmc_status_t hop_df(const Geom &g, int par, const float4 *links, const float4 *in, float4 *out, const float4 *self,
                     double a, int n, cudaStream_t s) {
  if (n < 1 || n > RHMC_MAX_NRHS || g.Vh * 3L * n > 0x7fffffffL) return RHMC_ERR_INVALID_ARG;
  const int tile = max(1, 128 / n);
  const int threads = ((tile * n + 31) / 32) * 32;
  const size_t smem = (size_t)tile * 72 * sizeof(float4) + (size_t)tile * 8 * sizeof(int);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_hop_df<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_hop_df<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  const float ah = (float)a, al = (float)(a - (double)ah);
  const unsigned grid = (unsigned)((g.Vh + tile - 1) / tile);
  prof_begin(PROF_HOP_DF, s);
  if (self)
    k_hop_df<true><<<grid, threads, smem, s>>>(g, par, links, in, out, self, ah, al, n, tile);
  else
    k_hop_df<false><<<grid, threads, smem, s>>>(g, par, links, in, out, self, ah, al, n, tile);
  prof_end(s, (double)g.Vh * sizeof(float4) * (72.0 + 3.0 * n * (self ? 3 : 2)));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

template rhmc_status_t hop<float>(const Geom &, int, const float2 *, const float2 *, float2 *, const float2 *, double,
                                  int, int, long, cudaStream_t, const float2 *, int);
template rhmc_status_t hop<double>(const Geom &, int, const double2 *, const double2 *, double2 *, const double2 *,
                                   double, int, int, long, cudaStream_t, const double2 *, int);

// 12-real copies of the FP32 records; returns through *ok whether every record
// is f V with V in SU(3) to FP32 accuracy (then the hop may use the copies).
rhmc_status_t stage_links12(const Geom &g, int bc_t, float2 *const l32[2], float2 *l12[2], bool *ok,
                            cudaStream_t s) {
  unsigned *dmax = nullptr;
  RHMC_CUDA_TRY(cudaMallocAsync(&dmax, sizeof(unsigned), s));
  RHMC_CUDA_TRY(cudaMemsetAsync(dmax, 0, sizeof(unsigned), s));
  const long items = g.Vh * 8;
  for (int p = 0; p < 2; ++p) {
    k_links12<<<(unsigned)((items + 255) / 256), 256, 0, s>>>(g, p, bc_t, l32[p], l12[p], dmax);
    RHMC_LAUNCH_CHECK();
  }
  unsigned h = 0;
  RHMC_CUDA_TRY(cudaMemcpyAsync(&h, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  RHMC_CUDA_TRY(cudaStreamSynchronize(s));
  RHMC_CUDA_TRY(cudaFreeAsync(dmax, s));
  float dev = 0.f;
  std::memcpy(&dev, &h, sizeof(float));
  *ok = dev < 1e-5f;
  return RHMC_OK;
}

}  // namespace rhmc
