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
#include "common.cuh"
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

// ------------------------------------------------------------ hop
// out[b] = (self ? a * self[b] : 0) - (self ? 1 : -1) * D in[b]   on parity `par`
// i.e. out = D in            when self == nullptr,
//      out = a self - D in   otherwise (the fused 4m^2 + sigma axpy of A).
// One thread per (site, right-hand side); `tile` sites per CTA; the batch
// loop reuses the staged links for `nbatch` independent fields.
template <typename T, bool SELF, bool STAGE>
__global__ void __launch_bounds__(256) k_hop(Geom g, int par, const C<T> *__restrict__ links,
                                             const C<T> *__restrict__ in, C<T> *__restrict__ out,
                                             const C<T> *__restrict__ self, T a, int n, int tile, int nbatch,
                                             long bstride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T> *sl = reinterpret_cast<C<T> *>(smem_raw);
  const long h0 = (long)blockIdx.x * tile;
  const int nsites = (int)min((long)tile, g.Vh - h0);
  if (STAGE) {
    // 16-byte vector copy of nsites * 72 complex
    const int nvec = nsites * 72 * (int)sizeof(C<T>) / 16;
    const int4 *src = reinterpret_cast<const int4 *>(links + h0 * 72);
    int4 *dst = reinterpret_cast<int4 *>(sl);
    for (int k = threadIdx.x; k < nvec; k += blockDim.x) dst[k] = __ldg(src + k);
    __syncthreads();
  }
  const int ls = threadIdx.x / n;
  const int j = threadIdx.x - ls * n;
  if (ls >= nsites) return;
  const long h = h0 + ls;
  int x[4];
  site_coords(g, par, h, x);
  long nb[8];
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    nb[mu] = nb_rank(g, x, mu, +1) * 3 * n + j;
    nb[4 + mu] = nb_rank(g, x, mu, -1) * 3 * n + j;
  }
  const C<T> *L = STAGE ? sl + ls * 72 : links + h * 72;
  for (int b = 0; b < nbatch; ++b) {
    const C<T> *inb = in + b * bstride;
    C<T> acc0 = czero<T>(), acc1 = czero<T>(), acc2 = czero<T>();
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const C<T> v0 = inb[nb[d]], v1 = inb[nb[d] + n], v2 = inb[nb[d] + 2 * n];
      const C<T> *l = L + d * 9;
      cmac<T>(acc0, l[0], v0);
      cmac<T>(acc0, l[1], v1);
      cmac<T>(acc0, l[2], v2);
      cmac<T>(acc1, l[3], v0);
      cmac<T>(acc1, l[4], v1);
      cmac<T>(acc1, l[5], v2);
      cmac<T>(acc2, l[6], v0);
      cmac<T>(acc2, l[7], v1);
      cmac<T>(acc2, l[8], v2);
    }
    const long o = b * bstride + h * 3 * n + j;
    if (SELF) {
      const C<T> s0 = self[o], s1 = self[o + n], s2 = self[o + 2 * n];
      out[o] = mk<T>(a * s0.x - acc0.x, a * s0.y - acc0.y);
      out[o + n] = mk<T>(a * s1.x - acc1.x, a * s1.y - acc1.y);
      out[o + 2 * n] = mk<T>(a * s2.x - acc2.x, a * s2.y - acc2.y);
    } else {
      out[o] = acc0;
      out[o + n] = acc1;
      out[o + 2 * n] = acc2;
    }
  }
}

template <typename T>
rhmc_status_t hop(const Geom &g, int par, const C<T> *links, const C<T> *in, C<T> *out, const C<T> *self, double a,
                  int n, int nbatch, long bstride, cudaStream_t s) {
  if (n < 1 || n > 256) return RHMC_ERR_INVALID_ARG;
  const bool stage = n >= 4;
  int tile = 256 / n;
  if (!stage) tile = (n == 1) ? 128 : 64;
  const int threads = ((tile * n + 31) / 32) * 32;
  const size_t smem = stage ? (size_t)tile * 72 * sizeof(C<T>) : 0;
  const long grid = (g.Vh + tile - 1) / tile;
  static bool attr_done = false;  // FP64 at n = 4 stages 72 KB of links
  if (!attr_done) {
    cudaFuncSetAttribute(k_hop<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    cudaFuncSetAttribute(k_hop<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
    attr_done = true;
  }
  prof_begin(sizeof(T) == 4 ? PROF_HOP32 : PROF_HOP64, s);
  if (self) {
    if (stage)
      k_hop<T, true, true><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
    else
      k_hop<T, true, false><<<grid, threads, 0, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
  } else {
    if (stage)
      k_hop<T, false, true><<<grid, threads, smem, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
    else
      k_hop<T, false, false><<<grid, threads, 0, s>>>(g, par, links, in, out, self, (T)a, n, tile, nbatch, bstride);
  }
  // algorithmic bytes: every link once, every input field once, the output once (+ self)
  prof_end(s, (double)g.Vh * sizeof(C<T>) * (72.0 + nbatch * 3.0 * n * (self ? 3 : 2)));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}

template rhmc_status_t hop<float>(const Geom &, int, const float2 *, const float2 *, float2 *, const float2 *, double,
                                  int, int, long, cudaStream_t);
template rhmc_status_t hop<double>(const Geom &, int, const double2 *, const double2 *, double2 *, const double2 *,
                                   double, int, int, long, cudaStream_t);

}  // namespace rhmc
