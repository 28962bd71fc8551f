// Stored-basis assembly of the shifted solutions (mixed precision).
//
// Algorithm 1's shifted updates for a shift s: X^(s) += P^(s) alpha^(s)_k and
// P^(s) = Q_k + P^(s) M2_k, M2_k = beta^(s)_k rho_k^dagger, starting from
// P^(s)_0 = Q_0, X^(s) = 0.  Unrolled, P^(s)_k = sum_{i <= k} Q_i D_{i,k}
// with D_{k,k} = 1, D_{i,k} = M2_{i+1} ... M2_k, and after the shift's last
// update L:
//   X^(s) = sum_{i < L} Q_i C_i,   C_{L-1} = alpha_L,  C_i = alpha_{i+1} + M2_{i+1} C_{i+1}.
// So instead of updating P^(s) and X^(s) in HBM at every iteration, the solve
// keeps the block basis Q_0, Q_1, ... (FP32) and the n x n coefficients of
// every iteration (FP64), and forms all X^(s) at the end in one contraction
//   [rows x K 2n] . [K 2n x (nshift - 1) 2n]
// of real-embedded blocks (row (re, im) of Q times the 2 x 2 real blocks
// (Re c, Im c; -Im c, Re c) of each coefficient gives (re, im) of the product).
// Only the base system keeps its recursion.
//
// The contraction runs on the tensor cores (k_basis_gemm_tc, tcgen05, FP16
// inputs, FP32 accumulation in tensor memory) with FP32-level accuracy:
//   * each FP32 operand value v (scaled by a power of two) is split exactly
//     into two FP16 pieces, v = h + l + r with h = fp16(v), l = fp16(v - h),
//     |r| <= 2^-22 |v| (v - h is exact in FP32);
//   * every K tile accumulates the three products whose order is above
//     2^-22: l_A h_B + h_A l_B + h_A h_B (the dropped l_A l_B is below 2^-22);
//   * FP16 has a narrow exponent range, so the basis is scaled by 2^12 (its
//     entries are bounded by 1: the blocks Q_i have orthonormal columns) and
//     the coefficients of each shift by the power of two that brings their
//     largest entry to [2^11, 2^12); the epilogue multiplies by the inverse
//     power (exact).  Coefficients far below a shift's largest lose relative
//     accuracy only below 2^-37 of that largest entry.
// The tensor cores' FP32 accumulation is not correctly rounded, and its error
// grows with the number of MMAs summed into one accumulator and with the
// accumulator's magnitude.  So every kGChunkKt K tiles the partial sum moves
// out of the accumulator into a running sum in tensor memory, added on the
// CUDA cores with round-to-nearest, and the accumulator restarts from zero.
// With one K tile per chunk, the small products of a tile enter an empty
// accumulator and only its four h_A h_B MMAs run at full magnitude.  Measured
// at 24^4 (16 shifts, drift of the shifted systems' true residuals after the
// multishift phase, largest shift): one accumulator for all 1656 MMAs 6.2e-5,
// 48 MMAs per chunk 5.8e-6, 12 MMAs per chunk 4.2e-6, FP32 products with FP64
// sums over blocks (CUDA cores) 2.6e-6; the last two need the same number of
// defect-correction iterations.  Two accumulators alternate, so the MMAs of
// one K tile run while the epilogue moves the other into the running sum:
// tensor memory holds both and the running sum (3 x 160 of its 512 columns),
// so an N tile is at most 160 columns (whole shifts: 5 at n = 16); each N
// tile runs only up to the last iteration that updated one of its shifts.
// Measured at 24^4: 8.4 ms with double-buffered accumulators against 17.5 ms
// with one accumulator of 256 columns (whose moves stalled the MMAs) and
// 17.4 ms for a library FP32-emulating GEMM.  The last chunk's epilogue writes running sum
// + accumulator straight into the FP64 solutions X^(s) (or P^(s)), so no
// temporary product matrix is stored.
// A CUDA-core kernel (k_basis_gemm_simt: FP32 products, FP64 sum per block) is
// the RHMC_TUNE_BASIS_GEMM = 1 alternative.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

// ------------------------------------------------------------ coefficients
// FP64 coefficient blocks cf[(s - 1) * cfstride + i][q][j] (n x n complex) of
// the expansion of X^(s) (want_p = 0: blocks i < min(last_s, K)) or of
// P^(s)_K (want_p = 1: blocks i <= K, active shifts only).  One CTA per shift.
__global__ void __launch_bounds__(256) k_basis_coef(int n, int nshift, const SolverState *__restrict__ st,
                                                    const double2 *__restrict__ hist, int K, int want_p,
                                                    double2 *__restrict__ cf, long cfstride) {
  __shared__ double2 Cm[kMaxN * kMaxN], Tm[kMaxN * kMaxN];
  const int s = blockIdx.x + 1;
  if (s >= nshift) return;
  const int nn = n * n, t = threadIdx.x;
  const bool own = t < nn;
  const int qi = own ? t / n : 0, qj = own ? t % n : 0;
  const int last = want_p ? (st->active[s] ? K : -1) : min(st->last_k[s], K);
  if (last < 0 || (!want_p && last == 0)) return;
  double2 *out = cf + (size_t)(s - 1) * cfstride * nn;
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
    if (own) out[(size_t)i * nn + t] = Cm[t];
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

// Blocks of shift s that carry a coefficient.
__device__ __forceinline__ int basis_nblk(const SolverState *st, int s, int K, int want_p) {
  if (want_p) return st->active[s] ? K + 1 : 0;
  return max(0, min(st->last_k[s], K));
}

// ------------------------------------------------------------ tensor-core operand layout
// An FP16 tile of R rows x 64 K-elements is stored K-major with 128-byte rows
// under the 128-byte swizzle: the 16-byte chunk c of row r sits at chunk
// position c ^ (r & 7) within its 1024-byte group of 8 rows.
__host__ __device__ __forceinline__ unsigned sw128h(int row, int k) {
  return (unsigned)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + (k & 7) * 2);
}

namespace {
constexpr int kGM = 128;            // rows per tile (MMA M)
constexpr int kGK = 64;             // FP16 K elements per stage (one 128-byte swizzle row)
constexpr int kGNmax = 160;         // columns per N tile (MMA N); tensor memory holds two accumulators and
                                    // the running sum: 3 x 160 <= 512 columns
constexpr int kGStages = 3;
constexpr int kGThreads = 576;      // warps 0-7 split A (two groups, alternate stages), 8-15 epilogue
                                    // (two per tensor-memory lane quarter, one column half each),
                                    // 16 loads B, 17 issues the MMAs
constexpr int kGChunkKt = 1;        // built-in K tiles per accumulation chunk (12 MMAs into one accumulator)
constexpr unsigned kGAPiece = kGM * 128;  // bytes of one FP16 piece of an A tile
constexpr float kGAScale = 4096.f;        // 2^12: |basis entries| <= 1
constexpr long long kGWaitCycles = 2000000000LL;  // about a second at the GPU's 2 GHz
}  // namespace

// The N tiling of the shifted columns: whole shifts per tile.
struct BasisTiles {
  int spt;       // shifts per tile
  int nnt;       // tiles
  int NT;        // MMA N of a tile (multiple of 16, <= kGNmax)
  int nkt;       // K tiles per N tile in the packed buffer (capacity)
  size_t chunk;  // bytes of the two FP16 pieces of one (N tile, K tile)
};

static BasisTiles basis_tiles(int n, int nshift, int cap) {
  BasisTiles t{};
  const int two_n = 2 * n;
  const int m = std::max(1, nshift - 1);
  t.spt = std::max(1, std::min(m, kGNmax / two_n));
  t.nnt = (m + t.spt - 1) / t.spt;
  t.NT = ((t.spt * two_n + 15) / 16) * 16;
  t.nkt = ((cap + 1) * two_n + kGK - 1) / kGK;
  t.chunk = (size_t)2 * t.NT * 128;
  return t;
}

size_t basis_pack_bytes(int n, int nshift, int cap) {
  const BasisTiles t = basis_tiles(n, nshift, cap);
  return (size_t)t.nnt * t.nkt * t.chunk;
}

// Packed FP16 pieces of the scaled real-embedded coefficients, one CTA per
// shift: bpack[(tile * nkt + kt)][piece][NT x 64] (layout sw128h), the scale
// 2^-(12 + e_s) of the shift's products in bscale[s], and the number of K
// tiles each N tile needs in tile_nkt (atomic max; zeroed before).
__global__ void __launch_bounds__(256) k_basis_pack(int n, int nshift, const SolverState *__restrict__ st, int K,
                                                    int want_p, const double2 *__restrict__ cf, long cfstride,
                                                    BasisTiles tl, unsigned char *__restrict__ bpack,
                                                    double *__restrict__ bscale, int *__restrict__ tile_nkt) {
  __shared__ double red[256];
  const int s = blockIdx.x + 1;
  if (s >= nshift) return;
  const int nn = n * n, two_n = 2 * n;
  const int nblk = basis_nblk(st, s, K, want_p);
  const double2 *c = cf + (size_t)(s - 1) * cfstride * nn;
  const long total = (long)nblk * nn;
  double mx = 0.0;
  for (long e = threadIdx.x; e < total; e += blockDim.x) {
    const double2 z = c[e];
    mx = fmax(mx, fmax(fabs(z.x), fabs(z.y)));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  mx = red[0];
  int e = 0;
  if (mx > 0.0 && isfinite(mx)) {
    int ex;
    frexp(mx, &ex);  // mx = f 2^ex, f in [0.5, 1)
    e = 12 - ex;     // mx 2^e in [2^11, 2^12)
  }
  const double up = ldexp(1.0, e);
  const int tile = (s - 1) / tl.spt;
  const int c0 = ((s - 1) % tl.spt) * two_n;
  if (threadIdx.x == 0) {
    bscale[s] = ldexp(1.0, -12 - e);
    if (nblk > 0) atomicMax(&tile_nkt[tile], (nblk * two_n + kGK - 1) / kGK);
  }
  // element (K index r = i 2n + 2q + a, column col = c0 + 2j + b)
  const long count = (long)nblk * two_n * two_n;
  for (long f = threadIdx.x; f < count; f += blockDim.x) {
    const int b = (int)(f & 1);
    const int j = (int)((f >> 1) % n);
    const long r = (f >> 1) / n;
    const int a = (int)(r & 1);
    const int q = (int)((r >> 1) % n);
    const int i = (int)((r >> 1) / n);
    const double2 z = c[(size_t)i * nn + q * n + j];
    // (a, b): (re, re) -> Re, (re, im) -> Im, (im, re) -> -Im, (im, im) -> Re
    const double v = (a == b) ? z.x : (a == 0 ? z.y : -z.y);
    const float v32 = (float)(v * up);
    const __half h = __float2half_rn(v32);
    const __half l = __float2half_rn(v32 - __half2float(h));
    const int kt = (int)(r / kGK), kk = (int)(r % kGK);
    const int col = c0 + 2 * j + b;
    unsigned char *dst = bpack + ((size_t)tile * tl.nkt + kt) * tl.chunk + sw128h(col, kk);
    *reinterpret_cast<__half *>(dst) = h;
    *reinterpret_cast<__half *>(dst + (size_t)tl.NT * 128) = l;
  }
}

// ------------------------------------------------------------ tcgen05 GEMM
struct GemmArgs {
  const float *basis;  // rows x lda floats (row r: the (re, im) of blocks 0 .. cap-1)
  long lda;
  long rows;
  int kdim;            // valid K extent in reals (written blocks x 2n); beyond it A is zero
  const unsigned char *bpack;
  BasisTiles tl;
  const int *tile_nkt;
  int kt0, kt1;        // K tiles [kt0, min(kt1, tile_nkt)) of every N tile
  const double *bscale;
  int n, nshift;
  double2 *X;          // X^(s) = product or, with x_add, X^(s) += product (FP64), or
  float2 *P;           // P^(s) = product (FP32)
  long fstride;
  int x_add;
  int acc_kt;          // K tiles per accumulation chunk
  int *err;
};

namespace {
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_try(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity`: false when another role gave up (abort set)
// or after kGWaitCycles, in which case abort and the error flag are set.
__device__ __forceinline__ bool bar_wait(unsigned addr, unsigned parity, volatile int *abort_flag, int *err) {
  if (bar_try(addr, parity)) return true;
  const long long t0 = clock64();
  for (;;) {
    if (bar_try(addr, parity)) return true;
    if (*abort_flag) return false;
    if (clock64() - t0 > kGWaitCycles) {
      *abort_flag = 1;
      atomicExch(err, 1);
      return false;
    }
  }
}
// The same without the abort check (used to drain async work before exit).
__device__ __forceinline__ bool bar_drain(unsigned addr, unsigned parity) {
  if (bar_try(addr, parity)) return true;
  const long long t0 = clock64();
  while (!bar_try(addr, parity))
    if (clock64() - t0 > kGWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void bar_arrive(unsigned addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

__device__ __forceinline__ unsigned long long umma_desc(unsigned saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFF);
  d |= (unsigned long long)1 << 16;            // leading byte offset (16 B units), unused for swizzled K-major
  d |= (unsigned long long)(1024 >> 4) << 32;  // stride byte offset: 8 rows of 128 bytes
  d |= (unsigned long long)1 << 46;            // descriptor version
  d |= (unsigned long long)2 << 61;            // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void umma_f16(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                         unsigned idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

#define RHMC_TMEM_LD32(taddr, v)                                                                                     \
  asm volatile(                                                                                                      \
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"  \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                                 \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), \
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),     \
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),    \
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])                  \
      : "r"(taddr))

#define RHMC_TMEM_LD16(taddr, v)                                                                                     \
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),       \
                 "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])  \
               : "r"(taddr))

#define RHMC_TMEM_ST16(taddr, v)                                                                                     \
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" \
               ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),   \
               "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])          \
               : "memory")

#define RHMC_TMEM_ST32(taddr, v)                                                                                     \
  asm volatile(                                                                                                      \
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18," \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),                                        \
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),  \
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),   \
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),   \
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])                                                                 \
      : "memory")

// Work item w: row tile mt, N tile nt (rotated by mt so that static
// round-robin spreads the long and the short N tiles evenly), and its K tiles.
__device__ __forceinline__ bool work_item(const GemmArgs &g, long w, long &mt, int &nt, int &nkt) {
  mt = w / g.tl.nnt;
  nt = (int)((w + mt) % g.tl.nnt);
  nkt = min(g.tile_nkt[nt], g.kt1) - g.kt0;
  return nkt > 0;
}

__device__ __forceinline__ float4 load_a4(const GemmArgs &g, long gr, int k) {
  if (gr >= g.rows || k >= g.kdim) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float *p = g.basis + gr * g.lda + k;
  if (k + 4 <= g.kdim) return __ldg(reinterpret_cast<const float4 *>(p));
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  v.x = p[0];
  if (k + 1 < g.kdim) v.y = p[1];
  if (k + 2 < g.kdim) v.z = p[2];
  return v;
}

__device__ __forceinline__ void split_store(unsigned char *hi, unsigned char *lo, unsigned off, float4 v) {
  v.x *= kGAScale, v.y *= kGAScale, v.z *= kGAScale, v.w *= kGAScale;
  const __half2 h01 = __floats2half2_rn(v.x, v.y), h23 = __floats2half2_rn(v.z, v.w);
  const float2 b01 = __half22float2(h01), b23 = __half22float2(h23);
  const __half2 l01 = __floats2half2_rn(v.x - b01.x, v.y - b01.y), l23 = __floats2half2_rn(v.z - b23.x, v.w - b23.y);
  uint2 hv, lv;
  hv.x = *reinterpret_cast<const unsigned *>(&h01);
  hv.y = *reinterpret_cast<const unsigned *>(&h23);
  lv.x = *reinterpret_cast<const unsigned *>(&l01);
  lv.y = *reinterpret_cast<const unsigned *>(&l23);
  *reinterpret_cast<uint2 *>(hi + off) = hv;
  *reinterpret_cast<uint2 *>(lo + off) = lv;
}
}  // namespace

__global__ void __launch_bounds__(kGThreads, 1) k_basis_gemm_tc(const GemmArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = smem_raw;
  base += (1024 - (smem_addr(smem_raw) & 1023)) & 1023;
  const unsigned stage_bytes = 2 * kGAPiece + 2u * g.tl.NT * 128;
  __shared__ __align__(8) unsigned long long bar_full_a[kGStages], bar_full_b[kGStages], bar_empty[kGStages];
  __shared__ __align__(8) unsigned long long bar_acc_full[2], bar_acc_empty[2], bar_final;
  __shared__ unsigned tmem_sh;
  __shared__ volatile int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_addr(&tmem_sh)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < kGStages; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar_full_a[q])), "r"(128));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_full_b[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_empty[q])));
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_acc_full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar_acc_empty[q])), "r"(256));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar_final)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    abort_sh = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = tmem_sh;
  const long mtiles = (g.rows + kGM - 1) / kGM;
  const long total = mtiles * g.tl.nnt;
  const int two_n = 2 * g.n;

  if (warp < 8) {
    // ---- A producers: FP32 basis rows -> scaled FP16 pieces (hi, lo) in shared memory.  Group
    // warp / 4 fills the K tiles with it & 1 == group (stage slot it % kGStages), so each group's
    // loads for its next tile are in flight while the MMAs of the tiles before it run.
    const int grp = warp >> 2, cw = warp & 3;
    const int half = lane >> 4, q = lane & 15;
    int it = 0;
    bool ok = true;
    for (long w = blockIdx.x; w < total && ok; w += gridDim.x) {
      long mt;
      int nt, nkt;
      if (!work_item(g, w, mt, nt, nkt)) continue;
      const long m0 = mt * kGM;
      const bool rows_in = m0 + kGM <= g.rows;
      for (int kk = 0; kk < nkt; ++kk, ++it) {
        if ((it & 1) != grp) continue;
        const int stage = it % kGStages;
        const int kt = g.kt0 + kk;
        const int k = kt * kGK + 4 * q;
        float4 v[16];
        if (rows_in && (kt + 1) * kGK <= g.kdim) {
          const float *src = g.basis + (m0 + 32 * cw + half) * g.lda + k;
#pragma unroll
          for (int r = 0; r < 16; ++r) v[r] = __ldg(reinterpret_cast<const float4 *>(src + 2 * r * g.lda));
        } else {
#pragma unroll
          for (int r = 0; r < 16; ++r) v[r] = load_a4(g, m0 + 32 * cw + 2 * r + half, k);
        }
        ok = bar_wait(smem_addr(&bar_empty[stage]), ((it / kGStages) & 1) ^ 1, &abort_sh, g.err);
        if (!ok) break;
        unsigned char *ahi = base + stage * stage_bytes, *alo = ahi + kGAPiece;
#pragma unroll
        for (int r = 0; r < 16; ++r) {
          const int row = 32 * cw + 2 * r + half;
          const unsigned off = (unsigned)((row >> 3) * 1024 + (row & 7) * 128 + ((((q >> 1) ^ (row & 7)) & 7) << 4) +
                                          (q & 1) * 8);
          split_store(ahi, alo, off, v[r]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        bar_arrive(smem_addr(&bar_full_a[stage]));
      }
    }
  } else if (warp < 16) {
    // ---- epilogue: per chunk, accumulator -> running sum (tensor memory, FP32 round-to-nearest);
    // after the last chunk running sum + accumulator -> X^(s) (FP64) or P^(s) (FP32)
    const int ew = warp & 3;         // tensor-memory lanes 32 ew .. 32 ew + 31 (a warp reaches lanes 32 (warp % 4) ..)
    const int cb = (warp - 8) >> 2;  // column half of the tile
    const unsigned tlane = tmem + ((unsigned)(32 * ew) << 16), trun = tlane + 2 * kGNmax;
    int cc = 0;
    bool ok = true;
    for (long w = blockIdx.x; w < total && ok; w += gridDim.x) {
      long mt;
      int nt, nkt;
      if (!work_item(g, w, mt, nt, nkt)) continue;
      const long row = mt * kGM + 32 * ew + lane;
      const int s_first = 1 + nt * g.tl.spt;
      const int ncols = min(g.tl.spt, g.nshift - s_first) * two_n;
      const int nch = (nkt + g.acc_kt - 1) / g.acc_kt;
      for (int ch = 0; ch < nch; ++ch, ++cc) {
        const int buf = cc & 1;
        ok = bar_wait(smem_addr(&bar_acc_full[buf]), (cc >> 1) & 1, &abort_sh, g.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const bool last = ch + 1 == nch;
        const unsigned tacc = tlane + (unsigned)(buf * kGNmax);
        for (int c0 = cb * (kGNmax / 2); c0 < min(ncols, (cb + 1) * (kGNmax / 2)); c0 += 16) {
          unsigned a[16];
          RHMC_TMEM_LD16(tacc + (unsigned)c0, a);
          if (ch > 0) {
            unsigned r[16];
            RHMC_TMEM_LD16(trun + (unsigned)c0, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int e = 0; e < 16; ++e) a[e] = __float_as_uint(__uint_as_float(a[e]) + __uint_as_float(r[e]));
          } else {
            asm volatile("tcgen05.wait::ld.sync.aligned;");
          }
          if (!last) {
            RHMC_TMEM_ST16(trun + (unsigned)c0, a);
            continue;
          }
          if (row >= g.rows) continue;
          double2 xv[8];
          if (g.X && g.x_add) {
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {  // eight loads in flight before their stores
              const int col = c0 + 2 * jj;
              if (col < ncols) xv[jj] = g.X[(s_first + col / two_n) * g.fstride + row * g.n + ((col % two_n) >> 1)];
            }
          }
#pragma unroll
          for (int jj = 0; jj < 8; ++jj) {
            const int col = c0 + 2 * jj;
            if (col >= ncols) continue;
            const int sh = s_first + col / two_n;
            const long o = sh * g.fstride + row * g.n + ((col % two_n) >> 1);
            const double sc = g.bscale[sh];
            double re = (double)__uint_as_float(a[2 * jj]) * sc;
            double im = (double)__uint_as_float(a[2 * jj + 1]) * sc;
            if (g.X) {
              if (g.x_add) re += xv[jj].x, im += xv[jj].y;
              g.X[o] = make_double2(re, im);
            } else {
              g.P[o] = make_float2((float)re, (float)im);
            }
          }
        }
        asm volatile("tcgen05.wait::st.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        bar_arrive(smem_addr(&bar_acc_empty[buf]));
      }
    }
  } else if (warp == 16) {
    // ---- B producer: one bulk copy of the packed FP16 pieces per stage
    if (lane == 0) {
      int it = 0;
      bool ok = true;
      for (long w = blockIdx.x; w < total && ok; w += gridDim.x) {
        long mt;
        int nt, nkt;
        if (!work_item(g, w, mt, nt, nkt)) continue;
        for (int kk = 0; kk < nkt; ++kk, ++it) {
          const int stage = it % kGStages;
          ok = bar_wait(smem_addr(&bar_empty[stage]), ((it / kGStages) & 1) ^ 1, &abort_sh, g.err);
          if (!ok) break;
          const unsigned bar = smem_addr(&bar_full_b[stage]);
          const unsigned dst = smem_addr(base + stage * stage_bytes + 2 * kGAPiece);
          const unsigned char *src = g.bpack + ((size_t)nt * g.tl.nkt + g.kt0 + kk) * g.tl.chunk;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((unsigned)g.tl.chunk)
                       : "memory");
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
              "l"(src), "r"((unsigned)g.tl.chunk), "r"(bar)
              : "memory");
        }
      }
      // copies still in flight (only after a failed wait) land before the CTA's memory is released
      if (abort_sh)
        for (int j = max(0, it - kGStages); j < it; ++j)
          bar_drain(smem_addr(&bar_full_b[j % kGStages]), (j / kGStages) & 1);
    }
  } else {
    // ---- MMA issuer: three FP16 products per K step, one accumulator per chunk of K tiles
    if (lane == 0) {
      const unsigned idesc = (1u << 4) | ((unsigned)(g.tl.NT >> 3) << 17) | ((unsigned)(kGM >> 4) << 24);
      int it = 0, cc = 0;
      bool ok = true;
      for (long w = blockIdx.x; w < total && ok; w += gridDim.x) {
        long mt;
        int nt, nkt;
        if (!work_item(g, w, mt, nt, nkt)) continue;
        for (int c0 = 0; c0 < nkt && ok; c0 += g.acc_kt, ++cc) {
          const int buf = cc & 1;
          ok = bar_wait(smem_addr(&bar_acc_empty[buf]), ((cc >> 1) & 1) ^ 1, &abort_sh, g.err);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;");
          const unsigned dt = tmem + (unsigned)(buf * kGNmax);
          const int c1 = min(c0 + g.acc_kt, nkt);
          for (int kk = c0; kk < c1; ++kk, ++it) {
            const int stage = it % kGStages;
            const unsigned par = (it / kGStages) & 1;
            ok = bar_wait(smem_addr(&bar_full_a[stage]), par, &abort_sh, g.err) &&
                 bar_wait(smem_addr(&bar_full_b[stage]), par, &abort_sh, g.err);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned sa = smem_addr(base + stage * stage_bytes);
            const unsigned sb = sa + 2 * kGAPiece;
            // (A piece, B piece): (lo, hi), (hi, lo), (hi, hi) -- smallest first
            const int pa[3] = {1, 0, 0}, pb[3] = {0, 1, 0};
#pragma unroll
            for (int p = 0; p < 3; ++p)
#pragma unroll
              for (int ks = 0; ks < 4; ++ks)  // K = 64 halves = 4 steps of 16 (32 bytes) inside the swizzle row
                umma_f16(dt, umma_desc(sa + pa[p] * kGAPiece + ks * 32),
                         umma_desc(sb + pb[p] * g.tl.NT * 128 + ks * 32), idesc, (kk - c0) | p | ks);
            umma_commit(smem_addr(&bar_empty[stage]));
          }
          if (!ok) break;
          umma_commit(smem_addr(&bar_acc_full[buf]));
        }
      }
      // every MMA this thread issued has completed before tensor memory is released
      umma_commit(smem_addr(&bar_final));
      bar_drain(smem_addr(&bar_final), 0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
}

// ------------------------------------------------------------ CUDA-core alternative
// X^(s) (+)= sum_{i in [kb0, kb1)} Q_i C_i (or P^(s) = ...): one thread per
// (row, output column) of one shift; FP32 products over the n inputs of a
// block, FP64 sum over blocks.
__global__ void __launch_bounds__(256) k_basis_gemm_simt(const float2 *__restrict__ basis, int cap, long rows, int n,
                                                         int nshift, const SolverState *__restrict__ st, int K,
                                                         int want_p, const double2 *__restrict__ cf, long cfstride,
                                                         int kb0, int kb1, int x_add, double2 *X, float2 *P,
                                                         long fstride) {
  const int s = blockIdx.y + 1;
  if (s >= nshift) return;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * n) return;
  const long r = e / n;
  const int j = (int)(e - r * n);
  const int nblk = min(basis_nblk(st, s, K, want_p), kb1);
  const int nn = n * n;
  const double2 *c = cf + (size_t)(s - 1) * cfstride * nn;
  const float2 *qrow = basis + r * (long)cap * n;
  double ar = 0.0, ai = 0.0;
  for (int i = kb0; i < nblk; ++i) {
    float pr = 0.f, pi = 0.f;
    for (int q = 0; q < n; ++q) {
      const float2 a = qrow[(long)i * n + q];
      const double2 z = c[(size_t)i * nn + q * n + j];
      const float zr = (float)z.x, zi = (float)z.y;
      pr = fmaf(a.x, zr, fmaf(-a.y, zi, pr));
      pi = fmaf(a.x, zi, fmaf(a.y, zr, pi));
    }
    ar += pr;
    ai += pi;
  }
  const long o = s * fstride + e;
  if (X) {
    if (x_add) {
      const double2 x = X[o];
      ar += x.x, ai += x.y;
    }
    X[o] = make_double2(ar, ai);
  } else {
    P[o] = make_float2((float)ar, (float)ai);
  }
}

// ------------------------------------------------------------ host
rhmc_status_t basis_assemble(const BasisBufs &bb, int n, int nshift, const SolverState *st, long rows, int K,
                             int want_p, double2 *X, float2 *P, long fstride, int chunk_blocks, int simt, int acc_kt,
                             int *err, cudaStream_t s) {
  if (nshift < 2 || (K <= 0 && !want_p)) return RHMC_OK;
  const long cfstride = bb.cap + 1;
  prof_begin(PROF_NXN_SHIFTS, s);
  k_basis_coef<<<nshift - 1, 256, 0, s>>>(n, nshift, st, bb.hist, K, want_p, bb.cf, cfstride);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  const int nblk_all = want_p ? K + 1 : K;
  const double out_bytes = (double)rows * n * (nshift - 1) * (want_p ? sizeof(float2) : sizeof(double2));
  if (simt) {
    const int chunk = (!want_p && chunk_blocks > 0) ? chunk_blocks : nblk_all;
    for (int b0 = 0; b0 < nblk_all; b0 += chunk) {
      const dim3 grid((unsigned)((rows * n + 255) / 256), (unsigned)(nshift - 1));
      prof_begin(PROF_OTHER, s);
      k_basis_gemm_simt<<<grid, 256, 0, s>>>(bb.basis, bb.cap, rows, n, nshift, st, K, want_p, bb.cf, cfstride, b0,
                                             std::min(b0 + chunk, nblk_all), b0 > 0, X, P, fstride);
      prof_end(s, (double)rows * n * std::min(chunk, nblk_all - b0) * sizeof(float2) + out_bytes * (b0 > 0 ? 2 : 1));
      RHMC_LAUNCH_CHECK();
    }
    return RHMC_OK;
  }
  const BasisTiles tl = basis_tiles(n, nshift, bb.cap);
  RHMC_CUDA_TRY(cudaMemsetAsync(bb.bpack, 0, (size_t)tl.nnt * tl.nkt * tl.chunk, s));
  RHMC_CUDA_TRY(cudaMemsetAsync(bb.tile_nkt, 0, sizeof(int) * tl.nnt, s));
  prof_begin(PROF_NXN_SHIFTS, s);
  k_basis_pack<<<nshift - 1, 256, 0, s>>>(n, nshift, st, K, want_p, bb.cf, cfstride, tl, bb.bpack, bb.bscale,
                                          bb.tile_nkt);
  prof_end(s, 0.0);
  RHMC_LAUNCH_CHECK();
  const size_t smem = 1024 + (size_t)kGStages * (2 * kGAPiece + (size_t)tl.NT * 256);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_basis_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(1024 + kGStages * (2 * kGAPiece + kGNmax * 256)));
  });
  GemmArgs g{};
  g.basis = reinterpret_cast<const float *>(bb.basis);
  g.lda = (long)bb.cap * 2 * n;
  g.rows = rows;
  g.kdim = std::min(K + 1, bb.cap) * 2 * n;  // blocks 0 .. K are written
  g.bpack = bb.bpack;
  g.tl = tl;
  g.tile_nkt = bb.tile_nkt;
  g.bscale = bb.bscale;
  g.n = n;
  g.nshift = nshift;
  g.X = want_p ? nullptr : X;
  g.P = want_p ? P : nullptr;
  g.fstride = fstride;
  g.acc_kt = acc_kt > 0 ? acc_kt : kGChunkKt;
  g.err = err;
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long mtiles = (rows + kGM - 1) / kGM;
  const int grid = (int)std::min<long>(mtiles * tl.nnt, std::max(nsm, 1));
  const int kt_all = (nblk_all * 2 * n + kGK - 1) / kGK;
  const int chunk_kt = (!want_p && chunk_blocks > 0) ? std::max(1, chunk_blocks * 2 * n / kGK) : kt_all;
  for (int kt0 = 0; kt0 < kt_all; kt0 += chunk_kt) {
    g.kt0 = kt0;
    g.kt1 = std::min(kt0 + chunk_kt, kt_all);
    g.x_add = kt0 > 0;  // X^(s), s >= 1, is zero before the assembly: the first K range stores
    prof_begin(PROF_BASIS_TC, s);
    k_basis_gemm_tc<<<grid, kGThreads, smem, s>>>(g);
    prof_end(s, (double)rows * (g.kt1 - kt0) * kGK * sizeof(float) + out_bytes * (kt0 > 0 ? 2 : 1));
    RHMC_LAUNCH_CHECK();
    if (prof_on()) {  // the MMA flops issued: three FP16 products per (row tile, N tile, K tile)
      int h[kMaxS];
      RHMC_CUDA_TRY(cudaMemcpyAsync(h, bb.tile_nkt, sizeof(int) * tl.nnt, cudaMemcpyDeviceToHost, s));
      RHMC_CUDA_TRY(cudaStreamSynchronize(s));
      double kts = 0.0;
      for (int t = 0; t < tl.nnt; ++t) kts += std::max(0, std::min(h[t], g.kt1) - kt0);
      prof_flops(3.0 * 2.0 * kGM * tl.NT * kGK * kts * mtiles);
    }
  }
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

}  // namespace rhmc
