// Shifted updates of SBCGrQ on the 5th-generation tensor cores (tcgen05).
//
// Algorithm 1's shifted updates for every shift updated in this iteration:
//   X^(s) += P^(s) alpha^(s)_k,   P^(s) = Q_k + P^(s) beta^(s)_k rho_k^dagger.
// Per 128-row tile of P^(s) (n = 16 complex = 32 reals per row) this is one
// real GEMM  D[128 x 64] = P[128 x 32] * B[32 x 64]  with B the real embedding
// of [alpha^(s) | beta^(s) rho^dagger]:
//   B[2k+0][2j+0] = Re M_kj,  B[2k+1][2j+0] = -Im M_kj,
//   B[2k+0][2j+1] = Im M_kj,  B[2k+1][2j+1] =  Re M_kj,
// so that row (p_0re, p_0im, p_1re, ...) * B gives (y_0re, y_0im, ...) = p M.
//
// FP32 accuracy from TF32 inputs: every operand is split exactly into three
// TF32 pieces, a = a0 + a1 + a2 with a0 = rna_tf32(a), a1 = rna_tf32(a - a0),
// a2 = rna_tf32(a - a0 - a1) (each difference is exact in FP32 and the pieces
// carry 11 + 11 + 2 significant bits), and D accumulates the six products
// whose order is above 2^-33 of the result, smallest first:
//   A2 B0 + A0 B2 + A1 B1 + A1 B0 + A0 B1 + A0 B0,
// in FP32 in tensor memory.  (A head + tail split keeps only about 22 of
// FP32's 24 bits and shows up as a larger drift of the shifted systems.)
//
// Per CTA (128 threads, one row per thread, three CTAs per SM): the threads
// load their rows of P^(s) and X^(s), write the split P tile to shared memory
// in the 128-byte-swizzled K-major layout; the B pieces of the shift (laid out
// once per iteration by k_tc_prepare_b) arrive by one bulk copy on an
// mbarrier; one thread issues the 24 tcgen05.mma (K = 32 in steps of 8, six
// products), commits them to a second mbarrier and, once they are done,
// starts the bulk copy of the next shift's B pieces; the threads then read
// their row of D with tcgen05.ld and write X^(s) and P^(s).  Every mbarrier
// wait is bounded: one that gives up sets an error flag, the kernel waits
// (bounded) for its copies and MMAs in flight, frees its tensor memory and
// returns.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

namespace {

constexpr int kTcRows = 128;         // tile rows (MMA M)
constexpr int kTcK = 32;             // reals per row (MMA K)
constexpr int kTcN = 64;             // output reals per row (MMA N): M1 | M2
constexpr int kTcCols = 64;          // tensor-memory columns allocated

// Byte offset of (row, k) in a K-major tile of 32-bit elements with 128-byte
// rows under the 128-byte swizzle: 16-byte chunk c of row r sits at chunk
// position c ^ (r & 7) within its 1024-byte group of 8 rows.
__host__ __device__ constexpr unsigned sw128(int row, int k) {
  return (unsigned)((row >> 3) * 1024 + (row & 7) * 128 + (((k >> 2) ^ (row & 7)) << 4) + (k & 3) * 4);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (unused for swizzled K-major), stride byte offset = 1024 (8 rows),
// descriptor version 1, 128-byte swizzle.
__device__ __forceinline__ unsigned long long make_desc(unsigned saddr) {
  unsigned long long d = 0;
  d |= (unsigned long long)((saddr >> 4) & 0x3FFF);
  d |= (unsigned long long)(1) << 16;             // leading byte offset (16 B units), ignored here
  d |= (unsigned long long)(1024 >> 4) << 32;     // stride byte offset
  d |= (unsigned long long)1 << 46;               // descriptor version
  d |= (unsigned long long)2 << 61;               // layout: 128-byte swizzle
  return d;
}

// Instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128.
constexpr unsigned kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((unsigned)(kTcN >> 3) << 17) |
                            ((unsigned)(kTcRows >> 4) << 24);

__device__ __forceinline__ float tf32_rna(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(unsigned dtmem, unsigned long long adesc, unsigned long long bdesc,
                                         int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_try_wait(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the mbarrier at addr for at most `cycles` SM
// clocks; false if the wait gave up.
__device__ __forceinline__ bool mbar_wait_for(unsigned addr, unsigned parity, long long cycles) {
  if (mbar_try_wait(addr, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(addr, parity))
    if (clock64() - t0 > cycles) return false;
  return true;
}
constexpr long long kWaitCycles = 2000000000LL;  // about a second at the GPU's 2 GHz

#define RHMC_TMEM_LD64(taddr, v)                                                                                      \
  asm volatile(                                                                                                       \
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"   \
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45," \
      "%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"                              \
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),  \
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),      \
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),     \
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]), "=r"(v[32]),     \
        "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]), "=r"(v[40]),     \
        "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]),     \
        "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]), "=r"(v[56]),     \
        "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])                   \
      : "r"(taddr))

}  // namespace

constexpr int kPieces = 3;
constexpr int kBTile = kTcN * kTcK;                               // floats per B piece
constexpr unsigned kBBytes = (unsigned)(kPieces * kBTile * sizeof(float));  // one shift's B pieces

// B pieces for every shift in [s_begin, s_end): [s][piece][64 x 32 floats,
// swizzled K-major, row n = output real index, k = input real index].
__global__ void __launch_bounds__(256) k_tc_prepare_b(const float2 *__restrict__ coef, int s_begin, int s_end,
                                                      float *__restrict__ btiles) {
  const int s = s_begin + blockIdx.x;
  if (s >= s_end) return;
  constexpr int N = 16;
  const float2 *m1 = coef + (1 + 2 * s) * N * N;
  const float2 *m2 = m1 + N * N;
  float *b0 = btiles + (size_t)s * kPieces * kBTile;
  for (int e = threadIdx.x; e < kBTile; e += blockDim.x) {
    const int n = e / kTcK, k = e % kTcK;  // B[k][n]
    const float2 *M = n < 32 ? m1 : m2;
    const int j = (n & 31) >> 1, b = n & 1, kc = k >> 1, a = k & 1;
    const float2 z = M[kc * N + j];
    // (a, b): (re, re) -> Re, (im, re) -> -Im, (re, im) -> Im, (im, im) -> Re
    const float v = (a == b) ? z.x : (a == 1 ? -z.y : z.y);
    const float p0 = tf32_rna(v);
    const float r1 = v - p0;
    const float p1 = tf32_rna(r1);
    const unsigned off = sw128(n, k) / 4;
    b0[off] = p0;
    b0[kBTile + off] = p1;
    b0[2 * kBTile + off] = tf32_rna(r1 - p1);
  }
}

__device__ __forceinline__ void mbar_expect_bulk(unsigned mbar, unsigned dst, const void *src, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__global__ void __launch_bounds__(kTcRows, 3) k_update_tc(const float2 *__restrict__ Q, float2 *__restrict__ P,
                                                       float2 *__restrict__ X, const float *__restrict__ btiles,
                                                       const int *__restrict__ upd, int s_begin, int s_end, long rows,
                                                       long fstride, int *__restrict__ err) {
  // shared: A pieces (3 x 16 KB), B pieces (3 x 8 KB, one bulk-copy target), all 1024-aligned
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = smem_raw;
  {  // align to 1024 bytes for the swizzle pattern
    const unsigned a = smem_u32(smem_raw);
    base += (1024 - (a & 1023)) & 1023;
  }
  float *As = reinterpret_cast<float *>(base);  // [3][128 x 32]
  float *Bs = As + kPieces * kTcRows * kTcK;    // [3][64 x 32]
  __shared__ __align__(8) unsigned long long mbar_mma, mbar_b;
  __shared__ unsigned tmem_base_sh;
  __shared__ int ok_sh, b_pending;
  __shared__ int live[kMaxS];
  __shared__ int nlive;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (tid == 0) {
    int m = 0;
    for (int q = s_begin; q < s_end; ++q)
      if (upd[q]) live[m++] = q;
    nlive = m;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  const unsigned amma = smem_u32(&mbar_mma), ab = smem_u32(&mbar_b);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(amma));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(ab));
    asm volatile("fence.mbarrier_init.release.cluster;");
    ok_sh = 1;
    b_pending = 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = tmem_base_sh;
  const int nl = nlive;
  const unsigned sA = smem_u32(As), sB = smem_u32(Bs);
  unsigned ph_mma = 0, ph_b = 0;
  const long ntiles = (rows + kTcRows - 1) / kTcRows;
  // the first work item's B pieces
  if (tid == 0 && nl > 0 && blockIdx.x < ntiles) {
    mbar_expect_bulk(ab, sB, btiles + (size_t)live[0] * kPieces * kBTile, kBBytes);
    b_pending = 1;
  }
  for (long tile = blockIdx.x; tile < ntiles && nl > 0; tile += gridDim.x) {
    const long r = tile * kTcRows + tid;
    const bool rlive = r < rows;
    float q[kTcK];
    {
      const float4 *src = reinterpret_cast<const float4 *>(Q + r * 16);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = rlive ? src[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        q[4 * c] = v.x, q[4 * c + 1] = v.y, q[4 * c + 2] = v.z, q[4 * c + 3] = v.w;
      }
    }
    int i = 0;
    for (; i < nl; ++i) {
      const int s = live[i];
      float2 *Ps = P + s * fstride;
      float2 *Xs = X + s * fstride;
      float4 xv[8];
      {  // this thread's rows of X^(s) and P^(s); P split into the three pieces, swizzled
        const float4 *xsrc = reinterpret_cast<const float4 *>(Xs + r * 16);
        const float4 *psrc = reinterpret_cast<const float4 *>(Ps + r * 16);
#pragma unroll
        for (int c = 0; c < 8; ++c) xv[c] = rlive ? xsrc[c] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = rlive ? psrc[c] : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 p0 = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
          const float4 r1 = make_float4(v.x - p0.x, v.y - p0.y, v.z - p0.z, v.w - p0.w);
          const float4 p1 = make_float4(tf32_rna(r1.x), tf32_rna(r1.y), tf32_rna(r1.z), tf32_rna(r1.w));
          const float4 p2 = make_float4(tf32_rna(r1.x - p1.x), tf32_rna(r1.y - p1.y), tf32_rna(r1.z - p1.z),
                                        tf32_rna(r1.w - p1.w));
          unsigned char *a0 = reinterpret_cast<unsigned char *>(As) + sw128(tid, 4 * c);
          *reinterpret_cast<float4 *>(a0) = p0;
          *reinterpret_cast<float4 *>(a0 + kTcRows * kTcK * 4) = p1;
          *reinterpret_cast<float4 *>(a0 + 2 * kTcRows * kTcK * 4) = p2;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        bool ok = mbar_wait_for(ab, ph_b, kWaitCycles);  // this shift's B pieces
        b_pending = ok ? 0 : 1;
        if (ok) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          // products (A piece, B piece), smallest first
          const int pa[6] = {2, 0, 1, 1, 0, 0}, pb[6] = {0, 2, 1, 0, 1, 0};
#pragma unroll
          for (int t = 0; t < 6; ++t)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {  // K = 32 reals = 4 steps of 8 (32 bytes) inside the swizzle atom
              const unsigned aoff = sA + pa[t] * (kTcRows * kTcK * 4) + kk * 32;
              const unsigned boff = sB + pb[t] * (kBTile * 4) + kk * 32;
              mma_tf32(tmem, make_desc(aoff), make_desc(boff), (t > 0 || kk > 0) ? 1 : 0);
            }
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(amma)
                       : "memory");
          ok = mbar_wait_for(amma, ph_mma, kWaitCycles);
          if (!ok) mbar_wait_for(amma, ph_mma, kWaitCycles);  // one more bounded chance before memory is reused
        }
        if (!ok) {
          ok_sh = 0;
          atomicExch(err, 1);
        } else {
          // the next work item's B pieces (the MMAs reading Bs are done)
          const bool next_in_tile = i + 1 < nl;
          const bool next_tile = tile + gridDim.x < ntiles;
          if (next_in_tile || next_tile) {
            const int sn = next_in_tile ? live[i + 1] : live[0];
            mbar_expect_bulk(ab, sB, btiles + (size_t)sn * kPieces * kBTile, kBBytes);
            b_pending = 1;
          }
        }
      }
      __syncthreads();
      ph_b ^= 1;
      ph_mma ^= 1;
      if (!ok_sh) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned d[64];
      RHMC_TMEM_LD64(tmem + ((unsigned)(warp * 32) << 16), d);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (rlive) {
        float4 *xs = reinterpret_cast<float4 *>(Xs + r * 16);
        float4 *ps = reinterpret_cast<float4 *>(Ps + r * 16);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float4 x = xv[c];
          x.x += __uint_as_float(d[4 * c]);
          x.y += __uint_as_float(d[4 * c + 1]);
          x.z += __uint_as_float(d[4 * c + 2]);
          x.w += __uint_as_float(d[4 * c + 3]);
          xs[c] = x;
          ps[c] = make_float4(q[4 * c] + __uint_as_float(d[32 + 4 * c]), q[4 * c + 1] + __uint_as_float(d[33 + 4 * c]),
                              q[4 * c + 2] + __uint_as_float(d[34 + 4 * c]),
                              q[4 * c + 3] + __uint_as_float(d[35 + 4 * c]));
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncthreads();  // tensor memory and the A pieces are rewritten by the next item
    }
    if (!ok_sh) break;
  }
  __syncthreads();
  // a bulk copy still in flight (only after a failed wait) lands before the CTA's memory is released
  if (tid == 0 && b_pending) mbar_wait_for(ab, ph_b, kWaitCycles);
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// Shifts [s_begin, s_end) with the tensor cores (mixed path, n = 16).
// btiles: 3 * 64 * 32 floats per shift of scratch; err: device flag.
rhmc_status_t update_shifts_tc(const float2 *Q, float2 *P, float2 *X, const float2 *coef, const int *upd,
                               int s_begin, int s_end, long rows, long fstride, float *btiles, int *err,
                               cudaStream_t s) {
  if (s_end <= s_begin) return RHMC_OK;
  if (((uintptr_t)btiles & 15) != 0) return RHMC_ERR_INVALID_ARG;  // bulk-copy source alignment
  k_tc_prepare_b<<<s_end - s_begin, 256, 0, s>>>(coef, s_begin, s_end, btiles);
  RHMC_LAUNCH_CHECK();
  const size_t smem = 1024 + (size_t)kPieces * (kTcRows * kTcK + kBTile) * sizeof(float);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const long tiles = (rows + kTcRows - 1) / kTcRows;
  const int grid = (int)std::min<long>(tiles, resident_ctas(k_update_tc, kTcRows, smem));
  int nupd = s_end - s_begin;
  if (prof_on()) {
    int h[kMaxS];
    cudaStreamSynchronize(s);
    cudaMemcpy(h, upd, sizeof(int) * s_end, cudaMemcpyDeviceToHost);
    nupd = 0;
    for (int q = s_begin; q < s_end; ++q) nupd += h[q] != 0;
  }
  prof_begin(PROF_UPDATE_TC, s);
  k_update_tc<<<grid, kTcRows, smem, s>>>(Q, P, X, btiles, upd, s_begin, s_end, rows, fstride, err);
  prof_end(s, (double)rows * 16 * sizeof(float2) * (1.0 + 4.0 * nupd));
  RHMC_LAUNCH_CHECK();
  return RHMC_OK;
}


// Self-test of the bounded wait: one warp waits on an mbarrier that nothing
// arrives at; the wait must give up after `cycles` clocks and set *err.
__global__ void k_wait_selftest(int *err, long long cycles) {
  __shared__ __align__(8) unsigned long long bar;
  const unsigned addr = smem_u32(&bar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(addr));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (!mbar_wait_for(addr, 0, cycles) && threadIdx.x == 0) atomicExch(err, 1);
}

}  // namespace rhmc

extern "C" rhmc_status_t rhmc_selftest_bounded_wait(int device, double seconds, rhmc_stream_t sv) {
  using namespace rhmc;
  if (!(seconds > 0.0 && seconds <= 2.0)) {
    set_error("rhmc_selftest_bounded_wait: seconds must be in (0, 2]");
    return RHMC_ERR_INVALID_ARG;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) RHMC_CUDA_TRY(cudaSetDevice(device));
  int khz = 0;
  cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device);
  const long long cycles = (long long)(seconds * (khz > 0 ? khz : 2000000) * 1e3);
  int *flag = nullptr;
  rhmc_status_t rc = RHMC_OK;
  cudaStream_t s = (cudaStream_t)sv;
  if (cudaMalloc(&flag, sizeof(int)) != cudaSuccess) {
    set_error("rhmc_selftest_bounded_wait: cudaMalloc failed");
    rc = RHMC_ERR_CUDA;
  } else {
    int h = 0;
    cudaMemsetAsync(flag, 0, sizeof(int), s);
    k_wait_selftest<<<1, 32, 0, s>>>(flag, cycles);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess) {
      if (h) {
        set_error("bounded device wait expired (self-test: nothing arrives at the barrier)");
        rc = RHMC_ERR_DEVICE_TIMEOUT;
      }
    } else {
      set_error("rhmc_selftest_bounded_wait: %s", cudaGetErrorString(e != cudaSuccess ? e : cudaGetLastError()));
      rc = RHMC_ERR_CUDA;
    }
    cudaFree(flag);
  }
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
