// Shifted updates of SBCGrQ on the 5th-generation tensor cores (tcgen05).
//
// Algorithm 1, lines 11-12, for every shift updated in this iteration:
//   X^(s) += P^(s) alpha^(s)_k,   P^(s) = Q_k + P^(s) beta^(s)_k rho_k^dagger.
// Per 128-row tile of P^(s) (n = 16 complex = 32 reals per row) this is one
// real GEMM  D[128 x 64] = P[128 x 32] * B[32 x 64]  with B the real embedding
// of [alpha^(s) | beta^(s) rho^dagger]:
//   B[2k+0][2j+0] = Re M_kj,  B[2k+1][2j+0] = -Im M_kj,
//   B[2k+0][2j+1] = Im M_kj,  B[2k+1][2j+1] =  Re M_kj,
// so that row (p_0re, p_0im, p_1re, ...) * B gives (y_0re, y_0im, ...) = p M.
//
// FP32 accuracy from TF32 inputs ("3xTF32"): every operand is split into a
// TF32 head and a TF32 tail, a = ah + al with ah = rna_tf32(a), al =
// rna_tf32(a - ah), and D = Ah Bh + Ah Bl + Al Bh accumulates in FP32 in tensor
// memory (the Al Bl term is below FP32 rounding).
//
// Per CTA (128 threads, one row per thread): the threads write the split P
// tile to shared memory in the 128-byte-swizzled K-major layout, copy the
// (pre-laid-out) B tiles, one elected thread issues the 12 tcgen05.mma
// (K = 32 in steps of 8, three products) and commits them to an mbarrier;
// after a bounded wait the threads read their row of D with tcgen05.ld and
// update X^(s) and P^(s).  A wait that does not finish within its iteration
// limit sets an error flag; the kernel then frees its tensor memory and
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

// B tiles for every shift in [s_begin, s_end): [s][head, tail][64 x 32 floats,
// swizzled K-major, row n = output real index, k = input real index].
__global__ void __launch_bounds__(256) k_tc_prepare_b(const float2 *__restrict__ coef, int s_begin, int s_end,
                                                      float *__restrict__ btiles) {
  const int s = s_begin + blockIdx.x;
  if (s >= s_end) return;
  constexpr int N = 16;
  const float2 *m1 = coef + (1 + 2 * s) * N * N;
  const float2 *m2 = m1 + N * N;
  float *hi = btiles + (size_t)s * 2 * kTcN * kTcK;
  float *lo = hi + kTcN * kTcK;
  for (int e = threadIdx.x; e < kTcN * kTcK; e += blockDim.x) {
    const int n = e / kTcK, k = e % kTcK;  // B[k][n]
    const float2 *M = n < 32 ? m1 : m2;
    const int j = (n & 31) >> 1, b = n & 1, kc = k >> 1, a = k & 1;
    const float2 z = M[kc * N + j];
    // (a, b): (re, re) -> Re, (im, re) -> -Im, (re, im) -> Im, (im, im) -> Re
    const float v = (a == b) ? z.x : (a == 1 ? -z.y : z.y);
    const float h = tf32_rna(v);
    const unsigned off = sw128(n, k) / 4;
    hi[off] = h;
    lo[off] = tf32_rna(v - h);
  }
}

__global__ void __launch_bounds__(kTcRows, 4) k_update_tc(const float2 *__restrict__ Q, float2 *__restrict__ P,
                                                       float2 *__restrict__ X, const float *__restrict__ btiles,
                                                       const int *__restrict__ upd, int s_begin, int s_end, long rows,
                                                       long fstride, int *__restrict__ err) {
  // shared: A head/tail (16 KB each), B head/tail (8 KB each), all 1024-aligned
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = smem_raw;
  {  // align to 1024 bytes for the swizzle pattern
    const unsigned a = smem_u32(smem_raw);
    base += (1024 - (a & 1023)) & 1023;
  }
  float *Ah = reinterpret_cast<float *>(base);
  float *Al = Ah + kTcRows * kTcK;
  float *Bh = Al + kTcRows * kTcK;
  float *Bl = Bh + kTcN * kTcK;
  __shared__ __align__(8) unsigned long long mbar;
  __shared__ unsigned tmem_base_sh;
  __shared__ int ok_sh;
  __shared__ int supd[kMaxS];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < s_end; k += blockDim.x) supd[k] = upd[k];
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    ok_sh = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const unsigned tmem = tmem_base_sh;
  const unsigned mbar_addr = smem_u32(&mbar);
  unsigned phase = 0;
  const unsigned sAh = smem_u32(Ah), sAl = smem_u32(Al), sBh = smem_u32(Bh), sBl = smem_u32(Bl);
  for (long tile = blockIdx.x; tile * kTcRows < rows && ok_sh; tile += gridDim.x) {
    const long r = tile * kTcRows + tid;
    const bool live = r < rows;
    float q[kTcK];
    if (live) {
      const float4 *src = reinterpret_cast<const float4 *>(Q + r * 16);
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = src[c];
        q[4 * c] = v.x, q[4 * c + 1] = v.y, q[4 * c + 2] = v.z, q[4 * c + 3] = v.w;
      }
    }
    for (int s = s_begin; s < s_end; ++s) {
      if (!supd[s]) continue;
      float2 *Ps = P + s * fstride;
      // A tile: this thread's row, head and tail, swizzled
      {
        float4 pv[8];
        if (live) {
          const float4 *src = reinterpret_cast<const float4 *>(Ps + r * 16);
#pragma unroll
          for (int c = 0; c < 8; ++c) pv[c] = src[c];
        } else {
#pragma unroll
          for (int c = 0; c < 8; ++c) pv[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4 v = pv[c];
          const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
          const float4 l = make_float4(tf32_rna(v.x - h.x), tf32_rna(v.y - h.y), tf32_rna(v.z - h.z),
                                       tf32_rna(v.w - h.w));
          const unsigned off = sw128(tid, 4 * c);
          *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(Ah) + off) = h;
          *reinterpret_cast<float4 *>(reinterpret_cast<unsigned char *>(Al) + off) = l;
        }
      }
      // B tiles (already in the swizzled layout): 16 KB copied by the CTA
      {
        const float4 *src = reinterpret_cast<const float4 *>(btiles + (size_t)s * 2 * kTcN * kTcK);
        float4 *dst = reinterpret_cast<float4 *>(Bh);
        for (int k = tid; k < 2 * kTcN * kTcK / 4; k += blockDim.x) dst[k] = src[k];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        // K = 32 reals = 4 steps of 8 (32 bytes) inside the 128-byte swizzle atom
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const unsigned off = kk * 32;
          mma_tf32(tmem, make_desc(sAh + off), make_desc(sBh + off), kk > 0);
          mma_tf32(tmem, make_desc(sAh + off), make_desc(sBl + off), 1);
          mma_tf32(tmem, make_desc(sAl + off), make_desc(sBh + off), 1);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_addr)
                     : "memory");
        if (!mbar_wait_for(mbar_addr, phase, kWaitCycles)) {
          ok_sh = 0;
          atomicExch(err, 1);
          // give the MMAs in flight one more bounded chance to land before the
          // tensor memory is released
          mbar_wait_for(mbar_addr, phase, kWaitCycles);
        }
      }
      __syncthreads();
      phase ^= 1;
      if (!ok_sh) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      unsigned d[64];
      RHMC_TMEM_LD64(tmem + ((unsigned)(warp * 32) << 16), d);
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      if (live) {
        float4 *xs = reinterpret_cast<float4 *>(X + s * fstride + r * 16);
        float4 *ps = reinterpret_cast<float4 *>(Ps + r * 16);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          float4 x = xs[c];
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
      __syncthreads();
    }
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcCols));
}

// Shifts [s_begin, s_end) with the tensor cores (mixed path, n = 16).
// btiles: 2 * 64 * 32 floats per shift of scratch; err: device flag.
rhmc_status_t update_shifts_tc(const float2 *Q, float2 *P, float2 *X, const float2 *coef, const int *upd,
                               int s_begin, int s_end, long rows, long fstride, float *btiles, int *err,
                               cudaStream_t s) {
  if (s_end <= s_begin) return RHMC_OK;
  k_tc_prepare_b<<<s_end - s_begin, 256, 0, s>>>(coef, s_begin, s_end, btiles);
  RHMC_LAUNCH_CHECK();
  const size_t smem = 1024 + (size_t)(2 * kTcRows * kTcK + 2 * kTcN * kTcK) * sizeof(float);
  static std::once_flag attr;
  std::call_once(attr, [&] {
    cudaFuncSetAttribute(k_update_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  const long tiles = (rows + kTcRows - 1) / kTcRows;
  const int grid = (int)std::min<long>(tiles, 4 * 152);
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
