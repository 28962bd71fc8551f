// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "../../include/rhmc.h"

namespace rhmc {

// ------------------------------------------------------------ complex types
template <typename T> struct cplx;
template <> struct cplx<float> { using t = float2; };
template <> struct cplx<double> { using t = double2; };
template <typename T> using C = typename cplx<T>::t;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T re, T im) {
  C<T> z;
  z.x = re;
  z.y = im;
  return z;
}
template <typename T> __host__ __device__ __forceinline__ C<T> czero() { return mk<T>(T(0), T(0)); }
// acc += a * b
template <typename T> __device__ __forceinline__ void cmac(C<T> &acc, C<T> a, C<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
template <typename T> __device__ __forceinline__ void cmac_cj(C<T> &acc, C<T> a, C<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}
// acc += a * conj(b)
template <typename T> __device__ __forceinline__ void cmac_bcj(C<T> &acc, C<T> a, C<T> b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.y, b.x, acc.y);
  acc.y = fma(-a.x, b.y, acc.y);
}

// ------------------------------------------------------------ lattice geometry
struct Geom {
  int L[4];
  int Lxh;   // Lx / 2
  long V, Vh;
};

// Coordinates of the site with parity `par` and parity rank h.  Because Lx is
// even, lex = 2h or 2h+1; the parity fixes which.
__device__ __forceinline__ void site_coords(const Geom &g, int par, long h, int x[4]) {
  long r = h / g.Lxh;  // (y, z, t) row index
  const int xh = (int)(h - r * g.Lxh);
  x[1] = (int)(r % g.L[1]);
  r /= g.L[1];
  x[2] = (int)(r % g.L[2]);
  x[3] = (int)(r / g.L[2]);
  const int rowpar = (x[1] + x[2] + x[3]) & 1;
  x[0] = 2 * xh + (rowpar ^ par);
}

__device__ __forceinline__ long lex_of(const Geom &g, const int x[4]) {
  return x[0] + (long)g.L[0] * (x[1] + (long)g.L[1] * (x[2] + (long)g.L[2] * x[3]));
}

// Parity rank of the neighbour of x in direction mu (dir = +1 / -1).
__device__ __forceinline__ long nb_rank(const Geom &g, const int x[4], int mu, int dir) {
  // the shifted coordinate is selected without dynamic indexing (no local memory)
  int y[4];
#pragma unroll
  for (int nu = 0; nu < 4; ++nu) {
    int v = x[nu];
    if (nu == mu) {
      v += dir;
      if (v < 0) v += g.L[nu];
      if (v >= g.L[nu]) v -= g.L[nu];
    }
    y[nu] = v;
  }
  return lex_of(g, y) >> 1;
}

// ------------------------------------------------------------ status handling
void set_error(const char *fmt, ...);
void count_launch();

// Optional per-kernel timing (rhmc_profile_enable): events recorded on the
// launching stream around each launch of a category, with the launch's
// algorithmic bytes.  No-ops when profiling is off.
enum ProfCat {
  PROF_HOP32 = 0, PROF_HOP64, PROF_GRAM32, PROF_GRAM64, PROF_AXPY, PROF_UPDATE32, PROF_UPDATE64,
  PROF_NXN, PROF_FORCE, PROF_OTHER, PROF_HOP_DF, PROF_NXN_SHIFTS, PROF_UPDATE_TC, PROF_UPDATE_SHIFTS32,
  PROF_BASIS_TC, PROF_NCAT
};
bool prof_on();

// Tunable launch parameters (rhmc_tune_set); 0 = built-in choice.
enum TuneKey {
  TUNE_HOP_RHS_PER_THREAD = 0,
  TUNE_UPDATE_THREADS,
  TUNE_FLUSH_EVERY,          // mixed: also flush FP32 increments every k iterations (0: at reliable updates only)
  TUNE_RELIABLE_DELTA_MILLI, // mixed: reliable update when the base residual fell by this / 1000 (0: 100)
  TUNE_CHECK_EVERY,          // iterations between host convergence checks (0: 8)
  TUNE_NATIVE_FP64_RESIDUALS, // mixed: native FP64 instead of double-float for residuals (0: double-float)
  TUNE_UPDATE_TENSOR,         // mixed, n = 16: shifted updates on tcgen05 (1) or CUDA cores (2); 0: built-in
  TUNE_GRAPHS,                // solver chunks as captured CUDA graphs (0/1) or eager launches (2)
  TUNE_HOP_STAGED,            // FP32 hop with cp.async-staged tiles: built-in (0), always (1), never (2)
  TUNE_REFINE_LANES,          // concurrent per-shift defect corrections (0: built-in 4)
  TUNE_LINKS12,               // FP32 hop reads 12-real links when all links are SU(3) (1); full records (0, 2)
  TUNE_SHIFT_FREEZE_NANO,     // mixed: freeze shifted systems below this recursive residual (x 1e-9; 0: built-in)
  TUNE_AXPY_SCALAR,           // mixed: scalar FP32 FMAs in the Y = C + A M kernels (1); packed FP32x2 (0)
  TUNE_NO_DEFECT_CORRECTION,  // 1: report the true residuals after the multishift phase, no corrections
  TUNE_BASIS_ITERS,           // mixed: stored-basis capacity in iterations (0: built-in, 1: off)
  TUNE_BASIS_GEMM,            // stored-basis assembly: FP32-accurate tcgen05 kernel (0) or CUDA-core kernel (1)
  TUNE_BASIS_CHUNK,           // stored-basis assembly: blocks per FP32 partial sum (0: one GEMM)
  TUNE_BASIS_ACC_KT,          // stored-basis assembly: K tiles per tensor-memory accumulation chunk (0: built-in)
  TUNE_NXN_FP64,              // mixed: base n x n steps in native FP64 (1) instead of double-float (0)
  TUNE_BASE_TILE,             // fused base step at n = 16: 0 = 8 rows x 16 warps, 1 = 16 x 12, 2 = 16 x 8, 3 = 8 x 12
  TUNE_GRAM_TILE,             // packed Gram at n = 16: 0 = 16 rows x 4 warps, 1 = 32 x 8, 2 = 16 x 8, 3 = 8 x 8
  TUNE_AXPY_ROWS,             // fused axpy + Gram at n = 16: 0 = 8-row tiles, 1 = 16-row tiles
  TUNE_CORRECTION_MARGIN_MILLI,  // defect corrections stop at this / 1000 x tol / r (0: built-in)
  TUNE_PHASE1_MARGIN_MILLI,   // the multishift phase runs to this / 1000 x tol (0: built-in)
  TUNE_CORRECTION_CHECK_EVERY,  // iterations between host checks of a defect correction (0: built-in 1)
  TUNE_NKEYS
};
int tune_get(int key);
void prof_begin(int cat, cudaStream_t s);
void prof_end(cudaStream_t s, double bytes);
void prof_flops(double flops);  // tensor-core flops of the launch just recorded

#define RHMC_CUDA_TRY(call)                                                                    \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      ::rhmc::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_));   \
      return RHMC_ERR_CUDA;                                                                    \
    }                                                                                          \
  } while (0)

#define RHMC_TRY(...)                   \
  do {                                  \
    rhmc_status_t st_ = (__VA_ARGS__);  \
    if (st_ != RHMC_OK) return st_;     \
  } while (0)

#define RHMC_LAUNCH_CHECK()                                                                    \
  do {                                                                                         \
    ::rhmc::count_launch();                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                       \
    if (e_ != cudaSuccess) {                                                                   \
      ::rhmc::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
      return RHMC_ERR_CUDA;                                                                    \
    }                                                                                          \
  } while (0)

// CTAs of kernel f resident on the whole GPU at once (cached per kernel and size).
template <typename F> static int resident_ctas(F f, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void *, int, size_t, int>, int> cache;
  int per_sm = 0, nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_tuple(reinterpret_cast<const void *>(f), threads, smem, dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  const int v = per_sm * std::max(nsm, 1);
  cache[key] = v;
  return v;
}

}  // namespace rhmc
