// Arithmetic peaks of the CUDA cores, measured (the denominators of the FP32
// and FP64 roofline fractions of the double-float hop, the n x n coefficient
// chain and the FP64 per-vector baseline).
//
// Every thread runs kChains independent fused multiply-add chains for `iters`
// rounds, so that the pipes see independent instructions back to back; the
// grid fills every SM with 8 CTAs of 256 threads.  Work counted: 2 flops per
// FMA lane (a packed FP32x2 FMA counts 4).  The chains' results are summed into
// one output word so that nothing is optimised away.
#include "common.cuh"

namespace rhmc {

namespace {
constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads) k_peak_fp32(float *out, int iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (float)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fmaf(a[j], b, c);
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.678f) out[0] = s;  // never true for the probe's inputs; keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_fp32x2(float *out, int iters, float b, float c) {
  unsigned long long a[kChains];
  const unsigned long long bb = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
  const unsigned long long cc = ((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(c);
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    const unsigned v = __float_as_uint((float)(threadIdx.x + j));
    a[j] = ((unsigned long long)v << 32) | v;
  }
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kChains; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[j]) : "l"(bb), "l"(cc));
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += __uint_as_float((unsigned)a[j]) + __uint_as_float((unsigned)(a[j] >> 32));
  if (s == 12345.678f) out[0] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_fp64(float *out, int iters, double b, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = (double)(threadIdx.x + j);
  for (int it = 0; it < iters; ++it)
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], b, c);
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  if (s == 12345.678) out[0] = (float)s;
}

// Best of `reps` launches, in TFLOP/s.
template <typename K, typename S>
static rhmc_status_t time_peak(K kern, S b, S c, int iters, int lanes_per_fma, int reps, cudaStream_t s,
                               float *out, double *tflops) {
  int nsm = 0, dev = 0;
  RHMC_CUDA_TRY(cudaGetDevice(&dev));
  RHMC_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = 8 * nsm;
  cudaEvent_t e0, e1;
  RHMC_CUDA_TRY(cudaEventCreate(&e0));
  RHMC_CUDA_TRY(cudaEventCreate(&e1));
  double best = 0.0;
  rhmc_status_t rc = RHMC_OK;
  for (int r = 0; r <= reps && rc == RHMC_OK; ++r) {
    cudaEventRecord(e0, s);
    kern<<<grid, kPeakThreads, 0, s>>>(out, iters, b, c);
    cudaEventRecord(e1, s);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      set_error("peak probe launch failed");
      rc = RHMC_ERR_CUDA;
      break;
    }
    count_launch();
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * lanes_per_fma * kChains * (double)iters * grid * kPeakThreads;
    if (r > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);  // launch 0 warms up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *tflops = best;
  return rc;
}
}  // namespace

}  // namespace rhmc

extern "C" rhmc_status_t rhmc_probe_alu_peaks(int device, double *fp32_tflops, double *fp32x2_tflops,
                                              double *fp64_tflops, rhmc_stream_t sv) {
  using namespace rhmc;
  if (!fp32_tflops || !fp32x2_tflops || !fp64_tflops) {
    set_error("rhmc_probe_alu_peaks: null output");
    return RHMC_ERR_INVALID_ARG;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) RHMC_CUDA_TRY(cudaSetDevice(device));
  cudaStream_t s = (cudaStream_t)sv;
  float *out = nullptr;
  rhmc_status_t rc = RHMC_OK;
  if (cudaMalloc(&out, sizeof(float)) != cudaSuccess) {
    set_error("rhmc_probe_alu_peaks: cudaMalloc failed");
    rc = RHMC_ERR_CUDA;
  }
  // a few milliseconds per launch at the expected rates
  if (rc == RHMC_OK) rc = time_peak(k_peak_fp32, 1.0000001f, 1e-7f, 1 << 16, 1, 5, s, out, fp32_tflops);
  if (rc == RHMC_OK) rc = time_peak(k_peak_fp32x2, 1.0000001f, 1e-7f, 1 << 15, 2, 5, s, out, fp32x2_tflops);
  if (rc == RHMC_OK) rc = time_peak(k_peak_fp64, 1.0000000001, 1e-12, 1 << 11, 1, 5, s, out, fp64_tflops);
  if (out) cudaFree(out);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
