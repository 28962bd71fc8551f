// Allocation-free variant of the FP64 operator application.
//
// rhmc_apply_mdagm_mrhs may grow the context's scratch pool with cudaMalloc
// on its first use.  Some callers cannot allow that: code running while a
// CUDA graph is being captured, real-time or embedded hosts whose memory
// budget is fixed at start-up, or frameworks that forbid allocation outside
// their own allocator.  rhmc_apply_mdagm_mrhs_noalloc gives them the same
// result with no allocation at all: the odd-parity intermediate D_oe X lives
// in a file-scope device array of fixed size, kNoAllocScratchBytes, which every
// GPU that loads this library holds until the process exits.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rhmc {

// 32 MiB: room for the intermediate of V/2 * 3 * n_rhs complex128 values,
// e.g. a 16^4 lattice with 16 right-hand sides (25.2 MB).
constexpr size_t kNoAllocScratchBytes = 32u << 20;
static __device__ __align__(256) double2 g_noalloc_scratch[kNoAllocScratchBytes / sizeof(double2)];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Device address of g_noalloc_scratch, per device, looked up on the first call.
// The address belongs to the device's primary context: it stays valid as long
// as that context lives, so a process that resets a device (cudaDeviceReset)
// must not call this entry point on that device afterwards.
double2 *g_scratch_ptr[kMaxDevices] = {};
}  // namespace

}  // namespace rhmc

extern "C" rhmc_status_t rhmc_apply_mdagm_mrhs_noalloc(rhmc_ctx_t *ctx, const void *X_dev, void *Y_dev, int n_rhs,
                                                       double sigma, rhmc_stream_t sv) {
  using namespace rhmc;
  if (!ctx || !X_dev || !Y_dev || X_dev == Y_dev) {
    set_error("rhmc_apply_mdagm_mrhs_noalloc: null or aliased argument");
    return RHMC_ERR_INVALID_ARG;
  }
  if (n_rhs < 1 || n_rhs > RHMC_MAX_NRHS) {
    set_error("rhmc_apply_mdagm_mrhs_noalloc: n_rhs = %d out of range [1, %d]", n_rhs, RHMC_MAX_NRHS);
    return RHMC_ERR_INVALID_ARG;
  }
  int device = 0;
  Geom g;
  double mass = 0.0;
  const double2 *le = nullptr, *lo = nullptr;
  rhmc_status_t rc = ctx_geometry(ctx, &device, &g, &mass, &le, &lo);
  if (rc != RHMC_OK) return rc;
  const size_t need = (size_t)g.Vh * 3 * n_rhs * sizeof(double2);
  if (need > kNoAllocScratchBytes) {
    set_error("rhmc_apply_mdagm_mrhs_noalloc: needs %zu bytes of scratch (V/2 * 3 * n_rhs complex128), "
              "more than its fixed %zu; use rhmc_apply_mdagm_mrhs",
              need, kNoAllocScratchBytes);
    return RHMC_ERR_INVALID_ARG;
  }
  if (device < 0 || device >= kMaxDevices) {
    set_error("rhmc_apply_mdagm_mrhs_noalloc: device %d out of range", device);
    return RHMC_ERR_INVALID_ARG;
  }
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != device) RHMC_CUDA_TRY(cudaSetDevice(device));
  double2 *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[device]) {
      // once per device, with that device current: the symbol's device address
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_error("rhmc_apply_mdagm_mrhs_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        if (prev >= 0 && prev != device) cudaSetDevice(prev);
        return RHMC_ERR_CUDA;
      }
      g_scratch_ptr[device] = static_cast<double2 *>(p);
    }
    scratch = g_scratch_ptr[device];
  }
  cudaStream_t s = (cudaStream_t)sv;
  CtxTuneScope tscope(ctx);  // the context's launch settings, as in rhmc_apply_mdagm_mrhs
  // the intermediate is fully overwritten by the first hop: nothing to clear
  rc = hop<double>(g, 1, lo, (const double2 *)X_dev, scratch, nullptr, 0.0, n_rhs, 1, 0, s);
  if (rc == RHMC_OK)
    rc = hop<double>(g, 0, le, scratch, (double2 *)Y_dev, (const double2 *)X_dev, 4.0 * mass * mass + sigma, n_rhs, 1,
                     0, s);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  return rc;
}
