// rsvd_small_svd_noalloc: the one-sided Jacobi SVD of rsvd_small_svd, for
// callers that cannot allocate device memory (their device memory is owned by
// a pool that has reserved it all, or they must not let cudaMalloc/cudaFree
// synchronise the device) and so cannot supply the workspace that
// rsvd_small_svd takes.
//
// The scratch lives in one file-scope device array sized for the largest
// supported r (RSVD_NOALLOC_MAX_R).  Every GPU that loads this library holds
// that array until the process exits.  Host code cannot use the array's name
// as a device address, so the address is looked up once per device with
// cudaGetSymbolAddress while that device is current, and passed to the kernel.
// All calls share the array and it keeps the previous call's contents; the
// words that must start at zero are cleared on every call.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int kMaxR = RSVD_NOALLOC_MAX_R;
// The same workspace as rsvd_small_svd at r = kMaxR, so that both entry points
// run the same phases: M and W (kMaxR^2 doubles each), the FP32 rotations
// (kMaxR^2 floats), the FP64 rotations, Newton-Schulz and product buffers
// (4 kMaxR^2 doubles), the split-K partials of the small GEMMs (32 kMaxR^2
// doubles), and the barrier, per-sweep flags, sweep count and status words;
// each carve rounded to 256 bytes.
constexpr size_t kScratchBytes =
    (2 + 4 + 32) * (size_t)kMaxR * kMaxR * sizeof(double) + (size_t)kMaxR * kMaxR * sizeof(float) + 8192;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up on the
// first call made on that device).
rsvd_status scratch_address(void** out) {
  int dev = 0;
  RSVD_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(RSVD_ERR_UNSUPPORTED, "rsvd_small_svd_noalloc: device index too large");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "rsvd_small_svd_noalloc: cudaGetSymbolAddress(scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return RSVD_OK;
}

}  // namespace
}  // namespace rsvd

extern "C" rsvd_status rsvd_small_svd_noalloc(int32_t r, const double* Mc, double* sigma, double* U, double* W,
                                              void* stream) {
  using namespace rsvd;
  if (r < 1 || !Mc || !sigma || !U || !W) return fail(RSVD_ERR_INVALID_ARG, "rsvd_small_svd_noalloc: bad arguments");
  if (r > kMaxR)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_small_svd_noalloc: r = " + std::to_string(r) +
                                          " exceeds the static scratch limit RSVD_NOALLOC_MAX_R = " +
                                          std::to_string(kMaxR));
  void* base = nullptr;
  RSVD_TRY(scratch_address(&base));
  Carver c(base, kScratchBytes);
  JacobiWs w = jacobi_ws_carve(c, r, r);
  if (c.overflow) return fail(RSVD_ERR_INVALID_ARG, "rsvd_small_svd_noalloc: scratch layout overflow");
  cudaStream_t st = as_stream(stream);
  // the status word must start at zero; jacobi_svd clears the barrier and flags
  RSVD_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), st));
  RSVD_TRY(jacobi_svd(r, r, Mc, sigma, U, W, w, st));
  return read_device_status(w.status, st);
}
