// Shared host/device helpers of the GB300 randomized-SVD library.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/rsvd.h"

namespace rsvd {

// ---- host-side error reporting --------------------------------------------

void set_error(const std::string& msg);
rsvd_status fail(rsvd_status st, const std::string& msg);
rsvd_status cuda_fail(cudaError_t e, const char* what);

#define RSVD_CUDA(call)                                              \
  do {                                                               \
    cudaError_t e__ = (call);                                        \
    if (e__ != cudaSuccess) return ::rsvd::cuda_fail(e__, #call);    \
  } while (0)

#define RSVD_TRY(call)                                               \
  do {                                                               \
    rsvd_status s__ = (call);                                        \
    if (s__ != RSVD_OK) return s__;                                  \
  } while (0)

// Every kernel launch site calls after_launch(): it counts the launch (for
// rsvd_kernel_launches) and returns the launch's error state.
cudaError_t after_launch();

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline int64_t round_up(int64_t a, int64_t b) { return cdiv(a, b) * b; }
template <typename T>
__host__ __device__ inline bool aligned16(const T* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// ---- device status word ----------------------------------------------------
// Kernels that can fail write one of these codes (first writer wins through
// atomicCAS) into a device int that the host reads back once per call.
enum DevStatus : int {
  DEV_OK = 0,
  DEV_NOT_SPD = 1,
  DEV_NO_CONVERGE = 2,
  DEV_TIMEOUT = 3,
  DEV_BAD_ARG = 4,
};

__device__ __forceinline__ void dev_set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

rsvd_status status_from_device(int code);

// Copy the device status word to the host (synchronising the stream).
rsvd_status read_device_status(const int* d_status, cudaStream_t stream);

// ---- workspace carving -------------------------------------------------------
// A bump allocator over one caller-provided device buffer; every carve is
// aligned to 256 bytes (enough for TMA's 128-byte and mbarrier rules).
struct Carver {
  char* base;
  size_t cap;
  size_t used = 0;
  bool overflow = false;
  Carver(void* b, size_t c) : base(static_cast<char*>(b)), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    size_t off = (used + 255) & ~size_t(255);
    size_t bytes = count * sizeof(T);
    if (off + bytes > cap) { overflow = true; used = off + bytes; return nullptr; }
    used = off + bytes;
    return reinterpret_cast<T*>(base ? base + off : nullptr);
  }
};

// Size-only counterpart of Carver (base == nullptr never overflows).
struct Sizer {
  size_t used = 0;
  template <typename T>
  void take(size_t count) { used = ((used + 255) & ~size_t(255)) + count * sizeof(T); }
};

// ---- small device helpers -----------------------------------------------------

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Bounded spin limit of every device-side wait (about a second at GB300 clocks
// with the 64 ns back-off used by the waits).
constexpr long long kSpinLimit = 20000000LL;

}  // namespace rsvd
