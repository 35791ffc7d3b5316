// Tensor-core A-passes (placeholder until the tcgen05 kernel lands).
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {

size_t tc_apass_ws_bytes(int64_t, int64_t, int, int, int, int64_t, int64_t) { return 256; }

rsvd_status tc_apass_from_f32(const rsvd_matrix&, int, int, int, const float*, int64_t, float*, int64_t,
                              int64_t, int64_t, void*, size_t, cudaStream_t) {
  return fail(RSVD_ERR_UNSUPPORTED, "tensor-core A-pass not built yet");
}

}  // namespace rsvd
