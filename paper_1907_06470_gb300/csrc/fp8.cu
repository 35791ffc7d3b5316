// FP8 (E4M3) storage of A with one power-of-two scale per tile, for the FP8
// variant of the A-passes (the precision choices of Section 3.2 taken below
// half precision; the products of Section 2.1 steps 2 and 5 and Eq. (3)).
//
// Tiles are the block-cyclic tiles of Section 3.1 (rows [I*qm, ...) x columns
// [J*qn, ...), qm and qn multiples of 128 or covering the whole dimension).
// For a tile with largest magnitude amax the scale s is the smallest power of
// two with amax / s <= 448 (the largest finite E4M3 value), and each entry is
// stored as the E4M3 code of x / s, rounded to nearest even with saturation.
// The tensor-core pass decodes the codes to BF16 (exact: E4M3 values have four
// significant bits) times s (exact: a power of two), so the only rounding of
// the FP8 path is the quantisation itself.
//
// Two passes over A: the per-tile maxima (one atomicMax per 128 x 128 block,
// order independent), then the codes.
#include <cuda_fp8.h>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int kQB = 128;  // block edge of the two kernels (tiles are multiples of it)

// One CTA (8 warps) per 128 x 128 block of A: warp w reads rows w, w+8, ...,
// lane l columns 4l..4l+3 (float4 when aligned).
__global__ void __launch_bounds__(256)
fp8_amax_kernel(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda, int64_t qm, int64_t qn, int64_t qtn,
                unsigned* __restrict__ amax_bits) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kQB, r0 = (int64_t)blockIdx.y * kQB;
  const bool vec = (lda % 4 == 0) && aligned16(A) && c0 + kQB <= n;
  float mx = 0.f;
  for (int64_t i = r0 + warp; i < min(m, r0 + kQB); i += 8) {
    const float* row = A + i * lda + c0;
    if (vec) {
      const float4 v = reinterpret_cast<const float4*>(row)[lane];
      mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    } else {
      for (int t = 0; t < 4; ++t) {
        const int64_t c = c0 + 4 * lane + t;
        if (c < n) mx = fmaxf(mx, fabsf(row[4 * lane + t]));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float red[8];
  if (lane == 0) red[warp] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = red[0];
    for (int w = 1; w < 8; ++w) b = fmaxf(b, red[w]);
    // non-negative floats order like their bit patterns
    atomicMax(&amax_bits[(r0 / qm) * qtn + (c0 / qn)], __float_as_uint(b));
  }
}

// scale = smallest power of two s with amax / s <= 448 (1 for an all-zero tile)
__global__ void fp8_scale_kernel(int64_t tiles, const unsigned* __restrict__ amax_bits, float* __restrict__ scales) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x) {
    const float amax = __uint_as_float(amax_bits[t]);
    float s = 1.f;
    if (amax > 0.f && isfinite(amax)) {
      int e = 0;
      const float f = frexpf(amax, &e);  // amax = f 2^e, f in [0.5, 1); 448 = 0.875 2^9
      s = ldexpf(1.f, e - 9 + (f > 0.875f ? 1 : 0));
    } else if (!(amax >= 0.f) || !isfinite(amax)) {
      s = __uint_as_float(0x7fc00000u);  // NaN or infinity in the tile: propagate
    }
    scales[t] = s;
  }
}

__global__ void __launch_bounds__(256)
fp8_quantize_kernel(int64_t m, int64_t n, const float* __restrict__ A, int64_t lda, int64_t qm, int64_t qn,
                    int64_t qtn, const float* __restrict__ scales, uint8_t* __restrict__ codes, int64_t ldc) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t c0 = (int64_t)blockIdx.x * kQB, r0 = (int64_t)blockIdx.y * kQB;
  const float s = scales[(r0 / qm) * qtn + (c0 / qn)];
  const float inv = 1.f / s;  // a power of two: exact, and x * inv is exact
  const bool vec = (lda % 4 == 0) && aligned16(A) && c0 + kQB <= n;
  for (int64_t i = r0 + warp; i < min(m, r0 + kQB); i += 8) {
    const float* row = A + i * lda + c0;
    uint8_t* out = codes + i * ldc + c0;
    float v[4];
    if (vec) {
      const float4 x = reinterpret_cast<const float4*>(row)[lane];
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
      for (int t = 0; t < 4; ++t) v[t] = c0 + 4 * lane + t < n ? row[4 * lane + t] : 0.f;
    }
    const __nv_fp8x2_storage_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[0] * inv, v[1] * inv), __NV_SATFINITE, __NV_E4M3);
    const __nv_fp8x2_storage_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[2] * inv, v[3] * inv), __NV_SATFINITE, __NV_E4M3);
    if (vec) {
      reinterpret_cast<uint32_t*>(out)[lane] = (uint32_t)lo | ((uint32_t)hi << 16);
    } else {
      const uint8_t b[4] = {(uint8_t)(lo & 0xff), (uint8_t)(lo >> 8), (uint8_t)(hi & 0xff), (uint8_t)(hi >> 8)};
      for (int t = 0; t < 4; ++t)
        if (c0 + 4 * lane + t < n) out[4 * lane + t] = b[t];
    }
  }
}

}  // namespace

bool fp8_tiles_ok(int64_t m, int64_t n, int64_t qm, int64_t qn) {
  return qm > 0 && qn > 0 && (qm % kQB == 0 || qm >= m) && (qn % kQB == 0 || qn >= n);
}

size_t fp8_amax_ws_bytes(int64_t m, int64_t n, int64_t qm, int64_t qn) {
  return (size_t)cdiv(m, qm) * cdiv(n, qn) * sizeof(unsigned) + 256;
}

rsvd_status fp8_quantize(const float* A, int64_t m, int64_t n, int64_t lda, int64_t qm, int64_t qn, uint8_t* codes,
                         int64_t ldc, float* scales, unsigned* amax_ws, cudaStream_t stream) {
  if (m <= 0 || n <= 0) return RSVD_OK;
  if (!fp8_tiles_ok(m, n, qm, qn))
    return fail(RSVD_ERR_INVALID_ARG, "fp8 quantize: tile edges must be multiples of 128 (or cover the matrix)");
  if (ldc < n || (ldc % 4) != 0 || (reinterpret_cast<uintptr_t>(codes) & 3) != 0)
    return fail(RSVD_ERR_INVALID_ARG, "fp8 quantize: codes need ld >= n, ld % 4 == 0 and a 4-byte aligned base");
  if (qm > m) qm = m;
  if (qn > n) qn = n;
  const int64_t qtm = cdiv(m, qm), qtn = cdiv(n, qn);
  RSVD_CUDA(cudaMemsetAsync(amax_ws, 0, (size_t)qtm * qtn * sizeof(unsigned), stream));
  const dim3 grid((unsigned)cdiv(n, kQB), (unsigned)cdiv(m, kQB));
  if (grid.y > 65535) return fail(RSVD_ERR_INVALID_ARG, "fp8 quantize: too many rows");
  fp8_amax_kernel<<<grid, 256, 0, stream>>>(m, n, A, lda, qm, qn, qtn, amax_ws);
  RSVD_CUDA(after_launch());
  fp8_scale_kernel<<<(int)cdiv(qtm * qtn, 256), 256, 0, stream>>>(qtm * qtn, amax_ws, scales);
  RSVD_CUDA(after_launch());
  fp8_quantize_kernel<<<grid, 256, 0, stream>>>(m, n, A, lda, qm, qn, qtn, scales, codes, ldc);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

}  // namespace rsvd
