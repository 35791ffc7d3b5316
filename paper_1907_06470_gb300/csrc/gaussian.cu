// Section 2.1 step 1: the n x r Gaussian test matrix O, entries i.i.d. N(0,1).
//
// Counter-based: entry (i, j) is element e = i*r + j of one stream, so every
// thread computes its entries independently of the launch shape.  Philox4x32-10
// (Salmon, Moraes, Dror, Shaw, SC'11) gives 128 random bits per pair of
// elements (2g, 2g+1); Box-Muller turns them into two normal deviates.  ln,
// sin and cos are evaluated from their atanh / Taylor series with separately
// rounded FP64 operations (__dmul_rn / __dadd_rn / __ddiv_rn never contract
// into FMAs), and the angle is reduced to [-pi/4, pi/4] exactly in integer
// arithmetic, so the values are reproducible bit for bit by any IEEE FP64
// implementation that follows the same operation order.
//
// bfloat16 outputs need each deviate only to its nearest bfloat16 (8
// significant bits), and FP64 arithmetic is slow on this GPU, so they are first
// evaluated in FP32 from the same random bits (bf16_pair_fp32); the FP64
// evaluation decides only the deviates whose FP32 value lies too close to a
// bfloat16 rounding boundary (about one in 1500).  The result is the rounding
// of the FP64 value either way.
#include "common.cuh"
#include "kernels.cuh"

#include <cuda_bf16.h>

namespace rsvd {
namespace {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) { k0 += kPhiloxW0; k1 += kPhiloxW1; }
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c[0];
    const uint64_t p1 = (uint64_t)kPhiloxM1 * c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    const uint32_t n0 = hi1 ^ c[1] ^ k0;
    const uint32_t n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// ln 2 as a 32-significant-bit head (E*head exact for |E| < 2^21) + FP64 tail.
__device__ __forceinline__ double ln2_hi() { return __longlong_as_double(0x3FE62E42FEE00000LL); }
__device__ __forceinline__ double ln2_lo() { return __longlong_as_double(0x3DEA39EF35793C76LL); }
__device__ __forceinline__ double sqrt2_rounded() { return __longlong_as_double(0x3FF6A09E667F3BCDLL); }
__device__ __forceinline__ double pi_times_2m53() {
  // fl(pi) = 0x400921FB54442D18; scaling by 2^-53 only changes the exponent.
  return __longlong_as_double(0x400921FB54442D18LL) * 0x1.0p-53;
}

// Horner evaluation c[0] + z*(c[1] + z*(...)), multiply and add rounded separately.
template <int N>
__device__ __forceinline__ double horner(const double (&c)[N], double z) {
  double acc = c[N - 1];
#pragma unroll
  for (int i = N - 2; i >= 0; --i) acc = __dadd_rn(c[i], __dmul_rn(z, acc));
  return acc;
}

// ln u for normal u > 0:  u = f 2^E, f in [sqrt2/2, sqrt2], s = (f-1)/(f+1),
// ln f = 2 atanh(s) = h + h*(z*P(z)), h = 2s, z = s^2, P = sum z^k/(2k+3).
__device__ double ln_series(double u) {
  const double kAtanh[10] = {1.0 / 3.0,  1.0 / 5.0,  1.0 / 7.0,  1.0 / 9.0,  1.0 / 11.0,
                             1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0, 1.0 / 21.0};
  const unsigned long long bits = (unsigned long long)__double_as_longlong(u);
  long long E = (long long)((bits >> 52) & 0x7FF) - 1023;
  double f = __longlong_as_double((long long)((bits & 0x000FFFFFFFFFFFFFULL) | 0x3FF0000000000000ULL));
  if (f > sqrt2_rounded()) { f = __dmul_rn(f, 0.5); E += 1; }
  const double s = __ddiv_rn(__dadd_rn(f, -1.0), __dadd_rn(f, 1.0));
  const double z = __dmul_rn(s, s);
  const double P = horner(kAtanh, z);
  const double h = __dmul_rn(2.0, s);
  const double t1 = __dmul_rn(z, P);
  const double t2 = __dmul_rn(h, t1);
  const double lnf = __dadd_rn(h, t2);
  const double Ef = (double)E;
  const double t3 = __dmul_rn(Ef, ln2_lo());
  const double t4 = __dadd_rn(t3, lnf);
  const double t5 = __dmul_rn(Ef, ln2_hi());
  return __dadd_rn(t5, t4);
}

// sin / cos on [-pi/4, pi/4] from their Taylor series (coefficients 1/k!).
__device__ __forceinline__ void sincos_reduced(double phi, double* s, double* c) {
  const double kSin[9] = {-1.0 / 6.0,
                          1.0 / 120.0,
                          -1.0 / 5040.0,
                          1.0 / 362880.0,
                          -1.0 / 39916800.0,
                          1.0 / 6227020800.0,
                          -1.0 / 1307674368000.0,
                          1.0 / 355687428096000.0,
                          -1.0 / 121645100408832000.0};
  const double kCos[9] = {-1.0 / 2.0,
                          1.0 / 24.0,
                          -1.0 / 720.0,
                          1.0 / 40320.0,
                          -1.0 / 3628800.0,
                          1.0 / 479001600.0,
                          -1.0 / 87178291200.0,
                          1.0 / 20922789888000.0,
                          -1.0 / 6402373705728000.0};
  const double z = __dmul_rn(phi, phi);
  const double S = horner(kSin, z);
  *s = __dadd_rn(phi, __dmul_rn(phi, __dmul_rn(z, S)));
  const double C = horner(kCos, z);
  *c = __dadd_rn(1.0, __dmul_rn(z, C));
}

// Round an FP64 value once to bfloat16 (nearest-even) on its bit pattern.
__device__ __forceinline__ uint16_t f64_to_bf16_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long sign = b >> 63;
  const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFULL;
  if (mag == 0) return (uint16_t)(sign << 15);
  const unsigned long long lsb = (mag >> 45) & 1ULL;
  const unsigned long long rnd = (mag + ((1ULL << 44) - 1) + lsb) >> 45;  // 11 exp + 7 mantissa bits
  const long long e64 = (long long)(rnd >> 7);
  const unsigned mant = (unsigned)(rnd & 0x7F);
  const long long e16 = e64 - 1023 + 127;  // Gaussian values stay inside the normal range
  return (uint16_t)((sign << 15) | ((unsigned long long)e16 << 7) | mant);
}

template <int kDtype>
__device__ __forceinline__ void store_value(void* out, int64_t idx, double v) {
  if constexpr (kDtype == RSVD_F64) {
    static_cast<double*>(out)[idx] = v;
  } else if constexpr (kDtype == RSVD_F32) {
    static_cast<float*>(out)[idx] = __double2float_rn(v);
  } else if constexpr (kDtype == kF32HoldingBf16) {
    // rounded once to bfloat16, stored exactly in an FP32 container
    static_cast<uint32_t*>(out)[idx] = (uint32_t)f64_to_bf16_bits(v) << 16;
  } else {
    static_cast<uint16_t*>(out)[idx] = f64_to_bf16_bits(v);
  }
}

// FP64 Box-Muller values of the 128 Philox bits c.
__device__ __forceinline__ void box_muller_f64(const uint32_t c[4], double* even, double* odd) {
  const uint64_t n1 = (((uint64_t)c[0] << 32) | c[1]) >> 11;
  const uint64_t n2 = (((uint64_t)c[2] << 32) | c[3]) >> 11;
  const double u1 = (double)(n1 + 1) * 0x1.0p-53;  // exact, in (0, 1]
  const double L = ln_series(u1);
  const double rho = __dsqrt_rn(__dmul_rn(-2.0, L));
  // theta = 2 pi t 2^-54, t = 2 n2 + 1; quadrant q = round(t / 2^52)
  const uint64_t t = 2 * n2 + 1;
  const uint64_t q = (t + (1ULL << 51)) >> 52;
  const int64_t d = (int64_t)t - (int64_t)(q << 52);
  const double phi = __dmul_rn((double)d, pi_times_2m53());
  double s, co;
  sincos_reduced(phi, &s, &co);
  double sin_t, cos_t;
  switch (q & 3) {
    case 0: sin_t = s; cos_t = co; break;
    case 1: sin_t = co; cos_t = -s; break;
    case 2: sin_t = -s; cos_t = -co; break;
    default: sin_t = -co; cos_t = s; break;
  }
  *even = __dmul_rn(rho, cos_t);
  *odd = __dmul_rn(rho, sin_t);
}

// FP64 values of stream elements 2g and 2g+1.
__device__ __forceinline__ void gaussian_pair(uint64_t seed, uint64_t g, double* even, double* odd) {
  uint32_t c[4] = {(uint32_t)g, (uint32_t)(g >> 32), 0u, 0u};
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  box_muller_f64(c, even, odd);
}

// bfloat16 bits of the nearest-even rounding shared by every real within a
// relative 2^-19 of v (v a nonzero normal FP32 value), or -1 when the band
// straddles a rounding boundary.  The band's ends are widened by 2^-22 for
// their own rounding, so they enclose the band; rounding is monotone, so equal
// roundings of the ends decide every value in it.
__device__ __forceinline__ int bf16_if_determined(float v) {
  const float a = fabsf(v);
  const uint32_t bl = __float_as_uint(a * (1.f - 0x1.2p-19f));
  const uint32_t bh = __float_as_uint(a * (1.f + 0x1.2p-19f));
  const uint32_t rl = (bl + 0x7FFFu + ((bl >> 16) & 1u)) >> 16;
  const uint32_t rh = (bh + 0x7FFFu + ((bh >> 16) & 1u)) >> 16;
  if (rl != rh) return -1;
  return (int)(rl | (v < 0.f ? 0x8000u : 0u));
}

// The bfloat16 roundings of the two FP64 deviates of the Philox bits c, from an
// FP32 evaluation of the same Box-Muller formula, when the error bound decides
// them; false otherwise.  Error of the FP32 values relative to the exact
// deviates (CUDA's documented bounds: logf, log1pf, sinpif, cospif 1 ulp,
// sqrtf correctly rounded; conversions of the integers 2^-24):
//   ln u1: u1 <= 1/2 from logf of u1 rounded (|ln u1| >= ln 2), u1 > 1/2 from
//          log1pf of 1 - u1 = m 2^-53 (m exact) rounded: at most 2^-22;
//   rho = sqrt(-2 ln u1): half that plus 2^-24; sin and cos of pi y with
//   y = d 2^-53 in [-1/4, 1/4] (the quadrant reduction is exact): 1.56 2^-23;
//   the final product 2^-24 --
// about 3.6 2^-23 = 2^-21.2 in all, within the 2^-19 band (the FP64 deviates
// differ from the exact ones by a few 2^-53).  t = 2 n2 + 1 is odd and q 2^52
// even, so d != 0: no deviate is zero, all are normal FP32 values.
__device__ __forceinline__ bool bf16_pair_fp32(const uint32_t c[4], uint16_t* even, uint16_t* odd) {
  const uint64_t n1 = (((uint64_t)c[0] << 32) | c[1]) >> 11;
  const uint64_t n2 = (((uint64_t)c[2] << 32) | c[3]) >> 11;
  float L;
  if (n1 + 1 <= (1ULL << 52)) {
    L = logf(__ull2float_rn(n1 + 1) * 0x1.0p-53f);
  } else {
    const uint64_t mm = (1ULL << 53) - (n1 + 1);  // 1 - u1 = mm 2^-53
    if (mm == 0) return false;                    // u1 = 1: deviates of zero, left to FP64
    L = log1pf(-(__ull2float_rn(mm) * 0x1.0p-53f));
  }
  const float rho = sqrtf(-2.f * L);
  const uint64_t t = 2 * n2 + 1;
  const uint64_t q = (t + (1ULL << 51)) >> 52;
  const int64_t d = (int64_t)t - (int64_t)(q << 52);
  const float y = __ll2float_rn(d) * 0x1.0p-53f;
  const float s = sinpif(y), co = cospif(y);
  float sin_t, cos_t;
  switch (q & 3) {
    case 0: sin_t = s; cos_t = co; break;
    case 1: sin_t = co; cos_t = -s; break;
    case 2: sin_t = -s; cos_t = -co; break;
    default: sin_t = -co; cos_t = s; break;
  }
  const int be = bf16_if_determined(rho * cos_t);
  const int bo = bf16_if_determined(rho * sin_t);
  if (be < 0 || bo < 0) return false;
  *even = (uint16_t)be;
  *odd = (uint16_t)bo;
  return true;
}

template <int kDtype>
__global__ void __launch_bounds__(256) gaussian_kernel(uint64_t seed, int64_t n, int64_t r,
                                                       int layout, void* out, int64_t ld) {
  const int64_t total = n * r;
  const int64_t pairs = (total + 1) / 2;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < pairs;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint32_t c[4] = {(uint32_t)g, (uint32_t)((uint64_t)g >> 32), 0u, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    if constexpr (kDtype == RSVD_BF16 || kDtype == kF32HoldingBf16) {
      uint16_t b2[2];
      if (!bf16_pair_fp32(c, &b2[0], &b2[1])) {
        double v2[2];
        box_muller_f64(c, &v2[0], &v2[1]);
        b2[0] = f64_to_bf16_bits(v2[0]);
        b2[1] = f64_to_bf16_bits(v2[1]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t e = 2 * g + h;
        if (e >= total) break;
        const int64_t i = e / r, j = e - i * r;
        const int64_t idx = layout == 0 ? i * ld + j : j * ld + i;
        if constexpr (kDtype == kF32HoldingBf16)
          static_cast<uint32_t*>(out)[idx] = (uint32_t)b2[h] << 16;
        else
          static_cast<uint16_t*>(out)[idx] = b2[h];
      }
    } else {
      double v2[2];
      box_muller_f64(c, &v2[0], &v2[1]);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t e = 2 * g + h;
        if (e >= total) break;
        const int64_t i = e / r, j = e - i * r;
        const int64_t idx = layout == 0 ? i * ld + j : j * ld + i;
        store_value<kDtype>(out, idx, v2[h]);
      }
    }
  }
}

// Each block first scans the r flags (almost always all zero) and returns at
// once when no column is dead; otherwise it fills its share of the rows of the
// dead columns.  Entry (i, k) is element k*M + i of the stream.
template <typename T>
__global__ void fill_dead_kernel(int64_t M, int r, const int* __restrict__ dead, T* __restrict__ Q,
                                 int64_t ldq, uint64_t seed, double scale) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < r; k += blockDim.x)
    if (dead[k]) any = 1;
  __syncthreads();
  if (!any) return;
  for (int k = 0; k < r; ++k) {
    if (!dead[k]) continue;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
      const int64_t e = (int64_t)k * M + i;
      double a, b;
      gaussian_pair(seed, (uint64_t)e >> 1, &a, &b);
      Q[i * ldq + k] = (T)(((e & 1) ? b : a) * scale);
    }
  }
}

}  // namespace

rsvd_status fill_dead_columns(int64_t M, int r, const int* dead, void* Q, int64_t ldq, int dtype,
                              uint64_t seed, cudaStream_t stream) {
  if (M * r == 0) return RSVD_OK;
  int64_t blocks = cdiv(M, 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  const double scale = 1.0 / sqrt((double)M);
  if (dtype == RSVD_F64)
    fill_dead_kernel<double><<<(int)blocks, 256, 0, stream>>>(M, r, dead, static_cast<double*>(Q), ldq, seed, scale);
  else
    fill_dead_kernel<float><<<(int)blocks, 256, 0, stream>>>(M, r, dead, static_cast<float*>(Q), ldq, seed, scale);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

rsvd_status launch_gaussian(uint64_t seed, int64_t n, int64_t r, int dtype, int layout, void* out,
                            int64_t ld, cudaStream_t stream) {
  const int64_t pairs = (n * r + 1) / 2;
  if (pairs == 0) return RSVD_OK;
  const int threads = 256;
  int64_t blocks = cdiv(pairs, threads);
  if (blocks > 152 * 16) blocks = 152 * 16;
  switch (dtype) {
    case RSVD_F64:
      gaussian_kernel<RSVD_F64><<<(int)blocks, threads, 0, stream>>>(seed, n, r, layout, out, ld);
      break;
    case RSVD_F32:
      gaussian_kernel<RSVD_F32><<<(int)blocks, threads, 0, stream>>>(seed, n, r, layout, out, ld);
      break;
    case RSVD_BF16:
      gaussian_kernel<RSVD_BF16><<<(int)blocks, threads, 0, stream>>>(seed, n, r, layout, out, ld);
      break;
    case kF32HoldingBf16:
      gaussian_kernel<kF32HoldingBf16><<<(int)blocks, threads, 0, stream>>>(seed, n, r, layout, out, ld);
      break;
    default:
      return fail(RSVD_ERR_INVALID_ARG, "gaussian: dtype must be F64, F32 or BF16");
  }
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

}  // namespace rsvd

extern "C" rsvd_status rsvd_gaussian(uint64_t seed, int64_t n, int64_t r, int32_t out_dtype,
                                     int32_t layout, void* out, int64_t ld, void* stream) {
  if (n < 0 || r < 0 || (layout != 0 && layout != 1))
    return rsvd::fail(RSVD_ERR_INVALID_ARG, "rsvd_gaussian: n, r >= 0 and layout 0 or 1");
  if (n * r == 0) return RSVD_OK;
  if (!out) return rsvd::fail(RSVD_ERR_INVALID_ARG, "rsvd_gaussian: out is NULL");
  if ((layout == 0 && ld < r) || (layout == 1 && ld < n))
    return rsvd::fail(RSVD_ERR_INVALID_ARG, "rsvd_gaussian: leading dimension too small");
  return rsvd::launch_gaussian(seed, n, r, out_dtype, layout, out, ld, rsvd::as_stream(stream));
}
