// Section 2.1 step 7 helpers: type conversion of the small factors and the
// sign convention of the singular-vector pairs.
//
// Sign rule (the paper leaves signs free): each pair (u_i, v_i) is negated
// when the largest-magnitude entry of u_i is negative; among entries of equal
// magnitude the lowest row index decides.  The column maxima are found per
// row chunk and combined with ties going to the lower chunk, so the first
// maximum wins.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

template <typename Tin, typename Tout>
__global__ void convert_kernel(int64_t rows, int64_t cols, const Tin* __restrict__ in, int64_t ldi,
                               Tout* __restrict__ out, int64_t ldo) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    out[i * ldo + j] = (Tout)in[i * ldi + j];
  }
}

template <typename T>
__global__ void gather_colmajor_kernel(int64_t rows, int64_t cols, const T* __restrict__ A, int64_t s_row,
                                       int64_t s_col, double* __restrict__ out) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, i = e - c * rows;
    out[e] = (double)A[i * s_row + c * s_col];
  }
}

// Rows per chunk: 64, more for tall panels so that at most about 4096 chunk
// maxima are stored.
inline int64_t sign_chunk(int64_t m) {
  const int64_t c = round_up(cdiv(m, 4096), 8);
  return c > 64 ? c : 64;
}

// Per chunk of rows and column j: the first entry of largest magnitude (value
// and magnitude), compared in the panel's own type (FP64 arithmetic is costly
// on this GPU).
template <typename T>
__global__ void colmax_kernel(int64_t m, int k, int64_t chunk, const T* __restrict__ U, int64_t ldu,
                              T* __restrict__ part) {
  const int j = threadIdx.x + blockIdx.y * blockDim.x;
  if (j >= k) return;
  const int64_t r0 = (int64_t)blockIdx.x * chunk;
  const int64_t r1 = min(m, r0 + chunk);
  T best = T(-1), val = T(0);
  for (int64_t i0 = r0; i0 < r1; i0 += 8) {
    T x[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) x[t] = i0 + t < r1 ? U[(i0 + t) * ldu + j] : T(0);
#pragma unroll
    for (int t = 0; t < 8; ++t) {
      const T ax = x[t] < T(0) ? -x[t] : x[t];
      if (i0 + t < r1 && ax > best) { best = ax; val = x[t]; }
    }
  }
  part[((int64_t)blockIdx.x * k + j) * 2 + 0] = best;
  part[((int64_t)blockIdx.x * k + j) * 2 + 1] = val;
}

// One warp per column: the chunk maxima combined so that the largest
// magnitude wins and, among equal magnitudes, the lowest chunk (row) does.
template <typename T>
__global__ void choose_flip_kernel(int k, int nchunks, const T* __restrict__ part, int* __restrict__ flip) {
  const int lane = threadIdx.x & 31;
  const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int j = w0; j < k; j += nw) {
    T best = T(-1), val = T(0);
    int idx = 0x7fffffff;
    for (int c = lane; c < nchunks; c += 32) {
      const T b = part[((int64_t)c * k + j) * 2];
      if (b > best) { best = b; val = part[((int64_t)c * k + j) * 2 + 1]; idx = c; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T b2 = __shfl_xor_sync(0xffffffffu, best, o);
      const T v2 = __shfl_xor_sync(0xffffffffu, val, o);
      const int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
      if (b2 > best || (b2 == best && i2 < idx)) { best = b2; val = v2; idx = i2; }
    }
    if (lane == 0) flip[j] = val < T(0) ? 1 : 0;
  }
}

// One warp per row of U (then of V): lanes over the columns, negating those
// whose pair was chosen for a flip.
template <typename T>
__global__ void flip_kernel(int64_t m, int64_t n, int k, const int* __restrict__ flip,
                            T* __restrict__ U, int64_t ldu, T* __restrict__ V, int64_t ldv) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w0; row < m + n; row += nw) {
    T* p = row < m ? U + row * ldu : V + (row - m) * ldv;
    for (int j = lane; j < k; j += 32)
      if (flip[j]) p[j] = -p[j];
  }
}

}  // namespace

template <typename Tin, typename Tout>
rsvd_status convert_matrix(int64_t rows, int64_t cols, const Tin* in, int64_t ldi, Tout* out,
                           int64_t ldo, cudaStream_t stream) {
  if (rows * cols == 0) return RSVD_OK;
  int64_t blocks = cdiv(rows * cols, 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  convert_kernel<Tin, Tout><<<(int)blocks, 256, 0, stream>>>(rows, cols, in, ldi, out, ldo);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

template rsvd_status convert_matrix<double, float>(int64_t, int64_t, const double*, int64_t, float*,
                                                   int64_t, cudaStream_t);
template rsvd_status convert_matrix<double, double>(int64_t, int64_t, const double*, int64_t, double*,
                                                    int64_t, cudaStream_t);
template rsvd_status convert_matrix<float, float>(int64_t, int64_t, const float*, int64_t, float*,
                                                  int64_t, cudaStream_t);

template <typename T>
rsvd_status gather_colmajor_f64(int64_t rows, int64_t cols, const T* A, int64_t s_row, int64_t s_col,
                                double* out, cudaStream_t stream) {
  if (rows * cols == 0) return RSVD_OK;
  int64_t blocks = cdiv(rows * cols, 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  gather_colmajor_kernel<T><<<(int)blocks, 256, 0, stream>>>(rows, cols, A, s_row, s_col, out);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}
template rsvd_status gather_colmajor_f64<double>(int64_t, int64_t, const double*, int64_t, int64_t, double*,
                                                 cudaStream_t);
template rsvd_status gather_colmajor_f64<float>(int64_t, int64_t, const float*, int64_t, int64_t, double*,
                                                cudaStream_t);

size_t sign_scratch_bytes(int64_t m, int k) {
  return (size_t)cdiv(m, sign_chunk(m)) * k * 2 * sizeof(double) + (size_t)k * sizeof(int) + 256;
}

template <typename T>
rsvd_status normalise_signs(int64_t m, int64_t n, int k, T* U, int64_t ldu, T* V, int64_t ldv,
                            void* scratch, size_t scratch_bytes, cudaStream_t stream) {
  if (k <= 0 || m <= 0) return RSVD_OK;
  if (sign_scratch_bytes(m, k) > scratch_bytes)
    return fail(RSVD_ERR_INVALID_ARG, "normalise_signs: scratch too small");
  const int64_t chunk = sign_chunk(m);
  const int64_t nchunks = cdiv(m, chunk);
  T* part = static_cast<T*>(scratch);
  int* flip = reinterpret_cast<int*>(static_cast<double*>(scratch) + nchunks * k * 2);
  const int tpb = k < 128 ? 32 * (int)cdiv(k, 32) : 128;
  colmax_kernel<T><<<dim3((unsigned)nchunks, (unsigned)cdiv(k, tpb)), tpb, 0, stream>>>(m, k, chunk, U, ldu,
                                                                                        part);
  RSVD_CUDA(after_launch());
  choose_flip_kernel<T><<<(int)cdiv((int64_t)k * 32, 256), 256, 0, stream>>>(k, (int)nchunks, part, flip);
  RSVD_CUDA(after_launch());
  int64_t blocks = cdiv((m + n) * 32, 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  flip_kernel<T><<<(int)blocks, 256, 0, stream>>>(m, n, k, flip, U, ldu, V, ldv);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

namespace {
// flag = 1 when ||s[:k] - prev[:k]||^2 <= tol^2 ||s[:k]||^2 (one block, fixed-order sums)
__global__ void sigma_change_kernel(int k, const double* __restrict__ s, const double* __restrict__ prev, double tol,
                                    int* flag) {
  __shared__ double red[2][32];
  double num = 0.0, den = 0.0;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    const double d = s[j] - prev[j];
    num += d * d;
    den += s[j] * s[j];
  }
  num = warp_sum(num);
  den = warp_sum(den);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red[0][w] = num; red[1][w] = den; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { a += red[0][i]; b += red[1][i]; }
    *flag = (a <= tol * tol * b) ? 1 : 0;
  }
}
}  // namespace

rsvd_status sigma_change_below(int k, const double* sigma, const double* prev, double tol, int* flag,
                               cudaStream_t stream) {
  sigma_change_kernel<<<1, 256, 0, stream>>>(k, sigma, prev, tol, flag);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

template rsvd_status normalise_signs<float>(int64_t, int64_t, int, float*, int64_t, float*, int64_t,
                                            void*, size_t, cudaStream_t);
template rsvd_status normalise_signs<double>(int64_t, int64_t, int, double*, int64_t, double*, int64_t,
                                             void*, size_t, cudaStream_t);

}  // namespace rsvd
