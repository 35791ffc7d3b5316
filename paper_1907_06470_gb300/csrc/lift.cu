// Section 2.1 step 7 helpers: type conversion of the small factors and the
// sign convention of the singular-vector pairs.
//
// Sign rule (the paper leaves signs free): each pair (u_i, v_i) is negated
// when the largest-magnitude entry of u_i is negative; among entries of equal
// magnitude the lowest row index decides.  The column maxima are found per
// row chunk and combined in chunk order, so the first maximum wins.
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

constexpr int kSignRows = 512;

template <typename T>
__global__ void colmax_kernel(int64_t m, int k, const T* __restrict__ U, int64_t ldu,
                              double* __restrict__ part) {
  const int j = threadIdx.x + blockIdx.y * blockDim.x;
  if (j >= k) return;
  const int64_t r0 = (int64_t)blockIdx.x * kSignRows;
  const int64_t r1 = min(m, r0 + kSignRows);
  double best = -1.0, val = 0.0;
  for (int64_t i = r0; i < r1; ++i) {
    const double x = (double)U[i * ldu + j];
    if (fabs(x) > best) { best = fabs(x); val = x; }
  }
  part[((int64_t)blockIdx.x * k + j) * 2 + 0] = best;
  part[((int64_t)blockIdx.x * k + j) * 2 + 1] = val;
}

__global__ void choose_flip_kernel(int k, int nchunks, const double* __restrict__ part,
                                   int* __restrict__ flip) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) {
    double best = -1.0, val = 0.0;
    for (int c = 0; c < nchunks; ++c) {
      const double b = part[((int64_t)c * k + j) * 2];
      if (b > best) { best = b; val = part[((int64_t)c * k + j) * 2 + 1]; }
    }
    flip[j] = val < 0.0 ? 1 : 0;
  }
}

template <typename T>
__global__ void flip_kernel(int64_t m, int64_t n, int k, const int* __restrict__ flip,
                            T* __restrict__ U, int64_t ldu, T* __restrict__ V, int64_t ldv) {
  const int64_t tu = m * k, tv = n * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tu + tv;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (e < tu) {
      const int64_t i = e / k; const int j = (int)(e - i * k);
      if (flip[j]) U[i * ldu + j] = -U[i * ldu + j];
    } else {
      const int64_t f = e - tu;
      const int64_t i = f / k; const int j = (int)(f - i * k);
      if (flip[j]) V[i * ldv + j] = -V[i * ldv + j];
    }
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
  return (size_t)cdiv(m, kSignRows) * k * 2 * sizeof(double) + (size_t)k * sizeof(int) + 256;
}

template <typename T>
rsvd_status normalise_signs(int64_t m, int64_t n, int k, T* U, int64_t ldu, T* V, int64_t ldv,
                            void* scratch, size_t scratch_bytes, cudaStream_t stream) {
  if (k <= 0 || m <= 0) return RSVD_OK;
  if (sign_scratch_bytes(m, k) > scratch_bytes)
    return fail(RSVD_ERR_INVALID_ARG, "normalise_signs: scratch too small");
  const int64_t nchunks = cdiv(m, kSignRows);
  double* part = static_cast<double*>(scratch);
  int* flip = reinterpret_cast<int*>(part + nchunks * k * 2);
  const int tpb = k < 128 ? 32 * (int)cdiv(k, 32) : 128;
  colmax_kernel<T><<<dim3((unsigned)nchunks, (unsigned)cdiv(k, tpb)), tpb, 0, stream>>>(m, k, U, ldu,
                                                                                        part);
  RSVD_CUDA(after_launch());
  choose_flip_kernel<<<(int)cdiv(k, 128), 128, 0, stream>>>(k, (int)nchunks, part, flip);
  RSVD_CUDA(after_launch());
  int64_t blocks = cdiv((m + n) * k, 256);
  if (blocks > 152 * 4) blocks = 152 * 4;
  flip_kernel<T><<<(int)blocks, 256, 0, stream>>>(m, n, k, flip, U, ldu, V, ldv);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

template rsvd_status normalise_signs<float>(int64_t, int64_t, int, float*, int64_t, float*, int64_t,
                                            void*, size_t, cudaStream_t);
template rsvd_status normalise_signs<double>(int64_t, int64_t, int, double*, int64_t, double*, int64_t,
                                             void*, size_t, cudaStream_t);

}  // namespace rsvd
