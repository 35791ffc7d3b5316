// Backward pass (adjoint) of the rank-k truncated SVD returned by rsvd_run.
//
// Not in the paper: the truncated-SVD adjoint of J. Townsend, "Differentiating
// the Singular Value Decomposition" (2016).  With F_ij = 1/(S_j^2 - S_i^2)
// (i != j; 0 on the diagonal and for numerically equal S_i, S_j),
//   J = F o (U^T dU - dU^T U),  K = F o (V^T dV - dV^T V),
//   M = J diag(S) + diag(dS) + diag(S) K,
//   P = (dU - U (U^T dU)) diag(S)^-1,   Q = (dV - V (V^T dV)) diag(S)^-1,
//   dA = [U | P] [V M^T + Q | V]^T        (one rank-2k product).
// The k x k pieces are formed in FP64 (the U^T dU and V^T dV reductions add
// FP64 chunk sums); the panels and the final product run in the data type.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int64_t kChunk = 256;

// One warp per entry: lane l adds the chunks l, l + 32, ... in FP64, then the
// 32 lane sums are added by a fixed shuffle tree (the same order every call).
template <typename T>
__global__ void sum_partials_f64_kernel(int k, int64_t nchunks, const T* __restrict__ P, double* __restrict__ out) {
  const int64_t kk = (int64_t)k * k;
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < kk; e += warps) {
    double s = 0.0;
    for (int64_t c = lane; c < nchunks; c += 32) s += (double)P[c * kk + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[e] = s;
  }
}

// The k x k matrices M^T (to multiply V), U^T dU and V^T dV in the data type,
// one entry per thread over the grid, and 1/S (block 0).  A pair with S_i^2 = S_j^2 to within 1e-12 S_max^2 gets F = 0.
template <typename T>
__global__ void small_adjoint_kernel(int k, const T* __restrict__ S, const T* __restrict__ dS,
                                     const double* __restrict__ UtdU, const double* __restrict__ VtdV,
                                     T* __restrict__ Mt, T* __restrict__ UtdU_t, T* __restrict__ VtdV_t,
                                     T* __restrict__ Sinv) {
  double smax = 0.0;
  for (int i = 0; i < k; ++i) smax = fmax(smax, fabs((double)S[i]));
  const double guard = 1e-12 * smax * smax;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < k * k; e += gridDim.x * blockDim.x) {
    const int i = e / k, j = e % k;
    const double si = (double)S[i], sj = (double)S[j];
    double Fij = 0.0;
    const double d = sj * sj - si * si;
    if (i != j && fabs(d) > guard) Fij = 1.0 / d;
    const double Jij = UtdU ? Fij * (UtdU[i * k + j] - UtdU[j * k + i]) : 0.0;
    const double Kij = VtdV ? Fij * (VtdV[i * k + j] - VtdV[j * k + i]) : 0.0;
    double Mij = Jij * sj + si * Kij;
    if (i == j && dS) Mij += (double)dS[i];
    Mt[j * k + i] = (T)Mij;  // M^T
    UtdU_t[e] = UtdU ? (T)UtdU[e] : T(0);
    VtdV_t[e] = VtdV ? (T)VtdV[e] : T(0);
  }
  if (blockIdx.x == 0)
    for (int i = threadIdx.x; i < k; i += blockDim.x) Sinv[i] = (T)(1.0 / (double)S[i]);
}

// L = [U | (dU - UX) diag(Sinv)]   (rows x 2k), UX = U (U^T dU) precomputed.
template <typename T>
__global__ void left_panel_kernel(int64_t rows, int k, const T* __restrict__ U, const T* __restrict__ dU,
                                  const T* __restrict__ UX, const T* __restrict__ Sinv, T* __restrict__ L) {
  const int64_t total = rows * 2 * k;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / (2 * k);
    const int c = (int)(e - i * 2 * k);
    T v;
    if (c < k) v = U[i * k + c];
    else {
      const int j = c - k;
      v = dU ? (dU[i * k + j] - UX[i * k + j]) * Sinv[j] : T(0);
    }
    L[e] = v;
  }
}

// Bt[0:k, :] = (V M^T + (dV - VY) diag(Sinv))^T,  Bt[k:2k, :] = V^T, with VM = V M^T
// and VY = V (V^T dV) precomputed (n x k each).  32 x 32 tiles through shared memory.
template <typename T>
__global__ void right_panel_kernel(int64_t n, int k, const T* __restrict__ V, const T* __restrict__ dV,
                                   const T* __restrict__ VM, const T* __restrict__ VY, const T* __restrict__ Sinv,
                                   T* __restrict__ Bt) {
  __shared__ T tile[2][32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;  // rows of V (columns of Bt)
  const int c0 = blockIdx.y * 32;               // columns of V (rows of Bt)
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int64_t i = r0 + t;
    const int j = c0 + threadIdx.x;
    T top = T(0), bot = T(0);
    if (i < n && j < k) {
      top = VM[i * k + j] + (dV ? (dV[i * k + j] - VY[i * k + j]) * Sinv[j] : T(0));
      bot = V[i * k + j];
    }
    tile[0][t][threadIdx.x] = top;
    tile[1][t][threadIdx.x] = bot;
  }
  __syncthreads();
  for (int t = threadIdx.y; t < 32; t += blockDim.y) {
    const int j = c0 + t;
    const int64_t i = r0 + threadIdx.x;
    if (j < k && i < n) {
      Bt[(int64_t)j * n + i] = tile[0][threadIdx.x][t];
      Bt[(int64_t)(k + j) * n + i] = tile[1][threadIdx.x][t];
    }
  }
}

template <typename T>
rsvd_status proj_gram(int64_t rows, int k, const T* X, const T* Y, T* partial, double* out, cudaStream_t st) {
  const int64_t nchunks = cdiv(rows, kChunk);
  RSVD_TRY(simt_gemm_partials<T>(k, k, rows, X, k, true, Y, k, (int)nchunks, kChunk, partial, st));
  sum_partials_f64_kernel<T><<<(int)std::min<int64_t>(cdiv((int64_t)k * k * 32, 256), 152 * 8), 256, 0, st>>>(
      k, nchunks, partial, out);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

}  // namespace

size_t backward_ws_bytes(int64_t m, int64_t n, int k, int dtype) {
  const size_t esz = dtype == RSVD_F64 ? 8 : 4;
  const int64_t mx = m > n ? m : n;
  Sizer s;
  s.take<char>((size_t)m * 2 * k * esz);           // L
  s.take<char>((size_t)2 * k * n * esz);           // Bt
  s.take<char>((size_t)mx * k * esz);              // UX / VY
  s.take<char>((size_t)mx * k * esz);              // VM
  s.take<char>((size_t)cdiv(mx, kChunk) * k * k * esz);  // partials
  s.take<double>((size_t)2 * k * k);               // U^T dU, V^T dV
  s.take<char>((size_t)(3 * k * k + k) * esz);     // M^T, U^T dU, V^T dV, 1/S in the data type
  if (dtype == RSVD_F32) s.take<char>(tc_gemm_wide_ws_bytes(m, 2 * k, n, RSVD_PREC_BF16X3));  // dA on the tensor cores
  return s.used + 256;
}

template <typename T>
rsvd_status backward_typed(int64_t m, int64_t n, int k, const T* U, const T* S, const T* V, const T* dU,
                           const T* dS, const T* dV, T* dA, void* ws, size_t ws_bytes, int* status, cudaStream_t st) {
  const int64_t mx = m > n ? m : n;
  Carver c(ws, ws_bytes);
  T* L = c.take<T>((size_t)m * 2 * k);
  T* Bt = c.take<T>((size_t)2 * k * n);
  T* XY = c.take<T>((size_t)mx * k);
  T* VM = c.take<T>((size_t)mx * k);
  T* partial = c.take<T>((size_t)cdiv(mx, kChunk) * k * k);
  double* UtdU = c.take<double>((size_t)2 * k * k);
  double* VtdV = UtdU ? UtdU + (size_t)k * k : nullptr;
  T* small = c.take<T>((size_t)3 * k * k + k);
  const size_t tcb = std::is_same<T, float>::value ? tc_gemm_wide_ws_bytes(m, 2 * k, n, RSVD_PREC_BF16X3) : 0;
  void* tcws = tcb ? c.take<char>(tcb) : nullptr;
  if (c.overflow) return fail(RSVD_ERR_INVALID_ARG, "rsvd_backward: workspace too small");
  T* Mt = small;
  T* UtdU_t = small + (size_t)k * k;
  T* VtdV_t = small + 2 * (size_t)k * k;
  T* Sinv = small + 3 * (size_t)k * k;
  if (dU) RSVD_TRY(proj_gram<T>(m, k, U, dU, partial, UtdU, st));
  if (dV) RSVD_TRY(proj_gram<T>(n, k, V, dV, partial, VtdV, st));
  small_adjoint_kernel<T><<<(int)cdiv((int64_t)k * k, 256), 256, 0, st>>>(k, S, dS, dU ? UtdU : nullptr,
                                                                          dV ? VtdV : nullptr, Mt, UtdU_t, VtdV_t,
                                                                          Sinv);
  RSVD_CUDA(after_launch());
  // left panel [U | P]
  if (dU) RSVD_TRY(simt_gemm<T>(m, k, k, U, k, false, UtdU_t, k, XY, k, false, 1, k, nullptr, st));
  int64_t lblocks = cdiv(m * 2 * k, 256);
  if (lblocks > 152 * 8) lblocks = 152 * 8;
  left_panel_kernel<T><<<(int)lblocks, 256, 0, st>>>(m, k, U, dU, XY, Sinv, L);
  RSVD_CUDA(after_launch());
  // right panel [V M^T + Q | V], stored transposed (2k x n)
  RSVD_TRY(simt_gemm<T>(n, k, k, V, k, false, Mt, k, VM, k, false, 1, k, nullptr, st));
  if (dV) RSVD_TRY(simt_gemm<T>(n, k, k, V, k, false, VtdV_t, k, XY, k, false, 1, k, nullptr, st));
  right_panel_kernel<T><<<dim3((unsigned)cdiv(n, 32), (unsigned)cdiv(k, 32)), dim3(32, 8), 0, st>>>(
      n, k, V, dV, VM, XY, Sinv, Bt);
  RSVD_CUDA(after_launch());
  // dA = L Bt  (m x n, K = 2k): FP32 data on the tensor cores in split BF16
  // (three products, about 16 significant bits per operand; the sums are
  // 2k = 128 terms long), FP64 data on the FP64 units
  if constexpr (std::is_same<T, float>::value) {
    if ((2 * k) % 4 == 0) {
      rsvd_matrix Lm = {};
      Lm.kind = RSVD_DENSE; Lm.dtype = RSVD_F32; Lm.location = RSVD_ON_DEVICE;
      Lm.m = m; Lm.n = 2 * k; Lm.data = L; Lm.ld = 2 * k;
      return tc_gemm_wide(Lm, RSVD_PREC_BF16X3, n, Bt, n, dA, n, tcws, tcb, status, st);
    }
  }
  RSVD_TRY(simt_gemm<T>(m, n, 2 * k, L, 2 * k, false, Bt, n, dA, n, false, 1, 2 * k, nullptr, st));
  return RSVD_OK;
}

template rsvd_status backward_typed<float>(int64_t, int64_t, int, const float*, const float*, const float*,
                                           const float*, const float*, const float*, float*, void*, size_t, int*,
                                           cudaStream_t);
template rsvd_status backward_typed<double>(int64_t, int64_t, int, const double*, const double*, const double*,
                                            const double*, const double*, const double*, double*, void*, size_t,
                                            int*, cudaStream_t);

}  // namespace rsvd
