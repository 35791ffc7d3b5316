// Section 2.1 steps 3-4: orthonormal basis Q_r of the sketch Y by CholeskyQR2.
//
//   G = Y^T Y          chunk partials (simt_gemm) added in FP64
//   G = L L^T          FP64 Cholesky, one CTA (cholesky_kernel)
//   Rinv = L^-T        triangular inverse, one warp per column (trilinv_kernel)
//   Q1 = Y Rinv        panel product in the panel's precision (simt_gemm)
// and the same once more on Q1 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto,
// "CholeskyQR2", 2014), which restores orthogonality to working precision
// whenever the first Cholesky succeeds.  The second Gram is close to the
// identity, so for FP32 panels its Cholesky and inverse run in FP32.
// R = R2 R1 is formed (in FP64) on request.
//
// Rank deficiency: a Cholesky pivot that has lost all but a tau fraction of its
// column's mass is deflated and the column of Q1 replaced by a unit random
// vector (from the library's Gaussian stream with a fixed seed), which the
// second sweep orthonormalises against the rest; R then has a zero row there.
//
// Gram accumulation: products are summed in the panel's type over chunks of
// 256 rows (more for panels over 2^19 rows; the SIMT GEMM, one partial per
// chunk) and the chunk partials are added in FP64 in chunk order.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

// Right-looking Cholesky G = L L^T of an r x r symmetric matrix in one CTA of
// 256 threads (the per-column barriers dominate, so fewer warps are faster).  The working copy A lives in shared memory when it fits
// (r <= kCholSmemMaxR), else in global memory (L2); the factor L (lower,
// row-major, zero above the diagonal) is written to `L`.  Step k: thread 0
// forms the pivot; then every thread writes its part of column k of L and
// applies the rank-1 update A[i][j] -= A[i][k] A[j][k] / d to the trailing
// lower triangle, reading column k unscaled (it is not written in that phase),
// so two barriers per column suffice.
//
// Pivot deflation: a pivot whose remaining mass d is at most tau * G_kk (the
// column is linearly dependent on the previous ones to the accuracy of G) is
// marked dead: L[k][k] = 1 and L[i][k] = 0 below it, so Y L^-T leaves that
// column as a negligible residual, to be replaced by a fresh random direction
// (fill_dead_columns).  A NaN or infinite pivot records DEV_NOT_SPD.
constexpr int kCholSmemBytes = 160 * 160 * 8;

template <typename T>
__global__ void __launch_bounds__(256)
cholesky_kernel(int r, const double* __restrict__ G, T* __restrict__ L, T* __restrict__ Awork,
                int* __restrict__ dead, double tau, int* status) {
  extern __shared__ __align__(16) unsigned char chol_smem[];
  __shared__ T s_inv, s_inv2;
  __shared__ int s_dead;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tx = tid & 31, ty = tid >> 5, nty = nt >> 5;
  const bool in_smem = (size_t)r * r * sizeof(T) + (size_t)r * sizeof(double) <= (size_t)kCholSmemBytes;
  T* gdiag = reinterpret_cast<T*>(chol_smem);  // tau * G_kk, the deflation floor
  T* A = in_smem ? reinterpret_cast<T*>(chol_smem + (size_t)r * sizeof(double)) : Awork;
  for (int e = tid; e < r * r; e += nt) { A[e] = (T)G[e]; L[e] = T(0); }
  for (int k = tid; k < r; k += nt) gdiag[k] = (T)(tau * G[(int64_t)k * r + k]);
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (tid == 0) {
      const T d = A[k * r + k];
      const T floor_k = gdiag[k];
      int is_dead = 0;
      if (!isfinite(d) || !isfinite(floor_k)) { is_dead = 1; dev_set_status(status, DEV_NOT_SPD); }
      else if (!(d > floor_k) || !(d > T(0))) is_dead = 1;
      dead[k] = is_dead;
      const T piv = is_dead ? T(0) : sqrt(d);
      s_inv = is_dead ? T(0) : T(1) / piv;
      s_inv2 = is_dead ? T(0) : T(1) / d;
      s_dead = is_dead;
      L[(int64_t)k * r + k] = is_dead ? T(1) : piv;
    }
    __syncthreads();
    const T inv = s_inv, inv2 = s_inv2;
    for (int i = k + 1 + tid; i < r; i += nt) L[(int64_t)i * r + k] = A[i * r + k] * inv;
    if (!s_dead) {
      for (int i = k + 1 + ty; i < r; i += nty) {
        const T cik = A[i * r + k] * inv2;
        for (int j = k + 1 + tx; j <= i; j += 32) A[i * r + j] -= cik * A[j * r + k];
      }
    }
    __syncthreads();
  }
}

// Any pivot dead in the second sweep means the panel stayed rank deficient
// after its dead columns were replaced: report it.
__global__ void check_dead_kernel(int r, const int* __restrict__ dead, int* status) {
  for (int k = threadIdx.x; k < r; k += blockDim.x)
    if (dead[k]) dev_set_status(status, DEV_NOT_SPD);
}

// X = L^-1 by forward substitution; Rinv = X^T (upper), in T and in the panel
// type TOUT.  Each CTA has four warps, one column j each; the rows of L from
// the CTA's first column down are staged in shared memory when they fit, and
// the reciprocals of the diagonal are formed once up front, so each sequential
// step of a column is a shared-memory dot product and one multiply.
constexpr int kInvCols = 4;
constexpr int kInvSmemBytes = 200 * 1024;

template <typename T, typename TOUT>
__global__ void __launch_bounds__(32 * kInvCols)
trilinv_kernel(int r, const T* __restrict__ L, T* __restrict__ Rinv, TOUT* __restrict__ Rinv_t, int staged) {
  extern __shared__ __align__(16) unsigned char inv_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j0 = blockIdx.x * kInvCols;
  const int rows = r - j0;                                  // rows/cols j0..r-1 of L
  T* xs = reinterpret_cast<T*>(inv_smem);                   // kInvCols x r solution vectors
  T* dinv = xs + kInvCols * r;                              // 1 / L[i][i]
  T* Ls = dinv + r;                                         // staged rows x rows block
  for (int e = threadIdx.x; e < kInvCols * r; e += blockDim.x) xs[e] = T(0);
  for (int i = j0 + threadIdx.x; i < r; i += blockDim.x) dinv[i] = T(1) / L[(int64_t)i * r + i];
  if (staged)
    for (int e = threadIdx.x; e < rows * rows; e += blockDim.x) {
      const int i = e / rows, l = e % rows;
      Ls[e] = l <= i ? L[(int64_t)(j0 + i) * r + (j0 + l)] : T(0);
    }
  __syncthreads();
  const int j = j0 + warp;
  if (j < r) {
    T* x = xs + warp * r;
    auto Lat = [&](int i, int l) -> T { return staged ? Ls[(i - j0) * rows + (l - j0)] : L[(int64_t)i * r + l]; };
    if (lane == 0) x[j] = dinv[j];
    __syncwarp();
    for (int i = j + 1; i < r; ++i) {
      T s = T(0);
      for (int l = j + lane; l < i; l += 32) s += Lat(i, l) * x[l];
      s = warp_sum(s);
      if (lane == 0) x[i] = -s * dinv[i];
      __syncwarp();
    }
    for (int i = lane; i < r; i += 32) {
      Rinv[(int64_t)j * r + i] = x[i];  // Rinv[j][i] = X[i][j]
      Rinv_t[(int64_t)j * r + i] = (TOUT)x[i];
    }
  }
}

// R = R2 R1 with R1 = L1^T, R2 = L2^T (both upper triangular).  A dead pivot l
// of the first sweep carries no part of Y (its column was a negligible
// residual), so row l of R1 counts as zero.
template <typename T2>
__global__ void rprod_kernel(int r, const double* __restrict__ L1, const int* __restrict__ dead1,
                             const T2* __restrict__ L2, double* __restrict__ R) {
  const int64_t total = (int64_t)r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    double s = 0.0;
    for (int l = i; l <= j; ++l)
      if (!dead1[l]) s += (double)L2[(int64_t)l * r + i] * L1[(int64_t)j * r + l];
    R[e] = j >= i ? s : 0.0;
  }
}

// Rows per partial Gram: each partial is a sum of gram_chunk(M) products in
// the panel's type -- 256 rows, or more for panels over 2^19 rows so that at
// most about kGramMaxChunks partials are stored -- and the partials are added
// in FP64 in chunk order.
constexpr int64_t kGramChunk = 256;
constexpr int64_t kGramMaxChunks = 2048;

int64_t gram_chunk(int64_t M) {
  const int64_t c = round_up(cdiv(M, kGramMaxChunks), kGramChunk);
  return c > kGramChunk ? c : kGramChunk;
}

int64_t gram_chunks(int64_t M) { return cdiv(M, gram_chunk(M)); }

template <typename T>
__global__ void gram_sum_partials_kernel(int r, int64_t nchunks, const T* __restrict__ P, double* __restrict__ G) {
  const int64_t rr = (int64_t)r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < rr; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = (int)(e / r), b = (int)(e % r);
    if (b < a) continue;
    double s = 0.0;
    for (int64_t c = 0; c < nchunks; ++c) s += (double)P[c * rr + e];
    G[(int64_t)a * r + b] = s;
    G[(int64_t)b * r + a] = s;
  }
}

// G = Y^T Y: the SIMT GEMM forms one r x r partial per chunk of kGramChunk rows
// (op(A) = Y^T), and the partials are added in FP64.
template <typename T>
rsvd_status gram(int64_t M, int r, const T* Y, int64_t ldy, const OrthWs& ws, cudaStream_t stream) {
  const int64_t nchunks = gram_chunks(M);
  T* P = static_cast<T*>(ws.gram_partial);
  RSVD_TRY(simt_gemm_partials<T>(r, r, M, Y, ldy, true, Y, ldy, (int)nchunks, gram_chunk(M), P, stream));
  const int64_t blocks = cdiv((int64_t)r * r, 256);
  gram_sum_partials_kernel<T><<<(int)blocks, 256, 0, stream>>>(r, nchunks, P, ws.G);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

// Relative pivot floor of the deflation test: a few hundred units of the Gram's
// accumulation accuracy (FP64 sums for FP64 panels, FP32 runs for FP32 panels).
template <typename T>
double pivot_tau();
template <>
double pivot_tau<double>() { return 1e-13; }
template <>
double pivot_tau<float>() { return 1e-5; }

// The second sweep factors Q1^T Q1, close to the identity: FP32 panels do it in
// FP32 (pivots far from the deflation floor), FP64 panels in FP64.
template <typename T>
struct SecondSweep { using type = double; };
template <>
struct SecondSweep<float> { using type = float; };

// Cholesky + triangular inverse.  TF is the arithmetic of the factorisation
// (FP64, or FP32 for the near-identity Gram of a second sweep on an FP32
// panel); T is the panel type that receives Rinv.
template <typename TF, typename T>
rsvd_status chol_inv(int r, const OrthWs& ws, TF* L, int* dead, double tau, cudaStream_t stream) {
  static bool attrs = false;
  if (!attrs) {
    RSVD_CUDA(cudaFuncSetAttribute(cholesky_kernel<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCholSmemBytes));
    RSVD_CUDA(cudaFuncSetAttribute(trilinv_kernel<TF, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kInvSmemBytes));
    attrs = true;
  }
  const size_t chol_need = (size_t)r * r * sizeof(TF) + (size_t)r * sizeof(double);
  const size_t chol_smem = chol_need <= (size_t)kCholSmemBytes ? chol_need : (size_t)r * sizeof(double);
  cholesky_kernel<TF><<<1, 256, chol_smem, stream>>>(r, ws.G, L, reinterpret_cast<TF*>(ws.Awork), dead, tau,
                                                      ws.status);
  RSVD_CUDA(after_launch());
  const size_t base = ((size_t)kInvCols * r + r) * sizeof(TF);
  const size_t staged_bytes = base + (size_t)r * r * sizeof(TF);
  const int staged = staged_bytes <= (size_t)kInvSmemBytes ? 1 : 0;
  trilinv_kernel<TF, T><<<(int)cdiv(r, kInvCols), 32 * kInvCols, staged ? staged_bytes : base, stream>>>(
      r, L, reinterpret_cast<TF*>(ws.Rinv), static_cast<T*>(ws.Rinv_t), staged);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

}  // namespace

size_t orth_ws_bytes(int64_t M, int r, int dtype) {
  Sizer s;
  const size_t esz = dtype == RSVD_F64 ? 8 : 4;
  s.take<double>((size_t)r * r * 5);
  s.take<int>((size_t)2 * r);
  s.take<char>((size_t)r * r * esz);
  s.take<char>((size_t)gram_chunks(M) * r * r * esz);
  s.take<char>((size_t)M * round_up(r, 4) * esz);
  s.take<int>(4);
  return s.used + 256;
}

OrthWs orth_ws_carve(Carver& c, int64_t M, int r, int dtype) {
  OrthWs w;
  const size_t esz = dtype == RSVD_F64 ? 8 : 4;
  double* base = c.take<double>((size_t)r * r * 5);
  if (base) {
    w.G = base; w.L1 = base + r * r; w.L2 = base + 2 * r * r; w.Rinv = base + 3 * r * r;
    w.Awork = base + 4 * r * r;
  }
  int* dd = c.take<int>((size_t)2 * r);
  if (dd) { w.dead1 = dd; w.dead2 = dd + r; }
  w.Rinv_t = c.take<char>((size_t)r * r * esz);
  w.gram_partial = c.take<char>((size_t)gram_chunks(M) * r * r * esz);
  w.gram_chunks = gram_chunks(M);
  w.ld_tmp = round_up(r, 4);
  w.tmp = c.take<char>((size_t)M * w.ld_tmp * esz);
  w.status = c.take<int>(4);
  return w;
}

template <typename T>
rsvd_status orth_panel(int64_t M, int r, const T* Y, int64_t ldy, T* Q, int64_t ldq, double* R,
                       const OrthWs& ws, cudaStream_t stream) {
  T* Q1 = static_cast<T*>(ws.tmp);
  const T* Rt = static_cast<const T*>(ws.Rinv_t);
  // sweep 1 (dead pivots: the panel is rank deficient to the Gram's accuracy;
  // their columns of Q1 are replaced by unit random directions)
  RSVD_TRY(gram<T>(M, r, Y, ldy, ws, stream));
  RSVD_TRY((chol_inv<double, T>(r, ws, ws.L1, ws.dead1, pivot_tau<T>(), stream)));
  RSVD_TRY(simt_gemm<T>(M, r, r, Y, ldy, false, Rt, r, Q1, ws.ld_tmp, false, 1, r, nullptr, stream));
  RSVD_TRY(fill_dead_columns(M, r, ws.dead1, Q1, ws.ld_tmp, sizeof(T) == 8 ? RSVD_F64 : RSVD_F32,
                             kDeadFillSeed, stream));
  // sweep 2
  RSVD_TRY(gram<T>(M, r, Q1, ws.ld_tmp, ws, stream));
  using TF2 = typename SecondSweep<T>::type;
  TF2* L2 = reinterpret_cast<TF2*>(ws.L2);
  RSVD_TRY((chol_inv<TF2, T>(r, ws, L2, ws.dead2, pivot_tau<T>(), stream)));
  check_dead_kernel<<<1, 256, 0, stream>>>(r, ws.dead2, ws.status);
  RSVD_CUDA(after_launch());
  RSVD_TRY(simt_gemm<T>(M, r, r, Q1, ws.ld_tmp, false, Rt, r, Q, ldq, false, 1, r, nullptr, stream));
  if (R) {
    rprod_kernel<TF2><<<(int)cdiv((int64_t)r * r, 256), 256, 0, stream>>>(r, ws.L1, ws.dead1, L2, R);
    RSVD_CUDA(after_launch());
  }
  return RSVD_OK;
}

template rsvd_status orth_panel<float>(int64_t, int, const float*, int64_t, float*, int64_t, double*,
                                       const OrthWs&, cudaStream_t);
template rsvd_status orth_panel<double>(int64_t, int, const double*, int64_t, double*, int64_t,
                                        double*, const OrthWs&, cudaStream_t);

}  // namespace rsvd
