// Section 2.1 steps 3-4: orthonormal basis Q_r of the sketch Y by CholeskyQR2.
//
//   G = Y^T Y          FP64 accumulation (gram_partial + gram_reduce)
//   G = L L^T          FP64 Cholesky, one CTA (cholesky_kernel)
//   Rinv = L^-T        FP64 triangular inverse, one warp per column (trilinv_kernel)
//   Q1 = Y Rinv        panel product in the panel's precision (simt_gemm)
// and the same once more on Q1 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto,
// "CholeskyQR2", 2014), which restores orthogonality to working precision
// whenever the first Cholesky succeeds.  R = R2 R1 is formed on request.
//
// Rank deficiency: a Cholesky pivot that has lost all but a tau fraction of its
// column's mass is deflated and the column of Q1 replaced by a unit random
// vector (from the library's Gaussian stream with a fixed seed), which the
// second sweep orthonormalises against the rest; R then has a zero row there.
//
// Gram accumulation: products of FP32 panels are summed in FP32 over runs of at
// most 128 rows and the run sums are added in FP64; FP64 panels are summed in
// FP64 throughout.  Per-CTA partial Grams are added in a fixed order.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int GB = 64;         // Gram output block edge
constexpr int GROWS = 32;      // rows staged per shared-memory load
constexpr int GFLUSH = 4;      // FP32 runs of GFLUSH*GROWS rows

__host__ __device__ inline void pair_of(int p, int nb, int* bi, int* bj) {
  // enumerate (bi, bj), bi <= bj, row by row
  int i = 0;
  while (p >= nb - i) { p -= nb - i; ++i; }
  *bi = i;
  *bj = i + p;
}

template <typename T, typename TACC>
__global__ void __launch_bounds__(256)
gram_partial_kernel(int64_t M, int r, const T* __restrict__ Y, int64_t ldy, int64_t rows_per,
                    int nb, double* __restrict__ partial) {
  __shared__ __align__(16) T Ya[GROWS][GB];
  __shared__ __align__(16) T Yb[GROWS][GB];
  int bi, bj;
  pair_of(blockIdx.x, nb, &bi, &bj);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.y * rows_per;
  const int64_t row1 = min(M, row0 + rows_per);
  double acc64[4][4];
  TACC acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) { acc64[a][b] = 0.0; acc[a][b] = TACC(0); }
  int run = 0;
  for (int64_t rb = row0; rb < row1; rb += GROWS) {
#pragma unroll
    for (int e = 0; e < (GROWS * GB) / 256; ++e) {
      const int idx = e * 256 + tid;
      const int rr = idx / GB, cc = idx % GB;
      const int64_t gr = rb + rr;
      const int ca = bi * GB + cc, cb = bj * GB + cc;
      Ya[rr][cc] = (gr < row1 && ca < r) ? Y[gr * ldy + ca] : T(0);
      Yb[rr][cc] = (gr < row1 && cb < r) ? Y[gr * ldy + cb] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < GROWS; ++rr) {
      TACC a[4], b[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) { a[e] = Ya[rr][ty * 4 + e]; b[e] = Yb[rr][tx * 4 + e]; }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
    if (++run == GFLUSH) {
      run = 0;
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) { acc64[x][y] += (double)acc[x][y]; acc[x][y] = TACC(0); }
    }
  }
  double* out = partial + ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * (GB * GB);
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y)
      out[(ty * 4 + x) * GB + tx * 4 + y] = acc64[x][y] + (double)acc[x][y];
}

// G[a][b] = G[b][a] = sum over chunks (fixed order) of the partial blocks.
__global__ void gram_reduce_kernel(int r, int nb, int npairs, int nchunks,
                                   const double* __restrict__ partial, double* __restrict__ G) {
  const int64_t total = (int64_t)npairs * GB * GB;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / (GB * GB));
    const int w = (int)(e % (GB * GB));
    int bi, bj;
    pair_of(p, nb, &bi, &bj);
    const int a = bi * GB + w / GB, b = bj * GB + w % GB;
    if (a >= r || b >= r) continue;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += partial[((int64_t)c * npairs + p) * (GB * GB) + w];
    G[(int64_t)a * r + b] = s;
    G[(int64_t)b * r + a] = s;
  }
}

// Right-looking Cholesky G = L L^T of an r x r symmetric matrix in one CTA.  L
// (lower, row-major, zero above the diagonal) is built in place in `L` after
// copying G.  Pivot deflation: a pivot whose remaining mass is at most
// tau * G_kk (the column is linearly dependent on the previous ones to the
// accuracy of G) is marked dead: L[k][k] = 1 and L[i][k] = 0 below it, so
// Y L^-T leaves that column as a negligible residual, to be replaced by a
// fresh random direction (fill_dead_columns).  A NaN or infinite pivot
// records DEV_NOT_SPD.
__global__ void __launch_bounds__(1024)
cholesky_kernel(int r, const double* __restrict__ G, double* __restrict__ L, int* __restrict__ dead,
                double tau, int* status) {
  __shared__ double piv;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < r * r; e += nt) L[e] = G[e];
  __syncthreads();
  for (int k = 0; k < r; ++k) {
    if (tid == 0) {
      const double d = L[(int64_t)k * r + k];
      const double g0 = G[(int64_t)k * r + k];
      int is_dead = 0;
      if (!isfinite(d) || !isfinite(g0)) { is_dead = 1; dev_set_status(status, DEV_NOT_SPD); }
      else if (!(d > tau * g0) || !(d > 0.0)) is_dead = 1;
      dead[k] = is_dead;
      piv = is_dead ? 0.0 : sqrt(d);
      L[(int64_t)k * r + k] = is_dead ? 1.0 : piv;
    }
    __syncthreads();
    const double inv = piv > 0.0 ? 1.0 / piv : 0.0;
    for (int i = k + 1 + tid; i < r; i += nt) L[(int64_t)i * r + k] *= inv;
    __syncthreads();
    if (piv > 0.0) {
      const int T = r - k - 1;
      for (int idx = tid; idx < T * T; idx += nt) {
        const int ii = idx / T, jj = idx % T;
        if (jj > ii) continue;
        const int i = k + 1 + ii, j = k + 1 + jj;
        L[(int64_t)i * r + j] -= L[(int64_t)i * r + k] * L[(int64_t)j * r + k];
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < r * r; e += nt) {
    const int i = e / r, j = e % r;
    if (j > i) L[e] = 0.0;
  }
}

// Any pivot dead in the second sweep means the panel stayed rank deficient
// after its dead columns were replaced: report it.
__global__ void check_dead_kernel(int r, const int* __restrict__ dead, int* status) {
  for (int k = threadIdx.x; k < r; k += blockDim.x)
    if (dead[k]) dev_set_status(status, DEV_NOT_SPD);
}

// X = L^-1 by forward substitution, one warp per column j; Rinv = X^T (upper),
// also written in the panel type TOUT.
template <typename TOUT>
__global__ void __launch_bounds__(32)
trilinv_kernel(int r, const double* __restrict__ L, double* __restrict__ Rinv,
               TOUT* __restrict__ Rinv_t) {
  extern __shared__ double xs[];
  const int j = blockIdx.x, lane = threadIdx.x;
  for (int i = lane; i < r; i += 32) xs[i] = 0.0;
  __syncwarp();
  if (lane == 0) xs[j] = 1.0 / L[(int64_t)j * r + j];
  __syncwarp();
  for (int i = j + 1; i < r; ++i) {
    double s = 0.0;
    for (int l = j + lane; l < i; l += 32) s += L[(int64_t)i * r + l] * xs[l];
    s = warp_sum(s);
    if (lane == 0) xs[i] = -s / L[(int64_t)i * r + i];
    __syncwarp();
  }
  for (int i = lane; i < r; i += 32) {
    Rinv[(int64_t)j * r + i] = xs[i];  // Rinv[j][i] = X[i][j]
    Rinv_t[(int64_t)j * r + i] = (TOUT)xs[i];
  }
}

// R = R2 R1 with R1 = L1^T, R2 = L2^T (both upper triangular).  A dead pivot l
// of the first sweep carries no part of Y (its column was a negligible
// residual), so row l of R1 counts as zero.
__global__ void rprod_kernel(int r, const double* __restrict__ L1, const int* __restrict__ dead1,
                             const double* __restrict__ L2, double* __restrict__ R) {
  const int64_t total = (int64_t)r * r;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / r), j = (int)(e % r);
    double s = 0.0;
    for (int l = i; l <= j; ++l)
      if (!dead1[l]) s += L2[(int64_t)l * r + i] * L1[(int64_t)j * r + l];
    R[e] = j >= i ? s : 0.0;
  }
}

int gram_chunks_for(int64_t M, int npairs) {
  int64_t want = cdiv(2 * 152, npairs);
  int64_t maxc = cdiv(M, GFLUSH * GROWS);
  int64_t c = want < maxc ? want : maxc;
  return (int)(c < 1 ? 1 : c);
}

template <typename T>
rsvd_status gram(int64_t M, int r, const T* Y, int64_t ldy, const OrthWs& ws, cudaStream_t stream) {
  const int nb = (int)cdiv(r, GB);
  const int npairs = nb * (nb + 1) / 2;
  int nchunks = gram_chunks_for(M, npairs);
  if (nchunks > ws.gram_chunks) nchunks = (int)ws.gram_chunks;
  const int64_t rows_per = round_up(cdiv(M, nchunks), GROWS);
  nchunks = (int)cdiv(M, rows_per);
  if (nchunks < 1) nchunks = 1;
  using TACC = T;
  gram_partial_kernel<T, TACC><<<dim3(npairs, nchunks), 256, 0, stream>>>(M, r, Y, ldy, rows_per, nb,
                                                                          ws.gram_partial);
  RSVD_CUDA(after_launch());
  gram_reduce_kernel<<<(int)cdiv((int64_t)npairs * GB * GB, 256), 256, 0, stream>>>(
      r, nb, npairs, nchunks, ws.gram_partial, ws.G);
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

template <typename T>
rsvd_status chol_inv(int r, const OrthWs& ws, double* L, int* dead, cudaStream_t stream) {
  cholesky_kernel<<<1, 1024, 0, stream>>>(r, ws.G, L, dead, pivot_tau<T>(), ws.status);
  RSVD_CUDA(after_launch());
  trilinv_kernel<T><<<r, 32, r * sizeof(double), stream>>>(r, L, ws.Rinv, static_cast<T*>(ws.Rinv_t));
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

}  // namespace

size_t orth_ws_bytes(int64_t M, int r, int dtype) {
  Sizer s;
  const size_t esz = dtype == RSVD_F64 ? 8 : 4;
  const int nb = (int)cdiv(r, GB);
  const int npairs = nb * (nb + 1) / 2;
  const int chunks = gram_chunks_for(M, npairs);
  s.take<double>((size_t)r * r * 4);
  s.take<int>((size_t)2 * r);
  s.take<char>((size_t)r * r * esz);
  s.take<double>((size_t)chunks * npairs * GB * GB);
  s.take<char>((size_t)M * round_up(r, 4) * esz);
  s.take<int>(4);
  return s.used + 256;
}

OrthWs orth_ws_carve(Carver& c, int64_t M, int r, int dtype) {
  OrthWs w;
  const size_t esz = dtype == RSVD_F64 ? 8 : 4;
  const int nb = (int)cdiv(r, GB);
  const int npairs = nb * (nb + 1) / 2;
  const int chunks = gram_chunks_for(M, npairs);
  double* base = c.take<double>((size_t)r * r * 4);
  if (base) { w.G = base; w.L1 = base + r * r; w.L2 = base + 2 * r * r; w.Rinv = base + 3 * r * r; }
  int* dd = c.take<int>((size_t)2 * r);
  if (dd) { w.dead1 = dd; w.dead2 = dd + r; }
  w.Rinv_t = c.take<char>((size_t)r * r * esz);
  w.gram_partial = c.take<double>((size_t)chunks * npairs * GB * GB);
  w.gram_chunks = chunks;
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
  RSVD_TRY(chol_inv<T>(r, ws, ws.L1, ws.dead1, stream));
  RSVD_TRY(simt_gemm<T>(M, r, r, Y, ldy, false, Rt, r, Q1, ws.ld_tmp, false, 1, r, nullptr, stream));
  RSVD_TRY(fill_dead_columns(M, r, ws.dead1, Q1, ws.ld_tmp, sizeof(T) == 8 ? RSVD_F64 : RSVD_F32,
                             kDeadFillSeed, stream));
  // sweep 2
  RSVD_TRY(gram<T>(M, r, Q1, ws.ld_tmp, ws, stream));
  RSVD_TRY(chol_inv<T>(r, ws, ws.L2, ws.dead2, stream));
  check_dead_kernel<<<1, 256, 0, stream>>>(r, ws.dead2, ws.status);
  RSVD_CUDA(after_launch());
  RSVD_TRY(simt_gemm<T>(M, r, r, Q1, ws.ld_tmp, false, Rt, r, Q, ldq, false, 1, r, nullptr, stream));
  if (R) {
    rprod_kernel<<<(int)cdiv((int64_t)r * r, 256), 256, 0, stream>>>(r, ws.L1, ws.dead1, ws.L2, R);
    RSVD_CUDA(after_launch());
  }
  return RSVD_OK;
}

template rsvd_status orth_panel<float>(int64_t, int, const float*, int64_t, float*, int64_t, double*,
                                       const OrthWs&, cudaStream_t);
template rsvd_status orth_panel<double>(int64_t, int, const double*, int64_t, double*, int64_t,
                                        double*, const OrthWs&, cudaStream_t);

}  // namespace rsvd
