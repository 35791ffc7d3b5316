// Block-wise SIMT products (FP32 FFMA / FP64 DFMA): the plain-precision
// A-passes of Section 2.1 steps 2 and 5 and Eq. (3), and the small panel
// products of the orthonormalisation and of the lift (Section 2.1 step 7).
//
// C[M x N] (+)= op(A)[M x K] * B[K x N], all row-major.  op(A) = A reads
// A[i*lda + k]; op(A) = A^T reads A[k*lda + i] (A stored K x M), which is how
// the transposed A-pass reads the same row-major tiles of A without a copy.
// The K range is cut into chunks (the tile columns / rows of Section 2.3);
// each chunk writes its own partial product and a second kernel adds the
// partials in chunk order, so results do not depend on scheduling.
//
// Tiling: 128 x 128 output tile per 256-thread CTA, 8 x 8 outputs per thread
// as two 4-wide halves in each direction (conflict-free shared-memory
// broadcasts), K step 8, double-buffered shared memory.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int BM = 128, BN = 128, BK = 8, PAD = 4, THREADS = 256;

template <typename T, bool VEC>
__device__ __forceinline__ void load4(const T* p, bool ok, int64_t valid, T out[4]) {
  if (VEC && ok && valid >= 4) {
    if constexpr (sizeof(T) == 4) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(p));
      out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else {
      const double2 v0 = __ldg(reinterpret_cast<const double2*>(p));
      const double2 v1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
      out[0] = v0.x; out[1] = v0.y; out[2] = v1.x; out[3] = v1.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < 4; ++e) out[e] = (ok && e < valid) ? p[e] : T(0);
  }
}

template <typename T, bool TRANS_A, bool VEC>
__global__ void __launch_bounds__(THREADS)
simt_gemm_kernel(int64_t M, int64_t N, int64_t K, const T* __restrict__ A, int64_t lda,
                 const T* __restrict__ B, int64_t ldb, T* __restrict__ C, int64_t ldc,
                 int64_t c_split_stride, int64_t kchunk, int accumulate) {
  __shared__ __align__(16) T As[2][BK][BM + PAD];
  __shared__ __align__(16) T Bs[2][BK][BN + PAD];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t i0 = (int64_t)blockIdx.x * BM;
  const int64_t j0 = (int64_t)blockIdx.y * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);
  T* Cz = C + (int64_t)blockIdx.z * c_split_stride;

  T acc[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 8; ++b) acc[a][b] = T(0);

  // Per-thread load coordinates.
  // A, not transposed: row ar = tid/2 of the tile, k offset ak = (tid&1)*4.
  // A transposed and B: k row = tid/32, 4 consecutive columns at (tid&31)*4.
  const int ar = tid >> 1, ak = (tid & 1) * 4;
  const int lr = tid >> 5, lc = (tid & 31) * 4;

  T ra[4], rb[4];
  auto load_tiles = [&](int64_t k0) {
    if constexpr (!TRANS_A) {
      const int64_t gi = i0 + ar, gk = k0 + ak;
      load4<T, VEC>(A + gi * lda + gk, gi < M && gk < kend, kend - gk, ra);
    } else {
      const int64_t gk = k0 + lr, gi = i0 + lc;
      load4<T, VEC>(A + gk * lda + gi, gk < kend && gi < M, M - gi, ra);
    }
    const int64_t gk = k0 + lr, gj = j0 + lc;
    load4<T, VEC>(B + gk * ldb + gj, gk < kend && gj < N, N - gj, rb);
  };
  auto store_tiles = [&](int buf) {
    if constexpr (!TRANS_A) {
#pragma unroll
      for (int e = 0; e < 4; ++e) As[buf][ak + e][ar] = ra[e];
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) As[buf][lr][lc + e] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) Bs[buf][lr][lc + e] = rb[e];
  };

  if (kbeg < kend) {
    load_tiles(kbeg);
    store_tiles(0);
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) load_tiles(k0 + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        T a[8], b[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          a[e] = As[buf][kk][ty * 4 + e];
          a[4 + e] = As[buf][kk][64 + ty * 4 + e];
          b[e] = Bs[buf][kk][tx * 4 + e];
          b[4 + e] = Bs[buf][kk][64 + tx * 4 + e];
        }
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 8; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
      }
      if (more) {
        store_tiles(buf ^ 1);
        __syncthreads();
        buf ^= 1;
      }
    }
  }

#pragma unroll
  for (int x = 0; x < 8; ++x) {
    const int64_t gi = i0 + (x < 4 ? ty * 4 + x : 64 + ty * 4 + (x - 4));
    if (gi >= M) continue;
#pragma unroll
    for (int y = 0; y < 8; ++y) {
      const int64_t gj = j0 + (y < 4 ? tx * 4 + y : 64 + tx * 4 + (y - 4));
      if (gj >= N) continue;
      T* dst = Cz + gi * ldc + gj;
      *dst = accumulate ? *dst + acc[x][y] : acc[x][y];
    }
  }
}

// out[i, j] (+)= sum_z P[z][i, j] in increasing z.
template <typename T>
__global__ void __launch_bounds__(256)
reduce_partials_kernel(int64_t M, int64_t N, int nsplit, const T* __restrict__ P, int64_t ldp,
                       int64_t pstride, T* __restrict__ out, int64_t ldo, int accumulate) {
  const int64_t total = M * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N, j = e - i * N;
    T s = T(0);
    for (int z = 0; z < nsplit; ++z) s += P[z * pstride + i * ldp + j];
    T* dst = out + i * ldo + j;
    *dst = accumulate ? *dst + s : s;
  }
}

// The same sum with 4 consecutive columns per thread (16-byte loads) and the
// partials of up to 16 splits loaded together; the order of the additions
// (split 0, 1, 2, ...) is the same as above.
// One warp per output float4: lane l adds the partials of a contiguous block
// of splits in order, then the 32 lane sums are combined by a fixed butterfly,
// so the result does not depend on scheduling.
__global__ void reduce_partials_warp_vec4_kernel(int64_t M, int64_t N4, int nsplit, const float4* __restrict__ P,
                                                 int64_t ldp4, int64_t pstride4, float4* __restrict__ out,
                                                 int64_t ldo4, int accumulate) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= M * N4) return;  // whole warps only (blockDim is a multiple of 32)
  const int64_t i = w / N4, j = w - i * N4;
  const float4* src = P + i * ldp4 + j;
  const int per = (nsplit + 31) / 32;
  const int z0 = lane * per, z1 = min(nsplit, z0 + per);
  float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int z = z0; z < z1; ++z) {
    const float4 v = src[(int64_t)z * pstride4];
    s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
    s.z += __shfl_xor_sync(0xffffffffu, s.z, o);
    s.w += __shfl_xor_sync(0xffffffffu, s.w, o);
  }
  if (lane == 0) {
    float4* dst = out + i * ldo4 + j;
    if (accumulate) {
      const float4 d = *dst;
      s.x += d.x; s.y += d.y; s.z += d.z; s.w += d.w;
    }
    *dst = s;
  }
}

template <int U>
__global__ void reduce_partials_vec4_kernel(int64_t M, int64_t N4, int nsplit, const float4* __restrict__ P,
                                            int64_t ldp4, int64_t pstride4, float4* __restrict__ out, int64_t ldo4,
                                            int accumulate) {
  const int64_t total = M * N4;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / N4, j = e - i * N4;
    const float4* src = P + i * ldp4 + j;
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    // U partials loaded together (one wait per U), then added in order
    for (int z0 = 0; z0 < nsplit; z0 += U) {
      float4 v[U];
#pragma unroll
      for (int u = 0; u < U; ++u)  // past the last split: the last one again (in cache, not added)
        v[u] = src[(int64_t)min(z0 + u, nsplit - 1) * pstride4];
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (z0 + u < nsplit) { s.x += v[u].x; s.y += v[u].y; s.z += v[u].z; s.w += v[u].w; }
    }
    float4* dst = out + i * ldo4 + j;
    if (accumulate) {
      const float4 d = *dst;
      s.x += d.x; s.y += d.y; s.z += d.z; s.w += d.w;
    }
    *dst = s;
  }
}

}  // namespace

template <typename T>
rsvd_status simt_gemm(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, bool transA,
                      const T* B, int64_t ldb, T* C, int64_t ldc, bool accumulate, int nsplit,
                      int64_t kchunk, T* partial, cudaStream_t stream) {
  if (M <= 0 || N <= 0) return RSVD_OK;
  if (nsplit < 1) nsplit = 1;
  if (nsplit == 1) kchunk = K > 0 ? K : 1;
  if (nsplit > 1 && !partial) return fail(RSVD_ERR_INVALID_ARG, "simt_gemm: partial buffer missing");
  kchunk = round_up(kchunk, 4);
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) && aligned16(A) && aligned16(B);
  dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), (unsigned)nsplit);
  if (grid.y > 65535 || grid.z > 65535) return fail(RSVD_ERR_INVALID_ARG, "simt_gemm: grid too large");
  T* dst = nsplit > 1 ? partial : C;
  const int64_t ldd = nsplit > 1 ? N : ldc;
  const int64_t stride = nsplit > 1 ? M * N : 0;
  const int acc = nsplit > 1 ? 0 : (accumulate ? 1 : 0);
#define RSVD_LAUNCH(TR, VE)                                                              \
  simt_gemm_kernel<T, TR, VE><<<grid, THREADS, 0, stream>>>(M, N, K, A, lda, B, ldb, dst, \
                                                            ldd, stride, kchunk, acc)
  if (transA) {
    if (vec) RSVD_LAUNCH(true, true); else RSVD_LAUNCH(true, false);
  } else {
    if (vec) RSVD_LAUNCH(false, true); else RSVD_LAUNCH(false, false);
  }
#undef RSVD_LAUNCH
  RSVD_CUDA(after_launch());
  if (nsplit > 1) {
    int64_t blocks = cdiv(M * N, 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    reduce_partials_kernel<T><<<(int)blocks, 256, 0, stream>>>(M, N, nsplit, partial, N, M * N, C,
                                                                ldc, accumulate ? 1 : 0);
    RSVD_CUDA(after_launch());
  }
  return RSVD_OK;
}

template <typename T>
rsvd_status simt_gemm_partials(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, bool transA,
                               const T* B, int64_t ldb, int nsplit, int64_t kchunk, T* partial,
                               cudaStream_t stream) {
  if (M <= 0 || N <= 0) return RSVD_OK;
  if (nsplit < 1 || kchunk % 4 != 0 || !partial)
    return fail(RSVD_ERR_INVALID_ARG, "simt_gemm_partials: bad split");
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) && aligned16(A) && aligned16(B);
  dim3 grid((unsigned)cdiv(M, BM), (unsigned)cdiv(N, BN), (unsigned)nsplit);
  if (grid.y > 65535 || grid.z > 65535) return fail(RSVD_ERR_INVALID_ARG, "simt_gemm_partials: grid too large");
#define RSVD_LAUNCH(TR, VE)                                                                      \
  simt_gemm_kernel<T, TR, VE><<<grid, THREADS, 0, stream>>>(M, N, K, A, lda, B, ldb, partial, N, \
                                                            M * N, kchunk, 0)
  if (transA) {
    if (vec) RSVD_LAUNCH(true, true); else RSVD_LAUNCH(true, false);
  } else {
    if (vec) RSVD_LAUNCH(false, true); else RSVD_LAUNCH(false, false);
  }
#undef RSVD_LAUNCH
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

template rsvd_status simt_gemm_partials<float>(int64_t, int64_t, int64_t, const float*, int64_t, bool, const float*,
                                               int64_t, int, int64_t, float*, cudaStream_t);
template rsvd_status simt_gemm_partials<double>(int64_t, int64_t, int64_t, const double*, int64_t, bool,
                                                const double*, int64_t, int, int64_t, double*, cudaStream_t);

template <typename T>
rsvd_status reduce_partials(int64_t M, int64_t N, int nsplit, const T* P, int64_t ldp, int64_t pstride, T* out,
                            int64_t ldo, bool accumulate, cudaStream_t stream) {
  if (M * N == 0) return RSVD_OK;
  if constexpr (std::is_same<T, float>::value) {
    const bool vec = N % 4 == 0 && ldp % 4 == 0 && pstride % 4 == 0 && ldo % 4 == 0 && aligned16(P) && aligned16(out);
    if (vec && nsplit >= 64 && M * (N / 4) <= 152 * 64) {
      // few outputs, many partials (the Grams of tall panels): a warp per float4
      const int64_t warps = M * (N / 4);
      reduce_partials_warp_vec4_kernel<<<(int)cdiv(warps * 32, 256), 256, 0, stream>>>(
          M, N / 4, nsplit, reinterpret_cast<const float4*>(P), ldp / 4, pstride / 4, reinterpret_cast<float4*>(out),
          ldo / 4, accumulate ? 1 : 0);
      RSVD_CUDA(after_launch());
      return RSVD_OK;
    }
    if (vec) {
      // a thread per output float4 where the grid allows (one round of loads)
      int64_t blocks = cdiv(M * (N / 4), 256);
      if (blocks > 152 * 64) blocks = 152 * 64;
      // as many partials in flight as there are splits (up to 16)
      const float4* P4 = reinterpret_cast<const float4*>(P);
      float4* o4 = reinterpret_cast<float4*>(out);
      const int acc = accumulate ? 1 : 0;
      if (nsplit <= 4)
        reduce_partials_vec4_kernel<4><<<(int)blocks, 256, 0, stream>>>(M, N / 4, nsplit, P4, ldp / 4, pstride / 4, o4,
                                                                       ldo / 4, acc);
      else if (nsplit <= 8)
        reduce_partials_vec4_kernel<8><<<(int)blocks, 256, 0, stream>>>(M, N / 4, nsplit, P4, ldp / 4, pstride / 4, o4,
                                                                       ldo / 4, acc);
      else
        reduce_partials_vec4_kernel<16><<<(int)blocks, 256, 0, stream>>>(M, N / 4, nsplit, P4, ldp / 4, pstride / 4,
                                                                        o4, ldo / 4, acc);
      RSVD_CUDA(after_launch());
      return RSVD_OK;
    }
  }
  int64_t blocks = cdiv(M * N, 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  reduce_partials_kernel<T><<<(int)blocks, 256, 0, stream>>>(M, N, nsplit, P, ldp, pstride, out, ldo,
                                                              accumulate ? 1 : 0);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

template rsvd_status reduce_partials<float>(int64_t, int64_t, int, const float*, int64_t, int64_t, float*,
                                            int64_t, bool, cudaStream_t);
template rsvd_status reduce_partials<double>(int64_t, int64_t, int, const double*, int64_t, int64_t, double*,
                                             int64_t, bool, cudaStream_t);

template rsvd_status simt_gemm<float>(int64_t, int64_t, int64_t, const float*, int64_t, bool,
                                      const float*, int64_t, float*, int64_t, bool, int, int64_t,
                                      float*, cudaStream_t);
template rsvd_status simt_gemm<double>(int64_t, int64_t, int64_t, const double*, int64_t, bool,
                                       const double*, int64_t, double*, int64_t, bool, int, int64_t,
                                       double*, cudaStream_t);

}  // namespace rsvd
