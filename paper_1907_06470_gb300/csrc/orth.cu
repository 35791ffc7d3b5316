// Section 2.1 steps 3-4: orthonormal basis Q_r of the sketch Y by CholeskyQR2.
//
//   G = Y^T Y          chunk partials (simt_gemm) added in FP64
//   G = L L^T,         Cholesky and triangular inverse together, one CTA, in
//   Rinv = L^-T        the panel's type (chol_inv_fused_kernel)
//   Q1 = Y Rinv        panel product in the panel's precision (simt_gemm)
// and the same once more on Q1 (Fukaya, Nakatsukasa, Yanagisawa, Yamamoto,
// "CholeskyQR2", 2014), which restores orthogonality to working precision
// whenever the first Cholesky succeeds.  R = R2 R1 is formed (in FP64) on
// request.
//
// Rank deficiency: a Cholesky pivot that has lost all but a tau fraction of its
// column's mass is deflated and the column of Q1 replaced by a unit random
// vector (from the library's Gaussian stream with a fixed seed), which the
// second sweep orthonormalises against the rest; R then has a zero row there.
//
// Gram accumulation: products are summed in the panel's type over chunks of
// 256 rows (more for panels over 2^19 rows; the SIMT GEMM, one partial per
// chunk) and the chunk partials are added in FP64 in a fixed order.
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

// Pivot deflation: a pivot whose remaining mass d is at most tau * G_kk (the
// column is linearly dependent on the previous ones to the accuracy of G) is
// marked dead: L[k][k] = 1 and L[i][k] = 0 below it, so Y L^-T leaves that
// column as a negligible residual, to be replaced by a fresh random direction
// (fill_dead_columns).  A NaN or infinite pivot records DEV_NOT_SPD.

// Any pivot dead in the second sweep means the panel stayed rank deficient
// after its dead columns were replaced: report it.
__global__ void check_dead_kernel(int r, const int* __restrict__ dead, int* status) {
  for (int k = threadIdx.x; k < r; k += blockDim.x)
    if (dead[k]) dev_set_status(status, DEV_NOT_SPD);
}


// Cholesky and triangular inverse in one CTA: the working matrices in shared
// memory when they fit, else in a global scratch (L2 resident at these sizes;
// the algorithm is the same).
//
// Cholesky, blocked right-looking with kCholB = 16 columns per panel: warp 0
// factors the diagonal block column by column in registers (the pivot test
// and deflation above), each thread solves one row of the panel below it, and
// the trailing lower triangle takes the panel's rank-16 update -- with
// lookahead: warp 0 updates and factors the next diagonal block while the
// other warps update the rest, two barriers per panel.  Rows are stored with
// a stride that is a multiple of 16 bytes, so a row segment of the panel moves
// in 16-byte loads (4 for FP32, 8 for FP64); the padding columns are zero.
//
// Inverse X = L^-1 blocked by block diagonals: the diagonal blocks are inverted
// by one warp each; then for d = 1, 2, ... every block X_ij with i - j = d is
// X_ij = -X_ii (sum_{j<=t<i} L_it X_tj), whose right-hand side only needs
// blocks of smaller d.  Each thread forms a 2 x 4 tile of a block (two rows of
// L against a 16-byte row segment of X per term).  Rinv_t = X^T (upper) and L
// are written to global memory as their entries become final.
constexpr int kCholB = 16;
constexpr int kFusedThreads = 512;
constexpr size_t kFusedSmemMax = 220 * 1024;

template <typename T>
__host__ __device__ inline int fused_ld(int r) {
  constexpr int e = 16 / (int)sizeof(T);
  return (r + e - 1) / e * e + e;
}

// bytes of the matrices the fused kernel keeps in shared or global memory:
// A (L), X (L^-1) and the block scratch S
// slices of the block scratch S: the inverse splits the terms of a block over
// up to this many slices when a block diagonal has few blocks
template <typename T>
__host__ __device__ constexpr int inv_slices() { return 64 / (int)sizeof(T); }

template <typename T>
__host__ __device__ inline size_t fused_big_bytes(int r) {
  const int nb = (r + kCholB - 1) / kCholB;
  const int ns = nb > inv_slices<T>() ? nb : inv_slices<T>();
  return 2 * (size_t)r * fused_ld<T>(r) * sizeof(T) + (size_t)ns * kCholB * kCholB * sizeof(T) + 64;
}

// bytes of the per-pivot vectors (always in shared memory)
template <typename T>
__host__ __device__ inline size_t fused_small_bytes(int r) {
  return ((3 * (size_t)r * sizeof(T) + 15) & ~(size_t)15);
}

template <typename T>
__host__ __device__ inline size_t fused_smem_bytes(int r) {
  return fused_small_bytes<T>(r) + fused_big_bytes<T>(r);
}

template <typename T>
struct alignas(16) Vec16 {
  static constexpr int E = 16 / (int)sizeof(T);
  T v[E];
};

template <typename T>
__device__ __forceinline__ Vec16<T> ld16(const T* p) { return *reinterpret_cast<const Vec16<T>*>(p); }

// L_kk = sqrt(d) and its reciprocal (0, 0 for a dead pivot).  FP32: from the
// hardware reciprocal square root refined by one Newton step (within about an
// ulp; the Gram itself carries errors far above that); FP64: IEEE sqrt and
// division.
__device__ __forceinline__ void pivot_sqrt(float d, int is_dead, float& piv, float& inv) {
  float y = rsqrtf(d);
  y = y * fmaf(-0.5f * d, y * y, 1.5f);
  inv = is_dead ? 0.f : y;
  piv = is_dead ? 0.f : d * y;
}
__device__ __forceinline__ void pivot_sqrt(double d, int is_dead, double& piv, double& inv) {
  piv = is_dead ? 0.0 : sqrt(d);
  inv = is_dead ? 0.0 : 1.0 / piv;
}

// Warp 0: Cholesky of the diagonal block at p (w <= 16 columns) in place in A,
// with its pivot test and the reciprocals of its diagonal.
template <typename T>
__device__ __forceinline__ void factor_diag_block(T* A, int lda, int p, int w, const T* gdiag, T* invs, T* xdg,
                                                  int* dead, int* status, int lane, T* Lout, int r) {
  constexpr int NB = kCholB;
  constexpr int E = Vec16<T>::E;
  constexpr int NV = NB / E;

  // Diagonal block in registers: lane i (< w) holds row p+i.  Every lane
  // forms each pivot from the broadcast diagonal entry, so no lane waits
  // on another beyond the shuffles.
  T row[NB];
  if (lane < w) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const Vec16<T> x = ld16(A + (p + lane) * lda + p + E * v);
#pragma unroll
      for (int e = 0; e < E; ++e) row[E * v + e] = x.v[e];
    }
  } else {
#pragma unroll
    for (int t = 0; t < NB; ++t) row[t] = T(0);
  }
  const T fl = lane < w ? gdiag[p + lane] : T(0);
  int my_dead = 0;
  T my_inv = T(0);
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (k < w) {
      const T d = __shfl_sync(0xffffffffu, row[k], k);
      const T floor_k = __shfl_sync(0xffffffffu, fl, k);
      int is_dead = 0;
      if (!isfinite(d) || !isfinite(floor_k)) is_dead = 2;
      else if (!(d > floor_k) || !(d > T(0))) is_dead = 1;
      T piv, inv;
      pivot_sqrt(d, is_dead, piv, inv);
      if (lane == k) {
        my_dead = is_dead;
        my_inv = inv;
        row[k] = is_dead ? T(1) : piv;
      }
      if (lane > k) row[k] *= inv;                 // L_{lane,k}
#pragma unroll
      for (int j = k + 1; j < NB; ++j) {
        const T ljk = __shfl_sync(0xffffffffu, row[k], j);  // L_{j,k}
        if (lane >= j) row[j] -= row[k] * ljk;
      }
    }
  }
  if (lane < w) {
    dead[p + lane] = my_dead ? 1 : 0;
    if (my_dead == 2) dev_set_status(status, DEV_NOT_SPD);
    invs[p + lane] = my_inv;
    xdg[p + lane] = my_dead ? T(1) : my_inv;
#pragma unroll
    for (int t = 0; t < NB; ++t)
      if (t <= lane) {
        A[(p + lane) * lda + p + t] = row[t];
        Lout[(int64_t)(p + lane) * r + p + t] = row[t];
      }
  }
}

template <typename T>
__global__ void __launch_bounds__(kFusedThreads, 1)
chol_inv_fused_kernel(int r, const double* __restrict__ G, T* __restrict__ Lout, int* __restrict__ dead,
                      double tau, int* status, T* __restrict__ Rinv_t, int ldr, unsigned char* gscratch) {
  extern __shared__ __align__(16) unsigned char fsm[];
  constexpr int NB = kCholB;
  constexpr int E = Vec16<T>::E;       // entries per 16 bytes
  constexpr int NV = NB / E;           // 16-byte vectors per panel row segment
  const int lda = fused_ld<T>(r);
  const int nb = (r + NB - 1) / NB;
  T* gdiag = reinterpret_cast<T*>(fsm);  // tau * G_kk
  T* invs = gdiag + r;                   // 1 / L_kk (0 for a dead pivot)
  T* xdg = invs + r;                     // X_kk = 1 / L_kk (1 for a dead pivot)
  unsigned char* big = gscratch ? gscratch : fsm + fused_small_bytes<T>(r);
  T* A = reinterpret_cast<T*>(big);      // r x lda, lower triangle used
  T* X = A + (size_t)r * lda;            // r x lda: L^-1
  T* S = X + (size_t)r * lda;            // nb blocks of NB^2 scratch
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nt >> 5;

  // G (L2 resident, just written): eight loads in flight per thread per round;
  // the padding columns r .. lda-1 are zeroed (they enter masked products)
  for (int k = tid; k < r; k += nt) gdiag[k] = (T)(tau * G[(int64_t)k * r + k]);
  {
    const int rr = r * r;
    constexpr int U = 8;
    for (int e0 = tid; e0 < rr; e0 += U * nt) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = e0 + u * nt < rr ? G[e0 + u * nt] : 0.0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * nt;
        if (e < rr) {
          const int i = e / r;
          A[i * lda + (e - i * r)] = (T)v[u];
        }
      }
    }
    const int pad = lda - r;
    for (int e = tid; e < r * pad; e += nt) A[(e / pad) * lda + r + e % pad] = T(0);
    // the zero triangles of the outputs: L above its diagonal, Rinv_t below
    for (int i = warp; i < r; i += nwarps)
      for (int j = lane; j < r; j += 32) {
        if (j > i) Lout[(int64_t)i * r + j] = T(0);
        else if (j < i) Rinv_t[(int64_t)i * ldr + j] = T(0);
      }
  }
  __syncthreads();

  // Panels with lookahead: while warps 1.. apply panel p's rank-16 update to
  // the trailing matrix, warp 0 applies it to the next diagonal block alone and
  // factors that block, so the diagonal factorisations overlap the updates.
  // (p = -NB: only the first diagonal block, so that its code exists once)
  for (int p = -NB; p < r; p += NB) {
    const int pe = min(p + NB, r), w = pe - p;
    // Panel rows below the block: x L_D^T = a, one thread per row, x in registers.
    for (int i = p < 0 ? r : pe + tid; i < r; i += nt) {
      T x[NB];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const Vec16<T> y = ld16(A + i * lda + p + E * v);
#pragma unroll
        for (int e = 0; e < E; ++e) x[E * v + e] = y.v[e];
      }
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (k < w) {
          T v = x[k];
#pragma unroll
          for (int t = 0; t < k; ++t) v -= x[t] * A[(p + k) * lda + p + t];
          x[k] = v * invs[p + k];
        }
      }
#pragma unroll
      for (int t = 0; t < NB; ++t)
        if (t < w) {
          A[i * lda + p + t] = x[t];
          Lout[(int64_t)i * r + p + t] = x[t];
        }
    }
    __syncthreads();
    const int pn = pe, wn = min(NB, r - pn);  // the next panel (wn <= 0: none); w == NB when it exists
    if (warp == 0) {
      if (wn > 0) {
        // next diagonal block: lane l updates row pn + l (entries pn .. pn + l)
        if (p >= 0 && lane < wn) {
          T li[NB];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Vec16<T> y = ld16(A + (pn + lane) * lda + p + E * v);
#pragma unroll
            for (int e = 0; e < E; ++e) li[E * v + e] = y.v[e];
          }
          for (int jj = 0; jj <= lane; ++jj) {
            T sum = A[(pn + lane) * lda + pn + jj];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              const Vec16<T> y = ld16(A + (pn + jj) * lda + p + E * v);
#pragma unroll
              for (int e = 0; e < E; ++e) sum -= li[E * v + e] * y.v[e];
            }
            A[(pn + lane) * lda + pn + jj] = sum;
          }
        }
        __syncwarp();
        factor_diag_block(A, lda, pn, wn, gdiag, invs, xdg, dead, status, lane, Lout, r);
      }
    } else {
      // Trailing lower triangle without the next diagonal block: lane owns
      // column j, warps 1.. the rows i >= max(j, next block end) in pairs.
      const int wi = warp - 1, nw = nwarps - 1;
      for (int j = p < 0 ? r : pe + lane; j < r; j += 32) {
        T lj[NB];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const Vec16<T> y = ld16(A + j * lda + p + E * v);
#pragma unroll
          for (int e = 0; e < E; ++e) lj[E * v + e] = E * v + e < w ? y.v[e] : T(0);
        }
        const int i_lo = j < pn + wn ? pn + wn : j;
        int i = pe + wi;
        if (i < i_lo) i += ((i_lo - i + nw - 1) / nw) * nw;  // first of the warp's rows >= i_lo
        for (; i + nw < r; i += 2 * nw) {
          const int i2 = i + nw;
          T s1 = A[i * lda + j], s2 = A[i2 * lda + j];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Vec16<T> y1 = ld16(A + i * lda + p + E * v), y2 = ld16(A + i2 * lda + p + E * v);
#pragma unroll
            for (int e = 0; e < E; ++e) {
              s1 -= y1.v[e] * lj[E * v + e];
              s2 -= y2.v[e] * lj[E * v + e];
            }
          }
          A[i * lda + j] = s1;
          A[i2 * lda + j] = s2;
        }
        if (i < r) {
          T s1 = A[i * lda + j];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Vec16<T> y1 = ld16(A + i * lda + p + E * v);
#pragma unroll
            for (int e = 0; e < E; ++e) s1 -= y1.v[e] * lj[E * v + e];
          }
          A[i * lda + j] = s1;
        }
      }
    }
    __syncthreads();
  }
  // diagonal blocks: X_bb = L_bb^-1, lane c of warp b solves column c of block b
  for (int b = warp; b < nb; b += nwarps) {
    const int o = b * NB, w = min(NB, r - o);
    if (lane < w) {
      T col[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i < w) {
          // row i of the block (entries past w are padding or later columns, masked by t < i < w)
          T li[NB];
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const Vec16<T> y = ld16(A + (o + i) * lda + o + E * v);
#pragma unroll
            for (int e = 0; e < E; ++e) li[E * v + e] = y.v[e];
          }
          T x = i == lane ? T(1) : T(0);
#pragma unroll
          for (int t = 0; t < NB; ++t)
            if (t >= lane && t < i) x -= li[t] * col[t];
          col[i] = i < lane ? T(0) : x * xdg[o + i];
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < w) {
          X[(o + i) * lda + o + lane] = col[i];
          if (i >= lane) Rinv_t[(int64_t)(o + lane) * ldr + o + i] = col[i];  // Rinv_t[j][i] = X[i][j]
        }
    }
  }
  __syncthreads();
  // off-diagonal blocks by block diagonal d: S_ij = sum_{j<=t<i} L_it X_tj, then
  // X_ij = -X_ii S_ij.  L is read from A (unchanged since the factorisation);
  // X_tj for t in blocks j .. i-1 lies on block diagonals below d, finished in
  // earlier steps.  Work unit: block q (bi = q + d, bj = q), a slice of its d
  // sub-blocks of terms (when the diagonal has few blocks), and a 2 x 4 tile
  // (rows 2 ti, 2 ti + 1; columns 4 tj .. 4 tj + 3).  The slices' partial sums
  // are added in slice order.
  for (int d = 1; d < nb; ++d) {
    const int nblk = nb - d;
    int ks = inv_slices<T>() / nblk;
    ks = ks < 1 ? 1 : (ks > d ? d : ks);
    const int db = (d + ks - 1) / ks;          // sub-blocks per slice
    ks = (d + db - 1) / db;
    for (int u = tid; u < nblk * ks * 32; u += nt) {
      const int q = u / (ks * 32), sl = (u >> 5) % ks, tl = u & 31;
      const int bi = q + d, bj = q;
      const int pi = 2 * (tl >> 2), pj = 4 * (tl & 3);
      const int i0 = bi * NB + pi, j0 = bj * NB + pj;
      const bool r0 = i0 < r, r1 = i0 + 1 < r;
      const int t0 = (bj + sl * db) * NB, t1 = (bj + min(d, (sl + 1) * db)) * NB;
      T acc[2][4] = {};
#pragma unroll 4
      for (int t = t0; t < t1; ++t) {
        const T a0 = r0 ? A[i0 * lda + t] : T(0);
        const T a1 = r1 ? A[(i0 + 1) * lda + t] : T(0);
        T xv[4];
#pragma unroll
        for (int h = 0; h < 4 / E; ++h) {
          const Vec16<T> y = ld16(X + t * lda + j0 + E * h);
#pragma unroll
          for (int e = 0; e < E; ++e) xv[E * h + e] = y.v[e];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          acc[0][c] += a0 * xv[c];
          acc[1][c] += a1 * xv[c];
        }
      }
      T* Sq = S + (q * ks + sl) * NB * NB;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        Sq[pi * NB + pj + c] = acc[0][c];
        Sq[(pi + 1) * NB + pj + c] = acc[1][c];
      }
    }
    __syncthreads();
    if (ks > 1) {
      for (int e = tid; e < nblk * NB * NB; e += nt) {
        const int q = e / (NB * NB), o = e % (NB * NB);
        T* Sq = S + q * ks * NB * NB + o;
        T sum = Sq[0];
        for (int sl = 1; sl < ks; ++sl) sum += Sq[sl * NB * NB];
        Sq[0] = sum;
      }
      __syncthreads();
    }
    for (int u = tid; u < nblk * 32; u += nt) {
      const int q = u >> 5, tl = u & 31;
      const int bi = q + d, bj = q;
      const int pi = 2 * (tl >> 2), pj = 4 * (tl & 3);
      const int i0 = bi * NB + pi, j0 = bj * NB + pj;
      const T* Sq = S + q * ks * NB * NB;
      T acc[2][4] = {};
#pragma unroll
      for (int s2 = 0; s2 < NB; ++s2) {
        const int t = bi * NB + s2;   // X_ii is zero above its diagonal and outside r
        const T x0 = i0 < r && t < r ? X[i0 * lda + t] : T(0);
        const T x1 = i0 + 1 < r && t < r ? X[(i0 + 1) * lda + t] : T(0);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const T sv = Sq[s2 * NB + pj + c];
          acc[0][c] -= x0 * sv;
          acc[1][c] -= x1 * sv;
        }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (i0 < r) {
          X[i0 * lda + j0 + c] = acc[0][c];
          Rinv_t[(int64_t)(j0 + c) * ldr + i0] = acc[0][c];
        }
        if (i0 + 1 < r) {
          X[(i0 + 1) * lda + j0 + c] = acc[1][c];
          Rinv_t[(int64_t)(j0 + c) * ldr + i0 + 1] = acc[1][c];
        }
      }
    }
    __syncthreads();
  }
}

// R = R2 R1 with R1 = L1^T, R2 = L2^T (both upper triangular).  A dead pivot l
// of the first sweep carries no part of Y (its column was a negligible
// residual), so row l of R1 counts as zero.
// One warp per entry (i, j): lanes over l in [i, j], their partial sums added
// by a fixed shuffle tree (FP64, every SM busy: the sum is short, the FP64
// latency long); entries below the diagonal are zero.
template <typename T1, typename T2>
__global__ void rprod_kernel(int r, const T1* __restrict__ L1, const int* __restrict__ dead1,
                             const T2* __restrict__ L2, double* __restrict__ R) {
  const int lane = threadIdx.x & 31;
  const int64_t total = (int64_t)r * r;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < total; e += nw) {
    const int i = (int)(e / r), j = (int)(e % r);
    double s = 0.0;
    for (int l = i + lane; l <= j; l += 32)
      if (!dead1[l]) s += (double)L2[(int64_t)l * r + i] * (double)L1[(int64_t)j * r + l];
    s = warp_sum(s);
    if (lane == 0) R[e] = j >= i ? s : 0.0;
  }
}

int rprod_blocks(int r) {
  const int64_t b = cdiv((int64_t)r * r * 32, 256);
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

// Rows per partial Gram: each partial is a sum of gram_chunk(M) products in
// the panel's type -- 256 rows, or more for panels over 2^19 rows so that at
// most about kGramMaxChunks partials are stored -- and the partials are added
// in FP64 in a fixed order (gram_sum_partials_kernel).
constexpr int64_t kGramChunk = 256;
constexpr int64_t kGramMaxChunks = 2048;

int64_t gram_chunk(int64_t M) {
  const int64_t c = round_up(cdiv(M, kGramMaxChunks), kGramChunk);
  return c > kGramChunk ? c : kGramChunk;
}

int64_t gram_chunks(int64_t M) { return cdiv(M, gram_chunk(M)); }

// One warp per upper-triangle entry (a, b): lane l adds chunks l, l+32, ... in
// order, then the 32 lane sums are combined by a fixed shuffle tree, so the
// result does not depend on scheduling.
template <typename T>
__global__ void gram_sum_partials_kernel(int r, int64_t nchunks, const T* __restrict__ P, double* __restrict__ G) {
  const int64_t rr = (int64_t)r * r;
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t e = w0; e < rr; e += nw) {
    const int a = (int)(e / r), b = (int)(e % r);
    if (b < a) continue;
    double s = 0.0;
    for (int64_t c = lane; c < nchunks; c += 32) s += (double)P[c * rr + e];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      G[(int64_t)a * r + b] = s;
      G[(int64_t)b * r + a] = s;
    }
  }
}

// G = Y^T Y: the SIMT GEMM forms one r x r partial per chunk of kGramChunk rows
// (op(A) = Y^T), and the partials are added in FP64.
template <typename T>
rsvd_status gram(int64_t M, int r, const T* Y, int64_t ldy, const OrthWs& ws, cudaStream_t stream) {
  const int64_t nchunks = gram_chunks(M);
  T* P = static_cast<T*>(ws.gram_partial);
  RSVD_TRY(simt_gemm_partials<T>(r, r, M, Y, ldy, true, Y, ldy, (int)nchunks, gram_chunk(M), P, stream));
  int64_t blocks = cdiv((int64_t)r * r * 32, 256);
  if (blocks > 152 * 32) blocks = 152 * 32;
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

// Arithmetic of the two factorisations: the panel's type.  The Gram of an FP32
// panel carries FP32 accuracy (FP32 products summed in chunks), and
// CholeskyQR in working precision u leaves Q1 orthogonal to about
// u cond(Y)^2, which the second sweep restores to u whenever cond(Y) is below
// about u^-1/2 (about 4e3 in FP32) -- the range finder's panels Y = A Z with
// orthonormal Z have cond(Y) near sigma_1 / sigma_r of A.  Pivots below
// tau = 1e-5 of their diagonal (the deflation floor of FP32 panels) are
// deflated either way.  The second sweep factors Q1^T Q1, close to the identity.

// Cholesky + triangular inverse in the arithmetic T of the factorisation
// (FP64 for FP64 panels, FP32 for FP32 panels), which is also the panel type
// that receives Rinv.
template <typename T>
rsvd_status chol_inv(int r, const OrthWs& ws, T* L, int* dead, double tau, cudaStream_t stream) {
  const size_t fused = fused_smem_bytes<T>(r);
  const bool in_smem = fused <= kFusedSmemMax;
  if (!in_smem && !(ws.chol_scratch && ws.chol_scratch_bytes >= fused_big_bytes<T>(r)))
    return fail(RSVD_ERR_INVALID_ARG, "orth: workspace lacks the factorisation scratch for this r");
  static bool fattr = false;
  if (!fattr) {
    RSVD_CUDA(cudaFuncSetAttribute(chol_inv_fused_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)kFusedSmemMax));
    fattr = true;
  }
  chol_inv_fused_kernel<T><<<1, kFusedThreads, in_smem ? fused : fused_small_bytes<T>(r), stream>>>(
      r, ws.G, L, dead, tau, ws.status, static_cast<T*>(ws.Rinv_t), ws.ld_rt,
      in_smem ? nullptr : static_cast<unsigned char*>(ws.chol_scratch));
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

}  // namespace

namespace {
// global scratch for the blocked factorisation when r is too large for shared
// memory (sized for FP64, which covers FP32)
size_t chol_scratch_bytes(int r) {
  if (fused_smem_bytes<double>(r) <= kFusedSmemMax) return 0;
  return fused_big_bytes<double>(r);
}

size_t tc_orth_ws(int64_t M, int r) {
  const size_t g = tc_apass_ws_bytes(M, r, r, 1, RSVD_PREC_BF16X3, 0, 0);
  const size_t p = tc_apass_ws_bytes(M, r, r, 0, RSVD_PREC_BF16X3, 0, 0);
  return g > p ? g : p;
}
bool tc_orth_ok(int r, int dtype, bool tc) { return tc && dtype == RSVD_F32 && r <= 512; }

// G = widened lower triangle of the FP32 Gram, mirrored
__global__ void widen_gram_kernel(int r, const float* __restrict__ g32, double* __restrict__ G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x) {
    const int i = e / r, j = e % r;
    G[e] = (double)(i >= j ? g32[i * r + j] : g32[j * r + i]);
  }
}
}  // namespace

size_t orth_ws_bytes(int64_t M, int r, int dtype, bool tc) {
  Sizer s;
  const size_t esz = dtype == RSVD_F64 ? 8 : 4;
  s.take<double>((size_t)r * r * 3);
  s.take<int>((size_t)2 * r);
  s.take<char>((size_t)r * round_up(r, 4) * esz);
  s.take<char>((size_t)gram_chunks(M) * r * r * esz);
  s.take<char>((size_t)M * round_up(r, 4) * esz);
  s.take<int>(4);
  if (tc_orth_ok(r, dtype, tc)) {
    s.take<float>((size_t)r * r);
    s.take<char>(tc_orth_ws(M, r));
  }
  s.take<char>(chol_scratch_bytes(r));
  return s.used + 256;
}

OrthWs orth_ws_carve(Carver& c, int64_t M, int r, int dtype, bool tc) {
  OrthWs w;
  const size_t esz = dtype == RSVD_F64 ? 8 : 4;
  double* base = c.take<double>((size_t)r * r * 3);
  if (base) { w.G = base; w.L1 = base + r * r; w.L2 = base + 2 * r * r; }
  int* dd = c.take<int>((size_t)2 * r);
  if (dd) { w.dead1 = dd; w.dead2 = dd + r; }
  w.ld_rt = (int)round_up(r, 4);
  w.Rinv_t = c.take<char>((size_t)r * w.ld_rt * esz);
  w.gram_partial = c.take<char>((size_t)gram_chunks(M) * r * r * esz);
  w.gram_chunks = gram_chunks(M);
  w.ld_tmp = round_up(r, 4);
  w.tmp = c.take<char>((size_t)M * w.ld_tmp * esz);
  w.status = c.take<int>(4);
  if (tc_orth_ok(r, dtype, tc)) {
    w.gram32 = c.take<float>((size_t)r * r);
    w.tc_ws_bytes = tc_orth_ws(M, r);
    w.tc_ws = c.take<char>(w.tc_ws_bytes);
  }
  w.chol_scratch_bytes = chol_scratch_bytes(r);
  w.chol_scratch = w.chol_scratch_bytes ? c.take<char>(w.chol_scratch_bytes) : nullptr;
  return w;
}

// Tensor-core Gram G = Y^T Y (split BF16, FP32 accumulation), widened to FP64.
rsvd_status gram_tc(int64_t M, int r, const float* Y, int64_t ldy, const OrthWs& ws, cudaStream_t stream) {
  rsvd_matrix A = {};
  A.kind = RSVD_DENSE; A.dtype = RSVD_F32; A.location = RSVD_ON_DEVICE;
  A.m = M; A.n = r; A.data = Y; A.ld = ldy;
  RSVD_TRY(tc_apass_from_f32(A, 1, RSVD_PREC_BF16X3, r, Y, ldy, ws.gram32, r, 0, 0, ws.tc_ws, ws.tc_ws_bytes,
                             ws.status, stream));
  widen_gram_kernel<<<(int)cdiv((int64_t)r * r, 256), 256, 0, stream>>>(r, ws.gram32, ws.G);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

// Tensor-core panel product Q = Y Rinv (split BF16).
rsvd_status panel_times_tc(int64_t M, int r, const float* Y, int64_t ldy, const float* Rt, float* Q, int64_t ldq,
                           const OrthWs& ws, cudaStream_t stream) {
  rsvd_matrix A = {};
  A.kind = RSVD_DENSE; A.dtype = RSVD_F32; A.location = RSVD_ON_DEVICE;
  A.m = M; A.n = r; A.data = Y; A.ld = ldy;
  return tc_apass_from_f32(A, 0, RSVD_PREC_BF16X3, r, Rt, ws.ld_rt, Q, ldq, 0, 0, ws.tc_ws, ws.tc_ws_bytes, ws.status,
                           stream);
}

template <typename T>
rsvd_status orth_panel(int64_t M, int r, const T* Y, int64_t ldy, T* Q, int64_t ldq, double* R,
                       const OrthWs& ws, cudaStream_t stream, bool tc, bool one_sweep) {
  // one sweep: Q = Y R1^-1 spans the columns of Y (dead pivots refilled) but is
  // orthonormal only to about eps cond(Y)^2 -- enough where only the span is
  // used; the second sweep restores orthonormality to rounding
  if (R) one_sweep = false;
  T* Q1 = one_sweep ? Q : static_cast<T*>(ws.tmp);
  const int64_t ld1 = one_sweep ? ldq : ws.ld_tmp;
  const T* Rt = static_cast<const T*>(ws.Rinv_t);
  if constexpr (std::is_same<T, float>::value) {
    if (tc && ws.tc_ws && ldy % 4 == 0 && ldq % 4 == 0 && aligned16(Y) && aligned16(Q)) {
      // the same two sweeps with the Grams and panel products on the tensor cores
      RSVD_TRY(gram_tc(M, r, Y, ldy, ws, stream));
      float* L1 = reinterpret_cast<float*>(ws.L1);
      RSVD_TRY(chol_inv<float>(r, ws, L1, ws.dead1, pivot_tau<float>(), stream));
      RSVD_TRY(panel_times_tc(M, r, Y, ldy, Rt, Q1, ld1, ws, stream));
      RSVD_TRY(fill_dead_columns(M, r, ws.dead1, Q1, ld1, RSVD_F32, kDeadFillSeed, stream));
      if (one_sweep) return RSVD_OK;
      RSVD_TRY(gram_tc(M, r, Q1, ws.ld_tmp, ws, stream));
      float* L2 = reinterpret_cast<float*>(ws.L2);
      RSVD_TRY(chol_inv<float>(r, ws, L2, ws.dead2, pivot_tau<float>(), stream));
      check_dead_kernel<<<1, 256, 0, stream>>>(r, ws.dead2, ws.status);
      RSVD_CUDA(after_launch());
      RSVD_TRY(panel_times_tc(M, r, Q1, ws.ld_tmp, Rt, Q, ldq, ws, stream));
      if (R) {
        rprod_kernel<float, float><<<rprod_blocks(r), 256, 0, stream>>>(r, L1, ws.dead1, L2, R);
        RSVD_CUDA(after_launch());
      }
      return RSVD_OK;
    }
  }
  // sweep 1 (dead pivots: the panel is rank deficient to the Gram's accuracy;
  // their columns of Q1 are replaced by unit random directions)
  RSVD_TRY(gram<T>(M, r, Y, ldy, ws, stream));
  T* L1 = reinterpret_cast<T*>(ws.L1);
  RSVD_TRY(chol_inv<T>(r, ws, L1, ws.dead1, pivot_tau<T>(), stream));
  RSVD_TRY(simt_gemm<T>(M, r, r, Y, ldy, false, Rt, ws.ld_rt, Q1, ld1, false, 1, r, nullptr, stream));
  RSVD_TRY(fill_dead_columns(M, r, ws.dead1, Q1, ld1, sizeof(T) == 8 ? RSVD_F64 : RSVD_F32, kDeadFillSeed, stream));
  if (one_sweep) return RSVD_OK;
  // sweep 2
  RSVD_TRY(gram<T>(M, r, Q1, ws.ld_tmp, ws, stream));
  T* L2 = reinterpret_cast<T*>(ws.L2);
  RSVD_TRY(chol_inv<T>(r, ws, L2, ws.dead2, pivot_tau<T>(), stream));
  check_dead_kernel<<<1, 256, 0, stream>>>(r, ws.dead2, ws.status);
  RSVD_CUDA(after_launch());
  RSVD_TRY(simt_gemm<T>(M, r, r, Q1, ws.ld_tmp, false, Rt, ws.ld_rt, Q, ldq, false, 1, r, nullptr, stream));
  if (R) {
    rprod_kernel<T, T><<<rprod_blocks(r), 256, 0, stream>>>(r, L1, ws.dead1, L2, R);
    RSVD_CUDA(after_launch());
  }
  return RSVD_OK;
}

template rsvd_status orth_panel<float>(int64_t, int, const float*, int64_t, float*, int64_t, double*,
                                       const OrthWs&, cudaStream_t, bool, bool);
template rsvd_status orth_panel<double>(int64_t, int, const double*, int64_t, double*, int64_t,
                                        double*, const OrthWs&, cudaStream_t, bool, bool);

}  // namespace rsvd
