// Section 2.1 step 6: SVD of the small factor by one-sided (Hestenes) Jacobi
// in FP64, with the relative stopping test of Demmel & Veselic (1992).
//
// Three phases for square inputs with 8 <= r <= 512: FP32 sweeps to FP32
// convergence (one CTA with shared memory for r <= 160, a 16-CTA cluster over
// global memory above); Newton-Schulz steps that make the accumulated FP32
// rotation orthogonal in FP64, applied to M; FP64 sweeps to FP64
// convergence, which then take few sweeps -- or none, for callers whose
// inputs carry far less than FP32 accuracy (only the outputs are formed).
// Other shapes run the FP64 sweeps from the start.
//
// M (rows x r, column-major, rows >= 1) is driven to orthogonal columns by
// plane rotations from the right, M W = U diag(sigma).  The sweep order is round-robin: in
// each of the r'-1 rounds of a sweep (r' = r rounded up to even) the r'/2
// column pairs are disjoint, so one CTA rotates each pair concurrently.
// FP64 throughput on one GB300 SM is low (about 2 DFMA per clock), so the
// pairs of a round are spread over the warps of a thread-block cluster of up to
// 16 CTAs (one warp per pair) and rounds are separated by the hardware cluster
// barrier.  Columns are read and written through L2 (ld/st .cg) because another
// SM may have rotated them in the previous round.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

__device__ __forceinline__ int rr_column(int pos, int round, int rp) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (rp - 1);
}

// All threads of all CTAs of the cluster: release this CTA's memory operations
// and wait until every thread of the cluster has arrived.
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Rotation that annihilates g in the 2 x 2 Gram [[a, g], [g, b]] of a column
// pair: t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / (2 g),
// c = (1 + t^2)^-1/2, s = c t.  FP64 instructions are costly on this GPU
// (about 2 FMA per clock per SM), so only what must hold to double precision is
// formed in FP64: the angle itself may be off in the 8th digit (the sweep then
// leaves |g| ~ 1e-7 |g| instead of 0, far below what the next sweep needs),
// but c^2 + s^2 = c^2 (1 + t^2) must be 1 to rounding, so t is taken in FP32
// (exact in FP64, 1 + t^2 exact) and c is refined from the FP32 estimate by two
// Newton steps for (1 + t^2)^-1/2.  |zeta| stays below about 1e27 here (both
// columns are above the rounding-level floor), so no FP32 overflow.
__device__ __forceinline__ void jacobi_rotation(double a, double b, double g, double& c, double& s) {
  const float z = (float)((b - a) / (2.0 * g));
  const float tf = fabsf(z) > 1e18f ? 0.5f / z : copysignf(1.f, z) / (fabsf(z) + sqrtf(fmaf(z, z, 1.f)));
  const double t = (double)tf;
  const double x = fma(t, t, 1.0);
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  c = y;
  s = y * t;
}

// Outputs of a finished one-sided Jacobi: column norms sigma_c = ||M_c||, a
// stable descending order, U_c = M_c / sigma_c and W_c.  Signs: each pair of
// columns (U_c, W_c) is turned so that the entry of W_c largest in magnitude
// (the first such) is positive, so that the output does not depend on the
// path the sweeps took.  M (rows x r) and W (r x r) are column-major and read
// through L2.

// Warp-collective: the norm of column c and its sign (valid in every lane).
__device__ __forceinline__ void column_norm_sign(int rows, int r, int c, const double* __restrict__ M,
                                                 const double* __restrict__ W, int lane, double& nrm, double& sgn) {
  double s2 = 0.0;
  for (int i = lane; i < rows; i += 32) { const double x = __ldcg(&M[(int64_t)c * rows + i]); s2 = fma(x, x, s2); }
  s2 = warp_sum_d(s2);
  double wm = -1.0;
  int wi = r;
  for (int i = lane; i < r; i += 32) {
    const double x = fabs(__ldcg(&W[(int64_t)c * r + i]));
    if (x > wm) { wm = x; wi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double om = __shfl_xor_sync(0xffffffffu, wm, o);
    const int oi = __shfl_xor_sync(0xffffffffu, wi, o);
    if (om > wm || (om == wm && oi < wi)) { wm = om; wi = oi; }
  }
  nrm = sqrt(s2);
  sgn = wi < r && __ldcg(&W[(int64_t)c * r + wi]) < 0.0 ? -1.0 : 1.0;
}

// Warp-collective: the rank of column c among the norms nrms[0..r) (ties by
// index) and its normalised outputs.
__device__ __forceinline__ void write_column(int rows, int r, int c, const double* __restrict__ M,
                                             const double* __restrict__ W, const double* nrms, double sgn, int lane,
                                             double* __restrict__ sigma, double* __restrict__ Uout,
                                             double* __restrict__ Wout) {
  const double sc = nrms[c];
  int cnt = 0;
  for (int d = lane; d < r; d += 32) cnt += (nrms[d] > sc) || (nrms[d] == sc && d < c);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  const int rank = cnt;
  if (lane == 0) sigma[rank] = sc;
  const double inv = sc > 0.0 ? sgn / sc : 0.0;
  for (int i = lane; i < rows; i += 32) Uout[(int64_t)i * r + rank] = __ldcg(&M[(int64_t)c * rows + i]) * inv;
  for (int i = lane; i < r; i += 32) Wout[(int64_t)i * r + rank] = sgn * __ldcg(&W[(int64_t)c * r + i]);
}

// All warps of one CTA (sh: 2 r doubles of shared memory).
__device__ void form_outputs(int rows, int r, const double* __restrict__ M, const double* __restrict__ W,
                             double* sh, double* __restrict__ sigma, double* __restrict__ Uout,
                             double* __restrict__ Wout) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, warps = blockDim.x >> 5;
  double* sgn = sh + r;
  for (int c = warp; c < r; c += warps) {
    double nv, sg;
    column_norm_sign(rows, r, c, M, W, lane, nv, sg);
    if (lane == 0) { sh[c] = nv; sgn[c] = sg; }
  }
  __syncthreads();
  for (int c = warp; c < r; c += warps) write_column(rows, r, c, M, W, sh, sgn[c], lane, sigma, Uout, Wout);
}

// Finish only: the columns of M W were orthogonalised before (the FP32
// phase), so no sweeps run and the outputs are formed straight from M and W,
// one warp per column over many SMs (FP64 arithmetic is slow on one SM): the
// norms and signs (into nrm_sgn, 2 r doubles), then, after the launch
// boundary, the ranks and the outputs.
constexpr int kFinishWarps = 8;

__global__ void __launch_bounds__(32 * kFinishWarps)
jacobi_finish_norms_kernel(int rows, int r, const double* __restrict__ M, const double* __restrict__ W,
                           double* __restrict__ nrm_sgn, int* sweeps_out) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * kFinishWarps + (threadIdx.x >> 5);
  if (blockIdx.x == 0 && threadIdx.x == 0) *sweeps_out = 0;
  if (c >= r) return;
  double nv, sg;
  column_norm_sign(rows, r, c, M, W, lane, nv, sg);
  if (lane == 0) { nrm_sgn[c] = nv; nrm_sgn[r + c] = sg; }
}

__global__ void __launch_bounds__(32 * kFinishWarps)
jacobi_finish_out_kernel(int rows, int r, const double* __restrict__ M, const double* __restrict__ W,
                         const double* __restrict__ nrm_sgn, double* sigma, double* Uout, double* Wout) {
  const int lane = threadIdx.x & 31;
  const int c = blockIdx.x * kFinishWarps + (threadIdx.x >> 5);
  if (c >= r) return;
  write_column(rows, r, c, M, W, nrm_sgn, nrm_sgn[r + c], lane, sigma, Uout, Wout);
}

// One cluster of up to 16 CTAs; warp w of CTA b owns pair slot b*warps + w of
// every round.  Rounds are separated by the hardware cluster barrier; the
// columns live in global memory and are accessed through L2 (.cg).
constexpr int kMaxPerLane = 8;  // rows <= 256: column values held in registers
constexpr int kClusterCheckSmem = 200 * 1024;

__global__ void jacobi_cluster_kernel(int rows, int r, const double* __restrict__ Min,
                                      const double* __restrict__ W0, double* M, double* W, int* rotated,
                                      int* sweeps_out, int* status, double* sigma, double* Uout, double* Wout,
                                      int check, double tol, int max_sweeps) {
  __shared__ double red[32];
  extern __shared__ double sh[];  // check pass: M staged (rows x r) + column norms (r); end: sigma_c, signs
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, warps = nthr >> 5;
  const int ncta = gridDim.x;
  const int rp = r + (r & 1);
  const int npairs = rp / 2;
  const int64_t mm = (int64_t)rows * r;
  const int64_t ww = (int64_t)r * r;
  const int64_t gtid = (int64_t)blockIdx.x * nthr + tid, gstride = (int64_t)ncta * nthr;

  for (int64_t e = gtid; e < mm; e += gstride) __stcg(&M[e], Min[e]);
  for (int64_t e = gtid; e < ww; e += gstride) __stcg(&W[e], W0 ? W0[e] : ((e / r) == (e % r) ? 1.0 : 0.0));
  // Frobenius norm of the input (every CTA computes it), for the rounding-level
  // column test of the sweeps
  double f = 0.0;
  for (int64_t e = tid; e < mm; e += nthr) f += Min[e] * Min[e];
  f = warp_sum_d(f);
  if (lane == 0) red[warp] = f;
  __syncthreads();
  double fro2 = 0.0;
  for (int i = 0; i < warps; ++i) fro2 += red[i];
  const double eps = 2.220446049250313e-16;
  const double big = (double)(rows > r ? rows : r);
  const double zero2 = (big * eps) * (big * eps) * fro2;
  const double tol2 = tol * tol;
  cluster_sync_all();

  int sweep = 0;
  bool converged = false;
  const int s = blockIdx.x * warps + warp;  // this warp's pair slot
  for (; sweep < max_sweeps; ++sweep) {
    // this warp's rotations in the sweep (one flag and one maximum per warp,
    // published before the barrier that ends the sweep's last round)
    bool my_rot = false;
    float my_mrel = 0.f;
    for (int round = 0; round < rp - 1; ++round) {
      if (s < npairs) {
        int p = rr_column(s, round, rp), q = rr_column(rp - 1 - s, round, rp);
        if (p < r && q < r) {
          if (p > q) { const int t = p; p = q; q = t; }
          double* mp = M + (int64_t)p * rows;
          double* mq = M + (int64_t)q * rows;
          double xv[kMaxPerLane], yv[kMaxPerLane];
          double a = 0.0, b = 0.0, g = 0.0;
          const bool in_regs = rows <= 32 * kMaxPerLane;
#pragma unroll
          for (int t = 0; t < kMaxPerLane; ++t) {
            const int i = lane + 32 * t;
            const bool ok = in_regs && i < rows;
            xv[t] = ok ? __ldcg(&mp[i]) : 0.0;
            yv[t] = ok ? __ldcg(&mq[i]) : 0.0;
          }
          // FP64 instructions are expensive here (about 2 FMA per clock per SM):
          // skip the slots no lane of the warp holds
#pragma unroll
          for (int t = 0; t < kMaxPerLane; ++t)
            if (in_regs && 32 * t < rows) {
              a = fma(xv[t], xv[t], a); b = fma(yv[t], yv[t], b); g = fma(xv[t], yv[t], g);
            }
          double* wp = W + (int64_t)p * r;
          double* wq = W + (int64_t)q * r;
          double wu[kMaxPerLane], wv[kMaxPerLane];
          const bool w_in_regs = r <= 32 * kMaxPerLane;
#pragma unroll
          for (int t = 0; t < kMaxPerLane; ++t) {
            const int i = lane + 32 * t;
            const bool ok = w_in_regs && i < r;
            wu[t] = ok ? __ldcg(&wp[i]) : 0.0;
            wv[t] = ok ? __ldcg(&wq[i]) : 0.0;
          }
          if (!in_regs)
            for (int i = lane; i < rows; i += 32) {
              const double x = __ldcg(&mp[i]), y = __ldcg(&mq[i]);
              a = fma(x, x, a); b = fma(y, y, b); g = fma(x, y, g);
            }
          a = warp_sum_d(a);
          b = warp_sum_d(b);
          g = warp_sum_d(g);
          if (g * g > tol2 * (a * b) && a > zero2 && b > zero2) {
            my_rot = true;
            my_mrel = fmaxf(my_mrel, fabsf((float)g) * rsqrtf((float)a) * rsqrtf((float)b));
            double c, sn;
            jacobi_rotation(a, b, g, c, sn);
            if (in_regs) {
#pragma unroll
              for (int u = 0; u < kMaxPerLane; ++u) {
                const int i = lane + 32 * u;
                if (i < rows) {
                  __stcg(&mp[i], c * xv[u] - sn * yv[u]);
                  __stcg(&mq[i], sn * xv[u] + c * yv[u]);
                }
              }
            } else {
              for (int i = lane; i < rows; i += 32) {
                const double x = __ldcg(&mp[i]), y = __ldcg(&mq[i]);
                __stcg(&mp[i], c * x - sn * y);
                __stcg(&mq[i], sn * x + c * y);
              }
            }
            if (w_in_regs) {
#pragma unroll
              for (int u = 0; u < kMaxPerLane; ++u) {
                const int i = lane + 32 * u;
                if (i < r) {
                  __stcg(&wp[i], c * wu[u] - sn * wv[u]);
                  __stcg(&wq[i], sn * wu[u] + c * wv[u]);
                }
              }
            } else {
              for (int i = lane; i < r; i += 32) {
                const double u = __ldcg(&wp[i]), v = __ldcg(&wq[i]);
                __stcg(&wp[i], c * u - sn * v);
                __stcg(&wq[i], sn * u + c * v);
              }
            }
          }
        }
      }
      if (round == rp - 2 && lane == 0 && my_rot) {
        atomicMax(&rotated[2 * kJacobiMaxSweeps + sweep], __float_as_int(my_mrel));
        __stcg(&rotated[sweep], 1);
      }
      cluster_sync_all();
    }
    if (__ldcg(&rotated[sweep]) == 0) { converged = true; break; }
    // Jacobi converges quadratically near the end: when the largest relative
    // off-diagonal rotated in this sweep, squared, is below the tolerance, the
    // next sweep would most likely find nothing -- check instead of sweeping.
    const float mrel = __int_as_float(__ldcg(&rotated[2 * kJacobiMaxSweeps + sweep]));
    if (check && (double)mrel * (double)mrel <= tol) {
      // Check pass instead of one more sweep: every pair's test on the
      // current columns (a sweep that found no pair to rotate would leave the
      // columns as they are, so this is the same stopping test), as dot
      // products from a staged copy of M, spread over all warps of the cluster.
      double* Ms = sh;
      double* nrm = sh + mm;
      for (int64_t e = tid; e < mm; e += nthr) Ms[e] = __ldcg(&M[e]);
      __syncthreads();
      for (int c = warp; c < r; c += warps) {
        double s2 = 0.0;
        for (int i = lane; i < rows; i += 32) s2 = fma(Ms[(int64_t)c * rows + i], Ms[(int64_t)c * rows + i], s2);
        s2 = warp_sum_d(s2);
        if (lane == 0) nrm[c] = s2;
      }
      __syncthreads();
      bool bad = false;
      for (int p = blockIdx.x * warps + warp; p < r; p += ncta * warps) {
        const double* xp = Ms + (int64_t)p * rows;
        const double a = nrm[p];
        for (int q = p + 1 + lane; q < r; q += 32) {
          const double* xq = Ms + (int64_t)q * rows;
          double g0 = 0.0, g1 = 0.0, g2 = 0.0, g3 = 0.0;
          int i = 0;
          for (; i + 4 <= rows; i += 4) {
            g0 = fma(xp[i], xq[i], g0);
            g1 = fma(xp[i + 1], xq[i + 1], g1);
            g2 = fma(xp[i + 2], xq[i + 2], g2);
            g3 = fma(xp[i + 3], xq[i + 3], g3);
          }
          for (; i < rows; ++i) g0 = fma(xp[i], xq[i], g0);
          const double g = (g0 + g1) + (g2 + g3);
          const double b = nrm[q];
          if (g * g > tol2 * (a * b) && a > zero2 && b > zero2) bad = true;
        }
      }
      if (__any_sync(0xffffffffu, bad) && lane == 0) __stcg(&rotated[kJacobiMaxSweeps + sweep], 1);
      cluster_sync_all();
      if (__ldcg(&rotated[kJacobiMaxSweeps + sweep]) == 0) { converged = true; break; }
    }
  }
  if (blockIdx.x != 0) return;
  if (!converged) dev_set_status(status, DEV_NO_CONVERGE);
  if (tid == 0) *sweeps_out = sweep + (converged ? 1 : 0);
  form_outputs(rows, r, M, W, sh, sigma, Uout, Wout);
}

// FP32 first phase for r too large for one CTA's shared memory: the same
// round-robin sweeps as jacobi_cluster_kernel in FP32, with the columns of M
// (rows x r) and W (r x r) in global memory.  It stops once the largest
// relative off-diagonal rotated in a sweep, squared, is below r eps32 (the next
// sweep would leave only FP32 rounding; the FP64 phase finishes from there).
constexpr int kF32ClusterPerLane = 16;  // rows <= 512 in registers

__global__ void jacobi_cluster_f32_kernel(int rows, int r, const double* __restrict__ Min, float* M, float* W,
                                          int* rotated, int* sweeps_out) {
  __shared__ float red[32];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, warps = nthr >> 5;
  const int rp = r + (r & 1);
  const int npairs = rp / 2;
  const int64_t mm = (int64_t)rows * r;
  const int64_t ww = (int64_t)r * r;
  const int64_t gtid = (int64_t)blockIdx.x * nthr + tid, gstride = (int64_t)gridDim.x * nthr;
  for (int64_t e = gtid; e < mm; e += gstride) __stcg(&M[e], (float)Min[e]);
  for (int64_t e = gtid; e < ww; e += gstride) __stcg(&W[e], (e / r) == (e % r) ? 1.f : 0.f);
  float f = 0.f;
  for (int64_t e = tid; e < mm; e += nthr) { const float v = (float)Min[e]; f = fmaf(v, v, f); }
  f = warp_sum(f);
  if (lane == 0) red[warp] = f;
  __syncthreads();
  float fro2 = 0.f;
  for (int i = 0; i < warps; ++i) fro2 += red[i];
  const float eps = 1.1920929e-7f;
  const float big = (float)(rows > r ? rows : r);
  const float zero2 = (big * eps) * (big * eps) * fro2;
  const float tol = (float)r * eps;
  cluster_sync_all();

  int sweep = 0;
  const int s = blockIdx.x * warps + warp;  // this warp's pair slot
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    bool my_rot = false;
    float my_mrel = 0.f;
    for (int round = 0; round < rp - 1; ++round) {
      if (s < npairs) {
        int p = rr_column(s, round, rp), q = rr_column(rp - 1 - s, round, rp);
        if (p < r && q < r) {
          if (p > q) { const int t = p; p = q; q = t; }
          float* mp = M + (int64_t)p * rows;
          float* mq = M + (int64_t)q * rows;
          float* wp = W + (int64_t)p * r;
          float* wq = W + (int64_t)q * r;
          float xv[kF32ClusterPerLane], yv[kF32ClusterPerLane];
          float a = 0.f, b = 0.f, g = 0.f;
#pragma unroll
          for (int t = 0; t < kF32ClusterPerLane; ++t) {
            const int i = lane + 32 * t;
            xv[t] = i < rows ? __ldcg(&mp[i]) : 0.f;
            yv[t] = i < rows ? __ldcg(&mq[i]) : 0.f;
            a = fmaf(xv[t], xv[t], a); b = fmaf(yv[t], yv[t], b); g = fmaf(xv[t], yv[t], g);
          }
          a = warp_sum(a); b = warp_sum(b); g = warp_sum(g);
          if (fabsf(g) > tol * sqrtf(a * b) && a > zero2 && b > zero2) {
            my_rot = true;
            my_mrel = fmaxf(my_mrel, fabsf(g) * rsqrtf(a * b));
            const float zeta = (b - a) / (2.f * g);
            const float az = fabsf(zeta);
            const float t = az > 1e18f ? 0.5f / zeta : copysignf(1.f, zeta) / (az + sqrtf(fmaf(zeta, zeta, 1.f)));
            const float x = fmaf(t, t, 1.f);
            float c = rsqrtf(x);
            c = c * fmaf(-0.5f * x, c * c, 1.5f);
            const float sn = c * t;
#pragma unroll
            for (int u = 0; u < kF32ClusterPerLane; ++u) {
              const int i = lane + 32 * u;
              if (i < rows) {
                __stcg(&mp[i], c * xv[u] - sn * yv[u]);
                __stcg(&mq[i], sn * xv[u] + c * yv[u]);
              }
              if (i < r) {
                const float wu = __ldcg(&wp[i]), wv = __ldcg(&wq[i]);
                __stcg(&wp[i], c * wu - sn * wv);
                __stcg(&wq[i], sn * wu + c * wv);
              }
            }
          }
        }
      }
      if (round == rp - 2 && lane == 0 && my_rot) {
        atomicMax(&rotated[2 * kJacobiMaxSweeps + sweep], __float_as_int(my_mrel));
        __stcg(&rotated[sweep], 1);
      }
      cluster_sync_all();
    }
    if (__ldcg(&rotated[sweep]) == 0) { ++sweep; break; }
    const float mrel = __int_as_float(__ldcg(&rotated[2 * kJacobiMaxSweeps + sweep]));
    if (mrel * mrel <= tol) { ++sweep; break; }
  }
  if (blockIdx.x == 0 && tid == 0) *sweeps_out = sweep;
}

// FP32 one-sided Jacobi in one CTA with M and W in shared memory: the cheap
// first phase.  Columns are stored with stride ldm = r rounded up to 4; each
// group of kF32PairLanes (8) lanes rotates one column pair, lane l of the
// group holding the float4s l, l + 8, ... (V of them, V = ceil(r / 32)) of
// both columns, so a group reads 128 contiguous bytes per access (no bank
// conflicts).  The CTA has a group per pair of a round (480 threads at
// r = 120).  A round is bound by instruction issue: every group computes the
// rotation's scalars, so eight lanes per pair (rather than a half-warp) issue
// half the warp-instructions per round.  The rotations are accumulated in W32
// (column-major r x r), which the FP64 phase then orthonormalises and applies
// to M before finishing in FP64.
constexpr int kF32MaxR = 160;
constexpr int kF32PairLanes = 8;

__device__ __forceinline__ float pair_group_sum(float v) {
#pragma unroll
  for (int o = kF32PairLanes / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Packed FP32 pairs (two floats in 64 bits) on the SM's two-wide FP32 path:
// each half is one IEEE round-to-nearest multiply or fused multiply-add, as
// the scalar instruction would give, at half the instructions.
__device__ __forceinline__ unsigned long long f2_splat(float a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ float f2_hsum(unsigned long long a) {
  float lo, hi;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(a));
  return lo + hi;
}

// column of round-robin position pos in round `round` (positions 1 .. rp-1 rotate)
__device__ __forceinline__ int rr_col_fast(int pos, int round, int rp) {
  if (pos == 0) return 0;
  int v = pos - 1 + round;
  if (v >= rp - 1) v -= rp - 1;
  return 1 + v;
}

size_t f32_jacobi_smem(int r) {
  const size_t ldm = (size_t)round_up(r, 4);
  return (2 * (size_t)r * ldm + r) * sizeof(float);
}

template <int V>
__global__ void __launch_bounds__(kF32PairLanes * kF32MaxR / 2, 1)
jacobi_f32_kernel(int r, const double* __restrict__ Mc, float* __restrict__ W32, int* sweeps_out) {
  extern __shared__ __align__(16) float smf[];
  const int ldm = (r + 3) & ~3;
  const int ld4 = ldm / 4;                // float4 per column
  float* M = smf;
  float* W = smf + (size_t)r * ldm;
  float* nrm = W + (size_t)r * ldm;
  __shared__ float redf[32];
  __shared__ int s_rot;
  __shared__ int s_maxrel;  // bits of the largest relative off-diagonal rotated in the sweep
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, warps = nt >> 5;
  const int hw = tid / kF32PairLanes, hl = tid % kF32PairLanes, nhw = nt / kF32PairLanes;  // group, lane in it
  const int rp = r + (r & 1), npairs = rp / 2;
  float f = 0.f;
  for (int c = warp; c < r; c += warps)
    for (int i = lane; i < ldm; i += 32) {
      const float v = i < r ? (float)Mc[(int64_t)c * r + i] : 0.f;
      M[c * ldm + i] = v;
      W[c * ldm + i] = (i == c) ? 1.f : 0.f;
      f = fmaf(v, v, f);
    }
  f = warp_sum(f);
  if (lane == 0) redf[warp] = f;
  __syncthreads();
  float fro2 = 0.f;
  for (int i = 0; i < warps; ++i) fro2 += redf[i];
  const float eps = 1.1920929e-7f;
  const float zero2 = ((float)r * eps) * ((float)r * eps) * fro2;
  const float tol = (float)r * eps;
  int sweep = 0;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    __syncthreads();
    if (tid == 0) { s_rot = 0; s_maxrel = 0; }
    // squared column norms, exact at the start of each sweep and then carried
    // through the rotations (||c m_p - s m_q||^2 = c^2 a - 2 c s g + s^2 b), so
    // that each pair reduces only its inner product
    for (int c = warp; c < r; c += warps) {
      float s2 = 0.f;
      for (int i = lane; i < r; i += 32) s2 = fmaf(M[c * ldm + i], M[c * ldm + i], s2);
      s2 = warp_sum(s2);
      if (lane == 0) nrm[c] = s2;
    }
    __syncthreads();
    // whether this thread's pairs rotated in the sweep, and the largest relative
    // off-diagonal they rotated: kept in registers, reduced once per sweep
    bool my_rot = false;
    float my_mrel = 0.f;
    for (int round = 0; round < rp - 1; ++round) {
      // every group takes the same number of iterations (shuffles need the full warp)
      for (int s0 = 0; s0 < npairs; s0 += nhw) {
        const int sl = s0 + hw;
        int p = 0, q = 0;
        bool active = sl < npairs;
        if (active) {
          p = rr_col_fast(sl, round, rp);
          q = rr_col_fast(rp - 1 - sl, round, rp);
          if (p >= r || q >= r) active = false;
          if (p > q) { const int t = p; p = q; q = t; }
        }
        // 16 bytes per access as two packed pairs
        const ulonglong2* mp4 = reinterpret_cast<const ulonglong2*>(M + p * ldm);
        const ulonglong2* mq4 = reinterpret_cast<const ulonglong2*>(M + q * ldm);
        ulonglong2 xv[V], yv[V];
        const float a = active ? nrm[p] : 0.f, b = active ? nrm[q] : 0.f;
        unsigned long long g2 = 0ull;  // (+0, +0)
#pragma unroll
        for (int t = 0; t < V; ++t) {
          const int i4 = hl + kF32PairLanes * t;
          const bool ok = active && i4 < ld4;
          xv[t] = ok ? mp4[i4] : make_ulonglong2(0ull, 0ull);
          yv[t] = ok ? mq4[i4] : make_ulonglong2(0ull, 0ull);
          g2 = f2_fma(xv[t].x, yv[t].x, f2_fma(xv[t].y, yv[t].y, g2));
        }
        float g = pair_group_sum(f2_hsum(g2));
        if (active && fabsf(g) > tol * sqrtf(a * b) && a > zero2 && b > zero2) {
          my_rot = true;
          my_mrel = fmaxf(my_mrel, fabsf(g) * rsqrtf(a * b));
          // t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), zeta = (b - a) / 2g; for
          // |zeta| > 1e18 (zeta^2 would overflow) t = 1 / (2 zeta) to rounding.
          // c = (1 + t^2)^-1/2 from the hardware estimate and one Newton step:
          // the FP32 rotations only need to converge, W32 is orthonormalised
          // in FP64 afterwards.
          const float zeta = (b - a) / (2.f * g);
          const float az = fabsf(zeta);
          const float t = az > 1e18f ? 0.5f / zeta : copysignf(1.f, zeta) / (az + sqrtf(fmaf(zeta, zeta, 1.f)));
          const float x = fmaf(t, t, 1.f);
          float c = rsqrtf(x);
          c = c * fmaf(-0.5f * x, c * c, 1.5f);
          const float sn = c * t;
          if (hl == 0) {
            const float cc = c * c, ss = sn * sn, cs2 = 2.f * c * sn * g;
            nrm[p] = fmaxf(fmaf(cc, a, fmaf(ss, b, -cs2)), 0.f);
            nrm[q] = fmaxf(fmaf(ss, a, fmaf(cc, b, cs2)), 0.f);
          }
          // x' = c x - s y, y' = s x + c y on packed pairs: the product with s
          // rounded, then one fused multiply-add
          ulonglong2* mp = reinterpret_cast<ulonglong2*>(M + p * ldm);
          ulonglong2* mq = reinterpret_cast<ulonglong2*>(M + q * ldm);
          ulonglong2* wp = reinterpret_cast<ulonglong2*>(W + p * ldm);
          ulonglong2* wq = reinterpret_cast<ulonglong2*>(W + q * ldm);
          const unsigned long long c2 = f2_splat(c), s2 = f2_splat(sn), ns2 = f2_splat(-sn);
#pragma unroll
          for (int u = 0; u < V; ++u) {
            const int i4 = hl + kF32PairLanes * u;
            if (i4 < ld4) {
              const ulonglong2 xx = xv[u], yy = yv[u];
              const ulonglong2 wu = wp[i4], wv = wq[i4];
              mp[i4] = make_ulonglong2(f2_fma(c2, xx.x, f2_mul(ns2, yy.x)), f2_fma(c2, xx.y, f2_mul(ns2, yy.y)));
              mq[i4] = make_ulonglong2(f2_fma(c2, yy.x, f2_mul(s2, xx.x)), f2_fma(c2, yy.y, f2_mul(s2, xx.y)));
              wp[i4] = make_ulonglong2(f2_fma(c2, wu.x, f2_mul(ns2, wv.x)), f2_fma(c2, wu.y, f2_mul(ns2, wv.y)));
              wq[i4] = make_ulonglong2(f2_fma(c2, wv.x, f2_mul(s2, wu.x)), f2_fma(c2, wv.y, f2_mul(s2, wu.y)));
            }
          }
        }
      }
      __syncthreads();
    }
    {
      const bool wr = __any_sync(0xffffffffu, my_rot);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) my_mrel = fmaxf(my_mrel, __shfl_xor_sync(0xffffffffu, my_mrel, o));
      if (lane == 0 && wr) {
        s_rot = 1;
        atomicMax(&s_maxrel, __float_as_int(my_mrel));  // non-negative floats order like their bits
      }
      __syncthreads();
    }
    const int rot = s_rot;
    const float mrel = __int_as_float(s_maxrel);
    __syncthreads();  // every thread has read s_rot before it is reset below
    if (!rot) { ++sweep; break; }
    if (mrel * mrel > tol) continue;  // far from convergence: sweep again without checking
    // check pass: the same stopping test on every pair, from the current
    // columns, without rotating (replaces the final sweep that finds nothing)
    for (int c = warp; c < r; c += warps) {
      float s2 = 0.f;
      for (int i = lane; i < r; i += 32) s2 = fmaf(M[c * ldm + i], M[c * ldm + i], s2);
      s2 = warp_sum(s2);
      if (lane == 0) nrm[c] = s2;
    }
    if (tid == 0) s_rot = 0;
    __syncthreads();
    bool bad = false;
    for (int p = warp; p < r; p += warps) {
      const float a = nrm[p];
      const float4* xp = reinterpret_cast<const float4*>(M + p * ldm);
      for (int q = p + 1 + lane; q < r; q += 32) {
        const float4* xq = reinterpret_cast<const float4*>(M + q * ldm);
        float g0 = 0.f, g1 = 0.f;
        for (int i = 0; i < ld4; ++i) {
          const float4 x = xp[i], y = xq[i];
          g0 = fmaf(x.x, y.x, fmaf(x.y, y.y, g0));
          g1 = fmaf(x.z, y.z, fmaf(x.w, y.w, g1));
        }
        const float g = g0 + g1;
        const float b = nrm[q];
        if (fabsf(g) > tol * sqrtf(a * b) && a > zero2 && b > zero2) bad = true;
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) s_rot = 1;
    __syncthreads();
    if (!s_rot) { ++sweep; break; }
  }
  for (int c = warp; c < r; c += warps)
    for (int i = lane; i < r; i += 32) W32[(int64_t)c * r + i] = W[c * ldm + i];
  if (tid == 0) *sweeps_out = sweep;
}

__global__ void ns_shift_kernel(int r, const double* __restrict__ P, double* __restrict__ T) {
  // T = 1.5 I - 0.5 P
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < r * r; e += gridDim.x * blockDim.x)
    T[e] = ((e / r) == (e % r) ? 1.5 : 0.0) - 0.5 * P[e];
}

__global__ void widen_kernel(int n, const float* __restrict__ in, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) out[e] = (double)in[e];
}

}  // namespace

size_t jacobi_ws_bytes(int64_t rows, int r, bool precondition) {
  Sizer s;
  s.take<double>((size_t)rows * r);
  s.take<double>((size_t)r * r);
  s.take<unsigned>(2);
  s.take<int>(3 * kJacobiMaxSweeps);
  s.take<int>(1);
  s.take<int>(1);
  if (precondition) {
    s.take<float>((size_t)r * r);               // W32
    s.take<double>((size_t)4 * r * r);          // W64, P, T, M64
    s.take<double>((size_t)32 * r * r);         // split-K partials of the small GEMMs
  }
  return s.used + 256;
}

JacobiWs jacobi_ws_carve(Carver& c, int64_t rows, int r, bool precondition) {
  JacobiWs w;
  w.M = c.take<double>((size_t)rows * r);
  w.W = c.take<double>((size_t)r * r);
  w.barrier = c.take<unsigned>(2);
  w.rotated = c.take<int>(3 * kJacobiMaxSweeps);
  w.sweeps = c.take<int>(1);
  w.status = c.take<int>(1);
  if (precondition) {
    w.W32 = c.take<float>((size_t)r * r);
    double* d = c.take<double>((size_t)4 * r * r);
    if (d) { w.W64 = d; w.P = d + (size_t)r * r; w.T = d + 2 * (size_t)r * r; w.M64 = d + 3 * (size_t)r * r; }
    w.gemm_partial = c.take<double>((size_t)32 * r * r);
  }
  return w;
}

namespace {

// C (r x r, FP64) = op(A) B with the K range split over up to 32 CTAs (one
// 128 x 128 output tile each), partials added in order.
rsvd_status small_gemm64(int r, const double* A, bool transA, const double* B, double* C, double* partial,
                         cudaStream_t stream) {
  int nsplit = (int)cdiv(r, 8);
  if (nsplit > 32) nsplit = 32;
  const int64_t kchunk = round_up(cdiv(r, nsplit), 4);
  nsplit = (int)cdiv(r, kchunk);
  return simt_gemm<double>(r, r, r, A, r, transA, B, r, C, r, false, nsplit, kchunk, partial, stream);
}

rsvd_status launch_cluster_jacobi(int rows, int r, const double* Min, const double* W0, double* sigma, double* U,
                                  double* W, const JacobiWs& ws, cudaStream_t stream, double tol,
                                  int max_sweeps = kJacobiMaxSweeps) {
  if (max_sweeps == 0) {
    // finish only: a warp per column forms the outputs from M and the
    // rotation W0; the norms and signs go through ws.M (rows x r >= 2 r doubles)
    if (!W0 || rows < 2) return RSVD_ERR_INVALID_ARG;
    const int grid = (int)cdiv(r, kFinishWarps);
    jacobi_finish_norms_kernel<<<grid, 32 * kFinishWarps, 0, stream>>>(rows, r, Min, W0, ws.M, ws.sweeps);
    RSVD_CUDA(after_launch());
    jacobi_finish_out_kernel<<<grid, 32 * kFinishWarps, 0, stream>>>(rows, r, Min, W0, ws.M, sigma, U, W);
    RSVD_CUDA(after_launch());
    return RSVD_OK;
  }
  RSVD_CUDA(cudaMemsetAsync(ws.rotated, 0, 3 * kJacobiMaxSweeps * sizeof(int), stream));
  const int rp = r + (r & 1);
  const int npairs = rp / 2;
  // FP64 work per round is spread over up to 16 SMs (a non-portable cluster
  // size); fall back to smaller clusters where the device refuses it.
  int ncta = (int)cdiv(npairs, 4);
  if (ncta > 16) ncta = 16;
  if (ncta < 1) ncta = 1;
  // the check pass stages M in shared memory when it fits
  const size_t check_bytes = ((size_t)rows * r + r) * sizeof(double);
  const int check = max_sweeps > 0 && check_bytes <= (size_t)kClusterCheckSmem ? 1 : 0;
  const size_t smem = check ? check_bytes : 2 * (size_t)r * sizeof(double);
  static bool attr_set = false;
  if (!attr_set) {
    RSVD_CUDA(cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    RSVD_CUDA(cudaFuncSetAttribute(jacobi_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   kClusterCheckSmem));
    attr_set = true;
  }
  for (;;) {
    const int warps = (int)cdiv(npairs, ncta);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncta);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    const cudaError_t qe = cudaOccupancyMaxActiveClusters(&clusters, jacobi_cluster_kernel, &cfg);
    if ((qe != cudaSuccess || clusters < 1) && ncta > 1) {
      (void)cudaGetLastError();
      ncta = ncta > 8 ? 8 : ncta / 2;
      continue;
    }
    RSVD_CUDA(cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel, rows, r, Min, W0, ws.M, ws.W, ws.rotated, ws.sweeps,
                                 ws.status, sigma, U, W, check, tol, max_sweeps));
    RSVD_CUDA(after_launch());
    return RSVD_OK;
  }
}

// Phase 1 for 160 < r <= 512: FP32 sweeps over a cluster (up to 16 CTAs, one
// warp per pair), with M staged in the FP64 phase's working buffer.
rsvd_status launch_cluster_f32(int r, const double* Mc, const JacobiWs& ws, cudaStream_t stream) {
  RSVD_CUDA(cudaMemsetAsync(ws.rotated, 0, 3 * kJacobiMaxSweeps * sizeof(int), stream));
  const int npairs = (r + (r & 1)) / 2;
  int ncta = (int)cdiv(npairs, 4);
  if (ncta > 16) ncta = 16;
  static bool attr_set = false;
  if (!attr_set) {
    RSVD_CUDA(cudaFuncSetAttribute(jacobi_cluster_f32_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    attr_set = true;
  }
  for (;;) {
    const int warps = (int)cdiv(npairs, ncta);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncta);
    cfg.blockDim = dim3(32 * warps);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    const cudaError_t qe = cudaOccupancyMaxActiveClusters(&clusters, jacobi_cluster_f32_kernel, &cfg);
    if ((qe != cudaSuccess || clusters < 1) && ncta > 1) {
      (void)cudaGetLastError();
      ncta = ncta > 8 ? 8 : ncta / 2;
      continue;
    }
    RSVD_CUDA(cudaLaunchKernelEx(&cfg, jacobi_cluster_f32_kernel, r, r, Mc, reinterpret_cast<float*>(ws.M), ws.W32,
                                 ws.rotated, ws.sweeps));
    RSVD_CUDA(after_launch());
    return RSVD_OK;
  }
}

}  // namespace

rsvd_status jacobi_svd(int rows, int r, const double* Mc, double* sigma, double* U, double* W,
                       const JacobiWs& ws, cudaStream_t stream, double tol, bool fp64_sweeps) {
  if (r <= 0) return RSVD_OK;
  if (!(tol > 0.0)) tol = (double)r * 2.220446049250313e-16;  // r eps: the FP64 stopping test
  if (rows != r || r > 32 * kF32ClusterPerLane || r < 8 || !ws.W32)
    return launch_cluster_jacobi(rows, r, Mc, nullptr, sigma, U, W, ws, stream, tol);
  // Phase 1: FP32 sweeps to FP32 convergence -- one CTA with M and W in shared
  // memory, or for r > 160 a cluster with them in global memory.
  if (r > kF32MaxR) {
    RSVD_TRY(launch_cluster_f32(r, Mc, ws, stream));
  } else {
    static bool attr = false;
    if (!attr) {
      const int mx = (int)f32_jacobi_smem(kF32MaxR);
      RSVD_CUDA(cudaFuncSetAttribute(jacobi_f32_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      RSVD_CUDA(cudaFuncSetAttribute(jacobi_f32_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      RSVD_CUDA(cudaFuncSetAttribute(jacobi_f32_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      RSVD_CUDA(cudaFuncSetAttribute(jacobi_f32_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      RSVD_CUDA(cudaFuncSetAttribute(jacobi_f32_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
      attr = true;
    }
    // float4s per lane and column: ceil(ceil(r / 4) / 8); a group of lanes per
    // column pair of a round (a multiple of 32 threads, at most 1024)
    const int V = (int)cdiv(cdiv(r, 4), kF32PairLanes);
    const int npairs = (r + (r & 1)) / 2;
    const int nt = (int)round_up((int64_t)npairs * kF32PairLanes, 32);  // at most 640 (r <= 160)
    const size_t sm = f32_jacobi_smem(r);
    if (V <= 1) jacobi_f32_kernel<1><<<1, nt, sm, stream>>>(r, Mc, ws.W32, ws.sweeps);
    else if (V == 2) jacobi_f32_kernel<2><<<1, nt, sm, stream>>>(r, Mc, ws.W32, ws.sweeps);
    else if (V == 3) jacobi_f32_kernel<3><<<1, nt, sm, stream>>>(r, Mc, ws.W32, ws.sweeps);
    else if (V == 4) jacobi_f32_kernel<4><<<1, nt, sm, stream>>>(r, Mc, ws.W32, ws.sweeps);
    else jacobi_f32_kernel<5><<<1, nt, sm, stream>>>(r, Mc, ws.W32, ws.sweeps);
    RSVD_CUDA(after_launch());
  }
  // Phase 2: Newton-Schulz steps make W orthogonal to FP64 accuracy:
  // W' = (1.5 I - 0.5 W W^T) W, i.e. on the column-major storage (= W^T row-major)
  // Wt' = Wt (1.5 I - 0.5 P) with P = Wt^T Wt.  The accumulated FP32 rotation
  // is orthogonal to about 1e-6; each step squares that error, so two steps
  // reach FP64 rounding.  Without FP64 sweeps (inputs far less accurate than
  // FP32) the FP32 rotation is kept as it is: 1e-6 is already below the
  // orthogonality of U that the FP32 stopping test leaves (r eps32).
  widen_kernel<<<(int)cdiv((int64_t)r * r, 256), 256, 0, stream>>>(r * r, ws.W32, ws.T);
  RSVD_CUDA(after_launch());
  const int ns_steps = fp64_sweeps ? 2 : 0;
  for (int step = 0; step < ns_steps; ++step) {
    double* src = step == 0 ? ws.T : ws.W64;
    double* dst = step == 0 ? ws.W64 : ws.T;
    RSVD_TRY(small_gemm64(r, src, true, src, ws.P, ws.gemm_partial, stream));
    ns_shift_kernel<<<(int)cdiv((int64_t)r * r, 256), 256, 0, stream>>>(r, ws.P, ws.P);
    RSVD_CUDA(after_launch());
    RSVD_TRY(small_gemm64(r, src, false, ws.P, dst, ws.gemm_partial, stream));
  }
  // the (orthonormalised) rotation is now in T; move it to W64
  RSVD_CUDA(cudaMemcpyAsync(ws.W64, ws.T, sizeof(double) * (size_t)r * r, cudaMemcpyDeviceToDevice, stream));
  // M64 = M W': column-major M64 = Wt' (row-major) times Mc viewed row-major.
  RSVD_TRY(small_gemm64(r, ws.W64, false, Mc, ws.M64, ws.gemm_partial, stream));
  // Phase 3: FP64 sweeps to convergence, starting from the rotated matrix --
  // or, where the caller's inputs carry far less than FP32 accuracy, none: the
  // FP32 convergence stands and only the outputs are formed (norms, order,
  // normalisation) from the FP64 product M W.
  return launch_cluster_jacobi(rows, r, ws.M64, ws.W64, sigma, U, W, ws, stream, tol,
                               fp64_sweeps ? kJacobiMaxSweeps : 0);
}

}  // namespace rsvd
