// Section 2.1 step 6: SVD of the small factor by one-sided (Hestenes) Jacobi
// in FP64, with the relative stopping test of Demmel & Veselic (1992).
//
// M (rows x r, column-major, rows >= 1) is driven to orthogonal columns by plane rotations
// from the right, M W = U diag(sigma).  The sweep order is round-robin: in
// each of the r'-1 rounds of a sweep (r' = r rounded up to even) the r'/2
// column pairs are disjoint, so one CTA rotates each pair concurrently.
// FP64 throughput on one GB300 SM is low, so the rounds are spread over up to
// r'/2 co-resident CTAs (cooperative launch) separated by a grid barrier whose
// waits are bounded: a barrier that times out records DEV_TIMEOUT and every
// CTA returns.  Columns are read and written through L2 (ld/st .cg) because
// another SM may have rotated them in the previous round.
#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int JT = 128;  // threads per CTA

__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* p) {
  return *reinterpret_cast<const volatile unsigned*>(p);
}

// Sense-by-generation grid barrier with a bounded spin.  bar[0] = arrivals,
// bar[1] = generation.  Returns false if the wait timed out or another CTA
// recorded an error.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* status) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    const unsigned gen = ld_volatile_u32(&bar[1]);
    __threadfence();
    const unsigned arrived = atomicAdd(&bar[0], 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      long long spins = 0;
      while (ld_volatile_u32(&bar[1]) == gen) {
        if (++spins > kSpinLimit) { dev_set_status(status, DEV_TIMEOUT); ok = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*reinterpret_cast<volatile int*>(status) == DEV_TIMEOUT) ok = 0;
  }
  __syncthreads();
  return ok != 0;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < JT / 32; ++i) s += red[i];
  return s;
}

__device__ __forceinline__ int rr_column(int pos, int round, int rp) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (rp - 1);
}

__global__ void __launch_bounds__(JT)
jacobi_kernel(int rows, int r, const double* __restrict__ Min, double* M, double* W, unsigned* bar,
              int* rotated, int* sweeps_out, int* status, double* sigma, double* Uout, double* Wout) {
  __shared__ double red[JT / 32];
  const int tid = threadIdx.x;
  const unsigned nblocks = gridDim.x;
  const int rp = r + (r & 1);
  const int npairs = rp / 2;
  const int64_t mm = (int64_t)rows * r;
  const int64_t ww = (int64_t)r * r;

  // copy the input and set W = I (each CTA a strided share)
  for (int64_t e = (int64_t)blockIdx.x * JT + tid; e < mm; e += (int64_t)nblocks * JT)
    __stcg(&M[e], Min[e]);
  for (int64_t e = (int64_t)blockIdx.x * JT + tid; e < ww; e += (int64_t)nblocks * JT)
    __stcg(&W[e], (e / r) == (e % r) ? 1.0 : 0.0);
  // Frobenius norm of the input, for the rounding-level column test
  double f = 0.0;
  for (int64_t e = tid; e < mm; e += JT) f += Min[e] * Min[e];
  const double fro2 = block_sum(f, red);
  const double eps = 2.220446049250313e-16;
  const double big = (double)(rows > r ? rows : r);
  const double zero2 = (big * eps) * (big * eps) * fro2;
  const double tol = (double)r * eps;
  if (!grid_barrier(bar, nblocks, status)) return;

  int sweep = 0;
  bool converged = false;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    for (int round = 0; round < rp - 1; ++round) {
      for (int s = blockIdx.x; s < npairs; s += nblocks) {
        int p = rr_column(s, round, rp), q = rr_column(rp - 1 - s, round, rp);
        if (p >= r || q >= r) continue;  // dummy column of an odd r
        if (p > q) { const int t = p; p = q; q = t; }
        double* mp = M + (int64_t)p * rows;
        double* mq = M + (int64_t)q * rows;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = tid; i < rows; i += JT) {
          const double x = __ldcg(&mp[i]), y = __ldcg(&mq[i]);
          a += x * x; b += y * y; g += x * y;
        }
        a = block_sum(a, red);
        b = block_sum(b, red);
        g = block_sum(g, red);
        if (!(fabs(g) > tol * sqrt(a * b)) || !(a > zero2) || !(b > zero2)) continue;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double sn = c * t;
        double* wp = W + (int64_t)p * r;
        double* wq = W + (int64_t)q * r;
        for (int i = tid; i < rows; i += JT) {
          const double x = __ldcg(&mp[i]), y = __ldcg(&mq[i]);
          __stcg(&mp[i], c * x - sn * y);
          __stcg(&mq[i], sn * x + c * y);
        }
        for (int i = tid; i < r; i += JT) {
          const double u = __ldcg(&wp[i]), v = __ldcg(&wq[i]);
          __stcg(&wp[i], c * u - sn * v);
          __stcg(&wq[i], sn * u + c * v);
        }
        if (tid == 0) *reinterpret_cast<volatile int*>(&rotated[sweep]) = 1;
      }
      if (!grid_barrier(bar, nblocks, status)) return;
    }
    if (*reinterpret_cast<volatile int*>(&rotated[sweep]) == 0) { converged = true; break; }
  }
  if (blockIdx.x != 0) return;
  if (!converged) dev_set_status(status, DEV_NO_CONVERGE);
  if (tid == 0) *sweeps_out = sweep + (converged ? 1 : 0);
  // column norms, stable descending order, normalised outputs
  extern __shared__ double sh[];  // sigma_c for c < r
  for (int c = tid; c < r; c += JT) {
    double s2 = 0.0;
    for (int i = 0; i < rows; ++i) { const double x = __ldcg(&M[(int64_t)c * rows + i]); s2 += x * x; }
    sh[c] = sqrt(s2);
  }
  __syncthreads();
  for (int c = tid; c < r; c += JT) {
    const double sc = sh[c];
    int rank = 0;
    for (int d = 0; d < r; ++d) rank += (sh[d] > sc) || (sh[d] == sc && d < c);
    sigma[rank] = sc;
    const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
    for (int i = 0; i < rows; ++i) Uout[(int64_t)i * r + rank] = __ldcg(&M[(int64_t)c * rows + i]) * inv;
    for (int i = 0; i < r; ++i) Wout[(int64_t)i * r + rank] = __ldcg(&W[(int64_t)c * r + i]);
  }
}

}  // namespace

size_t jacobi_ws_bytes(int64_t rows, int r) {
  Sizer s;
  s.take<double>((size_t)rows * r);
  s.take<double>((size_t)r * r);
  s.take<unsigned>(2);
  s.take<int>(kJacobiMaxSweeps);
  s.take<int>(1);
  s.take<int>(1);
  return s.used + 256;
}

JacobiWs jacobi_ws_carve(Carver& c, int64_t rows, int r) {
  JacobiWs w;
  w.M = c.take<double>((size_t)rows * r);
  w.W = c.take<double>((size_t)r * r);
  w.barrier = c.take<unsigned>(2);
  w.rotated = c.take<int>(kJacobiMaxSweeps);
  w.sweeps = c.take<int>(1);
  w.status = c.take<int>(1);
  return w;
}

rsvd_status jacobi_svd(int rows, int r, const double* Mc, double* sigma, double* U, double* W,
                       const JacobiWs& ws, cudaStream_t stream) {
  if (r <= 0) return RSVD_OK;
  RSVD_CUDA(cudaMemsetAsync(ws.barrier, 0, 2 * sizeof(unsigned), stream));
  RSVD_CUDA(cudaMemsetAsync(ws.rotated, 0, kJacobiMaxSweeps * sizeof(int), stream));
  const int rp = r + (r & 1);
  int nblocks = rp / 2;
  if (nblocks > 128) nblocks = 128;
  if (nblocks < 1) nblocks = 1;
  const size_t smem = (size_t)r * sizeof(double);
  int dev = 0, coop = 0, per_sm = 0, sms = 0;
  RSVD_CUDA(cudaGetDevice(&dev));
  RSVD_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  RSVD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  RSVD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_kernel, JT, smem));
  if (!coop || per_sm * sms < nblocks) nblocks = 1;  // a single CTA never waits on another
  int rows_ = rows, r_ = r;
  const double* Min = Mc;
  double* Mw = ws.M;
  double* Ww = ws.W;
  unsigned* bar = ws.barrier;
  int* rot = ws.rotated;
  int* sw = ws.sweeps;
  int* st = ws.status;
  void* args[] = {&rows_, &r_, &Min, &Mw, &Ww, &bar, &rot, &sw, &st, &sigma, &U, &W};
  if (nblocks > 1) {
    RSVD_CUDA(cudaLaunchCooperativeKernel((const void*)jacobi_kernel, dim3(nblocks), dim3(JT), args,
                                          smem, stream));
    RSVD_CUDA(after_launch());
  } else {
    jacobi_kernel<<<1, JT, smem, stream>>>(rows_, r_, Min, Mw, Ww, bar, rot, sw, st, sigma, U, W);
    RSVD_CUDA(after_launch());
  }
  return RSVD_OK;
}

}  // namespace rsvd
