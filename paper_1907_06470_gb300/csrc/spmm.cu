// A-passes for a sparse A in compressed sparse row form (Section 3.3: the
// sparse x dense product; Section 2.1 step 2 and Eq. (3)).
//
//   forward     Y = A X      one warp per row of A
//   transposed  Z = A^T Y    the same kernel on the CSR of A^T (the CSC of A)
//
// Each output row is computed by one warp.  The row's entries are read 32 at
// a time (one (column, value) pair per lane, coalesced), then broadcast lane
// by lane; for each entry the warp gathers one row of the dense panel (r
// values, 16-byte vector loads, lane l holding columns 4l..4l+3 + 128t) and
// accumulates in FP32 registers in entry order, so every output row is a fixed
// sequence of FMAs and the result does not depend on scheduling.  The gathers
// dominate: a pass reads nnz * r * 4 bytes of panel rows, which the
// Zipf-skewed column popularity of the sparse workloads serves largely from L2.
//
// The grid is persistent (the resident blocks of every SM) and its warps draw
// rows kSpmmGrab at a time from a counter, so a warp that drew short rows
// draws again instead of idling beside a long row of its block.  The CSR
// arrays and the output are touched once per pass and move with streaming
// (evict-first) loads and stores, leaving L2 to the gathered panel rows.
//
// The CSR of A^T is built on the host once (csr_transpose_host): a stable
// counting sort over columns, split over threads by row ranges, so its entry
// order (increasing row of A within each column) and hence the transposed
// pass are deterministic.
#include <cuda_bf16.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace rsvd {
namespace {

constexpr int kSpmmThreads = 256;
constexpr int kSpmmGrab = 2;  // rows a warp takes per draw
constexpr int kSpmmBuckets = 4096;             // panel row blocks the segment tasks are grouped by
constexpr int64_t kSpmmBlockBytes = 32 << 20;  // bytes of panel rows per block

__device__ __forceinline__ void fma4(float4& a, float v, const float4& x) {
  a.x = fmaf(v, x.x, a.x);
  a.y = fmaf(v, x.y, a.y);
  a.z = fmaf(v, x.z, a.z);
  a.w = fmaf(v, x.w, a.w);
}

// The gathered panel, in one of three formats (SpmmPanel::fmt):
//   0  FP32 rows (f, ld floats per row)
//   1  BF16 rows (h, ld 16-bit values per row): X rounded to BF16
//   2  24-bit rows (p24, rb bytes per row): X rounded to 16 significant bits;
//      each group of 128 values takes 384 bytes, the high 16 bits of the 128
//      values (256 bytes) followed by their next 8 bits (128 bytes), so a
//      value's bits are hi << 16 | lo << 8 and a gathered row is one
//      contiguous 3-bytes-per-value run
// Lane l of a warp holds the values 4l..4l+3 + 128t of a row, so a lane loads
// one float4 (FP32), one uint2 (BF16), or one uint2 and one uint32 from the
// same 384-byte group (24-bit) per slot t.
template <int FMT>
struct PanelSlot;

template <>
struct PanelSlot<0> {
  float4 v;
  __device__ __forceinline__ void load(const SpmmPanel& P, int64_t row, int q) {
    v = __ldg(reinterpret_cast<const float4*>(P.f + row * P.ld) + q);
  }
  __device__ __forceinline__ void zero() { v = make_float4(0.f, 0.f, 0.f, 0.f); }
  __device__ __forceinline__ float4 get() const { return v; }
};

template <>
struct PanelSlot<1> {
  uint2 h;
  __device__ __forceinline__ void load(const SpmmPanel& P, int64_t row, int q) {
    h = __ldg(reinterpret_cast<const uint2*>(P.h + row * P.ld) + q);
  }
  __device__ __forceinline__ void zero() { h = make_uint2(0u, 0u); }
  __device__ __forceinline__ float4 get() const {
    return make_float4(__uint_as_float(h.x << 16), __uint_as_float(h.x & 0xffff0000u), __uint_as_float(h.y << 16),
                       __uint_as_float(h.y & 0xffff0000u));
  }
};

template <>
struct PanelSlot<2> {
  uint2 h;
  uint32_t l;
  __device__ __forceinline__ void load(const SpmmPanel& P, int64_t row, int q) {
    const uint8_t* g = P.p24 + row * P.rb + (q >> 5) * 384;
    h = __ldg(reinterpret_cast<const uint2*>(g) + (q & 31));
    l = __ldg(reinterpret_cast<const uint32_t*>(g + 256) + (q & 31));
  }
  __device__ __forceinline__ void zero() {
    h = make_uint2(0u, 0u);
    l = 0u;
  }
  __device__ __forceinline__ float4 get() const {
    return make_float4(__uint_as_float((h.x << 16) | ((l & 0xffu) << 8)),
                       __uint_as_float((h.x & 0xffff0000u) | (l & 0xff00u)),
                       __uint_as_float((h.y << 16) | ((l >> 8) & 0xff00u)),
                       __uint_as_float((h.y & 0xffff0000u) | ((l >> 16) & 0xff00u)));
  }
};

// V4 slots per lane: panel rows of at most 128*V4 values.  Rows start 16-byte
// (FP32, 24-bit) or 8-byte (BF16) aligned; values r..4*ceil(r/4)-1 are read
// (inside ld) but never written to Y.
// Sum over entries [e0, e1) of one row into acc (lane l: columns 4l..4l+3 + 128t).
template <int V4, int FMT>
__device__ __forceinline__ void row_segment_vec(int64_t e0, int64_t e1, int lane, int nv,
                                                const int32_t* __restrict__ colidx, const float* __restrict__ val,
                                                const SpmmPanel& P, float4 (&acc)[V4]) {
  for (int64_t b = e0; b < e1; b += 32) {
    const int64_t e = b + lane;
    int c = 0;
    float v = 0.f;
    if (e < e1) {
      c = __ldcs(colidx + e);
      v = __ldcs(val + e);
    }
    const int cnt = (int)(e1 - b < 32 ? e1 - b : 32);
    int j = 0;
    // four entries at a time: their gathers are issued before the FMAs
    for (; j + 4 <= cnt; j += 4) {
      int cj[4];
      float vj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        cj[u] = __shfl_sync(0xffffffffu, c, j + u);
        vj[u] = __shfl_sync(0xffffffffu, v, j + u);
      }
      PanelSlot<FMT> x[4][V4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int t = 0; t < V4; ++t) {
          const int q = lane + 32 * t;
          if (q < nv) x[u][t].load(P, cj[u], q);
          else x[u][t].zero();
        }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int t = 0; t < V4; ++t) fma4(acc[t], vj[u], x[u][t].get());
    }
    for (; j < cnt; ++j) {
      const int cj = __shfl_sync(0xffffffffu, c, j);
      const float vj = __shfl_sync(0xffffffffu, v, j);
#pragma unroll
      for (int t = 0; t < V4; ++t) {
        const int q = lane + 32 * t;
        if (q < nv) {
          PanelSlot<FMT> x;
          x.load(P, cj, q);
          fma4(acc[t], vj, x.get());
        }
      }
    }
  }
}

// Write (or add) acc to the output row yr, columns < r only.
template <int V4>
__device__ __forceinline__ void store_row_vec(float* yr, int r, int lane, int nv, int accumulate,
                                              const float4 (&acc)[V4]) {
#pragma unroll
  for (int t = 0; t < V4; ++t) {
    const int q = lane + 32 * t;
    if (q >= nv) continue;
    const int c0 = 4 * q;
    float4 o = acc[t];
    if (c0 + 4 <= r) {
      float4* p = reinterpret_cast<float4*>(yr + c0);
      if (accumulate) {
        const float4 y = __ldcs(p);
        o.x += y.x; o.y += y.y; o.z += y.z; o.w += y.w;
      }
      __stcs(p, o);
    } else {  // the panel's last, partial group of four columns
      yr[c0] = accumulate ? yr[c0] + o.x : o.x;
      if (c0 + 1 < r) yr[c0 + 1] = accumulate ? yr[c0 + 1] + o.y : o.y;
      if (c0 + 2 < r) yr[c0 + 2] = accumulate ? yr[c0 + 2] + o.z : o.z;
    }
  }
}

// Persistent grid: warps draw kSpmmGrab rows at a time, from *next when it is
// given (zeroed before the launch), else by a fixed stride.  With split != 0,
// rows of more than kSpmmSeg entries are left to the segment tasks
// (spmm_segment_kernel + spmm_combine_kernel).
template <int V4, int FMT>
__global__ void __launch_bounds__(kSpmmThreads, V4 >= 4 ? 2 : 3)
spmm_csr_vec_kernel(int64_t M, int r, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                    const float* __restrict__ val, const SpmmPanel P, float* __restrict__ Y, int64_t ldy,
                    int accumulate, int split, unsigned long long* next) {
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = ((int64_t)blockIdx.x * kSpmmThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kSpmmThreads) >> 5;
  const int nv = (r + 3) >> 2;
  for (int64_t it = 0;; ++it) {
    int64_t base;
    if (next) {
      unsigned long long b = 0;
      if (lane == 0) b = atomicAdd(next, (unsigned long long)kSpmmGrab);
      base = (int64_t)__shfl_sync(0xffffffffu, b, 0);
    } else {
      base = (gwarp + it * nwarps) * kSpmmGrab;
    }
    if (base >= M) break;
    const int64_t end = base + kSpmmGrab < M ? base + kSpmmGrab : M;
    for (int64_t row = base; row < end; ++row) {
      const int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
      if (split && e1 - e0 > kSpmmSeg) continue;
      float4 acc[V4];
#pragma unroll
      for (int t = 0; t < V4; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      row_segment_vec<V4, FMT>(e0, e1, lane, nv, colidx, val, P, acc);
      store_row_vec<V4>(Y + row * ldy, r, lane, nv, accumulate, acc);
    }
  }
}

// Task list of the long rows: a row of len > kSpmmSeg entries takes
// ceil(len / kSpmmSeg) consecutive task slots (segment s of the row in slot
// base + s) from an atomic counter.  Which base a row gets depends on timing,
// but the partials of a row are always added in segment order.
__global__ void spmm_tasks_kernel(int64_t M, const int32_t* __restrict__ rowptr, int* counter, int max_tasks,
                                  int* __restrict__ task_row, int* __restrict__ task_seg) {
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < M; row += (int64_t)gridDim.x * blockDim.x) {
    const int64_t len = (int64_t)rowptr[row + 1] - rowptr[row];
    if (len <= kSpmmSeg) continue;
    const int nseg = (int)((len + kSpmmSeg - 1) / kSpmmSeg);
    const int base = atomicAdd(counter, nseg);
    for (int s = 0; s < nseg && base + s < max_tasks; ++s) {
      task_row[base + s] = (int)row;
      task_seg[base + s] = s;
    }
  }
}

// The segment tasks are run grouped by the panel row block (kSpmmBlockBytes
// of panel rows) that holds the panel row of their first entry, so that the
// warps running at any one time gather from a window of the panel that L2
// keeps: the long rows' head segments share their panel rows, and so do the
// segments of the dense columns of A (rows of the CSR of A^T).
// Bucket of each task; counts per bucket.
__global__ void spmm_task_bucket_kernel(const int* __restrict__ counter, int64_t max_tasks,
                                        const int* __restrict__ task_row, const int* __restrict__ task_seg,
                                        const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                        int64_t width, int* __restrict__ bucket_of, int* __restrict__ bucket_cnt) {
  int64_t ntask = *counter;
  if (ntask > max_tasks) ntask = max_tasks;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntask; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e0 = (int64_t)rowptr[task_row[t]] + (int64_t)task_seg[t] * kSpmmSeg;
    int64_t b = (int64_t)colidx[e0] / width;
    if (b >= kSpmmBuckets) b = kSpmmBuckets - 1;
    bucket_of[t] = (int)b;
    atomicAdd(&bucket_cnt[b], 1);
  }
}

// Exclusive prefix sum of the kSpmmBuckets counts, in place (one block of 1024).
__global__ void __launch_bounds__(1024) spmm_bucket_scan_kernel(int* __restrict__ bucket_cnt) {
  constexpr int per = kSpmmBuckets / 1024;
  __shared__ int wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int v[per];
  int s = 0;
#pragma unroll
  for (int i = 0; i < per; ++i) {
    v[i] = bucket_cnt[tid * per + i];
    s += v[i];
  }
  int incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    wsum[lane] = w;
  }
  __syncthreads();
  int run = incl - s + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
  for (int i = 0; i < per; ++i) {
    bucket_cnt[tid * per + i] = run;
    run += v[i];
  }
}

// order[]: the tasks grouped by bucket (their order inside a bucket does not
// matter: each task writes its own partial slot).
__global__ void spmm_bucket_scatter_kernel(const int* __restrict__ counter, int64_t max_tasks,
                                           const int* __restrict__ bucket_of, int* __restrict__ bucket_cur,
                                           int* __restrict__ order) {
  int64_t ntask = *counter;
  if (ntask > max_tasks) ntask = max_tasks;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ntask; t += (int64_t)gridDim.x * blockDim.x)
    order[atomicAdd(&bucket_cur[bucket_of[t]], 1)] = (int)t;
}

// Persistent grid, one warp per task at a time (positions gw, gw + warps, ...
// of order[]): the partial product of one segment of a long row, written to
// partial[task * ldp ...] (ldp = 4 ceil(r/4)).
template <int V4, int FMT>
__global__ void __launch_bounds__(kSpmmThreads, V4 >= 4 ? 2 : 3)
spmm_segment_kernel(int r, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                    const float* __restrict__ val, const SpmmPanel P, const int* __restrict__ counter,
                    const int* __restrict__ task_row, const int* __restrict__ task_seg,
                    const int* __restrict__ order, int64_t max_tasks, float* __restrict__ partial, int64_t ldp) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * kSpmmThreads) >> 5;
  const int nv = (r + 3) >> 2;
  int64_t ntask = *counter;
  if (ntask > max_tasks) ntask = max_tasks;
  for (int64_t i = ((int64_t)blockIdx.x * kSpmmThreads + threadIdx.x) >> 5; i < ntask; i += nwarps) {
    const int64_t task = order[i];
    const int row = task_row[task], seg = task_seg[task];
    const int64_t e0 = (int64_t)rowptr[row] + (int64_t)seg * kSpmmSeg;
    const int64_t e1 = min((int64_t)rowptr[row + 1], e0 + kSpmmSeg);
    float4 acc[V4];
#pragma unroll
    for (int t = 0; t < V4; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    row_segment_vec<V4, FMT>(e0, e1, lane, nv, colidx, val, P, acc);
    float4* p = reinterpret_cast<float4*>(partial + task * ldp);
#pragma unroll
    for (int t = 0; t < V4; ++t) {
      const int q = lane + 32 * t;
      if (q < nv) p[q] = acc[t];
    }
  }
}

// Persistent grid, one warp per long row at a time (found at its segment-0
// task): the row's partials added in segment order, then stored like a short
// row.
template <int V4>
__global__ void __launch_bounds__(kSpmmThreads)
spmm_combine_kernel(int r, const int32_t* __restrict__ rowptr, const int* __restrict__ counter,
                    const int* __restrict__ task_row, const int* __restrict__ task_seg, int64_t max_tasks,
                    const float* __restrict__ partial, int64_t ldp, float* __restrict__ Y, int64_t ldy,
                    int accumulate) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * kSpmmThreads) >> 5;
  const int nv = (r + 3) >> 2;
  int64_t ntask = *counter;
  if (ntask > max_tasks) ntask = max_tasks;
  for (int64_t task = ((int64_t)blockIdx.x * kSpmmThreads + threadIdx.x) >> 5; task < ntask; task += nwarps) {
    if (task_seg[task] != 0) continue;
    const int row = task_row[task];
    const int64_t len = (int64_t)rowptr[row + 1] - rowptr[row];
    const int nseg = (int)((len + kSpmmSeg - 1) / kSpmmSeg);
    if (task + nseg > max_tasks) continue;  // only if rowptr holds more than nnz entries
    float4 acc[V4];
#pragma unroll
    for (int t = 0; t < V4; ++t) acc[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    // eight segments' partials loaded together, then added in segment order
    for (int s0 = 0; s0 < nseg; s0 += 8) {
      float4 x[8][V4];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        // past the last segment: the last one again (in cache, not added)
        const float4* p = reinterpret_cast<const float4*>(partial + (task + min(s0 + u, nseg - 1)) * ldp);
#pragma unroll
        for (int t = 0; t < V4; ++t) {
          const int q = lane + 32 * t;
          x[u][t] = q < nv ? p[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (s0 + u < nseg) {
#pragma unroll
          for (int t = 0; t < V4; ++t) {
            acc[t].x += x[u][t].x; acc[t].y += x[u][t].y; acc[t].z += x[u][t].z; acc[t].w += x[u][t].w;
          }
        }
    }
    store_row_vec<V4>(Y + (int64_t)row * ldy, r, lane, nv, accumulate, acc);
  }
}

// Panel conversion for the compact formats: rows of X (K x r, ldx) rounded to
// BF16 (fmt 1, into h, ld values per row) or to 16 significant bits (fmt 2,
// into p24, rb bytes per row in 384-byte groups of 128 values), both
// round-to-nearest-even; values r..ld-1 are zero.  One thread per value.
__global__ void spmm_pack_kernel(int fmt, int64_t K, int r, const float* __restrict__ X, int64_t ldx,
                                 uint16_t* __restrict__ h, uint8_t* __restrict__ p24, int64_t ld, int64_t rb) {
  const int64_t total = K * ld;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t row = i / ld;
    const int c = (int)(i - row * ld);
    const float x = c < r ? X[row * ldx + c] : 0.f;
    if (fmt == 1) {
      h[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    } else {
      uint32_t b = __float_as_uint(x);
      if ((b & 0x7fffffffu) > 0x7f800000u) b |= 0x00400000u;  // NaN stays NaN in 24 bits
      else if ((b & 0x7f800000u) != 0x7f800000u) b += 0x7fu + ((b >> 8) & 1u);
      uint8_t* g = p24 + row * rb + (c >> 7) * 384;
      const int w = c & 127;
      reinterpret_cast<uint16_t*>(g)[w] = (uint16_t)(b >> 16);
      g[256 + w] = (uint8_t)((b >> 8) & 0xffu);
    }
  }
}

// Scalar variant for panels that are not 16-byte aligned: lane l holds columns
// l + 32t, t < VS.
template <int VS>
__global__ void __launch_bounds__(kSpmmThreads)
spmm_csr_scalar_kernel(int64_t M, int r, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                       const float* __restrict__ val, const float* __restrict__ X, int64_t ldx,
                       float* __restrict__ Y, int64_t ldy, int accumulate) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (kSpmmThreads / 32) + (threadIdx.x >> 5);
  if (row >= M) return;
  float acc[VS];
#pragma unroll
  for (int t = 0; t < VS; ++t) acc[t] = 0.f;
  const int64_t e0 = rowptr[row], e1 = rowptr[row + 1];
  for (int64_t b = e0; b < e1; b += 32) {
    const int64_t e = b + lane;
    int c = 0;
    float v = 0.f;
    if (e < e1) {
      c = __ldg(colidx + e);
      v = __ldg(val + e);
    }
    const int cnt = (int)(e1 - b < 32 ? e1 - b : 32);
    for (int j = 0; j < cnt; ++j) {
      const int cj = __shfl_sync(0xffffffffu, c, j);
      const float vj = __shfl_sync(0xffffffffu, v, j);
      const float* xr = X + (int64_t)cj * ldx;
#pragma unroll
      for (int t = 0; t < VS; ++t) {
        const int q = lane + 32 * t;
        if (q < r) acc[t] = fmaf(vj, __ldg(xr + q), acc[t]);
      }
    }
  }
  float* yr = Y + row * ldy;
#pragma unroll
  for (int t = 0; t < VS; ++t) {
    const int q = lane + 32 * t;
    if (q < r) yr[q] = accumulate ? yr[q] + acc[t] : acc[t];
  }
}

// Blocks of a kSpmmThreads-thread kernel resident on the whole device at once.
int64_t resident_blocks_of(const void* kernel) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, kSpmmThreads, 0);
  return (int64_t)(sms > 0 ? sms : 152) * (occ > 0 ? occ : 1);
}

// The same, cached per kernel instance.
template <int V4, int FMT>
int64_t resident_vec() {
  static const int64_t b = resident_blocks_of(reinterpret_cast<const void*>(spmm_csr_vec_kernel<V4, FMT>));
  return b;
}
template <int V4, int FMT>
int64_t resident_seg() {
  static const int64_t b = resident_blocks_of(reinterpret_cast<const void*>(spmm_segment_kernel<V4, FMT>));
  return b;
}
template <int V4>
int64_t resident_comb() {
  static const int64_t b = resident_blocks_of(reinterpret_cast<const void*>(spmm_combine_kernel<V4>));
  return b;
}

template <int V4, int FMT>
rsvd_status launch_vec(int64_t M, int r, const int32_t* rowptr, const int32_t* colidx, const float* val,
                       const SpmmPanel& X, float* Y, int64_t ldy, int acc, bool split, unsigned long long* next,
                       const int* counter, const int* task_row, const int* task_seg, const int* order,
                       int64_t max_tasks, float* partial, int64_t ldp, cudaStream_t stream) {
  const int64_t row_blocks = cdiv(cdiv(M, kSpmmGrab), kSpmmThreads / 32);
  const int64_t res = resident_vec<V4, FMT>();
  spmm_csr_vec_kernel<V4, FMT><<<(unsigned)(row_blocks < res ? row_blocks : res), kSpmmThreads, 0, stream>>>(
      M, r, rowptr, colidx, val, X, Y, ldy, acc, split ? 1 : 0, next);
  RSVD_CUDA(after_launch());
  if (!split) return RSVD_OK;
  const int64_t task_blocks = cdiv(max_tasks, kSpmmThreads / 32);
  const int64_t sres = resident_seg<V4, FMT>();
  spmm_segment_kernel<V4, FMT><<<(unsigned)(task_blocks < sres ? task_blocks : sres), kSpmmThreads, 0, stream>>>(
      r, rowptr, colidx, val, X, counter, task_row, task_seg, order, max_tasks, partial, ldp);
  RSVD_CUDA(after_launch());
  const int64_t cres = resident_comb<V4>();
  spmm_combine_kernel<V4><<<(unsigned)(task_blocks < cres ? task_blocks : cres), kSpmmThreads, 0, stream>>>(
      r, rowptr, counter, task_row, task_seg, max_tasks, partial, ldp, Y, ldy, acc);
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

}  // namespace

size_t spmm_ws_bytes(int64_t nnz, int r) {
  const int64_t tasks = spmm_max_tasks(nnz);
  Sizer s;
  s.take<int>(4);
  s.take<int>(kSpmmBuckets);
  s.take<int>((size_t)tasks);  // task_row
  s.take<int>((size_t)tasks);  // task_seg
  s.take<int>((size_t)tasks);  // bucket_of
  s.take<int>((size_t)tasks);  // order
  s.take<float>((size_t)tasks * round_up(r, 4));
  return s.used + 256;
}

int64_t spmm_p24_row_bytes(int64_t ld) { return cdiv(ld, 128) * 384; }

rsvd_status spmm_pack(int fmt, int64_t K, int r, const float* X, int64_t ldx, uint16_t* h, uint8_t* p24, int64_t ld,
                      cudaStream_t stream) {
  if (K <= 0) return RSVD_OK;
  if ((fmt != 1 && fmt != 2) || r < 1 || ldx < r || ld < round_up(r, 4) || ld % 4 || !X || (fmt == 1 && !h) ||
      (fmt == 2 && !p24))
    return fail(RSVD_ERR_INVALID_ARG, "spmm_pack: bad arguments");
  const int64_t blocks = std::min<int64_t>(cdiv(K * ld, 256), 152 * 32);
  spmm_pack_kernel<<<(unsigned)blocks, 256, 0, stream>>>(fmt, K, r, X, ldx, h, p24, ld, spmm_p24_row_bytes(ld));
  RSVD_CUDA(after_launch());
  return RSVD_OK;
}

rsvd_status spmm_csr_panel(int64_t M, int r, const int32_t* rowptr, const int32_t* colidx, const float* val,
                           int64_t nnz, const SpmmPanel& X, float* Y, int64_t ldy, bool accumulate, void* ws,
                           size_t ws_bytes, cudaStream_t stream) {
  if (M <= 0) return RSVD_OK;
  const bool fp32 = X.fmt == 0;
  if (r < 1 || r > kSpmmMaxR || X.ld < r || ldy < r || !rowptr || !Y || X.fmt < 0 || X.fmt > 2 ||
      (fp32 && !X.f) || (X.fmt == 1 && (!X.h || X.ld % 4)) ||
      (X.fmt == 2 && (!X.p24 || X.ld % 4 || X.rb != spmm_p24_row_bytes(X.ld))))
    return fail(RSVD_ERR_INVALID_ARG, "spmm_csr: bad arguments");
  const int64_t blocks = cdiv(M, kSpmmThreads / 32);
  if (blocks > 0x7fffffffLL) return fail(RSVD_ERR_INVALID_ARG, "spmm_csr: too many rows");
  const int acc = accumulate ? 1 : 0;
  const bool vec = !fp32 || (X.ld % 4 == 0 && ldy % 4 == 0 && aligned16(X.f) && aligned16(Y));
  if (!vec) {
    const dim3 grid((unsigned)blocks);
    const int vs = (int)cdiv(r, 32);
#define RSVD_SCA(V) \
  spmm_csr_scalar_kernel<V><<<grid, kSpmmThreads, 0, stream>>>(M, r, rowptr, colidx, val, X.f, X.ld, Y, ldy, acc)
    if (vs <= 4) RSVD_SCA(4);
    else if (vs <= 8) RSVD_SCA(8);
    else RSVD_SCA(16);
#undef RSVD_SCA
    RSVD_CUDA(after_launch());
    return RSVD_OK;
  }
  if (ldy % 4 || !aligned16(Y)) return fail(RSVD_ERR_INVALID_ARG, "spmm_csr: compact panels need 16-byte output rows");
  const int v4 = (int)cdiv(cdiv(r, 4), 32);
  // rows of more than kSpmmSeg entries are split into segment tasks when the
  // workspace allows; the row counter of the persistent grid sits beside the
  // task counter
  const bool ws_ok = ws && reinterpret_cast<uintptr_t>(ws) % 16 == 0;
  const int64_t max_tasks = spmm_max_tasks(nnz);
  const bool split = ws_ok && ws_bytes >= spmm_ws_bytes(nnz, r) && nnz > kSpmmSeg;
  int *counter = nullptr, *task_row = nullptr, *task_seg = nullptr, *bucket_cnt = nullptr, *bucket_of = nullptr,
      *order = nullptr;
  unsigned long long* next = nullptr;
  float* partial = nullptr;
  const int64_t ldp = round_up(r, 4);
  if (ws_ok && ws_bytes >= 256) {
    Carver c(ws, ws_bytes);
    counter = c.take<int>(4);
    next = reinterpret_cast<unsigned long long*>(counter + 2);
    if (split) {
      bucket_cnt = c.take<int>(kSpmmBuckets);
      task_row = c.take<int>((size_t)max_tasks);
      task_seg = c.take<int>((size_t)max_tasks);
      bucket_of = c.take<int>((size_t)max_tasks);
      order = c.take<int>((size_t)max_tasks);
      partial = c.take<float>((size_t)max_tasks * ldp);
    }
    // the counters, and the bucket counts carved right after them
    const size_t zero = split ? (size_t)(reinterpret_cast<char*>(bucket_cnt + kSpmmBuckets) -
                                         reinterpret_cast<char*>(counter))
                              : 4 * sizeof(int);
    RSVD_CUDA(cudaMemsetAsync(counter, 0, zero, stream));
  }
  if (split) {
    int tb = (int)cdiv(M, 256);
    if (tb > 152 * 16) tb = 152 * 16;
    spmm_tasks_kernel<<<tb, 256, 0, stream>>>(M, rowptr, counter, (int)max_tasks, task_row, task_seg);
    RSVD_CUDA(after_launch());
    // group the tasks by the block of panel rows of their first entry
    const int64_t row_bytes = X.fmt == 0 ? X.ld * 4 : (X.fmt == 1 ? X.ld * 2 : X.rb);
    const int64_t width = std::max<int64_t>(1, kSpmmBlockBytes / row_bytes);
    const int gb = (int)std::min<int64_t>(cdiv(max_tasks, 256), 152 * 8);
    spmm_task_bucket_kernel<<<gb, 256, 0, stream>>>(counter, max_tasks, task_row, task_seg, rowptr, colidx, width,
                                                    bucket_of, bucket_cnt);
    RSVD_CUDA(after_launch());
    spmm_bucket_scan_kernel<<<1, 1024, 0, stream>>>(bucket_cnt);
    RSVD_CUDA(after_launch());
    spmm_bucket_scatter_kernel<<<gb, 256, 0, stream>>>(counter, max_tasks, bucket_of, bucket_cnt, order);
    RSVD_CUDA(after_launch());
  }
#define RSVD_VEC(V, F)                                                                                           \
  return launch_vec<V, F>(M, r, rowptr, colidx, val, X, Y, ldy, acc, split, next, counter, task_row, task_seg, \
                          order, max_tasks, partial, ldp, stream)
#define RSVD_VEC_F(V)                  \
  do {                                 \
    if (X.fmt == 0) RSVD_VEC(V, 0);    \
    else if (X.fmt == 1) RSVD_VEC(V, 1); \
    else RSVD_VEC(V, 2);               \
  } while (0)
  switch (v4) {
    case 1: RSVD_VEC_F(1);
    case 2: RSVD_VEC_F(2);
    case 3: RSVD_VEC_F(3);
    default: RSVD_VEC_F(4);
  }
#undef RSVD_VEC_F
#undef RSVD_VEC
}

rsvd_status spmm_csr(int64_t M, int r, const int32_t* rowptr, const int32_t* colidx, const float* val,
                     int64_t nnz, const float* X, int64_t ldx, float* Y, int64_t ldy, bool accumulate, void* ws,
                     size_t ws_bytes, cudaStream_t stream) {
  SpmmPanel P;
  P.fmt = 0;
  P.f = X;
  P.ld = ldx;
  return spmm_csr_panel(M, r, rowptr, colidx, val, nnz, P, Y, ldy, accumulate, ws, ws_bytes, stream);
}

// Stable counting-sort transpose on the host.  Rows are split into T ranges of
// about equal entry counts; thread t counts its entries per column, the
// per-(thread, column) offsets are laid out column-major (thread 0 first), and
// every thread scatters its rows in increasing order, so the entries of each
// output row come in increasing row index of A whatever T is.
// per-(thread, row) counters of the host counting sorts: 32-bit (nnz < 2^31),
// at most 64 Mi of them (256 MB), which bounds the thread count for long outputs
constexpr int64_t kCountScratch = (int64_t)1 << 26;

rsvd_status csr_transpose_host(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                               const float* val, int32_t* t_rowptr, int32_t* t_colidx, float* t_val) {
  if (m < 0 || n < 0 || !rowptr || !t_rowptr) return fail(RSVD_ERR_INVALID_ARG, "csr_transpose: bad arguments");
  if (rowptr[0] != 0) return fail(RSVD_ERR_INVALID_ARG, "csr_transpose: rowptr[0] != 0");
  for (int64_t i = 0; i < m; ++i)
    if (rowptr[i + 1] < rowptr[i]) return fail(RSVD_ERR_INVALID_ARG, "csr_transpose: rowptr decreases");
  const int64_t nnz = rowptr[m];
  if (nnz > 0 && (!colidx || !val || !t_colidx || !t_val))
    return fail(RSVD_ERR_INVALID_ARG, "csr_transpose: NULL index or value array");
  unsigned hw = std::thread::hardware_concurrency();
  int T = (int)std::min<int64_t>({(int64_t)(hw ? hw : 1), 32, std::max<int64_t>(1, nnz >> 20),
                                    std::max<int64_t>(1, kCountScratch / std::max<int64_t>(1, n))});
  if (T < 1) T = 1;
  std::vector<int64_t> r0(T + 1);
  for (int t = 0; t <= T; ++t) {
    const int64_t target = nnz * t / T;
    r0[t] = t == T ? m : std::lower_bound(rowptr, rowptr + m + 1, (int32_t)target) - rowptr;
    if (r0[t] > m) r0[t] = m;
  }
  for (int t = 1; t <= T; ++t)
    if (r0[t] < r0[t - 1]) r0[t] = r0[t - 1];
  std::vector<int32_t> cnt((size_t)T * n, 0);  // cnt[t*n + j]
  std::vector<int> bad(T, 0);
  auto count = [&](int t) {
    int32_t* c = cnt.data() + (size_t)t * n;
    for (int64_t i = r0[t]; i < r0[t + 1]; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int32_t j = colidx[e];
        if (j < 0 || j >= n) { bad[t] = 1; return; }
        ++c[j];
      }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(count, t);
  count(0);
  for (auto& x : th) x.join();
  th.clear();
  for (int t = 0; t < T; ++t)
    if (bad[t]) return fail(RSVD_ERR_INVALID_ARG, "csr_transpose: column index out of range");
  // offsets: column j's block starts at t_rowptr[j]; thread t writes after threads < t
  int64_t run = 0;
  for (int64_t j = 0; j < n; ++j) {
    t_rowptr[j] = (int32_t)run;
    for (int t = 0; t < T; ++t) {
      const int64_t c = cnt[(size_t)t * n + j];
      cnt[(size_t)t * n + j] = (int32_t)run;
      run += c;
    }
  }
  t_rowptr[n] = (int32_t)run;
  auto scatter = [&](int t) {
    int32_t* off = cnt.data() + (size_t)t * n;
    for (int64_t i = r0[t]; i < r0[t + 1]; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        const int64_t pos = off[colidx[e]]++;
        t_colidx[pos] = (int32_t)i;
        t_val[pos] = val[e];
      }
  };
  for (int t = 1; t < T; ++t) th.emplace_back(scatter, t);
  scatter(0);
  for (auto& x : th) x.join();
  return RSVD_OK;
}

// COO (Section 3.3: the paper's sparse format, row and column index arrays of
// 32 or 64 bits, structure of arrays) to CSR on the host: a stable counting
// sort by row.  T threads take contiguous chunks of the entries; the
// per-(thread, row) offsets are laid out row-major over threads, so thread t's
// entries of a row follow those of threads < t and the entries of each row
// keep their COO order whatever T is.
template <typename I>
rsvd_status coo_to_csr_typed(int64_t m, int64_t n, int64_t nnz, const I* rowidx, const I* colidx,
                             const float* val, int32_t* rowptr, int32_t* out_colidx, float* out_val) {
  unsigned hw = std::thread::hardware_concurrency();
  int T = (int)std::min<int64_t>({(int64_t)(hw ? hw : 1), 32, std::max<int64_t>(1, nnz >> 20),
                                    std::max<int64_t>(1, kCountScratch / std::max<int64_t>(1, m))});
  if (T < 1) T = 1;
  std::vector<int64_t> e0(T + 1);
  for (int t = 0; t <= T; ++t) e0[t] = nnz * t / T;
  std::vector<int32_t> cnt((size_t)T * m, 0);  // cnt[t*m + i]
  std::vector<int> bad(T, 0);
  auto count = [&](int t) {
    int32_t* c = cnt.data() + (size_t)t * m;
    for (int64_t e = e0[t]; e < e0[t + 1]; ++e) {
      const int64_t i = (int64_t)rowidx[e], j = (int64_t)colidx[e];
      if (i < 0 || i >= m || j < 0 || j >= n) { bad[t] = 1; return; }
      ++c[i];
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(count, t);
  count(0);
  for (auto& x : th) x.join();
  th.clear();
  for (int t = 0; t < T; ++t)
    if (bad[t]) return fail(RSVD_ERR_INVALID_ARG, "coo_to_csr: index out of range");
  int64_t run = 0;
  for (int64_t i = 0; i < m; ++i) {
    rowptr[i] = (int32_t)run;
    for (int t = 0; t < T; ++t) {
      const int64_t c = cnt[(size_t)t * m + i];
      cnt[(size_t)t * m + i] = (int32_t)run;
      run += c;
    }
  }
  rowptr[m] = (int32_t)run;
  auto scatter = [&](int t) {
    int32_t* off = cnt.data() + (size_t)t * m;
    for (int64_t e = e0[t]; e < e0[t + 1]; ++e) {
      const int64_t pos = off[(int64_t)rowidx[e]]++;
      out_colidx[pos] = (int32_t)colidx[e];
      out_val[pos] = val[e];
    }
  };
  for (int t = 1; t < T; ++t) th.emplace_back(scatter, t);
  scatter(0);
  for (auto& x : th) x.join();
  return RSVD_OK;
}

rsvd_status coo_to_csr_host(int64_t m, int64_t n, int64_t nnz, int index_bits, const void* rowidx,
                            const void* colidx, const float* val, int32_t* rowptr, int32_t* out_colidx,
                            float* out_val) {
  if (m < 0 || n < 0 || nnz < 0 || !rowptr) return fail(RSVD_ERR_INVALID_ARG, "coo_to_csr: bad arguments");
  if (index_bits != 32 && index_bits != 64) return fail(RSVD_ERR_INVALID_ARG, "coo_to_csr: index_bits must be 32 or 64");
  if (nnz >= ((int64_t)1 << 31) || n > ((int64_t)1 << 31) - 1)
    return fail(RSVD_ERR_INVALID_ARG, "coo_to_csr: the CSR holds 32-bit offsets and column indices");
  if (nnz > 0 && (!rowidx || !colidx || !val || !out_colidx || !out_val))
    return fail(RSVD_ERR_INVALID_ARG, "coo_to_csr: NULL index or value array");
  if (index_bits == 32)
    return coo_to_csr_typed<int32_t>(m, n, nnz, static_cast<const int32_t*>(rowidx),
                                     static_cast<const int32_t*>(colidx), val, rowptr, out_colidx, out_val);
  return coo_to_csr_typed<int64_t>(m, n, nnz, static_cast<const int64_t*>(rowidx),
                                   static_cast<const int64_t*>(colidx), val, rowptr, out_colidx, out_val);
}

}  // namespace rsvd
