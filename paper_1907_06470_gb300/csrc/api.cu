// C ABI: planner (Section 3.4 / 3.5), the randomized SVD driver (Section 2.1
// steps 1-7 with the power scheme of Section 2.2), the exact small SVD, and
// the per-step entry points.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"
#include "rsvd_pipeline.h"

namespace rsvd {

// ---- errors -------------------------------------------------------------------

namespace {
thread_local std::string g_last_error;
std::atomic<unsigned long long> g_launches{0};
}

cudaError_t after_launch() {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

void set_error(const std::string& msg) { g_last_error = msg; }

rsvd_status fail(rsvd_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

rsvd_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return e == cudaErrorMemoryAllocation ? RSVD_ERR_OOM : RSVD_ERR_CUDA;
}

rsvd_status status_from_device(int code) {
  switch (code) {
    case DEV_OK: return RSVD_OK;
    case DEV_NOT_SPD: return fail(RSVD_ERR_NOT_SPD, "Cholesky breakdown: Gram matrix not positive definite");
    case DEV_NO_CONVERGE: return fail(RSVD_ERR_NO_CONVERGE, "one-sided Jacobi reached its sweep limit");
    case DEV_TIMEOUT: return fail(RSVD_ERR_TIMEOUT, "a device-side wait exceeded its spin limit");
    default: return fail(RSVD_ERR_INVALID_ARG, "device reported an invalid argument");
  }
}

rsvd_status read_device_status(const int* d_status, cudaStream_t stream) {
  int h = 0;
  RSVD_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  RSVD_CUDA(cudaStreamSynchronize(stream));
  if (h == DEV_TIMEOUT) {
    // the tensor-core pipeline records where its first expired wait was (the
    // words after the status of the workspaces it writes to)
    int w[2] = {0, 0};
    if (cudaMemcpy(w, d_status + 1, sizeof(w), cudaMemcpyDeviceToHost) == cudaSuccess && w[0]) {
      static const char* roles[] = {"?", "A loads (operand slot free)", "A loads (staging slot free)",
                                    "panel loads (operand slot free)", "MMA (accumulator free)",
                                    "MMA (A operand full)", "MMA (panel full)", "converter", "epilogue"};
      const int role = (w[0] >> 24) & 15;
      return fail(RSVD_ERR_TIMEOUT, std::string("a device-side wait exceeded its spin limit: ") +
                                        roles[role < 9 ? role : 0] + ", ring slot " +
                                        std::to_string((w[0] >> 16) & 255) + ", K step " +
                                        std::to_string(w[0] & 0xffff) + ", unit " + std::to_string(w[1]));
    }
  }
  return status_from_device(h);
}

// ---- A-pass dispatch -----------------------------------------------------------

namespace {

// Chunking of the reduction dimension follows the tile map: the forward pass
// (K = n) is split at tile columns, the transposed pass (K = m) at tile rows.
struct PassShape {
  int64_t M, K, kchunk;
  int nsplit;
};

PassShape pass_shape(int64_t m, int64_t n, int trans, int64_t mb, int64_t nb) {
  PassShape s;
  s.M = trans ? n : m;
  s.K = trans ? m : n;
  s.kchunk = trans ? mb : nb;
  if (s.kchunk <= 0 || s.kchunk > s.K) s.kchunk = s.K;
  s.kchunk = round_up(s.kchunk, 8);
  s.nsplit = (int)cdiv(s.K, s.kchunk);
  if (s.nsplit < 1) s.nsplit = 1;
  return s;
}

size_t elem_size(int dtype) { return dtype == RSVD_F64 ? 8 : ((dtype == RSVD_BF16 || dtype == RSVD_F16) ? 2 : 4); }

}  // namespace

size_t apass_ws_bytes(int64_t m, int64_t n, int r, int trans, int prec, int64_t mb, int64_t nb) {
  const PassShape s = pass_shape(m, n, trans, mb, nb);
  const size_t esz = prec == RSVD_PREC_FP64 ? 8 : 4;
  if (prec == RSVD_PREC_BF16 || prec == RSVD_PREC_BF16X3 || prec == RSVD_PREC_FP8)
    return tc_apass_ws_bytes(m, n, r, trans, prec == RSVD_PREC_FP8 ? RSVD_PREC_BF16 : prec, mb, nb);
  return s.nsplit > 1 ? (size_t)s.nsplit * s.M * r * esz + 256 : 256;
}

rsvd_status apass_dense(const rsvd_matrix& A, int trans, int prec, int r, const void* X, int64_t ldx,
                        void* Y, int64_t ldy, int64_t mb, int64_t nb, void* ws, size_t ws_bytes,
                        int* status, cudaStream_t stream, bool accumulate) {
  if (A.kind != RSVD_DENSE || A.location != RSVD_ON_DEVICE)
    return fail(RSVD_ERR_INVALID_ARG, "apass: A must be a dense device matrix");
  if (ws_bytes < apass_ws_bytes(A.m, A.n, r, trans, prec, mb, nb))
    return fail(RSVD_ERR_INVALID_ARG, "apass: workspace too small");
  const PassShape s = pass_shape(A.m, A.n, trans, mb, nb);
  if (prec == RSVD_PREC_FP64) {
    if (A.dtype != RSVD_F64) return fail(RSVD_ERR_INVALID_ARG, "apass: FP64 precision needs FP64 A");
    return simt_gemm<double>(s.M, r, s.K, static_cast<const double*>(A.data), A.ld, trans != 0,
                             static_cast<const double*>(X), ldx, static_cast<double*>(Y), ldy, accumulate,
                             s.nsplit, s.kchunk, static_cast<double*>(ws), stream);
  }
  if (A.dtype == RSVD_BF16 || A.dtype == RSVD_F16) {  // Section 3.2: A stored in 16 bits
    Bf16Source a16;
    a16.data = static_cast<const uint16_t*>(A.data);
    a16.m = A.m; a16.n = A.n; a16.ld = A.ld;
    a16.f16 = A.dtype == RSVD_F16 ? 1 : 0;
    return tc_apass_from_16(a16, trans, prec, r, static_cast<const float*>(X), ldx, static_cast<float*>(Y), ldy, ws,
                            ws_bytes, status, stream, accumulate);
  }
  if (A.dtype != RSVD_F32) return fail(RSVD_ERR_INVALID_ARG, "apass: FP32/BF16 precision needs FP32 A");
  if (prec == RSVD_PREC_FP32) {
    return simt_gemm<float>(s.M, r, s.K, static_cast<const float*>(A.data), A.ld, trans != 0,
                            static_cast<const float*>(X), ldx, static_cast<float*>(Y), ldy, accumulate,
                            s.nsplit, s.kchunk, static_cast<float*>(ws), stream);
  }
  if (prec != RSVD_PREC_BF16 && prec != RSVD_PREC_BF16X3)
    return fail(RSVD_ERR_INVALID_ARG, "apass: unknown precision");
  return tc_apass_from_f32(A, trans, prec, r, static_cast<const float*>(X), ldx,
                           static_cast<float*>(Y), ldy, mb, nb, ws, ws_bytes, status, stream, accumulate);
}

}  // namespace rsvd

using namespace rsvd;

// ---- plan -----------------------------------------------------------------------

namespace {

// CUDA-event spans around the stages of one rsvd_run.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;
  std::vector<std::pair<int, int>> spans;  // (stage, index of the start event)
  size_t used = 0;
  double ms[RSVD_STAGE_COUNT] = {};
  int apass_calls = 0;

  rsvd_status reserve(size_t pairs) {
    while (ev.size() < 2 * pairs) {
      cudaEvent_t e;
      RSVD_CUDA(cudaEventCreate(&e));
      ev.push_back(e);
    }
    return RSVD_OK;
  }
  void begin() { used = 0; spans.clear(); apass_calls = 0; }
  int start(int stage, cudaStream_t s) {
    if (!on || used + 2 > ev.size()) return -1;
    cudaEventRecord(ev[used], s);
    spans.push_back({stage, (int)used});
    used += 2;
    return (int)used - 2;
  }
  void stop(int idx, cudaStream_t s) {
    if (idx >= 0) cudaEventRecord(ev[idx + 1], s);
  }
  void collect() {
    for (double& x : ms) x = 0.0;
    for (auto& sp : spans) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[sp.second], ev[sp.second + 1]) == cudaSuccess) ms[sp.first] += t;
    }
  }
  ~Profiler() {
    for (auto e : ev) cudaEventDestroy(e);
  }
};

struct Span {
  Profiler& p;
  cudaStream_t s;
  int idx;
  Span(Profiler& p_, int stage, cudaStream_t s_) : p(p_), s(s_), idx(p_.start(stage, s_)) {}
  ~Span() { p.stop(idx, s); }
};

}  // namespace

struct rsvd_plan_s {
  int64_t m = 0, n = 0;
  int k = 0, p = 0, q = 0, r = 0, ldr = 0;
  uint64_t seed = 0;
  int prec = RSVD_PREC_FP32, dtype = RSVD_F32, refine = 1, n_slots = 2;
  int64_t mb = 0, nb = 0;
  size_t mem_cap = 0, ws_bytes = 0, a_copy_bytes = 0;
  void* ws = nullptr;
  // carved device buffers
  void* X = nullptr;    // n x ldr  (test matrix / Z panel)
  void* Y = nullptr;    // m x ldr
  void* Qm = nullptr;   // m x ldr
  void* Bt = nullptr;   // n x ldr
  void* Qb = nullptr;   // n x ldr
  void* apass_ws = nullptr;
  size_t apass_ws_bytes = 0;
  uint16_t* pk_h = nullptr;   // CSR plans of BF16 precision: the panel in BF16
  uint8_t* pk_24 = nullptr;   // CSR plans of BF16X3 precision: the panel in 24 bits
  OrthWs orth;
  JacobiWs jac;
  double* R = nullptr;      // r x r
  double* sigma = nullptr;  // r
  double* sigma_prev = nullptr;  // r: estimates of the previous power iteration (automatic q)
  int* q_flag = nullptr;    // device word: 1 when the change fell below the tolerance
  int auto_q = 0;           // choose q automatically (q is then the maximum)
  int fused = 0;            // power iterations as fused sweeps W = orth(A^T (A W))
  double auto_q_tol = 1e-3;
  int q_used = 0;           // power iterations applied by the last run
  std::string ckpt_path;    // checkpoint file of the range finder ("" = off)
  int ckpt_stop_after = -1; // stop (RSVD_ERR_INTERRUPTED) after writing this step's checkpoint
  int resumed_from = -1;    // step the last run resumed after (-1: started afresh)
  double* UR = nullptr;     // r x r
  double* WR = nullptr;     // r x r
  void* URk = nullptr;      // r x k in dtype
  void* WRk = nullptr;      // r x k in dtype
  void* sign_scratch = nullptr;
  size_t sign_scratch_bytes = 0;
  void* lift_ws = nullptr;  // the lift's tensor-core products (BF16-family plans)
  size_t lift_ws_bytes = 0;
  void* bwd_ws = nullptr;   // backward pass (rsvd_backward)
  size_t bwd_ws_bytes = 0;
  int* status = nullptr;
  void* Adev = nullptr;     // device copy of a host-resident A
  // In-core copy of a host A in row chunks on a side stream (Section 3.7: I/O
  // overlapped with compute): the first forward pass takes each chunk as it
  // lands; everything else waits for the whole copy.
  cudaStream_t h2d_stream = nullptr;
  std::vector<cudaEvent_t> h2d_ev;  // one per chunk, then one for "all landed"
  int64_t h2d_chunk_rows = 0;
  int h2d_chunks = 0;
  bool h2d_pending = false;          // the current run's copy is in flight
  // Host matrices prefetched for later runs (rsvd_plan_prefetch): up to two
  // copies pending on h2d_stream, each into its own device buffer; rsvd_run
  // takes the oldest when its descriptor is the run's A.
  struct Prefetch {
    void* dev = nullptr;
    size_t bytes = 0;
    bool pending = false;
    uint64_t seq = 0;
    rsvd_matrix desc{};
    int64_t ldd = 0, chunk_rows = 0;
    int chunks = 0;
    std::vector<cudaEvent_t> ev;  // as h2d_ev
  };
  Prefetch pre[2];
  uint64_t pre_seq = 0;
  uint16_t* a16 = nullptr;  // BF16 plans in core: BF16 copy of A, written by the first forward pass
  size_t a16_bytes = 0;
  int64_t a16_ld = 0;
  bool a16_ready = false;   // the current run's copy is complete (enqueued)
  int64_t mb_req = 0, nb_req = 0;  // tile edges asked for in the options (0: none)
  StreamState* ss = nullptr;       // out-of-core state (created on the first streamed run)
  bool streaming = false;          // the current run streams A from the host
  CsrStream* cs = nullptr;         // out-of-core state of a host CSR A
  bool csr_streaming = false;      // the current run streams CSR tiles from the host
  int32_t* h_tpinned = nullptr;    // pinned host CSR of A^T built for streaming (n + 1 + nnz indices)
  float* h_tval_pinned = nullptr;
  size_t h_tpinned_nnz = 0;
  int64_t h_tpinned_n = -1;
  int kind = RSVD_DENSE;           // rsvd_kind the plan runs on
  bool tc_orth_all = false;        // range-finder Grams / panel products on the tensor cores
  bool tc_orth_inner = false;      // the same except for the final Q
  Fp8Source f8;                    // FP8 plans: E4M3 codes of A and tile scales (in the workspace)
  unsigned* f8_amax = nullptr;
  void* csr_dev = nullptr;         // device copies of a CSR A and/or its transpose, SpMM workspace
  size_t csr_dev_bytes = 0;
  void* spmm_ws = nullptr;         // long-row tasks of the CSR passes (inside csr_dev)
  size_t spmm_ws_bytes = 0;
  std::vector<int32_t> h_idx;      // host staging for a transpose built by the library
  std::vector<float> h_val;
  Profiler prof;
};

namespace {

rsvd_status check_args(int64_t m, int64_t n, int k, int p, int q, const rsvd_opts* o) {
  if (m <= 0 || n <= 0 || k < 1 || p < 0 || q < 0 || q > 64)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: need m, n >= 1, k >= 1, p >= 0, 0 <= q <= 64");
  const int64_t r = (int64_t)k + p;
  if (r > m || r > n) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: k + p must not exceed min(m, n)");
  const bool csr = o && o->kind == RSVD_CSR;
  if (o && o->kind != RSVD_DENSE && o->kind != RSVD_CSR) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: unknown kind");
  if (!csr && r > 256) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: k + p must not exceed 256 (dense)");
  if (csr && r > kSpmmMaxR) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: k + p must not exceed 512 (CSR)");
  if (csr && (o->dtype != RSVD_F32 ||
              (o->prec != RSVD_PREC_FP32 && o->prec != RSVD_PREC_BF16 && o->prec != RSVD_PREC_BF16X3)))
    return fail(RSVD_ERR_UNSUPPORTED, "rsvd_plan: CSR plans take F32 values and FP32, BF16 or BF16X3 precision");
  if (o) {
    if (o->dtype != RSVD_F32 && o->dtype != RSVD_F64)
      return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: dtype must be F32 or F64");
    if (o->prec < RSVD_PREC_FP64 || o->prec > RSVD_PREC_FP8)
      return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: unknown precision");
    if (o->prec == RSVD_PREC_FP8 && (csr || o->dtype != RSVD_F32))
      return fail(RSVD_ERR_UNSUPPORTED, "rsvd_plan: FP8 precision takes dense F32 matrices");
    if ((o->prec == RSVD_PREC_FP64) != (o->dtype == RSVD_F64))
      return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: FP64 precision goes with FP64 data and only with it");
    if (o->mb < 0 || o->nb < 0 || o->n_slots < 0)
      return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: negative tile edge or slot count");
    if (o->auto_q_tol < 0.0 || !(o->auto_q_tol == o->auto_q_tol))
      return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: auto_q_tol must be >= 0 (0: default 1e-3)");
    if (o->fused && (csr || o->prec == RSVD_PREC_FP8 || o->auto_q))
      return fail(RSVD_ERR_UNSUPPORTED, "rsvd_plan: fused sweeps take dense plans of FP64, FP32, BF16 or BF16X3 "
                                        "precision with a fixed q");
  }
  return RSVD_OK;
}

void apply_opts(rsvd_plan_s* P, const rsvd_opts* o) {
  if (o) {
    P->dtype = o->dtype;
    P->prec = o->prec;
    P->refine = o->refine;
    P->mb = o->mb;
    P->nb = o->nb;
    P->mb_req = o->mb;
    P->nb_req = o->nb;
    P->n_slots = o->n_slots > 0 ? o->n_slots : 2;
    P->kind = o->kind;
    P->auto_q = o->auto_q ? 1 : 0;
    P->fused = o->fused ? 1 : 0;
    if (o->auto_q_tol > 0.0) P->auto_q_tol = o->auto_q_tol;
  }
  if (P->mb <= 0) P->mb = P->m;  // in core: one block row unless asked otherwise
  if (P->nb <= 0) P->nb = P->n;
  if (P->mb > P->m) P->mb = P->m;
  if (P->nb > P->n) P->nb = P->n;
}

// Carve (or, with base == nullptr, size) the plan's workspace.
size_t layout(rsvd_plan_s* P, void* base, size_t cap) {
  Carver c(base, base ? cap : ~size_t(0) / 2);
  const size_t esz = elem_size(P->dtype);
  const int64_t mx = P->m > P->n ? P->m : P->n;
  P->X = c.take<char>((size_t)P->n * P->ldr * esz);
  P->Y = c.take<char>((size_t)P->m * P->ldr * esz);
  P->Qm = c.take<char>((size_t)P->m * P->ldr * esz);
  P->Bt = c.take<char>((size_t)P->n * P->ldr * esz);
  P->Qb = c.take<char>((size_t)P->n * P->ldr * esz);
  const bool dense = P->kind == RSVD_DENSE;  // CSR passes need no workspace here
  if (!dense && (P->prec == RSVD_PREC_BF16 || P->prec == RSVD_PREC_BF16X3)) {
    if (P->prec == RSVD_PREC_BF16) P->pk_h = c.take<uint16_t>((size_t)mx * P->ldr);
    else P->pk_24 = c.take<uint8_t>((size_t)mx * spmm_p24_row_bytes(P->ldr));
  }
  const size_t a0 = dense ? apass_ws_bytes(P->m, P->n, P->r, 0, P->prec, P->mb, P->nb) : 0;
  const size_t a1 = dense ? apass_ws_bytes(P->m, P->n, P->r, 1, P->prec, P->mb, P->nb) : 0;
  size_t a2 = 0;
  if (dense && (P->prec == RSVD_PREC_BF16 || P->prec == RSVD_PREC_FP8) && P->refine)
    a2 = apass_ws_bytes(P->m, P->n, P->r, 1, RSVD_PREC_BF16X3, P->mb, P->nb);
  P->apass_ws_bytes = a0 > a1 ? a0 : a1;
  if (a2 > P->apass_ws_bytes) P->apass_ws_bytes = a2;
  P->apass_ws = c.take<char>(P->apass_ws_bytes);
  // Range-finder bases only have to span the sketch: FP32 data orthonormalises
  // them on the tensor cores (split BF16) -- every basis for the BF16 / FP8
  // paths, every basis but the final Q (whose orthonormality enters B = Q^T A:
  // a Q orthonormal to 2^-16 moves the singular values of Q^T A by about as
  // much) for the FP32 and split-BF16 paths, which aim at FP32 accuracy
  P->tc_orth_all = P->dtype == RSVD_F32 && (P->prec == RSVD_PREC_BF16 || P->prec == RSVD_PREC_FP8);
  P->tc_orth_inner = P->dtype == RSVD_F32;
  P->orth = orth_ws_carve(c, mx, P->r, P->dtype, P->tc_orth_inner);
  P->jac = jacobi_ws_carve(c, P->r, P->r);
  P->R = c.take<double>((size_t)P->r * P->r);
  P->sigma = c.take<double>((size_t)P->r);
  P->sigma_prev = c.take<double>((size_t)P->r);
  P->q_flag = c.take<int>(4);
  P->UR = c.take<double>((size_t)P->r * P->r);
  P->WR = c.take<double>((size_t)P->r * P->r);
  P->URk = c.take<char>((size_t)P->r * P->k * esz);
  P->WRk = c.take<char>((size_t)P->r * P->k * esz);
  P->sign_scratch_bytes = sign_scratch_bytes(P->m, P->k);
  P->sign_scratch = c.take<char>(P->sign_scratch_bytes);
  P->bwd_ws_bytes = dense ? backward_ws_bytes(P->m, P->n, P->k, P->dtype) : 0;
  P->bwd_ws = c.take<char>(P->bwd_ws_bytes);
  P->lift_ws_bytes = P->dtype == RSVD_F32 ? tc_gemm_wide_ws_bytes(mx, P->r, P->k, RSVD_PREC_BF16X3) : 0;
  P->lift_ws = c.take<char>(P->lift_ws_bytes);
  if (P->prec == RSVD_PREC_FP8) {
    // quantisation tiles: the plan's tiles rounded up to multiples of 128
    Fp8Source& f = P->f8;
    f.m = P->m;
    f.n = P->n;
    f.ldc = round_up(P->n, 16);
    f.qm = P->mb >= P->m ? P->m : round_up(P->mb, 128);
    f.qn = P->nb >= P->n ? P->n : round_up(P->nb, 128);
    if (f.qm > P->m) f.qm = P->m;
    if (f.qn > P->n) f.qn = P->n;
    f.codes = c.take<uint8_t>((size_t)P->m * f.ldc);
    f.scales = c.take<float>((size_t)cdiv(P->m, f.qm) * cdiv(P->n, f.qn));
    P->f8_amax = c.take<unsigned>((size_t)cdiv(P->m, f.qm) * cdiv(P->n, f.qn));
  }
  P->status = c.take<int>(4);
  if (base) {
    P->orth.status = P->status;
    P->jac.status = P->status;
  }
  return c.used + 256;
}

template <typename T>
rsvd_status run_typed(rsvd_plan_s* P, const rsvd_matrix& A, T* U, T* S, T* V, cudaStream_t st) {
  const int64_t m = P->m, n = P->n;
  const int r = P->r, k = P->k, ldr = P->ldr;
  T* X = static_cast<T*>(P->X);
  T* Y = static_cast<T*>(P->Y);
  T* Q = static_cast<T*>(P->Qm);
  T* Bt = static_cast<T*>(P->Bt);
  T* Qb = static_cast<T*>(P->Qb);
  const int prec = P->prec;
  // the final B^T = A^T Q: split BF16 for dense BF16 / FP8 plans (refine);
  // an FP32 panel for CSR plans whose range finder gathers compact panels
  const bool csr_compact = P->kind == RSVD_CSR && (prec == RSVD_PREC_BF16 || prec == RSVD_PREC_BF16X3);
  const int final_prec = csr_compact ? RSVD_PREC_FP32
                         : ((prec == RSVD_PREC_BF16 || prec == RSVD_PREC_FP8) && P->refine) ? RSVD_PREC_BF16X3
                                                                                             : prec;
  Profiler& pf = P->prof;
  // BF16 plans in core stream a BF16 copy of A after the first plain forward
  // pass has written it: half the bytes per pass, the same operands.  BF16X3
  // plans keep the split copy (hi and lo parts, 4 bytes per entry like the
  // FP32 A) so that their later passes move the operands without converting.
  bool use16 = false;
  const bool split_copy = prec == RSVD_PREC_BF16X3;
  // A stored in 16 bits by the caller (Section 3.2): every pass reads it as is
  const bool a16_in = A.kind == RSVD_DENSE && (A.dtype == RSVD_BF16 || A.dtype == RSVD_F16);
  if constexpr (std::is_same<T, float>::value) {
    if ((prec == RSVD_PREC_BF16 || prec == RSVD_PREC_BF16X3) && A.kind == RSVD_DENSE && !a16_in &&
        !P->streaming && round_up(r, 16) <= (split_copy ? 192 : 256)) {
      const int64_t ld16 = round_up(n, 64);
      const size_t need = (size_t)m * ld16 * sizeof(uint16_t) * (split_copy ? 2 : 1);
      const bool fits = P->mem_cap == 0 || P->ws_bytes + P->a_copy_bytes + need <= P->mem_cap;
      if (fits && P->a16_bytes < need) {
        if (P->a16) cudaFree(P->a16);
        P->a16 = nullptr;
        P->a16_bytes = 0;
        if (cudaMalloc(reinterpret_cast<void**>(&P->a16), need) == cudaSuccess) {
          P->a16_bytes = need;
        } else {
          (void)cudaGetLastError();  // no room: the passes read the FP32 A (same results)
          P->a16 = nullptr;
        }
      }
      use16 = fits && P->a16 && P->a16_bytes >= need;
      P->a16_ld = ld16;
    }
  }
  P->a16_ready = false;
  // A copied from the host in chunks: the first forward pass may take the
  // chunks as they land; any other use of A waits for the whole copy
  auto await_copy = [&]() -> rsvd_status {
    if (P->h2d_pending) {
      RSVD_CUDA(cudaStreamWaitEvent(st, P->h2d_ev[P->h2d_chunks], 0));
      P->h2d_pending = false;
    }
    return RSVD_OK;
  };
  // the first forward pass over A chunk by chunk (rows [r0, r0 + rows)), each
  // chunk after its copy: the same products per row as one pass over A
  auto chunked_forward = [&](int pr, const T* Xin, T* Yout, bool& done) -> rsvd_status {
    done = false;
    if (!P->h2d_pending || P->streaming || A.kind != RSVD_DENSE || pr == RSVD_PREC_FP8) return RSVD_OK;
    const size_t esz = elem_size(A.dtype);
    uint16_t* lo = (prec == RSVD_PREC_BF16X3 && P->a16) ? P->a16 + (size_t)m * P->a16_ld : nullptr;
    const bool write_copy = use16 && pr == prec && !P->a16_ready;
    // every chunk takes the K split of the whole pass: the same sums per row
    const int64_t kps = tc_ksteps_per_split(m, n, r, 0, pr);
    for (int c = 0; c < P->h2d_chunks; ++c) {
      const int64_t r0 = (int64_t)c * P->h2d_chunk_rows, rows = std::min<int64_t>(P->h2d_chunk_rows, m - r0);
      RSVD_CUDA(cudaStreamWaitEvent(st, P->h2d_ev[c], 0));
      rsvd_matrix Ac = A;
      Ac.m = rows;
      Ac.data = static_cast<const char*>(A.data) + (size_t)r0 * A.ld * esz;
      T* Yc = Yout + (size_t)r0 * ldr;
      if constexpr (std::is_same<T, float>::value) {
        if (write_copy) {
          RSVD_TRY(tc_apass_from_f32(Ac, 0, pr, r, Xin, ldr, Yc, ldr, P->mb, P->nb, P->apass_ws, P->apass_ws_bytes,
                                     P->status, st, false, P->a16 + (size_t)r0 * P->a16_ld, P->a16_ld,
                                     lo ? lo + (size_t)r0 * P->a16_ld : nullptr, kps));
          continue;
        }
        if (a16_in) {
          Bf16Source b;
          b.data = static_cast<const uint16_t*>(Ac.data); b.m = rows; b.n = n; b.ld = A.ld;
          b.f16 = A.dtype == RSVD_F16 ? 1 : 0;
          RSVD_TRY(tc_apass_from_16(b, 0, pr, r, Xin, ldr, Yc, ldr, P->apass_ws, P->apass_ws_bytes, P->status, st,
                                    false, kps));
          continue;
        }
        if (pr == RSVD_PREC_BF16 || pr == RSVD_PREC_BF16X3) {
          RSVD_TRY(tc_apass_from_f32(Ac, 0, pr, r, Xin, ldr, Yc, ldr, P->mb, P->nb, P->apass_ws, P->apass_ws_bytes,
                                     P->status, st, false, nullptr, 0, nullptr, kps));
          continue;
        }
      }
      RSVD_TRY(apass_dense(Ac, 0, pr, r, Xin, ldr, Yc, ldr, P->mb, P->nb, P->apass_ws, P->apass_ws_bytes,
                           P->status, st));
    }
    if (write_copy) P->a16_ready = true;
    P->h2d_pending = false;  // every chunk has been waited for
    done = true;
    return RSVD_OK;
  };
  auto apass = [&](int trans, int pr, const T* Xin, T* Yout) -> rsvd_status {
    Span sp(pf, trans ? RSVD_STAGE_APASS_TRANS : RSVD_STAGE_APASS_FWD, st);
    ++pf.apass_calls;
    if (!trans && P->h2d_pending) {
      bool done = false;
      RSVD_TRY(chunked_forward(pr, Xin, Yout, done));
      if (done) return RSVD_OK;
    }
    RSVD_TRY(await_copy());
    if constexpr (std::is_same<T, float>::value) {
      if (a16_in) {
        Bf16Source b;
        b.data = static_cast<const uint16_t*>(A.data); b.m = m; b.n = n; b.ld = A.ld;
        b.f16 = A.dtype == RSVD_F16 ? 1 : 0;
        return tc_apass_from_16(b, trans, pr, r, Xin, ldr, Yout, ldr, P->apass_ws, P->apass_ws_bytes, P->status, st);
      }
      if (use16 && pr == prec) {
        uint16_t* lo = split_copy ? P->a16 + (size_t)m * P->a16_ld : nullptr;
        if (P->a16_ready) {
          Bf16Source b;
          b.data = P->a16; b.m = m; b.n = n; b.ld = P->a16_ld; b.lo = lo;
          return tc_apass_from_16(b, trans, pr, r, Xin, ldr, Yout, ldr, P->apass_ws, P->apass_ws_bytes, P->status,
                                  st);
        }
        if (!trans) {
          RSVD_TRY(tc_apass_from_f32(A, 0, pr, r, Xin, ldr, Yout, ldr, P->mb, P->nb, P->apass_ws,
                                     P->apass_ws_bytes, P->status, st, false, P->a16, P->a16_ld, lo));
          P->a16_ready = true;
          return RSVD_OK;
        }
      }
    }
    if constexpr (std::is_same<T, float>::value) {
      if (A.kind == RSVD_CSR) {
        // Section 3.3: sparse x dense; A^T through the CSR of A^T.  BF16 and
        // BF16X3 passes gather the panel rounded to 16 or 24 bits.
        SpmmPanel px;
        px.f = Xin;
        px.ld = ldr;
        if (pr == RSVD_PREC_BF16 || pr == RSVD_PREC_BF16X3) {
          px.fmt = pr == RSVD_PREC_BF16 ? 1 : 2;
          RSVD_TRY(spmm_pack(px.fmt, trans ? m : n, r, Xin, ldr, P->pk_h, P->pk_24, ldr, st));
          px.f = nullptr;
          px.h = P->pk_h;
          px.p24 = P->pk_24;
          px.rb = spmm_p24_row_bytes(ldr);
        }
        if (P->csr_streaming)  // Sections 3.5, 3.7: CSR tiles streamed from the host
          return csr_apass_streamed(P->cs, trans, r, px, Yout, ldr, st);
        return trans ? spmm_csr_panel(n, r, A.t_rowptr, A.t_colidx, A.t_val, A.nnz, px, Yout, ldr, false,
                                      P->spmm_ws, P->spmm_ws_bytes, st)
                     : spmm_csr_panel(m, r, A.rowptr, A.colidx, A.val, A.nnz, px, Yout, ldr, false, P->spmm_ws,
                                      P->spmm_ws_bytes, st);
      }
    }
    if (P->streaming) return apass_streamed(P->ss, A, trans, pr, r, Xin, Yout, ldr, P->status, st);
    if constexpr (std::is_same<T, float>::value) {
      if (pr == RSVD_PREC_FP8)
        return tc_apass_from_fp8(P->f8, trans, r, Xin, ldr, Yout, ldr, P->apass_ws, P->apass_ws_bytes, P->status, st);
    }
    return apass_dense(A, trans, pr, r, Xin, ldr, Yout, ldr, P->mb, P->nb, P->apass_ws, P->apass_ws_bytes,
                       P->status, st);
  };
  // Range-finder bases only carry the sketch's span to the next product: one
  // CholeskyQR sweep for them; the final Q, whose orthonormality enters
  // B = Q^T A, takes both sweeps
  auto orth = [&](int64_t M, const T* Yin, T* Qout, bool final_q) -> rsvd_status {
    Span sp(pf, RSVD_STAGE_ORTH, st);
    const bool tc = P->tc_orth_all || (P->tc_orth_inner && !final_q);
    const bool one = !final_q;
    return orth_panel<T>(M, r, Yin, ldr, Qout, ldr, nullptr, P->orth, st, tc, one);
  };
  // Section 3.8 persistence: the header of each checkpoint places its basis in
  // the execution plan; a matching checkpoint lets the run skip its steps.
  const bool ckpt_on = !P->ckpt_path.empty() && !P->auto_q && !P->fused;
  CkptHeader hdr;
  std::memset(&hdr, 0, sizeof(hdr));
  int first_step = 0;
  P->resumed_from = -1;
  if (ckpt_on) {
    hdr.m = m; hdr.n = n; hdr.k = k; hdr.p = P->p; hdr.q = P->q; hdr.r = r; hdr.ldr = ldr;
    hdr.prec = prec; hdr.dtype = P->dtype; hdr.kind = A.kind; hdr.seed = P->seed;
    RSVD_TRY(await_copy());
    RSVD_TRY(matrix_fingerprint(A, &hdr.fingerprint, st));
    const int done = ckpt_try_load(P->ckpt_path, hdr, Q, X, st);
    if (done >= 0) {
      first_step = done + 1;
      P->resumed_from = done;
    }
  }
  auto checkpoint = [&](int step) -> rsvd_status {
    if (!ckpt_on) return RSVD_OK;
    CkptHeader h = hdr;
    h.step = step;
    h.panel_rows = (step % 2 == 0) ? m : n;
    h.panel_bytes = (uint64_t)h.panel_rows * ldr * (P->dtype == RSVD_F64 ? 8 : 4);
    RSVD_TRY(read_device_status(P->status, st));  // never persist a basis from a failed step
    RSVD_TRY(ckpt_save(P->ckpt_path, h, (step % 2 == 0) ? (const void*)Q : (const void*)X, st));
    if (P->ckpt_stop_after == step)
      return fail(RSVD_ERR_INTERRUPTED, "rsvd_run: stopped after checkpoint step " + std::to_string(step));
    return RSVD_OK;
  };
  {
    Span total(pf, RSVD_STAGE_TOTAL, st);
    RSVD_CUDA(cudaMemsetAsync(P->status, 0, 4 * sizeof(int), st));
    if (first_step == 0) {  // step 1: Gaussian test matrix (n x r); X may hold a resumed Z otherwise
      Span sp(pf, RSVD_STAGE_GAUSSIAN, st);
      // BF16-valued test matrices for the tensor-core and BF16-panel paths; the
      // 24-bit panels of CSR BF16X3 plans round an FP32 test matrix
      const bool bf16_panel = A.kind == RSVD_CSR ? prec == RSVD_PREC_BF16
                                                 : (prec == RSVD_PREC_BF16 || prec == RSVD_PREC_BF16X3 ||
                                                    prec == RSVD_PREC_FP8);
      RSVD_TRY(launch_gaussian(P->seed, n, r, bf16_panel ? kF32HoldingBf16 : P->dtype, 0, X, ldr, st));
    }
    if constexpr (std::is_same<T, float>::value) {
      if (prec == RSVD_PREC_FP8) {  // E4M3 codes of A with tile scales, once per run
        Span sp(pf, RSVD_STAGE_QUANTIZE, st);
        RSVD_TRY(await_copy());
        RSVD_TRY(fp8_quantize(static_cast<const float*>(A.data), m, n, A.ld, P->f8.qm, P->f8.qn,
                              const_cast<uint8_t*>(P->f8.codes), P->f8.ldc, const_cast<float*>(P->f8.scales),
                              P->f8_amax, st));
      }
    }
    // step 2 and steps 3-4: Y = A O, Q = orth(Y) (range-finder step 0), unless
    // a checkpoint of this plan and this A lets the run resume later
    if (first_step == 0 && !P->fused) {
      RSVD_TRY(apass(0, prec, X, Y));
      RSVD_TRY(orth(m, Y, Q, P->q == 0));
      RSVD_TRY(checkpoint(0));
    }
    auto small_svd = [&]() -> rsvd_status {  // step 6 on the current B^T
      Span sp(pf, RSVD_STAGE_SMALL_SVD, st);
      RSVD_TRY(orth_panel<T>(n, r, Bt, ldr, Qb, ldr, P->R, P->orth, st));
      // FP32 outputs: off-diagonals below 1e-11 r (relative) change sigma by their
      // square and the vectors by them over the relative gap, both far below the
      // FP32 rounding of U, S, V; FP64 outputs take the FP64 test (r eps).  BF16
      // and FP8 products carry errors of order 2^-8 relative, so the FP32
      // convergence (r eps32, sigma moved by ~1e-10) is already far below them
      // and the FP64 sweeps are left out.
      const bool low = prec == RSVD_PREC_BF16 || prec == RSVD_PREC_FP8;
      return jacobi_svd(r, r, P->R, P->sigma, P->UR, P->WR, P->jac, st,
                        P->dtype == RSVD_F64 ? 0.0 : 1e-11 * (double)r, !low);
    };
    bool have_final = false;  // Bt, Qb, R and the small SVD already hold the final result
    P->q_used = P->q;
    if (P->fused) {
      // Eq. (3) right to left with the products A^T (A W) grouped per sweep
      // and only the n-side orthonormalised: W = O; q times W = orth(A^T (A W));
      // then Q = orth(A W).  Streamed, each sweep reads every row panel once.
      const int prec_t = sweep_trans_prec(prec);
      for (int i = 0; i < P->q; ++i) {
        if (P->streaming) {
          Span sp(pf, RSVD_STAGE_SWEEP, st);
          ++pf.apass_calls;
          RSVD_TRY(sweep_streamed(P->ss, A, prec, prec_t, r, X, Bt, ldr, P->status, st));
        } else {
          RSVD_TRY(apass(0, prec, X, Y));
          RSVD_TRY(apass(1, prec_t, Y, Bt));
        }
        RSVD_TRY(orth(n, Bt, X, false));
      }
      RSVD_TRY(apass(0, prec, X, Y));
      RSVD_TRY(orth(m, Y, Q, true));
    } else if (!P->auto_q) {
      // Eq. (3), right to left: q times Z = orth(A^T Q), Q = orth(A Z); step
      // 2i+1 leaves Z in X, step 2i+2 leaves Q (checkpointed when enabled)
      for (int s = first_step > 0 ? first_step : 1; s <= 2 * P->q; ++s) {
        if (s & 1) {
          RSVD_TRY(apass(1, prec, Q, Bt));
          RSVD_TRY(orth(n, Bt, X, false));
        } else {
          RSVD_TRY(apass(0, prec, X, Y));
          RSVD_TRY(orth(m, Y, Q, s == 2 * P->q));
        }
        RSVD_TRY(checkpoint(s));
      }
    } else {
      // Section 2.2, automatic iteration parameter: after each power iteration
      // the small SVD of B_i^T = A^T Q_i gives sigma^(i); stop once
      // ||sigma^(i) - sigma^(i-1)|| / ||sigma^(i)|| (top k) <= tol, or at q.  The
      // next basis is Q_b of that small SVD (= orth(A^T Q_i)), so the
      // monitoring costs one small SVD per iteration and no extra pass.
      int it = 0;
      for (;; ++it) {
        RSVD_TRY(apass(1, prec, Q, Bt));
        RSVD_TRY(small_svd());
        if (it > 0) {
          RSVD_TRY(sigma_change_below(k, P->sigma, P->sigma_prev, P->auto_q_tol, P->q_flag, st));
          int h = 0;
          RSVD_CUDA(cudaMemcpyAsync(&h, P->q_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
          RSVD_CUDA(cudaStreamSynchronize(st));
          if (h) break;
        }
        if (it == P->q) break;
        RSVD_CUDA(cudaMemcpyAsync(P->sigma_prev, P->sigma, (size_t)r * sizeof(double), cudaMemcpyDeviceToDevice, st));
        RSVD_TRY(apass(0, prec, Qb, Y));
        RSVD_TRY(orth(m, Y, Q, true));  // any Q may turn out to be the final one
      }
      P->q_used = it;
      have_final = final_prec == prec;  // else recompute B^T in the refinement precision
    }
    if (!have_final) {
      // step 5: B^T = A^T Q
      RSVD_TRY(apass(1, final_prec, Q, Bt));
      // step 6: B^T = Q_b R, R^T = U_R diag(sigma) W^T  =>  B = U_R diag(sigma) (Q_b W)^T
      RSVD_TRY(small_svd());
    }
    {  // step 7: U = Q U_R[:, :k], V = Q_b W[:, :k]
      Span sp(pf, RSVD_STAGE_LIFT, st);
      T* URk = static_cast<T*>(P->URk);
      T* WRk = static_cast<T*>(P->WRk);
      RSVD_TRY((convert_matrix<double, T>(r, k, P->UR, r, URk, k, st)));
      RSVD_TRY((convert_matrix<double, T>(r, k, P->WR, r, WRk, k, st)));
      bool tc_lift = false;
      if constexpr (std::is_same<T, float>::value) {
        // BF16-family plans lift on the tensor cores in split BF16 (about 16
        // significant bits per operand, far below their products' errors);
        // FP32 plans keep the FP32 SIMT product
        tc_lift = (prec == RSVD_PREC_BF16 || prec == RSVD_PREC_BF16X3 || prec == RSVD_PREC_FP8) &&
                  P->lift_ws_bytes >= tc_gemm_wide_ws_bytes(m > n ? m : n, r, k, RSVD_PREC_BF16X3);
        if (tc_lift) {
          rsvd_matrix Qm{}, Qbm{};
          Qm.kind = Qbm.kind = RSVD_DENSE;
          Qm.dtype = Qbm.dtype = RSVD_F32;
          Qm.location = Qbm.location = RSVD_ON_DEVICE;
          Qm.m = m; Qm.n = r; Qm.data = Q; Qm.ld = ldr;
          Qbm.m = n; Qbm.n = r; Qbm.data = Qb; Qbm.ld = ldr;
          RSVD_TRY(tc_gemm_wide(Qm, RSVD_PREC_BF16X3, k, URk, k, U, k, P->lift_ws, P->lift_ws_bytes, P->status, st));
          RSVD_TRY(tc_gemm_wide(Qbm, RSVD_PREC_BF16X3, k, WRk, k, V, k, P->lift_ws, P->lift_ws_bytes, P->status,
                                st));
        }
      }
      if (!tc_lift) {
        RSVD_TRY(simt_gemm<T>(m, k, r, Q, ldr, false, URk, k, U, k, false, 1, r, nullptr, st));
        RSVD_TRY(simt_gemm<T>(n, k, r, Qb, ldr, false, WRk, k, V, k, false, 1, r, nullptr, st));
      }
      RSVD_TRY((convert_matrix<double, T>(1, k, P->sigma, k, S, k, st)));
      RSVD_TRY(normalise_signs<T>(m, n, k, U, k, V, k, P->sign_scratch, P->sign_scratch_bytes, st));
    }
  }
  const rsvd_status res = read_device_status(P->status, st);
  if (pf.on) pf.collect();
  if (res == RSVD_OK && ckpt_on) std::remove(P->ckpt_path.c_str());  // the run is complete
  return res;
}

// Make a device CSR descriptor (with the CSR of A^T) for rsvd_run.  Device
// arrays of A are used in place; host arrays, and a transpose the library
// builds on the host, are copied into the plan's CSR buffer (kept between
// runs and grown when needed).
rsvd_status prepare_csr(rsvd_plan_s* P, const rsvd_matrix& A, rsvd_matrix* out, cudaStream_t st) {
  const int64_t m = A.m, n = A.n, nnz = A.nnz;
  if (nnz < 0 || nnz > 0x7fffffffLL || !A.rowptr || (nnz > 0 && (!A.colidx || !A.val)))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: bad CSR descriptor (nnz, rowptr, colidx, val)");
  if (A.dtype != RSVD_F32) return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: CSR values must be F32");
  const bool host = A.location == RSVD_ON_HOST;
  const bool have_t = A.t_rowptr != nullptr;
  if (have_t && nnz > 0 && (!A.t_colidx || !A.t_val))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: t_rowptr set without t_colidx/t_val");
  *out = A;
  out->location = RSVD_ON_DEVICE;
  // device bytes needed: A's arrays when on the host, the transpose when on the host or built here
  const size_t a_bytes = host ? (size_t)(m + 1) * 4 + (size_t)nnz * 8 : 0;
  const size_t t_bytes = (host || !have_t) ? (size_t)(n + 1) * 4 + (size_t)nnz * 8 : 0;
  const size_t sws = spmm_ws_bytes(nnz, P->r);
  const size_t need = a_bytes + t_bytes + sws + 1024;
  // Section 3.5: a host CSR whose copies do not fit under the cap is processed
  // out of core, its tiles (and those of its transpose) streamed per pass; so
  // is a host CSR for which the options set tile edges (Section 3.1: the
  // blocks of the block-cyclic map, resident after the first pass when they
  // all fit)
  const bool stream_it =
      host && ((P->mem_cap && P->ws_bytes + need > P->mem_cap) || P->mb_req > 0 || P->nb_req > 0);
  // host views of the transpose's source, and of the transpose
  const int32_t *hrp = nullptr, *hci = nullptr;
  const float* hv = nullptr;
  std::vector<int32_t> tmp_idx;
  std::vector<float> tmp_val;
  if (!have_t) {
    if (host) {
      hrp = A.rowptr; hci = A.colidx; hv = A.val;
    } else {  // bring A to the host to build its transpose
      tmp_idx.resize((size_t)(m + 1) + (size_t)nnz);
      tmp_val.resize((size_t)nnz);
      RSVD_CUDA(cudaMemcpyAsync(tmp_idx.data(), A.rowptr, (size_t)(m + 1) * 4, cudaMemcpyDeviceToHost, st));
      if (nnz) {
        RSVD_CUDA(cudaMemcpyAsync(tmp_idx.data() + m + 1, A.colidx, (size_t)nnz * 4, cudaMemcpyDeviceToHost, st));
        RSVD_CUDA(cudaMemcpyAsync(tmp_val.data(), A.val, (size_t)nnz * 4, cudaMemcpyDeviceToHost, st));
      }
      RSVD_CUDA(cudaStreamSynchronize(st));
      hrp = tmp_idx.data(); hci = tmp_idx.data() + m + 1; hv = tmp_val.data();
    }
    if (hrp[m] != nnz) return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: rowptr[m] != nnz");
    int32_t* ti;
    float* tv;
    if (stream_it) {  // pinned, for copies that overlap the products
      if (P->h_tpinned_nnz < (size_t)nnz || P->h_tpinned_n != n) {
        if (P->h_tpinned) cudaFreeHost(P->h_tpinned);
        if (P->h_tval_pinned) cudaFreeHost(P->h_tval_pinned);
        P->h_tpinned = nullptr;
        P->h_tval_pinned = nullptr;
        P->h_tpinned_nnz = 0;
        RSVD_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->h_tpinned), ((size_t)n + 1 + (size_t)nnz) * 4,
                                cudaHostAllocDefault));
        RSVD_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&P->h_tval_pinned), (size_t)nnz * 4 + 4,
                                cudaHostAllocDefault));
        P->h_tpinned_nnz = (size_t)nnz;
        P->h_tpinned_n = n;
      }
      ti = P->h_tpinned;
      tv = P->h_tval_pinned;
    } else {
      P->h_idx.resize((size_t)(n + 1) + (size_t)nnz);
      P->h_val.resize((size_t)nnz);
      ti = P->h_idx.data();
      tv = P->h_val.data();
    }
    RSVD_TRY(csr_transpose_host(m, n, hrp, hci, hv, ti, ti + n + 1, tv));
  } else if (host && A.rowptr[m] != nnz) {
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: rowptr[m] != nnz");
  }
  if (stream_it) {
    size_t budget = 0;
    if (P->mem_cap) {
      if (P->ws_bytes >= P->mem_cap) return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_run: no room left for streaming");
      budget = P->mem_cap - P->ws_bytes;
    } else {  // no cap: the device memory free now, less a margin for the caller
      size_t free_b = 0, total_b = 0;
      RSVD_CUDA(cudaMemGetInfo(&free_b, &total_b));
      budget = free_b > ((size_t)1 << 30) ? free_b - ((size_t)1 << 30) : free_b / 2;
    }
    rsvd_matrix H = A;
    if (!have_t) {  // the transpose built above, in pinned host memory
      H.t_rowptr = P->h_tpinned;
      H.t_colidx = P->h_tpinned + n + 1;
      H.t_val = P->h_tval_pinned;
    }
    RSVD_TRY(csr_stream_prepare(&P->cs, H, P->mb_req, P->nb_req, P->n_slots, budget, P->r));
    csr_stream_begin_run(P->cs);
    P->csr_streaming = true;
    *out = H;
    return RSVD_OK;
  }
  {
    if (P->mem_cap && P->ws_bytes + need > P->mem_cap)
      return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_run: the CSR copies and SpMM workspace do not fit under mem_cap");
    if (P->csr_dev_bytes < need) {
      if (P->csr_dev) cudaFree(P->csr_dev);
      P->csr_dev = nullptr;
      P->csr_dev_bytes = 0;
      RSVD_CUDA(cudaMalloc(&P->csr_dev, need));
      P->csr_dev_bytes = need;
    }
    Carver c(P->csr_dev, P->csr_dev_bytes);
    P->spmm_ws = c.take<char>(sws);
    P->spmm_ws_bytes = sws;
    if (host) {
      int32_t* rp = c.take<int32_t>((size_t)m + 1);
      int32_t* ci = c.take<int32_t>((size_t)nnz);
      float* v = c.take<float>((size_t)nnz);
      Span sp(P->prof, RSVD_STAGE_H2D, st);
      RSVD_CUDA(cudaMemcpyAsync(rp, A.rowptr, (size_t)(m + 1) * 4, cudaMemcpyHostToDevice, st));
      if (nnz) {
        RSVD_CUDA(cudaMemcpyAsync(ci, A.colidx, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
        RSVD_CUDA(cudaMemcpyAsync(v, A.val, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
      }
      out->rowptr = rp; out->colidx = ci; out->val = v;
    }
    if (t_bytes) {
      int32_t* trp = c.take<int32_t>((size_t)n + 1);
      int32_t* tci = c.take<int32_t>((size_t)nnz);
      float* tv = c.take<float>((size_t)nnz);
      const int32_t* s_rp = have_t ? A.t_rowptr : P->h_idx.data();
      const int32_t* s_ci = have_t ? A.t_colidx : P->h_idx.data() + n + 1;
      const float* s_v = have_t ? A.t_val : P->h_val.data();
      Span sp(P->prof, RSVD_STAGE_H2D, st);
      RSVD_CUDA(cudaMemcpyAsync(trp, s_rp, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, st));
      if (nnz) {
        RSVD_CUDA(cudaMemcpyAsync(tci, s_ci, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
        RSVD_CUDA(cudaMemcpyAsync(tv, s_v, (size_t)nnz * 4, cudaMemcpyHostToDevice, st));
      }
      out->t_rowptr = trp; out->t_colidx = tci; out->t_val = tv;
    }
  }
  return RSVD_OK;
}

}  // namespace

namespace {

// rsvd_full for the larger shapes: T = A (m >= n) or A^T (m < n), rows x cols
// with cols = min(m, n) <= 512, in FP64.  T = Q R by CholeskyQR2, R^T W =
// U_J diag(s) by the square one-sided Jacobi (the column-major view of the
// row-major R is R^T), so T = (Q W) diag(s) U_J^T: the left singular vectors
// of T are Q W, the right ones U_J.
rsvd_status full_svd_tall(const rsvd_matrix& A, void* U, void* S, void* V, cudaStream_t st) {
  const int64_t m = A.m, n = A.n;
  const int64_t rows = m >= n ? m : n;
  const int cols = (int)(m >= n ? n : m);
  const size_t rc = (size_t)rows * cols, cc = (size_t)cols * cols;
  const size_t ob = orth_ws_bytes(rows, cols, RSVD_F64, false);
  const size_t jb = jacobi_ws_bytes(cols, cols);
  const size_t sb = sign_scratch_bytes(m, cols);
  Sizer sz;
  sz.take<double>(rc); sz.take<double>(rc); sz.take<double>(rc);
  sz.take<double>(cc); sz.take<double>(cols); sz.take<double>(cc); sz.take<double>(cc);
  sz.take<char>(ob); sz.take<char>(jb); sz.take<char>(sb);
  const size_t total = sz.used + 1024;
  void* ws = nullptr;
  RSVD_CUDA(cudaMalloc(&ws, total));
  Carver c(ws, total);
  double* T = c.take<double>(rc);
  double* Q = c.take<double>(rc);
  double* UA = c.take<double>(rc);
  double* R = c.take<double>(cc);
  double* sig = c.take<double>(cols);
  double* UJ = c.take<double>(cc);
  double* W = c.take<double>(cc);
  char* obase = c.take<char>(ob);
  char* jbase = c.take<char>(jb);
  void* sc = c.take<char>(sb);
  Carver oc(obase, ob), jc(jbase, jb);
  OrthWs ow = orth_ws_carve(oc, rows, cols, RSVD_F64, false);
  JacobiWs jw = jacobi_ws_carve(jc, cols, cols);
  rsvd_status s = RSVD_OK;
  auto run = [&]() -> rsvd_status {
    RSVD_CUDA(cudaMemsetAsync(ow.status, 0, sizeof(int), st));
    RSVD_CUDA(cudaMemsetAsync(jw.status, 0, sizeof(int), st));
    // row-major FP64 T: T[i][c] = A[i][c] (m >= n) or A[c][i] (m < n), written
    // as the column-major cols x rows gather
    if (A.dtype == RSVD_F64)
      RSVD_TRY(gather_colmajor_f64<double>(cols, rows, static_cast<const double*>(A.data), m >= n ? 1 : A.ld,
                                           m >= n ? A.ld : 1, T, st));
    else
      RSVD_TRY(gather_colmajor_f64<float>(cols, rows, static_cast<const float*>(A.data), m >= n ? 1 : A.ld,
                                          m >= n ? A.ld : 1, T, st));
    RSVD_TRY(orth_panel<double>(rows, cols, T, cols, Q, cols, R, ow, st, false));
    RSVD_TRY(jacobi_svd(cols, cols, R, sig, UJ, W, jw, st));
    RSVD_TRY(simt_gemm<double>(rows, cols, cols, Q, cols, false, W, cols, UA, cols, false, 1, cols, nullptr, st));
    const double* Usrc = m >= n ? UA : UJ;  // m x t
    const double* Vsrc = m >= n ? UJ : UA;  // n x t
    if (A.dtype == RSVD_F64) {
      double* Ud = static_cast<double*>(U);
      double* Vd = static_cast<double*>(V);
      RSVD_TRY((convert_matrix<double, double>(m, cols, Usrc, cols, Ud, cols, st)));
      RSVD_TRY((convert_matrix<double, double>(n, cols, Vsrc, cols, Vd, cols, st)));
      RSVD_TRY((convert_matrix<double, double>(1, cols, sig, cols, static_cast<double*>(S), cols, st)));
      RSVD_TRY(normalise_signs<double>(m, n, cols, Ud, cols, Vd, cols, sc, sb, st));
    } else {
      float* Uf = static_cast<float*>(U);
      float* Vf = static_cast<float*>(V);
      RSVD_TRY((convert_matrix<double, float>(m, cols, Usrc, cols, Uf, cols, st)));
      RSVD_TRY((convert_matrix<double, float>(n, cols, Vsrc, cols, Vf, cols, st)));
      RSVD_TRY((convert_matrix<double, float>(1, cols, sig, cols, static_cast<float*>(S), cols, st)));
      RSVD_TRY(normalise_signs<float>(m, n, cols, Uf, cols, Vf, cols, sc, sb, st));
    }
    RSVD_TRY(read_device_status(ow.status, st));
    return read_device_status(jw.status, st);
  };
  s = run();
  cudaStreamSynchronize(st);
  cudaFree(ws);
  return s;
}

}  // namespace

namespace rsvd {
namespace {

// Row chunks of about 256 MB (whole 128-row tiles) of a dense host A copied to
// dst (rows of ldd elements) on the plan's copy stream, one event after each
// chunk (ev[c]) and one after the last (ev[chunks]); ev[chunks + 1] orders the
// copies after the work queued on `after` when that is given.
rsvd_status copy_host_chunks(rsvd_plan_t P, const rsvd_matrix& A, void* dst, int64_t ldd,
                             std::vector<cudaEvent_t>& ev, cudaStream_t after, bool wait_after,
                             int64_t* chunk_rows, int* chunks) {
  const size_t esz = elem_size(A.dtype);
  const size_t row = (size_t)A.n * esz;
  const size_t dpitch = (size_t)ldd * esz, spitch = (size_t)A.ld * esz;
  int64_t crow = (int64_t)(((size_t)256 << 20) / std::max<size_t>(dpitch, 1));
  crow = std::max<int64_t>(128, crow / 128 * 128);
  const int nch = (int)cdiv(A.m, crow);
  if (!P->h2d_stream) RSVD_CUDA(cudaStreamCreateWithFlags(&P->h2d_stream, cudaStreamNonBlocking));
  while ((int)ev.size() < nch + 2) {
    cudaEvent_t e;
    RSVD_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ev.push_back(e);
  }
  if (wait_after) {
    RSVD_CUDA(cudaEventRecord(ev[nch + 1], after));
    RSVD_CUDA(cudaStreamWaitEvent(P->h2d_stream, ev[nch + 1], 0));
  }
  for (int c = 0; c < nch; ++c) {
    const int64_t r0 = (int64_t)c * crow, rows = std::min<int64_t>(crow, A.m - r0);
    RSVD_CUDA(cudaMemcpy2DAsync(static_cast<char*>(dst) + (size_t)r0 * dpitch, dpitch,
                                static_cast<const char*>(A.data) + (size_t)r0 * spitch, spitch, row, rows,
                                cudaMemcpyHostToDevice, P->h2d_stream));
    RSVD_CUDA(cudaEventRecord(ev[c], P->h2d_stream));
  }
  RSVD_CUDA(cudaEventRecord(ev[nch], P->h2d_stream));
  *chunk_rows = crow;
  *chunks = nch;
  return RSVD_OK;
}

bool same_host_matrix(const rsvd_matrix& a, const rsvd_matrix& b) {
  return a.kind == b.kind && a.dtype == b.dtype && a.location == b.location && a.m == b.m && a.n == b.n &&
         a.ld == b.ld && a.data == b.data;
}

// Pending prefetches dropped: their copies complete in order on h2d_stream
// and their buffers are reused by later prefetches only.
void drop_prefetches(rsvd_plan_t P) {
  for (auto& e : P->pre) e.pending = false;
}

// Under a memory cap, a run that does not take a prefetch gives the room of
// the idle prefetch buffers back (their copies finish first).
void release_idle_prefetch_buffers(rsvd_plan_t P) {
  bool any = false;
  for (auto& e : P->pre) any |= !e.pending && e.dev;
  if (!any) return;
  if (P->h2d_stream) cudaStreamSynchronize(P->h2d_stream);
  for (auto& e : P->pre)
    if (!e.pending && e.dev) {
      cudaFree(e.dev);
      e.dev = nullptr;
      e.bytes = 0;
    }
}

}  // namespace
}  // namespace rsvd

extern "C" {

const char* rsvd_status_str(rsvd_status s) {
  switch (s) {
    case RSVD_OK: return "RSVD_OK";
    case RSVD_ERR_INVALID_ARG: return "RSVD_ERR_INVALID_ARG";
    case RSVD_ERR_OOM: return "RSVD_ERR_OOM";
    case RSVD_ERR_CAP_TOO_SMALL: return "RSVD_ERR_CAP_TOO_SMALL";
    case RSVD_ERR_CUDA: return "RSVD_ERR_CUDA";
    case RSVD_ERR_NOT_SPD: return "RSVD_ERR_NOT_SPD";
    case RSVD_ERR_NO_CONVERGE: return "RSVD_ERR_NO_CONVERGE";
    case RSVD_ERR_TIMEOUT: return "RSVD_ERR_TIMEOUT";
    case RSVD_ERR_UNSUPPORTED: return "RSVD_ERR_UNSUPPORTED";
    case RSVD_ERR_INTERRUPTED: return "RSVD_ERR_INTERRUPTED";
  }
  return "RSVD_ERR_UNKNOWN";
}

const char* rsvd_last_error(void) { return g_last_error.c_str(); }

rsvd_status rsvd_tile_map(int64_t m, int64_t n, int64_t mb, int64_t nb, int32_t n_slots, rsvd_tile* out,
                          int64_t cap, int64_t* count) {
  if (m < 0 || n < 0 || mb <= 0 || nb <= 0 || n_slots <= 0 || cap < 0 || !count)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_tile_map: bad arguments");
  const int64_t Tm = cdiv(m, mb), Tn = cdiv(n, nb);
  *count = Tm * Tn;
  if (cap > 0 && !out) return fail(RSVD_ERR_INVALID_ARG, "rsvd_tile_map: out is NULL");
  int64_t t = 0;
  for (int64_t I = 0; I < Tm && t < cap; ++I)
    for (int64_t J = 0; J < Tn && t < cap; ++J, ++t) {
      rsvd_tile& x = out[t];
      x.t = t; x.I = I; x.J = J;
      x.row0 = I * mb; x.row1 = (I + 1) * mb < m ? (I + 1) * mb : m;
      x.col0 = J * nb; x.col1 = (J + 1) * nb < n ? (J + 1) * nb : n;
      x.slot = t % n_slots;
    }
  return RSVD_OK;
}

size_t rsvd_spmm_workspace(int64_t nnz, int32_t r) { return spmm_ws_bytes(nnz < 0 ? 0 : nnz, r); }

size_t rsvd_csr_apass_workspace(int64_t nnz, int64_t K, int32_t r, int32_t prec) {
  if (r < 1 || K < 0) return 0;
  const size_t sws = spmm_ws_bytes(nnz < 0 ? 0 : nnz, r);
  if (prec != RSVD_PREC_BF16 && prec != RSVD_PREC_BF16X3) return sws;
  const int64_t ld = round_up(r, 4);
  Sizer z;
  z.take<char>(sws);
  if (prec == RSVD_PREC_BF16) z.take<uint16_t>((size_t)K * ld);
  else z.take<uint8_t>((size_t)K * spmm_p24_row_bytes(ld));
  return z.used + 256;
}

size_t rsvd_apass_workspace(int64_t m, int64_t n, int32_t r, int32_t trans, int32_t prec, int64_t mb,
                            int64_t nb) {
  if (prec == RSVD_PREC_FP8) {
    const int64_t qm = (mb <= 0 || mb >= m) ? m : round_up(mb, 128);
    const int64_t qn = (nb <= 0 || nb >= n) ? n : round_up(nb, 128);
    const int64_t tiles = cdiv(m, qm < m ? qm : m) * cdiv(n, qn < n ? qn : n);
    Sizer z;
    z.take<uint8_t>((size_t)m * round_up(n, 16));
    z.take<float>((size_t)tiles);
    z.take<unsigned>((size_t)tiles);
    z.take<int>(4);
    z.take<char>(tc_apass_ws_bytes(m, n, r, trans, RSVD_PREC_BF16, mb, nb));
    return z.used + 512;
  }
  return apass_ws_bytes(m, n, r, trans, prec, mb, nb) + 512;
}

rsvd_status rsvd_fp8_quantize(const rsvd_matrix* A, int64_t qm, int64_t qn, uint8_t* codes, int64_t ldc,
                              float* scales, void* stream) {
  if (!A || !codes || !scales || A->kind != RSVD_DENSE || A->dtype != RSVD_F32 || A->location != RSVD_ON_DEVICE ||
      A->ld < A->n || A->m < 1 || A->n < 1)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_fp8_quantize: need a dense F32 device matrix and outputs");
  if (!fp8_tiles_ok(A->m, A->n, qm, qn))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_fp8_quantize: tile edges must be multiples of 128 or cover the matrix");
  const int64_t cqm = qm > A->m ? A->m : qm, cqn = qn > A->n ? A->n : qn;
  const size_t tiles = (size_t)cdiv(A->m, cqm) * cdiv(A->n, cqn);
  cudaStream_t st = as_stream(stream);
  unsigned* amax = nullptr;
  RSVD_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&amax), tiles * sizeof(unsigned), st));
  const rsvd_status s = fp8_quantize(static_cast<const float*>(A->data), A->m, A->n, A->ld, cqm, cqn, codes, ldc,
                                     scales, amax, st);
  cudaFreeAsync(amax, st);
  return s;
}

rsvd_status rsvd_apass(const rsvd_matrix* A, int32_t trans, int32_t prec, int32_t r, const void* X,
                       int64_t ldx, void* Y, int64_t ldy, int64_t mb, int64_t nb, void* ws,
                       size_t ws_bytes, void* stream) {
  if (!A || !X || !Y || r < 1 || (trans != 0 && trans != 1) || ldx < r || ldy < r)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_apass: bad arguments");
  if (A->kind == RSVD_CSR) {
    if (r > kSpmmMaxR || A->dtype != RSVD_F32 || A->location != RSVD_ON_DEVICE ||
        (prec != RSVD_PREC_FP32 && prec != RSVD_PREC_BF16 && prec != RSVD_PREC_BF16X3))
      return fail(RSVD_ERR_INVALID_ARG,
                  "rsvd_apass: CSR needs a device F32 matrix, prec FP32, BF16 or BF16X3, r <= 512");
    const int32_t* rp = trans ? A->t_rowptr : A->rowptr;
    const int32_t* ci = trans ? A->t_colidx : A->colidx;
    const float* v = trans ? A->t_val : A->val;
    if (!rp || (A->nnz > 0 && (!ci || !v)))
      return fail(RSVD_ERR_INVALID_ARG, "rsvd_apass: CSR arrays missing (trans = 1 needs t_rowptr/t_colidx/t_val)");
    const int64_t M = trans ? A->n : A->m, K = trans ? A->m : A->n;
    SpmmPanel px;
    px.f = static_cast<const float*>(X);
    px.ld = ldx;
    void* sws = ws;
    size_t sws_bytes = ws_bytes;
    if (prec != RSVD_PREC_FP32) {
      // the workspace holds the split-row tasks, then the compact panel
      const size_t need = rsvd_csr_apass_workspace(A->nnz, K, r, prec);
      if (!ws || ws_bytes < need || reinterpret_cast<uintptr_t>(ws) % 16 != 0)
        return fail(RSVD_ERR_INVALID_ARG,
                    "rsvd_apass: CSR BF16 / BF16X3 passes need rsvd_csr_apass_workspace bytes, 16-byte aligned");
      const int64_t ld = round_up(r, 4);
      Carver c(ws, ws_bytes);
      sws_bytes = spmm_ws_bytes(A->nnz, r);
      sws = c.take<char>(sws_bytes);
      uint16_t* h = prec == RSVD_PREC_BF16 ? c.take<uint16_t>((size_t)K * ld) : nullptr;
      uint8_t* p24 = prec == RSVD_PREC_BF16X3 ? c.take<uint8_t>((size_t)K * spmm_p24_row_bytes(ld)) : nullptr;
      px.fmt = prec == RSVD_PREC_BF16 ? 1 : 2;
      RSVD_TRY(spmm_pack(px.fmt, K, r, static_cast<const float*>(X), ldx, h, p24, ld, as_stream(stream)));
      px.f = nullptr;
      px.h = h;
      px.p24 = p24;
      px.rb = spmm_p24_row_bytes(ld);
      px.ld = ld;
    }
    return spmm_csr_panel(M, r, rp, ci, v, A->nnz, px, static_cast<float*>(Y), ldy, false, sws, sws_bytes,
                          as_stream(stream));
  }
  if (r > 256) return fail(RSVD_ERR_INVALID_ARG, "rsvd_apass: r must not exceed 256 (dense)");
  if (A->kind == RSVD_DENSE && A->ld < A->n) return fail(RSVD_ERR_INVALID_ARG, "rsvd_apass: ld < n");
  if (prec == RSVD_PREC_FP8) {
    // quantise A (tiles mb x nb, rounded up to multiples of 128) into the
    // workspace, then the pass on the codes
    if (A->kind != RSVD_DENSE || A->dtype != RSVD_F32 || A->location != RSVD_ON_DEVICE)
      return fail(RSVD_ERR_INVALID_ARG, "rsvd_apass: FP8 needs a dense F32 device matrix");
    Fp8Source f;
    f.m = A->m; f.n = A->n; f.ldc = round_up(A->n, 16);
    f.qm = (mb <= 0 || mb >= A->m) ? A->m : round_up(mb, 128);
    f.qn = (nb <= 0 || nb >= A->n) ? A->n : round_up(nb, 128);
    if (f.qm > A->m) f.qm = A->m;
    if (f.qn > A->n) f.qn = A->n;
    const size_t need = rsvd_apass_workspace(A->m, A->n, r, trans, prec, mb, nb);
    if (!ws || ws_bytes < need) return fail(RSVD_ERR_INVALID_ARG, "rsvd_apass: workspace too small");
    Carver c(ws, ws_bytes);
    f.codes = c.take<uint8_t>((size_t)A->m * f.ldc);
    f.scales = c.take<float>((size_t)cdiv(A->m, f.qm) * cdiv(A->n, f.qn));
    unsigned* amax = c.take<unsigned>((size_t)cdiv(A->m, f.qm) * cdiv(A->n, f.qn));
    int* st_word = c.take<int>(4);
    const size_t tws = tc_apass_ws_bytes(A->m, A->n, r, trans, RSVD_PREC_BF16, mb, nb);
    void* tw = c.take<char>(tws);
    cudaStream_t st = as_stream(stream);
    RSVD_CUDA(cudaMemsetAsync(st_word, 0, 4 * sizeof(int), st));
    RSVD_TRY(fp8_quantize(static_cast<const float*>(A->data), A->m, A->n, A->ld, f.qm, f.qn,
                          const_cast<uint8_t*>(f.codes), f.ldc, const_cast<float*>(f.scales), amax, st));
    RSVD_TRY(tc_apass_from_fp8(f, trans, r, static_cast<const float*>(X), ldx, static_cast<float*>(Y), ldy, tw, tws,
                               st_word, st));
    return read_device_status(st_word, st);
  }
  if (prec == RSVD_PREC_BF16 || prec == RSVD_PREC_BF16X3) {
    // The tensor-core pipeline reports an expired wait through a device word:
    // this call synchronises the stream and returns it.
    const size_t need = apass_ws_bytes(A->m, A->n, r, trans, prec, mb, nb);
    if (ws_bytes < need + 512) return fail(RSVD_ERR_INVALID_ARG, "rsvd_apass: workspace too small");
    int* st_word = reinterpret_cast<int*>(static_cast<char*>(ws) + ((need + 255) & ~size_t(255)));
    cudaStream_t st = as_stream(stream);
    RSVD_CUDA(cudaMemsetAsync(st_word, 0, 4 * sizeof(int), st));
    RSVD_TRY(apass_dense(*A, trans, prec, r, X, ldx, Y, ldy, mb, nb, ws, need, st_word, st));
    return read_device_status(st_word, st);
  }
  return apass_dense(*A, trans, prec, r, X, ldx, Y, ldy, mb, nb, ws, ws_bytes, nullptr, as_stream(stream));
}

size_t rsvd_orth_workspace(int64_t M, int32_t r) { return orth_ws_bytes(M, r, RSVD_F64) + 1024; }

rsvd_status rsvd_orth(int32_t dtype, int64_t M, int32_t r, const void* Y, int64_t ldy, void* Q,
                      int64_t ldq, double* R, void* ws, size_t ws_bytes, void* stream) {
  if (r < 1 || r > 512 || M < r || ldy < r || ldq < r || !Y || !Q || (dtype != RSVD_F32 && dtype != RSVD_F64))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_orth: bad arguments");
  if (ws_bytes < rsvd_orth_workspace(M, r)) return fail(RSVD_ERR_INVALID_ARG, "rsvd_orth: workspace too small");
  Carver c(ws, ws_bytes);
  OrthWs w = orth_ws_carve(c, M, r, dtype);
  if (c.overflow) return fail(RSVD_ERR_INVALID_ARG, "rsvd_orth: workspace too small");
  cudaStream_t st = as_stream(stream);
  RSVD_CUDA(cudaMemsetAsync(w.status, 0, 4 * sizeof(int), st));
  if (dtype == RSVD_F64) {
    RSVD_TRY(orth_panel<double>(M, r, static_cast<const double*>(Y), ldy, static_cast<double*>(Q), ldq, R, w, st));
  } else {
    RSVD_TRY(orth_panel<float>(M, r, static_cast<const float*>(Y), ldy, static_cast<float*>(Q), ldq, R, w, st));
  }
  return read_device_status(w.status, st);
}

size_t rsvd_small_svd_workspace(int32_t r) { return jacobi_ws_bytes(r, r) + 512; }

rsvd_status rsvd_small_svd(int32_t r, const double* Mc, double* sigma, double* U, double* W, void* ws,
                           size_t ws_bytes, void* stream) {
  if (r < 1 || r > 256 || !Mc || !sigma || !U || !W)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_small_svd: bad arguments");
  if (ws_bytes < rsvd_small_svd_workspace(r)) return fail(RSVD_ERR_INVALID_ARG, "rsvd_small_svd: workspace too small");
  Carver c(ws, ws_bytes);
  JacobiWs w = jacobi_ws_carve(c, r, r);
  cudaStream_t st = as_stream(stream);
  RSVD_CUDA(cudaMemsetAsync(w.status, 0, sizeof(int), st));
  RSVD_TRY(jacobi_svd(r, r, Mc, sigma, U, W, w, st));
  return read_device_status(w.status, st);
}

rsvd_status rsvd_plan_min_cap(int64_t m, int64_t n, int k, int p, const rsvd_opts* opts, size_t* out_bytes) {
  RSVD_TRY(check_args(m, n, k, p, 0, opts));
  if (!out_bytes) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_min_cap: out is NULL");
  rsvd_plan_s P;
  P.m = m; P.n = n; P.k = k; P.p = p; P.r = k + p; P.ldr = (int)round_up(P.r, 4);
  apply_opts(&P, opts);
  *out_bytes = layout(&P, nullptr, 0);
  return RSVD_OK;
}

rsvd_status rsvd_plan(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, size_t mem_cap_bytes,
                      const rsvd_opts* opts, rsvd_plan_t* out) {
  if (!out) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan: out is NULL");
  *out = nullptr;
  RSVD_TRY(check_args(m, n, k, p, q, opts));
  rsvd_plan_s* P = new (std::nothrow) rsvd_plan_s();
  if (!P) return fail(RSVD_ERR_OOM, "rsvd_plan: host allocation failed");
  P->m = m; P->n = n; P->k = k; P->p = p; P->q = q; P->r = k + p; P->seed = seed;
  P->ldr = (int)round_up(P->r, 4);
  apply_opts(P, opts);
  P->mem_cap = mem_cap_bytes;
  P->ws_bytes = layout(P, nullptr, 0);
  if (mem_cap_bytes && P->ws_bytes > mem_cap_bytes) {
    delete P;
    return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_plan: mem_cap below the workspace this plan needs");
  }
  cudaError_t e = cudaMalloc(&P->ws, P->ws_bytes);
  if (e != cudaSuccess) {
    delete P;
    return cuda_fail(e, "rsvd_plan: cudaMalloc(workspace)");
  }
  layout(P, P->ws, P->ws_bytes);
  *out = P;
  return RSVD_OK;
}

rsvd_status rsvd_plan_info(rsvd_plan_t P, rsvd_plan_info_t* o) {
  if (!P || !o) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_info: NULL argument");
  std::memset(o, 0, sizeof(*o));
  o->m = P->m; o->n = P->n; o->k = P->k; o->p = P->p; o->q = P->q; o->r = P->r;
  o->prec = P->prec; o->dtype = P->dtype; o->mb = P->mb; o->nb = P->nb;
  o->tiles_m = cdiv(P->m, P->mb); o->tiles_n = cdiv(P->n, P->nb); o->n_slots = P->n_slots;
  o->resident = 1; o->workspace_bytes = P->ws_bytes; o->min_cap_bytes = P->ws_bytes; o->seed = P->seed;
  o->q_used = P->q_used;
  o->resumed_from = P->resumed_from;
  o->bf16_copy = P->a16_ready ? 1 : 0;
  return RSVD_OK;
}

rsvd_status rsvd_run(rsvd_plan_t P, const rsvd_matrix* A, void* U, void* S, void* V, void* stream) {
  if (!P || !A || !U || !S || !V) return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: NULL argument");
  const bool a16 = A->dtype == RSVD_BF16 || A->dtype == RSVD_F16;
  if (A->m != P->m || A->n != P->n || (A->dtype != P->dtype && !a16))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: A does not match the plan (shape or dtype)");
  if (a16 && (P->dtype != RSVD_F32 || P->prec != RSVD_PREC_BF16 || A->kind != RSVD_DENSE))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: a BF16 or FP16 A needs a dense F32 plan with BF16 precision");
  if (a16 && A->location == RSVD_ON_DEVICE && (A->ld % 8 != 0 || (reinterpret_cast<uintptr_t>(A->data) & 15) != 0))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: a BF16 or FP16 A needs ld % 8 == 0 and a 16-byte aligned base");
  if (A->kind != P->kind) return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: A's kind (dense/CSR) differs from the plan's");
  cudaStream_t st = as_stream(stream);
  if (A->kind == RSVD_CSR) {
    rsvd_matrix Ad;
    P->prof.begin();
    P->streaming = false;
    P->csr_streaming = false;
    RSVD_TRY(prepare_csr(P, *A, &Ad, st));
    return run_typed<float>(P, Ad, static_cast<float*>(U), static_cast<float*>(S), static_cast<float*>(V), st);
  }
  if (A->ld < A->n || !A->data) return fail(RSVD_ERR_INVALID_ARG, "rsvd_run: bad dense descriptor");
  rsvd_matrix Ad = *A;
  P->prof.begin();
  P->streaming = false;
  P->csr_streaming = false;
  if (A->location == RSVD_ON_HOST) {
    // Automatic in-core / out-of-core switch (Section 3.5): a host matrix that
    // fits under the cap (or any host matrix when there is no cap) is copied to
    // the device once and processed in core; otherwise its tiles are streamed.
    // device copy: rows of n values (16-bit A: padded to a multiple of 8 for the TMA)
    const int64_t ldd = a16 ? round_up(A->n, 8) : A->n;
    const size_t bytes = (size_t)A->m * ldd * elem_size(A->dtype);
    if (P->mem_cap && P->ws_bytes + bytes > P->mem_cap) {
      if (a16) return fail(RSVD_ERR_UNSUPPORTED, "rsvd_run: a BF16 or FP16 A is not streamed (it must fit the cap)");
      if (P->Adev) { cudaFree(P->Adev); P->Adev = nullptr; P->a_copy_bytes = 0; }
      drop_prefetches(P);
      release_idle_prefetch_buffers(P);
      if (P->ws_bytes >= P->mem_cap) return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_run: no room left for streaming");
      if (P->prec == RSVD_PREC_FP8)
        return fail(RSVD_ERR_UNSUPPORTED, "rsvd_run: FP8 precision needs A in device memory (no streaming)");
      const int final_prec =
          ((P->prec == RSVD_PREC_BF16 || P->prec == RSVD_PREC_FP8) && P->refine) ? RSVD_PREC_BF16X3 : P->prec;
      // fused sweeps stream full-width row panels (the default tile shape)
      if (P->fused && P->nb_req > 0 && P->nb_req < A->n)
        return fail(RSVD_ERR_UNSUPPORTED, "rsvd_run: fused sweeps stream full-width row panels (nb = 0 or n)");
      // BF16 plans keep their resident tiles as BF16 copies (twice as many fit)
      const bool bf16_cache = P->prec == RSVD_PREC_BF16 && P->dtype == RSVD_F32 && !P->fused &&
                              round_up(P->r, 16) <= 256;
      RSVD_TRY(stream_prepare(&P->ss, A->m, A->n, elem_size(A->dtype), P->mb_req, P->nb_req, P->n_slots,
                              P->mem_cap - P->ws_bytes, P->r, P->prec, final_prec, bf16_cache));
      stream_begin_run(P->ss);
      P->streaming = true;
      if (P->dtype == RSVD_F64)
        return run_typed<double>(P, Ad, static_cast<double*>(U), static_cast<double*>(S), static_cast<double*>(V), st);
      return run_typed<float>(P, Ad, static_cast<float*>(U), static_cast<float*>(S), static_cast<float*>(V), st);
    }
    // the oldest pending prefetch, when it is this A, replaces the copy
    rsvd_plan_s::Prefetch* pre = nullptr;
    for (auto& e : P->pre)
      if (e.pending && (!pre || e.seq < pre->seq)) pre = &e;
    if (pre && !same_host_matrix(pre->desc, *A)) {
      drop_prefetches(P);
      pre = nullptr;
    }
    if (pre) {
      pre->pending = false;
      std::swap(P->h2d_ev, pre->ev);  // the first pass waits on the prefetch's chunk events
      P->h2d_chunk_rows = pre->chunk_rows;
      P->h2d_chunks = pre->chunks;
      Ad.data = pre->dev;
      Ad.ld = pre->ldd;
      if (P->prof.on) {
        Span sp(P->prof, RSVD_STAGE_H2D, st);
        RSVD_CUDA(cudaStreamWaitEvent(st, P->h2d_ev[P->h2d_chunks], 0));
      }
    } else {
      if (P->mem_cap) release_idle_prefetch_buffers(P);
      if (P->a_copy_bytes < bytes) {
        if (P->Adev) cudaFree(P->Adev);
        P->Adev = nullptr;
        P->a_copy_bytes = 0;
        RSVD_CUDA(cudaMalloc(&P->Adev, bytes));
        P->a_copy_bytes = bytes;
      }
      Span sp(P->prof, RSVD_STAGE_H2D, st);
      // the copies start after the work already queued on the caller's stream
      RSVD_TRY(copy_host_chunks(P, *A, P->Adev, ldd, P->h2d_ev, st, true, &P->h2d_chunk_rows, &P->h2d_chunks));
      if (P->prof.on) RSVD_CUDA(cudaStreamWaitEvent(st, P->h2d_ev[P->h2d_chunks], 0));  // the stage time covers the copy
      Ad.data = P->Adev;
    }
    P->h2d_pending = true;
    Ad.ld = ldd;
    Ad.location = RSVD_ON_DEVICE;
  }
  const rsvd_status res =
      P->dtype == RSVD_F64
          ? run_typed<double>(P, Ad, static_cast<double*>(U), static_cast<double*>(S), static_cast<double*>(V), st)
          : run_typed<float>(P, Ad, static_cast<float*>(U), static_cast<float*>(S), static_cast<float*>(V), st);
  if (P->h2d_pending) {  // a run that stopped before using A: the copy still ends before the call returns
    cudaStreamSynchronize(P->h2d_stream);
    P->h2d_pending = false;
  }
  return res;
}

rsvd_status rsvd_plan_prefetch(rsvd_plan_t P, const rsvd_matrix* A) {
  if (!P || !A) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_prefetch: NULL argument");
  const bool a16 = A->dtype == RSVD_BF16 || A->dtype == RSVD_F16;
  if (P->kind != RSVD_DENSE || A->kind != RSVD_DENSE || A->location != RSVD_ON_HOST || !A->data)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_prefetch: a dense host A of a dense plan");
  if (A->m != P->m || A->n != P->n || A->ld < A->n || (A->dtype != P->dtype && !a16))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_prefetch: A does not match the plan (shape or dtype)");
  if (a16 && (P->dtype != RSVD_F32 || P->prec != RSVD_PREC_BF16))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_prefetch: a BF16 or FP16 A needs an F32 plan with BF16 precision");
  const int64_t ldd = a16 ? round_up(A->n, 8) : A->n;
  const size_t bytes = (size_t)A->m * ldd * elem_size(A->dtype);
  if (P->mem_cap && P->ws_bytes + bytes > P->mem_cap)
    return fail(RSVD_ERR_UNSUPPORTED, "rsvd_plan_prefetch: A does not fit the cap in core (rsvd_run streams it)");
  rsvd_plan_s::Prefetch* e = nullptr;
  for (auto& x : P->pre)
    if (!x.pending) { e = &x; break; }
  if (!e) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_prefetch: two prefetches are already pending");
  if (P->mem_cap) {
    size_t held = P->ws_bytes + P->a_copy_bytes + P->a16_bytes;
    for (auto& x : P->pre) held += &x == e ? std::max(x.bytes, bytes) : x.bytes;
    if (held > P->mem_cap) return fail(RSVD_ERR_CAP_TOO_SMALL, "rsvd_plan_prefetch: no room for the prefetch buffers");
  }
  if (e->bytes < bytes) {
    if (e->dev) cudaFree(e->dev);
    e->dev = nullptr;
    e->bytes = 0;
    if (cudaMalloc(&e->dev, bytes) != cudaSuccess) {
      (void)cudaGetLastError();
      return fail(RSVD_ERR_OOM, "rsvd_plan_prefetch: no device memory for the buffer");
    }
    e->bytes = bytes;
  }
  // the buffer is free: every run returns after its work has completed, and
  // an earlier copy into it precedes this one on the same stream
  RSVD_TRY(copy_host_chunks(P, *A, e->dev, ldd, e->ev, nullptr, false, &e->chunk_rows, &e->chunks));
  e->ldd = ldd;
  e->desc = *A;
  e->seq = ++P->pre_seq;
  e->pending = true;
  return RSVD_OK;
}

rsvd_status rsvd_csr_tile(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx, const float* val,
                          int64_t row0, int64_t row1, int64_t col0, int64_t col1, int32_t* t_rowptr,
                          int32_t* t_colidx, float* t_val, int64_t cap, int64_t* nnz) {
  return csr_tile_host(m, n, rowptr, colidx, val, row0, row1, col0, col1, t_rowptr, t_colidx, t_val, cap, nnz);
}

rsvd_status rsvd_csr_transpose(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                               const float* val, int32_t* t_rowptr, int32_t* t_colidx, float* t_val) {
  return csr_transpose_host(m, n, rowptr, colidx, val, t_rowptr, t_colidx, t_val);
}

rsvd_status rsvd_coo_to_csr(int64_t m, int64_t n, int64_t nnz, int32_t index_bits, const void* rowidx,
                            const void* colidx, const float* val, int32_t* rowptr, int32_t* out_colidx,
                            float* out_val) {
  return coo_to_csr_host(m, n, nnz, index_bits, rowidx, colidx, val, rowptr, out_colidx, out_val);
}

rsvd_status rsvd_plan_set_checkpoint(rsvd_plan_t P, const char* path, int32_t stop_after_step) {
  if (!P) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_set_checkpoint: NULL plan");
  if (path && *path && (P->auto_q || P->fused))
    return fail(RSVD_ERR_UNSUPPORTED, "rsvd_plan_set_checkpoint: not available with automatic q or fused sweeps");
  P->ckpt_path = path ? path : "";
  P->ckpt_stop_after = stop_after_step;
  return RSVD_OK;
}

rsvd_status rsvd_plan_set_profiling(rsvd_plan_t P, int32_t enable) {
  if (!P) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_set_profiling: NULL plan");
  if (enable) RSVD_TRY(P->prof.reserve(20 + 4 * ((size_t)P->q + 1)));
  P->prof.on = enable != 0;
  return RSVD_OK;
}

rsvd_status rsvd_plan_stage_ms(rsvd_plan_t P, double* ms, int32_t* apass_calls) {
  if (!P || !ms) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_stage_ms: NULL argument");
  for (int i = 0; i < RSVD_STAGE_COUNT; ++i) ms[i] = P->prof.ms[i];
  if (apass_calls) *apass_calls = P->prof.apass_calls;
  return RSVD_OK;
}

unsigned long long rsvd_kernel_launches(void) { return g_launches.load(); }

rsvd_status rsvd_backward(rsvd_plan_t P, const void* U, const void* S, const void* V, const void* dU,
                          const void* dS, const void* dV, void* dA, void* stream) {
  if (!P || !U || !S || !V || !dA) return fail(RSVD_ERR_INVALID_ARG, "rsvd_backward: NULL argument");
  if (P->kind != RSVD_DENSE) return fail(RSVD_ERR_UNSUPPORTED, "rsvd_backward: CSR plans have no backward pass");
  cudaStream_t st = as_stream(stream);
  if (P->dtype == RSVD_F64)
    return backward_typed<double>(P->m, P->n, P->k, static_cast<const double*>(U), static_cast<const double*>(S),
                                  static_cast<const double*>(V), static_cast<const double*>(dU),
                                  static_cast<const double*>(dS), static_cast<const double*>(dV),
                                  static_cast<double*>(dA), P->bwd_ws, P->bwd_ws_bytes, nullptr, st);
  // FP32: the rank-2k product runs on the tensor cores; its status word is read
  RSVD_CUDA(cudaMemsetAsync(P->status, 0, 4 * sizeof(int), st));
  RSVD_TRY(backward_typed<float>(P->m, P->n, P->k, static_cast<const float*>(U), static_cast<const float*>(S),
                                 static_cast<const float*>(V), static_cast<const float*>(dU),
                                 static_cast<const float*>(dS), static_cast<const float*>(dV),
                                 static_cast<float*>(dA), P->bwd_ws, P->bwd_ws_bytes, P->status, st));
  return read_device_status(P->status, st);
}

void rsvd_destroy(rsvd_plan_t P) {
  if (!P) return;
  if (P->h2d_stream) cudaStreamSynchronize(P->h2d_stream);  // no copy in flight into a freed buffer
  for (auto& e : P->pre) {
    if (e.dev) cudaFree(e.dev);
    for (auto ev : e.ev) cudaEventDestroy(ev);
  }
  if (P->ws) cudaFree(P->ws);
  if (P->Adev) cudaFree(P->Adev);
  if (P->a16) cudaFree(P->a16);
  if (P->csr_dev) cudaFree(P->csr_dev);
  if (P->h_tpinned) cudaFreeHost(P->h_tpinned);
  if (P->h_tval_pinned) cudaFreeHost(P->h_tval_pinned);
  for (auto e : P->h2d_ev) cudaEventDestroy(e);
  if (P->h2d_stream) cudaStreamDestroy(P->h2d_stream);
  stream_state_free(P->ss);
  csr_stream_free(P->cs);
  delete P;
}

rsvd_status rsvd_plan_stream_stats(rsvd_plan_t P, uint64_t* h2d_bytes, int64_t* tiles_streamed_per_pass,
                                   int64_t* tiles_resident) {
  if (!P) return fail(RSVD_ERR_INVALID_ARG, "rsvd_plan_stream_stats: NULL plan");
  if (P->csr_streaming) csr_stream_stats(P->cs, h2d_bytes, tiles_streamed_per_pass, tiles_resident);
  else stream_stats(P->streaming ? P->ss : nullptr, h2d_bytes, tiles_streamed_per_pass, tiles_resident);
  return RSVD_OK;
}

rsvd_status rsvd_full(const rsvd_matrix* A, void* U, void* S, void* V, void* stream) {
  if (!A || !U || !S || !V || A->kind != RSVD_DENSE || A->location != RSVD_ON_DEVICE || !A->data)
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_full: need a dense device matrix and outputs");
  const int64_t m = A->m, n = A->n, t = m < n ? m : n;
  if (m < 1 || n < 1 || t > 512 || A->ld < n || (A->dtype != RSVD_F64 && A->dtype != RSVD_F32))
    return fail(RSVD_ERR_INVALID_ARG, "rsvd_full: need min(m, n) <= 512, ld >= n, F32 or F64");
  cudaStream_t st = as_stream(stream);
  if (t > 256 || m * n > ((int64_t)1 << 24)) return full_svd_tall(*A, U, S, V, st);
  // One-sided Jacobi on the columns of A (m >= n) or of A^T (m < n), in FP64.
  //   m >= n: A W = U diag(s)   -> U = Uo, V = W
  //   m <  n: A^T W = V diag(s) -> V = Uo, U = W
  const int64_t rows = m >= n ? m : n, cols = t;
  const size_t jb = jacobi_ws_bytes(rows, (int)cols);
  const size_t sb = sign_scratch_bytes(m, (int)t);
  Sizer sz;
  sz.take<double>((size_t)rows * cols);
  sz.take<double>((size_t)cols);
  sz.take<double>((size_t)rows * cols);
  sz.take<double>((size_t)cols * cols);
  sz.take<char>(jb);
  sz.take<char>(sb);
  const size_t total = sz.used + 1024;
  void* ws = nullptr;
  RSVD_CUDA(cudaMalloc(&ws, total));
  Carver c(ws, total);
  double* Mc = c.take<double>((size_t)rows * cols);
  double* sig = c.take<double>((size_t)cols);
  double* Uo = c.take<double>((size_t)rows * cols);
  double* Wo = c.take<double>((size_t)cols * cols);
  char* jbase = c.take<char>(jb);
  void* sc = c.take<char>(sb);
  Carver jc(jbase, jb);
  JacobiWs jw = jacobi_ws_carve(jc, rows, (int)cols);
  rsvd_status s = RSVD_OK;
  const int64_t s_row = m >= n ? A->ld : 1;   // Mc[c*rows + i] = A at i*s_row + c*s_col
  const int64_t s_col = m >= n ? 1 : A->ld;
  if (cudaMemsetAsync(jw.status, 0, sizeof(int), st) != cudaSuccess) s = fail(RSVD_ERR_CUDA, "rsvd_full: memset");
  if (s == RSVD_OK) {
    s = A->dtype == RSVD_F64
            ? gather_colmajor_f64<double>(rows, cols, static_cast<const double*>(A->data), s_row, s_col, Mc, st)
            : gather_colmajor_f64<float>(rows, cols, static_cast<const float*>(A->data), s_row, s_col, Mc, st);
  }
  if (s == RSVD_OK) s = jacobi_svd((int)rows, (int)cols, Mc, sig, Uo, Wo, jw, st);
  const double* Usrc = m >= n ? Uo : Wo;
  const double* Vsrc = m >= n ? Wo : Uo;
  if (s == RSVD_OK) {
    if (A->dtype == RSVD_F64) {
      double* Ud = static_cast<double*>(U);
      double* Vd = static_cast<double*>(V);
      s = convert_matrix<double, double>(m, t, Usrc, t, Ud, t, st);
      if (s == RSVD_OK) s = convert_matrix<double, double>(n, t, Vsrc, t, Vd, t, st);
      if (s == RSVD_OK) s = convert_matrix<double, double>(1, t, sig, t, static_cast<double*>(S), t, st);
      if (s == RSVD_OK) s = normalise_signs<double>(m, n, (int)t, Ud, t, Vd, t, sc, sb, st);
    } else {
      float* Uf = static_cast<float*>(U);
      float* Vf = static_cast<float*>(V);
      s = convert_matrix<double, float>(m, t, Usrc, t, Uf, t, st);
      if (s == RSVD_OK) s = convert_matrix<double, float>(n, t, Vsrc, t, Vf, t, st);
      if (s == RSVD_OK) s = convert_matrix<double, float>(1, t, sig, t, static_cast<float*>(S), t, st);
      if (s == RSVD_OK) s = normalise_signs<float>(m, n, (int)t, Uf, t, Vf, t, sc, sb, st);
    }
  }
  if (s == RSVD_OK) s = read_device_status(jw.status, st);
  cudaStreamSynchronize(st);
  cudaFree(ws);
  return s;
}

}  // extern "C"
