// Internal launchers shared by the translation units of the library.
#pragma once
#include <string>

#include "common.cuh"

namespace rsvd {

// gaussian.cu -- Section 2.1 step 1.  Besides the public dtypes, kF32HoldingBf16
// writes the values rounded once to bfloat16 into an FP32 buffer (the test
// matrix of the BF16 path, whose A-pass converts its panel to BF16 exactly).
constexpr int kF32HoldingBf16 = 3;
rsvd_status launch_gaussian(uint64_t seed, int64_t n, int64_t r, int dtype, int layout, void* out,
                            int64_t ld, cudaStream_t stream);

// Replace column k of the M x r panel Q (k with dead[k] != 0) by a random
// vector of unit expected norm: entries stream(seed, k*M + i) / sqrt(M).
rsvd_status fill_dead_columns(int64_t M, int r, const int* dead, void* Q, int64_t ldq, int dtype,
                              uint64_t seed, cudaStream_t stream);
constexpr uint64_t kDeadFillSeed = 0x6A09E667F3BCC909ULL;

// gemm_simt.cu -- C (+)= op(A) B, K split into nsplit chunks of kchunk with
// partials (M*N each) in `partial`, added in chunk order.
template <typename T>
rsvd_status simt_gemm(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, bool transA,
                      const T* B, int64_t ldb, T* C, int64_t ldc, bool accumulate, int nsplit,
                      int64_t kchunk, T* partial, cudaStream_t stream);

// The GEMM of simt_gemm without the final reduction: partial z (the K chunk
// [z*kchunk, (z+1)*kchunk)) is written to partial + z*M*N (M x N, ld N).
template <typename T>
rsvd_status simt_gemm_partials(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda, bool transA,
                               const T* B, int64_t ldb, int nsplit, int64_t kchunk, T* partial,
                               cudaStream_t stream);

// out[i, j] (+)= sum_z P[z*pstride + i*ldp + j], z in increasing order.
template <typename T>
rsvd_status reduce_partials(int64_t M, int64_t N, int nsplit, const T* P, int64_t ldp, int64_t pstride, T* out,
                            int64_t ldo, bool accumulate, cudaStream_t stream);

// orth.cu -- CholeskyQR2 pieces.
struct OrthWs {
  double* G = nullptr;        // r x r Gram (FP64)
  double* L1 = nullptr;       // r x r Cholesky factors (lower, in the panel's type)
  double* L2 = nullptr;
  int* dead1 = nullptr;       // deflated pivots of the two sweeps (r each)
  int* dead2 = nullptr;
  void* Rinv_t = nullptr;     // R^-1 = L^-T (upper) in the panel dtype, row stride ld_rt
  int ld_rt = 0;              // r rounded up to 4 (16-byte rows for the vector loads of the products)
  void* gram_partial = nullptr;     // chunk partial Grams in the panel type
  int64_t gram_chunks = 0;
  void* tmp = nullptr;        // M x r panel (first-sweep result)
  int64_t ld_tmp = 0;
  int* status = nullptr;      // device status word
  void* tc_ws = nullptr;      // tensor-core Gram / panel product workspace (tc mode)
  size_t tc_ws_bytes = 0;
  float* gram32 = nullptr;    // r x r FP32 Gram from the tensor cores (tc mode)
  void* chol_scratch = nullptr;  // factorisation matrices when r is too large for shared memory
  size_t chol_scratch_bytes = 0;
};
// tc: FP32 panels may take their Grams and panel products on the tensor cores
// (split BF16, about 2e-5 relative) -- for bases whose only job is to span
// the sketch (the range finder of the BF16 / FP8 paths)
size_t orth_ws_bytes(int64_t M, int r, int dtype, bool tc = false);
OrthWs orth_ws_carve(Carver& c, int64_t M, int r, int dtype, bool tc = false);

// one_sweep (R == NULL only): a single CholeskyQR sweep, for bases whose only
// job is to span the sketch for the next product: Q spans Y as accurately as
// after two sweeps (the second changes orthonormality, not the span) but is
// orthonormal only to about eps cond(Y)^2.
template <typename T>
rsvd_status orth_panel(int64_t M, int r, const T* Y, int64_t ldy, T* Q, int64_t ldq, double* R,
                       const OrthWs& ws, cudaStream_t stream, bool tc = false, bool one_sweep = false);

// jacobi.cu -- Section 2.1 step 6 core.
struct JacobiWs {
  double* M = nullptr;        // rows x r working columns (column-major)
  double* W = nullptr;        // r x r accumulated rotations (column-major)
  unsigned* barrier = nullptr;  // grid barrier words (count, generation)
  int* rotated = nullptr;     // per sweep: rotation flag, check-pass flag, largest rotated off-diagonal
  int* sweeps = nullptr;      // sweeps used
  int* status = nullptr;
  float* W32 = nullptr;       // FP32-phase rotations (r x r)
  double* W64 = nullptr;      // orthonormalised rotations
  double* P = nullptr;        // Newton-Schulz Gram / shift
  double* T = nullptr;        // widened W32
  double* M64 = nullptr;      // M times the rotations
  double* gemm_partial = nullptr;
};
constexpr int kJacobiMaxSweeps = 64;
// `precondition` adds the buffers of the FP32 first phase (without them the
// FP64 sweeps run from the start).
size_t jacobi_ws_bytes(int64_t rows, int r, bool precondition = true);
JacobiWs jacobi_ws_carve(Carver& c, int64_t rows, int r, bool precondition = true);
// Mc column-major rows x r; outputs sigma (r), U (rows x r) and W (r x r)
// row-major with columns ordered like sigma (descending), each pair (U_c, W_c)
// signed so that the entry of W_c largest in magnitude is positive.
// tol: relative off-diagonal stopping test |c_ij| <= tol sqrt(c_ii c_jj) (0: r eps, FP64)
// fp64_sweeps = false (square inputs with the FP32 phase only): stop at FP32
// convergence (tol = r eps32) and form the outputs from the FP64 product M W.
rsvd_status jacobi_svd(int rows, int r, const double* Mc, double* sigma, double* U, double* W,
                       const JacobiWs& ws, cudaStream_t stream, double tol = 0.0, bool fp64_sweeps = true);

// lift.cu -- conversions, sign normalisation.
template <typename Tin, typename Tout>
rsvd_status convert_matrix(int64_t rows, int64_t cols, const Tin* in, int64_t ldi, Tout* out,
                           int64_t ldo, cudaStream_t stream);
template <typename T>
rsvd_status normalise_signs(int64_t m, int64_t n, int k, T* U, int64_t ldu, T* V, int64_t ldv,
                            void* scratch, size_t scratch_bytes, cudaStream_t stream);
size_t sign_scratch_bytes(int64_t m, int k);
// *flag = 1 when ||sigma[:k] - prev[:k]|| <= tol ||sigma[:k]|| (automatic q)
rsvd_status sigma_change_below(int k, const double* sigma, const double* prev, double tol, int* flag,
                               cudaStream_t stream);
// out[c*rows + i] = (double) A[i*s_row + c*s_col]  (column-major FP64 gather)
template <typename T>
rsvd_status gather_colmajor_f64(int64_t rows, int64_t cols, const T* A, int64_t s_row, int64_t s_col,
                                double* out, cudaStream_t stream);

// adjoint.cu -- backward pass of the truncated SVD.
size_t backward_ws_bytes(int64_t m, int64_t n, int k, int dtype);
template <typename T>
// status: device word (4 ints) that an expired tensor-core wait is recorded in
rsvd_status backward_typed(int64_t m, int64_t n, int k, const T* U, const T* S, const T* V, const T* dU,
                           const T* dS, const T* dV, T* dA, void* ws, size_t ws_bytes, int* status, cudaStream_t st);

// spmm.cu -- A-passes for a CSR matrix (FP32 values, int32 indices).
constexpr int kSpmmMaxR = 512;
// Rows with more entries than this are split into segments of this many
// entries, one warp each, when the workspace allows.
constexpr int kSpmmSeg = 1024;
// Upper bound on the segment tasks of a matrix with nnz entries: each long
// row of len entries takes ceil(len/kSpmmSeg) < 2 len/kSpmmSeg tasks.
inline int64_t spmm_max_tasks(int64_t nnz) { return 2 * (nnz / kSpmmSeg) + 1; }
size_t spmm_ws_bytes(int64_t nnz, int r);
// The dense panel of a CSR A-pass: fmt 0 FP32 rows (f, ld floats per row);
// fmt 1 BF16 rows (h, ld values per row, ld a multiple of 4); fmt 2 24-bit
// rows (p24, rb = spmm_p24_row_bytes(ld) bytes per row: groups of 128 values
// as 256 bytes of high 16-bit parts then 128 bytes of low bytes).
struct SpmmPanel {
  int fmt = 0;
  const float* f = nullptr;
  const uint16_t* h = nullptr;
  const uint8_t* p24 = nullptr;
  int64_t ld = 0;
  int64_t rb = 0;
};
int64_t spmm_p24_row_bytes(int64_t ld);
// Rows of X (K x r, ldx) rounded into the compact formats (fmt 1 into h, fmt 2
// into p24).
rsvd_status spmm_pack(int fmt, int64_t K, int r, const float* X, int64_t ldx, uint16_t* h, uint8_t* p24, int64_t ld,
                      cudaStream_t stream);
rsvd_status spmm_csr_panel(int64_t M, int r, const int32_t* rowptr, const int32_t* colidx, const float* val,
                           int64_t nnz, const SpmmPanel& X, float* Y, int64_t ldy, bool accumulate, void* ws,
                           size_t ws_bytes, cudaStream_t stream);
// Y (M x r, ldy) = (or +=) A X for the M-row CSR (rowptr, colidx, val; nnz
// entries), X row-major (ldx).  ws (may be NULL) enables the long-row split.
rsvd_status spmm_csr(int64_t M, int r, const int32_t* rowptr, const int32_t* colidx, const float* val,
                     int64_t nnz, const float* X, int64_t ldx, float* Y, int64_t ldy, bool accumulate, void* ws,
                     size_t ws_bytes, cudaStream_t stream);
// Host CSR of A^T (n rows) from the CSR of A (m rows); stable, deterministic.
rsvd_status csr_transpose_host(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                               const float* val, int32_t* t_rowptr, int32_t* t_colidx, float* t_val);
// COO (index arrays of index_bits = 32 or 64) to CSR, stable within rows.
rsvd_status coo_to_csr_host(int64_t m, int64_t n, int64_t nnz, int index_bits, const void* rowidx,
                            const void* colidx, const float* val, int32_t* rowptr, int32_t* out_colidx,
                            float* out_val);

// checkpoint.cu -- persistence of the range finder's basis (Section 3.8).
struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int64_t m, n;
  int32_t k, p, q, r, ldr, prec, dtype, kind;
  uint64_t seed, fingerprint;
  int32_t step, pad;
  int64_t panel_rows;
  uint64_t panel_bytes, panel_checksum, header_checksum;
};
rsvd_status matrix_fingerprint(const rsvd_matrix& A, uint64_t* out, cudaStream_t st);
// writes header + device panel (h.panel_bytes) to path (via path.tmp and rename)
rsvd_status ckpt_save(const std::string& path, CkptHeader h, const void* dev_panel, cudaStream_t st);
// loads the checkpoint at path if it matches `expect`; returns its step (or -1)
int ckpt_try_load(const std::string& path, const CkptHeader& expect, void* dev_q, void* dev_z, cudaStream_t st);

// stream.cu -- out-of-core A-passes over tiles of a pinned host matrix.
struct StreamState;
rsvd_status stream_prepare(StreamState** ps, int64_t m, int64_t n, size_t esz, int64_t mb_req, int64_t nb_req,
                           int slots, size_t budget, int r, int prec, int final_prec, bool bf16_cache);
void stream_begin_run(StreamState* s);
rsvd_status apass_streamed(StreamState* s, const rsvd_matrix& Ah, int trans, int prec, int r, const void* X,
                           void* Y, int64_t ldr, int* status, cudaStream_t st);
// Precision of the products A^T (A W) in a fused sweep for a plan precision.
int sweep_trans_prec(int prec);
// One fused power sweep Z = A^T (A W) over streamed full-width row panels.
rsvd_status sweep_streamed(StreamState* s, const rsvd_matrix& Ah, int prec, int prec_t, int r, const void* W,
                           void* Z, int64_t ldr, int* status, cudaStream_t st);
void stream_state_free(StreamState* s);
void stream_stats(const StreamState* s, uint64_t* h2d, int64_t* per_pass, int64_t* cached);

// csr_stream.cu -- out-of-core sparse A-passes over CSR tiles of a host matrix.
// Entries of rows [row0, row1) x columns [col0, col1) of a host CSR as a local
// CSR (offsets from 0, column indices minus col0); with cap == 0 only counts.
rsvd_status csr_tile_host(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx, const float* val,
                          int64_t row0, int64_t row1, int64_t col0, int64_t col1, int32_t* t_rowptr,
                          int32_t* t_colidx, float* t_val, int64_t cap, int64_t* nnz_out);
struct CsrStream;
// A: host CSR with host t_rowptr/t_colidx/t_val (the CSR of A^T).
rsvd_status csr_stream_prepare(CsrStream** ps, const rsvd_matrix& A, int64_t mb_req, int64_t nb_req, int slots,
                               size_t budget, int r);
void csr_stream_begin_run(CsrStream* s);
rsvd_status csr_apass_streamed(CsrStream* s, int trans, int r, const SpmmPanel& X, float* Y, int64_t ldy,
                               cudaStream_t st);
void csr_stream_free(CsrStream* s);
void csr_stream_stats(const CsrStream* s, uint64_t* h2d, int64_t* per_pass, int64_t* cached);

// api.cu -- A-pass dispatch.
size_t apass_ws_bytes(int64_t m, int64_t n, int r, int trans, int prec, int64_t mb, int64_t nb);
rsvd_status apass_dense(const rsvd_matrix& A, int trans, int prec, int r, const void* X, int64_t ldx,
                        void* Y, int64_t ldy, int64_t mb, int64_t nb, void* ws, size_t ws_bytes,
                        int* status, cudaStream_t stream, bool accumulate = false);

// gemm_tc.cu -- tensor-core (tcgen05) A-passes on FP32 A with in-kernel BF16 conversion.
size_t tc_apass_ws_bytes(int64_t m, int64_t n, int r, int trans, int prec, int64_t mb, int64_t nb);
// `status` (may be NULL: a workspace word is used) receives DEV_TIMEOUT if a
// pipeline wait expires.
// fp8.cu -- E4M3 codes of A with one power-of-two scale per block-cyclic tile.
struct Fp8Source {
  const uint8_t* codes = nullptr;  // m x ldc bytes
  int64_t m = 0, n = 0, ldc = 0;
  const float* scales = nullptr;   // cdiv(m, qm) x cdiv(n, qn)
  int64_t qm = 0, qn = 0;          // tile edges, clamped to m and n
};
bool fp8_tiles_ok(int64_t m, int64_t n, int64_t qm, int64_t qn);
size_t fp8_amax_ws_bytes(int64_t m, int64_t n, int64_t qm, int64_t qn);
rsvd_status fp8_quantize(const float* A, int64_t m, int64_t n, int64_t lda, int64_t qm, int64_t qn, uint8_t* codes,
                         int64_t ldc, float* scales, unsigned* amax_ws, cudaStream_t stream);
// The A-pass on the FP8 source (BF16 panel, FP32 accumulation).
rsvd_status tc_apass_from_fp8(const Fp8Source& f8, int trans, int r, const float* X, int64_t ldx, float* Y,
                              int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream,
                              bool accumulate = false);
// copy16 (optional, forward pass only): the pass also stores BF16(A), rounded
// as its operands are, row-major with stride ld16 (a multiple of 64 >= n),
// for tc_apass_from_bf16; copy16lo (optional, split mode only) receives
// BF16(A - BF16(A)) in the same layout, the lo part of the split operand.
// kps (optional): K steps per split, to give a row block of a larger pass the
// larger pass's split of the K range (tc_ksteps_per_split), hence its sums.
rsvd_status tc_apass_from_f32(const rsvd_matrix& A, int trans, int prec, int r, const float* X,
                              int64_t ldx, float* Y, int64_t ldy, int64_t mb, int64_t nb, void* ws,
                              size_t ws_bytes, int* status, cudaStream_t stream, bool accumulate = false,
                              uint16_t* copy16 = nullptr, int64_t ld16 = 0, uint16_t* copy16lo = nullptr,
                              int64_t kps = 0);
// Y (M x N, ldy) = A X for an FP32 A (M x K, A.ld % 4 == 0, 16-byte aligned)
// and X (K x N, ldx) with any N, in output tiles of up to 192 (split) or 256
// columns: the tensor-core product of a short K and a wide output (the
// adjoint's rank-2k product).  prec BF16 or BF16X3.
size_t tc_gemm_wide_ws_bytes(int64_t M, int64_t K, int64_t N, int prec);
rsvd_status tc_gemm_wide(const rsvd_matrix& A, int prec, int64_t N, const float* X, int64_t ldx, float* Y,
                         int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream);
// The K steps per split a pass over an m x n A chooses (0 where the pass
// runs over column halves of the panel).
int64_t tc_ksteps_per_split(int64_t m, int64_t n, int r, int trans, int prec);
// A BF16 copy of a dense m x n A (row-major, stride ld elements).
struct Bf16Source {
  const uint16_t* data = nullptr;
  int64_t m = 0, n = 0, ld = 0;
  int f16 = 0;  // 1: the values are IEEE FP16 (the panel is then rounded to FP16)
  // optional second part of the same layout: A = data + lo (the split copy of
  // an FP32 A, BF16 only); split-mode passes then form three products
  const uint16_t* lo = nullptr;
};
// The BF16 A-pass over the copy: the same operands, hence the same result, as
// tc_apass_from_f32 with prec BF16 on the FP32 A the copy was made from.
rsvd_status tc_apass_from_bf16(const Bf16Source& b16, int trans, int r, const float* X, int64_t ldx, float* Y,
                               int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream);
// A-pass over a 16-bit A (BF16 or FP16, m x n, row stride ld % 8 == 0, 16-byte
// aligned): prec BF16 rounds the panel to A's type; BF16X3 splits it in two
// (hi + lo) and adds the two products, and when A has a lo part (the split
// copy of an FP32 A) the product of that part with the panel's hi part too.
rsvd_status tc_apass_from_16(const Bf16Source& a16, int trans, int prec, int r, const float* X, int64_t ldx,
                             float* Y, int64_t ldy, void* ws, size_t ws_bytes, int* status, cudaStream_t stream,
                             bool accumulate = false, int64_t kps = 0);

}  // namespace rsvd
