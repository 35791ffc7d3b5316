/*
 * rsvd.h - C ABI of the GB300 randomized-SVD library (librsvd_gb300.so).
 *
 * The library computes the rank-k randomized SVD of Halko, Martinsson & Tropp
 * as described in Demchik, Bacak, Bordag, "Out-of-core singular value
 * decomposition" (arXiv:1907.06470), Section 2.1 (steps 1-7) with the power
 * scheme of Section 2.2 (Eq. (2), evaluated right to left as in Eq. (3)),
 * over the block-wise / block-cyclic matrix partition of Section 2.3 and
 * Section 3.1.  Every step runs in CUDA kernels on one GB300 (sm_103a).
 *
 * Conventions (all entry points):
 *   - Every call returns an rsvd_status; nothing aborts and nothing prints.
 *     rsvd_last_error() returns a per-thread text detail of the last failure.
 *   - Matrices are row-major.  "device" pointers are CUDA global memory of the
 *     current device; "host" pointers are ordinary (preferably pinned) memory.
 *   - The caller owns every buffer it passes; the library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls that return a device status (rsvd_run, rsvd_orth, rsvd_small_svd,
 *     rsvd_full) synchronise `stream` once before returning; the others only
 *     enqueue work.
 */
#ifndef RSVD_GB300_H
#define RSVD_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RSVD_OK = 0,
  RSVD_ERR_INVALID_ARG = 1,   /* an argument breaks a documented rule */
  RSVD_ERR_OOM = 2,           /* cudaMalloc / host allocation failed */
  RSVD_ERR_CAP_TOO_SMALL = 3, /* mem_cap below the planner's minimum */
  RSVD_ERR_CUDA = 4,          /* a CUDA runtime/driver call failed */
  RSVD_ERR_NOT_SPD = 5,       /* Cholesky breakdown: Gram matrix not positive definite */
  RSVD_ERR_NO_CONVERGE = 6,   /* Jacobi sweep limit reached */
  RSVD_ERR_TIMEOUT = 7,       /* a device-side wait exceeded its spin limit */
  RSVD_ERR_UNSUPPORTED = 8,   /* valid request this build does not implement */
  RSVD_ERR_INTERRUPTED = 9    /* the run stopped on request after writing a checkpoint */
} rsvd_status;

/* Arithmetic of the A-passes (the products with A of Section 2.1 steps 2 and 5
 * and of Eq. (3)).  FP64: everything FP64.  FP32: FP32 FMA products.  BF16:
 * A and the panel rounded to bfloat16, products on the tensor cores with FP32
 * accumulation; the final pass B^T = A^T Q is recomputed in split-BF16
 * (hi+lo, three products, about FP32 accuracy) when opts.refine != 0.
 * BF16X3: every A-pass in split-BF16.  FP8 (an experiment): A is stored once
 * per run as E4M3 codes with one power-of-two scale per tile (the plan's
 * tiles rounded up to multiples of 128; one tile when no tiles are set; see
 * rsvd_fp8_quantize), the A-passes decode the codes to BF16 on the fly and
 * multiply with the BF16 panel on the tensor cores (FP32 accumulation); the
 * final B^T = A^T Q is recomputed in split-BF16 from the FP32 A when
 * opts.refine != 0.  Dense F32 matrices held in device memory during the run. */
typedef enum {
  RSVD_PREC_FP64 = 0,
  RSVD_PREC_FP32 = 1,
  RSVD_PREC_BF16 = 2,
  RSVD_PREC_BF16X3 = 3,
  RSVD_PREC_FP8 = 4
} rsvd_prec;

typedef enum { RSVD_F64 = 0, RSVD_F32 = 1, RSVD_BF16 = 2, RSVD_F16 = 3 } rsvd_dtype;
typedef enum { RSVD_DENSE = 0, RSVD_CSR = 1 } rsvd_kind;
typedef enum { RSVD_ON_DEVICE = 0, RSVD_ON_HOST = 1 } rsvd_location;

/* Options of rsvd_plan; a NULL pointer selects the defaults given here. */
typedef struct {
  int32_t prec;      /* rsvd_prec; default FP64 for FP64 plans, FP32 otherwise */
  int32_t refine;    /* BF16 only: split-BF16 recompute of B^T (default 1) */
  int64_t mb, nb;    /* block-cyclic tile edges (Section 3.1); 0 = planner choice */
  int32_t n_slots;   /* block-cyclic slots = copy/compute buffer pairs (default 2) */
  int32_t dtype;     /* rsvd_dtype of A and of the outputs: F64 or F32 (default F32) */
  int32_t kind;      /* rsvd_kind of the matrices this plan runs on (default DENSE);
                        CSR plans take dtype F32 and prec FP32, BF16 or
                        BF16X3: the range-finder passes of BF16 / BF16X3 CSR
                        plans gather the panel rounded to BF16 / to 24 bits
                        (see rsvd_apass), their final B^T = A^T Q an FP32
                        panel */
  int32_t auto_q;    /* 1: choose the number of power iterations automatically,
                        with q (rsvd_plan) as the maximum (Section 2.2): after i
                        iterations the singular values sigma^(i) of B_i = Q_i^T A
                        are formed; iterations stop at the first i >= 1 with
                        ||sigma^(i) - sigma^(i-1)||_2 <= auto_q_tol ||sigma^(i)||_2
                        over the top k, or at i = q.  Costs one small SVD per
                        iteration; rsvd_plan_info reports the count used. */
  double auto_q_tol; /* tolerance of auto_q; 0 selects 1e-3 */
  int32_t fused;     /* 1: fused power sweeps (Section 2.2, Eq. (3) evaluated
                        right to left with the products A^T (A W) grouped):
                        W = O; q times W = orth(A^T (A W)); Q = orth(A W).  Only
                        the n-side basis is orthonormalised between products;
                        the span is that of the default scheme in exact
                        arithmetic, but the sweep squares the spectrum, so
                        directions below about sqrt(eps) sigma_1 are lost.  Out
                        of core each sweep streams every row panel once (Y_I =
                        A_I W, then Z += A_I^T Y_I while the panel is on the
                        device): q + 2 reads of A instead of 2q + 2.  BF16 plans
                        form A^T Y in split BF16.  Dense plans of FP64, FP32,
                        BF16 or BF16X3 precision with a fixed q; streamed
                        tiles must be full-width row panels (nb = 0 or n);
                        no checkpoints. */
  int32_t reserved;
} rsvd_opts;

/* Descriptor of the input matrix A (m x n). */
typedef struct {
  int32_t kind;      /* rsvd_kind: DENSE row-major, or CSR */
  int32_t dtype;     /* rsvd_dtype of the values: F64 or F32 (CSR: F32); a dense
                        A may also be stored in 16 bits, BF16 or F16 (IEEE
                        half), for F32 plans with BF16 precision (rsvd_run) */
  int32_t location;  /* rsvd_location of the data */
  int32_t reserved;
  int64_t m, n;
  const void* data;  /* DENSE: element (i,j) at data[i*ld + j] */
  int64_t ld;        /* DENSE: leading dimension in elements, >= n */
  const int32_t* rowptr;  /* CSR: m+1 offsets, rowptr[0] = 0, rowptr[m] = nnz */
  const int32_t* colidx;  /* CSR: nnz column indices in [0, n) */
  const float* val;       /* CSR: nnz values */
  int64_t nnz;            /* CSR: number of stored entries, < 2^31 */
  /* CSR only, optional: the CSR of A^T (n+1 offsets, nnz row indices of A,
   * nnz values), used by the products A^T X; built by the library from the
   * CSR of A (rsvd_csr_transpose) when t_rowptr is NULL.  Same location as
   * rowptr/colidx/val. */
  const int32_t* t_rowptr;
  const int32_t* t_colidx;
  const float* t_val;
} rsvd_matrix;

/* One tile of the block-cyclic map (Section 3.1): rows [row0,row1) x cols [col0,col1). */
typedef struct {
  int64_t t, I, J, row0, row1, col0, col1, slot;
} rsvd_tile;

typedef struct rsvd_plan_s* rsvd_plan_t;

/* Planner summary, filled by rsvd_plan_info. */
typedef struct {
  int64_t m, n;
  int32_t k, p, q, r;        /* r = k + p */
  int32_t prec, dtype;
  int64_t mb, nb;            /* tile edges in use */
  int64_t tiles_m, tiles_n;  /* tile grid */
  int32_t n_slots;
  int32_t resident;          /* 1: A is used from device memory during rsvd_run */
  size_t workspace_bytes;    /* device memory owned by the plan */
  size_t min_cap_bytes;      /* smallest mem_cap this problem can be planned in */
  uint64_t seed;
  int32_t q_used;            /* power iterations applied by the last rsvd_run */
  int32_t resumed_from;      /* checkpoint step the last rsvd_run resumed after; -1: none */
  int32_t bf16_copy;         /* 1: the last rsvd_run's later passes read a BF16 copy of A
                                (BF16X3 plans: the split copy) */
} rsvd_plan_info_t;

/* Header of a checkpoint file (rsvd_plan_set_checkpoint). */
typedef struct {
  int64_t m, n;
  int32_t k, p, q, r, prec, dtype, kind;
  uint64_t seed, fingerprint;
  int32_t step;               /* range-finder step whose basis the file holds */
  int64_t panel_rows;         /* m (Q after an even step) or n (Z after an odd step) */
  uint64_t panel_bytes;
} rsvd_checkpoint_info_t;

/* ---- Section 2.1 / 2.2: plan and run -------------------------------------- */

/* Plan a rank-k randomized SVD of an m x n matrix with oversampling p
 * (r = k + p columns in the sketch, Section 2.1 step 1) and q power
 * iterations (Section 2.2).  `seed` selects the Gaussian stream of the test
 * matrix (see rsvd_gaussian).  Device workspace is allocated here and owned by
 * the plan; `mem_cap_bytes` bounds it together with any device copy of A
 * (0 = no cap: run in core when A fits, the paper's default in Section 3.5).
 * Rules: 1 <= k, 0 <= p, k + p <= min(m, n), 0 <= q <= 64, and k + p <= 256
 * for dense plans, k + p <= 512 for CSR plans (opts.kind = CSR: dtype F32,
 * prec FP32, BF16 or BF16X3; they hold no backward workspace).
 * Errors: INVALID_ARG, CAP_TOO_SMALL (see rsvd_plan_min_cap), OOM, CUDA.
 * On success *out receives a plan that must be released with rsvd_destroy. */
rsvd_status rsvd_plan(int64_t m, int64_t n, int k, int p, int q, uint64_t seed,
                      size_t mem_cap_bytes, const rsvd_opts* opts, rsvd_plan_t* out);

/* Smallest mem_cap_bytes that rsvd_plan accepts for these arguments (host only). */
rsvd_status rsvd_plan_min_cap(int64_t m, int64_t n, int k, int p, const rsvd_opts* opts,
                              size_t* out_bytes);

rsvd_status rsvd_plan_info(rsvd_plan_t plan, rsvd_plan_info_t* out);

/* Run the planned randomized SVD on A (Section 2.1 steps 1-7 with Eq. (3)).
 * A: of the plan's kind and dtype.  Dense: device or pinned host.  CSR
 * (Section 3.3, sparse x dense products): device or host arrays; the products
 * A X run on the CSR of A and the products A^T X on the CSR of A^T, which is
 * built on the host (rsvd_csr_transpose, once per call) when A.t_rowptr is
 * NULL.  A host CSR (and a built transpose) is copied into device memory owned
 * by the plan when the copies fit under the cap (or there is no cap);
 * otherwise it is processed out of core (Section 3.5): the blocks of the CSR
 * of A (forward products) and of the CSR of A^T (transposed products) are
 * streamed from host memory through opts.n_slots device buffers, overlapped
 * with the products, and the blocks that fit in the rest of the cap stay
 * resident for the later passes.  Blocks: with opts.mb / opts.nb set, the
 * block-cyclic grid mb x nb of A (nb x mb for A^T; narrower than the matrix:
 * cut once per call into a pinned host store, see rsvd_csr_tile); by default
 * full-width row ranges of at most 2^25 entries (fewer when the cap is
 * tight), copied straight from the host arrays (pinned memory lets the
 * copies overlap; a transpose the library builds is pinned).
 * A host A is copied to the device and processed in core when the plan has no
 * cap or the copy fits under it; otherwise it is processed out of core: its
 * block-cyclic tiles (edges opts.mb x opts.nb; by default full-width row
 * panels of about 512 MB, whose rows are contiguous in host memory; shrunk to
 * fit) are streamed from host memory through opts.n_slots device buffers on a side
 * stream, overlapped with the tile products, and the tiles that fit in the
 * rest of the cap stay resident for the later passes of the run (Section 3.5,
 * Section 3.7).  Streaming needs A in pinned host memory for the copies to
 * overlap.
 * BF16 plans processing A in core also keep a BF16 copy of A (2 m
 * round_up(n, 64) bytes, owned by the plan from the first such run, within the
 * cap when there is one): the first forward pass writes it and the later
 * BF16 passes read it (the same operands, so the same result; half the bytes
 * per pass).  BF16X3 plans (k + p <= 192) keep the split copy instead, BF16(A)
 * and BF16(A - BF16(A)) (4 m round_up(n, 64) bytes): the later passes read the
 * two parts the FP32 A would be split into, with no conversion.  Without room
 * for the copy every pass reads the FP32 A (the same results).
 * 16-bit storage (Section 3.2): an F32 plan with BF16 precision also takes a
 * dense A stored as BF16 or F16 (IEEE half; device: ld % 8 == 0 and a 16-byte
 * aligned base; host: copied to the device in core, never streamed), read
 * as is by every pass: the panels are rounded to A's 16-bit type (one
 * tensor-core product takes both operands in one type), and with opts.refine
 * the pass forming B^T splits its panel in two 16-bit parts (A X_hi + A X_lo,
 * about 16 significant bits) instead of splitting A, which is exact.  The
 * SVD is that of the matrix the 16-bit values represent.
 * Outputs (device, plan dtype): U m x k row-major, S k values descending,
 * V n x k row-major, so that A ~ U diag(S) V^T.  Each pair (u_i, v_i) is signed
 * so that the largest-magnitude entry of u_i is positive.  Synchronises
 * `stream`.  Errors: INVALID_ARG (shape/dtype mismatch), NOT_SPD, NO_CONVERGE,
 * TIMEOUT, CUDA.  The plan stays valid after an error. */
rsvd_status rsvd_run(rsvd_plan_t plan, const rsvd_matrix* A, void* U, void* S, void* V,
                     void* stream);

/* Persistence and recoverability (Section 3.8).  With a path set, rsvd_run
 * writes the range finder's basis after each of its steps -- step 0: Q_0 =
 * orth(A O); step 2i+1: Z_{i+1} = orth(A^T Q_i); step 2i+2: Q_{i+1} =
 * orth(A Z_{i+1}) -- to `path` (through path.tmp and a rename), with a header
 * holding the plan's m, n, k, p, q, seed, precision, dtype, kind, the step and
 * a fingerprint of A (sampled entries).  An rsvd_run whose plan and A match a
 * valid checkpoint at `path` loads its basis and continues after that step
 * (rsvd_plan_info: resumed_from); the result is the same as without the
 * interruption.  The file is removed when the run completes.
 * stop_after_step >= 0 makes rsvd_run return RSVD_ERR_INTERRUPTED right after
 * writing that step's checkpoint (a planned interruption).  path NULL or ""
 * turns checkpoints off.  Fixed q only (UNSUPPORTED with auto_q).  Host only. */
rsvd_status rsvd_plan_set_checkpoint(rsvd_plan_t plan, const char* path, int32_t stop_after_step);

/* Reads and validates the header of a checkpoint file (host only; magic,
 * version and header checksum).  Errors: INVALID_ARG if there is no valid
 * checkpoint at `path`. */
rsvd_status rsvd_checkpoint_info(const char* path, rsvd_checkpoint_info_t* out);

/* Exact thin SVD of a dense device matrix (Section 3: the library's
 * non-approximate path), t = min(m, n) <= 512: U m x t, S t, V n x t, same
 * dtype as A, signs as in rsvd_run.  All arithmetic in FP64 on T = A (m >= n)
 * or A^T (m < n).  t <= 256 and m*n <= 2^24: one-sided Jacobi on the columns
 * of T.  Otherwise T = Q R by CholeskyQR2 and the one-sided Jacobi on the t x t
 * R.  That path forms the Gram of T, so singular values below about 1e-7 of
 * the largest keep an absolute, not a relative, FP64 accuracy (columns
 * dependent to that level give zeros in S); a non-finite entry gives
 * RSVD_ERR_NOT_SPD.  On both paths the singular vectors of zero (or
 * rounding-level) singular values are not completed to an orthonormal set:
 * such columns of U or V may be zero.  Allocates and frees its own device
 * workspace (about 3 m n + 4 t^2 doubles on the CholeskyQR2 path).
 * Synchronises `stream`. */
rsvd_status rsvd_full(const rsvd_matrix* A, void* U, void* S, void* V, void* stream);

/* Backward pass (no counterpart in the paper): the adjoint of the rank-k
 * truncated SVD (Townsend, "Differentiating the Singular Value
 * Decomposition", 2016) evaluated at U, S, V as returned by rsvd_run on this
 * plan.  With F_ij = 1/(S_j^2 - S_i^2) (i != j; 0 on the diagonal and for
 * S_i^2, S_j^2 equal to within 1e-12 S_max^2),
 *   dA = U M V^T + (I - U U^T) dU S^-1 V^T + U S^-1 dV^T (I - V V^T),
 *   M  = (F o (U^T dU - dU^T U)) S + diag(dS) + S (F o (V^T dV - dV^T V)).
 * The projector terms treat the discarded spectrum as zero: this is the exact
 * derivative when A has rank k (or k = min(m, n)), and the usual truncated
 * approximation otherwise.  The range finder is not differentiated.
 * Inputs (device, plan dtype): U m x k, S k, V n x k, and the cotangents
 * dU m x k, dS k, dV n x k, any of which may be NULL (zero).  Output dA: m x n
 * row-major (leading dimension n), overwritten.  FP32 plans form the final
 * rank-2k product dA = [U M + P | U S^-1] [V | Q]^T on the tensor cores in
 * split BF16 (about 16 significant bits per operand, FP32 accumulation over
 * the 2k terms) and synchronise `stream` to read its status (TIMEOUT if a
 * pipeline wait expired); FP64 plans compute in FP64 and enqueue only.  Uses
 * the plan's workspace.  Errors: INVALID_ARG, TIMEOUT. */
rsvd_status rsvd_backward(rsvd_plan_t plan, const void* U, const void* S, const void* V,
                          const void* dU, const void* dS, const void* dV, void* dA, void* stream);

void rsvd_destroy(rsvd_plan_t plan);

/* ---- Tracing (Section 4.1 stage breakdown) ----------------------------------- */

/* Stages of rsvd_run, after the paper's list of processing stages in
 * Section 4.1 ("Preparation of O", "O*A^T", "Orthogonalization", "A^T*Q_r",
 * "SVD0 Preparation" + "SVD0", "Postprocessing") plus the host-to-device copy of a
 * host-resident A. */
typedef enum {
  RSVD_STAGE_GAUSSIAN = 0,    /* test matrix O */
  RSVD_STAGE_APASS_FWD = 1,   /* products A X */
  RSVD_STAGE_APASS_TRANS = 2, /* products A^T X, including B^T = A^T Q */
  RSVD_STAGE_ORTH = 3,        /* CholeskyQR2 of the range-finder panels */
  RSVD_STAGE_SMALL_SVD = 4,   /* QR of B^T + one-sided Jacobi */
  RSVD_STAGE_LIFT = 5,        /* U = Q U_B, V = Q_b W, signs */
  RSVD_STAGE_H2D = 6,         /* copy of a host-resident A */
  RSVD_STAGE_TOTAL = 7,       /* whole rsvd_run on the device */
  RSVD_STAGE_QUANTIZE = 8,    /* FP8 codes of A (FP8 precision only) */
  RSVD_STAGE_SWEEP = 9,       /* fused sweeps A^T (A W) over streamed row panels */
  RSVD_STAGE_COUNT = 10
} rsvd_stage;

/* Enable (1) or disable (0) stage timing: rsvd_run then records CUDA events
 * around each stage on its stream.  Host only; cheap when disabled. */
rsvd_status rsvd_plan_set_profiling(rsvd_plan_t plan, int32_t enable);

/* Times (ms, summed per stage) of the last profiled rsvd_run: `ms` receives
 * RSVD_STAGE_COUNT values; *apass_calls (may be NULL) the number of A-passes. */
rsvd_status rsvd_plan_stage_ms(rsvd_plan_t plan, double* ms, int32_t* apass_calls);

/* Out-of-core statistics of the last rsvd_run (all zero when it ran in core):
 * bytes copied host-to-device, tiles streamed per A-pass, and tiles kept
 * resident in device memory across the passes of the run.  Any pointer may be
 * NULL. */
rsvd_status rsvd_plan_stream_stats(rsvd_plan_t plan, uint64_t* h2d_bytes, int64_t* tiles_streamed_per_pass,
                                   int64_t* tiles_resident);

/* Number of CUDA kernels this library has launched in this process so far. */
unsigned long long rsvd_kernel_launches(void);

const char* rsvd_status_str(rsvd_status status);
const char* rsvd_last_error(void);

/* ---- Individual steps (used by the parity tests) -------------------------- */

/* Section 2.1 step 1: entries of the n x r Gaussian matrix O.  Entry (i, j) is
 * element e = i*r + j of one stream: Philox4x32-10 (Salmon et al., SC'11) with
 * key (seed mod 2^32, seed >> 32) and counter (g mod 2^32, g >> 32, 0, 0),
 * g = e >> 1, gives words x0..x3; N1 = ((x0<<32)|x1) >> 11, N2 = ((x2<<32)|x3) >> 11;
 * u1 = (N1+1)*2^-53; theta = 2 pi (2 N2 + 1) 2^-54; the value is
 * sqrt(-2 ln u1) * (e even ? cos theta : sin theta), computed in FP64 with
 * the library's own ln/sin/cos and rounded once (nearest-even) to out_dtype.
 * layout 0: out[i*ld + j] (ld >= r); layout 1 (transposed): out[j*ld + i]
 * (ld >= n).  out_dtype: F64, F32 or BF16.  Device output; enqueues only. */
rsvd_status rsvd_gaussian(uint64_t seed, int64_t n, int64_t r, int32_t out_dtype,
                          int32_t layout, void* out, int64_t ld, void* stream);

/* Block-cyclic tile map of Section 3.1 (host only): tile t = I*Tn + J covers
 * rows [I*mb, min(m,(I+1)*mb)) x cols [J*nb, min(n,(J+1)*nb)) and goes to slot
 * t mod n_slots.  Writes at most `cap` tiles to `out` (may be NULL when cap is
 * 0) and the total count to *count. */
rsvd_status rsvd_tile_map(int64_t m, int64_t n, int64_t mb, int64_t nb, int32_t n_slots,
                          rsvd_tile* out, int64_t cap, int64_t* count);

/* One A-pass (Section 2.1 steps 2 and 5, Eq. (3)): Y = A X (trans = 0) or
 * Y = A^T X (trans = 1), block-wise over the tile grid (mb, nb) of Section 2.3,
 * with the partial products of each tile row/column added in a fixed order.
 * A: dense device matrix (F64 or F32), or a CSR device matrix (below).
 * X: K x r row-major of A's dtype (K = n for trans = 0, m for trans = 1),
 * leading dimension ldx.  Y: M x r row-major of A's dtype, leading dimension
 * ldy.  prec: FP64 (A F64), FP32, BF16, BF16X3 or FP8 (A F32; A 16-byte
 * aligned with ld % 4 == 0; FP8 quantises A into the workspace with tiles
 * mb x nb rounded up to multiples of 128, or one tile when mb/nb are 0).  r <= 256 (CSR: 512, see below).  Needs `ws_bytes` >=
 * rsvd_apass_workspace(...).  FP64/FP32 enqueue only; BF16/BF16X3
 * synchronise `stream` and return TIMEOUT if a wait of the tensor-core
 * pipeline expired. */
size_t rsvd_apass_workspace(int64_t m, int64_t n, int32_t r, int32_t trans, int32_t prec,
                            int64_t mb, int64_t nb);
rsvd_status rsvd_apass(const rsvd_matrix* A, int32_t trans, int32_t prec, int32_t r,
                       const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t mb, int64_t nb,
                       void* ws, size_t ws_bytes, void* stream);

/* Section 2.1 steps 3-4: orthonormal basis of the columns of a device panel
 * Y (M x r row-major, F64 or F32, leading dimension ldy) by CholeskyQR2:
 * G = Y^T Y, G = R1^T R1 (Cholesky), Q1 = Y R1^-1, repeated once on Q1.  F64:
 * all in FP64.  F32: FP32 products summed in FP64 over row chunks, FP32
 * Cholesky and inverse (accurate while cond(Y) is below about 4e3).  Pivots
 * below 1e-13 (F64) / 1e-5 (F32) of their diagonal entry are deflated: the
 * column of Q is replaced by a fresh random direction and R gets a zero row.
 * Writes Q (M x r, same dtype, leading dimension ldq, may
 * not alias Y) and, when R is not NULL, the FP64 upper-triangular r x r factor
 * R = R2 R1 (row-major) with Y = Q R.  r <= 512, M >= r.  Needs `ws_bytes` >=
 * rsvd_orth_workspace(M, r).  Errors: NOT_SPD.  Synchronises `stream`. */
size_t rsvd_orth_workspace(int64_t M, int32_t r);
rsvd_status rsvd_orth(int32_t dtype, int64_t M, int32_t r, const void* Y, int64_t ldy,
                      void* Q, int64_t ldq, double* R, void* ws, size_t ws_bytes, void* stream);

/* Section 2.1 step 6 core: one-sided Jacobi SVD (Hestenes; stopping test of
 * Demmel & Veselic) of a device FP64 square matrix, given column-major as Mc
 * (column c at Mc + c*r, r <= 256): Mc W = U diag(sigma).  Outputs (device,
 * FP64): sigma (r, descending), U and W as r x r row-major with the columns
 * ordered like sigma, each pair (U_c, W_c) signed so that the entry of W_c
 * largest in magnitude is positive.  Needs `ws_bytes` >=
 * rsvd_small_svd_workspace(r).
 * Errors: NO_CONVERGE, TIMEOUT.  Synchronises `stream`. */
size_t rsvd_small_svd_workspace(int32_t r);
rsvd_status rsvd_small_svd(int32_t r, const double* Mc, double* sigma, double* U, double* W,
                           void* ws, size_t ws_bytes, void* stream);

/* Section 3.3 (sparse x dense product): Y = A X (trans = 0, CSR of A) or
 * Y = A^T X (trans = 1, using A.t_rowptr/t_colidx/t_val, which must be set)
 * for a CSR device matrix with FP32 values and FP32 accumulation in entry
 * order (deterministic).  X: K x r row-major FP32 (ldx), Y: M x r row-major
 * (ldy), overwritten; r <= 512.  Goes through rsvd_apass (mb, nb ignored)
 * with prec
 *   FP32    the panel X as given;
 *   BF16    X rounded to BF16 (round to nearest even) before the gathers;
 *   BF16X3  X rounded to 24-bit floats (sign, 8-bit exponent, 15 stored
 *           mantissa bits; round to nearest even on the FP32 bits), stored as
 *           a BF16 high part and a low byte: 3 bytes per gathered value,
 *           relative rounding error below 2^-16.
 * The gathers of panel rows (r values per stored entry) bound the pass, so
 * the compact panels move 1/2 and 3/4 of the FP32 bytes.  BF16 / BF16X3
 * passes need ws (16-byte aligned) of rsvd_csr_apass_workspace(A.nnz, K, r,
 * prec) bytes and ldy % 4 == 0 with Y 16-byte aligned.  For FP32 the
 * workspace is optional: ws may be NULL, and then every row is summed by one
 * warp; with ws_bytes >= rsvd_spmm_workspace(A.nnz, r), rows of more than
 * 1024 entries are split into 1024-entry segments summed by separate warps and
 * added in segment order (same result for any timing; the compact passes
 * always split).  A.nnz must equal rowptr[M] of the CSR used.  Enqueues only. */
size_t rsvd_spmm_workspace(int64_t nnz, int32_t r);

/* Workspace bytes of rsvd_apass on a CSR matrix with nnz entries whose panel X
 * has K rows (K = n for trans = 0, m for trans = 1), r columns, precision
 * prec (FP32: rsvd_spmm_workspace(nnz, r); BF16, BF16X3: that plus the
 * compact panel).  0 for r < 1 or K < 0. */
size_t rsvd_csr_apass_workspace(int64_t nnz, int64_t K, int32_t r, int32_t prec);

/* Host (CPU) transpose of a CSR matrix: from the CSR of the m x n matrix A
 * (rowptr m+1, colidx and val nnz = rowptr[m]) writes the CSR of A^T into
 * caller-allocated host arrays t_rowptr (n+1), t_colidx (nnz, row indices of
 * A) and t_val (nnz).  Within each row of A^T the entries come in increasing
 * row index of A (a stable counting sort), so the result does not depend on
 * the number of threads it uses.  Errors: INVALID_ARG (decreasing rowptr,
 * column index outside [0, n), NULL array). */
rsvd_status rsvd_csr_transpose(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx,
                               const float* val, int32_t* t_rowptr, int32_t* t_colidx, float* t_val);

/* Block (I, J) of the block-cyclic map of Section 3.1 for a CSR matrix (host
 * only, Section 3.3 sparse storage): the entries of the m x n CSR (rowptr
 * m+1, colidx and val rowptr[m]) that lie in rows [row0, row1) and columns
 * [col0, col1), as a CSR of row1 - row0 rows: t_rowptr (row1 - row0 + 1
 * offsets from 0), t_colidx (column indices minus col0) and t_val, each row's
 * entries in the order of the source row.  Caller-allocated arrays; with
 * cap = 0 only t_rowptr (may be NULL) and *nnz are written (a counting call),
 * otherwise t_colidx and t_val receive the entries and cap must be at least
 * their count.  The out-of-core sparse passes stream such blocks.
 * Errors: INVALID_ARG (ranges outside the matrix, decreasing rowptr, cap
 * below the count, NULL arrays with cap > 0). */
rsvd_status rsvd_csr_tile(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* colidx, const float* val,
                          int64_t row0, int64_t row1, int64_t col0, int64_t col1, int32_t* t_rowptr,
                          int32_t* t_colidx, float* t_val, int64_t cap, int64_t* nnz);

/* Host (CPU) conversion of a sparse m x n matrix in coordinate (COO) format
 * (Section 3.3: structure of arrays, row and column indices of 32 or 64 bits)
 * into the CSR the sparse A-passes take.  Inputs: nnz entries (rowidx[e],
 * colidx[e], val[e]), index arrays of index_bits = 32 (int32_t) or 64
 * (int64_t), in any order; repeated (i, j) pairs stay separate entries, so the
 * products see their sum.  Outputs, caller-allocated host arrays: rowptr
 * (m+1), out_colidx and out_val (nnz).  Within each row the entries keep their
 * COO order (a stable counting sort; the result does not depend on the
 * number of threads used).  The CSR of A^T, for A.t_rowptr/t_colidx/t_val,
 * is the same call with m and n and the two index arrays swapped.
 * Errors: INVALID_ARG (index outside [0, m) x [0, n), index_bits not 32 or 64,
 * nnz >= 2^31 or n >= 2^31, NULL array). */
rsvd_status rsvd_coo_to_csr(int64_t m, int64_t n, int64_t nnz, int32_t index_bits, const void* rowidx,
                            const void* colidx, const float* val, int32_t* rowptr, int32_t* out_colidx,
                            float* out_val);

/* FP8 storage of a dense F32 device matrix A (m x n): E4M3 codes (OCP 8-bit
 * floating point, 2023: bias 7, three mantissa bits, largest finite 448,
 * rounding to nearest even, saturating) with one scale per tile of rows
 * [I*qm, ...) x columns [J*qn, ...) (qm, qn multiples of 128, or at least m /
 * n for a single tile row / column).  The scale of a tile is the smallest
 * power of two s with amax / s <= 448 (amax: the tile's largest magnitude; s =
 * 1 for an all-zero tile, NaN for a tile holding NaN or infinity); entry
 * (i, j) is stored as code(a_ij / s).  Outputs (device, caller-owned): codes
 * m x ldc bytes (ldc >= n, ldc % 4 == 0, 4-byte aligned base), scales
 * cdiv(m, qm) x cdiv(n, qn) floats, row-major.  Enqueues only (one
 * stream-ordered allocation of the tile maxima).  Errors: INVALID_ARG. */
rsvd_status rsvd_fp8_quantize(const rsvd_matrix* A, int64_t qm, int64_t qn, uint8_t* codes, int64_t ldc,
                              float* scales, void* stream);

/* ---- Variant without allocation (no counterpart in the paper) --------------- */

/* Largest r accepted by rsvd_small_svd_noalloc. */
#define RSVD_NOALLOC_MAX_R 256

/* rsvd_small_svd for callers that cannot allocate device memory -- for example
 * code whose device memory is entirely reserved by a framework's memory pool,
 * or latency-sensitive code that must not let cudaMalloc/cudaFree synchronise
 * the device -- and therefore cannot provide the workspace rsvd_small_svd
 * takes.  Same arguments and results as rsvd_small_svd, minus the workspace;
 * it calls no allocation routine, and runs the same phases as rsvd_small_svd
 * (so both give the same results).  Its scratch is one static device array of
 * about 19 MiB (rsvd_small_svd's workspace at r = RSVD_NOALLOC_MAX_R: 38
 * FP64 and one FP32 RSVD_NOALLOC_MAX_R^2 matrices plus a few words) that
 * every GPU loading this library keeps until the process exits.  The first
 * call on a device looks up that array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call uses the same
 * array: calls whose work overlaps on the GPU (other streams, other host
 * threads) race and return wrong results; serialise them.  The words that must
 * start at zero are cleared by each call.  Errors: INVALID_ARG for r outside
 * [1, RSVD_NOALLOC_MAX_R] (checked on the host before any GPU work),
 * NO_CONVERGE, TIMEOUT, CUDA.  Synchronises `stream`. */
rsvd_status rsvd_small_svd_noalloc(int32_t r, const double* Mc, double* sigma, double* U, double* W,
                                   void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RSVD_GB300_H */
