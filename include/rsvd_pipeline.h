/*
 * rsvd_pipeline.h - pipelined host inputs for consecutive rsvd_run calls of
 * one plan (librsvd_gb300.so).
 *
 * Section 3.7 of arXiv:1907.06470 overlaps the transfers of the matrix with
 * the computation.  Within one call, rsvd_run already lets its first forward
 * pass take the rows of a host A as they land; across calls, a stream of
 * host matrices can keep the link busy while the previous matrix is being
 * factored: each call's copy is issued (rsvd_plan_prefetch) before the
 * previous call runs, so the link and the passes work at the same time.
 * Every matrix still crosses the link once per call.
 *
 * Typical use, factoring A_0, A_1, ... in turn:
 *     rsvd_plan_prefetch(plan, &A_0);
 *     for i = 0, 1, ...:
 *         rsvd_plan_prefetch(plan, &A_{i+1});    (when there is a next one)
 *         rsvd_run(plan, &A_i, U, S, V, stream); (takes the copy of A_i)
 */
#ifndef RSVD_GB300_PIPELINE_H
#define RSVD_GB300_PIPELINE_H

#include "rsvd.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Starts copying the dense host matrix A to a device buffer of the plan and
 * returns without waiting for the copy.
 *   A: the plan's m x n, kind DENSE, location HOST, the plan's dtype (or BF16 /
 *      FP16 for a BF16 plan, as rsvd_run allows); row-major with ld >= n.
 *      Pinned host memory (cudaHostAlloc / cudaHostRegister) lets the copy
 *      run asynchronously; the caller must not change or free A until the run
 *      that takes it has returned.
 * The copy goes in row chunks of about 256 MB on the plan's copy stream,
 * after the plan's earlier copies, into one of two device buffers of the
 * plan (allocated on first use, m x n elements each, rows padded to 8 for
 * 16-bit A; counted against the plan's memory cap).  At most two prefetches
 * are pending at a time.
 * The next rsvd_run of the plan takes the oldest pending prefetch when its A
 * has the same descriptor (data, m, n, ld, dtype): its first forward pass
 * consumes the rows as they land, exactly as for a copy rsvd_run makes itself
 * (the results are the same bits).  A run given any other matrix drops the
 * pending prefetches (their copies still complete in order) and copies its A
 * itself; under a memory cap, such a run (and a streamed run) first frees the
 * idle prefetch buffers, so that the plan stays within the cap.
 * Errors: INVALID_ARG (NULL, a matrix that is not the plan's shape and dtype,
 * not dense on the host, or two prefetches already pending), UNSUPPORTED (A
 * would be streamed: it does not fit the plan's cap in core), CAP_TOO_SMALL
 * (the prefetch buffers do not fit the cap), OOM, CUDA. */
rsvd_status rsvd_plan_prefetch(rsvd_plan_t plan, const rsvd_matrix* A);

#ifdef __cplusplus
}
#endif

#endif /* RSVD_GB300_PIPELINE_H */
