/*
 * lu_batched.h -- many independent small dense solves in one persistent launch.
 *
 * Each system i is the HPL problem of arxiv 2202.13995 (section "High
 * Performance Linpack": A_i x_i = b_i by A_i = L_i U_i, then L y = b,
 * U x = y), factored by the same blocked right-looking LU with partial
 * pivoting as lu_factor (block width 32), in FP32, then brought to FP64
 * accuracy by iterative refinement: r = b - A x in FP64, stop a system once
 * every column's HPL scaled residual ||r||/(eps (||A|| ||x|| + ||b||) n),
 * eps = 2^-53, is below tol, else d = solve(r) in FP32 and x += d in FP64.
 *
 * One CTA solves one system start to finish, so a system's result does not
 * depend on which other systems share the batch, on their order, or on the
 * tuned launch shape: a system gives the same bits alone and in any batch.
 *
 * Conventions: as lu.h (column-major FP64 device buffers, caller-owned).
 * Limits: 1 <= n_i <= 512, 1 <= nrhs_i <= 8.
 */
#ifndef GB300_LU_BATCHED_H
#define GB300_LU_BATCHED_H

#include "lu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lu_batch_s *lu_batch;

/* Plan a batch of `count` systems.  Host arrays (count entries each): n, nrhs,
 * lda, ldb, ldx, and the device pointers dA (n x n), dB (n x nrhs, right-hand
 * sides, read only), dX (n x nrhs, solutions; may equal dB).  prec must be
 * LU_F32 (FP32 factor + FP64 refinement).  The plan copies the descriptors to
 * the device, orders the systems by decreasing n, sizes its scratch, and
 * captures the launch in a CUDA graph.  tune != 0 times the candidate launch
 * shapes (threads per CTA, CTAs per SM) on this batch (running it) and keeps
 * the fastest; the choice changes timing only, never results. */
int lu_batch_create(lu_ctx ctx, int count, const int *n, const int *nrhs, const double *const *dA, const int *lda,
                    const double *const *dB, const int *ldb, double *const *dX, const int *ldx, lu_prec prec,
                    double tol, int max_iter, int tune, lu_batch *out);

/* Run the plan on the context's stream (one graph launch).  Device outputs
 * (count entries each, may be NULL except dInfo): dInfo[i] = 0 converged,
 * j > 0 first zero pivot (1-based; x_i untouched), -1 not converged within
 * max_iter (x_i = last iterate), -2 a bounded device wait timed out;
 * dIters[i] = corrections applied; dResid[i] = largest final scaled residual. */
int lu_batch_run(lu_batch b, int *dInfo, int *dIters, double *dResid);

/* Launch shape chosen for the plan (threads per CTA, CTAs per SM) and, if it
 * was tuned, the best measured time in milliseconds (else 0). */
int lu_batch_shape(lu_batch b, int *threads, int *ctas_per_sm, float *ms);

/* Release the plan (stream-ordered). */
void lu_batch_free(lu_batch b);

/* One-call form: plan, run and free; dB holds b on entry and
 * x on return; dInfo as in lu_batch_run.  Synchronizes the stream. */
int lu_solve_batched(lu_ctx ctx, int count, const int *n, const int *nrhs, const double *const *dA, const int *lda,
                     double *const *dB, const int *ldb, lu_prec prec, int *dInfo);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LU_BATCHED_H */
