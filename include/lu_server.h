/*
 * lu_server.h -- a serving loop for dense solves (continuous batching).
 *
 * Each request is the HPL problem of arxiv 2202.13995 (section "High
 * Performance Linpack": A x = b via A = L U, L y = b, U x = y), solved by
 * lu_factor (the blocked right-looking LU with partial pivoting) in the
 * server's factor precision plus lu_refine (FP64 iterative refinement to HPL
 * scaled residual < 16).  The paper has no serving layer; this one follows the
 * serving pattern of the solver's specification: requests that arrive while
 * others run are admitted as slots and memory free up, and their work overlaps
 * on the GPU.
 *
 * Slots: max_slots worker threads, each with its own library context and CUDA
 * stream on the device current at lu_server_create.  A free slot takes the
 * oldest queued request whose memory fits the HBM budget (factor working copy,
 * operands, scratch and refinement vectors, counted exactly as the library
 * allocates them), evicting least-recently-used resident factors first.
 * Requests overlap on the device, factorizations included: the trailing-update
 * CTAs leave room for a panel CTA on every SM, and a cooperative panel launch
 * that finds no room retries (bounded).  The environment variable
 * GB300LU_SERVER_SERIAL_FACTOR runs factorizations one at a time instead.
 * Requests with n >= 2048 in BF16 or FP16 are factored with block width 256
 * (lu_factor's default is 128 up to n = 12288): with many requests on the
 * device their trailing updates share HBM, and the wider block halves their
 * traffic per FLOP.
 * The slots' contexts factor without the lookahead (other requests fill the
 * SMs it would use), run their triangular solves on 8 persistent CTAs
 * (GB300LU_SERVER_SOLVE_CTAS) and wait for the device asleep rather than
 * spinning.  A serving process should set CUDA_DEVICE_MAX_CONNECTIONS=32 in
 * its environment before it creates its CUDA context: with the default of 8
 * hardware work queues, the slots' streams share queues and one request's
 * kernels wait behind another's (measured on GB300 with the served mix: 973
 * solves/s at 8 slots with 8 queues, 1204 with 32).
 *
 * Small requests (n <= 512 and nrhs <= 8) go to a batch slot instead: it
 * takes every queued small request at once (up to 4096), solves them in one
 * persistent launch of the batched solver (lu_batched.h: FP32 factor + FP64
 * refinement to scaled residual < 16, whatever the server's factor precision)
 * and reports them with slot = max_slots.  Its working memory is counted in
 * the budget while it runs.  Small requests never leave a factor resident and
 * never use one (refactoring them in the batch costs less than any reuse).
 *
 * Resident factors: a request with keep_factor != 0 leaves its factor resident
 * under factor_key (counted in the budget).  A later request with the same
 * key and use_resident != 0 skips the factorization; if the factor was evicted
 * it is factored again and the result says so.
 *
 * Determinism: a request's route (worker slot or batch slot), kernels and
 * launch shapes depend only on the request (n, nrhs, precision), and the
 * batched solver computes each system in one CTA independently of the rest of
 * its batch, so a result has the same bits whether it runs alone or among
 * others.
 *
 * Thread safety: every lu_server_* call may come from any host thread.
 * Buffers: the caller owns A, B and X (device, column-major FP64) and keeps
 * them alive and unchanged until the request is done (and A while its factor
 * is resident and may be reused).
 */
#ifndef GB300_LU_SERVER_H
#define GB300_LU_SERVER_H

#include <stddef.h>
#include <stdint.h>

#include "lu.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lu_server_s *lu_server;

typedef struct {
  int n, nrhs;            /* 1 <= nrhs <= 32 */
  const double *dA;       /* n x n */
  int lda;
  const double *dB;       /* n x nrhs, read */
  int ldb;
  double *dX;             /* n x nrhs, written (must not alias dB) */
  int ldx;
  uint64_t factor_key;    /* resident-factor key (0 = none) */
  int keep_factor;        /* keep this request's factor resident under factor_key */
  int use_resident;       /* reuse the resident factor of factor_key if present */
} lu_request;

typedef struct {
  int status;             /* LU_OK, LU_ENOTCONV, LU_ESINGULAR, LU_ENOMEM, LU_ERANGE, LU_ETIMEOUT, ... */
  int iters;              /* refinement corrections applied */
  double scaled_resid;    /* largest final HPL scaled residual */
  int reused_factor;      /* 1 if a resident factor was used */
  int refactored;         /* 1 if a requested resident factor had been evicted */
  int slot;               /* worker slot that ran it (max_slots: the batch slot) */
  uint64_t t_submit_ns, t_start_ns, t_done_ns; /* CLOCK_MONOTONIC */
} lu_result;

/* Start a server on the current device.  hbm_budget_bytes bounds the memory
 * of running requests plus resident factors; prec is the factor precision
 * (LU_BF16, LU_FP16, LU_F32 or LU_F64); max_slots in 1..64. */
int lu_server_create(lu_server *out, size_t hbm_budget_bytes, lu_prec prec, int max_slots);

/* Queue a request; *ticket identifies it.  Returns -k for an invalid
 * argument k, LU_ENOMEM if the request alone exceeds the budget. */
int lu_server_submit(lu_server s, const lu_request *req, uint64_t *ticket);

/* LU_EAGAIN while the ticket is queued or running; LU_OK with *out filled once
 * it is done (the result stays readable until the server is destroyed). */
int lu_server_poll(lu_server s, uint64_t ticket, lu_result *out);

/* Block until the ticket is done, then as lu_server_poll. */
int lu_server_wait(lu_server s, uint64_t ticket, lu_result *out);

/* Counters: requests done, resident factors, bytes in use, evictions. */
int lu_server_stats(lu_server s, uint64_t *done, int *resident, size_t *bytes_in_use, uint64_t *evictions);

/* Finish every queued request, stop the slots and free resident factors. */
int lu_server_destroy(lu_server s);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LU_SERVER_H */
