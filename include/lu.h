/*
 * lu.h -- C ABI of the GB300 dense LU solver (libgb300lu.so).
 *
 * The solver answers the problem of the HPL benchmark (arxiv 2202.13995,
 * section "High Performance Linpack", first paragraph): solve A x = b for a
 * dense A in R^{n x n} by factoring A = L U, then solving L y = b and
 * U x = y.  The factorization is the blocked right-looking iteration of the
 * paper's "Base Implementation" (figure "lu_iteration": factor a block column,
 * update the top blocks with L, update the inner blocks by a matrix
 * multiplication), here with partial pivoting (P A = L U, L unit lower).
 *
 * Conventions (all entry points):
 *   - Matrices are column-major FP64 in device memory: element (i, j) of A is
 *     dA[i + j*lda], lda >= n.  Right-hand sides B are n x nrhs with ldb >= n.
 *   - Pointers named d* are device pointers; the caller owns every buffer it
 *     passes and must keep it alive until the work enqueued on the context's
 *     stream has finished.
 *   - All work is enqueued on the CUDA stream given to lu_create (the caller's
 *     stream, e.g. torch.cuda.current_stream().cuda_stream); unless stated
 *     otherwise a call returns once its work is enqueued.
 *   - Return value: LU_OK (0), a negative value -k when argument k (1-based)
 *     is invalid, or one of the LU_E* codes below.  No C++ exception crosses
 *     this boundary.
 *   - ipiv / info use the LAPACK convention: 1-based; info = j > 0 means
 *     U(j, j) is exactly zero (the factorization still completes).
 */
#ifndef GB300_LU_H
#define GB300_LU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Factor precision.  LU_F64: FP64 panel, FP64 trailing update (the plain
 * FP64 solve).  LU_BF16 / LU_FP16: FP32 working matrix and panel, trailing
 * update on the tensor cores with BF16 / FP16 operands and FP32 accumulation;
 * solutions are brought to FP64 accuracy by lu_refine.  LU_F32: FP32 panel and
 * FP32 trailing update on the CUDA cores. */
typedef enum { LU_F64 = 0, LU_BF16 = 1, LU_FP16 = 2, LU_F32 = 3 } lu_prec;

enum {
  LU_OK = 0,
  LU_ESINGULAR = 1, /* a solve was asked of factors with an exactly zero pivot */
  LU_ENOMEM = 2,    /* device allocation failed */
  LU_ENOTCONV = 3,  /* lu_refine reached max_iter; x holds the last iterate */
  LU_ERANGE = 4,    /* a 16-bit cast overflowed (FP16 > 65504) or a NaN was met */
  LU_ETIMEOUT = 5,  /* a bounded device wait hit its limit; results are invalid */
  LU_EAGAIN = 6,    /* (server) the ticket is not finished yet */
  LU_ECUDA = 7,     /* a CUDA runtime call failed (launch, copy, ...) */
  LU_EINTERNAL = 8  /* anything else */
};

typedef struct lu_ctx_s *lu_ctx;
typedef struct lu_fact_s *lu_fact;

/* Create a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  The context owns a few
 * KB of device scratch and a pinned status word; its device memory comes from
 * the stream-ordered pool (lu_create_ex takes an allocator instead).  Not
 * thread-safe: one host thread per context at a time. */
int lu_create(lu_ctx *out, void *cuda_stream);

/* Device-memory callbacks for a context's workspace (lu_create_ex).
 * alloc(user, bytes, stream) returns device memory usable by work enqueued on
 * `stream` from now on (NULL on failure: the call then returns LU_ENOMEM);
 * release(user, ptr, bytes, stream) gives a block back once the work already
 * enqueued on `stream` has no further use for it -- the block must not be
 * reused for other work until that work has finished, as with cudaFreeAsync
 * or a caching allocator that records the stream (torch's
 * caching_allocator_alloc / caching_allocator_delete behave this way).
 * `bytes` is the size the block was allocated with.  The callbacks run on
 * the host thread that calls into the library. */
typedef void *(*lu_alloc_fn)(void *user, size_t bytes, void *cuda_stream);
typedef void (*lu_free_fn)(void *user, void *ptr, size_t bytes, void *cuda_stream);

/* lu_create with the context's device memory drawn from the caller's
 * allocator: every buffer the context and the factorizations, solves,
 * refinements, batches and step calls made through it allocate (factors,
 * pivots, workspaces, status words) comes from alloc and goes back through
 * release, on the context's stream; lu_destroy releases the context's own.
 * Factors keep the allocator of the context that created them.  alloc and
 * release both NULL = the stream-ordered pool (cudaMallocAsync), as
 * lu_create; -3 when only one of them is given. */
int lu_create_ex(lu_ctx *out, void *cuda_stream, lu_alloc_fn alloc, lu_free_fn release, void *user);

/* Synchronize the context's stream and free everything the context owns.
 * Factors created from it must be freed first. */
void lu_destroy(lu_ctx ctx);

/* Text of a status code (static storage). */
const char *lu_strerror(int code);

/* Factor P A = L U of the n x n matrix dA (not modified; read during this
 * call's enqueued work only).  nb is the block width of the paper's blocked
 * iteration (its LOCAL_MEM_BLOCK size); nb = 0 picks the block width of the
 * library's tuning table for (n, prec, flags) -- the fastest of an offline
 * sweep of whole solves on this GPU (lu_default_nb tells which).  The factors, pivots and workspace are owned by *out, which
 * lu_fact_free releases.  If info is non-NULL the call synchronizes the stream
 * and stores the LAPACK info (0, or the first zero pivot j, 1-based); with
 * info NULL the call is asynchronous and lu_fact_info reads it later.
 * Returns LU_ETIMEOUT / LU_ERANGE if a device status bit was raised (only
 * seen when info is non-NULL). */
int lu_factor(lu_ctx ctx, int n, const double *dA, int lda, lu_prec prec, int nb, lu_fact *out, int *info);

/* lu_factor with options.  flags = 0 is lu_factor.  LU_FACTOR_NOPIV: the
 * paper's own variant (HPL-AI rules: A diagonally dominant, so no pivoting;
 * section "High Performance Linpack"), with its four block operations per
 * iteration: LU of the diagonal block, top blocks A12 <- L11^-1 A12, left
 * blocks A21 <- A21 U11^-1, inner blocks A22 <- A22 - A21 A12.  ipiv is then
 * the identity.  Without diagonal dominance this variant can be unstable or
 * hit a zero pivot (info > 0).
 * LU_FACTOR_OZAKI (prec = LU_F64 only, nb <= 256): the FP64 trailing update
 * C -= L21 U12 (section "Base Implementation", the inner blocks) runs on the
 * BF16 tensor cores by error-free splitting (Ozaki scheme): each operand row
 * or column is scaled by a power of two and cut into 8 slices of 7-bit
 * integers, the 36 slice products with p + q <= 7 are exact in the FP32
 * accumulator, and they are combined exactly in 64-bit integers before one
 * FP64 rounding.  The error of an update element C - sum_k a b is below
 * 2^-53 * ((1.13 k + 4) * 2^(e_i + f_j) + sum_k |a b| + |result|), with 2^e_i and
 * 2^f_j the powers of two just above the largest |L21| of row i and |U12| of
 * column j: the order of an FP64 dot product's error bound.  Non-finite
 * operands fail with LU_ERANGE. */
enum { LU_FACTOR_NOPIV = 1, LU_FACTOR_OZAKI = 2 };
int lu_factor_ex(lu_ctx ctx, int n, const double *dA, int lda, lu_prec prec, int nb, int flags, lu_fact *out,
                 int *info);

/* Synchronize and read the LAPACK info of a factorization (and the device
 * status: LU_ETIMEOUT / LU_ERANGE when raised). */
int lu_fact_info(lu_fact f, int *info);

/* Copy the pivots (n ints, 1-based, LAPACK ipiv) to device memory dIpiv. */
int lu_fact_ipiv(lu_fact f, int *dIpiv);

/* Copy the factors, in the factor precision widened to FP64, to the n x n
 * column-major device buffer dLU (L strictly below the diagonal, U on and
 * above it, rows in pivoted order as in LAPACK dgetrf). */
int lu_fact_lu(lu_fact f, double *dLU, int ldlu);

/* Solve A X = B from the factors: B (n x nrhs, FP64) is overwritten with X.
 * For LU_F64 factors this is the FP64 solve; for lower-precision factors it is
 * the first iterate x0 (the solve runs in the factor's working precision).
 * Returns LU_ESINGULAR (without touching B) if the factorization met a zero
 * pivot; synchronizes only in that check's first call per factorization. */
int lu_solve(lu_fact f, int nrhs, double *dB, int ldb);

/* Mixed-precision iterative refinement: x0 = solve(b); then repeat
 * r = b - A x (FP64), stop for a column once its HPL scaled residual
 * ||r||_inf / (eps (||A||_inf ||x||_inf + ||b||_inf) n), eps = 2^-53, is below
 * tol, else d = solve(r) and x += d (FP64).  dA must be the matrix that was
 * factored.  dX (n x nrhs) receives the solution.  iters (host, may be NULL)
 * receives the number of corrections applied, scaled_resid (host, may be
 * NULL) the largest final scaled residual over the columns.  Synchronizes the
 * stream once per iteration.  Returns LU_ENOTCONV after max_iter corrections
 * without convergence (dX still holds the last iterate). */
int lu_refine(lu_fact f, const double *dA, int lda, const double *dB, int ldb, double *dX, int ldx, int nrhs,
              double tol, int max_iter, int *iters, double *scaled_resid);

/* HPL scaled residual of dX against (dA, dB), per column, computed in FP64 on
 * the device; out (host, nrhs doubles) receives the values.  Synchronizes. */
int lu_scaled_residual(lu_ctx ctx, int n, int nrhs, const double *dA, int lda, const double *dX, int ldx,
                       const double *dB, int ldb, double *out);

/* The infinity norms behind the scaled residual, per column q of dX:
 * out[4q] = ||b - A x||, out[4q+1] = ||A||, out[4q+2] = ||x||, out[4q+3] =
 * ||b|| (r computed in FP64 on the device; out is host memory, 4*nrhs
 * doubles).  They give the HPL form above and the paper's own shape of the
 * check, ||r|| / (n ||b|| eps) (arxiv 2202.13995, section "High Performance
 * Linpack", where its printed formula has no residual in it and is read this
 * way).  Synchronizes.  Errors as lu_scaled_residual. */
int lu_residual_norms(lu_ctx ctx, int n, int nrhs, const double *dA, int lda, const double *dX, int ldx,
                      const double *dB, int ldb, double *out);

/* The block width nb = 0 selects for an n x n factorization of precision
 * prec with lu_factor_ex flags `flags` (the tuning table's entry; at most n).
 * Returns -1 (n < 0), -2 (prec invalid). */
int lu_default_nb(int n, lu_prec prec, int flags);

/* Device bytes that lu_factor (block width nb, 0 = default) plus lu_refine
 * with nrhs right-hand sides allocate for an n x n system on the current
 * device (0 on an invalid argument).  For memory budgeting. */
size_t lu_fact_bytes(int n, int nrhs, lu_prec prec, int nb);

/* Release a factorization (stream-ordered: safe to call with work in flight). */
void lu_fact_free(lu_fact f);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LU_H */
