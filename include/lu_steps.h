/*
 * lu_steps.h -- step-level entry points of libgb300lu.so, one per step of the
 * blocked LU iteration, so that each step can be checked on its own.
 *
 * The steps are those of the paper's blocked right-looking LU (arxiv
 * 2202.13995, section "Base Implementation", figure "lu_iteration"): factor
 * the block column ("LU" and "left" blocks, here one panel with partial
 * pivoting), update the "top" blocks with L (a triangular solve), and update
 * the "inner" blocks by a matrix multiplication.
 *
 * Conventions: as lu.h, except that every matrix here is ROW-major (element
 * (i, j) at p[i*ld + j]), which is the library's internal working layout.
 * Each call enqueues its work on the context's stream and returns; status bits
 * raised on the device (timeout, range) are reported by lu_ctx_status.
 */
#ifndef GB300_LU_STEPS_H
#define GB300_LU_STEPS_H

#include "lu.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Panel factorization with partial pivoting of the m x w row-major panel dP
 * (FP64 when prec is LU_F64, FP32 otherwise), m >= w, w <= 512, in place:
 * L below the diagonal (unit diagonal implied), U on and above it.
 * dIpiv (device, w ints) receives the 1-based pivot rows (relative to the
 * panel), dInfo (device, 1 int) the first zero pivot (1-based) or 0. */
int lu_step_panel(lu_ctx ctx, lu_prec prec, int m, int w, void *dP, int ld, int *dIpiv, int *dInfo);

/* The same panel factorization for callers that cannot allocate device
 * memory.  The paper has no counterpart: this entry point exists for callers
 * that must not call cudaMalloc when they factor a panel -- for instance code
 * that runs while another thread captures a CUDA graph in global capture
 * mode, or a service that reserves all of its device memory at start-up and
 * allows no allocation afterwards.  lu_step_panel allocates its scratch on
 * first use; this variant allocates nothing and creates no context object.
 *
 * Its scratch is one fixed array of about 96 KB in device memory, held on
 * every GPU that loads the library until the process exits.  Limits: w <= 512
 * (a wider panel returns -4, argument 4 invalid) and a panel whose rows fit
 * the CTAs' shared memory (on GB300 about 78,000 rows in FP64 and 200,000 in
 * FP32; a taller one returns -3); both are checked before anything is
 * enqueued.  The panel runs
 * on at most 160 CTAs (one per SM on GB300's 152 SMs; a larger device uses
 * 160 of its SMs).  The first call on each device (with that device current)
 * looks up the array's device address and the SM count; make that first call
 * before any stream capture begins.
 *
 * Every call uses the same array and leaves its last contents there: calls
 * whose work overlaps on the GPU (on different streams, or from different
 * threads without ordering) race on it and give wrong results.
 *
 * Arguments as lu_step_panel, with the stream passed directly (a
 * cudaStream_t, NULL = legacy default stream) and dStatus (device, 1 int),
 * which the call zeroes and the kernel then ORs device status bits into
 * (1 = a bounded device wait timed out, 2 = a NaN was met).  dInfo receives
 * 0 or the first zero pivot (1-based).  Asynchronous: returns once enqueued. */
int lu_step_panel_static(void *cuda_stream, lu_prec prec, int m, int w, void *dP, int ld, int *dIpiv, int *dInfo,
                         int *dStatus);

/* Top-block update U12 = L11^-1 A12: dL (w x w row-major, only the strict
 * lower triangle is read; unit diagonal), dX (w x N row-major) overwritten,
 * 1 <= w <= 512.  LU_F64 and LU_F32: substitution in that precision.
 * LU_BF16 / LU_FP16: the form the mixed-precision factorizations use -- FP32,
 * with each 32 x 32 diagonal block of L11 inverted and applied as a product
 * (the rounding of U12 differs from substitution; the factor is refined). */
int lu_step_trsm(lu_ctx ctx, lu_prec prec, int w, int N, const void *dL, int ldl, void *dX, int ldx);

/* Inner-block update C -= A B with C m x n, A m x k, B k x n, row-major.
 * LU_F64: FP64 A, B, C on the CUDA cores.  LU_F32: FP32 on the CUDA cores.
 * LU_BF16 / LU_FP16: FP32 A, B, C; A and B are rounded to BF16 / FP16
 * (round-to-nearest-even) and multiplied on the tensor cores (tcgen05) with
 * FP32 accumulation, then subtracted from C in FP32. */
int lu_step_gemm(lu_ctx ctx, lu_prec prec, int m, int n, int k, void *dC, int ldc, const void *dA, int lda,
                 const void *dB, int ldb);

/* Inner-block update C -= A B in FP64 (row-major FP64 device arrays, C m x n,
 * A m x k, B k x n, 1 <= k <= 256) with the products on the BF16 tensor cores
 * by error-free splitting, as lu_factor_ex's LU_FACTOR_OZAKI (same error
 * bound).  Workspace: the context's step scratch (grown as needed).  Returns
 * -5 for k outside 1..256, LU_ERANGE (at the next lu_ctx_status) for
 * non-finite operands. */
int lu_step_gemm_ozaki(lu_ctx ctx, int m, int n, int k, double *dC, int ldc, const double *dA, int lda,
                       const double *dB, int ldb);

/* Failure-path probe: runs one of the library's bounded device waits on a
 * condition that nothing ever satisfies -- kind 0: a triangular solve's wait
 * for a solution block that is never published; 1: a panel's grid barrier
 * that the other CTA never reaches; 2: a tensor-core kernel's mbarrier wait
 * for a copy that never lands.  The wait gives up after the library's
 * compiled-in limit (2 s), the kernel sets the timeout bit and returns, and
 * the call returns LU_ETIMEOUT with the status cleared; the context stays
 * usable.  Synchronizes.  Returns -1 (ctx NULL), -2 (kind not 0..2). */
int lu_step_wait_probe(lu_ctx ctx, int kind);

/* The seeded synthetic input of the benchmarks, generated on the device
 * (HPL generates its input: arxiv 2202.13995, section "High Performance
 * Linpack").  Fills the rows x cols column-major FP64 block dA (ld >= rows):
 * element (i, j) is draw k = i + j * rows of stream stream_id of `seed` --
 * SplitMix64 in counter mode, z = mix64(mix64(seed ^ stream_id *
 * 0xD1B54A32D192ED03) + (k + 1) * 0x9E3779B97F4A7C15), value (z >> 11) *
 * 2^-53 - 0.5, uniform in [-0.5, 0.5) -- plus diag_shift where i == j.
 * Stream 0 with rows = cols = n is the matrix A of the workloads (shift 0 or
 * n/4), stream 1 with rows = n, cols = nrhs their right-hand sides.  The same
 * bits as the package's host generator.  Enqueued on cuda_stream (a
 * cudaStream_t); returns -1..-4 for invalid arguments. */
int lu_generate(double *dA, int rows, int cols, int ld, uint64_t seed, int stream_id, double diag_shift,
                void *cuda_stream);

/* Arithmetic-rate probe of the current device, for roofline denominators
 * (the paper has no counterpart): kind 0 = FP64 fused multiply-add on the
 * CUDA cores, 1 = FP64 warp matrix multiply-accumulate (mma.sync m8n8k4),
 * 2 = FP32 fused multiply-add on the CUDA cores.  Runs a register-only kernel
 * on every SM for a few tens of milliseconds and stores the best of three
 * timed launches in *tflops (host).  Synchronizes; allocates 64 bytes.
 * Returns -1 (kind not 0..2), -2 (tflops NULL), LU_ECUDA / LU_ENOMEM. */
int lu_peak_probe(int kind, double *tflops);

/* Read and clear the context's device status bits (synchronizes): returns
 * LU_OK, LU_ETIMEOUT or LU_ERANGE. */
int lu_ctx_status(lu_ctx ctx);

/* Phase profiling.  When enabled, the library records a CUDA event pair on
 * the context's stream around every kernel launch of the factorization and
 * solve, per phase.  lu_profile_read synchronizes and returns, per phase, the
 * summed device milliseconds and the number of launches since the last read
 * (phases: 0 panel, 1 laswp, 2 trsm, 3 cast, 4 gemm, 5 solve, 6 residual,
 * 7 other; arrays of LU_NPHASE entries), then clears the record. */
#define LU_NPHASE 8
int lu_profile_enable(lu_ctx ctx, int enable);
/* Phases recorded while profiling is enabled: bit p of phase_mask selects
 * phase p (default: every phase).  Selecting one phase keeps the other
 * launches free of events, e.g. to time one kernel inside a timed region. */
int lu_profile_select(lu_ctx ctx, unsigned phase_mask);
int lu_profile_read(lu_ctx ctx, double *ms, long long *launches);

/* Kernels this context has launched so far (all phases, profiling or not). */
long long lu_launch_count(lu_ctx ctx);

/* Number of SMs of the context's device and the library's build tag (static
 * string naming the target architecture). */
int lu_device_sm_count(lu_ctx ctx);
const char *lu_build_tag(void);

#ifdef __cplusplus
}
#endif
#endif /* GB300_LU_STEPS_H */
