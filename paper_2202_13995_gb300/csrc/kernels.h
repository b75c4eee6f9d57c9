// Internal launchers of the LU library (not part of the C ABI).
//
// Layout of the working matrix W: ROW-major, W[i*ldw + j] = A(i, j), in the
// factor's working type T (double for LU_F64, float otherwise).  Row
// interchanges are then contiguous copies, and the trailing update's A operand
// (L21) is K-major as stored.  The caller's A stays column-major FP64.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {

struct DevInfo {
  int sm_count;
  int max_smem_optin;
};

// Raise a kernel's dynamic shared-memory limit to the device maximum, once per
// kernel and device (thread-safe).  Launches then never depend on a per-call
// attribute value, which concurrent host threads launching the same kernel
// with different sizes would race on.
cudaError_t allow_max_smem(const void* func);

// ---------------------------------------------------------------- panel.cu
// Scratch of the cooperative panel kernel (global memory, owned by the caller).
struct PanelScratch {
  unsigned* bar;   // 2 words: grid barrier (zeroed by the launcher)
  void* xval;      // [2][Gmax] T
  int* xidx;       // [2][Gmax]
  void* xrow;      // [2][Gmax][ib] T
  void* xrowj;     // [2][ib] T
  int* perm;       // 1 + 4*wmax ints: count, dst positions, src positions
  int gmax;        // capacity in CTAs
  int ibmax;
  int wmax;
  int gtarget = 0; // preferred CTA count (0: the default for the element size)
};
// Most CTAs one cooperative panel launch may use: every CTA's candidate row
// of a column must fit the exchange buffer each CTA reads after the barrier.
constexpr int kPanelMaxCtas = 160;
// Bytes of PanelScratch for up to gmax CTAs, sub-panels of ibmax columns,
// panels up to wmax wide, elements of tsize bytes (each part 256-aligned).
constexpr size_t panel_scratch_bytes(int gmax, int ibmax, int wmax, int tsize) {
  return 64                                                  // barrier
         + (2 * (size_t)gmax * tsize + 256)                  // xval
         + (2 * (size_t)gmax * sizeof(int) + 256)            // xidx
         + (2 * (size_t)gmax * ibmax * tsize + 256)          // xrow
         + (2 * (size_t)ibmax * tsize + 256)                 // xrowj
         + ((1 + 4 * (size_t)wmax) * sizeof(int) + 256);     // perm
}
void panel_scratch_carve(PanelScratch* s, void* base, int gmax, int ibmax, int wmax, int tsize);

// CTAs that launch_panel uses for an m x w panel of element size tsize
// (gtarget > 0 replaces the default target count).
int panel_grid_size(int m, int w, int tsize, const DevInfo& dev, int gmax, int gtarget = 0);

// Factor the m x w panel whose (0,0) element is W(k,k) (row stride ldw) with
// partial pivoting.  Writes ipiv[k..k+w) (1-based, absolute), lowers *info to
// the first zero pivot (absolute, 1-based; the caller initialises it to
// INT_MAX), and the panel's net row permutation into scratch.perm.
// With spec_flag set (the diagonal-pivot check ran first, see SpecArgs) the
// launch returns at once when the check passed, and otherwise restores the
// rows the check changed from spec_backup (row-major, ld = w) before it
// factors the panel.
template <typename T>
cudaError_t launch_panel(T* Wkk, int64_t ldw, int m, int w, int kabs, int* ipiv, int* info, int* status,
                         const PanelScratch& s, const DevInfo& dev, cudaStream_t st, const int* spec_flag = nullptr,
                         const T* spec_backup = nullptr);

// The FP32 panel on one thread-block cluster (panel_cluster.cu): same
// arguments and outputs as launch_panel; used by launch_panel<float> when
// panel_cluster_available(m, w).  panel_cluster_size gives its CTA count.
int panel_cluster_size(int m, int w);
bool panel_cluster_available(int m, int w);
cudaError_t launch_panel_cluster(float* Wkk, int64_t ldw, int m, int w, int kabs, int* ipiv, int* info, int* status,
                                 int* perm, cudaStream_t st);
// SMs one panel launch occupies (for the lookahead's trailing-update cap).
int panel_sm_use(int m, int w, int tsize, const DevInfo& dev, const PanelScratch& s);

// Apply the panel permutation in scratch.perm (positions relative to row k) to
// columns [0, k) and [k + w, n) of W, and to the row-index vector rowid.
template <typename T>
cudaError_t launch_laswp(T* W, int64_t ldw, int n, int k, int w, const int* perm, int* rowid, cudaStream_t st);

// U12 <- L11^-1 A12: L11 = unit-lower w x w at W(k,k), A12 = w x N at W(k,k+w).
template <typename T>
cudaError_t launch_trsm_lower(const T* L11, T* A12, int64_t ldw, int w, int N, cudaStream_t st);

// ---------------------------------------------------------------- trsm_inv.cu
// The same top-block solve in FP32 for the mixed-precision factorizations, by
// the inverses of L11's 32 x 32 diagonal blocks (each CTA inverts them, then
// applies each block as a product and updates the rows below it), w <= 512.
// With kind 1 (BF16) or 2 (FP16) it also writes the trailing update's B
// operand of the solved columns, Bop[j * kpad + t] = U12(t, j) rounded (zero
// for w <= t < kpad), and raises ST_RANGE in *status for a non-finite result,
// as launch_cast_b does; kind 0 writes no operand.
cudaError_t launch_trsm_inv(const float* L11, float* A12, int64_t ldw, int w, int N, int kind, void* Bop, int kpad,
                            int* status, cudaStream_t st);

// W (row-major T) <- A (column-major FP64), n x n.
template <typename T>
cudaError_t launch_to_working(const double* A, int64_t lda, T* W, int64_t ldw, int n, cudaStream_t st);
// LU (column-major FP64) <- W (row-major T), n x n.
template <typename T>
cudaError_t launch_from_working(const T* W, int64_t ldw, double* LU, int64_t ldlu, int n, cudaStream_t st);

cudaError_t launch_iota(int* v, int n, cudaStream_t st, int base = 0);

// ---------------------------------------------------------------- nopiv.cu
// Diagonal-pivot check of a pivoted panel (FP32 panels).  Partial pivoting
// picks row j in column j when |a_jj| is the largest candidate; the block
// column kernels below first factor the m x w panel as if every pivot were on
// the diagonal and accept the result only if every multiplier satisfies
// |l_ij| <= 1/2 (the diagonal candidate at least twice any other, so the pivot
// search would have chosen it) and every pivot is finite and nonzero.
// Otherwise they record the failure, the panel kernel restores the rows they
// changed from `backup` and factors the panel with the full pivot search.
//   flag[0]: 0 while every checked stage passed, 1 after a failure (sticky);
//   flag[1]: kabs + 1 of a panel whose slab (see launch_block_column) failed,
//            flag[2]: the rows to restore then (the first slab's rows, or all);
//   flag[3]: kabs + 1 of a panel whose rows below a slab failed (all rows).
// A panel whose check fails leaves speculation off for the later panels of
// the factorization (their check kernels return at once).
struct SpecArgs {
  int* flag = nullptr;     // 4 ints, device (zeroed per factorization)
  void* backup = nullptr;  // m x w, row-major, ld = w: the panel's rows before the check
  int* ipiv = nullptr;     // absolute ipiv (identity written by the first slab)
  int* perm = nullptr;     // panel permutation record (count 0 written likewise)
};

// Factor the m x w block column at P (row-major, ld; m >= w) without
// pivoting -- the paper's "LU" (diagonal block) and "left" (A21 U11^-1)
// operations -- slab by slab: one CTA factors a slab of up to 128 rows in
// shared memory (its diagonal block and U rows), then a CTA per 64 rows below
// solves their L columns and updates the rest.  Zero pivots lower *info
// (absolute column + 1; kabs = P's first column).  With spec.flag set the
// kernels are the diagonal-pivot check of a pivoted panel instead (info
// unused).  block_column_launches gives the number of kernels it launches.
// uinv: scratch of w x 32 elements (the inverses of U's 32 x 32 diagonal
// blocks, passed from the slab kernel to the kernel of the rows below).
template <typename T>
cudaError_t launch_block_column(T* P, int64_t ld, int m, int w, int kabs, int* info, T* uinv, cudaStream_t st,
                                const SpecArgs& spec = SpecArgs());
int block_column_launches(int m, int w, int tsize);

// ---------------------------------------------------------------- gemm_simt.cu
// C (m x n) -= A (m x k) * B (k x n), all row-major in T, CUDA-core FMA.
template <typename T>
cudaError_t launch_gemm_simt(T* C, int64_t ldc, const T* A, int64_t lda, const T* B, int64_t ldb, int m, int n,
                             int k, cudaStream_t st);

// ---------------------------------------------------------------- gemm_tc.cu
// Operand casts for the tensor-core update (kind 1 = BF16, 2 = FP16):
//   Aop[i*kpad + t] = L21(i, t)     (K-major, m x k)
//   Bop[j*kpad + t] = U12(t, j)     (K-major, n x k)
// kpad >= k is a multiple of 64 with zero fill.  Overflow or NaN sets ST_RANGE.
cudaError_t launch_cast_operands(int kind, const float* L21, const float* U12, int64_t ldw, int m, int n, int k,
                                 void* Aop, void* Bop, int kpad, int* status, cudaStream_t st);
// The A half of launch_cast_operands alone (rows of L21 into Aop).
cudaError_t launch_cast_a(int kind, const float* L21, int64_t ldw, int m, int k, void* Aop, int kpad, int* status,
                          cudaStream_t st);
// C (row-major FP32, m x n) -= Aop * Bop^T on tcgen05 (FP32 accumulate in TMEM).
// max_ctas > 0 caps the persistent grid (to leave SMs to a concurrent kernel).
cudaError_t tc_gemm_run(int kind, float* C, int64_t ldc, const void* Aop, const void* Bop, int m, int n, int kpad,
                        int* status, const DevInfo& dev, cudaStream_t st, int max_ctas = 0);

// ---------------------------------------------------------------- gemm_ozaki.cu
// FP64 C -= A B with the products on BF16 tensor cores by error-free splitting
// (Ozaki scheme, 8 slices of 7 bits, exact integer combination).  k <= 256.
// ozaki_split cuts A (m x k) and B (k x n), both row-major FP64, into the
// workspace (ozaki_ws_bytes(m, n, k, sm_count) bytes, sm_count of the device
// that runs it); ozaki_gemm then updates columns
// [col0, col0 + ncols) of the m x n product into C (row-major FP64, column 0
// of C is column col0 of the product).  Non-finite operands set ST_RANGE.
size_t ozaki_ws_bytes(int m, int n, int k, int sm_count);
cudaError_t ozaki_split(const double* A, int64_t lda, const double* B, int64_t ldb, int m, int n, int k, void* ws,
                        int* status, cudaStream_t st);
cudaError_t ozaki_gemm(double* C, int64_t ldc, const void* ws, int m, int n, int k, int col0, int ncols, int* status,
                       const DevInfo& dev, cudaStream_t st, int max_ctas = 0);
// M (w x w, row-major) = I - L^-1 for the unit-lower block L (w <= 256), so that
// the top block solve L^-1 A12 is the split update A12 - M A12.
cudaError_t launch_unit_lower_inv_comp(const double* L, int64_t ldl, int w, double* M, int64_t ldm, cudaStream_t st);

// ---------------------------------------------------------------- solve.cu
struct SolveScratch {
  int* sync;       // flags [nblk] + ticket (zeroed per launch by the launcher)
  void* y;         // n x NR (T) workspace
  void* z;         // n x NR (T) workspace
  int nblk_max;
  void* dinv = nullptr;     // optional inverses of the 64 x 64 diagonal blocks
  bool dinv_ready = false;
  int max_ctas = 0;         // CTAs per triangle launch (0: one per 64-row block)
};
size_t solve_dinv_bytes(int n, int tsize);
template <typename T>
cudaError_t launch_trinv(const T* W, int64_t ldw, int n, T* Dinv, cudaStream_t st);
size_t solve_scratch_bytes(int n, int tsize);
void solve_scratch_carve(SolveScratch* s, void* base, int n, int tsize);

// X = U^-1 L^-1 P B for one chunk of <= 32 right-hand sides.  B, X: FP64
// column-major (may alias).  Computed in T.
template <typename T>
cudaError_t launch_lu_solve(const T* W, int64_t ldw, const int* rowid, int n, int nrhs, const double* B,
                            int64_t ldb, double* X, int64_t ldx, const SolveScratch& s, int* status, cudaStream_t st);

// R = B - A X (FP64), with per-column max |r|, max |x|, max |b| into norms
// (3*nrhs doubles, zeroed by the launcher).  partial: workspace of
// residual_partial_bytes(n, nrhs).
size_t residual_partial_bytes(int n, int nrhs);
cudaError_t launch_residual(const double* A, int64_t lda, const double* X, int64_t ldx, const double* B,
                            int64_t ldb, double* R, int64_t ldr, int n, int nrhs, double* partial, double* norms,
                            cudaStream_t st);
// anorm[0] = ||A||_inf (max row sum of |A|).
// Per-column max |r|, |x|, |b| (norms layout as launch_residual) of an R
// formed by another kernel.
cudaError_t launch_colmax3(const double* R, int64_t ldr, const double* X, int64_t ldx, const double* B, int64_t ldb,
                           int n, int nrhs, double* norms, cudaStream_t st);
cudaError_t launch_norm_inf(const double* A, int64_t lda, int n, double* partial, double* anorm, cudaStream_t st);
// X[:, q] += D[:, q] for columns q with active[q] != 0.
cudaError_t launch_add_update(double* X, int64_t ldx, const double* D, int64_t ldd, int n, int nrhs,
                              const int* active, cudaStream_t st);

// Bounded-wait probe (waitprobe.cu): kind 0 flag wait, 1 grid barrier, 2
// mbarrier wait, each on a condition nothing satisfies; 8 bytes of scratch.
cudaError_t launch_wait_probe(int kind, void* scratch, int* status, cudaStream_t st);

}  // namespace gb
