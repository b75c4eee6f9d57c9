// Forward/back substitution, FP64 residual and the refinement update.
//
// The solve answers the second step of the HPL problem statement (arxiv
// 2202.13995, section "High Performance Linpack", first paragraph): with
// P A = L U, solve L y = P b, then U x = y.  The paper runs this step on the
// CPU; here it is one kernel per triangle.
//
// Triangular solve design (one launch per triangle): the rows are cut in
// blocks of 64.  Each CTA takes a block in dependency order from an atomic
// ticket (so a CTA only ever waits on blocks taken by CTAs already running),
// accumulates the products of its block row with every finished solution
// block as soon as that block's flag is published, then solves its own
// 64 x 64 diagonal block and publishes its solution block.  Every matrix entry
// is read once, and the only serial chain is the diagonal solves.
#include "common.cuh"
#include "kernels.h"

namespace gb {

constexpr int TS_BS = 64;

template <typename T, int NR>
struct TrsvSmem {
  T Ls[TS_BS][TS_BS + 1];
  T ys[TS_BS][NR];
  T red[3][NR][TS_BS];
  int flag;
  int blk;
};

// LOWER: Y = L^-1 (P B) with unit-lower L; the right-hand side is gathered
//        from B through rowid (P b)[i] = b[rowid[i]].
// UPPER: X = U^-1 Y with non-unit upper U; the result goes to Yout (T) for
//        the later blocks and to X (FP64).
template <typename T, int NR, bool LOWER>
__global__ void __launch_bounds__(256) trsv_kernel(const T* __restrict__ W, int64_t ldw, int n, int nrhs,
                                                   const double* __restrict__ B, int64_t ldb,
                                                   const int* __restrict__ rowid, const T* __restrict__ Yin,
                                                   T* Yout, double* X, int64_t ldx, int* flags, int* ticket,
                                                   int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrsvSmem<T, NR>& sm = *reinterpret_cast<TrsvSmem<T, NR>*>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = tid & 63, g = tid >> 6;
  const int nblk = (n + TS_BS - 1) / TS_BS;
  if (tid == 0) sm.blk = atomicAdd(ticket, 1);
  __syncthreads();
  const int t_ = sm.blk;
  const int ib = LOWER ? t_ : nblk - 1 - t_;
  const int i0 = ib * TS_BS;
  const int rows = min(TS_BS, n - i0);

  T acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = T(0);

  const int jfirst = LOWER ? 0 : nblk - 1;
  const int jstep = LOWER ? 1 : -1;
  const int count = LOWER ? ib : nblk - 1 - ib;
  for (int it = 0; it < count; ++it) {
    const int jb = jfirst + it * jstep;
    const int j0 = jb * TS_BS;
    const int cols = min(TS_BS, n - j0);
    // matrix block first: it does not depend on the flag
    for (int e = tid; e < TS_BS * TS_BS; e += 256) {
      const int rr = e >> 6, cc = e & 63;
      sm.Ls[rr][cc] = (rr < rows && cc < cols) ? W[(int64_t)(i0 + rr) * ldw + j0 + cc] : T(0);
    }
    if (tid == 0) sm.flag = wait_flag_eq(flags + jb, 1, status) ? 1 : 0;
    __syncthreads();
    if (!sm.flag) return;
    for (int e = tid; e < TS_BS * NR; e += 256) {
      const int c = e & 63, q = e >> 6;
      sm.ys[c][q] = (q < nrhs && c < cols) ? __ldcg(Yout + (int64_t)q * n + j0 + c) : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int cc = 0; cc < 16; ++cc) {
      const int c = g * 16 + cc;
      const T l = sm.Ls[r][c];
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] = fma(l, sm.ys[c][q], acc[q]);
    }
    __syncthreads();
  }
  // reduce the four column groups in a fixed order
  if (g > 0) {
#pragma unroll
    for (int q = 0; q < NR; ++q) sm.red[g - 1][q][r] = acc[q];
  }
  // diagonal block
  for (int e = tid; e < TS_BS * TS_BS; e += 256) {
    const int rr = e >> 6, cc = e & 63;
    sm.Ls[rr][cc] = (rr < rows && cc < rows) ? W[(int64_t)(i0 + rr) * ldw + i0 + cc] : T(0);
  }
  __syncthreads();
  if (g == 0) {
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const T tot = acc[q] + sm.red[0][q][r] + sm.red[1][q][r] + sm.red[2][q][r];
      T v = T(0);
      if (r < rows && q < nrhs) {
        if (LOWER)
          v = (T)B[(int64_t)q * ldb + rowid[i0 + r]] - tot;
        else
          v = Yin[(int64_t)q * n + i0 + r] - tot;
      }
      sm.ys[r][q] = v;
    }
  }
  __syncthreads();
  for (int q = warp; q < nrhs; q += 8) {
    T x0 = sm.ys[lane][q], x1 = sm.ys[lane + 32][q];
    if (LOWER) {
      for (int t = 0; t < rows; ++t) {
        const T xt = __shfl_sync(0xffffffffu, t < 32 ? x0 : x1, t & 31);
        if (lane > t) x0 -= sm.Ls[lane][t] * xt;
        if (lane + 32 > t) x1 -= sm.Ls[lane + 32][t] * xt;
      }
    } else {
      for (int t = rows - 1; t >= 0; --t) {
        T xt;
        if (t >= 32) {
          if (lane == t - 32) x1 = x1 / sm.Ls[t][t];
          xt = __shfl_sync(0xffffffffu, x1, t - 32);
        } else {
          if (lane == t) x0 = x0 / sm.Ls[t][t];
          xt = __shfl_sync(0xffffffffu, x0, t);
        }
        if (lane < t) x0 -= sm.Ls[lane][t] * xt;
        if (lane + 32 < t) x1 -= sm.Ls[lane + 32][t] * xt;
      }
    }
    sm.ys[lane][q] = x0;
    sm.ys[lane + 32][q] = x1;
  }
  __syncthreads();
  for (int e = tid; e < TS_BS * NR; e += 256) {
    const int rr = e & 63, q = e >> 6;
    if (rr < rows && q < nrhs) {
      const T v = sm.ys[rr][q];
      Yout[(int64_t)q * n + i0 + rr] = v;
      if (!LOWER) X[(int64_t)q * ldx + i0 + rr] = (double)v;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release_s32(flags + ib, 1);
}

size_t solve_scratch_bytes(int n, int tsize) {
  const int nblk = (int)cdiv(n, TS_BS);
  return 256 + (size_t)(nblk + 2) * sizeof(int) + 2 * (size_t)n * 32 * tsize + 512;
}

void solve_scratch_carve(SolveScratch* s, void* base, int n, int tsize) {
  const int nblk = (int)cdiv(n, TS_BS);
  char* p = (char*)base;
  s->sync = (int*)p;
  p += ((size_t)(nblk + 2) * sizeof(int) + 255) / 256 * 256;
  s->y = p;
  p += ((size_t)n * 32 * tsize + 255) / 256 * 256;
  s->z = p;
  s->nblk_max = nblk;
}

template <typename T, int NR>
static cudaError_t run_solve(const T* W, int64_t ldw, const int* rowid, int n, int nrhs, const double* B,
                             int64_t ldb, double* X, int64_t ldx, const SolveScratch& s, int* status,
                             cudaStream_t st) {
  const int nblk = (int)cdiv(n, TS_BS);
  const size_t smem = sizeof(TrsvSmem<T, NR>);
  auto kl = trsv_kernel<T, NR, true>;
  auto ku = trsv_kernel<T, NR, false>;
  cudaError_t e = cudaFuncSetAttribute(kl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(ku, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int* flags = s.sync;
  int* ticket = s.sync + nblk;
  T* y = (T*)s.y;
  T* z = (T*)s.z;
  e = cudaMemsetAsync(s.sync, 0, (size_t)(nblk + 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  kl<<<nblk, 256, smem, st>>>(W, ldw, n, nrhs, B, ldb, rowid, nullptr, y, nullptr, 0, flags, ticket, status);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.sync, 0, (size_t)(nblk + 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  ku<<<nblk, 256, smem, st>>>(W, ldw, n, nrhs, nullptr, 0, nullptr, y, z, X, ldx, flags, ticket, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lu_solve(const T* W, int64_t ldw, const int* rowid, int n, int nrhs, const double* B,
                            int64_t ldb, double* X, int64_t ldx, const SolveScratch& s, int* status,
                            cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs > 32) return cudaErrorInvalidValue;
  if (nrhs == 1) return run_solve<T, 1>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  if (nrhs <= 4) return run_solve<T, 4>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  if (nrhs <= 8) return run_solve<T, 8>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  if (nrhs <= 16) return run_solve<T, 16>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  return run_solve<T, 32>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
}

template cudaError_t launch_lu_solve<double>(const double*, int64_t, const int*, int, int, const double*, int64_t,
                                             double*, int64_t, const SolveScratch&, int*, cudaStream_t);
template cudaError_t launch_lu_solve<float>(const float*, int64_t, const int*, int, int, const double*, int64_t,
                                            double*, int64_t, const SolveScratch&, int*, cudaStream_t);

// ============================================================ residual r = b - A x (FP64)
// Partial products over column slabs, then a fixed-order sum: deterministic.
constexpr int RS_ROWS = 256;
constexpr int RS_CHUNK = 64;

static int residual_splits(int n) {
  const int rt = (int)cdiv(n, RS_ROWS);
  int ks = (int)cdiv(608, rt);  // about four CTAs per SM in all
  const int kmax = (int)cdiv(n, RS_CHUNK);
  if (ks > kmax) ks = kmax;
  if (ks < 1) ks = 1;
  return ks;
}

size_t residual_partial_bytes(int n, int nrhs) { return (size_t)residual_splits(n) * n * (nrhs > 0 ? nrhs : 1) * 8; }

template <int NR, bool ABS>
__global__ void __launch_bounds__(RS_ROWS) residual_partial_kernel(const double* __restrict__ A, int64_t lda,
                                                                   const double* __restrict__ X, int64_t ldx, int n,
                                                                   int nrhs, int kc, double* __restrict__ partial) {
  __shared__ double xs[RS_CHUNK][NR];
  const int i = blockIdx.x * RS_ROWS + threadIdx.x;
  const int ks = blockIdx.y;
  const int c_begin = ks * kc, c_end = min(n, c_begin + kc);
  double acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = 0.0;
  for (int c0 = c_begin; c0 < c_end; c0 += RS_CHUNK) {
    const int cw = min(RS_CHUNK, c_end - c0);
    for (int e = threadIdx.x; e < RS_CHUNK * NR; e += RS_ROWS) {
      const int c = e % RS_CHUNK, q = e / RS_CHUNK;
      xs[c][q] = (c < cw && q < nrhs) ? (ABS ? 1.0 : X[(int64_t)q * ldx + c0 + c]) : 0.0;
    }
    __syncthreads();
    if (i < n) {
      for (int c = 0; c < cw; ++c) {
        double a = A[(int64_t)(c0 + c) * lda + i];
        if (ABS) a = fabs(a);
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = fma(a, xs[c][q], acc[q]);
      }
    }
    __syncthreads();
  }
  if (i < n) {
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (q < nrhs) partial[((int64_t)ks * nrhs + q) * n + i] = acc[q];
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// norms layout: [0, nrhs) max|r|, [nrhs, 2 nrhs) max|x|, [2 nrhs, 3 nrhs) max|b|
__global__ void residual_finish_kernel(const double* __restrict__ partial, int ks, const double* __restrict__ X,
                                       int64_t ldx, const double* __restrict__ B, int64_t ldb, double* R,
                                       int64_t ldr, int n, int nrhs, double* norms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  double rv = 0.0, xv = 0.0, bv = 0.0;
  if (i < n) {
    double s = 0.0;
    for (int k = 0; k < ks; ++k) s += partial[((int64_t)k * nrhs + q) * n + i];
    const double b = B[(int64_t)q * ldb + i];
    const double r = b - s;
    if (R) R[(int64_t)q * ldr + i] = r;
    rv = fabs(r);
    xv = fabs(X[(int64_t)q * ldx + i]);
    bv = fabs(b);
  }
  rv = warp_max(rv);
  xv = warp_max(xv);
  bv = warp_max(bv);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(norms + q, rv);
    atomic_max_nonneg(norms + nrhs + q, xv);
    atomic_max_nonneg(norms + 2 * nrhs + q, bv);
  }
}

__global__ void rowsum_finish_kernel(const double* __restrict__ partial, int ks, int n, double* anorm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n)
    for (int k = 0; k < ks; ++k) s += partial[(int64_t)k * n + i];
  s = warp_max(s);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(anorm, s);
}

template <int NR, bool ABS>
static cudaError_t run_partial(const double* A, int64_t lda, const double* X, int64_t ldx, int n, int nrhs, int ks,
                               double* partial, cudaStream_t st) {
  const int kc = (int)cdiv(cdiv(n, ks), RS_CHUNK) * RS_CHUNK;
  dim3 grid((unsigned)cdiv(n, RS_ROWS), (unsigned)ks);
  residual_partial_kernel<NR, ABS><<<grid, RS_ROWS, 0, st>>>(A, lda, X, ldx, n, nrhs, kc, partial);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* A, int64_t lda, const double* X, int64_t ldx, const double* B,
                            int64_t ldb, double* R, int64_t ldr, int n, int nrhs, double* partial, double* norms,
                            cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs > 32) return cudaErrorInvalidValue;
  const int ks = residual_splits(n);
  cudaError_t e;
  if (nrhs == 1)
    e = run_partial<1, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else if (nrhs <= 4)
    e = run_partial<4, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else if (nrhs <= 8)
    e = run_partial<8, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else if (nrhs <= 16)
    e = run_partial<16, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else
    e = run_partial<32, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(norms, 0, (size_t)3 * nrhs * sizeof(double), st);
  if (e != cudaSuccess) return e;
  residual_finish_kernel<<<dim3((unsigned)cdiv(n, 256), (unsigned)nrhs), 256, 0, st>>>(partial, ks, X, ldx, B, ldb,
                                                                                      R, ldr, n, nrhs, norms);
  return cudaGetLastError();
}

cudaError_t launch_norm_inf(const double* A, int64_t lda, int n, double* partial, double* anorm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int ks = residual_splits(n);
  cudaError_t e = run_partial<1, true>(A, lda, nullptr, 0, n, 1, ks, partial, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(anorm, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  rowsum_finish_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(partial, ks, n, anorm);
  return cudaGetLastError();
}

__global__ void add_update_kernel(double* X, int64_t ldx, const double* D, int64_t ldd, int n, const int* active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (i < n && active[q]) X[(int64_t)q * ldx + i] += D[(int64_t)q * ldd + i];
}

cudaError_t launch_add_update(double* X, int64_t ldx, const double* D, int64_t ldd, int n, int nrhs,
                              const int* active, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  add_update_kernel<<<dim3((unsigned)cdiv(n, 256), (unsigned)nrhs), 256, 0, st>>>(X, ldx, D, ldd, n, active);
  return cudaGetLastError();
}

}  // namespace gb
