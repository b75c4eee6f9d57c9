// Batched dense solves: one persistent kernel, one CTA per system at a time.
//
// Each system is the HPL problem (arxiv 2202.13995, section "High Performance
// Linpack") factored by the paper's blocked right-looking iteration (section
// "Base Implementation"), here inside one CTA with block width 32 and partial
// pivoting, in FP32, followed by FP64 iterative refinement.
//
// Partial pivoting without moving rows: the CTA keeps the logical-to-physical
// row map `perm` in shared memory.  A pivot swaps two entries of perm (and two
// rows of the shared-memory panel); every other access goes through perm, so
// the row interchanges of the other columns cost nothing.  L and U stay in the
// working copy in physical row order, and P b is a gather through perm.
//
// The systems are taken from an atomic queue in decreasing n (largest first
// for balance).  The arithmetic of a system depends on its n only, never on
// the CTA, the launch shape or the rest of the batch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "lu_batched.h"

namespace gb {

constexpr int BT_NMAX = 512;
constexpr int BT_NB = 32;
constexpr int BT_CW = 256;    // column chunk of the trailing update
constexpr int BT_RHSMAX = 8;

struct BatchDesc {
  const double* A;
  const double* B;
  double* X;
  int n, nrhs, lda, ldb, ldx, pad;
};

struct BatchSmem {
  // factor phase
  float P[BT_NB][BT_NMAX];  // panel, column-major: P[c][r]
  float Us[BT_NB][BT_CW];   // U12 chunk
  int perm[BT_NMAX];
  float Ld[BT_NB][BT_NB + 1];
  float redf[32];
  int redi[32];
  double redd[3 * BT_RHSMAX * 32];  // >= 16 warps x 32 + 32
  int misc[8];
};
// refinement phase views (alias P/Us): x (FP64), r (FP64), y (FP32), 8 x 512 each
static_assert(sizeof(float) * BT_NB * (BT_NMAX + BT_CW) >=
                  2 * sizeof(double) * BT_RHSMAX * BT_NMAX + sizeof(float) * BT_RHSMAX * BT_NMAX,
              "refinement vectors must fit in the factor-phase buffers");
static_assert(3 * BT_RHSMAX * 32 >= 16 * 32 + 32, "block_max_many needs 16 warps x 32 + 32 slots");

__device__ __forceinline__ void block_argmax_f(float& v, int& i, BatchSmem& sm, int nt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  warp_argmax(v, i);
  if (lane == 0) {
    sm.redf[warp] = v;
    sm.redi[warp] = i;
  }
  __syncthreads();
  v = lane < nt / 32 ? sm.redf[lane] : -1.0f;
  i = lane < nt / 32 ? sm.redi[lane] : INT_MAX;
  warp_argmax(v, i);  // every warp computes the same result
}

// FP32 LU with partial pivoting of the n x n row-major W (ld), rows through perm.
// Returns the first zero pivot (1-based) or 0.
template <int NT>
__device__ int bt_factor(float* W, int ld, int n, BatchSmem& sm, int* status) {
  const int tid = threadIdx.x;
  int info = 0;
  for (int i = tid; i < n; i += NT) sm.perm[i] = i;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += BT_NB) {
    const int kb = min(BT_NB, n - k0);
    const int m = n - k0;
    // thread = row, four columns per load (rows and k0 are 16-byte aligned):
    // the column-major panel is then written without bank conflicts
    for (int e = tid; e < m * (BT_NB / 4); e += NT) {
      const int r = e % m, c = (e / m) * 4;
      if (c >= kb) continue;
      const float* src = W + (int64_t)sm.perm[k0 + r] * ld + k0 + c;
      if (c + 4 <= kb) {
        const float4 v = *reinterpret_cast<const float4*>(src);
        sm.P[c][r] = v.x;
        sm.P[c + 1][r] = v.y;
        sm.P[c + 2][r] = v.z;
        sm.P[c + 3][r] = v.w;
      } else {
        for (int x = 0; c + x < kb; ++x) sm.P[c + x][r] = src[x];
      }
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
      float bv = -1.0f;
      int bi = INT_MAX;
      for (int r = j + tid; r < m; r += NT) {
        const float v = fabsf(sm.P[j][r]);
        if (v != v) atomicOr(status, ST_RANGE);
        argmax_merge(bv, bi, v, r);
      }
      block_argmax_f(bv, bi, sm, NT);
      int p = bi;
      if (!GB_IN_BOUNDS(status, p >= j && p < m)) p = j;
      if (tid < kb && p != j) {
        const float t = sm.P[tid][j];
        sm.P[tid][j] = sm.P[tid][p];
        sm.P[tid][p] = t;
      }
      if (tid == 0 && p != j) {
        const int t = sm.perm[k0 + j];
        sm.perm[k0 + j] = sm.perm[k0 + p];
        sm.perm[k0 + p] = t;
      }
      __syncthreads();
      const float piv = sm.P[j][j];
      if (piv == 0.0f && info == 0) info = k0 + j + 1;
      for (int r = j + 1 + tid; r < m; r += NT) {
        float l = sm.P[j][r];
        if (piv != 0.0f) l = l / piv;
        sm.P[j][r] = l;
        for (int c = j + 1; c < kb; ++c) sm.P[c][r] -= l * sm.P[c][j];
      }
      __syncthreads();
    }
    for (int e = tid; e < m * (BT_NB / 4); e += NT) {
      const int r = e % m, c = (e / m) * 4;
      if (c >= kb) continue;
      float* dst = W + (int64_t)sm.perm[k0 + r] * ld + k0 + c;
      if (c + 4 <= kb) {
        *reinterpret_cast<float4*>(dst) = make_float4(sm.P[c][r], sm.P[c + 1][r], sm.P[c + 2][r], sm.P[c + 3][r]);
      } else {
        for (int x = 0; c + x < kb; ++x) dst[x] = sm.P[c + x][r];
      }
    }
    __syncthreads();
    // U12 (top blocks) and the inner update, in column chunks
    for (int c0 = k0 + kb; c0 < n; c0 += BT_CW) {
      const int cw = min(BT_CW, n - c0);
      for (int c = tid; c < cw; c += NT) {
        // the column's kb entries are loaded together, then solved in registers
        float v[BT_NB];
#pragma unroll
        for (int j = 0; j < BT_NB; ++j) v[j] = j < kb ? W[(int64_t)sm.perm[k0 + j] * ld + c0 + c] : 0.0f;
#pragma unroll
        for (int j = 1; j < BT_NB; ++j)
#pragma unroll
          for (int i = 0; i < j; ++i) v[j] -= sm.P[i][j] * v[i];
#pragma unroll
        for (int j = 0; j < BT_NB; ++j) {
          if (j < kb) {
            sm.Us[j][c] = v[j];
            W[(int64_t)sm.perm[k0 + j] * ld + c0 + c] = v[j];
          }
        }
      }
      __syncthreads();
      // rows kb .. m of the panel (logical k0 + kb ..), columns c0 .. c0 + cw:
      // 4 x 4 register tiles, products accumulated in order of k
      const int rows = m - kb;
      const int rt = (rows + 3) / 4, ct = (cw + 3) / 4;
      for (int t = tid; t < rt * ct; t += NT) {
        const int r0 = kb + (t / ct) * 4, cc = (t % ct) * 4;
        // the tile's entries of W first: their latency runs under the products
        float cw4[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float* wr = W + (int64_t)sm.perm[k0 + min(r0 + i, m - 1)] * ld + c0 + cc;
#pragma unroll
          for (int q = 0; q < 4; ++q) cw4[i][q] = (r0 + i < m && cc + q < cw) ? wr[q] : 0.0f;
        }
        float acc[4][4] = {};
        // kb = 32 here (the last block has no rows below it), so r0 and cc
        // are multiples of 4: one 16-byte shared load per operand and k.
        // Lanes past m or cw read stale entries into rows / columns of acc
        // that are never stored.
        for (int k = 0; k < kb; ++k) {
          const float4 a4 = *reinterpret_cast<const float4*>(&sm.P[k][r0]);
          const float4 b4 = *reinterpret_cast<const float4*>(&sm.Us[k][cc]);
          const float a[4] = {a4.x, a4.y, a4.z, a4.w};
          const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = fmaf(a[i], b[q], acc[i][q]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (r0 + i >= m) break;
          float* wr = W + (int64_t)sm.perm[k0 + r0 + i] * ld + c0 + cc;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (cc + q < cw) wr[q] = cw4[i][q] - acc[i][q];
        }
      }
      __syncthreads();
    }
  }
  return info;
}

// y <- U^-1 L^-1 (P rhs) in FP32 for nr right-hand sides held in y[q][0..n)
// (already gathered through perm).  Blocked by 32: one warp per right-hand side
// solves a diagonal block, then all threads update the rows beyond it.
template <int NT>
__device__ void bt_solve(const float* W, int ld, int n, int nr, float* y, BatchSmem& sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // forward, unit lower
  for (int b0 = 0; b0 < n; b0 += BT_NB) {
    const int bw = min(BT_NB, n - b0);
    for (int e = tid; e < BT_NB * BT_NB; e += NT) {
      const int r = e / BT_NB, c = e % BT_NB;
      sm.Ld[r][c] = (r < bw && c < bw) ? W[(int64_t)sm.perm[b0 + r] * ld + b0 + c] : 0.0f;
    }
    __syncthreads();
    for (int q = warp; q < nr; q += NT / 32) {
      float x = lane < bw ? y[q * BT_NMAX + b0 + lane] : 0.0f;
      for (int t = 0; t < bw; ++t) {
        const float xt = __shfl_sync(0xffffffffu, x, t);
        if (lane > t) x -= sm.Ld[lane][t] * xt;
      }
      if (lane < bw) y[q * BT_NMAX + b0 + lane] = x;
    }
    __syncthreads();
    for (int r = b0 + bw + tid; r < n; r += NT) {
      const float* wr = W + (int64_t)sm.perm[r] * ld + b0;
      float l[BT_NB];
#pragma unroll
      for (int t = 0; t < BT_NB; ++t) l[t] = t < bw ? wr[t] : 0.0f;
      for (int q = 0; q < nr; ++q) {
        float v = y[q * BT_NMAX + r];
#pragma unroll
        for (int t = 0; t < BT_NB; ++t)
          if (t < bw) v -= l[t] * y[q * BT_NMAX + b0 + t];
        y[q * BT_NMAX + r] = v;
      }
    }
    __syncthreads();
  }
  // backward, upper
  const int nblk = (n + BT_NB - 1) / BT_NB;
  for (int bi = nblk - 1; bi >= 0; --bi) {
    const int b0 = bi * BT_NB;
    const int bw = min(BT_NB, n - b0);
    for (int e = tid; e < BT_NB * BT_NB; e += NT) {
      const int r = e / BT_NB, c = e % BT_NB;
      sm.Ld[r][c] = (r < bw && c < bw) ? W[(int64_t)sm.perm[b0 + r] * ld + b0 + c] : 0.0f;
    }
    __syncthreads();
    for (int q = warp; q < nr; q += NT / 32) {
      float x = lane < bw ? y[q * BT_NMAX + b0 + lane] : 0.0f;
      for (int t = bw - 1; t >= 0; --t) {
        if (lane == t) x = x / sm.Ld[t][t];
        const float xt = __shfl_sync(0xffffffffu, x, t);
        if (lane < t) x -= sm.Ld[lane][t] * xt;
      }
      if (lane < bw) y[q * BT_NMAX + b0 + lane] = x;
    }
    __syncthreads();
    for (int r = tid; r < b0; r += NT) {
      const float* wr = W + (int64_t)sm.perm[r] * ld + b0;
      float u[BT_NB];
#pragma unroll
      for (int t = 0; t < BT_NB; ++t) u[t] = t < bw ? wr[t] : 0.0f;
      for (int q = 0; q < nr; ++q) {
        float v = y[q * BT_NMAX + r];
#pragma unroll
        for (int t = 0; t < BT_NB; ++t)
          if (t < bw) v -= u[t] * y[q * BT_NMAX + b0 + t];
        y[q * BT_NMAX + r] = v;
      }
    }
    __syncthreads();
  }
}

// r = b - A x in FP64 for the rows of this thread (A FP64 column-major), with
// the column maxima of |r|, |x|, |b| and, on the first pass, the row sums of |A|.
template <int NR, bool FIRST>
__device__ __forceinline__ void bt_resid_rows(const BatchDesc& d, int n, const double* xs, double* rs, double& amax,
                                              double* rmax, double* xmax, double* bmax, int tid, int nt) {
  for (int i = tid; i < n; i += nt) {
    double acc[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      acc[q] = d.B[(int64_t)q * d.ldb + i];
      bmax[q] = fmax(bmax[q], fabs(acc[q]));
    }
    double asum = 0.0;
    for (int j = 0; j < n; ++j) {
      const double a = d.A[(int64_t)j * d.lda + i];
      if (FIRST) asum += fabs(a);
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[q] = fma(-a, xs[q * BT_NMAX + j], acc[q]);
    }
    amax = fmax(amax, asum);
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      rs[q * BT_NMAX + i] = acc[q];
      rmax[q] = fmax(rmax[q], fabs(acc[q]));
      xmax[q] = fmax(xmax[q], fabs(xs[q * BT_NMAX + i]));
    }
  }
}

// Block-wide maxima of 3 nr (+1) per-thread values in one shared-memory round:
// returns a shared array (valid until the next call) with rmax[0..nr),
// xmax[0..nr), bmax[0..nr) and, if with_a, amax.  Maxima do not depend on the
// order of reduction.
__device__ __forceinline__ const double* block_max_many(const double* rmax, const double* xmax, const double* bmax,
                                                        double amax, int nr, bool with_a, double* red, int nt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int K = 3 * nr + (with_a ? 1 : 0);  // <= 25
  __syncthreads();  // the previous results have been read
  for (int k = 0; k < K; ++k) {
    double v = k < nr ? rmax[k] : k < 2 * nr ? xmax[k - nr] : k < 3 * nr ? bmax[k - 2 * nr] : amax;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if (lane == 0) red[warp * 32 + k] = v;
  }
  __syncthreads();
  if ((int)threadIdx.x < K) {
    double m = 0.0;
    for (int w = 0; w < nt / 32; ++w) m = fmax(m, red[w * 32 + threadIdx.x]);
    red[16 * 32 + threadIdx.x] = m;
  }
  __syncthreads();
  return red + 16 * 32;
}

template <int NT>
__global__ void __launch_bounds__(NT) batched_kernel(const BatchDesc* __restrict__ desc, const int* __restrict__ order,
                                                     int count, int* next, float* scratch, int64_t slot_floats,
                                                     int* info_out, int* iters_out, double* resid_out, double tol,
                                                     int max_iter, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BatchSmem& sm = *reinterpret_cast<BatchSmem*>(smem_raw);
  double* xs = reinterpret_cast<double*>(&sm.P[0][0]);  // [8][512] FP64
  double* rs = xs + BT_RHSMAX * BT_NMAX;                // [8][512] FP64
  float* ys = reinterpret_cast<float*>(rs + BT_RHSMAX * BT_NMAX);  // [8][512] FP32
  const int tid = threadIdx.x;
  float* W = scratch + (int64_t)blockIdx.x * slot_floats;
  const double eps = 1.1102230246251565e-16;  // 2^-53

  while (true) {
    if (tid == 0) sm.misc[0] = atomicAdd(next, 1);
    __syncthreads();
    const int s = sm.misc[0];
    __syncthreads();
    if (s >= count) break;
    const int sys = order[s];
    const BatchDesc d = desc[sys];
    const int n = d.n, nr = d.nrhs;
    const int ld = (n + 3) & ~3;
    // W <- A (FP64 column-major -> FP32 row-major), through 32 x 32 tiles
    for (int i0 = 0; i0 < n; i0 += BT_NB) {
      for (int j0 = 0; j0 < n; j0 += BT_NB) {
        for (int e = tid; e < BT_NB * BT_NB; e += NT) {
          const int i = e % BT_NB, j = e / BT_NB;
          sm.Ld[j][i] = (i0 + i < n && j0 + j < n) ? (float)d.A[(int64_t)(j0 + j) * d.lda + i0 + i] : 0.0f;
        }
        __syncthreads();
        for (int e = tid; e < BT_NB * BT_NB; e += NT) {
          const int j = e % BT_NB, i = e / BT_NB;
          if (i0 + i < n && j0 + j < n) W[(int64_t)(i0 + i) * ld + j0 + j] = sm.Ld[j][i];
        }
        __syncthreads();
      }
    }
    const int info = bt_factor<NT>(W, ld, n, sm, status);
    if (info != 0) {
      if (tid == 0) {
        info_out[sys] = info;
        if (iters_out) iters_out[sys] = 0;
        if (resid_out) resid_out[sys] = INFINITY;
      }
      __syncthreads();
      continue;
    }
    // x0 = solve(b)
    for (int e = tid; e < nr * n; e += NT) {
      const int q = e / n, r = e % n;
      ys[q * BT_NMAX + r] = (float)d.B[(int64_t)q * d.ldb + sm.perm[r]];
    }
    __syncthreads();
    bt_solve<NT>(W, ld, n, nr, ys, sm);
    for (int e = tid; e < nr * n; e += NT) {
      const int q = e / n, r = e % n;
      xs[q * BT_NMAX + r] = (double)ys[q * BT_NMAX + r];
    }
    __syncthreads();
    double anorm = 0.0;
    int it = 0, result = -1;
    double worst = 0.0;
    unsigned active = (1u << nr) - 1u;
    while (true) {
      // r = b - A x (FP64), row sums of |A| on the first pass, column maxima
      double rmax[BT_RHSMAX], xmax[BT_RHSMAX], bmax[BT_RHSMAX];
#pragma unroll
      for (int q = 0; q < BT_RHSMAX; ++q) rmax[q] = xmax[q] = bmax[q] = 0.0;
      double amax = 0.0;
      // one instantiation per right-hand-side count, so that no FP64
      // operation is issued for absent columns
#define GB_RESID_CASE(NRC)                                                              \
  case NRC:                                                                             \
    if (it == 0)                                                                        \
      bt_resid_rows<NRC, true>(d, n, xs, rs, amax, rmax, xmax, bmax, tid, NT);          \
    else                                                                                \
      bt_resid_rows<NRC, false>(d, n, xs, rs, amax, rmax, xmax, bmax, tid, NT);         \
    break;
      switch (nr) {
        GB_RESID_CASE(1)
        GB_RESID_CASE(2)
        GB_RESID_CASE(3)
        GB_RESID_CASE(4)
        GB_RESID_CASE(5)
        GB_RESID_CASE(6)
        GB_RESID_CASE(7)
        GB_RESID_CASE(8)
        default:
          break;
      }
#undef GB_RESID_CASE
      // all column maxima (and max_i sum_j |a_ij| on the first pass) in one
      // block reduction: value k < nr is |r_k|, then |x_k|, |b_k|, ||A||
      const double* cm = block_max_many(rmax, xmax, bmax, amax, nr, it == 0, sm.redd, NT);
      if (it == 0) anorm = cm[3 * nr];
      worst = 0.0;
      unsigned still = 0u;
      for (int q = 0; q < nr; ++q) {
        const double rn = cm[q];
        const double xn = cm[nr + q];
        const double bn = cm[2 * nr + q];
        const double den = eps * (anorm * xn + bn) * (double)n;
        const double sc = den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
        worst = fmax(worst, sc);
        if (!(sc < tol)) still |= 1u << q;
      }
      active = still;
      if (still == 0u) {
        result = 0;
        break;
      }
      if (it >= max_iter) {
        result = -1;
        break;
      }
      // d = solve(r) in FP32, x += d for the columns not yet converged
      __syncthreads();
      for (int e = tid; e < nr * n; e += NT) {
        const int q = e / n, r = e % n;
        ys[q * BT_NMAX + r] = (float)rs[q * BT_NMAX + sm.perm[r]];
      }
      __syncthreads();
      bt_solve<NT>(W, ld, n, nr, ys, sm);
      for (int e = tid; e < nr * n; e += NT) {
        const int q = e / n, r = e % n;
        if ((active >> q) & 1u) xs[q * BT_NMAX + r] += (double)ys[q * BT_NMAX + r];
      }
      __syncthreads();
      ++it;
    }
    for (int e = tid; e < nr * n; e += NT) {
      const int q = e / n, r = e % n;
      d.X[(int64_t)q * d.ldx + r] = xs[q * BT_NMAX + r];
    }
    if (tid == 0) {
      info_out[sys] = result;
      if (iters_out) iters_out[sys] = it;
      if (resid_out) resid_out[sys] = worst;
    }
    __syncthreads();
  }
}

}  // namespace gb

using namespace gb;

// ------------------------------------------------------------------ host side
struct lu_batch_s {
  lu_ctx ctx = nullptr;
  cudaStream_t stream = nullptr;
  int count = 0;
  int nmax = 0;
  double tol = 16.0;
  int max_iter = 50;
  BatchDesc* d_desc = nullptr;
  int* d_order = nullptr;
  int* d_next = nullptr;
  float* d_scratch = nullptr;
  int64_t slot_floats = 0;
  int threads = 256;
  int ctas_per_sm = 1;
  int grid = 0;
  float tuned_ms = 0.f;
  int sm_count = 0;
  // graph of the current launch shape, keyed by the output pointers
  cudaGraphExec_t exec = nullptr;
  int* g_info = nullptr;
  int* g_iters = nullptr;
  double* g_resid = nullptr;
};

// accessors of the context (defined in lu_api.cu)
cudaStream_t gb_ctx_stream(lu_ctx c);
int gb_ctx_sm_count(lu_ctx c);
int* gb_ctx_status(lu_ctx c);
void gb_ctx_count_launches(lu_ctx c, long long k);
void* gb_ctx_alloc(lu_ctx c, size_t bytes);
void gb_ctx_free(lu_ctx c, void* p);

template <int NT>
static cudaError_t launch_batched(lu_batch b, int* info, int* iters, double* resid, cudaStream_t st) {
  auto kern = batched_kernel<NT>;
  const size_t smem = sizeof(BatchSmem);  // opt-in size set by occupancy() at plan time
  cudaError_t e = cudaMemsetAsync(b->d_next, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  kern<<<b->grid, NT, smem, st>>>(b->d_desc, b->d_order, b->count, b->d_next, b->d_scratch, b->slot_floats, info,
                                  iters, resid, b->tol, b->max_iter, gb_ctx_status(b->ctx));
  return cudaGetLastError();
}

static cudaError_t launch_shape(lu_batch b, int* info, int* iters, double* resid, cudaStream_t st) {
  return b->threads == 512 ? launch_batched<512>(b, info, iters, resid, st)
                           : launch_batched<256>(b, info, iters, resid, st);
}

static int occupancy(int threads) {
  int per = 0;
  const size_t smem = sizeof(BatchSmem);
  if (threads == 512) {
    allow_max_smem((const void*)batched_kernel<512>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel<512>, 512, smem);
  } else {
    allow_max_smem((const void*)batched_kernel<256>);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batched_kernel<256>, 256, smem);
  }
  return per;
}

extern "C" void lu_batch_free(lu_batch b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  gb_ctx_free(b->ctx, b->d_desc);
  gb_ctx_free(b->ctx, b->d_scratch);
  delete b;
}

extern "C" int lu_batch_create(lu_ctx ctx, int count, const int* n, const int* nrhs, const double* const* dA,
                               const int* lda, const double* const* dB, const int* ldb, double* const* dX,
                               const int* ldx, lu_prec prec, double tol, int max_iter, int tune, lu_batch* out) {
  if (!ctx) return -1;
  if (count < 0) return -2;
  if (!out) return -15;
  *out = nullptr;
  if (count > 0 && (!n || !nrhs || !dA || !lda || !dB || !ldb || !dX || !ldx)) return -3;
  if (prec != LU_F32) return -11;
  if (!(tol > 0)) return -12;
  if (max_iter < 0) return -13;
  std::vector<BatchDesc> h(count);
  int nmax = 1;
  for (int i = 0; i < count; ++i) {
    if (n[i] < 1 || n[i] > BT_NMAX) return -3;
    if (nrhs[i] < 1 || nrhs[i] > BT_RHSMAX) return -4;
    if (!dA[i] || !dB[i] || !dX[i]) return -5;
    if (lda[i] < n[i] || ldb[i] < n[i] || ldx[i] < n[i]) return -6;
    h[i] = BatchDesc{dA[i], dB[i], dX[i], n[i], nrhs[i], lda[i], ldb[i], ldx[i], 0};
    nmax = std::max(nmax, n[i]);
  }
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return n[a] > n[c]; });

  lu_batch b = new (std::nothrow) lu_batch_s();
  if (!b) return LU_ENOMEM;
  b->ctx = ctx;
  b->stream = gb_ctx_stream(ctx);
  b->count = count;
  b->nmax = nmax;
  b->tol = tol;
  b->max_iter = max_iter;
  b->sm_count = gb_ctx_sm_count(ctx);
  const int ldmax = (nmax + 3) & ~3;
  b->slot_floats = ((int64_t)nmax * ldmax + 63) / 64 * 64;
  // launch shape: threads per CTA and CTAs per SM (scratch sized for the most)
  const int occ256 = occupancy(256);
  const int maxper = std::max(1, std::min(2, occ256));
  b->threads = 256;
  b->ctas_per_sm = maxper;
  const int slots = b->sm_count * maxper;
  const size_t desc_bytes = ((sizeof(BatchDesc) * std::max(count, 1) + 255) / 256) * 256;
  const size_t order_bytes = ((sizeof(int) * std::max(count, 1) + 255) / 256) * 256;
  void* p = gb_ctx_alloc(ctx, desc_bytes + order_bytes + 256);
  if (!p) {
    delete b;
    return LU_ENOMEM;
  }
  b->d_desc = (BatchDesc*)p;
  b->d_order = (int*)((char*)p + desc_bytes);
  b->d_next = (int*)((char*)p + desc_bytes + order_bytes);
  b->d_scratch = (float*)gb_ctx_alloc(ctx, sizeof(float) * b->slot_floats * slots);
  if (!b->d_scratch) {
    lu_batch_free(b);
    return LU_ENOMEM;
  }
  if (count > 0) {
    // the descriptors: a stream-ordered copy from this call's host arrays
    if (cudaMemcpyAsync(b->d_desc, h.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
      lu_batch_free(b);
      return LU_ECUDA;
    }
  }
  b->grid = std::min(std::max(count, 1), b->sm_count * b->ctas_per_sm);
  if (tune && count > 0) {
    // time each candidate shape on this batch and keep the fastest
    int* tinfo = (int*)gb_ctx_alloc(ctx, sizeof(int) * count);
    if (!tinfo) {
      lu_batch_free(b);
      return LU_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bt = 256, bc = 1;
    const int cand_t[2] = {256, 512};
    for (int ti = 0; ti < 2; ++ti) {
      const int per = std::max(1, std::min(maxper, occupancy(cand_t[ti])));
      for (int cps = 1; cps <= per; ++cps) {
        b->threads = cand_t[ti];
        b->ctas_per_sm = cps;
        b->grid = std::min(count, b->sm_count * cps);
        float ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
          cudaEventRecord(e0, b->stream);
          if (launch_shape(b, tinfo, nullptr, nullptr, b->stream) != cudaSuccess) break;
          cudaEventRecord(e1, b->stream);
          cudaEventSynchronize(e1);
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          if (rep > 0) ms = std::min(ms, t);
        }
        if (ms < best) {
          best = ms;
          bt = cand_t[ti];
          bc = cps;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    gb_ctx_free(ctx, tinfo);
    b->threads = bt;
    b->ctas_per_sm = bc;
    b->grid = std::min(count, b->sm_count * bc);
    b->tuned_ms = best;
  }
  *out = b;
  return LU_OK;
}

extern "C" int lu_batch_shape(lu_batch b, int* threads, int* ctas_per_sm, float* ms) {
  if (!b) return -1;
  if (threads) *threads = b->threads;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (ms) *ms = b->tuned_ms;
  return LU_OK;
}

extern "C" int lu_batch_run(lu_batch b, int* dInfo, int* dIters, double* dResid) {
  if (!b) return -1;
  if (!dInfo && b->count > 0) return -2;
  if (b->count == 0) return LU_OK;
  // (re)capture the launch as a graph when the outputs change
  if (!b->exec || b->g_info != dInfo || b->g_iters != dIters || b->g_resid != dResid) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return LU_ECUDA;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = launch_shape(b, dInfo, dIters, dResid, cs);
      e = cudaStreamEndCapture(cs, &g);
      if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b->exec = nullptr;
      return LU_ECUDA;
    }
    b->g_info = dInfo;
    b->g_iters = dIters;
    b->g_resid = dResid;
  }
  if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess) return LU_ECUDA;
  gb_ctx_count_launches(b->ctx, 1);
  return LU_OK;
}

// Device bytes a plan of `count` systems (largest n = nmax) allocates, for a
// caller that budgets memory (the solve server): descriptors, order, queue
// counter and the per-CTA working copies at the largest launch shape.
size_t gb_batch_bytes(int count, int nmax, int sm_count) {
  const int ldmax = (nmax + 3) & ~3;
  const int64_t slot_floats = ((int64_t)nmax * ldmax + 63) / 64 * 64;
  const size_t desc_bytes = ((sizeof(BatchDesc) * std::max(count, 1) + 255) / 256) * 256;
  const size_t order_bytes = ((sizeof(int) * std::max(count, 1) + 255) / 256) * 256;
  return desc_bytes + order_bytes + 256 + sizeof(float) * (size_t)slot_floats * (size_t)sm_count * 2;
}

extern "C" int lu_solve_batched(lu_ctx ctx, int count, const int* n, const int* nrhs, const double* const* dA,
                                const int* lda, double* const* dB, const int* ldb, lu_prec prec, int* dInfo) {
  lu_batch b = nullptr;
  int rc = lu_batch_create(ctx, count, n, nrhs, dA, lda, (const double* const*)dB, ldb, dB, ldb, prec, 16.0, 50, 0,
                           &b);
  if (rc) return rc;
  rc = lu_batch_run(b, dInfo, nullptr, nullptr);
  cudaStream_t st = gb_ctx_stream(ctx);
  if (cudaStreamSynchronize(st) != cudaSuccess && rc == LU_OK) rc = LU_ECUDA;
  lu_batch_free(b);
  return rc;
}
