// The paper's own LU variant: no pivoting on a diagonally dominant A (HPL-AI
// rules, arxiv 2202.13995, section "High Performance Linpack"), with the four
// per-block operations of its "Base Implementation" (figure "lu_iteration"):
//   LU    -- factor the diagonal block,
//   top   -- A12 <- L11^-1 A12           (trsm_lower_kernel, panel.cu),
//   left  -- A21 <- A21 U11^-1           (below_solve_kernel, here),
//   inner -- A22 <- A22 - A21 A12        (the trailing-update GEMMs).
// Without pivoting no column needs a search over all rows, so the latency of
// the partial-pivot panel disappears; the price is stability, which the
// diagonal dominance of the matrix provides.
//
// Here the "LU" and "left" operations factor a whole m x w block column
// without pivoting, slab by slab: the block column's top h rows (a slab) are
// factored by one CTA in shared memory -- the LU of the slab's h x h diagonal
// block and its U rows to the right -- and then every row below the slab gets
// its L columns (X <- X U^-1 for the slab's h columns) and the update of the
// block column's remaining columns, a CTA per 64 rows.  The next slab starts
// h rows and h columns further down.  The same two kernels serve the
// diagonal-pivot check of a pivoted panel (SpecArgs in kernels.h).
#include "common.cuh"
#include "kernels.h"

namespace gb {

// Device view of SpecArgs.  Flags: [0] sticky failure, [1] kabs + 1 of a panel
// whose slab failed and [2] the rows to restore then, [3] kabs + 1 of a panel
// whose rows below a slab failed (every row to restore).
template <typename T>
struct SpecDev {
  int* flag;
  T* backup;
  int* ipiv;
  int* perm;
};

template <typename T>
__device__ __forceinline__ bool spec_ok_mult(T l) {
  return l <= T(0.5) && l >= T(-0.5);  // false for NaN
}

template <typename T>
__device__ __forceinline__ bool finite_nonzero(T v) {
  return v != T(0) && v - v == T(0);
}

// 16-byte vector of T
template <typename T>
struct V16;
template <>
struct V16<float> {
  using type = float4;
  static constexpr int n = 4;
};
template <>
struct V16<double> {
  using type = double2;
  static constexpr int n = 2;
};
template <typename T>
__device__ __forceinline__ void v16_get(const typename V16<T>::type& v, T* out);
template <>
__device__ __forceinline__ void v16_get<float>(const float4& v, float* o) {
  o[0] = v.x;
  o[1] = v.y;
  o[2] = v.z;
  o[3] = v.w;
}
template <>
__device__ __forceinline__ void v16_get<double>(const double2& v, double* o) {
  o[0] = v.x;
  o[1] = v.y;
}

template <typename T>
__device__ __forceinline__ typename V16<T>::type v16_make(const T* e);
template <>
__device__ __forceinline__ float4 v16_make<float>(const float* e) {
  return make_float4(e[0], e[1], e[2], e[3]);
}
template <>
__device__ __forceinline__ double2 v16_make<double>(const double* e) {
  return make_double2(e[0], e[1]);
}

// Rows [0, nrows) x columns [0, ncol) of G (row-major, ld) into S (row
// stride sld), and, when B is set, to B too (row stride ncol).  Each warp
// takes four rows at a time with all their loads in flight; 16-byte loads
// when G's rows are 16-byte aligned.  Rows nrows .. rows_alloc of S are
// zero-filled.
template <typename T, int NT>
__device__ __forceinline__ void load_rows(const T* G, int64_t ld, int nrows, int rows_alloc, int ncol, T* S,
                                          int sld, T* B) {
  constexpr int VN = V16<T>::n;
  using VT = typename V16<T>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NT / 32;
  const bool vec = ((reinterpret_cast<uintptr_t>(G) & 15) == 0) && ((ld * (int64_t)sizeof(T)) & 15) == 0;
  const int nvec = vec ? ncol / VN : 0;  // whole vectors per row
  for (int r0 = warp * 4; r0 < rows_alloc; r0 += NW * 4) {
    // the vector part: 4 rows x 4 vectors per lane in flight at a time
    for (int v0 = 0; v0 < nvec; v0 += 32 * 4) {
      VT buf[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = r0 + i, v = v0 + lane + 32 * q;
          if (r < nrows && v < nvec) buf[i][q] = reinterpret_cast<const VT*>(G + (int64_t)r * ld)[v];
        }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int r = r0 + i, v = v0 + lane + 32 * q;
          if (r < rows_alloc && v < nvec) {
            T e[VN];
            if (r < nrows) {
              v16_get<T>(buf[i][q], e);
            } else {
#pragma unroll
              for (int x = 0; x < VN; ++x) e[x] = T(0);
            }
#pragma unroll
            for (int x = 0; x < VN; ++x) {
              S[(size_t)r * sld + v * VN + x] = e[x];
              if (B && r < nrows) B[(int64_t)r * ncol + v * VN + x] = e[x];
            }
          }
        }
    }
    // the scalar rest of each row
    for (int i = 0; i < 4; ++i) {
      const int r = r0 + i;
      if (r >= rows_alloc) break;
      for (int c = nvec * VN + lane; c < ncol; c += 32) {
        const T e = r < nrows ? G[(int64_t)r * ld + c] : T(0);
        S[(size_t)r * sld + c] = e;
        if (B && r < nrows) B[(int64_t)r * ncol + c] = e;
      }
    }
  }
}

// ============================================================ slab LU
// One CTA factors the slab D (hs rows x wt columns, row-major, ld) in shared
// memory: the LU of its hs x hs diagonal block without pivoting, blocked by 32
// columns, and U's rows right of the block (columns hs .. wt).  Per block of
// 32 columns:
//   (i)  the block's columns, one at a time: the multipliers of the column (a
//        thread per row, dividing by the pivot as in the definition), then a
//        rank-1 update of the rows below it within the block's columns (a
//        thread per row); two barriers per column;
//   (i') the block's rows right of the block (U's rows there) by forward
//        substitution with the block's L, a thread per column;
//   (ii) a rank-32 update of the rows below the block and the columns right
//        of it (register tiles).
// Then, for the rows below the slab, (iii) the inverses of U's 32 x 32
// diagonal blocks (a warp per block), written to uinv.
// The loops stay rolled, with their shared-memory loads batched ahead of the
// products: the kernel runs once per launch on one SM, where a long
// straight-line body would be fetched from L2 at every block.
// A zero pivot lowers *info to its absolute column + 1 (kabs = D's first
// column) and skips its scaling.  With sp.flag set it is a stage of a pivoted
// panel's diagonal-pivot check: the first slab (first != 0) saves its rows to
// sp.backup and writes the identity pivots and an empty permutation record
// for the panel's wt columns; *info is left alone; a multiplier above 1/2, or
// a zero or non-finite pivot, records the failure (flag[1] = tag, flag[2] =
// restore_rows, then flag[0]).  It returns at once when an earlier stage or
// panel failed.
constexpr int SL_THREADS = 256;

// Row stride of the slab in shared memory, in elements: at least the width
// and whole 32-column blocks, and VN (mod 2 VN) for VN elements per 16 bytes,
// so that each thread's 16-byte piece of its own row falls in banks of its
// own within a quarter-warp.
__host__ __device__ inline int slab_wp(int hs, int wt, int tsize) {
  const int vn = 16 / tsize;
  const int w = wt > ((hs + 31) & ~31) ? wt : ((hs + 31) & ~31);
  return (w + 2 * vn - 1) / (2 * vn) * (2 * vn) + vn;
}
// shared memory of one slab: rows, the pivot row's block columns, the
// multipliers, and a 32 x 33 scratch per diagonal block for its U's inverse
inline size_t slab_smem_bytes(int hs, int wt, int tsize) {
  return ((size_t)hs * slab_wp(hs, wt, tsize) + 32 + (size_t)hs + (size_t)((hs + 31) / 32) * 32 * 33) * tsize;
}

template <typename T>
__global__ void __launch_bounds__(SL_THREADS) slab_lu_kernel(T* D, int64_t ld, int hs, int wt, int kabs, int* info,
                                                             SpecDev<T> sp, int first, int tag, int restore_rows,
                                                             T* uinv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int VN = V16<T>::n;
  using VT = typename V16<T>::type;
  const int wp = slab_wp(hs, wt, sizeof(T));
  T* A = reinterpret_cast<T*>(smem_raw);  // [hs][wp]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool spec = sp.flag != nullptr;
  bool bad = false;
  if (spec) {
    const int f0 = __ldcg(sp.flag), f3 = __ldcg(sp.flag + 3);
    if (f0 != 0 || f3 != 0) {
      if (tid == 0 && f0 == 0) sp.flag[0] = 1;  // a failure of the rows below an earlier slab
      return;
    }
  }
  load_rows<T, SL_THREADS>(D, ld, hs, hs, wt, A, wp, (spec && first) ? sp.backup : nullptr);
  if (spec && first) {
    for (int j = tid; j < wt; j += SL_THREADS) sp.ipiv[kabs + j] = kabs + j + 1;
    if (tid == 0) sp.perm[0] = 0;
  }
  __syncthreads();
  T* pr = A + (size_t)hs * wp;  // [32]: the pivot row's block columns right of the pivot, zero elsewhere
  T* lcol = pr + 32;            // [hs]: the current column's multipliers
  for (int c0 = 0; c0 < hs; c0 += 32) {
    const int bw = min(32, hs - c0);
    const int r1 = c0 + bw;
    // (i) the block's columns, one at a time.  Column cj: (a) a thread per
    //     row below the pivot divides by the pivot (as in the definition),
    //     and the last warp copies the pivot row's block columns right of cj;
    //     (b) a thread per row below cj applies the rank-1 update to its
    //     row's 32 block columns in 16-byte pieces (the copy's zeros leave
    //     the columns at and left of cj as they are).
    for (int j = 0; j < bw; ++j) {
      const int cj = c0 + j;
      const T piv = A[cj * wp + cj];
      const bool pz = !(piv != T(0));
      if (tid == 0) {
        if (spec) {
          if (!finite_nonzero(piv)) bad = true;
        } else if (pz) {
          atomicMin(info, kabs + cj + 1);
        }
      }
      for (int r = cj + 1 + tid; r < hs; r += SL_THREADS) {
        T l = A[r * wp + cj];
        if (!pz) l = l / piv;
        if (spec && !spec_ok_mult(l)) bad = true;
        A[r * wp + cj] = l;
        lcol[r] = l;
      }
      if (warp == SL_THREADS / 32 - 1) {  // (never a row thread: a slab has at most 128 rows)
        const int k = c0 + lane;
        pr[lane] = (k > cj && k < r1) ? A[cj * wp + k] : T(0);
      }
      __syncthreads();
      for (int r = cj + 1 + tid; r < hs; r += SL_THREADS) {
        const T nl = -lcol[r];
        VT* y = reinterpret_cast<VT*>(A + r * wp + c0);
        const VT* x = reinterpret_cast<const VT*>(pr);
#pragma unroll
        for (int v = 0; v < 32 / VN; ++v) {
          T yv[VN], xv[VN];
          v16_get<T>(y[v], yv);
          v16_get<T>(x[v], xv);
#pragma unroll
          for (int e = 0; e < VN; ++e) yv[e] = fma(nl, xv[e], yv[e]);
          y[v] = v16_make<T>(yv);
        }
      }
      __syncthreads();
    }
    // (i') the block's rows right of the block: forward substitution with the
    //      block's unit lower L, a thread per column -- the same products in
    //      the same order as rank-1 updates column by column would apply them
    for (int k = r1 + tid; k < wt; k += SL_THREADS) {
      for (int t = c0 + 1; t < r1; ++t) {
        T v = A[t * wp + k];
        for (int s0 = c0; s0 < t; s0 += 8) {
          T lv[8], xv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int ss = s0 + u < t ? s0 + u : t - 1;
            lv[u] = A[t * wp + ss];
            xv[u] = A[ss * wp + k];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (s0 + u < t) v = fma(-lv[u], xv[u], v);
        }
        A[t * wp + k] = v;
      }
    }
    __syncthreads();
    // (ii) rank-bw update of rows [r1, hs) x columns [r1, wt): a thread per
    //       4 rows x 4 columns 32 apart (the warp reads consecutive columns)
    const int nr = hs - r1, nc = wt - r1;
    if (nr > 0 && nc > 0) {
      const int ntr = (nr + 3) / 4, ncg = (nc + 127) / 128;
      for (int it = tid; it < ntr * ncg * 32; it += SL_THREADS) {
        const int cl = it & 31, g = (it >> 5) % ncg, tr = (it >> 5) / ncg;
        const int rr = r1 + 4 * tr, cc = r1 + 128 * g + cl;
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = T(0);
#pragma unroll 4
        for (int j = 0; j < bw; ++j) {
          T av[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) av[i] = rr + i < hs ? A[(rr + i) * wp + c0 + j] : T(0);
#pragma unroll
          for (int q = 0; q < 4; ++q) bv[q] = cc + 32 * q < wt ? A[(c0 + j) * wp + cc + 32 * q] : T(0);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = fma(av[i], bv[q], acc[i][q]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (rr + i < hs && cc + 32 * q < wt) A[(rr + i) * wp + cc + 32 * q] -= acc[i][q];
      }
    }
    __syncthreads();
  }
  for (int r = warp; r < hs; r += SL_THREADS / 32)
    for (int c = lane; c < wt; c += 32) D[(int64_t)r * ld + c] = A[r * wp + c];
  // (iii) for the rows below the slab: the inverse of each 32 x 32 diagonal
  //       block of U, a warp per block, a lane per column of the inverse:
  //       back substitution with the division by U's diagonal; uinv[b]
  //       (32 x 32, row-major), the identity outside a ragged last block
  if (uinv != nullptr) {
    T* Zs = lcol + hs;
    for (int b = warp; 32 * b < hs; b += SL_THREADS / 32) {
      const int c0 = 32 * b, bw = min(32, hs - c0);
      T* Z = Zs + (size_t)b * 32 * 33;  // [32][33]
      const T* Ub = A + (size_t)c0 * wp + c0;
      for (int t = 0; t < 32; ++t) Z[t * 33 + lane] = (t == lane) ? T(1) : T(0);
      __syncwarp();
      for (int t = bw - 1; t >= 0; --t) {
        const T zt = Z[t * 33 + lane] / Ub[t * wp + t];
        Z[t * 33 + lane] = zt;
        for (int q0 = 0; q0 < t; q0 += 8) {
          T uq[8], zq[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int q = q0 + u < t ? q0 + u : t - 1;
            uq[u] = Ub[q * wp + t];
            zq[u] = Z[q * 33 + lane];
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (q0 + u < t) Z[(q0 + u) * 33 + lane] = zq[u] - uq[u] * zt;
        }
        __syncwarp();
      }
      T* ub = uinv + (size_t)b * 1024;
      for (int t = 0; t < 32; ++t) ub[t * 32 + lane] = Z[t * 33 + lane];
    }
  }
  if (spec && __syncthreads_or(bad) && tid == 0) {
    sp.flag[1] = tag;
    sp.flag[2] = restore_rows;
    __threadfence();
    sp.flag[0] = 1;
  }
}

// ============================================================ rows below a slab
// X (m x wt, row-major, ld): the ws columns of a slab's rows below it are
// solved against the slab's upper ws x ws block U (X <- X U^-1, the paper's
// "left" block update) and the other wt - ws columns updated with U's rows
// right of the block (U is ws x wt at U, row-major, ld).  CTA = RB rows of X
// in shared memory; by 32-column blocks of the ws:
//   1. U's 32 rows of the block staged in shared memory (cp.async);
//   2. the diagonal block: X_b <- X_b U_bb^-1, a small product with the
//      inverse of U's 32 x 32 diagonal block, which the slab kernel wrote to
//      uinv (32 x 32 per block, row-major);
//   3. the columns to the right: a rank-32 update, each thread a register
//      tile of RB/16 rows x 4 columns per 64-column chunk, its rows' values
//      of the block read from a transposed copy (one 16-byte load per k).
// With sp.flag set it is a stage of the diagonal-pivot check: for the first
// slab (first != 0) the rows are saved to sp.backup first and the stage runs
// unless flag[0] is set; a later stage returns on flag[0] or flag[3].  A
// multiplier above 1/2 in magnitude (or not finite) records flag[3] = tag.
constexpr int LS_THREADS = 256;

template <typename T, int RB>
__global__ void __launch_bounds__(LS_THREADS) below_solve_kernel(const T* __restrict__ U, const T* __restrict__ uinv,
                                                                 T* X, int64_t ld, int m, int ws, int wt,
                                                                 SpecDev<T> sp, int first, int tag) {
  static_assert(RB % 16 == 0 && RB <= LS_THREADS, "RB rows: 16 row groups, one thread per row");
  constexpr int RT = RB / 16;  // rows per thread in the update
  constexpr int VN = V16<T>::n;
  using VT = typename V16<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wx = wt | 1;          // odd row stride: a row per thread is free of bank conflicts
  const int wu = (wt + 3) & ~3;   // U stage row stride: 16-byte rows
  T* Us = reinterpret_cast<T*>(smem_raw);  // [32][wu]: rows c0 .. c0 + 31 of U, columns c0 .. wt
  T* Ui = Us + 32 * wu;                    // [32][32]: the inverse of U's current 32 x 32 diagonal block
  T* Xs = Ui + 32 * 32;                    // [RB][wx]
  T* XT = Xs + RB * wx;                    // [32][RB]: the solved block, transposed (16-byte aligned)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = blockIdx.x * RB;
  const int rows = min(RB, m - r0);
  const bool spec = sp.flag != nullptr;
  if (spec) {
    const bool stop = first ? __ldcg(sp.flag) != 0 : (__ldcg(sp.flag) != 0 || __ldcg(sp.flag + 3) != 0);
    if (stop) return;
  }
  bool bad = false;
  const bool uvec = ((reinterpret_cast<uintptr_t>(U) & 15) == 0) && ((ld * (int64_t)sizeof(T)) & 15) == 0;
  load_rows<T, LS_THREADS>(X + (int64_t)r0 * ld, ld, rows, RB, wt, Xs, wx,
                           (spec && first) ? sp.backup + (int64_t)r0 * wt : nullptr);
  for (int c0 = 0; c0 < ws; c0 += 32) {
    const int bw = min(32, ws - c0);
    __syncthreads();  // the previous block's update is done with Us
    // U's rows c0 .. c0 + bw, columns c0 .. wt: asynchronous copies, all in flight together
    {
      const int nv = uvec ? (wt - c0) / VN : 0;  // c0 is a multiple of 32: 16-byte aligned when U's rows are
      for (int e = tid; e < bw * nv; e += LS_THREADS) {
        const int k = e / nv, v = e % nv;
        cp_async<16>(&Us[k * wu + c0 + v * VN], &U[(int64_t)(c0 + k) * ld + c0 + v * VN]);
      }
      const int done = c0 + nv * VN, rest = wt - done;
      for (int e = tid; e < bw * rest; e += LS_THREADS) {
        const int k = e / rest, c = done + e % rest;
        cp_async<sizeof(T)>(&Us[k * wu + c], &U[(int64_t)(c0 + k) * ld + c]);
      }
      const T* ub = uinv + (size_t)(c0 / 32) * 1024;
      for (int e = tid; e < 1024 / VN; e += LS_THREADS) cp_async<16>(&Ui[e * VN], &ub[e * VN]);
      cp_async_wait_all();
    }
    __syncthreads();
    // the diagonal block: X_b <- X_b Ui, a small product over the whole CTA
    // (rows x quads of columns; results held until every thread has read)
    {
      T res[(RB * 8 + LS_THREADS - 1) / LS_THREADS][4];
#pragma unroll
      for (int it = 0; it < (RB * 8 + LS_THREADS - 1) / LS_THREADS; ++it) {
        const int e = tid + it * LS_THREADS;
        const int r = e >> 3, cq = (e & 7) * 4;
#pragma unroll
        for (int q = 0; q < 4; ++q) res[it][q] = T(0);
        if (e < RB * 8) {
#pragma unroll 8
          for (int k = 0; k < bw; ++k) {
            const T xk = Xs[r * wx + c0 + k];
            T uv[4];
            v16_get<T>(*reinterpret_cast<const VT*>(&Ui[k * 32 + cq]), uv);
            if (VN == 2) v16_get<T>(*reinterpret_cast<const VT*>(&Ui[k * 32 + cq + 2]), uv + 2);
#pragma unroll
            for (int q = 0; q < 4; ++q) res[it][q] = fma(xk, uv[q], res[it][q]);
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int it = 0; it < (RB * 8 + LS_THREADS - 1) / LS_THREADS; ++it) {
        const int e = tid + it * LS_THREADS;
        const int r = e >> 3, cq = (e & 7) * 4;
        if (e < RB * 8) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (cq + q < bw) {
              Xs[r * wx + c0 + cq + q] = res[it][q];
              if (spec && r < rows && !spec_ok_mult(res[it][q])) bad = true;
            }
          }
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < 32 * RB; e += LS_THREADS) {
      const int k = e / RB, r = e % RB;
      XT[k * RB + r] = k < bw ? Xs[r * wx + c0 + k] : T(0);
    }
    __syncthreads();
    const int c1 = c0 + bw;  // columns [c1, wt) remain
    const int rg = tid >> 4, cg = tid & 15;
    for (int cc = c1 + 4 * cg; cc < wt; cc += 64) {
      T acc[RT][4];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = T(0);
#pragma unroll 4
      for (int k = 0; k < bw; ++k) {
        // columns past wt are never stored; c1 and cc are multiples of 4 (a
        // remaining column exists only after a full 32-column block), so the
        // 16-byte loads stay inside the stage's 16-byte rows
        T ub[4], xa[RT];
        const T* up = &Us[k * wu + cc];
        v16_get<T>(*reinterpret_cast<const VT*>(up), ub);
        if (VN == 2) v16_get<T>(*reinterpret_cast<const VT*>(up + 2), ub + 2);
        if constexpr (RT % VN == 0) {
#pragma unroll
          for (int i = 0; i < RT; i += VN) v16_get<T>(*reinterpret_cast<const VT*>(&XT[k * RB + RT * rg + i]), xa + i);
        } else {
#pragma unroll
          for (int i = 0; i < RT; ++i) xa[i] = XT[k * RB + RT * rg + i];
        }
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = fma(xa[i], ub[q], acc[i][q]);
      }
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (cc + q < wt) Xs[(RT * rg + i) * wx + cc + q] -= acc[i][q];
    }
  }
  __syncthreads();
  for (int r = warp; r < rows; r += LS_THREADS / 32)
    for (int c = lane; c < wt; c += 32) X[(int64_t)(r0 + r) * ld + c] = Xs[r * wx + c];
  if (spec && __syncthreads_or(bad) && tid == 0) sp.flag[3] = tag;
}

// ============================================================ launchers
template <typename T>
static SpecDev<T> spec_dev(const SpecArgs& a, int64_t backup_offset) {
  SpecDev<T> d;
  d.flag = a.flag;
  d.backup = a.backup ? reinterpret_cast<T*>(a.backup) + backup_offset : nullptr;
  d.ipiv = a.ipiv;
  d.perm = a.perm;
  return d;
}

static int device_smem_optin() {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return optin;
}

// Slab height: the largest multiple of 32, at most 128, whose slab fits in
// 168 KB of shared memory.
static int slab_rows(int w, int tsize) {
  int h = 128;
  while (h > 32 && slab_smem_bytes(h, w, tsize) > 168 * 1024) h -= 32;
  return h;
}

static size_t ls_smem(int rb, int wt, int tsize) {
  const size_t wu = (size_t)((wt + 3) & ~3);
  return (32 * wu + 32 * 32 + (size_t)rb * (wt | 1) + 32 * (size_t)rb) * tsize;
}

template <typename T, int RB>
static cudaError_t launch_ls(const T* U, const T* uinv, T* X, int64_t ld, int m, int ws, int wt,
                             const SpecDev<T>& sp, int first, int tag, cudaStream_t st) {
  auto kern = below_solve_kernel<T, RB>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)cdiv(m, RB), LS_THREADS, ls_smem(RB, wt, sizeof(T)), st>>>(U, uinv, X, ld, m, ws, wt, sp, first,
                                                                               tag);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_below(const T* U, const T* uinv, T* X, int64_t ld, int m, int ws, int wt,
                                const SpecDev<T>& sp, int first, int tag, cudaStream_t st) {
  const int optin = device_smem_optin();
  if (ls_smem(64, wt, sizeof(T)) <= (size_t)optin)
    return launch_ls<T, 64>(U, uinv, X, ld, m, ws, wt, sp, first, tag, st);
  if (ls_smem(32, wt, sizeof(T)) <= (size_t)optin)
    return launch_ls<T, 32>(U, uinv, X, ld, m, ws, wt, sp, first, tag, st);
  if (ls_smem(16, wt, sizeof(T)) <= (size_t)optin)
    return launch_ls<T, 16>(U, uinv, X, ld, m, ws, wt, sp, first, tag, st);
  return cudaErrorInvalidValue;
}

// One slab: a CTA with the slab in shared memory.
template <typename T>
static cudaError_t launch_slab(T* D, int64_t ld, int hs, int wt, int kabs, int* info, const SpecDev<T>& sp,
                               int first, int tag, int restore, T* uinv, cudaStream_t st) {
  auto kern = slab_lu_kernel<T>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<1, SL_THREADS, slab_smem_bytes(hs, wt, sizeof(T)), st>>>(D, ld, hs, wt, kabs, info, sp, first, tag, restore,
                                                                   uinv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_block_column(T* P, int64_t ld, int m, int w, int kabs, int* info, T* uinv, cudaStream_t st,
                                const SpecArgs& spec) {
  if (w <= 0) return cudaSuccess;
  if (m < w) return cudaErrorInvalidValue;
  const int h = slab_rows(w, sizeof(T));
  cudaError_t e = cudaSuccess;
  const int tag = kabs + 1;
  for (int s0 = 0; s0 < w; s0 += h) {
    const int hs = (w - s0) < h ? (w - s0) : h;
    const int wt = w - s0;
    const int first = s0 == 0;
    T* D = P + (int64_t)s0 * ld + s0;
    // a failed check of the first slab changed only its rows; any later
    // failure, every row of the block column
    const int restore = first ? hs : m;
    const int below = m - s0 - hs;
    T* ui = uinv + (size_t)(s0 / 32) * 1024;  // the slab's diagonal blocks' inverses (for the rows below)
    if ((e = launch_slab<T>(D, ld, hs, wt, kabs + s0, info, spec_dev<T>(spec, 0), first, tag, restore,
                            below > 0 ? ui : nullptr, st)) != cudaSuccess)
      return e;
    if (below > 0) {
      // the first slab's rows below it follow its rows in the backup (row stride w)
      e = launch_below<T>(D, ui, D + (int64_t)hs * ld, ld, below, hs, wt, spec_dev<T>(spec, (int64_t)hs * w), first,
                          tag, st);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

int block_column_launches(int m, int w, int tsize) {
  if (w <= 0) return 0;
  const int h = slab_rows(w, tsize);
  int n = 0;
  for (int s0 = 0; s0 < w; s0 += h) {
    const int hs = (w - s0) < h ? (w - s0) : h;
    n += (m - s0 - hs) > 0 ? 2 : 1;
  }
  return n;
}

template cudaError_t launch_block_column<double>(double*, int64_t, int, int, int, int*, double*, cudaStream_t,
                                                 const SpecArgs&);
template cudaError_t launch_block_column<float>(float*, int64_t, int, int, int, int*, float*, cudaStream_t,
                                                const SpecArgs&);

}  // namespace gb
