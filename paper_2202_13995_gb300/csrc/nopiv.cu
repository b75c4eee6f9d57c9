// The paper's own LU variant: no pivoting on a diagonally dominant A (HPL-AI
// rules, arxiv 2202.13995, section "High Performance Linpack"), with the four
// per-block operations of its "Base Implementation" (figure "lu_iteration"):
//   LU    -- factor the diagonal block (one CTA: no grid-wide step at all),
//   top   -- A12 <- L11^-1 A12           (trsm_lower_kernel, panel.cu),
//   left  -- A21 <- A21 U11^-1           (trsm_right_upper_kernel, here),
//   inner -- A22 <- A22 - A21 A12        (the trailing-update GEMMs).
// Without pivoting no column needs a search over all rows, so the latency of
// the partial-pivot panel disappears; the price is stability, which the
// diagonal dominance of the matrix provides.
#include "common.cuh"
#include "kernels.h"

namespace gb {

constexpr int NP_NB = 32;

// 16-byte global accesses of 16 / sizeof(T) elements, and a 4-element
// shared-memory load (one or two 16-byte accesses); the addresses are aligned.
template <typename T>
__device__ __forceinline__ void load16(const T* p, T* v);
template <>
__device__ __forceinline__ void load16<float>(const float* p, float* v) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
template <>
__device__ __forceinline__ void load16<double>(const double* p, double* v) {
  const double2 x = *reinterpret_cast<const double2*>(p);
  v[0] = x.x;
  v[1] = x.y;
}
template <typename T>
__device__ __forceinline__ void store16(T* p, const T* v);
template <>
__device__ __forceinline__ void store16<float>(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void store16<double>(double* p, const double* v) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
}
template <typename T>
__device__ __forceinline__ void load4s(const T* p, T* v) {
  load16<T>(p, v);
  if (sizeof(T) == 8) load16<T>(p + 2, v + 2);
}
constexpr int NP_CW = 128;  // column chunk of the in-block update
// threads of the diagonal-block CTA: 512 for FP32 (the update loads its C
// tile ahead of the products, which needs more than the 64 registers a thread
// of a 1024-thread CTA has), 256 for FP64 (a thread holds 32 doubles in
// registers)
template <typename T>
constexpr int np_threads() {
  return sizeof(T) == 8 ? 256 : 512;
}

// Device view of SpecArgs (the diagonal-pivot check of a pivoted panel).
// Flags: [0] sticky failure, [1] kabs + 1 of a panel whose diagonal block
// failed, [3] kabs + 1 of a panel whose rows below the block failed.
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

// In-place LU (no pivoting) of the w x w block at D (row-major, ld), blocked by
// 32 columns; one CTA of np_threads<T>() threads.  Lowers *info to kabs + j + 1 at the
// first exactly zero pivot j (and skips that column's scaling).
// With sp.flag set it is the first stage of a pivoted panel's diagonal-pivot
// check: it saves the block to sp.backup, writes the identity pivots and an
// empty permutation record, leaves *info alone, and on a multiplier above 1/2
// or a zero or non-finite pivot records the failure (flag[1], then flag[0]).
template <typename T>
__global__ void __launch_bounds__(np_threads<T>()) diag_lu_kernel(T* D, int64_t ld, int w, int kabs, int* info,
                                                                  SpecDev<T> sp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wp = (w + 3) & ~3;
  T* P = reinterpret_cast<T*>(smem_raw);  // [NP_NB][wp]: column c of the sub-panel, row r
  T* Us = P + (size_t)NP_NB * wp;         // [NP_NB][NP_CW]
  const int tid = threadIdx.x;
  constexpr int NP_NT = np_threads<T>();
  constexpr int CH = 16 / sizeof(T);  // elements per 16-byte access
  const bool vec = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && (ld % CH) == 0;
  const bool spec = sp.flag != nullptr;
  bool bad = false;  // a multiplier above 1/2 or a zero / non-finite pivot (spec only)
  if (spec) {
    // the check is off once a panel has failed it; a failure of the previous
    // panel's rows below its block turns it off here
    const int f0 = __ldcg(sp.flag), f3 = __ldcg(sp.flag + 3);
    if (f0 != 0 || f3 != 0) {
      if (tid == 0 && f0 == 0) sp.flag[0] = 1;
      return;
    }
    for (int r = tid / 32; r < w; r += NP_NT / 32)
      for (int c = tid % 32; c < w; c += 32) sp.backup[(int64_t)r * w + c] = D[(int64_t)r * ld + c];
    for (int j = tid; j < w; j += NP_NT) sp.ipiv[kabs + j] = kabs + j + 1;
    if (tid == 0) sp.perm[0] = 0;
    __syncthreads();
  }
  for (int k0 = 0; k0 < w; k0 += NP_NB) {
    const int kb = min(NP_NB, w - k0), m = w - k0;
    // thread = row (consecutive threads, consecutive rows: the column-major
    // sub-panel is written without bank conflicts), CH columns per load
    for (int e = tid; e < m * (NP_NB / CH); e += NP_NT) {
      const int r = e % m, c = (e / m) * CH;
      if (c >= kb) continue;
      const T* src = D + (int64_t)(k0 + r) * ld + k0 + c;
      if (vec && c + CH <= kb) {
        T v[CH];
        load16<T>(src, v);
#pragma unroll
        for (int x = 0; x < CH; ++x) P[(c + x) * wp + r] = v[x];
      } else {
        for (int x = 0; c + x < kb; ++x) P[(c + x) * wp + r] = src[x];
      }
    }
    __syncthreads();
    for (int j = 0; j < kb; ++j) {
      const T piv = P[j * wp + j];
      if (spec) {
        if (tid == 0 && !(piv != T(0) && piv - piv == T(0))) bad = true;  // zero or non-finite pivot
      } else if (tid == 0 && piv == T(0)) {
        atomicMin(info, kabs + k0 + j + 1);
      }
      for (int r = j + 1 + tid; r < m; r += NP_NT) {
        T l = P[j * wp + r];
        if (piv != T(0)) l = l / piv;
        if (spec && !spec_ok_mult(l)) bad = true;
        P[j * wp + r] = l;
        for (int c = j + 1; c < kb; ++c) P[c * wp + r] -= l * P[c * wp + j];
      }
      __syncthreads();
    }
    for (int e = tid; e < m * (NP_NB / CH); e += NP_NT) {
      const int r = e % m, c = (e / m) * CH;
      if (c >= kb) continue;
      T* dst = D + (int64_t)(k0 + r) * ld + k0 + c;
      if (vec && c + CH <= kb) {
        T v[CH];
#pragma unroll
        for (int x = 0; x < CH; ++x) v[x] = P[(c + x) * wp + r];
        store16<T>(dst, v);
      } else {
        for (int x = 0; c + x < kb; ++x) dst[x] = P[(c + x) * wp + r];
      }
    }
    __syncthreads();
    for (int c0 = k0 + kb; c0 < w; c0 += NP_CW) {
      const int cw = min(NP_CW, w - c0);
      for (int c = tid; c < cw; c += NP_NT) {
        // the column's kb values in registers (loads issued together), then
        // forward substitution with the unit-lower block
        T v[NP_NB];
#pragma unroll
        for (int j = 0; j < NP_NB; ++j) v[j] = j < kb ? D[(int64_t)(k0 + j) * ld + c0 + c] : T(0);
#pragma unroll
        for (int j = 1; j < NP_NB; ++j) {
#pragma unroll
          for (int i = 0; i < NP_NB; ++i)
            if (i < j) v[j] -= P[i * wp + j] * v[i];
        }
#pragma unroll
        for (int j = 0; j < NP_NB; ++j) {
          if (j < kb) {
            Us[j * NP_CW + c] = v[j];
            D[(int64_t)(k0 + j) * ld + c0 + c] = v[j];
          }
        }
      }
      __syncthreads();
      const int rows = m - kb;
      const int rt = (rows + 3) / 4, ct = (cw + 3) / 4;
      for (int t = tid; t < rt * ct; t += NP_NT) {
        const int r0 = kb + (t / ct) * 4, cc = (t % ct) * 4;
        // the tile's entries of D first: their latency runs under the products
        T dv[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const T* dr = D + (int64_t)(k0 + min(r0 + i, m - 1)) * ld + c0 + cc;
#pragma unroll
          for (int q = 0; q < 4; ++q) dv[i][q] = (r0 + i < m && cc + q < cw) ? dr[q] : T(0);
        }
        T acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = T(0);
        // kb = NP_NB here (the last block has no rows below it), so r0 and cc
        // are multiples of 4: 16-byte shared loads.  Lanes past m or cw read
        // stale entries into rows / columns of acc that are never stored.
        for (int k = 0; k < kb; ++k) {
          T a[4], b[4];
          load4s<T>(&P[k * wp + r0], a);
          load4s<T>(&Us[k * NP_CW + cc], b);
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][q] = fma(a[i], b[q], acc[i][q]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if (r0 + i >= m) break;
          T* dr = D + (int64_t)(k0 + r0 + i) * ld + c0 + cc;
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (cc + q < cw) dr[q] = dv[i][q] - acc[i][q];
        }
      }
      __syncthreads();
    }
  }
  if (spec && __syncthreads_or(bad) && tid == 0) {
    sp.flag[1] = kabs + 1;
    __threadfence();
    sp.flag[0] = 1;
  }
}

// X (m x w, row-major, ld) <- X U^-1 with U the upper (non-unit) w x w block at
// U (row-major, ld): the paper's "left" block update.  CTA = RB rows of X in
// shared memory; by 32-column blocks:
//   1. the diagonal block: one thread per row substitutes its 32 values in
//      registers against U's 32 x 32 diagonal block, multiplying by the
//      reciprocals of U's diagonal (computed once per CTA);
//   2. the columns to the right: a rank-32 update, each thread a register tile
//      of RB/16 rows x 4 columns per 64-column chunk, U's rows staged in shared
//      memory.
// With sp.flag set it is the second stage of a pivoted panel's diagonal-pivot
// check: the rows are saved to sp.backup first, and a multiplier above 1/2 in
// magnitude (or not finite) records the panel in flag[3].  It returns at once
// when flag[0] is set (the check is off, or the diagonal block failed it).
constexpr int LS_THREADS = 256;

template <typename T, int RB>
__global__ void __launch_bounds__(LS_THREADS) trsm_right_upper_kernel(const T* __restrict__ U, T* X, int64_t ld,
                                                                      int m, int w, int kabs, SpecDev<T> sp) {
  static_assert(RB % 16 == 0 && RB <= LS_THREADS, "RB rows: 16 row groups, one thread per row");
  constexpr int RT = RB / 16;  // rows per thread in the update
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wx = w | 1;          // odd row stride: a row per thread is free of bank conflicts
  const int wu = (w + 3) & ~3;   // U stage row stride: 16-byte rows
  T* Us = reinterpret_cast<T*>(smem_raw);  // [32][wu]: rows c0 .. c0 + 31 of U, columns c0 .. w
  T* rcp = Us + 32 * wu;                   // [wu]: 1 / U(j, j)
  T* Xs = rcp + wu;                        // [RB][wx]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r0 = blockIdx.x * RB;
  const int rows = min(RB, m - r0);
  const bool spec = sp.flag != nullptr;
  if (spec && __ldcg(sp.flag) != 0) return;
  bool bad = false;
  for (int j = tid; j < w; j += LS_THREADS) rcp[j] = T(1) / U[(int64_t)j * ld + j];
  for (int r = warp; r < RB; r += LS_THREADS / 32) {
    const bool ok = r < rows;
    for (int c = lane; c < w; c += 32) {
      const T v = ok ? X[(int64_t)(r0 + r) * ld + c] : T(0);
      Xs[r * wx + c] = v;
      if (spec && ok) sp.backup[(int64_t)(r0 + r) * w + c] = v;
    }
  }
  for (int c0 = 0; c0 < w; c0 += 32) {
    const int bw = min(32, w - c0);
    __syncthreads();  // the previous block's update is done with Us
    for (int k = warp; k < bw; k += LS_THREADS / 32)
      for (int c = c0 + lane; c < w; c += 32) Us[k * wu + c] = U[(int64_t)(c0 + k) * ld + c];
    __syncthreads();
    if (tid < rows) {
      T a[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) a[j] = j < bw ? Xs[tid * wx + c0 + j] : T(0);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        if (j < bw) {
          const T x = a[j] * rcp[c0 + j];
          if (spec && !spec_ok_mult(x)) bad = true;
          a[j] = x;
#pragma unroll
          for (int k = j + 1; k < 32; ++k)
            if (k < bw) a[k] -= x * Us[j * wu + c0 + k];
        }
      }
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (j < bw) Xs[tid * wx + c0 + j] = a[j];
    }
    __syncthreads();
    const int c1 = c0 + bw;  // columns [c1, w) remain (only when bw == 32)
    const int rg = tid >> 4, cg = tid & 15;
    for (int cc = c1 + 4 * cg; cc < w; cc += 64) {
      T acc[RT][4];
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = T(0);
#pragma unroll 8
      for (int k = 0; k < 32; ++k) {
        T ub[4], xa[RT];
        load4s<T>(&Us[k * wu + cc], ub);  // columns past w are never stored
#pragma unroll
        for (int i = 0; i < RT; ++i) xa[i] = Xs[(RT * rg + i) * wx + c0 + k];
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int q = 0; q < 4; ++q) acc[i][q] = fma(xa[i], ub[q], acc[i][q]);
      }
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (cc + q < w) Xs[(RT * rg + i) * wx + cc + q] -= acc[i][q];
    }
  }
  __syncthreads();
  for (int r = warp; r < rows; r += LS_THREADS / 32)
    for (int c = lane; c < w; c += 32) X[(int64_t)(r0 + r) * ld + c] = Xs[r * wx + c];
  if (spec && __syncthreads_or(bad) && tid == 0) sp.flag[3] = kabs + 1;
}

template <typename T>
static SpecDev<T> spec_dev(const SpecArgs& a, int64_t backup_offset) {
  SpecDev<T> d;
  d.flag = a.flag;
  d.backup = a.backup ? reinterpret_cast<T*>(a.backup) + backup_offset : nullptr;
  d.ipiv = a.ipiv;
  d.perm = a.perm;
  return d;
}

template <typename T>
cudaError_t launch_diag_lu(T* D, int64_t ld, int w, int kabs, int* info, cudaStream_t st, const SpecArgs& spec) {
  if (w <= 0) return cudaSuccess;
  const int wp = (w + 3) & ~3;
  const size_t smem = ((size_t)NP_NB * wp + (size_t)NP_NB * NP_CW) * sizeof(T);
  auto kern = diag_lu_kernel<T>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<1, np_threads<T>(), smem, st>>>(D, ld, w, kabs, info, spec_dev<T>(spec, 0));
  return cudaGetLastError();
}

static size_t ls_smem(int rb, int w, int tsize) {
  const size_t wu = (size_t)((w + 3) & ~3);
  return (32 * wu + wu + (size_t)rb * (w | 1)) * tsize;
}

template <typename T, int RB>
static cudaError_t launch_ls(const T* U, T* X, int64_t ld, int m, int w, int kabs, const SpecDev<T>& sp,
                             cudaStream_t st) {
  auto kern = trsm_right_upper_kernel<T, RB>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)cdiv(m, RB), LS_THREADS, ls_smem(RB, w, sizeof(T)), st>>>(U, X, ld, m, w, kabs, sp);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trsm_right_upper(const T* U, T* X, int64_t ld, int m, int w, cudaStream_t st,
                                    const SpecArgs& spec, int kabs) {
  if (m <= 0 || w <= 0) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // the rows below the panel's w x w block follow it in the backup
  const SpecDev<T> sp = spec_dev<T>(spec, (int64_t)w * w);
  if (ls_smem(64, w, sizeof(T)) <= (size_t)optin) return launch_ls<T, 64>(U, X, ld, m, w, kabs, sp, st);
  if (ls_smem(32, w, sizeof(T)) <= (size_t)optin) return launch_ls<T, 32>(U, X, ld, m, w, kabs, sp, st);
  if (ls_smem(16, w, sizeof(T)) <= (size_t)optin) return launch_ls<T, 16>(U, X, ld, m, w, kabs, sp, st);
  return cudaErrorInvalidValue;
}

template cudaError_t launch_diag_lu<double>(double*, int64_t, int, int, int*, cudaStream_t, const SpecArgs&);
template cudaError_t launch_diag_lu<float>(float*, int64_t, int, int, int*, cudaStream_t, const SpecArgs&);
template cudaError_t launch_trsm_right_upper<double>(const double*, double*, int64_t, int, int, cudaStream_t,
                                                     const SpecArgs&, int);
template cudaError_t launch_trsm_right_upper<float>(const float*, float*, int64_t, int, int, cudaStream_t,
                                                    const SpecArgs&, int);

}  // namespace gb
