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

// In-place LU (no pivoting) of the w x w block at D (row-major, ld), blocked by
// 32 columns; one CTA of np_threads<T>() threads.  Lowers *info to kabs + j + 1 at the
// first exactly zero pivot j (and skips that column's scaling).
template <typename T>
__global__ void __launch_bounds__(np_threads<T>()) diag_lu_kernel(T* D, int64_t ld, int w, int kabs, int* info) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wp = (w + 3) & ~3;
  T* P = reinterpret_cast<T*>(smem_raw);  // [NP_NB][wp]: column c of the sub-panel, row r
  T* Us = P + (size_t)NP_NB * wp;         // [NP_NB][NP_CW]
  const int tid = threadIdx.x;
  constexpr int NP_NT = np_threads<T>();
  constexpr int CH = 16 / sizeof(T);  // elements per 16-byte access
  const bool vec = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && (ld % CH) == 0;
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
      if (tid == 0 && piv == T(0)) atomicMin(info, kabs + k0 + j + 1);
      for (int r = j + 1 + tid; r < m; r += NP_NT) {
        T l = P[j * wp + r];
        if (piv != T(0)) l = l / piv;
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
}

// X (m x w, row-major, ld) <- X U^-1 with U the upper (non-unit) w x w block at
// U (row-major, ld): the paper's "left" block update.  CTA = 32 rows of X in
// shared memory; by 32-column blocks: warps solve their rows against the
// diagonal block (division by the pivot, as in the definition), then all
// threads update the columns to the right.
template <typename T>
__global__ void __launch_bounds__(256) trsm_right_upper_kernel(const T* __restrict__ U, T* X, int64_t ld, int m,
                                                               int w) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int wp = w + 1;
  T* Xs = reinterpret_cast<T*>(smem_raw);  // [32][wp]
  T* Ud = Xs + 32 * wp;                    // [32][33] diagonal block
  T* Ub = Ud + 32 * 33;                    // [32][w] U rows b0.. b0+32, columns right of the block
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int r0 = blockIdx.x * 32;
  const int rows = min(32, m - r0);
  for (int e = threadIdx.x; e < 32 * w; e += 256) {
    const int r = e / w, c = e % w;
    Xs[r * wp + c] = r < rows ? X[(int64_t)(r0 + r) * ld + c] : T(0);
  }
  for (int b0 = 0; b0 < w; b0 += 32) {
    const int bw = min(32, w - b0);
    const int c1 = b0 + bw, nr = w - c1;
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int s = e >> 5, t = e & 31;
      Ud[s * 33 + t] = (s < bw && t < bw) ? U[(int64_t)(b0 + s) * ld + b0 + t] : T(0);
    }
    for (int e = threadIdx.x; e < bw * nr; e += 256) {
      const int s = e / nr, c = e % nr;
      Ub[s * w + c] = U[(int64_t)(b0 + s) * ld + c1 + c];
    }
    __syncthreads();
    for (int r = warp; r < 32; r += 8) {
      T x = lane < bw ? Xs[r * wp + b0 + lane] : T(0);
      for (int s = 0; s < bw; ++s) {
        if (lane == s) x = x / Ud[s * 33 + s];
        const T xs = __shfl_sync(0xffffffffu, x, s);
        if (lane > s && lane < bw) x -= xs * Ud[s * 33 + lane];
      }
      if (lane < bw) Xs[r * wp + b0 + lane] = x;
    }
    __syncthreads();
    // columns right of the block: X[r][c] -= sum_s X[r][b0 + s] U[b0 + s][c]
    for (int e = threadIdx.x; e < 32 * nr; e += 256) {
      const int r = e / nr, c = e % nr;
      T acc = Xs[r * wp + c1 + c];
      for (int s = 0; s < bw; ++s) acc -= Xs[r * wp + b0 + s] * Ub[s * w + c];
      Xs[r * wp + c1 + c] = acc;
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < 32 * w; e += 256) {
    const int r = e / w, c = e % w;
    if (r < rows) X[(int64_t)(r0 + r) * ld + c] = Xs[r * wp + c];
  }
}

template <typename T>
cudaError_t launch_diag_lu(T* D, int64_t ld, int w, int kabs, int* info, cudaStream_t st) {
  if (w <= 0) return cudaSuccess;
  const int wp = (w + 3) & ~3;
  const size_t smem = ((size_t)NP_NB * wp + (size_t)NP_NB * NP_CW) * sizeof(T);
  auto kern = diag_lu_kernel<T>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<1, np_threads<T>(), smem, st>>>(D, ld, w, kabs, info);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trsm_right_upper(const T* U, T* X, int64_t ld, int m, int w, cudaStream_t st) {
  if (m <= 0 || w <= 0) return cudaSuccess;
  const size_t smem = ((size_t)32 * (w + 1) + 32 * 33 + (size_t)32 * w) * sizeof(T);
  auto kern = trsm_right_upper_kernel<T>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)cdiv(m, 32), 256, smem, st>>>(U, X, ld, m, w);
  return cudaGetLastError();
}

template cudaError_t launch_diag_lu<double>(double*, int64_t, int, int, int*, cudaStream_t);
template cudaError_t launch_diag_lu<float>(float*, int64_t, int, int, int*, cudaStream_t);
template cudaError_t launch_trsm_right_upper<double>(const double*, double*, int64_t, int, int, cudaStream_t);
template cudaError_t launch_trsm_right_upper<float>(const float*, float*, int64_t, int, int, cudaStream_t);

}  // namespace gb
