// Trailing update on the CUDA cores: C -= A * B (row-major), FP64 (DFMA) or FP32.
//
// This is the paper's "inner" block update (arxiv 2202.13995, section "Base
// Implementation": the inner blocks are updated by matrix multiplication of
// the left and top blocks), A22 <- A22 - L21 * U12.  On GB300 the FP64 rate is
// a small fraction of the FP32 rate and tcgen05 has no FP64 kind, so the FP64
// path is bound by DFMA issue: a 64 x 64 CTA tile with a 4 x 4 register tile
// per thread keeps the FP64 pipes fed from shared memory with ample slack.
#include "common.cuh"
#include "kernels.h"

namespace gb {

constexpr int SG_BM = 64, SG_BN = 64, SG_BK = 16;

template <typename T>
__global__ void __launch_bounds__(256) gemm_simt_kernel(T* __restrict__ C, int64_t ldc, const T* __restrict__ A,
                                                        int64_t lda, const T* __restrict__ B, int64_t ldb, int m,
                                                        int n, int k) {
  __shared__ T As[2][SG_BK][SG_BM];
  __shared__ T Bs[2][SG_BK][SG_BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * SG_BM, n0 = blockIdx.x * SG_BN;

  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  T ra[4], rb[4];
  auto load_regs = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      const int ar = e >> 4, ak = e & 15;
      const int gr = m0 + ar, gk = k0 + ak;
      ra[q] = (gr < m && gk < k) ? A[(int64_t)gr * lda + gk] : T(0);
      const int bk = e >> 6, bc = e & 63;
      const int gbk = k0 + bk, gc = n0 + bc;
      rb[q] = (gbk < k && gc < n) ? B[(int64_t)gbk * ldb + gc] : T(0);
    }
  };
  auto store_smem = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = tid + 256 * q;
      As[buf][e & 15][e >> 4] = ra[q];
      Bs[buf][e >> 6][e & 63] = rb[q];
    }
  };

  const int nk = (k + SG_BK - 1) / SG_BK;
  load_regs(0);
  store_smem(0);
  __syncthreads();
  for (int t = 0; t < nk; ++t) {
    const int buf = t & 1;
    if (t + 1 < nk) load_regs((t + 1) * SG_BK);
#pragma unroll
    for (int kk = 0; kk < SG_BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (t + 1 < nk) {
      store_smem(buf ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty + 16 * i;
    if (r >= m) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx + 16 * j;
      if (c < n) C[(int64_t)r * ldc + c] -= acc[i][j];
    }
  }
}

template <typename T>
cudaError_t launch_gemm_simt(T* C, int64_t ldc, const T* A, int64_t lda, const T* B, int64_t ldb, int m, int n,
                             int k, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  dim3 grid((unsigned)cdiv(n, SG_BN), (unsigned)cdiv(m, SG_BM));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  gemm_simt_kernel<T><<<grid, 256, 0, st>>>(C, ldc, A, lda, B, ldb, m, n, k);
  return cudaGetLastError();
}

template cudaError_t launch_gemm_simt<double>(double*, int64_t, const double*, int64_t, const double*, int64_t, int,
                                              int, int, cudaStream_t);
template cudaError_t launch_gemm_simt<float>(float*, int64_t, const float*, int64_t, const float*, int64_t, int, int,
                                             int, cudaStream_t);

}  // namespace gb
