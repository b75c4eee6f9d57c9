// Seeded synthetic inputs on the device: the HPL-shaped matrices and
// right-hand sides of the benchmarks, generated where they are used.
//
// The HPL benchmark generates its own input (arxiv 2202.13995, section "High
// Performance Linpack": the matrix is generated, the solution known); here
// every entry is a pure function of (seed, stream, index): SplitMix64
// (Steele, Lea, Flood, OOPSLA 2014) in counter mode, the k-th draw of a stream
// being mix64(state0 + (k + 1) * GAMMA) with state0 = mix64(seed XOR stream *
// STREAM_MULT), mapped to (z >> 11) * 2^-53 - 0.5, a uniform value in
// [-0.5, 0.5) that is exact in FP64.  The host forms of the same draws (numpy
// and torch, in the Python package) give the same bits.
#include <cuda_runtime.h>
#include <stdint.h>

#include "lu_steps.h"
#include "common.cuh"

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kMix1 = 0xBF58476D1CE4E5B9ull;
constexpr uint64_t kMix2 = 0x94D049BB133111EBull;
constexpr uint64_t kStreamMult = 0xD1B54A32D192ED03ull;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * kMix1;
  z = (z ^ (z >> 27)) * kMix2;
  return z ^ (z >> 31);
}

// element (i, j) of the rows x cols column-major block at A (ld) is draw
// i + j * rows of the stream, plus `shift` where i == j
__global__ void generate_kernel(double* A, int64_t ld, int rows, int cols, uint64_t s0, double shift) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = k / rows, i = k - j * rows;
    const uint64_t z = mix64(s0 + (uint64_t)(k + 1) * kGamma);
    double v = (double)(z >> 11) * 0x1.0p-53 - 0.5;
    if (i == j) v += shift;
    A[i + j * ld] = v;
  }
}

}  // namespace

extern "C" int lu_generate(double* dA, int rows, int cols, int ld, uint64_t seed, int stream_id, double diag_shift,
                           void* cuda_stream) {
  if (rows < 0) return -2;
  if (cols < 0) return -3;
  if (ld < (rows > 1 ? rows : 1)) return -4;
  if (!dA && rows > 0 && cols > 0) return -1;
  if (rows == 0 || cols == 0) return LU_OK;
  const uint64_t s0 = mix64(seed ^ ((uint64_t)stream_id * kStreamMult));
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t total = (int64_t)rows * cols;
  const int64_t want = gb::cdiv(total, 256);
  const int grid = (int)(want < (int64_t)sms * 16 ? want : (int64_t)sms * 16);
  generate_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(dA, ld, rows, cols, s0, diag_shift);
  return cudaGetLastError() == cudaSuccess ? LU_OK : LU_ECUDA;
}
