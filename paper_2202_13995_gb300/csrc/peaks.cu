// Arithmetic-rate probes of the device: the denominators of the roofline
// fractions of the FP64 and FP32 CUDA-core kernels (the FP64 trailing update,
// the batched FP32 factor).  Each kernel keeps every lane busy with eight
// independent chains of one operation and no memory traffic; the rate is the
// operation count over the CUDA-event time of the launch.
#include <cuda_runtime.h>

#include "lu_steps.h"
#include "common.cuh"

namespace {

constexpr int PK_THREADS = 256;

__global__ void __launch_bounds__(PK_THREADS) dfma_kernel(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = b + (double)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 12345.678) out[0] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(PK_THREADS) ffma_kernel(float* out, int iters, float a, float b) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = b + (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  if (s == 12345.678f) out[0] = s;
}

// FP64 warp-level matrix multiply-accumulate (m8n8k4, the FP64 tensor-core
// instruction of the mma.sync family): four independent accumulators per warp
__global__ void __launch_bounds__(PK_THREADS) dmma_kernel(double* out, int iters, double a, double b) {
  const double av = a + 1e-3 * (threadIdx.x & 31), bv = b - 1e-3 * (threadIdx.x & 31);
  double c[4][2];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i][0] = c[i][1] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};"
                   : "+d"(c[i][0]), "+d"(c[i][1])
                   : "d"(av), "d"(bv));
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) s += c[i][0] + c[i][1];
  if (s == 12345.678) out[0] = s;
}

}  // namespace

extern "C" int lu_peak_probe(int kind, double* tflops) {
  if (kind < 0 || kind > 2) return -1;
  if (!tflops) return -2;
  *tflops = 0.0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LU_ECUDA;
  double* buf = nullptr;
  if (cudaMalloc(&buf, 64) != cudaSuccess) return LU_ENOMEM;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = LU_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = LU_ECUDA;
  const int grid = sms * 8;  // eight CTAs of 256 threads per SM: every scheduler has warps to pick
  // operations per launch: kind 0 / 2: 2 flops x 8 chains x iters per thread;
  // kind 1: 512 flops per mma (2 x 8 x 8 x 4) x 4 per iteration per warp
  // about 150 ms per launch, long enough for the clocks to settle
  const int iters = kind == 2 ? 1 << 21 : (kind == 1 ? 1 << 13 : 1 << 15);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && rc == LU_OK; ++rep) {
    cudaEventRecord(e0, st);
    if (kind == 0)
      dfma_kernel<<<grid, PK_THREADS, 0, st>>>(buf, iters, 0.999999, 1e-6);
    else if (kind == 1)
      dmma_kernel<<<grid, PK_THREADS, 0, st>>>(buf, iters, 0.5, 0.25);
    else
      ffma_kernel<<<grid, PK_THREADS, 0, (cudaStream_t)st>>>((float*)buf, iters, 0.999999f, 1e-6f);
    cudaEventRecord(e1, st);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      rc = LU_ECUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // the first launch warms up
  }
  if (rc == LU_OK) {
    const double threads = (double)grid * PK_THREADS;
    const double flops = kind == 1 ? (threads / 32.0) * 4.0 * 512.0 * iters : threads * 8.0 * 2.0 * iters;
    *tflops = flops / (best * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(buf);
  return rc;
}
