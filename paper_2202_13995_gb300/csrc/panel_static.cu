// Panel factorization for callers that cannot allocate device memory.
//
// lu_step_panel obtains the panel kernel's global scratch (the candidate
// exchange buffers, the grid barrier and the permutation record) with
// cudaMalloc on first use.  Some callers must not allocate at that point: code
// running while another thread captures a CUDA graph in global capture mode
// (where cudaMalloc is an error), and services that reserve all of their
// device memory up front and forbid any later allocation.  For them,
// lu_step_panel_static runs the same kernel with its scratch in the fixed
// array below, which lives in device memory from the moment the library is
// loaded until the process exits (on every GPU that loads the library).
#include <climits>
#include <mutex>

#include "lu_steps.h"
#include "common.cuh"
#include "kernels.h"

namespace {

// CTAs of one cooperative panel launch: the panel kernel's own limit (every
// CTA's candidate row must fit the exchange buffer); a device with more SMs
// runs the panel on this many of them.
constexpr int kStaticGmax = gb::kPanelMaxCtas;
constexpr int kStaticIb = 32;
constexpr int kStaticWmax = 512;   // widest panel accepted
// the scratch of the largest launch (FP64, widest panel), with room for the
// 256-byte alignment of its parts
constexpr size_t kStaticBytes = gb::panel_scratch_bytes(kStaticGmax, kStaticIb, kStaticWmax, 8) + 1024;

__device__ __align__(256) static unsigned char g_panel_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};
gb::DevInfo g_dev[kMaxDevices] = {};

// Per-device set-up, done by the first call on each device with that device
// current: the device address of the scratch array (host code only sees a
// host-side stand-in of its name) and the device's SM count.
int setup_device(int dev, void** addr, gb::DevInfo* info) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_addr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_panel_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return LU_ECUDA;
    }
    gb::DevInfo d{};
    if (cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return LU_ECUDA;
    }
    g_dev[dev] = d;
    g_addr[dev] = p;
  }
  *addr = g_addr[dev];
  *info = g_dev[dev];
  return LU_OK;
}

__global__ void finalize_info_kernel(int* info) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *info == 0x7f7f7f7f) *info = 0;
}

}  // namespace

extern "C" int lu_step_panel_static(void* cuda_stream, lu_prec prec, int m, int w, void* dP, int ld, int* dIpiv,
                                    int* dInfo, int* dStatus) {
  if (prec < LU_F64 || prec > LU_F32) return -2;
  if (m < 1) return -3;
  if (w < 1 || w > m || w > kStaticWmax) return -4;
  if (!dP) return -5;
  if (ld < w) return -6;
  if (!dIpiv) return -7;
  if (!dInfo) return -8;
  if (!dStatus) return -9;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return LU_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return LU_EINTERNAL;
  void* base = nullptr;
  gb::DevInfo info{};
  int rc = setup_device(dev, &base, &info);
  if (rc) return rc;
  const int tsize = prec == LU_F64 ? 8 : 4;
  const int gmax = info.sm_count < kStaticGmax ? info.sm_count : kStaticGmax;
  if (gb::panel_scratch_bytes(gmax, kStaticIb, w, tsize) > kStaticBytes) return LU_EINTERNAL;
  // a panel too tall for the CTAs' shared memory is refused here, before
  // anything is enqueued (dStatus and dInfo are left untouched)
  if (gb::panel_grid_size(m, w, tsize, info, gmax) <= 0) return -3;
  gb::PanelScratch ps;
  gb::panel_scratch_carve(&ps, base, gmax, kStaticIb, w, tsize);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (cudaMemsetAsync(dStatus, 0, sizeof(int), st) != cudaSuccess) return LU_ECUDA;
  if (cudaMemsetAsync(dInfo, 0x7f, sizeof(int), st) != cudaSuccess) return LU_ECUDA;
  cudaError_t e;
  if (prec == LU_F64)
    e = gb::launch_panel<double>((double*)dP, ld, m, w, 0, dIpiv, dInfo, dStatus, ps, info, st);
  else
    e = gb::launch_panel<float>((float*)dP, ld, m, w, 0, dIpiv, dInfo, dStatus, ps, info, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorCooperativeLaunchTooLarge ? -3 : LU_ECUDA;
  }
  finalize_info_kernel<<<1, 32, 0, st>>>(dInfo);
  if (cudaGetLastError() != cudaSuccess) return LU_ECUDA;
  return LU_OK;
}
