// Bounded-wait probe: runs each kind of device wait the library uses on a
// condition that nothing ever satisfies, so that the failure path (the limit
// runs out, the kernel raises ST_TIMEOUT and returns, the host reports
// LU_ETIMEOUT and the context stays usable) can be tested without faulting or
// hanging the GPU.  The waits are the library's own helpers with their
// compiled-in limit.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace gb {

__global__ void wait_probe_kernel(int kind, int* flag, unsigned* counter, int* status) {
  __shared__ int smem_flag;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int abort_flag;
  if (kind == 0) {
    // a solve's wait for a block that is never published
    if (threadIdx.x == 0) wait_flag_eq(flag, 1, status);
  } else if (kind == 1) {
    // a panel's grid barrier that the other (absent) CTA never reaches
    grid_sync_mono(counter, 2u, status, &smem_flag);
  } else {
    // a tensor-core kernel's mbarrier wait for a copy or MMA that never arrives
    if (threadIdx.x == 0) {
      abort_flag = 0;
      mbar_init(smem_u32(&bar), 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      mbar_wait(smem_u32(&bar), 0u, status, (volatile int*)&abort_flag);
    }
  }
}

cudaError_t launch_wait_probe(int kind, void* scratch, int* status, cudaStream_t st) {
  int* flag = reinterpret_cast<int*>(scratch);
  unsigned* counter = reinterpret_cast<unsigned*>(flag + 1);
  cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(int), st);
  if (e != cudaSuccess) return e;
  wait_probe_kernel<<<1, 32, 0, st>>>(kind, flag, counter, status);
  return cudaGetLastError();
}

}  // namespace gb
