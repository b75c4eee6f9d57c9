// Device helpers shared by the kernels of the LU library: status bits, bounded
// waits on %globaltimer, and a grid barrier for cooperative launches.
//
// Every spin in this library is bounded: a wait that runs past its limit sets
// ST_TIMEOUT in the caller's device status word and returns false, and the
// kernel then leaves without touching the data any further.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gb {

// device status bits (OR-ed into a status word that the host reads)
enum StatusBits : int {
  ST_TIMEOUT = 1,   // a bounded device wait hit its limit
  ST_RANGE = 2,     // a cast to a 16-bit format overflowed, or a NaN was met
  ST_BADARG = 4,    // a kernel was given a size it cannot handle
  ST_BOUNDS = 8,    // an index guard of the bounds-checking build fired
};

// Index guards.  The bounds-checking build (-DLU_BOUNDS_CHECK) tests `cond`,
// records ST_BOUNDS and lets the caller take a safe path when it fails; the
// normal build compiles the guard away.
#ifdef LU_BOUNDS_CHECK
#define GB_IN_BOUNDS(status, cond) ((cond) ? true : (atomicOr((status), ST_BOUNDS), false))
#else
#define GB_IN_BOUNDS(status, cond) true
#endif

// limit of every device spin (nanoseconds of %globaltimer)
#ifndef GB_SPIN_LIMIT_NS
#define GB_SPIN_LIMIT_NS 2000000000ull
#endif

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_s32(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *flag == want (acquire).  Called by one thread.  Returns false
// (and sets ST_TIMEOUT) if the limit runs out first.
__device__ __forceinline__ bool wait_flag_eq(const int* flag, int want, int* status) {
  if (ld_acquire_s32(flag) == want) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    for (int i = 0; i < 64; ++i) {
      if (ld_acquire_s32(flag) == want) return true;
    }
    if (gtimer() - t0 > GB_SPIN_LIMIT_NS) {
      atomicOr(status, ST_TIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// bar[0] = arrival count, bar[1] = generation.  The host zeroes both before
// the launch.  Returns false in every thread of the CTA if the wait timed out.
struct GridBarrier {
  unsigned* bar;
  unsigned nblocks;
};

__device__ __forceinline__ bool grid_sync(const GridBarrier& gbar, int* status, int* smem_flag) {
  __syncthreads();
  if (gbar.nblocks > 1) {
    if (threadIdx.x == 0) {
      int ok = 1;
      unsigned gen = ld_acquire_u32(gbar.bar + 1);
      __threadfence();
      unsigned arrived = atomicAdd(gbar.bar, 1u);
      if (arrived == gbar.nblocks - 1) {
        atomicExch(gbar.bar, 0u);
        __threadfence();
        st_release_u32(gbar.bar + 1, gen + 1);
      } else {
        const uint64_t t0 = gtimer();
        while (ld_acquire_u32(gbar.bar + 1) == gen) {
          if (gtimer() - t0 > GB_SPIN_LIMIT_NS) {
            atomicOr(status, ST_TIMEOUT);
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
      *smem_flag = ok;
    }
    __syncthreads();
    return *smem_flag != 0;
  }
  return true;
}

// (|v|, index) pair reduction used by the pivot search: larger |v| wins, and on
// equal |v| the smaller row index wins (the first row of largest magnitude).
template <typename T>
__device__ __forceinline__ void argmax_merge(T& v, int& i, T v2, int i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

// Pivot-search magnitude |x|, with NaN as +infinity: a NaN entry is then
// chosen as a pivot (and the non-finite pivot reported) instead of never
// comparing and leaving a column without a candidate row.
template <typename T>
__device__ __forceinline__ T pivot_mag(T x) {
  const T a = x < T(0) ? -x : x;
  return a == a ? a : T(INFINITY);
}

// FP64 specialisations on the bit patterns: GB300 runs FP64 instructions,
// comparisons included, at two per clock per SM, while a pivot search
// compares magnitudes only.  A magnitude (non-negative, +inf for NaN) and the
// "no candidate" value -1 order as their bit patterns read as signed 64-bit
// integers, so the integer pipe gives the same answer.
template <>
__device__ __forceinline__ void argmax_merge<double>(double& v, int& i, double v2, int i2) {
  const long long a = __double_as_longlong(v), b = __double_as_longlong(v2);
  if (b > a || (b == a && i2 < i)) {
    v = v2;
    i = i2;
  }
}

template <>
__device__ __forceinline__ double pivot_mag<double>(double x) {
  const unsigned long long m = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  return __longlong_as_double((long long)(m > 0x7ff0000000000000ull ? 0x7ff0000000000000ull : m));
}

// x != 0 (either sign of zero); the FP64 form tests the bits on the integer pipe.
__device__ __forceinline__ bool nonzero(float x) { return x != 0.0f; }
__device__ __forceinline__ bool nonzero(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) != 0ull;
}

// A pivot-search magnitude that is +inf (a non-finite entry).
__device__ __forceinline__ bool is_inf_mag(float v) { return !(v < INFINITY); }
__device__ __forceinline__ bool is_inf_mag(double v) {
  return (unsigned long long)__double_as_longlong(v) == 0x7ff0000000000000ull;
}

template <typename T>
__device__ __forceinline__ void warp_argmax(T& v, int& i) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    T v2 = __shfl_xor_sync(0xffffffffu, v, off);
    int i2 = __shfl_xor_sync(0xffffffffu, i, off);
    argmax_merge(v, i, v2, i2);
  }
}

__host__ __device__ __forceinline__ int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

// ---- asynchronous global -> shared copies (cp.async), 4, 8 or 16 bytes
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async sizes");
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(smem)), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// close the copies issued so far into a group; wait until at most N groups are pending
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---- thread-block clusters: rank, peer shared-memory addresses, barrier
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// the address of this CTA's shared variable at `addr` in the CTA of rank `rank`
__device__ __forceinline__ uint32_t cluster_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ float cluster_ld(uint32_t addr, float) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ double cluster_ld(uint32_t addr, double) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}
// the hardware cluster barrier, release / acquire at cluster scope: every
// CTA's prior shared and global writes are visible to every peer after it
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Grid barrier on a monotonic arrival counter (zeroed by the launcher): the
// k-th barrier waits until the counter reaches k * G.  Arrival is a release
// reduction, so a CTA never waits on its own arrival round trip.
__device__ __forceinline__ bool grid_sync_mono(unsigned* count, unsigned target, int* status, int* smem_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(count) : "memory");
    int ok = 1;
    if (ld_acquire_u32(count) < target) {
      const uint64_t t0 = gtimer();
      while (ld_acquire_u32(count) < target) {
        if (gtimer() - t0 > GB_SPIN_LIMIT_NS) {
          atomicOr(status, ST_TIMEOUT);
          ok = 0;
          break;
        }
      }
    }
    *smem_flag = ok;
  }
  __syncthreads();
  return *smem_flag != 0;
}

}  // namespace gb
