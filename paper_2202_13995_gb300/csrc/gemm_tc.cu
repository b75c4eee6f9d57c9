// Tensor-core trailing update for the mixed-precision factorization:
//   C (FP32, row-major) -= Aop * Bop^T,  Aop = L21 and Bop = U12^T in BF16 or
//   FP16 (K-major), products accumulated in FP32.
//
// This is the paper's "inner" block update by matrix multiplication (arxiv
// 2202.13995, section "Base Implementation"; the paper's own design unrolls a
// register-blocked GEMM in FPGA DSPs), here on the 5th-generation tensor cores:
//   - warp 0 (one thread) streams K-chunks of 64 elements of both operands
//     into a 2-stage shared-memory ring with TMA (128-byte swizzle);
//   - warp 1 (one thread) issues tcgen05.mma (M=128, N=256, K=16) into one of
//     two TMEM accumulators (2 x 256 columns), committing each stage back to
//     the producer and each finished tile to the epilogue;
//   - warps 2..9 drain a finished accumulator with tcgen05.ld while the next
//     tile accumulates in the other one, and subtract it from C in place.
//     C moves through shared memory in 32 x 32 chunks: each epilogue warp
//     keeps four chunk buffers and loads C (cp.async, row-contiguous
//     16-byte pieces, four full 128-byte lines per warp instruction) three
//     chunks ahead of the one it drains.  TMEM hands each thread one row: the
//     thread subtracts its row in shared memory, and the warp writes the chunk
//     back row-contiguously.  The CTA's next tile is also prefetched into L2.
// Persistent CTAs (one per SM) walk the output tiles.  Every mbarrier wait is
// bounded; on timeout the kernel raises ST_TIMEOUT, lets its TMA loads and
// MMAs land, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <mutex>

#include "cast16.cuh"
#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace gb {

constexpr int TC_BM = 128;
constexpr int TC_BN = 256;
constexpr int TC_BK = 64;  // one 128-byte swizzle row of 16-bit elements
constexpr int TC_STAGES = 2;  // 96 KB ring: the MMAs of a tile take a fraction of its epilogue
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;  // 16 KB
constexpr int TC_B_BYTES = TC_BN * TC_BK * 2;  // 32 KB
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_THREADS = 32 * (2 + TC_EPI_WARPS);
constexpr int TC_TMEM_COLS = 512;
constexpr int TC_CHUNK_BYTES = 32 * 32 * 4;  // 32 rows x 32 columns of FP32 C
constexpr int TC_CBUF = 4;                    // chunk buffers per epilogue warp (3 loads ahead)
constexpr int TC_STG_BYTES = TC_CBUF * TC_CHUNK_BYTES;
constexpr size_t TC_SMEM = 1024 + (size_t)TC_STAGES * (TC_A_BYTES + TC_B_BYTES) + TC_EPI_WARPS * TC_STG_BYTES + 256;
static_assert(TC_SMEM <= 232448, "tc_gemm_kernel shared memory");

// ------------------------------------------------------------ kernel
struct TcParams {
  float* C;
  int64_t ldc;
  int m, n, kchunks;
  int tiles_m, tiles_n;
  int vec_ok;  // C rows 16-byte aligned
  uint32_t idesc;
  int* status;
};

__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcParams P) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t sA = base;
  const uint32_t sB = base + TC_STAGES * TC_A_BYTES;
  float4* stg_all = reinterpret_cast<float4*>(gbase + TC_STAGES * (TC_A_BYTES + TC_B_BYTES));
  unsigned char* ctl = gbase + TC_STAGES * (TC_A_BYTES + TC_B_BYTES) + TC_EPI_WARPS * TC_STG_BYTES;
  const uint32_t bar_full = smem_u32(ctl);
  const uint32_t bar_empty = bar_full + 8 * TC_STAGES;
  const uint32_t bar_tfull = bar_empty + 8 * TC_STAGES;
  const uint32_t bar_tempty = bar_tfull + 16;
  const uint32_t bar_drain = bar_tempty + 16;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctl + 8 * (2 * TC_STAGES + 5));
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctl + 8 * (2 * TC_STAGES + 5) + 8);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = P.tiles_m * P.tiles_n;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(bar_full + 8 * s, 1);
      mbar_init(bar_empty + 8 * s, 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(bar_tfull + 8 * a, 1);
      mbar_init(bar_tempty + 8 * a, TC_EPI_WARPS);
    }
    mbar_init(bar_drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int last_par[TC_STAGES];
#pragma unroll
      for (int s = 0; s < TC_STAGES; ++s) last_par[s] = -1;
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int tm = t % P.tiles_m, tn = t / P.tiles_m;
        for (int kc = 0; kc < P.kchunks; ++kc) {
          if (!mbar_wait(bar_empty + 8 * s, ph ^ 1u, P.status, abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(bar_full + 8 * s, TC_A_BYTES + TC_B_BYTES);
          tma_load_2d(sA + s * TC_A_BYTES, &tmA, kc * TC_BK, tm * TC_BM, bar_full + 8 * s);
          tma_load_2d(sB + s * TC_B_BYTES, &tmB, kc * TC_BK, tn * TC_BN, bar_full + 8 * s);
          last_par[s] = (int)ph;
          if (++s == TC_STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (!ok) {
        // let every issued copy land before the CTA can exit
        for (int q = 0; q < TC_STAGES; ++q) {
          if (last_par[q] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try(bar_full + 8 * q, (uint32_t)last_par[q]) && gtimer() - t0 < GB_SPIN_LIMIT_NS) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int acc = 0;
      uint32_t aph = 0;
      bool ok = true;
      bool issued = false;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        if (!mbar_wait(bar_tempty + 8 * acc, aph ^ 1u, P.status, abort_flag)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dtm = tmem_base + (uint32_t)(acc * TC_BN);
        for (int kc = 0; kc < P.kchunks; ++kc) {
          if (!mbar_wait(bar_full + 8 * s, ph, P.status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = sA + s * TC_A_BYTES, b0 = sB + s * TC_B_BYTES;
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk) {
            tc_mma(dtm, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), P.idesc, (kc | kk) ? 1u : 0u);
          }
          issued = true;
          tc_commit(bar_empty + 8 * s);
          if (++s == TC_STAGES) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(bar_tfull + 8 * acc);
        if (++acc == 2) {
          acc = 0;
          aph ^= 1u;
        }
      }
      if (!ok && issued) {
        // let the MMAs already issued finish before TMEM is freed
        tc_commit(bar_drain);
        const uint64_t t0 = gtimer();
        while (!mbar_try(bar_drain, 0) && gtimer() - t0 < GB_SPIN_LIMIT_NS) {
        }
      }
    }
  } else {
    // ---------------- epilogue: C -= accumulator
    const int q = warp & 3;              // TMEM lane quarter this warp may access
    const int half = (warp - 2) >> 2;    // which 128 columns of the tile
    const uint32_t cbuf = smem_u32(stg_all) + (uint32_t)((warp - 2) * TC_STG_BYTES);
    float4* const cbuf_p = stg_all + (warp - 2) * (TC_STG_BYTES / 16);
    // Coalesced view of a chunk: lane -> rows 4i + lane/8 (i < 8), 16-byte
    // unit lane%8.  In a buffer, (row r, unit u) sits at float4 r*8 +
    // (u ^ (r & 7)), so that the row-per-lane accesses and the coalesced ones
    // are both free of bank conflicts; (4i + lane/8) & 7 depends on i only
    // through its parity.
    const int rsub = lane >> 3, unit = lane & 7;
    const uint32_t coff0 = (uint32_t)(rsub * 8 + (unit ^ rsub)) * 16u;        // even i
    const uint32_t coff1 = (uint32_t)(rsub * 8 + (unit ^ (rsub + 4))) * 16u;  // odd i, less 512 B
    const int64_t ldc4 = 4 * P.ldc;
    // A lane's view of one tile: its first row and column, rows and columns left.
    struct View {
      float* p;
      int rows, cols;  // rows and columns of C from the lane's first ones on
      bool vec;        // C rows 16-byte aligned (else the element-wise path only)
    };
    auto view_of = [&](int t) -> View {
      View v;
      const int tm = t % P.tiles_m, tn = t / P.tiles_m;
      const int r0 = tm * TC_BM + q * 32 + rsub, c0 = tn * TC_BN + half * 128 + 4 * unit;
      v.p = P.C + (int64_t)r0 * P.ldc + c0;
      v.rows = P.m - r0;
      v.cols = P.n - c0;
      v.vec = P.vec_ok != 0;
      return v;
    };
    // cp.async of chunk cc of a tile (zero-filled where C is ragged: those
    // pieces are updated in global memory directly)
    auto load_chunk = [&](const View& v, int cc, int slot) {
      const bool full = v.vec && cc * 32 + 4 <= v.cols;
      const uint32_t b = cbuf + (uint32_t)(slot * TC_CHUNK_BYTES);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const bool ok = full && 4 * i < v.rows;
        const float* src = v.p + i * ldc4 + cc * 32;
        cpa16_zfill(b + (uint32_t)(i >> 1) * 1024u + ((i & 1) ? coff1 + 512u : coff0), ok ? (const void*)src
                                                                                         : (const void*)P.C,
                    ok ? 16u : 0u);
      }
    };
    // L2 prefetch of this thread's 128-column row segment of tile t
    auto prefetch_c = [&](int t) {
      if (t >= ntiles || !P.vec_ok) return;
      const int r = (t % P.tiles_m) * TC_BM + q * 32 + lane;
      const int c0 = (t / P.tiles_m) * TC_BN + half * 128;
      const int nc = min(128, P.n - c0);
      if (r >= P.m || nc < 4) return;
      l2_prefetch_bulk(P.C + (int64_t)r * P.ldc + c0, (uint32_t)(nc & ~3) * 4u);
    };
    // the load side runs TC_CBUF - 1 chunks ahead of the drain side
    int lt = blockIdx.x, lcc = 0, lslot = 0;
    View lv = view_of(lt < ntiles ? lt : 0);
    auto load_next = [&]() {
      if (lt < ntiles) load_chunk(lv, lcc, lslot);
      cpa_commit();  // one group per chunk, empty past the last one
      if (++lslot == TC_CBUF) lslot = 0;
      if (++lcc == 4) {
        lcc = 0;
        lt += gridDim.x;
        if (lt < ntiles) lv = view_of(lt);
      }
    };
    prefetch_c(blockIdx.x);
#pragma unroll 1
    for (int g = 0; g < TC_CBUF - 1; ++g) load_next();
    int acc = 0;
    uint32_t aph = 0;
    int slot = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      prefetch_c(t + gridDim.x);
      const View dv = view_of(t);
      int okw = 1;
      if (lane == 0) okw = mbar_wait(bar_tfull + 8 * acc, aph, P.status, abort_flag) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      tc_fence_after();
#pragma unroll 1
      for (int cc = 0; cc < 4; ++cc) {
        load_next();
        uint32_t v[32];
        const uint32_t taddr =
            tmem_base + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * TC_BN + half * 128 + cc * 32);
        TMEM_LD_X32(taddr, v);
        cpa_wait<TC_CBUF - 1>();  // this thread's pieces of the chunk have landed
        tmem_wait_ld();
        __syncwarp();  // ... and every other lane's
        float4* buf = cbuf_p + slot * (TC_CHUNK_BYTES / 16);
        // row `lane`: C -= accumulator in shared memory
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          float4* p = buf + lane * 8 + (u ^ (lane & 7));
          float4 c = *p;
          c.x -= __uint_as_float(v[4 * u + 0]);
          c.y -= __uint_as_float(v[4 * u + 1]);
          c.z -= __uint_as_float(v[4 * u + 2]);
          c.w -= __uint_as_float(v[4 * u + 3]);
          *p = c;
        }
        __syncwarp();
        const unsigned char* bb = reinterpret_cast<const unsigned char*>(buf);
        const bool full = dv.vec && cc * 32 + 4 <= dv.cols;
        if (full && dv.rows >= 29) {
          // whole chunk in range for this lane
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const float4 a = *reinterpret_cast<const float4*>(bb + (i >> 1) * 1024 + ((i & 1) ? coff1 + 512 : coff0));
            *reinterpret_cast<float4*>(dv.p + i * ldc4 + cc * 32) = a;
          }
        } else {
          const int gcols = dv.cols - cc * 32;
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            if (4 * i >= dv.rows) break;
            const float4 a = *reinterpret_cast<const float4*>(bb + (i >> 1) * 1024 + ((i & 1) ? coff1 + 512 : coff0));
            float* cp = dv.p + i * ldc4 + cc * 32;
            if (full) {
              *reinterpret_cast<float4*>(cp) = a;
            } else {
              // the buffer held zeros here: a = -accumulator, and C + a == C - accumulator
              if (0 < gcols) cp[0] += a.x;
              if (1 < gcols) cp[1] += a.y;
              if (2 < gcols) cp[2] += a.z;
              if (3 < gcols) cp[3] += a.w;
            }
          }
        }
        __syncwarp();  // the buffer is refilled by a later load
        if (++slot == TC_CBUF) slot = 0;
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_tempty + 8 * acc);
      if (++acc == 2) {
        acc = 0;
        aph ^= 1u;
      }
    }
    cpa_wait<0>();  // no copy may land after the CTA exits
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TC_TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ operand casts
// Aop[i*kpad + t] = L21(i, t), Bop[j*kpad + t] = U12(t, j), zero for t >= k.
template <typename H>
__global__ void cast_a_kernel(const float* __restrict__ L21, int64_t ld, int m, int k, H* __restrict__ Aop, int kpad,
                              int* status) {
  const int i = blockIdx.y;
  bool bad = false;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < kpad; t += gridDim.x * blockDim.x) {
    H h = to16<H>(t < k ? L21[(int64_t)i * ld + t] : 0.0f);
    bad |= bad16<H>(h);
    Aop[(int64_t)i * kpad + t] = h;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_RANGE);
}

template <typename H>
__global__ void cast_b_kernel(const float* __restrict__ U12, int64_t ld, int n, int k, H* __restrict__ Bop, int kpad,
                              int* status) {
  __shared__ float tile[32][33];
  const int j0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int t = t0 + r, j = j0 + tx;
    tile[r][tx] = (t < k && j < n) ? U12[(int64_t)t * ld + j] : 0.0f;
  }
  __syncthreads();
  bool bad = false;
  for (int r = ty; r < 32; r += 8) {
    const int j = j0 + r, t = t0 + tx;
    if (j < n && t < kpad) {
      H h = to16<H>(tile[tx][r]);
      bad |= bad16<H>(h);
      Bop[(int64_t)j * kpad + t] = h;
    }
  }
  if (__any_sync(0xffffffffu, bad) && tx == 0) atomicOr(status, ST_RANGE);
}

cudaError_t launch_cast_operands(int kind, const float* L21, const float* U12, int64_t ldw, int m, int n, int k,
                                 void* Aop, void* Bop, int kpad, int* status, cudaStream_t st) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  // the A cast runs one grid row per operand row
  if (m > 65535 || (kpad % 64) != 0 || k > kpad) return cudaErrorInvalidValue;
  dim3 ga((unsigned)cdiv(kpad, 256), (unsigned)m);
  dim3 gb_((unsigned)cdiv(n, 32), (unsigned)cdiv(kpad, 32));
  if (kind == 1) {
    cast_a_kernel<__nv_bfloat16><<<ga, 256, 0, st>>>(L21, ldw, m, k, (__nv_bfloat16*)Aop, kpad, status);
    cast_b_kernel<__nv_bfloat16><<<gb_, dim3(32, 8), 0, st>>>(U12, ldw, n, k, (__nv_bfloat16*)Bop, kpad, status);
  } else {
    cast_a_kernel<__half><<<ga, 256, 0, st>>>(L21, ldw, m, k, (__half*)Aop, kpad, status);
    cast_b_kernel<__half><<<gb_, dim3(32, 8), 0, st>>>(U12, ldw, n, k, (__half*)Bop, kpad, status);
  }
  return cudaGetLastError();
}

// The A operand alone, eight elements per thread: two 16-byte loads of L21
// and one 16-byte store of the operand (L21's rows 16-byte aligned, k a
// multiple of 8; launch_cast_a checks and otherwise uses cast_a_kernel).
template <typename H>
__global__ void cast_a8_kernel(const float* __restrict__ L21, int64_t ld, int m, int k, H* __restrict__ Aop, int kpad,
                               int* status) {
  const int per_row = kpad / 8;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool bad = false;
  if (e < (int64_t)m * per_row) {
    const int i = (int)(e / per_row), t = (int)(e % per_row) * 8;
    float v[8];
    if (t < k) {
      const float4 x0 = *reinterpret_cast<const float4*>(L21 + (int64_t)i * ld + t);
      const float4 x1 = *reinterpret_cast<const float4*>(L21 + (int64_t)i * ld + t + 4);
      v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
      v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = 0.0f;
    }
    unsigned w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const H lo = to16<H>(v[2 * u]), hi = to16<H>(v[2 * u + 1]);
      bad |= bad16<H>(lo) || bad16<H>(hi);
      w[u] = (unsigned)bits16<H>(lo) | ((unsigned)bits16<H>(hi) << 16);
    }
    *reinterpret_cast<uint4*>(Aop + (int64_t)i * kpad + t) = make_uint4(w[0], w[1], w[2], w[3]);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, ST_RANGE);
}

cudaError_t launch_cast_a(int kind, const float* L21, int64_t ldw, int m, int k, void* Aop, int kpad, int* status,
                          cudaStream_t st) {
  if (m <= 0) return cudaSuccess;
  if ((kpad % 64) != 0 || k > kpad) return cudaErrorInvalidValue;
  const bool vec = (k % 8) == 0 && ((uintptr_t)L21 & 15u) == 0 && (ldw % 4) == 0 && ((uintptr_t)Aop & 15u) == 0;
  if (vec) {
    const int64_t items = (int64_t)m * (kpad / 8);
    const unsigned grid = (unsigned)cdiv(items, 256);
    if (kind == 1)
      cast_a8_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(L21, ldw, m, k, (__nv_bfloat16*)Aop, kpad, status);
    else
      cast_a8_kernel<__half><<<grid, 256, 0, st>>>(L21, ldw, m, k, (__half*)Aop, kpad, status);
    return cudaGetLastError();
  }
  if (m > 65535) return cudaErrorInvalidValue;
  dim3 ga((unsigned)cdiv(kpad, 256), (unsigned)m);
  if (kind == 1)
    cast_a_kernel<__nv_bfloat16><<<ga, 256, 0, st>>>(L21, ldw, m, k, (__nv_bfloat16*)Aop, kpad, status);
  else
    cast_a_kernel<__half><<<ga, 256, 0, st>>>(L21, ldw, m, k, (__half*)Aop, kpad, status);
  return cudaGetLastError();
}

// ------------------------------------------------------------ host side
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled get_encode() {
  static PFN_encodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_encodeTiled)p;
  });
  return fn;
}

static bool make_map(CUtensorMap* map, int kind, const void* ptr, int rows, int kpad, int box_rows) {
  PFN_encodeTiled enc = get_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, kind == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                   const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

cudaError_t tc_gemm_run(int kind, float* C, int64_t ldc, const void* Aop, const void* Bop, int m, int n, int kpad,
                        int* status, const DevInfo& dev, cudaStream_t st, int max_ctas) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  if (kind != 1 && kind != 2) return cudaErrorInvalidValue;
  if (kpad <= 0 || (kpad % TC_BK) != 0) return cudaErrorInvalidValue;
  if (((uintptr_t)Aop & 15u) || ((uintptr_t)Bop & 15u)) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  if (!make_map(&ma, kind, Aop, m, kpad, TC_BM) || !make_map(&mb, kind, Bop, n, kpad, TC_BN))
    return cudaErrorInvalidValue;
  {
    cudaError_t e = allow_max_smem((const void*)tc_gemm_kernel);
    if (e != cudaSuccess) return e;
  }
  TcParams P;
  P.C = C;
  P.ldc = ldc;
  P.m = m;
  P.n = n;
  P.kchunks = kpad / TC_BK;
  P.tiles_m = (int)cdiv(m, TC_BM);
  P.tiles_n = (int)cdiv(n, TC_BN);
  P.vec_ok = (((uintptr_t)C & 15u) == 0 && (ldc % 4) == 0) ? 1 : 0;
  P.idesc = tc_idesc_mn(kind == 1 ? 1u : 0u, TC_BM, TC_BN);
  P.status = status;
  const int ntiles = P.tiles_m * P.tiles_n;
  int grid = ntiles < dev.sm_count ? ntiles : dev.sm_count;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  tc_gemm_kernel<<<grid, TC_THREADS, TC_SMEM, st>>>(ma, mb, P);
  return cudaGetLastError();
}


}  // namespace gb
