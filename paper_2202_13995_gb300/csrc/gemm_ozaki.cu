// FP64 trailing update C -= A B on the BF16 tensor cores by error-free
// splitting (the Ozaki scheme: K. Ozaki, T. Ogita, S. Oishi, S. M. Rump,
// "Error-free transformations of matrix multiplication by using fast routines
// of matrix multiplication and its applications", Numer. Algorithms 59, 2012;
// on tensor cores: D. Mukunoki, K. Ozaki, T. Ogita, T. Imamura, "DGEMM using
// Tensor Cores, and Its Accurate and Reproducible Versions", ISC 2020).
//
// This is the paper's "inner" block update (arxiv 2202.13995, section "Base
// Implementation") in FP64 accuracy without FP64 multiply-adds for the
// products: GB300's FP64 rate is a small fraction of its BF16 tensor rate, and
// tcgen05 has no FP64 kind.
//
// Splitting.  Row i of A is scaled by 2^-e_i (2^e_i the power of two just
// above its largest |a|) and cut into S = 8 slices of 7-bit integers d_p:
//   a = 2^e_i * sum_p d_p 2^(-7(p+1))  + (remainder below 2^(e_i - 56)).
// Column j of B likewise (2^f_j, slices g_q).  Every slice is an integer in
// [-127, 127], exact in BF16.
//
// Products.  For each slice pair (p, q) with t = p + q <= S - 1 (36 pairs) the
// tensor cores form G = sum_k d_p(i,k) g_q(k,j) over the full k <= 256: an
// integer of magnitude < 256 * 127^2 < 2^22, exact in the FP32 accumulator.
//
// Combination, exact and in integers.  G + 1.5 * 2^23 is exact in FP32 and
// its bit pattern is 0x4B400000 + G; the epilogue adds that pattern, shifted
// by 40 - 7t, into a 64-bit integer per element (the constant part is
// subtracted once at the end).  The sum I is the product's scaled value in
// units of 2^(e_i + f_j - 54); |I| < 2^63 by the bound on G.  The 15 pairs of
// the two smallest orders (t = 6, 7) are shifted right, rounded to nearest.
// Finally C -= I * 2^(e_i + f_j - 54): one rounding in the conversion of I and
// one in the subtraction.
//
// Error of I * 2^(e_i + f_j - 54) against the exact sum of products, in units
// of 2^-53 * 2^(e_i + f_j): dropped pairs (t >= 8) < 0.87 k, splitting
// remainders < 0.25 k, rounded shifts <= 3.75; so below (1.13 k + 4).  The
// conversion adds at most 2^-53 sum_k |a b|, the subtraction 2^-53 |result|:
// the order of the rounding error bound of a k-term FP64 dot product.
//
// Kernel.  Persistent CTAs (one per SM) walk 128 x 128 output tiles.  For a
// tile, A's slice p (128 rows x k) sits in shared memory (double-buffered, the
// next slice loads while the current one is used) while B's slices q stream
// through a 6-stage ring; warp 0 issues the TMA loads, warp 1 the tcgen05.mma
// (M = 128, N = 128, K = 16) into one of four TMEM accumulators per pair, and
// warps 4..11 drain each finished accumulator into their 64 per-thread 64-bit
// sums (registers moved to them from warps 0..3 by setmaxnreg).  A finished
// tile's sums are parked in a per-CTA scratch (L2-resident) and applied to C
// two columns per slice pair of the next tile, so the FP64 conversion and
// subtraction (GB300 runs about two FP64 operations per clock per SM) overlap
// the next tile's products instead of stalling them.  With m = 32 (the
// refinement's residual for 32 right-hand sides) A's slices lie 32 rows apart,
// so the box of slice p holds slices p .. p + 3 in its four TMEM lane quarters:
// a tile then takes the products of slices 0 and 4 only (12 instead of 36),
// each epilogue warp weights its quarter by that quarter's slice order, and
// the four quarters' exact partial sums are added before the FP64 update,
// which every quarter applies to a quarter of the columns.  Every mbarrier
// wait is bounded; on timeout the kernel raises ST_TIMEOUT, lets issued copies
// and MMAs land, frees TMEM and returns.
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace gb {

constexpr int OZ_S = 8;        // slices per operand
constexpr int OZ_BITS = 7;     // bits per slice
constexpr int OZ_KMAX = 256;   // exactness bound on k (k * 127^2 < 2^22)
constexpr int OZ_F = 40;       // fraction bits of the integer sum below the t = 0 term
constexpr int OZ_BM = 128, OZ_BN = 128, OZ_BK = 64;
constexpr int OZ_CHUNK = OZ_BM * OZ_BK * 2;          // 16 KB: one 128 x 64 BF16 box (A or B)
constexpr int OZ_ABUF = (OZ_KMAX / OZ_BK) * OZ_CHUNK;  // 64 KB: one resident A slice
constexpr int OZ_BSTAGES = 6;
constexpr int OZ_NACC = 4;     // TMEM accumulators of 128 columns
constexpr int OZ_EPI_WARPS = 8;                  // warpgroups 1 and 2
constexpr int OZ_THREADS = 32 * (4 + OZ_EPI_WARPS);  // warpgroup 0: TMA warp, MMA warp, two idle warps
// Register split (setmaxnreg): warpgroup 0 gives registers to the two epilogue
// warpgroups, which hold 64 64-bit sums per thread.  The split must fit the
// block's launch allocation (OZ_THREADS x the kernel's register count); the
// launcher checks that before every launch, so an increase never waits.
constexpr int OZ_REG_LOW = 56, OZ_REG_HIGH = 224;
constexpr int OZ_REG_POOL = OZ_REG_LOW * 128 + OZ_REG_HIGH * 256;
constexpr int OZ_TMEM_COLS = OZ_NACC * OZ_BN;
constexpr size_t OZ_SMEM = 1024 + 2 * (size_t)OZ_ABUF + (size_t)OZ_BSTAGES * OZ_CHUNK + 256;
constexpr uint32_t OZ_MAGIC_BITS = 0x4B400000u;  // bit pattern of 1.5 * 2^23
constexpr float OZ_MAGIC = 12582912.0f;

static_assert(OZ_KMAX * 127 * 127 < (1 << 22), "a slice-pair product must stay below 2^22");
static_assert(OZ_SMEM <= 232448, "shared memory per CTA");

// ------------------------------------------------------------ splitting
// The slices of x with |x| < 2^e: d_p = trunc(128 r_p), r_{p+1} = 128 r_p - d_p,
// r_0 = x 2^-e.  Every step is exact in FP64, so d_p is digit p of the base-128
// expansion of |x| 2^-e with x's sign; it is taken here from the bit pattern
// (integer operations only: GB300's FP64 rate would make the FP64 form the
// cost of the split).  The 56-bit magnitude M = floor(|x| 2^(56 - e)) holds the
// eight digits, d_p = (M >> (49 - 7p)) & 127.
__device__ __forceinline__ uint64_t oz_fixed56(uint64_t bits, int e) {
  const int field = (int)((bits >> 52) & 0x7ff);
  uint64_t mant = bits & 0xfffffffffffffull;
  if (field) mant |= 1ull << 52;
  const int sh = (field ? field : 1) - 1075 + 56 - e;  // |x| = mant 2^(field' - 1075)
  if (sh >= 0) return sh < 64 ? mant << sh : 0ull;
  return -sh < 64 ? mant >> (-sh) : 0ull;
}

// BF16 pattern of the integer sign * d, 0 <= d <= 127 (exact: <= 7 significant bits)
__device__ __forceinline__ uint32_t oz_bf16_digit(uint32_t d, uint32_t sign) {
  if (d == 0) return 0u;
  const int k = 31 - __clz(d);  // leading bit
  return sign | ((127u + (uint32_t)k) << 7) | ((d << (7 - k)) & 0x7fu);
}

// e with |x| < 2^e <= 2|x| for the largest |x| of a line, from its pattern (0 for 0)
__device__ __forceinline__ int oz_expo(uint64_t absbits) {
  if (absbits == 0) return 0;
  const int field = (int)(absbits >> 52);
  if (field) return field - 1022;
  return (63 - __clzll((long long)absbits)) - 1074 + 1;  // subnormal
}

// A (m x k, row-major FP64) -> As[p][i][kpad] (BF16 integers), ea[i] = e_i.
// One warp per row; a lane takes element pairs (2 lane + 64 u, + 1).
__global__ void __launch_bounds__(256) oz_split_rows_kernel(const double* __restrict__ A, int64_t lda, int m, int k,
                                                            int kpad, __nv_bfloat16* __restrict__ As,
                                                            int* __restrict__ ea, int* status) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= m) return;
  constexpr int U = OZ_KMAX / 64;
  uint64_t v[U][2];
  uint64_t mx = 0;
  bool bad = false;
  const double* row = A + (int64_t)i * lda;
#pragma unroll
  for (int u = 0; u < U; ++u) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = 64 * u + 2 * lane + h;
      v[u][h] = c < k ? (uint64_t)__double_as_longlong(row[c]) : 0ull;
      const uint64_t a = v[u][h] & 0x7fffffffffffffffull;
      bad |= (a >> 52) == 0x7ff;
      mx = a > mx ? a : mx;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const uint64_t o = __shfl_xor_sync(0xffffffffu, mx, off);
    mx = o > mx ? o : mx;
  }
  const bool zero = __any_sync(0xffffffffu, bad);
  if (zero && lane == 0) atomicOr(status, ST_RANGE);
  const int e = zero ? 0 : oz_expo(mx);
  if (lane == 0) ea[i] = e;
  uint32_t* out = reinterpret_cast<uint32_t*>(As);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int c = 64 * u + 2 * lane;
    if (c >= kpad) break;
    const uint64_t M0 = zero ? 0ull : oz_fixed56(v[u][0], e);
    const uint64_t M1 = zero ? 0ull : oz_fixed56(v[u][1], e);
    const uint32_t s0 = (uint32_t)(v[u][0] >> 48) & 0x8000u, s1 = (uint32_t)(v[u][1] >> 48) & 0x8000u;
#pragma unroll
    for (int p = 0; p < OZ_S; ++p) {
      const int sh = 49 - OZ_BITS * p;
      const uint32_t w = oz_bf16_digit((uint32_t)(M0 >> sh) & 127u, s0) |
                         (oz_bf16_digit((uint32_t)(M1 >> sh) & 127u, s1) << 16);
      out[(((int64_t)p * m + i) * kpad + c) >> 1] = w;
    }
  }
}

// B (k x n, row-major FP64) -> Bs[q][j][kpad] (column j's slice, K contiguous),
// fb[j] = f_j.  CTA = 32 columns; 64-row blocks go through shared memory.
__global__ void __launch_bounds__(256) oz_split_cols_kernel(const double* __restrict__ B, int64_t ldb, int k, int n,
                                                            int kpad, __nv_bfloat16* __restrict__ Bs,
                                                            int* __restrict__ fb, int* status) {
  __shared__ uint64_t tile[OZ_BK][33];
  __shared__ uint64_t red[8][32];
  __shared__ int fe[32];
  constexpr int ZERO_COL = 1 << 20;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j0 = blockIdx.x * 32, j = j0 + lane;
  uint64_t mx = 0;
  bool bad = false;
  for (int r = warp; r < k; r += 8) {
    const uint64_t a = j < n ? ((uint64_t)__double_as_longlong(B[(int64_t)r * ldb + j]) & 0x7fffffffffffffffull) : 0ull;
    bad |= (a >> 52) == 0x7ff;
    mx = a > mx ? a : mx;
  }
  red[warp][lane] = bad ? ~0ull : mx;
  __syncthreads();
  if (warp == 0) {
    bool b2 = false;
    mx = 0;
    for (int w = 0; w < 8; ++w) {
      const uint64_t o = red[w][lane];
      b2 |= o == ~0ull;
      if (o != ~0ull) mx = o > mx ? o : mx;
    }
    if (b2) atomicOr(status, ST_RANGE);
    const int e = b2 ? 0 : oz_expo(mx);
    fe[lane] = (b2 || mx == 0) ? ZERO_COL : e;
    if (j < n) fb[j] = e;
  }
  __syncthreads();
  uint32_t* out = reinterpret_cast<uint32_t*>(Bs);
  for (int r0 = 0; r0 < kpad; r0 += OZ_BK) {
    for (int r = warp; r < OZ_BK; r += 8)
      tile[r][lane] = (r0 + r < k && j < n) ? (uint64_t)__double_as_longlong(B[(int64_t)(r0 + r) * ldb + j]) : 0ull;
    __syncthreads();
    for (int c = warp; c < 32; c += 8) {
      const int jj = j0 + c;
      if (jj >= n) continue;
      const int e = fe[c];
      const uint64_t x0 = tile[2 * lane][c], x1 = tile[2 * lane + 1][c];
      const uint64_t M0 = e == ZERO_COL ? 0ull : oz_fixed56(x0, e);
      const uint64_t M1 = e == ZERO_COL ? 0ull : oz_fixed56(x1, e);
      const uint32_t s0 = (uint32_t)(x0 >> 48) & 0x8000u, s1 = (uint32_t)(x1 >> 48) & 0x8000u;
#pragma unroll
      for (int q = 0; q < OZ_S; ++q) {
        const int sh = 49 - OZ_BITS * q;
        const uint32_t w = oz_bf16_digit((uint32_t)(M0 >> sh) & 127u, s0) |
                           (oz_bf16_digit((uint32_t)(M1 >> sh) & 127u, s1) << 16);
        out[(((int64_t)q * n + jj) * kpad + r0 + 2 * lane) >> 1] = w;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ the product kernel
struct OzParams {
  double* C;
  int64_t ldc;
  int m, n;        // rows and columns of this update
  int a_rows;      // rows of one A slice in the slice array
  int b_rows;      // columns of one B slice in the slice array
  int b_col0;      // first column of this update within the split
  int kchunks;
  int tiles_m, tiles_n;
  const int* ea;   // row exponents e_i
  const int* fb;   // column exponents f_j of this update's columns
  int vec_ok;      // C rows 16-byte aligned (vector loads and stores)
  int stacked;     // m == 32: an A box holds four consecutive slices (see the kernel)
  long long* scratch;  // per CTA: the previous tile's sums (OZ_BM x OZ_BN)
  uint32_t idesc;
  int* status;
};

// Output tile t -> (tm, tn), grouped by OZ_GROUP tile rows: within a group the
// tiles run down the rows first, so the tiles that the persistent CTAs hold at
// one time span about OZ_GROUP row blocks and gridDim / OZ_GROUP column
// blocks.  Their A and B slices (512 KB per block) then stay in L2 while C
// streams through it, instead of every row block's slices being evicted and
// read again from HBM for each column block.
constexpr int OZ_GROUP = 12;
__device__ __forceinline__ void oz_tile(int t, int tiles_m, int tiles_n, int& tm, int& tn) {
  const int per_group = OZ_GROUP * tiles_n;
  const int g = t / per_group;
  const int first = g * OZ_GROUP;
  const int gm = min(OZ_GROUP, tiles_m - first);
  const int r = t - g * per_group;
  tm = first + r % gm;
  tn = r / gm;
}

// 64-bit add of (xh:xl) into (h:l) through the carry flag.
__device__ __forceinline__ void oz_add64(uint32_t& l, uint32_t& h, uint32_t xl, uint32_t xh) {
  asm("add.cc.u32 %0, %0, %2;\n\taddc.u32 %1, %1, %3;" : "+r"(l), "+r"(h) : "r"(xl), "r"(xh));
}

// (hi:lo)[j] += pattern of (G_j + 1.5 * 2^23) shifted by 40 - 7t (64-bit sums
// kept as two 32-bit words).  t <= 1 touches the high word only; t = 6, 7 are
// right shifts rounded to nearest: half a unit of the shifted result rides in
// the float constant (G + 1.5 * 2^23 + 2^(r-1) is still exact), and since the
// constant's pattern has 22 low zero bits, the shifted pattern is the shifted
// constant plus floor((G + 2^(r-1)) / 2^r).
__device__ __forceinline__ void oz_acc32(uint32_t* lo, uint32_t* hi, const uint32_t* v, int t) {
  const int sh = OZ_F - OZ_BITS * t;
  if (sh >= 32) {
    const uint32_t mul = 1u << (sh - 32);
#pragma unroll
    for (int j = 0; j < 32; ++j) hi[j] += __float_as_uint(__uint_as_float(v[j]) + OZ_MAGIC) * mul;
  } else if (sh >= 0) {
    const int rs = 32 - sh;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint32_t b = __float_as_uint(__uint_as_float(v[j]) + OZ_MAGIC);
      oz_add64(lo[j], hi[j], b << sh, b >> rs);
    }
  } else {
    const int r = -sh;
    const float M = OZ_MAGIC + (float)(1 << (r - 1));
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const uint32_t b = __float_as_uint(__uint_as_float(v[j]) + M);
      oz_add64(lo[j], hi[j], b >> r, 0u);
    }
  }
}

__device__ __forceinline__ unsigned long long oz_corr(int t) {
  const int sh = OZ_F - OZ_BITS * t;
  return sh >= 0 ? (unsigned long long)OZ_MAGIC_BITS << sh : (unsigned long long)(OZ_MAGIC_BITS >> (-sh));
}

// C - I 2^E: I converted to FP64 (one rounding), scaled by 2^E through its
// exponent field (exact; two exact power-of-two products outside the normal
// range), then subtracted (one rounding).
__device__ __forceinline__ double oz_sub(double c, long long I, int E) {
  if (I == 0) return c;
  double d = __ll2double_rn(I);
  const long long bits = __double_as_longlong(d);
  const int ex = (int)((bits >> 52) & 0x7ff) + E;
  if (ex >= 1 && ex <= 2046) {
    d = __longlong_as_double(bits + ((long long)E << 52));
  } else {
    const int e1 = E / 2, e2 = E - e1;
    d = (d * __longlong_as_double((long long)(1023 + e1) << 52)) * __longlong_as_double((long long)(1023 + e2) << 52);
  }
  return c - d;
}

__global__ void __launch_bounds__(OZ_THREADS, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams P) {
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t sA = base;                 // 2 x OZ_ABUF
  const uint32_t sB = base + 2 * OZ_ABUF;   // OZ_BSTAGES x OZ_CHUNK
  unsigned char* ctl = gbase + 2 * OZ_ABUF + OZ_BSTAGES * OZ_CHUNK;
  const uint32_t bar_afull = smem_u32(ctl);
  const uint32_t bar_aempty = bar_afull + 16;
  const uint32_t bar_bfull = bar_aempty + 16;
  const uint32_t bar_bempty = bar_bfull + 8 * OZ_BSTAGES;
  const uint32_t bar_tfull = bar_bempty + 8 * OZ_BSTAGES;
  const uint32_t bar_tempty = bar_tfull + 8 * OZ_NACC;
  const uint32_t bar_drain = bar_tempty + 8 * OZ_NACC;
  const uint32_t bar_consumed = bar_drain + 8;  // stacked: every epilogue warp has read the parked sums
  const uint32_t bar_parked = bar_consumed + 8;  // stacked: every epilogue warp has parked its sums
  constexpr int NBAR = 4 + 2 * OZ_BSTAGES + 2 * OZ_NACC + 3;
  static_assert(8 * NBAR + 16 <= 256, "control block");
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(ctl + 8 * NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(ctl + 8 * NBAR + 8);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = P.tiles_m * P.tiles_n;
  // With m == 32 the 128-row box of A slice p holds slices p .. p + 3 in its
  // four 32-row quarters, so one product with B slice q serves the pairs
  // (p + g, q), g = 0..3: the tile walks p = 0, 4 (12 products instead of 36)
  // and each epilogue warp weights its quarter by that quarter's slice order.
  const int pstep = P.stacked ? 4 : 1;

  if (threadIdx.x == 0) {
    for (int a = 0; a < 2; ++a) {
      mbar_init(bar_afull + 8 * a, 1);
      mbar_init(bar_aempty + 8 * a, 1);
    }
    for (int s = 0; s < OZ_BSTAGES; ++s) {
      mbar_init(bar_bfull + 8 * s, 1);
      mbar_init(bar_bempty + 8 * s, 1);
    }
    for (int a = 0; a < OZ_NACC; ++a) {
      mbar_init(bar_tfull + 8 * a, 1);
      mbar_init(bar_tempty + 8 * a, OZ_EPI_WARPS);
    }
    mbar_init(bar_drain, 1);
    mbar_init(bar_consumed, OZ_EPI_WARPS);
    mbar_init(bar_parked, OZ_EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp < 4) {
   // warpgroup 0 (one setmaxnreg site for all four warps)
   asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(OZ_REG_LOW));
   if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      int apar[2] = {-1, -1};
      int bpar[OZ_BSTAGES];
#pragma unroll
      for (int s = 0; s < OZ_BSTAGES; ++s) bpar[s] = -1;
      int s = 0, ab = 0;
      uint32_t ph = 0, abph = 0;
      bool ok = true;
      // A slices load one slice ahead, into the buffer the MMA released last:
      // slice (tile, p + pstep) is issued once the B chunks of (p, q = 0) are.
      auto load_a = [&](int tile, int p) -> bool {
        if (!mbar_wait(bar_aempty + 8 * ab, abph ^ 1u, P.status, abort_flag)) return false;
        int tm, tn_unused;
        oz_tile(tile, P.tiles_m, P.tiles_n, tm, tn_unused);
        mbar_expect_tx(bar_afull + 8 * ab, (uint32_t)(P.kchunks * OZ_CHUNK));
        for (int kc = 0; kc < P.kchunks; ++kc)
          tma_load_2d(sA + ab * OZ_ABUF + kc * OZ_CHUNK, &tmA, kc * OZ_BK, p * P.a_rows + tm * OZ_BM,
                      bar_afull + 8 * ab);
        apar[ab] = (int)abph;
        if (++ab == 2) {
          ab = 0;
          abph ^= 1u;
        }
        return true;
      };
      if ((int)blockIdx.x < ntiles) ok = load_a(blockIdx.x, 0);
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        int tm_unused, tn;
        oz_tile(t, P.tiles_m, P.tiles_n, tm_unused, tn);
        for (int p = 0; p < OZ_S && ok; p += pstep) {
          for (int q = 0; q < OZ_S - p && ok; ++q) {
            for (int kc = 0; kc < P.kchunks; ++kc) {
              if (!mbar_wait(bar_bempty + 8 * s, ph ^ 1u, P.status, abort_flag)) {
                ok = false;
                break;
              }
              mbar_expect_tx(bar_bfull + 8 * s, OZ_CHUNK);
              tma_load_2d(sB + s * OZ_CHUNK, &tmB, kc * OZ_BK, q * P.b_rows + P.b_col0 + tn * OZ_BN,
                          bar_bfull + 8 * s);
              bpar[s] = (int)ph;
              if (++s == OZ_BSTAGES) {
                s = 0;
                ph ^= 1u;
              }
            }
            if (ok && q == 0) {
              if (p + pstep < OZ_S)
                ok = load_a(t, p + pstep);
              else if (t + (int)gridDim.x < ntiles)
                ok = load_a(t + gridDim.x, 0);
            }
          }
        }
      }
      if (!ok) {
        // let every issued copy land before the CTA can exit
        for (int a = 0; a < 2; ++a) {
          if (apar[a] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try(bar_afull + 8 * a, (uint32_t)apar[a]) && gtimer() - t0 < GB_SPIN_LIMIT_NS) {
          }
        }
        for (int q = 0; q < OZ_BSTAGES; ++q) {
          if (bpar[q] < 0) continue;
          const uint64_t t0 = gtimer();
          while (!mbar_try(bar_bfull + 8 * q, (uint32_t)bpar[q]) && gtimer() - t0 < GB_SPIN_LIMIT_NS) {
          }
        }
      }
    }
   } else if (warp == 1) {
    // ---------------- MMA issuer: one TMEM accumulator per slice pair
    if (lane == 0) {
      int s = 0, ab = 0, acc = 0;
      uint32_t ph = 0, abph = 0, tph = 0;
      bool ok = true, issued = false;
      for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        for (int p = 0; p < OZ_S && ok; p += pstep) {
          if (!mbar_wait(bar_afull + 8 * ab, abph, P.status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = sA + ab * OZ_ABUF;
          for (int q = 0; q < OZ_S - p && ok; ++q) {
            if (!mbar_wait(bar_tempty + 8 * acc, tph ^ 1u, P.status, abort_flag)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dtm = tmem_base + (uint32_t)(acc * OZ_BN);
            for (int kc = 0; kc < P.kchunks; ++kc) {
              if (!mbar_wait(bar_bfull + 8 * s, ph, P.status, abort_flag)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t b0 = sB + s * OZ_CHUNK;
#pragma unroll
              for (int kk = 0; kk < OZ_BK / 16; ++kk)
                tc_mma(dtm, sw128_desc(a0 + kc * OZ_CHUNK + kk * 32), sw128_desc(b0 + kk * 32), P.idesc,
                       (kc | kk) ? 1u : 0u);
              issued = true;
              tc_commit(bar_bempty + 8 * s);
              if (++s == OZ_BSTAGES) {
                s = 0;
                ph ^= 1u;
              }
            }
            if (!ok) break;
            tc_commit(bar_tfull + 8 * acc);
            if (++acc == OZ_NACC) {
              acc = 0;
              tph ^= 1u;
            }
          }
          if (!ok) break;
          tc_commit(bar_aempty + 8 * ab);
          if (++ab == 2) {
            ab = 0;
            abph ^= 1u;
          }
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
   }
  } else {
    // ---------------- epilogue: exact integer combination, then C -= I * 2^(e_i + f_j - 54)
    // (warpgroups 1 and 2, one setmaxnreg site)
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(OZ_REG_HIGH));
    const int quarter = warp & 3;          // TMEM lane quarter this warp may access
    const int half = (warp - 4) >> 2;      // which 64 columns of the tile
    const int et = threadIdx.x - 128;      // 0 .. 255
    const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
    // stacked: this warp's TMEM rows are slice p + gq of the box of slice p;
    // every quarter then updates C row `lane`, the column pairs 4 i + gq, from
    // the four quarters' parked sums
    const int gq = P.stacked ? quarter : 0;
    const int kstep = P.stacked ? 4 : 1;
    const int kn = 32 / kstep;  // column pairs of the deferred update per thread
    uint32_t sph = 0;  // stacked: phase parity of bar_consumed and bar_parked
    // This thread's 64 sums of the previous tile, parked in the CTA's scratch
    // ([pair of columns][thread][2]: a warp's accesses are contiguous) and
    // applied to C two columns per slice pair of the next tile, so that the
    // FP64 work of the update runs under that tile's products.
    long long* scr = P.scratch + (size_t)blockIdx.x * (OZ_BM * OZ_BN) + 2 * et;
    double* dcrow = nullptr;  // previous tile's C row segment (null: nothing pending)
    int dcol0 = 0, der = 0;
    long long qI[2];          // the chunk in flight: sums, C values, column exponents
    double qC[2];
    int qF[2], qk = -1;
    auto defer_issue = [&](int k) {  // columns 2k, 2k + 1 of the pending segment
      qk = -1;
      if (dcrow == nullptr || dcol0 + 2 * k >= P.n) return;
      qk = k;
      const longlong2 iv = *reinterpret_cast<const longlong2*>(scr + (size_t)k * (2 * 256));
      qI[0] = iv.x;
      qI[1] = iv.y;
      if (P.stacked) {
        // the same row's partial sums of the other quarters (threads
        // et + 32 (g - gq)): exact integers, so their sum is the whole product's
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          if (g == gq) continue;
          const longlong2 w =
              __ldcg(reinterpret_cast<const longlong2*>(scr + (size_t)k * (2 * 256) + 64 * (g - gq)));
          qI[0] = (long long)((unsigned long long)qI[0] + (unsigned long long)w.x);
          qI[1] = (long long)((unsigned long long)qI[1] + (unsigned long long)w.y);
        }
      }
      const int gc = dcol0 + 2 * k;
      if (P.vec_ok && gc + 2 <= P.n) {
        const double2 cv = *reinterpret_cast<const double2*>(dcrow + 2 * k);
        qC[0] = cv.x;
        qC[1] = cv.y;
      } else {
        qC[0] = dcrow[2 * k];
        qC[1] = gc + 1 < P.n ? dcrow[2 * k + 1] : 0.0;
      }
      qF[0] = P.fb[gc];
      qF[1] = gc + 1 < P.n ? P.fb[gc + 1] : 0;
    };
    auto defer_complete = [&]() {
      if (qk < 0) return;
      const int gc = dcol0 + 2 * qk;
      const double r0 = oz_sub(qC[0], qI[0], der + qF[0]);
      const double r1 = oz_sub(qC[1], qI[1], der + qF[1]);
      if (P.vec_ok && gc + 2 <= P.n) {
        *reinterpret_cast<double2*>(dcrow + 2 * qk) = make_double2(r0, r1);
      } else {
        dcrow[2 * qk] = r0;
        if (gc + 1 < P.n) dcrow[2 * qk + 1] = r1;
      }
      qk = -1;
    };
    int acc = 0;
    uint32_t tph = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      int tm, tn;
      oz_tile(t, P.tiles_m, P.tiles_n, tm, tn);
      const int row = P.stacked ? lane : tm * OZ_BM + quarter * 32 + lane;
      const bool rok = row < P.m;
      const int col0 = tn * OZ_BN + half * 64;
      double* crow = P.C + (int64_t)row * P.ldc + col0;
      uint32_t lo[64], hi[64];
#pragma unroll
      for (int j = 0; j < 64; ++j) lo[j] = hi[j] = 0u;
      unsigned long long corr = 0ull;
      int pi = 0;  // slice pair index within the tile
      for (int p = 0; p < OZ_S && ok; p += pstep) {
        if (p == (P.stacked ? 4 : 6) && rok) {
          // bring this tile's C segment into L2 for its deferred update
#pragma unroll
          for (int c = 0; c < 64; c += 16)
            if (col0 + c < P.n) asm volatile("prefetch.global.L2::evict_last [%0];" ::"l"(crow + c));
        }
        for (int q = 0; q < OZ_S - p; ++q, ++pi) {
          int okw = 1;
          if (lane == 0) okw = mbar_wait(bar_tfull + 8 * acc, tph, P.status, abort_flag) ? 1 : 0;
          okw = __shfl_sync(0xffffffffu, okw, 0);
          if (!okw) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int tt = p + gq + q;
          if (tt < OZ_S) {
            const uint32_t taddr = tmem_base + lane_addr + (uint32_t)(acc * OZ_BN + half * 64);
            uint32_t v[32];
            TMEM_LD_X16(taddr, v);
            TMEM_LD_X16(taddr + 16, (v + 16));
            tmem_wait_ld();
            oz_acc32(lo, hi, v, tt);
            TMEM_LD_X16(taddr + 32, v);
            TMEM_LD_X16(taddr + 48, (v + 16));
            tmem_wait_ld();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_tempty + 8 * acc);
            oz_acc32(lo + 32, hi + 32, v, tt);
            corr += oz_corr(tt);
          } else {
            // a stacked quarter whose pair order is past the last kept one
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_tempty + 8 * acc);
          }
          if (++acc == OZ_NACC) {
            acc = 0;
            tph ^= 1u;
          }
          // the previous tile's update, two columns per pair, loads one pair ahead
          defer_complete();
          if (pi < kn) defer_issue(pi * kstep + gq);
        }
      }
      if (!ok) break;
      defer_complete();
      // (every pair of a tile has passed: nothing of the previous update is left)
      for (; pi < kn; ++pi) {
        defer_issue(pi * kstep + gq);
        defer_complete();
      }
      if (P.stacked) {
        // every quarter has read the previous sums that this warp overwrites now
        __syncwarp();
        int okw = 1;
        if (lane == 0) {
          mbar_arrive(bar_consumed);
          okw = mbar_wait(bar_consumed, sph, P.status, abort_flag) ? 1 : 0;
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          ok = false;
          break;
        }
      }
      // park this tile's sums; their update runs during the next tile
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const unsigned long long i0 = (((unsigned long long)hi[2 * k] << 32) | lo[2 * k]) - corr;
        const unsigned long long i1 = (((unsigned long long)hi[2 * k + 1] << 32) | lo[2 * k + 1]) - corr;
        *reinterpret_cast<longlong2*>(scr + (size_t)k * (2 * 256)) = make_longlong2((long long)i0, (long long)i1);
      }
      if (P.stacked) {
        // the quarters read each other's parked sums only after all are written
        __threadfence_block();
        __syncwarp();
        int okw = 1;
        if (lane == 0) {
          mbar_arrive(bar_parked);
          okw = mbar_wait(bar_parked, sph, P.status, abort_flag) ? 1 : 0;
        }
        okw = __shfl_sync(0xffffffffu, okw, 0);
        if (!okw) {
          ok = false;
          break;
        }
        sph ^= 1u;
      }
      dcrow = rok ? crow : nullptr;
      dcol0 = col0;
      der = rok ? P.ea[row] - (OZ_F + 2 * OZ_BITS) : 0;
    }
    if (ok && dcrow != nullptr) {
      // the last tile's update
#pragma unroll 1
      for (int i = 0; i < kn; ++i) {
        defer_issue(i * kstep + gq);
        defer_complete();
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(OZ_TMEM_COLS)
                 : "memory");
  }
}

// ------------------------------------------------------------ host side
static size_t al1k(size_t b) { return (b + 1023) / 1024 * 1024; }

size_t ozaki_ws_bytes(int m, int n, int k, int sm_count) {
  const size_t kpad = (size_t)cdiv(k > 0 ? k : 1, OZ_BK) * OZ_BK;
  return al1k((size_t)OZ_S * m * kpad * 2) + al1k((size_t)OZ_S * n * kpad * 2) + al1k((size_t)m * 4) +
         al1k((size_t)n * 4) + (size_t)sm_count * OZ_BM * OZ_BN * 8;
}

struct OzLayout {
  __nv_bfloat16 *As, *Bs;
  int *ea, *fb;
  long long* scratch;
  int kpad;
};

static OzLayout oz_layout(void* ws, int m, int n, int k) {
  OzLayout L;
  L.kpad = (int)cdiv(k, OZ_BK) * OZ_BK;
  char* p = (char*)ws;
  L.As = (__nv_bfloat16*)p;
  p += al1k((size_t)OZ_S * m * L.kpad * 2);
  L.Bs = (__nv_bfloat16*)p;
  p += al1k((size_t)OZ_S * n * L.kpad * 2);
  L.ea = (int*)p;
  p += al1k((size_t)m * 4);
  L.fb = (int*)p;
  p += al1k((size_t)n * 4);
  L.scratch = (long long*)p;
  return L;
}

cudaError_t ozaki_split(const double* A, int64_t lda, const double* B, int64_t ldb, int m, int n, int k, void* ws,
                        int* status, cudaStream_t st) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  if (k > OZ_KMAX || ws == nullptr) return cudaErrorInvalidValue;
  const OzLayout L = oz_layout(ws, m, n, k);
  oz_split_rows_kernel<<<(unsigned)cdiv(m, 8), 256, 0, st>>>(A, lda, m, k, L.kpad, L.As, L.ea, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  oz_split_cols_kernel<<<(unsigned)cdiv(n, 32), 256, 0, st>>>(B, ldb, k, n, L.kpad, L.Bs, L.fb, status);
  return cudaGetLastError();
}

typedef CUresult (*PFN_encodeTiled_oz)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                       const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                       CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                       CUtensorMapFloatOOBfill);

static PFN_encodeTiled_oz oz_encode() {
  static PFN_encodeTiled_oz fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_encodeTiled_oz)p;
  });
  return fn;
}

static bool oz_map(CUtensorMap* map, const void* ptr, int64_t rows, int kpad) {
  PFN_encodeTiled_oz enc = oz_encode();
  if (!enc) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)OZ_BK, (cuuint32_t)OZ_BM};
  cuuint32_t estr[2] = {1, 1};
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t ozaki_gemm(double* C, int64_t ldc, const void* ws, int m, int n, int k, int col0, int ncols, int* status,
                       const DevInfo& dev, cudaStream_t st, int max_ctas) {
  if (m <= 0 || ncols <= 0 || k <= 0) return cudaSuccess;
  if (k > OZ_KMAX || col0 < 0 || col0 + ncols > n || ws == nullptr) return cudaErrorInvalidValue;
  const OzLayout L = oz_layout(const_cast<void*>(ws), m, n, k);
  CUtensorMap ma, mb;
  if (!oz_map(&ma, L.As, (int64_t)OZ_S * m, L.kpad) || !oz_map(&mb, L.Bs, (int64_t)OZ_S * n, L.kpad))
    return cudaErrorInvalidValue;
  cudaError_t e = allow_max_smem((const void*)oz_gemm_kernel);
  if (e != cudaSuccess) return e;
  {
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, (const void*)oz_gemm_kernel);
    if (e != cudaSuccess) return e;
    if (fa.numRegs * OZ_THREADS < OZ_REG_POOL) return cudaErrorInvalidConfiguration;
  }
  OzParams P;
  P.C = C;
  P.ldc = ldc;
  P.m = m;
  P.n = ncols;
  P.a_rows = m;
  P.b_rows = n;
  P.b_col0 = col0;
  P.kchunks = L.kpad / OZ_BK;
  P.tiles_m = (int)cdiv(m, OZ_BM);
  P.tiles_n = (int)cdiv(ncols, OZ_BN);
  P.ea = L.ea;
  P.fb = L.fb + col0;
  P.scratch = L.scratch;
  P.idesc = tc_idesc_mn(1u, OZ_BM, OZ_BN);
  P.vec_ok = (((uintptr_t)C & 15u) == 0 && (ldc % 2) == 0) ? 1 : 0;
  P.stacked = m == 32 ? 1 : 0;  // the slices of a 32-row A are 32 rows apart: four per 128-row box
  P.status = status;
  const int ntiles = P.tiles_m * P.tiles_n;
  int grid = ntiles < dev.sm_count ? ntiles : dev.sm_count;
  if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
  oz_gemm_kernel<<<grid, OZ_THREADS, OZ_SMEM, st>>>(ma, mb, P);
  return cudaGetLastError();
}

}  // namespace gb

namespace gb {

// M = I - L^-1 for the unit-lower w x w block L (row-major, ld ldl): the top
// block solve U12 = L^-1 A12 then becomes the update A12 - M A12, which the
// split product runs on the tensor cores.  One warp per column j of L^-1,
// forward substitution in its column (axpy) form: x = e_j, then for
// k = j, j+1, ...: x_i -= L(i,k) x_k for every i > k, so each x_i receives its
// terms in the order of k as in the definition.  Lane l holds x_i for
// i = l + 32 r (r < 8); x_k is broadcast by a shuffle.  No reduction: GB300
// runs FP64 at two operations per clock per SM, and a shuffle-add tree per
// row cost more than the products.  M(i,j) = -x_i below the diagonal, 0 on
// and above it.
template <int KB>
__device__ __forceinline__ void oz_inv_block(const double* __restrict__ L, int64_t ldl, int w, int j, int lane,
                                             double (&x)[8]) {
  if (j >= (KB + 1) * 32) return;  // this block of k lies left of column j
#pragma unroll
  for (int kk = 0; kk < 32; ++kk) {
    const int k = KB * 32 + kk;
    if (k < j) continue;
    if (k >= w - 1) return;
    const double xk = __shfl_sync(0xffffffffu, x[KB], kk);
#pragma unroll
    for (int r = KB; r < 8; ++r) {
      const int i = lane + 32 * r;
      if (i > k && i < w) x[r] = fma(-L[(int64_t)i * ldl + k], xk, x[r]);
    }
  }
}

__global__ void __launch_bounds__(32) unit_lower_inv_comp_kernel(const double* __restrict__ L, int64_t ldl, int w,
                                                                 double* __restrict__ M, int64_t ldm) {
  const int lane = threadIdx.x;
  const int j = blockIdx.x;
  double x[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) x[r] = (lane + 32 * r == j) ? 1.0 : 0.0;
  oz_inv_block<0>(L, ldl, w, j, lane, x);
  oz_inv_block<1>(L, ldl, w, j, lane, x);
  oz_inv_block<2>(L, ldl, w, j, lane, x);
  oz_inv_block<3>(L, ldl, w, j, lane, x);
  oz_inv_block<4>(L, ldl, w, j, lane, x);
  oz_inv_block<5>(L, ldl, w, j, lane, x);
  oz_inv_block<6>(L, ldl, w, j, lane, x);
  oz_inv_block<7>(L, ldl, w, j, lane, x);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int i = lane + 32 * r;
    if (i < w) M[(int64_t)i * ldm + j] = i > j ? -x[r] : 0.0;
  }
}

cudaError_t launch_unit_lower_inv_comp(const double* L, int64_t ldl, int w, double* M, int64_t ldm, cudaStream_t st) {
  if (w <= 0) return cudaSuccess;
  if (w > OZ_KMAX) return cudaErrorInvalidValue;
  static_assert(OZ_KMAX <= 8 * 32, "one warp holds a column of up to 256 entries");
  unit_lower_inv_comp_kernel<<<(unsigned)w, 32, 0, st>>>(L, ldl, w, M, ldm);
  return cudaGetLastError();
}

}  // namespace gb
