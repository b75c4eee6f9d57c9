// Forward/back substitution, FP64 residual and the refinement update.
//
// The solve answers the second step of the HPL problem statement (arxiv
// 2202.13995, section "High Performance Linpack", first paragraph): with
// P A = L U, solve L y = P b, then U x = y.  The paper runs this step on the
// CPU; here it is one kernel per triangle.
//
// Triangular solve design (one launch per triangle): the rows are cut in
// blocks of 64.  Each CTA takes a block in dependency order from an atomic
// ticket (so a CTA only ever waits on blocks taken by CTAs already running),
// accumulates the products of its block row with every finished solution
// block as soon as that block's flag is published, then solves its own
// 64 x 64 diagonal block and publishes its solution block.  Every matrix entry
// is read once per chunk of right-hand sides, and the only serial chain is
// the diagonal solves.  More right-hand sides than one CTA holds are cut in
// chunks whose blocks interleave on the one ticket counter (block b of chunk
// c is ticket b * chunks + c), so the chunks' chains run side by side in one
// launch instead of one after the other.
#include "common.cuh"
#include "kernels.h"

namespace gb {

constexpr int TS_BS = 64;
constexpr int TS_NRMAX = 16;  // right-hand sides per CTA: 16 for FP32 factors, 8 for FP64
constexpr int TS_RHS_MAX = 32;  // right-hand sides per launch (chunks of the above)
constexpr int TS_CHUNKS_MAX = TS_RHS_MAX / 8;

// Leading dimension of the solution workspaces: a multiple of 16 elements, so
// that every 16-byte chunk of a solution block starts 16-byte aligned.
__host__ __device__ __forceinline__ int64_t trsv_ldy(int n) { return ((int64_t)n + 15) / 16 * 16; }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

// Shared memory of one triangular-solve CTA: a ring of STAGES matrix blocks
// (64 x 64, rows contiguous) with the matching solution blocks, plus the
// padded diagonal block.
template <typename T, int NR, int STAGES>
struct TrsvSmem {
  T Lb[STAGES][TS_BS][TS_BS];
  T yb[STAGES][NR][TS_BS];
  T Ld[TS_BS][TS_BS + 1];  // diagonal block (or its inverse), padded rows
  T v[NR][TS_BS];
  T rinv[TS_BS];  // 1 / U(t,t) of the diagonal block (upper substitution)
  int flag;
  int blk;
};

// With DINV, the diagonal block's inverse (precomputed by trinv_kernel) turns
// the serial substitution into a parallel matrix-vector product; the FP32
// correction solves of the refinement use it.  The FP64 solve substitutes;
// its upper triangle multiplies by the reciprocals of the diagonal, computed
// when the block starts, off the chain of blocks (an FP64 division on GB300
// takes longer than the rest of a substitution step).

// LOWER: Y = L^-1 (P B) with unit-lower L; the right-hand side is gathered
//        from B through rowid: (P b)[i] = b[rowid[i]].
// UPPER: X = U^-1 Y with non-unit upper U; the result goes to Yout (T) for
//        the later blocks and to X (FP64).
// Y layouts: Yin/Yout[q * ldy + i] (column q of the n x nrhs block), ldy = trsv_ldy(n).
// nch chunks of NR right-hand sides (the last one possibly narrower); chunk c
// takes columns [c NR, c NR + NR) of B, Y and X and the flags [c nblk, (c+1) nblk).
// Requires ldw % (16 / sizeof(T)) == 0 and a 16-byte aligned W (the working
// matrix is allocated that way).
template <typename T, int NR, int STAGES, bool LOWER, bool DINV>
__global__ void __launch_bounds__(256) trsv_kernel(const T* __restrict__ W, int64_t ldw, int n, int nrhs_all, int nch,
                                                   const double* __restrict__ B0, int64_t ldb,
                                                   const int* __restrict__ rowid, const T* __restrict__ Yin0,
                                                   T* Yout0, double* X0, int64_t ldx, int* flags0, int* ticket,
                                                   int* status, const T* __restrict__ Dinv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrsvSmem<T, NR, STAGES>& sm = *reinterpret_cast<TrsvSmem<T, NR, STAGES>*>(smem_raw);
  constexpr int CH = 16 / sizeof(T);  // elements per 16-byte chunk
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nblk = (n + TS_BS - 1) / TS_BS;
  const int64_t ldy = trsv_ldy(n);
  // Persistent: a CTA takes blocks in ticket order until none is left (a
  // block waits only on lower tickets, all held by running CTAs or done, so
  // any grid size works; a capped grid leaves the other SMs to other work).
  for (;;) {
    if (tid == 0) {
      sm.blk = atomicAdd(ticket, 1);
      sm.flag = 1;
    }
    __syncthreads();
    const int tk = sm.blk;
    if (tk >= nblk * nch) return;  // uniform: sm.blk is the CTA's
    if (!GB_IN_BOUNDS(status, tk >= 0)) return;
    const int chunk = tk % nch, t_ = tk / nch;
    const int nrhs = min(NR, nrhs_all - chunk * NR);
    const double* B = B0 ? B0 + (int64_t)chunk * NR * ldb : nullptr;
    const T* Yin = Yin0 ? Yin0 + (int64_t)chunk * NR * ldy : nullptr;
    T* Yout = Yout0 + (int64_t)chunk * NR * ldy;
    double* X = X0 ? X0 + (int64_t)chunk * NR * ldx : nullptr;
    int* flags = flags0 + (int64_t)chunk * nblk;
    const int ib = LOWER ? t_ : nblk - 1 - t_;
    const int i0 = ib * TS_BS;
    const int rows = min(TS_BS, n - i0);
    const int count = LOWER ? ib : nblk - 1 - ib;
    auto jb_of = [&](int it) { return LOWER ? it : nblk - 1 - it; };

    // Off the dependency chain: the diagonal block (or its inverse) and this
    // block's right-hand side are loaded first; all loads issue before any use.
    {
      constexpr int PER = TS_BS * TS_BS / 256;
      T dv[PER];
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = tid + q * 256;
        const int rr = e >> 6, cc = e & 63;
        if (DINV)
          dv[q] = Dinv[((int64_t)ib * 2 + (LOWER ? 0 : 1)) * TS_BS * TS_BS + e];
        else
          dv[q] = (rr < rows && cc < rows) ? W[(int64_t)(i0 + rr) * ldw + i0 + cc] : T(0);
      }
#pragma unroll
      for (int q = 0; q < PER; ++q) {
        const int e = tid + q * 256;
        sm.Ld[e >> 6][e & 63] = dv[q];
      }
      if (!DINV && !LOWER) {
        __syncthreads();
        if (tid < TS_BS) sm.rinv[tid] = tid < rows ? T(1) / sm.Ld[tid][tid] : T(0);
      }
    }
    // this block's right-hand side: thread (row tid & 63) holds columns
    // q = (tid >> 6) + 4 u
    constexpr int NU = (NR + 3) / 4;
    T rhs[NU];
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      rhs[u] = T(0);
      const int r = tid & 63, q = (tid >> 6) + 4 * u;
      if (q < NR && r < rows && q < nrhs) {
        if (LOWER)
          rhs[u] = (T)B[(int64_t)q * ldb + rowid[i0 + r]];
        else
          rhs[u] = Yin[(int64_t)q * ldy + i0 + r];
      }
    }

    // warp 0: wait for the flag of iteration it's solution block, then copy
    // that block (written before the flag's release) into its stage
    auto load_y = [&](int it) {
      const int jb = jb_of(it);
      const int j0 = jb * TS_BS;
      const int cols = min(TS_BS, n - j0);
      const int st = it % STAGES;
      int ok = 1;
      if (lane == 0) ok = wait_flag_eq(flags + jb, 1, status) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      __syncwarp();  // orders lane 0's acquire before every lane's reads
      if (!ok) {
        if (lane == 0) sm.flag = 0;
        return;
      }
      for (int e = lane; e < NR * TS_BS / CH; e += 32) {
        const int q = e / (TS_BS / CH), cc = (e % (TS_BS / CH)) * CH;
        T* dst = &sm.yb[st][q][cc];
        if (q < nrhs && cc + CH <= cols) {
          cp_async16(dst, Yout + (int64_t)q * ldy + j0 + cc);
        } else {
#pragma unroll
          for (int u = 0; u < CH; ++u)
            dst[u] = (q < nrhs && cc + u < cols) ? __ldcg(Yout + (int64_t)q * ldy + j0 + cc + u) : T(0);
        }
      }
    };
    // issue the loads of iteration `it` into its stage (all threads): the
    // matrix block, and (warp 0, after its flag) the solution block -- except
    // for the last iteration, the block just before this one on the chain:
    // its solution block is fetched only when that iteration runs, so that
    // one product, not STAGES of them, follows the predecessor's flag
    auto issue = [&](int it) {
      if (it < count) {
        const int jb = jb_of(it);
        const int j0 = jb * TS_BS;
        const int cols = min(TS_BS, n - j0);
        const int st = it % STAGES;
        for (int e = tid; e < TS_BS * TS_BS / CH; e += 256) {
          const int rr = e / (TS_BS / CH), cc = (e % (TS_BS / CH)) * CH;
          T* dst = &sm.Lb[st][rr][cc];
          if (rr < rows && cc + CH <= cols) {
            cp_async16(dst, W + (int64_t)(i0 + rr) * ldw + j0 + cc);
          } else {
#pragma unroll
            for (int u = 0; u < CH; ++u)
              dst[u] = (rr < rows && cc + u < cols) ? W[(int64_t)(i0 + rr) * ldw + j0 + cc + u] : T(0);
          }
        }
        if (warp == 0 && it < count - 1) load_y(it);
      }
      cp_async_commit();
    };

    // acc[rr][q]: partial sums of rows 8*warp + rr over this lane's columns
    T acc[8][NR];
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
#pragma unroll
      for (int q = 0; q < NR; ++q) acc[rr][q] = T(0);

#pragma unroll 1
    for (int s0 = 0; s0 < STAGES - 1; ++s0) issue(s0);
#pragma unroll 1
    for (int it = 0; it < count; ++it) {
      issue(it + STAGES - 1);
      cp_async_wait_group<STAGES - 1>();
      if (it == count - 1 && warp == 0) {
        load_y(it);
        cp_async_wait_all();
      }
      __syncthreads();
      if (!sm.flag) {
        cp_async_wait_group<0>();
        return;
      }
      const int st = it % STAGES;
      T y0[NR], y1[NR];
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        y0[q] = sm.yb[st][q][lane];
        y1[q] = sm.yb[st][q][lane + 32];
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const T l0 = sm.Lb[st][warp * 8 + rr][lane];
        const T l1 = sm.Lb[st][warp * 8 + rr][lane + 32];
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[rr][q] = fma(l0, y0[q], fma(l1, y1[q], acc[rr][q]));
      }
      __syncthreads();
    }
    cp_async_wait_group<0>();
    // row sums: a fixed butterfly over the lanes (deterministic)
#pragma unroll
    for (int rr = 0; rr < 8; ++rr)
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        T v = acc[rr][q];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        acc[rr][q] = v;
      }
    if (lane < NR) {
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        T tot = T(0);
#pragma unroll
        for (int q = 0; q < NR; ++q)
          if (q == lane) tot = acc[rr][q];
        sm.v[lane][warp * 8 + rr] = tot;
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NU; ++u) {
      const int r = tid & 63, q = (tid >> 6) + 4 * u;
      if (q < NR) sm.v[q][r] = (r < rows && q < nrhs) ? rhs[u] - sm.v[q][r] : T(0);
    }
    __syncthreads();
    if (DINV) {
      // x = inverse(diagonal block) * v: warp w computes rows 8w .. 8w+7
      T xr[8][NR];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const T d0 = sm.Ld[warp * 8 + rr][lane], d1 = sm.Ld[warp * 8 + rr][lane + 32];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
          T v = d0 * sm.v[q][lane] + d1 * sm.v[q][lane + 32];
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
          xr[rr][q] = v;
        }
      }
      __syncthreads();
      if (lane < NR) {
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          T x = T(0);
#pragma unroll
          for (int q = 0; q < NR; ++q)
            if (q == lane) x = xr[rr][q];
          sm.v[lane][warp * 8 + rr] = x;
        }
      }
    } else
    for (int q = warp; q < nrhs; q += 8) {
      T x0 = sm.v[q][lane], x1 = sm.v[q][lane + 32];
      if (LOWER) {
        for (int t = 0; t < rows; ++t) {
          const T xt = __shfl_sync(0xffffffffu, t < 32 ? x0 : x1, t & 31);
          if (lane > t) x0 -= sm.Ld[lane][t] * xt;
          if (lane + 32 > t) x1 -= sm.Ld[lane + 32][t] * xt;
        }
      } else {
        for (int t = rows - 1; t >= 0; --t) {
          T xt;
          if (t >= 32) {
            if (lane == t - 32) x1 = x1 * sm.rinv[t];
            xt = __shfl_sync(0xffffffffu, x1, t - 32);
          } else {
            if (lane == t) x0 = x0 * sm.rinv[t];
            xt = __shfl_sync(0xffffffffu, x0, t);
          }
          if (lane < t) x0 -= sm.Ld[lane][t] * xt;
          if (lane + 32 < t) x1 -= sm.Ld[lane + 32][t] * xt;
        }
      }
      sm.v[q][lane] = x0;
      sm.v[q][lane + 32] = x1;
    }
    __syncthreads();
    for (int e = tid; e < TS_BS * NR; e += 256) {
      const int rr = e & 63, q = e >> 6;
      if (rr < rows && q < nrhs) {
        const T v = sm.v[q][rr];
        Yout[(int64_t)q * ldy + i0 + rr] = v;
        if (!LOWER) X[(int64_t)q * ldx + i0 + rr] = (double)v;
      }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release_s32(flags + ib, 1);
  }
}

// flags of every (block, chunk) and the ticket, then the two solution workspaces
size_t solve_scratch_bytes(int n, int tsize) {
  const int nblk = (int)cdiv(n, TS_BS);
  return 256 + (size_t)(nblk * TS_CHUNKS_MAX + 2) * sizeof(int) + 2 * (size_t)trsv_ldy(n) * TS_RHS_MAX * tsize +
         512;
}

void solve_scratch_carve(SolveScratch* s, void* base, int n, int tsize) {
  const int nblk = (int)cdiv(n, TS_BS);
  char* p = (char*)base;
  s->sync = (int*)p;
  p += ((size_t)(nblk * TS_CHUNKS_MAX + 2) * sizeof(int) + 255) / 256 * 256;
  s->y = p;
  p += ((size_t)trsv_ldy(n) * TS_RHS_MAX * tsize + 255) / 256 * 256;
  s->z = p;
  s->nblk_max = nblk;
}

// nrhs right-hand sides in nch = ceil(nrhs / NR) chunks of NR
template <typename T, int NR, bool DINV>
static cudaError_t run_solve(const T* W, int64_t ldw, const int* rowid, int n, int nrhs, const double* B,
                             int64_t ldb, double* X, int64_t ldx, const SolveScratch& s, int* status,
                             cudaStream_t st) {
  constexpr int STAGES = sizeof(T) == 8 ? 3 : 4;
  const int nblk = (int)cdiv(n, TS_BS);
  const size_t smem = sizeof(TrsvSmem<T, NR, STAGES>);
  auto kl = trsv_kernel<T, NR, STAGES, true, DINV>;
  auto ku = trsv_kernel<T, NR, STAGES, false, DINV>;
  const T* Dinv = (const T*)s.dinv;
  cudaError_t e = allow_max_smem((const void*)kl);
  if (e != cudaSuccess) return e;
  e = allow_max_smem((const void*)ku);
  if (e != cudaSuccess) return e;
  const int nch = (nrhs + NR - 1) / NR;
  if (nch > TS_CHUNKS_MAX || nrhs > TS_RHS_MAX) return cudaErrorInvalidValue;
  const int tickets = nblk * nch;
  int* flags = s.sync;
  int* ticket = s.sync + tickets;
  T* y = (T*)s.y;
  T* z = (T*)s.z;
  const int grid = (s.max_ctas > 0 && s.max_ctas < tickets) ? s.max_ctas : tickets;
  e = cudaMemsetAsync(s.sync, 0, (size_t)(tickets + 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  kl<<<grid, 256, smem, st>>>(W, ldw, n, nrhs, nch, B, ldb, rowid, nullptr, y, nullptr, 0, flags, ticket, status,
                              Dinv);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(s.sync, 0, (size_t)(tickets + 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  ku<<<grid, 256, smem, st>>>(W, ldw, n, nrhs, nch, nullptr, 0, nullptr, y, z, X, ldx, flags, ticket, status, Dinv);
  return cudaGetLastError();
}

// Inverses of the 64 x 64 diagonal blocks of L (unit lower) and U (upper):
// Dinv[(b*2 + 0)] = L_bb^-1, Dinv[(b*2 + 1)] = U_bb^-1, row-major 64 x 64,
// zero outside a ragged last block.  Thread c computes column c of each
// inverse by substitution.
template <typename T>
__global__ void __launch_bounds__(64) trinv_kernel(const T* __restrict__ W, int64_t ldw, int n, T* Dinv) {
  __shared__ T Ab[TS_BS][TS_BS + 1];
  __shared__ T Xb[TS_BS][TS_BS + 1];
  const int b = blockIdx.x, upper = blockIdx.y;
  const int i0 = b * TS_BS;
  const int bs = min(TS_BS, n - i0);
  const int c = threadIdx.x;
  for (int r = 0; r < TS_BS; ++r) Ab[r][c] = (r < bs && c < bs) ? W[(int64_t)(i0 + r) * ldw + i0 + c] : T(0);
  __syncthreads();
  for (int r = 0; r < TS_BS; ++r) Xb[r][c] = T(0);
  if (c < bs) {
    if (!upper) {
      Xb[c][c] = T(1);
      for (int r = c + 1; r < bs; ++r) {
        T sacc = T(0);
        for (int k = c; k < r; ++k) sacc += Ab[r][k] * Xb[k][c];
        Xb[r][c] = -sacc;
      }
    } else {
      Xb[c][c] = T(1) / Ab[c][c];
      for (int r = c - 1; r >= 0; --r) {
        T sacc = T(0);
        for (int k = r + 1; k <= c; ++k) sacc += Ab[r][k] * Xb[k][c];
        Xb[r][c] = -sacc / Ab[r][r];
      }
    }
  }
  __syncthreads();
  T* out = Dinv + ((int64_t)b * 2 + upper) * TS_BS * TS_BS;
  for (int r = 0; r < TS_BS; ++r) out[r * TS_BS + c] = Xb[r][c];
}

size_t solve_dinv_bytes(int n, int tsize) { return (size_t)cdiv(n, TS_BS) * 2 * TS_BS * TS_BS * tsize; }

template <typename T>
cudaError_t launch_trinv(const T* W, int64_t ldw, int n, T* Dinv, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  trinv_kernel<T><<<dim3((unsigned)cdiv(n, TS_BS), 2), 64, 0, st>>>(W, ldw, n, Dinv);
  return cudaGetLastError();
}
template cudaError_t launch_trinv<float>(const float*, int64_t, int, float*, cudaStream_t);
template cudaError_t launch_trinv<double>(const double*, int64_t, int, double*, cudaStream_t);

// One launch pair for up to 32 right-hand sides: a CTA holds up to 16 with
// FP32 factors, 8 with FP64 (whose accumulators take twice the registers);
// more are cut in chunks of that width whose chains of diagonal blocks run
// side by side in the same launches.
template <typename T>
cudaError_t launch_lu_solve(const T* W, int64_t ldw, const int* rowid, int n, int nrhs, const double* B,
                            int64_t ldb, double* X, int64_t ldx, const SolveScratch& s, int* status,
                            cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs > TS_RHS_MAX) return cudaErrorInvalidValue;
  if (((uintptr_t)W & 15u) || (ldw % (16 / sizeof(T))) != 0) return cudaErrorInvalidValue;
  constexpr int CHUNK = sizeof(T) == 4 ? 16 : 8;
  static_assert(CHUNK <= TS_NRMAX && TS_RHS_MAX / CHUNK <= TS_CHUNKS_MAX, "solve workspace holds the chunks");
  // a CTA's width: the right-hand sides rounded up to 1, 2, 4, 8 or the
  // chunk (a column's arithmetic is the same at every width)
  const bool dinv = s.dinv != nullptr && s.dinv_ready;
  if (dinv) {
    if (nrhs == 1) return run_solve<T, 1, true>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
    if (nrhs == 2) return run_solve<T, 2, true>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
    if (nrhs <= 4) return run_solve<T, 4, true>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
    if (nrhs <= 8) return run_solve<T, 8, true>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
    return run_solve<T, CHUNK, true>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  }
  if (nrhs == 1) return run_solve<T, 1, false>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  if (nrhs == 2) return run_solve<T, 2, false>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  if (nrhs <= 4) return run_solve<T, 4, false>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  if (nrhs <= 8) return run_solve<T, 8, false>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
  return run_solve<T, CHUNK, false>(W, ldw, rowid, n, nrhs, B, ldb, X, ldx, s, status, st);
}

template cudaError_t launch_lu_solve<double>(const double*, int64_t, const int*, int, int, const double*, int64_t,
                                             double*, int64_t, const SolveScratch&, int*, cudaStream_t);
template cudaError_t launch_lu_solve<float>(const float*, int64_t, const int*, int, int, const double*, int64_t,
                                            double*, int64_t, const SolveScratch&, int*, cudaStream_t);

// ============================================================ residual r = b - A x (FP64)
// Partial products over column slabs, then a fixed-order sum: deterministic.
constexpr int RS_ROWS = 256;
constexpr int RS_CHUNK = 64;

static int residual_splits(int n) {
  const int rt = (int)cdiv(n, RS_ROWS);
  int ks = (int)cdiv(608, rt);  // about four CTAs per SM in all
  const int kmax = (int)cdiv(n, RS_CHUNK);
  if (ks > kmax) ks = kmax;
  if (ks < 1) ks = 1;
  return ks;
}

size_t residual_partial_bytes(int n, int nrhs) { return (size_t)residual_splits(n) * n * (nrhs > 0 ? nrhs : 1) * 8; }

template <int NR, bool ABS>
__global__ void __launch_bounds__(RS_ROWS) residual_partial_kernel(const double* __restrict__ A, int64_t lda,
                                                                   const double* __restrict__ X, int64_t ldx, int n,
                                                                   int nrhs, int kc, double* __restrict__ partial) {
  __shared__ double xs[RS_CHUNK][NR];
  const int i = blockIdx.x * RS_ROWS + threadIdx.x;
  const int ks = blockIdx.y;
  const int c_begin = ks * kc, c_end = min(n, c_begin + kc);
  double acc[NR];
#pragma unroll
  for (int q = 0; q < NR; ++q) acc[q] = 0.0;
  for (int c0 = c_begin; c0 < c_end; c0 += RS_CHUNK) {
    const int cw = min(RS_CHUNK, c_end - c0);
    for (int e = threadIdx.x; e < RS_CHUNK * NR; e += RS_ROWS) {
      const int c = e % RS_CHUNK, q = e / RS_CHUNK;
      xs[c][q] = (c < cw && q < nrhs) ? (ABS ? 1.0 : X[(int64_t)q * ldx + c0 + c]) : 0.0;
    }
    __syncthreads();
    if (i < n) {
      for (int c = 0; c < cw; ++c) {
        double a = A[(int64_t)(c0 + c) * lda + i];
        if (ABS) a = fabs(a);
#pragma unroll
        for (int q = 0; q < NR; ++q) acc[q] = fma(a, xs[c][q], acc[q]);
      }
    }
    __syncthreads();
  }
  if (i < n) {
#pragma unroll
    for (int q = 0; q < NR; ++q)
      if (q < nrhs) partial[((int64_t)ks * nrhs + q) * n + i] = acc[q];
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

// norms layout: [0, nrhs) max|r|, [nrhs, 2 nrhs) max|x|, [2 nrhs, 3 nrhs) max|b|
__global__ void residual_finish_kernel(const double* __restrict__ partial, int ks, const double* __restrict__ X,
                                       int64_t ldx, const double* __restrict__ B, int64_t ldb, double* R,
                                       int64_t ldr, int n, int nrhs, double* norms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  double rv = 0.0, xv = 0.0, bv = 0.0;
  if (i < n) {
    double s = 0.0;
    for (int k = 0; k < ks; ++k) s += partial[((int64_t)k * nrhs + q) * n + i];
    const double b = B[(int64_t)q * ldb + i];
    const double r = b - s;
    if (R) R[(int64_t)q * ldr + i] = r;
    rv = fabs(r);
    xv = fabs(X[(int64_t)q * ldx + i]);
    bv = fabs(b);
  }
  rv = warp_max(rv);
  xv = warp_max(xv);
  bv = warp_max(bv);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(norms + q, rv);
    atomic_max_nonneg(norms + nrhs + q, xv);
    atomic_max_nonneg(norms + 2 * nrhs + q, bv);
  }
}

__global__ void rowsum_finish_kernel(const double* __restrict__ partial, int ks, int n, double* anorm) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (i < n)
    for (int k = 0; k < ks; ++k) s += partial[(int64_t)k * n + i];
  s = warp_max(s);
  if ((threadIdx.x & 31) == 0) atomic_max_nonneg(anorm, s);
}

template <int NR, bool ABS>
static cudaError_t run_partial(const double* A, int64_t lda, const double* X, int64_t ldx, int n, int nrhs, int ks,
                               double* partial, cudaStream_t st) {
  const int kc = (int)cdiv(cdiv(n, ks), RS_CHUNK) * RS_CHUNK;
  dim3 grid((unsigned)cdiv(n, RS_ROWS), (unsigned)ks);
  residual_partial_kernel<NR, ABS><<<grid, RS_ROWS, 0, st>>>(A, lda, X, ldx, n, nrhs, kc, partial);
  return cudaGetLastError();
}

cudaError_t launch_residual(const double* A, int64_t lda, const double* X, int64_t ldx, const double* B,
                            int64_t ldb, double* R, int64_t ldr, int n, int nrhs, double* partial, double* norms,
                            cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs > 32) return cudaErrorInvalidValue;
  const int ks = residual_splits(n);
  cudaError_t e;
  if (nrhs == 1)
    e = run_partial<1, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else if (nrhs <= 4)
    e = run_partial<4, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else if (nrhs <= 8)
    e = run_partial<8, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else if (nrhs <= 16)
    e = run_partial<16, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  else
    e = run_partial<32, false>(A, lda, X, ldx, n, nrhs, ks, partial, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(norms, 0, (size_t)3 * nrhs * sizeof(double), st);
  if (e != cudaSuccess) return e;
  residual_finish_kernel<<<dim3((unsigned)cdiv(n, 256), (unsigned)nrhs), 256, 0, st>>>(partial, ks, X, ldx, B, ldb,
                                                                                      R, ldr, n, nrhs, norms);
  return cudaGetLastError();
}

// max |r|, max |x|, max |b| per column of R, X, B (n x nrhs, column-major)
// into norms (layout as launch_residual), after R was formed elsewhere
__global__ void colmax3_kernel(const double* __restrict__ R, int64_t ldr, const double* __restrict__ X, int64_t ldx,
                               const double* __restrict__ B, int64_t ldb, int n, int nrhs, double* norms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  double rv = 0.0, xv = 0.0, bv = 0.0;
  if (i < n) {
    rv = fabs(R[(int64_t)q * ldr + i]);
    xv = fabs(X[(int64_t)q * ldx + i]);
    bv = fabs(B[(int64_t)q * ldb + i]);
  }
  rv = warp_max(rv);
  xv = warp_max(xv);
  bv = warp_max(bv);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(norms + q, rv);
    atomic_max_nonneg(norms + nrhs + q, xv);
    atomic_max_nonneg(norms + 2 * nrhs + q, bv);
  }
}

cudaError_t launch_colmax3(const double* R, int64_t ldr, const double* X, int64_t ldx, const double* B, int64_t ldb,
                           int n, int nrhs, double* norms, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(norms, 0, (size_t)3 * nrhs * sizeof(double), st);
  if (e != cudaSuccess) return e;
  colmax3_kernel<<<dim3((unsigned)cdiv(n, 256), (unsigned)nrhs), 256, 0, st>>>(R, ldr, X, ldx, B, ldb, n, nrhs,
                                                                               norms);
  return cudaGetLastError();
}

cudaError_t launch_norm_inf(const double* A, int64_t lda, int n, double* partial, double* anorm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int ks = residual_splits(n);
  cudaError_t e = run_partial<1, true>(A, lda, nullptr, 0, n, 1, ks, partial, st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(anorm, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  rowsum_finish_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(partial, ks, n, anorm);
  return cudaGetLastError();
}

__global__ void add_update_kernel(double* X, int64_t ldx, const double* D, int64_t ldd, int n, const int* active) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (i < n && active[q]) X[(int64_t)q * ldx + i] += D[(int64_t)q * ldd + i];
}

cudaError_t launch_add_update(double* X, int64_t ldx, const double* D, int64_t ldd, int n, int nrhs,
                              const int* active, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  add_update_kernel<<<dim3((unsigned)cdiv(n, 256), (unsigned)nrhs), 256, 0, st>>>(X, ldx, D, ldd, n, active);
  return cudaGetLastError();
}

}  // namespace gb
