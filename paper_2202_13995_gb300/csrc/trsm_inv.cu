// Top-block solve of the mixed-precision factorizations (the paper's "top"
// block update, arxiv 2202.13995 section "Base Implementation"):
//   U12 = L11^-1 A12,  L11 unit lower triangular (w x w), A12 w x N, FP32.
//
// Substitution row by row leaves the CUDA cores waiting on one short
// dependency after another.  Here every CTA first inverts L11's 32 x 32
// diagonal blocks (a warp per block, all at once, while its strip of A12 is
// still arriving), so that each block step is two small products:
//   X_b <- inv(L_bb) X_b,  then  X_r <- X_r - L_rb X_b for the rows r below,
// with the rows of L below the block staged in shared memory one block ahead
// (cp.async).  The CTA holds a strip of 32 columns of A12 in shared memory
// throughout (8 for a short solve); each thread of the update keeps a 4 x 8
// tile in registers (1 x 8 with 8 columns).
//
// Multiplying by the inverted diagonal block instead of substituting changes
// only the rounding of U12; the mixed-precision factor is refined in FP64
// afterwards.  With an operand kind the kernel also writes the solved strip
// as the trailing update's B operand (BF16 or FP16, K-major), which saves the
// separate cast of U12.
#include <cuda_runtime.h>

#include "cast16.cuh"
#include "common.cuh"
#include "kernels.h"

namespace gb {

constexpr int TI_THREADS = 256;
constexpr int TI_LDS = 33;      // row stride of staged rows of L: a column of them is conflict-free

struct TiLayout {
  int nblk;      // 32-row blocks
  int wr;        // rows rounded up to whole blocks
  int rb;        // rows of L staged per block at most (below the first block)
  int nbuf;      // staging buffers (2: the next block's rows load during this block)
  size_t xs, li, ls;  // floats
  size_t bytes;
};

// ns: columns of A12 per CTA (32, or 8 for short solves: four times the CTAs)
__host__ __device__ inline TiLayout ti_layout(int w, int kpad, int nbuf, int ns) {
  TiLayout t;
  t.nblk = (w + 31) / 32;
  t.wr = t.nblk * 32;
  t.rb = t.wr - 32;
  t.nbuf = nbuf;
  t.xs = (size_t)t.wr * ns;
  t.li = (size_t)t.nblk * 32 * TI_LDS;
  size_t ls = (size_t)nbuf * t.rb * TI_LDS;
  const size_t inv_stage = (size_t)(TI_THREADS / 32) * 32 * TI_LDS;  // each warp's copy of its diagonal block
  const size_t op = ((size_t)ns * (kpad + 2) + 1) / 2;               // the 16-bit transpose of the strip
  if (ls < inv_stage) ls = inv_stage;
  if (ls < op) ls = op;
  t.ls = ls;
  t.bytes = (t.xs + t.li + t.ls) * sizeof(float);
  return t;
}

// rows b0 + 32 .. w of L's columns b0 .. b0 + 31 -> buf[(r - b0 - 32) * TI_LDS + k]
__device__ __forceinline__ void ti_stage(const float* L, int64_t ld, int w, int b0, float* buf) {
  const int r0 = b0 + 32, R = w - r0;
  for (int e = threadIdx.x; e < R * 32; e += TI_THREADS) {
    const int rr = e >> 5, k = e & 31;
    cp_async<4>(&buf[rr * TI_LDS + k], L + (int64_t)(r0 + rr) * ld + b0 + k);
  }
}

template <int NS, typename H>
__device__ __forceinline__ bool ti_write_operand(const float* Xs, int w, int nc, int c0, H* Bop, int kpad,
                                                 unsigned short* O) {
  // transpose through shared memory: O[c * (kpad + 2) + t] (an odd word
  // stride, so a warp's 32 columns fall in 32 banks), then row-contiguous
  // 4-byte stores of each column's kpad values
  const int so = kpad + 2;
  bool bad = false;
  for (int e = threadIdx.x; e < NS * kpad; e += TI_THREADS) {
    const int c = e % NS, t = e / NS;
    const H h = to16<H>(t < w ? Xs[t * NS + c] : 0.0f);
    if (t < w && c < nc) bad |= bad16<H>(h);
    O[c * so + t] = bits16<H>(h);
  }
  __syncthreads();
  unsigned* B = reinterpret_cast<unsigned*>(Bop);
  const int hk = kpad / 2;
  for (int e = threadIdx.x; e < nc * hk; e += TI_THREADS) {
    const int c = e / hk, j = e - c * hk;
    const unsigned lo = O[c * so + 2 * j], hi = O[c * so + 2 * j + 1];
    B[(int64_t)(c0 + c) * hk + j] = lo | (hi << 16);
  }
  return bad;
}

template <int NS>
__global__ void __launch_bounds__(TI_THREADS) trsm_inv_kernel(const float* __restrict__ L, float* X, int64_t ld,
                                                              int w, int N, int nbuf, int kind, void* Bop, int kpad,
                                                              int* status) {
  static_assert(NS == 32 || NS == 8, "strip widths");
  constexpr int TQ = NS / 4;              // 16-byte pieces per strip row
  constexpr int RT = NS == 32 ? 4 : 1;    // rows per update tile (tiles are RT x 8)
  constexpr int CG = NS / 8;              // 8-column groups per strip
  extern __shared__ __align__(16) float smf[];
  const TiLayout lay = ti_layout(w, kind ? kpad : 0, nbuf, NS);
  float* Xs = smf;            // [wr][NS]: the strip of A12, solved in place
  float* Li = Xs + lay.xs;    // [nblk][32][33]: inverses of the diagonal blocks
  float* Ls = Li + lay.li;    // staged rows of L (also the inversion's copies and the operand transpose)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int c0 = blockIdx.x * NS;
  const int nc = min(NS, N - c0);

  // 1. the strip -> Xs (rows past w and columns past N zero)
  const bool vec = nc == NS && ((reinterpret_cast<uintptr_t>(X + c0) & 15) == 0) && (ld % 4) == 0;
  for (int e = tid; e < lay.wr * TQ; e += TI_THREADS) {
    const int r = e / TQ, q = (e % TQ) * 4;
    float* dst = &Xs[r * NS + q];
    if (r < w && vec) {
      cp_async<16>(dst, X + (int64_t)r * ld + c0 + q);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) dst[i] = (r < w && q + i < nc) ? X[(int64_t)r * ld + c0 + q + i] : 0.0f;
    }
  }
  cp_async_commit();

  // 2. inverses of the unit-lower diagonal blocks: warp per block, lane = a
  //    column j of the inverse Z, by Z[t][j] = -sum_{s<t} L[t][s] Z[s][j]
  //    (Z[s][j] = 0 for s < j, Z[j][j] = 1); padding rows of a partial last
  //    block invert to the identity
  for (int bi = warp; bi < lay.nblk; bi += TI_THREADS / 32) {
    const int b0 = bi * 32, bw = min(32, w - b0);
    float* D = Ls + warp * 32 * TI_LDS;
    {
      float v[32];  // all 32 loads in flight together (the strip's copies keep going)
#pragma unroll
      for (int t = 0; t < 32; ++t) v[t] = (t < bw && lane < t) ? __ldg(L + (int64_t)(b0 + t) * ld + b0 + lane) : 0.0f;
#pragma unroll
      for (int t = 0; t < 32; ++t) D[t * TI_LDS + lane] = v[t];
    }
    __syncwarp();
    float* Z = Li + bi * 32 * TI_LDS;
    for (int t = 0; t < 32; ++t) Z[t * TI_LDS + lane] = t == lane ? 1.0f : 0.0f;
    // eight terms at a time with their loads ahead of the products (D[t][s]
    // = 0 for s >= t, and rows of Z below the diagonal not yet computed are
    // still zero)
    for (int t = 1; t < 32; ++t) {
      float v[4] = {0.0f, 0.0f, 0.0f, 0.0f};
      for (int s0 = 0; s0 < t; s0 += 8) {
        float dv[8], zv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          dv[u] = D[t * TI_LDS + s0 + u];
          zv[u] = Z[(s0 + u) * TI_LDS + lane];
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u & 3] = fmaf(-dv[u], zv[u], v[u & 3]);
      }
      if (t > lane) Z[t * TI_LDS + lane] = (v[0] + v[1]) + (v[2] + v[3]);
    }
    __syncwarp();
  }
  cp_async_wait_group<0>();
  __syncthreads();

  const int rbs = lay.rb * TI_LDS;
  if (nbuf == 2 && lay.nblk > 1) ti_stage(L, ld, w, 0, Ls);
  cp_async_commit();

  for (int b = 0; b < lay.nblk; ++b) {
    const int b0 = b * 32, bw = min(32, w - b0);
    float* cur = Ls + (nbuf == 2 ? (b & 1) * rbs : 0);
    if (nbuf == 1) {
      ti_stage(L, ld, w, b0, cur);  // the single buffer was last read before the previous block's final barrier
      cp_async_commit();
    }
    // (i) X_b <- Z_b X_b: thread = one row t, four columns
    {
      const int t = tid / TQ, cq = (tid % TQ) * 4;
      const bool act = t < 32;
      const float* Z = Li + b * 32 * TI_LDS;
      float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
      for (int s = 0; act && s < bw; ++s) {  // Z[t][s] = 0 for s > t
        const float z = Z[t * TI_LDS + s];
        const float4 x = *reinterpret_cast<const float4*>(&Xs[(b0 + s) * NS + cq]);
        a0 = fmaf(z, x.x, a0);
        a1 = fmaf(z, x.y, a1);
        a2 = fmaf(z, x.z, a2);
        a3 = fmaf(z, x.w, a3);
      }
      __syncthreads();  // every thread has read X_b
      if (act && t < bw) *reinterpret_cast<float4*>(&Xs[(b0 + t) * NS + cq]) = make_float4(a0, a1, a2, a3);
    }
    if (nbuf == 2) {
      // the next block's rows go to the other buffer, last read in the
      // previous block's update (finished at its final barrier)
      if (b + 1 < lay.nblk) ti_stage(L, ld, w, b0 + 32, Ls + ((b + 1) & 1) * rbs);
      cp_async_commit();
      cp_async_wait_group<1>();  // this block's rows have landed
    } else {
      cp_async_wait_group<0>();
    }
    __syncthreads();
    // (ii) rows below: X_r -= L_rb X_b; item = RT rows x 8 columns
    const int R = w - b0 - 32;
    if (R > 0) {
      const int Rp = (R + RT - 1) / RT * RT;
      const float* xb = Xs + b0 * NS;
      for (int it = tid; it < Rp / RT * CG; it += TI_THREADS) {
        const int rg = it / CG, cg = it % CG;
        const float* lr = cur + RT * rg * TI_LDS;
        float acc[RT][8];
#pragma unroll
        for (int i = 0; i < RT; ++i)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[i][q] = 0.0f;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
          const float4 x0 = *reinterpret_cast<const float4*>(&xb[k * NS + 8 * cg]);
          const float4 x1 = *reinterpret_cast<const float4*>(&xb[k * NS + 8 * cg + 4]);
          const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
          for (int i = 0; i < RT; ++i) {
            const float l = lr[i * TI_LDS + k];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[i][q] = fmaf(l, xv[q], acc[i][q]);
          }
        }
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          const int r = b0 + 32 + RT * rg + i;
          if (r < w) {
            float4* p = reinterpret_cast<float4*>(&Xs[r * NS + 8 * cg]);
            float4 u = p[0], v = p[1];
            u.x -= acc[i][0]; u.y -= acc[i][1]; u.z -= acc[i][2]; u.w -= acc[i][3];
            v.x -= acc[i][4]; v.y -= acc[i][5]; v.z -= acc[i][6]; v.w -= acc[i][7];
            p[0] = u;
            p[1] = v;
          }
        }
      }
    }
    __syncthreads();
  }

  // 3. the solved strip back to A12, and the B operand
  for (int e = tid; e < w * TQ; e += TI_THREADS) {
    const int r = e / TQ, q = (e % TQ) * 4;
    if (vec) {
      *reinterpret_cast<float4*>(X + (int64_t)r * ld + c0 + q) = *reinterpret_cast<const float4*>(&Xs[r * NS + q]);
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (q + i < nc) X[(int64_t)r * ld + c0 + q + i] = Xs[r * NS + q + i];
    }
  }
  if (kind != 0) {
    unsigned short* O = reinterpret_cast<unsigned short*>(Ls);
    const bool bad = kind == 1 ? ti_write_operand<NS, __nv_bfloat16>(Xs, w, nc, c0, (__nv_bfloat16*)Bop, kpad, O)
                               : ti_write_operand<NS, __half>(Xs, w, nc, c0, (__half*)Bop, kpad, O);
    if (__syncthreads_or(bad) && tid == 0) atomicOr(status, ST_RANGE);
  }
}

cudaError_t launch_trsm_inv(const float* L11, float* A12, int64_t ldw, int w, int N, int kind, void* Bop, int kpad,
                            int* status, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  if (w < 1 || w > 512) return cudaErrorInvalidValue;
  if (kind != 0 && (kind > 2 || Bop == nullptr || status == nullptr || kpad < w || (kpad % 64) != 0 ||
                    ((uintptr_t)Bop & 3u)))
    return cudaErrorInvalidValue;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  // A short solve (fewer 32-column strips than half the SMs: the next
  // panel's columns) takes strips of 8 columns, four times the CTAs for the
  // same chain of blocks.  A grid of one wave loads the next block's rows
  // during this block (two buffers); a larger grid keeps one buffer, so that
  // two CTAs fit an SM and each hides the other's waits.
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ns = cdiv(N, 32) < sms / 2 ? 8 : 32;
  const bool one_wave = cdiv(N, ns) <= sms;
  TiLayout lay = ti_layout(w, kind ? kpad : 0, one_wave ? 2 : 1, ns);
  if (lay.bytes > (size_t)optin) lay = ti_layout(w, kind ? kpad : 0, 1, ns);
  if (lay.bytes > (size_t)optin) return cudaErrorInvalidValue;
  const void* kern = ns == 8 ? (const void*)trsm_inv_kernel<8> : (const void*)trsm_inv_kernel<32>;
  cudaError_t e = allow_max_smem(kern);
  if (e != cudaSuccess) return e;
  if (ns == 8)
    trsm_inv_kernel<8><<<(unsigned)cdiv(N, 8), TI_THREADS, lay.bytes, st>>>(L11, A12, ldw, w, N, lay.nbuf, kind, Bop,
                                                                            kpad, status);
  else
    trsm_inv_kernel<32><<<(unsigned)cdiv(N, 32), TI_THREADS, lay.bytes, st>>>(L11, A12, ldw, w, N, lay.nbuf, kind,
                                                                              Bop, kpad, status);
  return cudaGetLastError();
}

}  // namespace gb
