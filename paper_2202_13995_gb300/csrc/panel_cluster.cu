// FP32 panel factorization with partial pivoting on one thread-block cluster.
//
// The same computation as panel_getrf_kernel (the paper's diagonal and left
// blocks of a block iteration, factored together because partial pivoting
// searches every row below the diagonal; arxiv 2202.13995, section "Base
// Implementation"): for each column j, p = the first row of largest |a| at or
// below j, swap rows j and p, divide the entries below the diagonal by the
// pivot, rank-1 update of the columns to the right.
//
// The grid is one cluster of CL <= 16 CTAs (512 threads each); CTA c owns the
// panel rows [c R, c R + R).  Per column, the candidates are exchanged
// through distributed shared memory: every CTA publishes its best (|a|, row)
// and that row's sub-panel values in its own shared memory, the cluster
// barrier (release/acquire, cluster scope) follows, and every CTA reads all
// peers' candidates in one round of DSMEM loads.  That replaces the grid
// barrier and the L2 round trips of the cooperative kernel.
//
// The panel is processed in sub-panels of 16 columns.  A thread owns up to 4
// rows (tid + 512 q) of the sub-panel; the part of a row still being updated
// sits in registers, rotated so that the current column is always register 0
// (every register index is a compile-time constant and one copy of the column
// code serves all columns), and the finished part of every row goes to shared
// memory (Ls), where the sub-panel is whole when its last column is done.  After a sub-panel: its
// values are written back, its row interchanges are applied to the panel's
// other columns (columns distributed over the CTAs), every CTA solves the
// sub-panel's top rows of the columns to its right (U rows, into shared
// memory), and each CTA updates its own rows of those columns (a rank-16
// update, coalesced along the row, U in registers).  Three cluster
// synchronizations per sub-panel, one per column.
//
// The kernel spins on nothing: its only waits are hardware cluster barriers,
// and every CTA executes the same sequence of them (no CTA leaves early, the
// loop bounds are the same in all), so each one completes.
#include <climits>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "kernels.h"
#include "permrec.cuh"

namespace gb {

constexpr int PC_THREADS = 512;
constexpr int PC_WARPS = PC_THREADS / 32;
constexpr int PC_IB = 16;
constexpr int PC_RPT = 4;          // rows per thread at most: R <= 2048
constexpr int PC_CLMAX = 16;
constexpr int PC_WMAX = 512;
constexpr int PC_HF = 2048;        // hash buckets: rows outside the panel's top w rows
constexpr int PC_HS = 128;         // hash buckets: rows outside a sub-panel's top rows

struct alignas(16) PcSmem {
  float slot[2][2 + PC_IB];  // |a|, row (bits), the row's sub-panel values
  float rowj[2][PC_IB];      // row j's sub-panel values (its owner CTA)
  float stg[PC_WARPS][PC_IB];
  float redv[PC_WARPS];
  int redi[PC_WARPS];
  float xs[PC_CLMAX][2 + PC_IB];  // every CTA's slot, read through DSMEM
  float rj[PC_IB];
  int cnt[2];  // permutation record counts: whole panel, sub-panel
  float L11[PC_IB][PC_IB + 1];
  int fpos[2 * PC_WMAX], fcur[2 * PC_WMAX];
  int spos[2 * PC_IB], scur[2 * PC_IB];
  int hfk[PC_HF], hfv[PC_HF];
  int hsk[PC_HS], hsv[PC_HS];
  float U[PC_IB][PC_WMAX];
};

struct PcParams {
  float* A;  // W(k, k)
  int64_t ld;
  int m, w, R;
  int kabs;
  int* ipiv;
  int* info;
  int* status;
  int* perm;
};

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cl_map(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ float cl_ldf(uint32_t addr) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(addr) : "memory");
  return v;
}
__device__ __forceinline__ void cl_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t sm_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// v[q][c] for a run-time q, by predicated selects: an indexed read would move
// the whole register tile to local memory.
static_assert(PC_RPT == 4, "pc_pick selects among four rows");
__device__ __forceinline__ float pc_pick(const float (&v)[PC_RPT][PC_IB], int c, int q) {
  float x = v[0][c];
  asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %2, 1;\n\tselp.f32 %0, %1, %0, p;\n\t}" : "+f"(x) : "f"(v[1][c]), "r"(q));
  asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %2, 2;\n\tselp.f32 %0, %1, %0, p;\n\t}" : "+f"(x) : "f"(v[2][c]), "r"(q));
  asm("{\n\t.reg .pred p;\n\tsetp.eq.s32 p, %2, 3;\n\tselp.f32 %0, %1, %0, p;\n\t}" : "+f"(x) : "f"(v[3][c]), "r"(q));
  return x;
}

// Cluster synchronization (the hardware cluster barrier, release/acquire at
// cluster scope): this CTA's prior writes, shared and global, become visible
// to every peer, and the peers' to this CTA.  Every CTA runs the same
// sequence of synchronizations (the loop bounds are the same in all), so the
// barrier always completes.
#define PC_CSYNC() cl_barrier()

__global__ void __launch_bounds__(PC_THREADS, 1) panel_cluster_kernel(PcParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PcSmem& S = *reinterpret_cast<PcSmem*>(smem_raw);
  float* Ls = reinterpret_cast<float*>(smem_raw + sizeof(PcSmem));  // [R][PC_IB]: the sub-panel's L rows
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta = (int)cl_rank(), CL = (int)gridDim.x;
  const int R = P.R, w = P.w;
  const int64_t ld = P.ld;
  const int row0 = cta * R;
  const int rloc = max(0, min(P.m, row0 + R) - row0);
  float* A = P.A;

  for (int s = tid; s < w; s += PC_THREADS) {
    S.fpos[s] = s;
    S.fcur[s] = s;
  }
  for (int s = tid; s < PC_HF; s += PC_THREADS) S.hfk[s] = -1;
  if (tid == 0) S.cnt[0] = w;
  __syncthreads();
  cl_barrier();  // every peer has started before any DSMEM access
  const PermRec fperm{S.fpos, S.fcur, S.hfk, S.hfv, PC_HF - 1, 0, w, &S.cnt[0]};

  float v[PC_RPT][PC_IB];
  // 16-byte row segments: the tile moves in float4 when the rows allow it
  const bool aligned = ((uintptr_t)A & 15u) == 0 && (ld % 4) == 0;
  for (int j0 = 0; j0 < w; j0 += PC_IB) {
    const int ibs = min(PC_IB, w - j0);
    const bool vec = aligned && ibs == PC_IB;
    // ---- the sub-panel's rows into registers
#pragma unroll
    for (int q = 0; q < PC_RPT; ++q) {
      const int r = tid + PC_THREADS * q;
#pragma unroll
      for (int c = 0; c < PC_IB; ++c) v[q][c] = 0.f;
      if (r < rloc) {
        const float* src = A + (int64_t)(row0 + r) * ld + j0;
        if (vec) {
#pragma unroll
          for (int u = 0; u < PC_IB / 4; ++u) {
            const float4 x = __ldcg(reinterpret_cast<const float4*>(src) + u);
            v[q][4 * u] = x.x;
            v[q][4 * u + 1] = x.y;
            v[q][4 * u + 2] = x.z;
            v[q][4 * u + 3] = x.w;
          }
        } else {
#pragma unroll
          for (int c = 0; c < PC_IB; ++c)
            if (c < ibs) v[q][c] = __ldcg(src + c);
        }
      }
    }
    // every row's sub-panel values also start in Ls (rows above the
    // sub-panel keep them; the others are overwritten as they finish)
#pragma unroll
    for (int q = 0; q < PC_RPT; ++q) {
      const int r = tid + PC_THREADS * q;
      if (r < rloc) {
        float4* lsv = reinterpret_cast<float4*>(Ls + r * PC_IB);
#pragma unroll
        for (int u = 0; u < PC_IB / 4; ++u) lsv[u] = make_float4(v[q][4 * u], v[q][4 * u + 1], v[q][4 * u + 2], v[q][4 * u + 3]);
      }
    }
    for (int s = tid; s < ibs; s += PC_THREADS) {
      S.spos[s] = j0 + s;
      S.scur[s] = j0 + s;
    }
    for (int s = tid; s < PC_HS; s += PC_THREADS) S.hsk[s] = -1;
    if (tid == 0) S.cnt[1] = ibs;
    __syncthreads();
    const PermRec sperm{S.spos, S.scur, S.hsk, S.hsv, PC_HS - 1, j0, j0 + ibs, &S.cnt[1]};

    // local candidate of the sub-panel's first column
    float bv = -1.f;
    int bi = INT_MAX, bq = 0;
#pragma unroll
    for (int q = 0; q < PC_RPT; ++q) {
      const int r = tid + PC_THREADS * q;
      if (r < rloc && row0 + r >= j0) {
        const float a = pivot_mag(v[q][0]);
        if (a > bv || (a == bv && row0 + r < bi)) {
          bv = a;
          bi = row0 + r;
          bq = q;
        }
      }
    }
#pragma unroll 1
    for (int J = 0; J < ibs; ++J) {
      const int jg = j0 + J;
      const int par = jg & 1;
      // ---- 1. this CTA's candidate and its row; row jg from its owner.  A
      //      published row is whole: its finished part from Ls, the rest
      //      from the (rotated) registers.
      if (!(bv < INFINITY)) atomicOr(P.status, ST_RANGE);  // a non-finite candidate
      float wv = bv;
      int wi = bi;
      warp_argmax(wv, wi);
      if (wi != INT_MAX && bi == wi) {
        const int r = wi - row0;
        for (int c = 0; c < J; ++c) S.stg[warp][c] = Ls[r * PC_IB + c];
#pragma unroll
        for (int k = 0; k < PC_IB; ++k)
          if (J + k < PC_IB) S.stg[warp][J + k] = pc_pick(v, k, bq);
      }
      if (lane == 0) {
        S.redv[warp] = wv;
        S.redi[warp] = wi;
      }
      {
        const int lr = jg - row0;
        if (lr >= 0 && lr < rloc && (lr % PC_THREADS) == tid) {
          for (int c = 0; c < J; ++c) S.rowj[par][c] = Ls[lr * PC_IB + c];
#pragma unroll
          for (int k = 0; k < PC_IB; ++k)
            if (J + k < PC_IB) S.rowj[par][J + k] = pc_pick(v, k, lr / PC_THREADS);
        }
      }
      __syncthreads();
      if (warp == 0) {
        float cv = lane < PC_WARPS ? S.redv[lane] : -1.f;
        int ci = lane < PC_WARPS ? S.redi[lane] : INT_MAX;
        warp_argmax(cv, ci);
        const unsigned mk = __ballot_sync(0xffffffffu, lane < PC_WARPS && ci != INT_MAX && S.redi[lane] == ci);
        const int ww = mk ? __ffs(mk) - 1 : 0;
        if (lane == 0) {
          S.slot[par][0] = cv;
          S.slot[par][1] = __int_as_float(ci);
        }
        if (lane < PC_IB) S.slot[par][2 + lane] = ci != INT_MAX ? S.stg[ww][lane] : 0.f;
      }
      // ---- 2. exchange: every CTA's slot and row jg in one round of DSMEM reads
      PC_CSYNC();
      if (tid < CL * (2 + PC_IB)) {
        const int c_ = tid / (2 + PC_IB), k_ = tid % (2 + PC_IB);
        S.xs[c_][k_] = cl_ldf(cl_map(sm_u32(&S.slot[par][k_]), (uint32_t)c_));
      } else if (tid >= 320 && tid < 320 + PC_IB) {
        S.rj[tid - 320] = cl_ldf(cl_map(sm_u32(&S.rowj[par][tid - 320]), (uint32_t)(jg / R)));
      }
      __syncthreads();
      int p, cc = 0;
      {
        float cv = -1.f;
        int ci = INT_MAX;
        for (int c_ = 0; c_ < CL; ++c_) {
          const float v_ = S.xs[c_][0];
          const int i_ = __float_as_int(S.xs[c_][1]);
          if (v_ > cv || (v_ == cv && i_ < ci)) {
            cv = v_;
            ci = i_;
            cc = c_;
          }
        }
        p = ci;
      }
      const float* prow = p != INT_MAX ? &S.xs[cc][2] : S.rj;  // the whole pivot row
      if (p == INT_MAX) p = jg;  // no candidate at all (cannot happen: row jg is one)
      float pr[PC_IB];  // its part from column J on, rotated like the registers
#pragma unroll
      for (int k = 0; k < PC_IB; ++k) pr[k] = J + k < PC_IB ? prow[J + k] : 0.f;
      const float piv = pr[0];
      if (tid == 0) {
        if (cta == 0) {
          P.ipiv[P.kabs + jg] = P.kabs + p + 1;
          if (piv == 0.f) atomicMin(P.info, P.kabs + jg + 1);
        }
        if (p != jg) {
          if (cta == 0) fperm.swap_rows(jg, p);
          sperm.swap_rows(jg, p);
        }
      }
      // ---- 3. swap, scale (a division, as in the definition), rank-1
      //      update, rotation, and the next column's local candidate
      bv = -1.f;
      bi = INT_MAX;
      bq = 0;
#pragma unroll
      for (int q = 0; q < PC_RPT; ++q) {
        const int r = tid + PC_THREADS * q;
        const int rg = row0 + r;
        if (r < rloc) {
          if (p != jg && rg == p) {
            // row p takes row jg: its finished part and its current part
            for (int c = 0; c < J; ++c) Ls[r * PC_IB + c] = S.rj[c];
#pragma unroll
            for (int k = 0; k < PC_IB; ++k) v[q][k] = J + k < PC_IB ? S.rj[J + k] : 0.f;
          }
          if (rg == jg) {
            // the pivot row is final from here on
            for (int c = 0; c < PC_IB; ++c) Ls[r * PC_IB + c] = prow[c];
          }
          if (rg > jg) {
            float l = v[q][0];
            if (piv != 0.f) l = l / piv;
            Ls[r * PC_IB + J] = l;
#pragma unroll
            for (int k = 1; k < PC_IB; ++k) v[q][k] -= l * pr[k];
#pragma unroll
            for (int k = 0; k + 1 < PC_IB; ++k) v[q][k] = v[q][k + 1];
            v[q][PC_IB - 1] = 0.f;
            if (J + 1 < ibs) {
              const float a = pivot_mag(v[q][0]);
              if (a > bv || (a == bv && rg < bi)) {
                bv = a;
                bi = rg;
                bq = q;
              }
            }
          }
        }
      }
    }
    __syncthreads();

    // ---- (a) the sub-panel (whole in Ls) back to memory
#pragma unroll
    for (int q = 0; q < PC_RPT; ++q) {
      const int r = tid + PC_THREADS * q;
      if (r < rloc) {
        float* dst = A + (int64_t)(row0 + r) * ld + j0;
        const float4* lsv = reinterpret_cast<const float4*>(Ls + r * PC_IB);
        if (vec) {
#pragma unroll
          for (int u = 0; u < PC_IB / 4; ++u) reinterpret_cast<float4*>(dst)[u] = lsv[u];
        } else {
          for (int c = 0; c < ibs; ++c) dst[c] = Ls[r * PC_IB + c];
        }
      }
    }
    PC_CSYNC();
    // ---- (b) the sub-panel's interchanges on the panel's other columns:
    //      column o of the others goes to CTA o mod CL; a CTA reads every
    //      source row of a column before writing any destination row
    const int nout = w - ibs;
    const int scnt = S.cnt[1];
    for (int kb = 0; cta + CL * kb < nout; kb += PC_THREADS / 32) {
      const int o = cta + CL * (kb + tid / 32);
      const int s = tid % 32;
      const bool act = o < nout && s < scnt;
      const int c = o < j0 ? o : o + ibs;
      float val = 0.f;
      if (act) val = __ldcg(A + (int64_t)S.scur[s] * ld + c);
      __syncthreads();
      if (act) A[(int64_t)S.spos[s] * ld + c] = val;
      __syncthreads();
    }
    PC_CSYNC();
    const int nr = w - j0 - ibs;  // columns to the right of the sub-panel
    if (nr > 0) {
      // ---- (c) U rows of the right columns: L11^-1 A12, every CTA for itself
      for (int e = tid; e < ibs * ibs; e += PC_THREADS) {
        const int t = e / ibs, s = e % ibs;
        S.L11[t][s] = __ldcg(A + (int64_t)(j0 + t) * ld + j0 + s);
      }
      for (int e = tid; e < ibs * nr; e += PC_THREADS) {
        const int t = e / nr, c = e % nr;
        S.U[t][c] = __ldcg(A + (int64_t)(j0 + t) * ld + j0 + ibs + c);
      }
      __syncthreads();
      for (int c = tid; c < nr; c += PC_THREADS) {
        for (int t = 1; t < ibs; ++t) {
          float x = S.U[t][c];
          for (int s = 0; s < t; ++s) x -= S.L11[t][s] * S.U[s][c];
          S.U[t][c] = x;
        }
      }
    }
    PC_CSYNC();  // every CTA has read the top rows before their owners overwrite them
    if (nr > 0) {
      // ---- (d) own rows: top rows take U; rows below get the rank-ibs
      //      update.  A warp takes rows; a lane takes 4 columns 32 apart per
      //      pass, with their U column in registers (4 FMAs per shared-memory
      //      load of the row's L value), the next row's values loaded ahead.
      for (int r = warp; r < rloc; r += PC_WARPS) {
        const int rg = row0 + r;
        if (rg >= j0 && rg < j0 + ibs) {
          float* rowp = A + (int64_t)rg * ld + j0 + ibs;
          for (int c = lane; c < nr; c += 32) rowp[c] = S.U[rg - j0][c];
        }
      }
      const int rfirst = max(0, j0 + ibs - row0);  // first own row below the sub-panel
      constexpr int D = 2;                         // rows per step (and rows of loads in flight)
      for (int cb = 0; cb < nr; cb += 128) {
        float u[PC_IB][4];
#pragma unroll
        for (int t = 0; t < PC_IB; ++t)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const int c = cb + lane + 32 * k;
            u[t][k] = (t < ibs && c < nr) ? S.U[t][c] : 0.f;
          }
        bool cok[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) cok[k] = cb + lane + 32 * k < nr;
        auto load_rows = [&](int rb, float (&x)[D][4]) {
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const int r = rb + PC_WARPS * d;
            const float* rp = A + (int64_t)(row0 + r) * ld + j0 + ibs + cb + lane;
#pragma unroll
            for (int k = 0; k < 4; ++k) x[d][k] = (r < rloc && cok[k]) ? __ldcg(rp + 32 * k) : 0.f;
          }
        };
        float a[D][4], an[D][4];
        int rb = rfirst + warp;
        load_rows(rb, a);
        for (; rb < rloc; rb += PC_WARPS * D) {
          load_rows(rb + PC_WARPS * D, an);  // the next rows' values in flight
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const int r = rb + PC_WARPS * d;
            if (r < rloc) {
              const float4* lr4 = reinterpret_cast<const float4*>(Ls + r * PC_IB);
#pragma unroll
              for (int t4 = 0; t4 < PC_IB / 4; ++t4) {
                const float4 l4 = lr4[t4];
                const float lt[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int tt = 0; tt < 4; ++tt) {
                  if (4 * t4 + tt < ibs) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) a[d][k] -= lt[tt] * u[4 * t4 + tt][k];
                  }
                }
              }
              float* rowp = A + (int64_t)(row0 + r) * ld + j0 + ibs + cb + lane;
#pragma unroll
              for (int k = 0; k < 4; ++k)
                if (cok[k]) rowp[32 * k] = a[d][k];
            }
          }
#pragma unroll
          for (int d = 0; d < D; ++d)
#pragma unroll
            for (int k = 0; k < 4; ++k) a[d][k] = an[d][k];
        }
      }
    }
    __syncthreads();
  }

  // ---- whole-panel permutation for the row interchanges outside the panel
  if (cta == 0) {
    __syncthreads();
    const int fcnt = S.cnt[0];
    if (tid == 0) P.perm[0] = fcnt;
    for (int s = tid; s < fcnt; s += PC_THREADS) {
      P.perm[1 + s] = S.fpos[s];
      P.perm[1 + 2 * w + s] = S.fcur[s];
    }
  }
  cl_barrier();  // no CTA leaves while a peer may still read its shared memory
}

#undef PC_COLUMN
#undef PC_CSYNC

// The cluster of a panel: up to 16 CTAs of at most 2048 rows each, at least
// 256 rows per CTA; -1 when the panel does not fit this kernel.
int panel_cluster_size(int m, int w) {
  if (w < 1 || w > PC_WMAX || m < w) return -1;
  int cl = (m + 255) / 256;
  if (cl > PC_CLMAX) cl = PC_CLMAX;
  if (cl < 1) cl = 1;
  const int R = (m + cl - 1) / cl;
  if (R > PC_RPT * PC_THREADS) return -1;
  return cl;
}

cudaError_t launch_panel_cluster(float* Wkk, int64_t ldw, int m, int w, int kabs, int* ipiv, int* info, int* status,
                                 int* perm, cudaStream_t st) {
  const int cl = panel_cluster_size(m, w);
  if (cl < 0) return cudaErrorInvalidConfiguration;
  const int R = (m + cl - 1) / cl;
  const size_t smem = sizeof(PcSmem) + (size_t)R * PC_IB * sizeof(float);
  cudaError_t e = allow_max_smem((const void*)panel_cluster_kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute((const void*)panel_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  PcParams P;
  P.A = Wkk;
  P.ld = ldw;
  P.m = m;
  P.w = w;
  P.R = R;
  P.kabs = kabs;
  P.ipiv = ipiv;
  P.info = info;
  P.status = status;
  P.perm = perm;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl);
  cfg.blockDim = dim3(PC_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cl;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, panel_cluster_kernel, P);
}

// Whether a cluster of `cl` such CTAs can be placed on this device.
bool panel_cluster_available(int m, int w) {
  const int cl = panel_cluster_size(m, w);
  if (cl < 0) return false;
  static std::mutex mu;
  static int known[PC_CLMAX + 1] = {};  // 0 unknown, 1 yes, -1 no
  std::lock_guard<std::mutex> lk(mu);
  if (known[cl] == 0) {
    allow_max_smem((const void*)panel_cluster_kernel);
    cudaFuncSetAttribute((const void*)panel_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    const int R = PC_RPT * PC_THREADS;  // the largest shared-memory need
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cl);
    cfg.blockDim = dim3(PC_THREADS);
    cfg.dynamicSmemBytes = sizeof(PcSmem) + (size_t)R * PC_IB * sizeof(float);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    const cudaError_t e = cudaOccupancyMaxActiveClusters(&n, (const void*)panel_cluster_kernel, &cfg);
    if (e != cudaSuccess) cudaGetLastError();
    known[cl] = (e == cudaSuccess && n > 0) ? 1 : -1;
  }
  return known[cl] > 0;
}

}  // namespace gb
