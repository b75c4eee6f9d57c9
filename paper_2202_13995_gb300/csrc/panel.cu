// Panel factorization with partial pivoting, row interchanges (laswp), the
// top-block triangular solve (trsm) and the layout conversions.
//
// Method: the paper's blocked right-looking LU (arxiv 2202.13995, section
// "Base Implementation", figure "lu_iteration") factors the diagonal block,
// then updates the "top" blocks with L and the "left" blocks with U.  With
// partial pivoting the pivot of a column is searched over every row below the
// diagonal, so the diagonal block and the left blocks are factored together
// as one m x w panel here (LAPACK's dgetrf structure).
//
// The working matrix W is row-major (see kernels.h).
#include <chrono>
#include <climits>
#include <mutex>
#include <set>
#include <thread>
#include <utility>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "kernels.h"
#include "permrec.cuh"

namespace gb {

cudaError_t allow_max_smem(const void* func) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({func, dev})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, func);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({func, dev});
  return e;
}

template <typename T>
__device__ __forceinline__ T tabs(T v) {
  return v < T(0) ? -v : v;
}

// ============================================================ panel getrf
//
// One cooperative launch factors the whole panel.  CTA c owns the contiguous
// rows [c*R, c*R + R) of the panel.  The panel is processed in sub-panels of
// ib (<= 32) columns; a sub-panel's rows are held in shared memory, so each
// column step costs one grid barrier:
//   1. every CTA finds the first row of largest |a| among its rows >= j and
//      publishes (|a|, row) and that row's sub-panel values;
//   2. grid barrier;
//   3. every CTA reduces the G candidates (largest |a|, then lowest row) to
//      the pivot p, swaps rows j and p inside its tile where it owns them,
//      scales its column entries below j by 1/pivot (a division, as in the
//      definition) and applies the rank-1 update to the sub-panel columns.
// After a sub-panel, its interchanges are applied to the other panel columns,
// the sub-panel's L block solves the top rows of the panel columns to its
// right, and every CTA updates its own rows of those columns (a rank-ib GEMM).

constexpr int PNL_THREADS = 256;
constexpr int PNL_WARPS = PNL_THREADS / 32;
constexpr int PNL_IB = 32;
// After each column's barrier every CTA reads all candidate rows at once
// (one L2 round trip); up to PNL_XG CTAs.
constexpr int PNL_XG = kPanelMaxCtas;
constexpr int PNL_XQ = PNL_XG * PNL_IB / PNL_THREADS;  // candidate values per thread
constexpr int PNL_HF = 2048;  // hash buckets: rows outside the panel's top w rows
constexpr int PNL_HS = 128;   // hash buckets: rows outside a sub-panel's top rows

template <typename T>
struct PanelParams {
  T* A;  // W(k, k)
  int64_t ld;
  int m, w, ib, R, G;
  int kabs;
  int* ipiv;  // absolute ipiv array (entries kabs .. kabs + w written)
  int* info;
  int* status;
  unsigned* bar;
  T* xval;
  int* xidx;
  T* xrow;
  T* xrowj;
  int* perm;
  const int* spec;  // diagonal-pivot check flags (SpecArgs), or null
  const T* spec_backup;
};

__host__ __device__ inline size_t panel_smem_bytes(int R, int ib, int w, int tsize) {
  const int Rs = R | 1;
  size_t tcount = (size_t)ib * Rs + (size_t)ib * ib + (size_t)ib * 32 + 2 * (size_t)ib * 32 + PNL_WARPS +
                  (size_t)PNL_XG * ib;
  size_t icount = PNL_WARPS + 4 * (size_t)w + 4 * (size_t)ib + 2 * PNL_HF + 2 * PNL_HS + 8;
  return tcount * tsize + icount * sizeof(int) + 16;
}

template <typename T>
__global__ void __launch_bounds__(PNL_THREADS) panel_getrf_kernel(PanelParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cta = blockIdx.x;
  const int G = P.G, R = P.R, Rs = R | 1, ib = P.ib, w = P.w;
  const int64_t ld = P.ld;
  const int row0 = cta * R;
  const int rloc = max(0, min(P.m, row0 + R) - row0);

  T* S = reinterpret_cast<T*>(smem_raw);  // [ib][Rs]: column t of the tile, row r
  T* Lsub = S + (size_t)ib * Rs;          // [ib][ib] unit-lower block of the sub-panel
  T* Ust = Lsub + ib * ib;                // [ib][32] U rows for the in-panel update
  T* stage = Ust + ib * 32;               // [2*ib][32] interchange staging
  T* xall = stage + 2 * ib * 32;          // [PNL_XG][ib] all candidate rows
  T* redv = xall + PNL_XG * ib;           // [PNL_WARPS]
  int* redi = reinterpret_cast<int*>(redv + PNL_WARPS);
  int* fpos = redi + PNL_WARPS;  // [2w] whole-panel permutation record
  int* fcur = fpos + 2 * w;
  int* spos = fcur + 2 * w;      // [2ib] sub-panel permutation record
  int* scur = spos + 2 * ib;
  int* hfk = scur + 2 * ib;      // [PNL_HF] keys / values
  int* hfv = hfk + PNL_HF;
  int* hsk = hfv + PNL_HF;       // [PNL_HS]
  int* hsv = hsk + PNL_HS;
  int* misc = hsv + PNL_HS;      // 0: fcnt 1: scnt 2: barrier flag
  unsigned nbar = 0;

  if (P.spec != nullptr) {
    // the diagonal-pivot check ran first: nothing to do if the panel passed;
    // otherwise put back the rows it changed (this CTA's own rows; other CTAs
    // read them only after a grid barrier)
    const int f0 = __ldcg(P.spec), f1 = __ldcg(P.spec + 1), f2 = __ldcg(P.spec + 2), f3 = __ldcg(P.spec + 3);
    if (f0 == 0 && f3 == 0) return;
    const int tag = P.kabs + 1;
    const int rlim = f3 == tag ? P.m : (f1 == tag ? min(f2, P.m) : 0);
    const int rend = min(rloc, rlim - row0);
    for (int r = warp; r < rend; r += PNL_WARPS)
      for (int c = lane; c < w; c += 32) P.A[(int64_t)(row0 + r) * ld + c] = P.spec_backup[(int64_t)(row0 + r) * w + c];
    __syncthreads();
  }

  for (int s = tid; s < w; s += PNL_THREADS) {
    fpos[s] = s;
    fcur[s] = s;
  }
  for (int s = tid; s < PNL_HF; s += PNL_THREADS) hfk[s] = -1;
  if (tid == 0) misc[0] = w;
  const PermRec fperm{fpos, fcur, hfk, hfv, PNL_HF - 1, 0, w, &misc[0]};
  __syncthreads();

  for (int j0 = 0; j0 < w; j0 += ib) {
    const int ibs = min(ib, w - j0);
    for (int r = warp; r < rloc; r += PNL_WARPS)
      if (lane < ibs) S[lane * Rs + r] = __ldcg(P.A + (int64_t)(row0 + r) * ld + j0 + lane);
    for (int s = tid; s < ibs; s += PNL_THREADS) {
      spos[s] = j0 + s;
      scur[s] = j0 + s;
    }
    for (int s = tid; s < PNL_HS; s += PNL_THREADS) hsk[s] = -1;
    if (tid == 0) misc[1] = ibs;
    const PermRec sperm{spos, scur, hsk, hsv, PNL_HS - 1, j0, j0 + ibs, &misc[1]};
    __syncthreads();
    // local candidate of the sub-panel's first column
    T bv = T(-1);
    int bi = INT_MAX;
    for (int r = tid; r < rloc; r += PNL_THREADS) {
      const int gi = row0 + r;
      if (gi >= j0) argmax_merge(bv, bi, pivot_mag(S[r]), gi);
    }

    for (int j = 0; j < ibs; ++j) {
      const int jg = j0 + j;
      const int par = jg & 1;
      // ---- 1. this CTA's candidate: first row of largest |a| in column j
      //      among its rows >= jg; publish it with its sub-panel values
      if (is_inf_mag(bv)) atomicOr(P.status, ST_RANGE);  // a non-finite candidate
      warp_argmax(bv, bi);
      if (lane == 0) {
        redv[warp] = bv;
        redi[warp] = bi;
      }
      __syncthreads();
      if (warp == 0) {
        T v = lane < PNL_WARPS ? redv[lane] : T(-1);
        int i = lane < PNL_WARPS ? redi[lane] : INT_MAX;
        warp_argmax(v, i);
        if (lane == 0) {
          P.xval[par * G + cta] = v;
          P.xidx[par * G + cta] = i;
        }
        if (i != INT_MAX && lane < ibs) P.xrow[((int64_t)par * G + cta) * ib + lane] = S[lane * Rs + (i - row0)];
      } else if (warp == 1) {
        if (jg >= row0 && jg < row0 + rloc && lane < ibs) P.xrowj[par * ib + lane] = S[lane * Rs + (jg - row0)];
      }
      // ---- 2. exchange
      if (!grid_sync_mono(P.bar, (++nbar) * (unsigned)G, P.status, &misc[2])) return;
      // ---- 3. every candidate row, (|a|, row) pair and row jg in one round
      T xq[PNL_XQ];
#pragma unroll
      for (int q = 0; q < PNL_XQ; ++q) {
        const int e = tid + q * PNL_THREADS;
        xq[q] = e < G * ib ? __ldcg(P.xrow + (int64_t)par * G * ib + e) : T(0);
      }
      const T rjq = tid < ibs ? __ldcg(P.xrowj + par * ib + tid) : T(0);
      bv = T(-1);
      bi = INT_MAX;
      if (tid < G) {
        bv = __ldcg(P.xval + par * G + tid);
        bi = __ldcg(P.xidx + par * G + tid);
      }
#pragma unroll
      for (int q = 0; q < PNL_XQ; ++q) {
        const int e = tid + q * PNL_THREADS;
        if (e < G * ib) xall[e] = xq[q];
      }
      warp_argmax(bv, bi);
      if (lane == 0) {
        redv[warp] = bv;
        redi[warp] = bi;
      }
      __syncthreads();
      {
        T v = lane < PNL_WARPS ? redv[lane] : T(-1);
        int i = lane < PNL_WARPS ? redi[lane] : INT_MAX;
        warp_argmax(v, i);
        bi = i;  // the pivot row, in every thread
      }
      int p = bi;
      if (!GB_IN_BOUNDS(P.status, p >= jg && p < P.m)) p = jg;
      const T* prow = xall + (p / R) * ib;  // the pivot row's sub-panel values
      if (tid < ibs) {
        if (p != jg && p >= row0 && p < row0 + rloc) S[tid * Rs + (p - row0)] = rjq;
        if (jg >= row0 && jg < row0 + rloc) S[tid * Rs + (jg - row0)] = prow[tid];
      }
      if (tid == 0) {
        if (cta == 0) {
          P.ipiv[P.kabs + jg] = P.kabs + p + 1;
          if (prow[j] == T(0)) atomicMin(P.info, P.kabs + jg + 1);
        }
        if (p != jg) {
          fperm.swap_rows(jg, p);
          sperm.swap_rows(jg, p);
        }
      }
      __syncthreads();
      // ---- 4. scale the column below the pivot (a division, as in the
      //      definition), rank-1 update of the sub-panel, and the local
      //      candidate of the next column on the way
      const T piv = prow[j];
      bv = T(-1);
      bi = INT_MAX;
      for (int r = tid; r < rloc; r += PNL_THREADS) {
        const int gi = row0 + r;
        if (gi > jg) {
          T l = S[j * Rs + r];
          if (nonzero(piv)) l = l / piv;
          S[j * Rs + r] = l;
          for (int c = j + 1; c < ibs; ++c) S[c * Rs + r] -= l * prow[c];
          if (j + 1 < ibs) argmax_merge(bv, bi, pivot_mag(S[(j + 1) * Rs + r]), gi);
        }
      }
    }

    // ---- sub-panel done: write the tile back (after every thread's last update)
    __syncthreads();
    for (int r = warp; r < rloc; r += PNL_WARPS)
      if (lane < ibs) P.A[(int64_t)(row0 + r) * ld + j0 + lane] = S[lane * Rs + r];
    if (!grid_sync_mono(P.bar, (++nbar) * (unsigned)G, P.status, &misc[2])) return;

    // ---- interchanges of this sub-panel on the other panel columns, and the
    //      top-row triangular solve of the columns to its right
    const int nout = w - ibs;
    const int scnt = misc[1];
    const int nchunk = (nout + 31) / 32;
    if (nchunk > 0 && cta < nchunk) {
      for (int e = tid; e < ibs * ibs; e += PNL_THREADS) {
        const int t = e / ibs, s2 = e % ibs;
        Lsub[t * ib + s2] = __ldcg(P.A + (int64_t)(j0 + t) * ld + j0 + s2);
      }
      __syncthreads();
    }
    for (int q = cta; q < nchunk; q += G) {
      const int o = q * 32 + lane;
      const int c = o < j0 ? o : o + ibs;
      for (int s2 = warp; s2 < scnt; s2 += PNL_WARPS)
        if (o < nout) stage[s2 * 32 + lane] = __ldcg(P.A + (int64_t)scur[s2] * ld + c);
      __syncthreads();
      for (int s2 = warp; s2 < scnt; s2 += PNL_WARPS)
        if (o < nout) P.A[(int64_t)spos[s2] * ld + c] = stage[s2 * 32 + lane];
      __syncthreads();
      if (warp == 0 && o < nout && o >= j0) {
        // forward substitution with the unit-lower sub-panel block; the
        // column lives in the (now free) staging area, lane = column
        T* xs = stage;
        for (int t = 0; t < ibs; ++t) xs[t * 32 + lane] = __ldcg(P.A + (int64_t)(j0 + t) * ld + c);
        for (int t = 1; t < ibs; ++t) {
          T v = xs[t * 32 + lane];
          for (int s2 = 0; s2 < t; ++s2) v -= Lsub[t * ib + s2] * xs[s2 * 32 + lane];
          xs[t * 32 + lane] = v;
        }
        for (int t = 0; t < ibs; ++t) P.A[(int64_t)(j0 + t) * ld + c] = xs[t * 32 + lane];
      }
      __syncthreads();
    }
    if (j0 + ibs < w) {
      if (!grid_sync_mono(P.bar, (++nbar) * (unsigned)G, P.status, &misc[2])) return;
      // ---- rank-ibs update of own rows below the sub-panel, columns to its right
      const int c0 = j0 + ibs;
      for (int cc = c0; cc < w; cc += 32) {
        const int cw = min(32, w - cc);
        for (int t = warp; t < ibs; t += PNL_WARPS)
          if (lane < cw) Ust[t * 32 + lane] = __ldcg(P.A + (int64_t)(j0 + t) * ld + cc + lane);
        __syncthreads();
        // eight of the warp's rows per batch, their loads in flight together
        // (one L2 round trip per eight rows instead of one per row)
        for (int rb = warp; rb < rloc; rb += PNL_WARPS * 8) {
          T a[8];
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = rb + i * PNL_WARPS;
            const bool ok = r < rloc && row0 + r >= c0 && lane < cw;
            a[i] = ok ? __ldcg(P.A + (int64_t)(row0 + r) * ld + cc + lane) : T(0);
          }
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const int r = rb + i * PNL_WARPS;
            if (r < rloc && row0 + r >= c0 && lane < cw) {
              T v = a[i];
              for (int t = 0; t < ibs; ++t) v -= S[t * Rs + r] * Ust[t * 32 + lane];
              P.A[(int64_t)(row0 + r) * ld + cc + lane] = v;
            }
          }
        }
        __syncthreads();
      }
    }
  }
  // ---- whole-panel permutation for the row interchanges outside the panel:
  //      only the positions whose row moved (none when every pivot was on
  //      the diagonal, and the interchange kernel then has nothing to do)
  if (cta == 0) {
    __syncthreads();
    const int fcnt = misc[0];
    if (tid == 0) misc[3] = 0;
    __syncthreads();
    for (int s2 = tid; s2 < fcnt; s2 += PNL_THREADS) {
      if (fpos[s2] != fcur[s2]) {
        const int q = atomicAdd(&misc[3], 1);
        P.perm[1 + q] = fpos[s2];
        P.perm[1 + 2 * w + q] = fcur[s2];
      }
    }
    __syncthreads();
    if (tid == 0) P.perm[0] = misc[3];
  }
}

static inline char* align_up(char* p, size_t a) { return (char*)(((uintptr_t)p + a - 1) / a * a); }

void panel_scratch_carve(PanelScratch* s, void* base, int gmax, int ibmax, int wmax, int tsize) {
  char* p = (char*)base;
  s->bar = (unsigned*)p;
  p += 64;
  s->xval = p;
  p = align_up(p + 2 * (size_t)gmax * tsize, 256);
  s->xidx = (int*)p;
  p = align_up(p + 2 * (size_t)gmax * sizeof(int), 256);
  s->xrow = p;
  p = align_up(p + 2 * (size_t)gmax * ibmax * tsize, 256);
  s->xrowj = p;
  p = align_up(p + 2 * (size_t)ibmax * tsize, 256);
  s->perm = (int*)p;
  s->gmax = gmax;
  s->ibmax = ibmax;
  s->wmax = wmax;
}

// CTAs of one panel launch.  FP64 panels are bound by the (slow) FP64 pipes,
// so they spread over every SM; FP32 panels are bound by the per-column
// exchange, which is cheaper with fewer CTAs (one L2 round trip per column),
// and leave the other SMs to the concurrent trailing update.  Each CTA's
// sub-panel tile must fit in shared memory.
int panel_grid_size(int m, int w, int tsize, const DevInfo& dev, int gmax, int gtarget) {
  const int cap = dev.sm_count < gmax ? dev.sm_count : gmax;
  int target = tsize == 8 ? cap : (64 < cap ? 64 : cap);
  if (gtarget > 0) target = gtarget < cap ? gtarget : cap;
  static const int forced = getenv("GB300LU_PANEL_G") ? atoi(getenv("GB300LU_PANEL_G")) : 0;
  if (forced > 0) target = forced < cap ? forced : cap;
  const size_t budget = (size_t)dev.max_smem_optin - 48 * 1024;
  auto fits = [&](int r) {
    return (size_t)PNL_IB * (r | 1) * tsize <= budget &&
           panel_smem_bytes(r, PNL_IB, w, tsize) <= (size_t)dev.max_smem_optin;
  };
  int R = (int)cdiv(m, target);
  if (R < 64) R = 64;
  while (!fits(R) && target < cap) {
    ++target;
    R = (int)cdiv(m, target);
    if (R < 64) R = 64;
  }
  if (!fits(R)) return -1;
  return (int)cdiv(m, R);
}

// Panels use the cooperative grid kernel.  The cluster kernel (FP32 only;
// GB300LU_PANEL_CLUSTER set) computes the same factorization on at most 16
// SMs: about 4 us per column like the cooperative kernel, but its in-panel
// update on 16 SMs makes it slower alone (210 vs 185 ms of panels at
// n = 32768), and beside the lookahead update it waits for a free GPC.
static bool use_cluster_panel(int m, int w, int tsize) {
  static const bool cluster = getenv("GB300LU_PANEL_CLUSTER") != nullptr;
  return tsize == 4 && cluster && panel_cluster_available(m, w);
}

int panel_sm_use(int m, int w, int tsize, const DevInfo& dev, const PanelScratch& s) {
  if (use_cluster_panel(m, w, tsize)) return panel_cluster_size(m, w);
  return panel_grid_size(m, w, tsize, dev, s.gmax, s.gtarget);
}

template <typename T>
cudaError_t launch_panel(T* Wkk, int64_t ldw, int m, int w, int kabs, int* ipiv, int* info, int* status,
                         const PanelScratch& s, const DevInfo& dev, cudaStream_t st, const int* spec_flag,
                         const T* spec_backup) {
  if (w <= 0 || m < w || w > s.wmax) return cudaErrorInvalidValue;
  if constexpr (sizeof(T) == 4) {
    if (use_cluster_panel(m, w, 4)) {
      if (spec_flag != nullptr) return cudaErrorInvalidValue;  // no restore step in the cluster kernel
      return launch_panel_cluster(Wkk, ldw, m, w, kabs, ipiv, info, status, s.perm, st);
    }
  }
  if (s.gmax > PNL_XG) return cudaErrorInvalidValue;  // every candidate row fits the exchange buffer
  const int ib = PNL_IB < s.ibmax ? PNL_IB : s.ibmax;
  const int G0 = panel_grid_size(m, w, sizeof(T), dev, s.gmax, s.gtarget);
  if (G0 <= 0) return cudaErrorInvalidConfiguration;
  const int R = (int)cdiv(m, G0);
  const int G = (int)cdiv(m, R);  // <= G0; every CTA owns at least one row
  const size_t smem = panel_smem_bytes(R, ib, w, sizeof(T));
  auto kern = panel_getrf_kernel<T>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PNL_THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1 || G > per_sm * dev.sm_count || G > s.gmax) return cudaErrorCooperativeLaunchTooLarge;
  e = cudaMemsetAsync(s.bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  PanelParams<T> P;
  P.A = Wkk;
  P.ld = ldw;
  P.m = m;
  P.w = w;
  P.ib = ib;
  P.R = R;
  P.G = G;
  P.kabs = kabs;
  P.ipiv = ipiv;
  P.info = info;
  P.status = status;
  P.bar = s.bar;
  P.xval = (T*)s.xval;
  P.xidx = s.xidx;
  P.xrow = (T*)s.xrow;
  P.xrowj = (T*)s.xrowj;
  P.perm = s.perm;
  P.spec = spec_flag;
  P.spec_backup = spec_backup;
  void* args[] = {&P};
  // A cooperative launch is refused (without side effects) while other
  // in-flight cooperative grids -- other streams' panels -- hold the resources
  // it needs; those grids always finish, so retry with a short back-off
  // (bounded: 20 s).
  const auto t0 = std::chrono::steady_clock::now();
  while (true) {
    e = cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(PNL_THREADS), args, smem, st);
    if (e != cudaErrorCooperativeLaunchTooLarge && e != cudaErrorLaunchOutOfResources) return e;
    cudaGetLastError();
    if (std::chrono::steady_clock::now() - t0 > std::chrono::seconds(20)) return e;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

// ============================================================ laswp
// Apply a panel's net row permutation (count c, dst positions, src positions;
// relative to row k) to columns [0, k) and [k + w, n) of W.  CTA q handles a
// chunk of CW consecutive columns: it stages every source row segment in
// shared memory, then writes them to their destinations (so that sources are
// read before any destination is overwritten).  Block 0 also permutes rowid.

template <typename T>
__global__ void __launch_bounds__(256) laswp_kernel(T* W, int64_t ldw, int n, int k, int w, const int* perm,
                                                     int* rowid) {
  constexpr int CW = 128 / sizeof(T);  // columns per chunk: one 128-byte row segment
  constexpr int RPP = 256 / CW;        // row segments per pass
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* stage = reinterpret_cast<T*>(smem_raw);
  const int cnt = perm[0];
  if (cnt == 0) return;  // no row moved (every pivot on the diagonal)
  const int* dst = perm + 1;
  const int* src = perm + 1 + 2 * w;
  const int nout = n - w;
  const int rsub = threadIdx.x / CW;
  if (blockIdx.x == 0 && rowid != nullptr) {
    int* istage = reinterpret_cast<int*>(stage + (size_t)2 * w * CW);
    for (int s = threadIdx.x; s < cnt; s += 256) istage[s] = rowid[k + src[s]];
    __syncthreads();
    for (int s = threadIdx.x; s < cnt; s += 256) rowid[k + dst[s]] = istage[s];
  }
  // column chunks, grid-stride
  for (int q = blockIdx.x; q * CW < nout; q += gridDim.x) {
    const int o = q * CW + (threadIdx.x % CW);
    const int c = o < k ? o : o + w;
    for (int s = rsub; s < cnt; s += RPP)
      if (o < nout) stage[s * CW + (threadIdx.x % CW)] = W[(int64_t)(k + src[s]) * ldw + c];
    __syncthreads();
    for (int s = rsub; s < cnt; s += RPP)
      if (o < nout) W[(int64_t)(k + dst[s]) * ldw + c] = stage[s * CW + (threadIdx.x % CW)];
    __syncthreads();  // the stage is refilled by the next chunk
  }
}

template <typename T>
cudaError_t launch_laswp(T* W, int64_t ldw, int n, int k, int w, const int* perm, int* rowid, cudaStream_t st) {
  constexpr int CW = 128 / sizeof(T);
  const int nout = n - w;
  const int chunks = nout > 0 ? (int)cdiv(nout, CW) : 1;
  const size_t smem = (size_t)2 * w * CW * sizeof(T) + 2 * (size_t)w * sizeof(int) + 16;
  auto kern = laswp_kernel<T>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  // one resident wave (the launch is short and mostly waits on its first loads)
  static thread_local int per_sm = -1, sm_count = 0, per_sm_w = -1;
  if (per_sm < 0 || per_sm_w != w) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem) != cudaSuccess || per_sm < 1)
      per_sm = 1;
    per_sm_w = w;
  }
  const int wave = per_sm * sm_count;
  const int blocks = chunks < wave ? chunks : wave;
  laswp_kernel<T><<<blocks, 256, smem, st>>>(W, ldw, n, k, w, perm, rowid);
  return cudaGetLastError();
}

// ============================================================ trsm (top blocks)
// U12 <- L11^-1 A12 for the unit-lower w x w block L11 (the paper's "top"
// block update).  CTA = a strip of 32 columns of A12 held in shared memory
// (lane = column).  Blocked by 32 rows: warp 0 solves a 32 x 32 diagonal
// block by substitution, then all warps apply it to the rows below.

template <typename T>
__global__ void __launch_bounds__(256) trsm_lower_kernel(const T* L, T* X, int64_t ldw, int w, int N) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Xs = reinterpret_cast<T*>(smem_raw);  // [w][32]
  T* Ld = Xs + (size_t)w * 32;             // [32][33]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * 32 + lane;
  const bool cok = c < N;
  for (int r = warp; r < w; r += 8) Xs[r * 32 + lane] = cok ? X[(int64_t)r * ldw + c] : T(0);
  for (int b0 = 0; b0 < w; b0 += 32) {
    const int bw = min(32, w - b0);
    for (int e = threadIdx.x; e < bw * 32; e += 256) {
      const int t = e >> 5, s = e & 31;
      Ld[t * 33 + s] = (s < bw) ? L[(int64_t)(b0 + t) * ldw + b0 + s] : T(0);
    }
    __syncthreads();
    if (warp == 0) {
      T x[32];
#pragma unroll
      for (int t = 0; t < 32; ++t) x[t] = (t < bw) ? Xs[(b0 + t) * 32 + lane] : T(0);
#pragma unroll
      for (int t = 1; t < 32; ++t) {
        T v = x[t];
#pragma unroll
        for (int s = 0; s < 32; ++s)
          if (s < t) v -= Ld[t * 33 + s] * x[s];
        x[t] = v;
      }
#pragma unroll
      for (int t = 0; t < 32; ++t)
        if (t < bw) Xs[(b0 + t) * 32 + lane] = x[t];
    }
    __syncthreads();
    // rows below the block: each warp takes every 8th row, eight rows per
    // batch so that their L loads are in flight together
    T xb[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) xb[t] = (t < bw) ? Xs[(b0 + t) * 32 + lane] : T(0);
    for (int r0 = b0 + bw + warp; r0 < w; r0 += 64) {
      T lv[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = r0 + 8 * i;
        lv[i] = (r < w && lane < bw) ? L[(int64_t)r * ldw + b0 + lane] : T(0);
      }
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = r0 + 8 * i;
        if (r >= w) break;
        T acc = Xs[r * 32 + lane];
#pragma unroll
        for (int t = 0; t < 32; ++t) acc -= __shfl_sync(0xffffffffu, lv[i], t) * xb[t];
        Xs[r * 32 + lane] = acc;
      }
    }
    __syncthreads();
  }
  if (cok)
    for (int r = warp; r < w; r += 8) X[(int64_t)r * ldw + c] = Xs[r * 32 + lane];
}

template <typename T>
cudaError_t launch_trsm_lower(const T* L11, T* A12, int64_t ldw, int w, int N, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  const size_t smem = ((size_t)w * 32 + 32 * 33) * sizeof(T);
  auto kern = trsm_lower_kernel<T>;
  cudaError_t e = allow_max_smem((const void*)kern);
  if (e != cudaSuccess) return e;
  trsm_lower_kernel<T><<<(int)cdiv(N, 32), 256, smem, st>>>(L11, A12, ldw, w, N);
  return cudaGetLastError();
}

// ============================================================ layout conversions
template <typename T>
__global__ void to_working_kernel(const double* __restrict__ A, int64_t lda, T* __restrict__ W, int64_t ldw, int n) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = bi + tx, j = bj + jj;
    tile[jj][tx] = (i < n && j < n) ? A[(int64_t)j * lda + i] : 0.0;
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = bi + ii, j = bj + tx;
    if (i < n && j < n) W[(int64_t)i * ldw + j] = (T)tile[tx][ii];
  }
}

template <typename T>
__global__ void from_working_kernel(const T* __restrict__ W, int64_t ldw, double* __restrict__ LU, int64_t ldlu,
                                    int n) {
  __shared__ double tile[32][33];
  const int bi = blockIdx.y * 32, bj = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = bi + ii, j = bj + tx;
    tile[ii][tx] = (i < n && j < n) ? (double)W[(int64_t)i * ldw + j] : 0.0;
  }
  __syncthreads();
  for (int jj = ty; jj < 32; jj += 8) {
    const int i = bi + tx, j = bj + jj;
    if (i < n && j < n) LU[(int64_t)j * ldlu + i] = tile[tx][jj];
  }
}

template <typename T>
cudaError_t launch_to_working(const double* A, int64_t lda, T* W, int64_t ldw, int n, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(n, 32), (unsigned)cdiv(n, 32));
  to_working_kernel<T><<<grid, dim3(32, 8), 0, st>>>(A, lda, W, ldw, n);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_from_working(const T* W, int64_t ldw, double* LU, int64_t ldlu, int n, cudaStream_t st) {
  dim3 grid((unsigned)cdiv(n, 32), (unsigned)cdiv(n, 32));
  from_working_kernel<T><<<grid, dim3(32, 8), 0, st>>>(W, ldw, LU, ldlu, n);
  return cudaGetLastError();
}

__global__ void iota_kernel(int* v, int n, int base) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i + base;
}

cudaError_t launch_iota(int* v, int n, cudaStream_t st, int base) {
  iota_kernel<<<(int)cdiv(n, 256), 256, 0, st>>>(v, n, base);
  return cudaGetLastError();
}

#define GB_INST(T)                                                                                              \
  template cudaError_t launch_panel<T>(T*, int64_t, int, int, int, int*, int*, int*, const PanelScratch&,      \
                                       const DevInfo&, cudaStream_t, const int*, const T*);                     \
  template cudaError_t launch_laswp<T>(T*, int64_t, int, int, int, const int*, int*, cudaStream_t);            \
  template cudaError_t launch_trsm_lower<T>(const T*, T*, int64_t, int, int, cudaStream_t);                    \
  template cudaError_t launch_to_working<T>(const double*, int64_t, T*, int64_t, int, cudaStream_t);           \
  template cudaError_t launch_from_working<T>(const T*, int64_t, double*, int64_t, int, cudaStream_t);
GB_INST(double)
GB_INST(float)
#undef GB_INST

}  // namespace gb
