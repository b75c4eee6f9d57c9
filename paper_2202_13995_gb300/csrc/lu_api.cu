// C ABI of the LU library: contexts, the blocked factorization driver, the
// solve and the mixed-precision refinement loop (see include/lu.h).
//
// The driver follows the paper's blocked right-looking iteration (arxiv
// 2202.13995, section "Base Implementation", figure "lu_iteration"): per block
// column k of width nb,
//   1. panel   -- factor the m x nb block column with partial pivoting
//                 (the paper's "LU" + "left" blocks),
//   2. laswp   -- apply its row interchanges to the other columns,
//   3. trsm    -- U12 <- L11^-1 A12 (the "top" blocks),
//   4. update  -- A22 <- A22 - L21 U12 (the "inner" blocks, a GEMM).
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "lu.h"
#include "lu_steps.h"
#include "common.cuh"
#include "kernels.h"
#include "nb_table.h"

using namespace gb;

// Workspace allocation of a context: the caller's callbacks (lu_create_ex),
// or the stream-ordered pool (cudaMallocAsync).  Sizes are remembered so that
// a release can hand them back to the callback.
struct Allocator {
  lu_alloc_fn alloc = nullptr;
  lu_free_fn release = nullptr;
  void* user = nullptr;
  std::mutex mu;
  std::unordered_map<void*, size_t> sizes;
  void* get(size_t bytes, cudaStream_t st) {
    void* p = nullptr;
    if (alloc) {
      p = alloc(user, bytes, (void*)st);
      if (p) {
        std::lock_guard<std::mutex> lk(mu);
        sizes[p] = bytes;
      }
      return p;
    }
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void* p, cudaStream_t st) {
    if (!p) return;
    if (release) {
      size_t bytes = 0;
      {
        std::lock_guard<std::mutex> lk(mu);
        auto it = sizes.find(p);
        if (it != sizes.end()) {
          bytes = it->second;
          sizes.erase(it);
        }
      }
      release(user, p, bytes, (void*)st);
      return;
    }
    cudaFreeAsync(p, st);
  }
};

struct lu_ctx_s {
  cudaStream_t stream = nullptr;
  Allocator* mem = nullptr;  // owned; outlives the factors created from this context
  int device = 0;
  DevInfo dev{};
  int* d_status = nullptr;   // device status bits
  double* d_small = nullptr; // 4 + 3*32 doubles: anorm, norms
  int* d_active = nullptr;   // 32 ints: refinement column mask
  int* h_pinned = nullptr;   // pinned: 64 ints
  double* h_norms = nullptr; // pinned: 4 + 3*32 doubles
  // step-level scratch (lazily sized)
  void* step_ws = nullptr;
  size_t step_ws_bytes = 0;
  // launch accounting and optional per-phase event timing
  long long launches = 0;
  bool prof = false;
  unsigned prof_mask = ~0u;  // phases recorded while profiling (bit p = phase p)
  struct Rec {
    int phase;
    int nk;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> pool;
  // lookahead: a side stream for the next panel, joined back by events
  cudaStream_t side = nullptr;
  cudaEvent_t ev_next = nullptr, ev_panel = nullptr;
  cudaEvent_t ev_block = nullptr;  // shared contexts: host waits sleep on this event instead of spinning
  bool lookahead = true;
  int solve_ctas = 0;  // CTAs per triangular-solve launch (0: one per 64-row block)
  int gemm_ctas = 0;   // persistent CTAs of a trailing update without the lookahead (0: every SM)
  // diagonal-pivot check of FP32 panels, and the SMs its lookahead panels keep
  // (the trailing update gets the rest)
  bool spec = true;
  int spec_sms = 32;
  bool split_residual = true;  // the refinement's residual by the split product for > 16 right-hand sides
};

enum { PH_PANEL = 0, PH_LASWP, PH_TRSM, PH_CAST, PH_GEMM, PH_SOLVE, PH_RESID, PH_OTHER, PH_N };

static cudaEvent_t ev_get(lu_ctx c) {
  if (!c->pool.empty()) {
    cudaEvent_t e = c->pool.back();
    c->pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch wrapper: counts the kernels a launcher starts and, when profiling,
// brackets them with an event pair on the context's stream.
template <typename F>
static cudaError_t run_phase(lu_ctx c, int phase, int nk, cudaStream_t st, F&& launch) {
  cudaEvent_t a = nullptr, b = nullptr;
  const bool rec = c->prof && ((c->prof_mask >> phase) & 1u);
  if (rec) {
    a = ev_get(c);
    b = ev_get(c);
    cudaEventRecord(a, st);
  }
  cudaError_t e = launch();
  if (rec) {
    cudaEventRecord(b, st);
    c->recs.push_back({phase, nk, a, b});
  }
  if (e == cudaSuccess) c->launches += nk;
  return e;
}
#define PHASE(c, ph, nk, expr) run_phase((c), (ph), (nk), (c)->stream, [&]() { return (expr); })
#define PHASE_ON(c, st, ph, nk, expr) run_phase((c), (ph), (nk), (st), [&]() { return (expr); })

struct lu_fact_s {
  lu_ctx ctx = nullptr;
  Allocator* mem = nullptr;  // the creating context's (the context outlives the factor)
  int n = 0;
  lu_prec prec = LU_F64;
  int nb = 0;
  int64_t ldw = 0;
  int tsize = 8;
  void* W = nullptr;  // working matrix, row-major T
  int* ipiv = nullptr;
  int* rowid = nullptr;
  int* info_d = nullptr;
  void* panel_mem = nullptr;
  PanelScratch ps{};
  void* aop = nullptr;  // tensor-core operands (K-major, 16-bit)
  void* bop = nullptr;
  int kpad = 0;
  bool ozaki = false;   // FP64 trailing update by error-free splitting
  void* oz_ws = nullptr;
  double* oz_minv = nullptr;  // nb x nb: I - L11^-1 of the current block
  int* spec_flag = nullptr;   // diagonal-pivot check flags (SpecArgs), FP32 panels
  void* spec_backup = nullptr;  // n x nb FP32: a checked panel's rows before the check
  void* uinv = nullptr;         // nb x 32: inverses of the diagonal blocks of a block column's U
  void* solve_mem = nullptr;
  SolveScratch ss{};
  double* vec_ws = nullptr;  // refinement: R, D, partial sums
  void* res_ws = nullptr;    // refinement with > 16 right-hand sides: split operands of the residual product
  size_t res_ws_bytes = 0;
  size_t vec_ws_bytes = 0;
  int info = -1;             // cached host info (-1 = unknown)
};

static const char* k_err[] = {"ok",
                              "singular factor (exact zero pivot)",
                              "device allocation failed",
                              "refinement did not converge within max_iter",
                              "16-bit cast overflow or NaN",
                              "a bounded device wait timed out",
                              "not finished",
                              "CUDA runtime error",
                              "internal error"};

extern "C" const char* lu_strerror(int code) {
  if (code < 0) return "invalid argument";
  if (code <= LU_EINTERNAL) return k_err[code];
  return "unknown status";
}

extern "C" const char* lu_build_tag(void) { return "gb300lu sm_103a"; }

#define CU_TRY(expr)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      if (getenv("GB300LU_DEBUG")) fprintf(stderr, "gb300lu: %s -> %s\n", #expr, cudaGetErrorString(e_)); \
      return (e_ == cudaErrorMemoryAllocation) ? LU_ENOMEM : LU_ECUDA;                        \
    }                                                                                         \
  } while (0)

static int dalloc(lu_ctx c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return LU_OK;
  *p = c->mem->get(bytes, c->stream);
  return *p ? LU_OK : LU_ENOMEM;
}

static void dfree(lu_ctx c, void* p) { c->mem->put(p, c->stream); }

// a factor's buffers go back to the allocator it came from, on the stream of
// the context it is bound to now
static int falloc(lu_fact f, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return LU_OK;
  *p = f->mem->get(bytes, f->ctx->stream);
  return *p ? LU_OK : LU_ENOMEM;
}
static void ffree(lu_fact f, void* p) { f->mem->put(p, f->ctx->stream); }

extern "C" int lu_create(lu_ctx* out, void* cuda_stream) { return lu_create_ex(out, cuda_stream, nullptr, nullptr, nullptr); }

extern "C" int lu_create_ex(lu_ctx* out, void* cuda_stream, lu_alloc_fn alloc, lu_free_fn release, void* user) {
  if (!out) return -1;
  *out = nullptr;
  if ((alloc == nullptr) != (release == nullptr)) return -3;
  lu_ctx c = new (std::nothrow) lu_ctx_s();
  if (!c) return LU_ENOMEM;
  c->mem = new (std::nothrow) Allocator();
  if (!c->mem) {
    delete c;
    return LU_ENOMEM;
  }
  c->mem->alloc = alloc;
  c->mem->release = release;
  c->mem->user = user;
  c->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    delete c;
    return LU_ECUDA;
  }
  cudaDeviceGetAttribute(&c->dev.sm_count, cudaDevAttrMultiProcessorCount, c->device);
  cudaDeviceGetAttribute(&c->dev.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  if (dalloc(c, (void**)&c->d_status, 64 * sizeof(int)) != LU_OK ||
      dalloc(c, (void**)&c->d_small, 128 * sizeof(double)) != LU_OK ||
      dalloc(c, (void**)&c->d_active, 64 * sizeof(int)) != LU_OK ||
      cudaStreamSynchronize(c->stream) != cudaSuccess ||
      cudaMallocHost(&c->h_pinned, 64 * sizeof(int)) != cudaSuccess ||
      cudaMallocHost(&c->h_norms, 128 * sizeof(double)) != cudaSuccess) {
    lu_destroy(c);
    return LU_ENOMEM;
  }
  cudaMemsetAsync(c->d_status, 0, 64 * sizeof(int), c->stream);
  cudaMemsetAsync(c->d_small, 0, 128 * sizeof(double), c->stream);
  cudaStreamSynchronize(c->stream);
  // the side stream (lookahead panels) has the highest priority, so that a
  // panel waiting for SMs is placed before the concurrent update's CTAs
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_next, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_panel, cudaEventDisableTiming) != cudaSuccess) {
    lu_destroy(c);
    return LU_ECUDA;
  }
  if (getenv("GB300LU_NO_LOOKAHEAD")) c->lookahead = false;
  // the cluster panel kernel has no restore step for a failed check
  if (getenv("GB300LU_NO_SPEC") || getenv("GB300LU_PANEL_CLUSTER")) c->spec = false;
  if (const char* e = getenv("GB300LU_SPEC_SMS")) c->spec_sms = atoi(e);
  if (getenv("GB300LU_RESIDUAL_DFMA")) c->split_residual = false;
  *out = c;
  return LU_OK;
}

extern "C" void lu_destroy(lu_ctx c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  for (auto& r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->pool) cudaEventDestroy(e);
  if (c->side) {
    cudaStreamSynchronize(c->side);
    cudaStreamDestroy(c->side);
  }
  if (c->ev_block) cudaEventDestroy(c->ev_block);
  if (c->ev_next) cudaEventDestroy(c->ev_next);
  if (c->ev_panel) cudaEventDestroy(c->ev_panel);
  if (c->mem) {
    dfree(c, c->step_ws);
    dfree(c, c->d_status);
    dfree(c, c->d_small);
    dfree(c, c->d_active);
    cudaStreamSynchronize(c->stream);
  }
  if (c->h_pinned) cudaFreeHost(c->h_pinned);
  if (c->h_norms) cudaFreeHost(c->h_norms);
  delete c->mem;
  delete c;
}

extern "C" int lu_device_sm_count(lu_ctx c) { return c ? c->dev.sm_count : 0; }

extern "C" long long lu_launch_count(lu_ctx c) { return c ? c->launches : 0; }

extern "C" int lu_profile_enable(lu_ctx c, int enable) {
  if (!c) return -1;
  c->prof = enable != 0;
  return LU_OK;
}

extern "C" int lu_profile_select(lu_ctx c, unsigned phase_mask) {
  if (!c) return -1;
  c->prof_mask = phase_mask;
  return LU_OK;
}

extern "C" int lu_profile_read(lu_ctx c, double* ms, long long* launches) {
  if (!c) return -1;
  if (!ms) return -2;
  if (!launches) return -3;
  for (int p = 0; p < PH_N; ++p) {
    ms[p] = 0.0;
    launches[p] = 0;
  }
  CU_TRY(cudaStreamSynchronize(c->stream));
  for (auto& r : c->recs) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.phase] += t;
    launches[r.phase] += r.nk;
    c->pool.push_back(r.a);
    c->pool.push_back(r.b);
  }
  c->recs.clear();
  return LU_OK;
}

// The host waits for the context's stream: spinning (the lowest latency),
// or for a shared context, asleep on a blocking event, so that many contexts
// waiting at once do not hold a host core each.
static cudaError_t ctx_wait(lu_ctx c, cudaStream_t st) {
  if (c->ev_block == nullptr) return cudaStreamSynchronize(st);
  cudaError_t e = cudaEventRecord(c->ev_block, st);
  return e != cudaSuccess ? e : cudaEventSynchronize(c->ev_block);
}

static int read_status(lu_ctx c) {
  CU_TRY(cudaMemcpyAsync(c->h_pinned, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU_TRY(ctx_wait(c, c->stream));
  const int s = c->h_pinned[0];
  if (s) {
    CU_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
  }
  if (s & ST_TIMEOUT) return LU_ETIMEOUT;
  if (s & ST_RANGE) return LU_ERANGE;
  if (s & (ST_BADARG | ST_BOUNDS)) return LU_EINTERNAL;
  return LU_OK;
}

extern "C" int lu_ctx_status(lu_ctx c) {
  if (!c) return -1;
  return read_status(c);
}

// nb = 0: the block width of the offline sweep's table (nb_table.h), by
// factorization kind and size
static int default_nb(int n, lu_prec prec, bool split) {
  const int kind = prec == LU_F64 ? (split ? 1 : 0) : (prec == LU_F32 ? 3 : 2);
  for (const NbEntry& e : kNbTable)
    if (e.kind == kind && n <= e.nmax) return e.nb;
  return 256;
}

static int round_up(int v, int a) { return (v + a - 1) / a * a; }

// ------------------------------------------------------------------ factor
// The top block solve U12 = L11^-1 A12 with the split update: M = I - L11^-1
// in FP64, then A12 -= M A12 on the tensor cores (the split reads A12 before
// the product overwrites it, so the update runs in place).
static cudaError_t top_solve_split(lu_fact f, const double* L11, double* A12, int64_t ld, int w, int N) {
  lu_ctx c = f->ctx;
  cudaStream_t st = c->stream;
  cudaError_t e = PHASE(c, PH_TRSM, 1, launch_unit_lower_inv_comp(L11, ld, w, f->oz_minv, w, st));
  if (e != cudaSuccess) return e;
  e = PHASE(c, PH_TRSM, 2, ozaki_split(f->oz_minv, w, A12, ld, w, N, w, f->oz_ws, c->d_status, st));
  if (e != cudaSuccess) return e;
  return PHASE(c, PH_TRSM, 1, ozaki_gemm(A12, ld, f->oz_ws, w, N, w, 0, N, c->d_status, c->dev, st));
}

// Diagonal-pivot check (FP32 panels; SpecArgs in kernels.h).  The first
// panel is checked and the host waits for the verdict: if it passed, the
// later panels are checked too and their lookahead keeps only spec_sms SMs
// (the check's two kernels and, should a check fail, the pivoted panel that
// redoes it); if it failed, every panel takes the pivoted kernel at once and
// the lookahead keeps its usual share.  A later failure is seen by the host
// through an asynchronous copy of the flags and switches the rest of the
// factorization to the pivoted kernel's split.
enum { SPEC_OFF = 0, SPEC_TRY, SPEC_ON };

template <typename T>
static cudaError_t panel_step(lu_fact f, int mode, T* Wkk, int m, int w, int kabs, cudaStream_t s, int gtarget) {
  lu_ctx c = f->ctx;
  const int64_t ld = f->ldw;
  PanelScratch ps = f->ps;
  if (gtarget > 0) ps.gtarget = gtarget;
  if (mode == SPEC_OFF)
    return PHASE_ON(c, s, PH_PANEL, 1, launch_panel<T>(Wkk, ld, m, w, kabs, f->ipiv, f->info_d, c->d_status, ps,
                                                      c->dev, s));
  SpecArgs sa;
  sa.flag = f->spec_flag;
  sa.backup = f->spec_backup;
  sa.ipiv = f->ipiv;
  sa.perm = f->ps.perm;
  cudaError_t e = PHASE_ON(c, s, PH_PANEL, block_column_launches(m, w, sizeof(T)),
                           launch_block_column<T>(Wkk, ld, m, w, kabs, nullptr, (T*)f->uinv, s, sa));
  if (e != cudaSuccess) return e;
  return PHASE_ON(c, s, PH_PANEL, 1, launch_panel<T>(Wkk, ld, m, w, kabs, f->ipiv, f->info_d, c->d_status, ps,
                                                    c->dev, s, f->spec_flag, (const T*)f->spec_backup));
}

// Persistent CTAs of a trailing update that has the device to itself: all
// SMs; a shared context's (server slots) keep to gemm_ctas.
static int gemm_cap(lu_ctx c) { return c->gemm_ctas > 0 ? c->gemm_ctas : c->dev.sm_count; }

template <typename T>
static int factor_loop(lu_fact f) {
  lu_ctx c = f->ctx;
  cudaStream_t st = c->stream;
  T* W = (T*)f->W;
  const int n = f->n, nb = f->nb;
  const int64_t ld = f->ldw;
  const bool tc = f->prec == LU_BF16 || f->prec == LU_FP16;
  const int kind = f->prec == LU_BF16 ? 1 : 2;
  // Depth-1 lookahead (the paper's overlap of the next communication phase
  // with the update phase): the next panel's columns are updated first, then
  // that panel is factored on the side stream while the rest of the trailing
  // matrix is updated on the remaining SMs.
  // (the split FP64 update is not overlapped: its panel is FP64-bound and
  // runs fastest on every SM, and the update needs whole SMs for its shared
  // memory, so a concurrent panel would slow both)
  const bool lookahead = tc && c->lookahead && c->side != nullptr;
  int mode = (sizeof(T) == 4 && f->spec_flag != nullptr && n > nb) ? SPEC_TRY : SPEC_OFF;
  int* hflag = c->h_pinned + 48;  // [4]: verdict of the first panel; [4..8): later panels, copied asynchronously
  const int spec_sms = c->spec_sms > 0 ? c->spec_sms : 1;
  bool panel_ready = false;
  for (int k = 0; k < n; k += nb) {
    const int w = (n - k) < nb ? (n - k) : nb;
    T* Wkk = W + (int64_t)k * ld + k;
    if (mode == SPEC_ON && (hflag[4] != 0 || hflag[7] != 0)) mode = SPEC_OFF;  // a later panel failed its check
    if (panel_ready) {
      CU_TRY(cudaStreamWaitEvent(st, c->ev_panel, 0));
      panel_ready = false;
    } else {
      // a checked panel's pivoted kernel (a cooperative launch, whose CTAs
      // must all be resident at once) keeps to spec_sms CTAs: it returns at
      // once when the check passed, and a launch across the whole device
      // would wait for the device to drain whenever other work shares it
      CU_TRY(panel_step<T>(f, mode, Wkk, n - k, w, k, st, mode != SPEC_OFF ? spec_sms : 0));
      if (mode == SPEC_TRY) {
        CU_TRY(cudaMemcpyAsync(hflag, f->spec_flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
        CU_TRY(ctx_wait(c, st));
        mode = (hflag[0] == 0 && hflag[3] == 0) ? SPEC_ON : SPEC_OFF;
        hflag[4] = hflag[7] = 0;
      }
    }
    CU_TRY(PHASE(c, PH_LASWP, 1, launch_laswp<T>(W, ld, n, k, w, f->ps.perm, f->rowid, st)));
    const int rest = n - k - w;
    if (rest <= 0) continue;
    T* U12 = Wkk + w;
    T* L21 = Wkk + (int64_t)w * ld;
    T* A22 = L21 + w;
    const int w2 = rest < nb ? rest : nb;
    // with the lookahead, only the next panel's columns of the top block row
    // are solved and cast before the next panel starts; the rest follow on
    // this stream while the next panel runs on the side stream
    const bool split_top = tc && lookahead && rest > w2;
    if (f->ozaki) {
      CU_TRY(top_solve_split(f, (double*)Wkk, (double*)U12, ld, w, rest));
    } else if (tc) {
      // (the tensor-core form also writes the solved columns' B operand)
      CU_TRY(PHASE(c, PH_TRSM, 1, launch_trsm_inv((const float*)Wkk, (float*)U12, ld, w, split_top ? w2 : rest, kind,
                                                   f->bop, f->kpad, c->d_status, st)));
    } else {
      CU_TRY(PHASE(c, PH_TRSM, 1, launch_trsm_lower<T>(Wkk, U12, ld, w, split_top ? w2 : rest, st)));
    }
    if (f->ozaki) {
      CU_TRY(PHASE(c, PH_CAST, 2, ozaki_split((const double*)L21, ld, (const double*)U12, ld, rest, rest, w,
                                               f->oz_ws, c->d_status, st)));
      CU_TRY(PHASE(c, PH_GEMM, 1, ozaki_gemm((double*)A22, ld, f->oz_ws, rest, rest, w, 0, rest, c->d_status, c->dev,
                                              st)));
      continue;
    }
    if (!tc) {
      CU_TRY(PHASE(c, PH_GEMM, 1, launch_gemm_simt<T>(A22, ld, L21, ld, U12, ld, rest, rest, w, st)));
      continue;
    }
    CU_TRY(PHASE(c, PH_CAST, 1, launch_cast_a(kind, (const float*)L21, ld, rest, w, f->aop, f->kpad, c->d_status, st)));
    if (!split_top) {
      CU_TRY(PHASE(c, PH_GEMM, 1, tc_gemm_run(kind, (float*)A22, ld, f->aop, f->bop, rest, rest, f->kpad,
                                               c->d_status, c->dev, st, gemm_cap(c))));
      continue;
    }
    // columns of the next panel first
    CU_TRY(PHASE(c, PH_GEMM, 1, tc_gemm_run(kind, (float*)A22, ld, f->aop, f->bop, rest, w2, f->kpad, c->d_status,
                                             c->dev, st)));
    CU_TRY(cudaEventRecord(c->ev_next, st));
    CU_TRY(cudaStreamWaitEvent(c->side, c->ev_next, 0));
    T* Wn = A22;  // W(k + w, k + w)
    // the SMs the lookahead panel keeps: its checked form needs few; the
    // pivoted kernel keeps its usual share
    int gp = panel_sm_use(rest, w2, sizeof(T), c->dev, f->ps);
    if (mode == SPEC_ON) {
      // (a tall panel needs a few more CTAs than spec_sms for its tile to fit)
      const int gc = panel_grid_size(rest, w2, sizeof(T), c->dev, f->ps.gmax, spec_sms);
      gp = gc > spec_sms ? gc : spec_sms;
    }
    CU_TRY(panel_step<T>(f, mode, Wn, rest, w2, k + w, c->side, mode == SPEC_ON ? spec_sms : 0));
    if (mode == SPEC_ON)
      CU_TRY(cudaMemcpyAsync(hflag + 4, f->spec_flag, 4 * sizeof(int), cudaMemcpyDeviceToHost, c->side));
    CU_TRY(cudaEventRecord(c->ev_panel, c->side));
    panel_ready = true;
    // the rest of the top block row, then the rest of the trailing matrix on
    // the SMs the panel leaves free (the latency-bound panel runs slower on
    // SMs it shares with the update)
    void* bop2 = (char*)f->bop + (size_t)w2 * f->kpad * 2;
    CU_TRY(PHASE(c, PH_TRSM, 1, launch_trsm_inv((const float*)Wkk, (float*)(U12 + w2), ld, w, rest - w2, kind, bop2,
                                                 f->kpad, c->d_status, st)));
    const int cap = c->dev.sm_count - (gp > 0 ? gp : 0);
    CU_TRY(PHASE(c, PH_GEMM, 1, tc_gemm_run(kind, (float*)(A22 + w2), ld, f->aop, bop2, rest, rest - w2, f->kpad,
                                             c->d_status, c->dev, st, cap > 8 ? cap : 8)));
  }
  if (panel_ready) CU_TRY(cudaStreamWaitEvent(st, c->ev_panel, 0));
  return LU_OK;
}

// The paper's no-pivot iteration: LU of the diagonal block, left and top
// block solves, inner update.
template <typename T>
static cudaError_t nopiv_panel(lu_fact f, T* Wkk, int m, int w, int kabs, cudaStream_t s) {
  lu_ctx c = f->ctx;
  const int64_t ld = f->ldw;
  return PHASE_ON(c, s, PH_PANEL, block_column_launches(m, w, sizeof(T)),
                  launch_block_column<T>(Wkk, ld, m, w, kabs, f->info_d, (T*)f->uinv, s));
}

template <typename T>
static int factor_loop_nopiv(lu_fact f) {
  lu_ctx c = f->ctx;
  cudaStream_t st = c->stream;
  T* W = (T*)f->W;
  const int n = f->n, nb = f->nb;
  const int64_t ld = f->ldw;
  const bool tc = f->prec == LU_BF16 || f->prec == LU_FP16;
  const int kind = f->prec == LU_BF16 ? 1 : 2;
  // Lookahead (tensor-core form): the next block column is updated first, then
  // its diagonal-block LU and left-block solve run on the side stream, on the
  // few SMs the rest of the trailing update leaves them.
  const bool lookahead = tc && !f->ozaki && c->lookahead && c->side != nullptr;
  const int keep = c->spec_sms > 0 ? c->spec_sms : 1;
  bool panel_ready = false;
  for (int k = 0; k < n; k += nb) {
    const int w = (n - k) < nb ? (n - k) : nb;
    T* Wkk = W + (int64_t)k * ld + k;
    if (panel_ready) {
      CU_TRY(cudaStreamWaitEvent(st, c->ev_panel, 0));
      panel_ready = false;
    } else {
      CU_TRY(nopiv_panel<T>(f, Wkk, n - k, w, k, st));
    }
    const int rest = n - k - w;
    if (rest <= 0) continue;
    T* U12 = Wkk + w;
    T* L21 = Wkk + (int64_t)w * ld;
    T* A22 = L21 + w;
    const int w2 = rest < nb ? rest : nb;
    const bool split_top = tc && lookahead && rest > w2;  // as in factor_loop
    if (f->ozaki) {
      CU_TRY(top_solve_split(f, (double*)Wkk, (double*)U12, ld, w, rest));
    } else if (tc) {
      CU_TRY(PHASE(c, PH_TRSM, 1, launch_trsm_inv((const float*)Wkk, (float*)U12, ld, w, split_top ? w2 : rest, kind,
                                                   f->bop, f->kpad, c->d_status, st)));
    } else {
      CU_TRY(PHASE(c, PH_TRSM, 1, launch_trsm_lower<T>(Wkk, U12, ld, w, split_top ? w2 : rest, st)));
    }
    if (f->ozaki) {
      CU_TRY(PHASE(c, PH_CAST, 2, ozaki_split((const double*)L21, ld, (const double*)U12, ld, rest, rest, w,
                                               f->oz_ws, c->d_status, st)));
      CU_TRY(PHASE(c, PH_GEMM, 1, ozaki_gemm((double*)A22, ld, f->oz_ws, rest, rest, w, 0, rest, c->d_status, c->dev,
                                              st)));
    } else if (tc) {
      CU_TRY(PHASE(c, PH_CAST, 1, launch_cast_a(kind, (const float*)L21, ld, rest, w, f->aop, f->kpad, c->d_status,
                                                st)));
      if (!split_top) {
        CU_TRY(PHASE(c, PH_GEMM, 1, tc_gemm_run(kind, (float*)A22, ld, f->aop, f->bop, rest, rest, f->kpad,
                                                 c->d_status, c->dev, st, gemm_cap(c))));
        continue;
      }
      // the next block column, then its diagonal block and left blocks beside the rest
      CU_TRY(PHASE(c, PH_GEMM, 1, tc_gemm_run(kind, (float*)A22, ld, f->aop, f->bop, rest, w2, f->kpad,
                                               c->d_status, c->dev, st)));
      CU_TRY(cudaEventRecord(c->ev_next, st));
      CU_TRY(cudaStreamWaitEvent(c->side, c->ev_next, 0));
      CU_TRY(nopiv_panel<T>(f, A22, rest, w2, k + w, c->side));
      CU_TRY(cudaEventRecord(c->ev_panel, c->side));
      panel_ready = true;
      void* bop2 = (char*)f->bop + (size_t)w2 * f->kpad * 2;
      CU_TRY(PHASE(c, PH_TRSM, 1, launch_trsm_inv((const float*)Wkk, (float*)(U12 + w2), ld, w, rest - w2, kind,
                                                   bop2, f->kpad, c->d_status, st)));
      const int cap = c->dev.sm_count - keep;
      CU_TRY(PHASE(c, PH_GEMM, 1, tc_gemm_run(kind, (float*)(A22 + w2), ld, f->aop, bop2, rest, rest - w2, f->kpad,
                                               c->d_status, c->dev, st, cap > 8 ? cap : 8)));
    } else {
      CU_TRY(PHASE(c, PH_GEMM, 1, launch_gemm_simt<T>(A22, ld, L21, ld, U12, ld, rest, rest, w, st)));
    }
  }
  if (panel_ready) CU_TRY(cudaStreamWaitEvent(st, c->ev_panel, 0));
  return LU_OK;
}

extern "C" void lu_fact_free(lu_fact f) {
  if (!f) return;
  for (void* p : {f->W, (void*)f->ipiv, f->panel_mem, f->aop, f->oz_ws, (void*)f->oz_minv, (void*)f->spec_flag,
                  f->spec_backup, f->uinv, f->solve_mem, f->ss.dinv, (void*)f->vec_ws, f->res_ws})
    ffree(f, p);
  delete f;
}

extern "C" int lu_factor(lu_ctx c, int n, const double* dA, int lda, lu_prec prec, int nb, lu_fact* out,
                         int* info) {
  return lu_factor_ex(c, n, dA, lda, prec, nb, 0, out, info);
}

extern "C" int lu_factor_ex(lu_ctx c, int n, const double* dA, int lda, lu_prec prec, int nb, int flags,
                            lu_fact* out, int* info) {
  if (!c) return -1;
  if (flags & ~(LU_FACTOR_NOPIV | LU_FACTOR_OZAKI)) return -7;
  if ((flags & LU_FACTOR_OZAKI) && prec != LU_F64) return -7;
  const bool nopiv = (flags & LU_FACTOR_NOPIV) != 0;
  if (n < 0) return -2;
  if (!dA && n > 0) return -3;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (prec < LU_F64 || prec > LU_F32) return -5;
  if (nb < 0 || nb > 512) return -6;
  if (!out) return -8;
  *out = nullptr;
  if (nb == 0) nb = default_nb(n, prec, (flags & LU_FACTOR_OZAKI) != 0);
  if ((flags & LU_FACTOR_OZAKI) && nb > 256) return -6;
  lu_fact f = new (std::nothrow) lu_fact_s();
  if (!f) return LU_ENOMEM;
  f->ctx = c;
  f->mem = c->mem;
  f->n = n;
  f->prec = prec;
  f->nb = nb < n ? nb : (n > 0 ? n : 1);
  f->tsize = prec == LU_F64 ? 8 : 4;
  f->ldw = round_up(n > 0 ? n : 1, 64);
  const int nn = n > 0 ? n : 1;
  int rc = LU_OK;
  const int gmax = c->dev.sm_count;
  size_t pbytes = panel_scratch_bytes(gmax, 32, f->nb, f->tsize);
  if ((rc = falloc(f, &f->W, (size_t)f->ldw * nn * f->tsize)) ||
      (rc = falloc(f, (void**)&f->ipiv, (size_t)(2 * nn + 64) * sizeof(int))) ||
      (rc = falloc(f, &f->panel_mem, pbytes)) ||
      (rc = falloc(f, &f->solve_mem, solve_scratch_bytes(nn, f->tsize)))) {
    lu_fact_free(f);
    return rc;
  }
  f->rowid = f->ipiv + nn;
  f->info_d = f->rowid + nn;
  panel_scratch_carve(&f->ps, f->panel_mem, gmax, 32, f->nb, f->tsize);
  // With the lookahead, the FP32 panel shares the GPU with the update of the
  // rest of the trailing matrix: 5/8 of the SMs for the panel (measured at
  // n = 32768: 96 of 152 SMs, 238 ms per solve against 256 with 64 and 265
  // with 112, where the update runs short of SMs).
  if ((prec == LU_BF16 || prec == LU_FP16) && c->lookahead) f->ps.gtarget = (c->dev.sm_count * 5 + 7) / 8;
  solve_scratch_carve(&f->ss, f->solve_mem, nn, f->tsize);
  if (prec != LU_F64) {
    // FP32 factors: inverted diagonal blocks for the correction solves
    if ((rc = falloc(f, &f->ss.dinv, solve_dinv_bytes(nn, f->tsize)))) {
      lu_fact_free(f);
      return rc;
    }
  }
  if (flags & LU_FACTOR_OZAKI) {
    f->ozaki = true;
    if ((rc = falloc(f, &f->oz_ws, ozaki_ws_bytes(nn, nn, f->nb, c->dev.sm_count))) ||
        (rc = falloc(f, (void**)&f->oz_minv, (size_t)f->nb * f->nb * sizeof(double)))) {
      lu_fact_free(f);
      return rc;
    }
  }
  const bool spec = prec != LU_F64 && !nopiv && c->spec && n > f->nb;
  if (spec) {
    if ((rc = falloc(f, (void**)&f->spec_flag, 4 * sizeof(int))) ||
        (rc = falloc(f, &f->spec_backup, (size_t)nn * f->nb * f->tsize))) {
      lu_fact_free(f);
      return rc;
    }
  }
  if (spec || nopiv) {
    if ((rc = falloc(f, &f->uinv, (size_t)round_up(f->nb, 32) * 32 * f->tsize))) {
      lu_fact_free(f);
      return rc;
    }
  }
  if (prec == LU_BF16 || prec == LU_FP16) {
    f->kpad = round_up(f->nb, 64);
    if ((rc = falloc(f, &f->aop, (size_t)2 * nn * f->kpad * 2 + 1024))) {
      lu_fact_free(f);
      return rc;
    }
    f->bop = (char*)f->aop + ((size_t)nn * f->kpad * 2 + 1023) / 1024 * 1024;
  }
  cudaStream_t st = c->stream;
  auto fail = [&](int r) {
    lu_fact_free(f);
    return r;
  };
  if (cudaMemsetAsync(f->info_d, 0x7f, sizeof(int), st) != cudaSuccess) return fail(LU_ECUDA);
  if (f->spec_flag && cudaMemsetAsync(f->spec_flag, 0, 4 * sizeof(int), st) != cudaSuccess) return fail(LU_ECUDA);
  if (n > 0) {
    if (PHASE(c, PH_OTHER, 1, launch_iota(f->rowid, n, st)) != cudaSuccess) return fail(LU_ECUDA);
    if (nopiv && PHASE(c, PH_OTHER, 1, launch_iota(f->ipiv, n, st, 1)) != cudaSuccess) return fail(LU_ECUDA);
    if (prec == LU_F64) {
      if (PHASE(c, PH_OTHER, 1, launch_to_working<double>(dA, lda, (double*)f->W, f->ldw, n, st)) != cudaSuccess)
        return fail(LU_ECUDA);
      rc = nopiv ? factor_loop_nopiv<double>(f) : factor_loop<double>(f);
    } else {
      if (PHASE(c, PH_OTHER, 1, launch_to_working<float>(dA, lda, (float*)f->W, f->ldw, n, st)) != cudaSuccess)
        return fail(LU_ECUDA);
      rc = nopiv ? factor_loop_nopiv<float>(f) : factor_loop<float>(f);
      if (!rc && f->ss.dinv) {
        if (PHASE(c, PH_OTHER, 1, launch_trinv<float>((const float*)f->W, f->ldw, n, (float*)f->ss.dinv, st)) !=
            cudaSuccess)
          return fail(LU_ECUDA);
        f->ss.dinv_ready = true;
      }
    }
    if (rc) return fail(rc);
  }
  *out = f;
  if (info) {
    rc = lu_fact_info(f, info);
    if (rc) return rc;
  }
  return LU_OK;
}

extern "C" int lu_fact_info(lu_fact f, int* info) {
  if (!f) return -1;
  lu_ctx c = f->ctx;
  CU_TRY(cudaMemcpyAsync(c->h_pinned + 8, f->info_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  const int rs = read_status(c);  // synchronizes
  const int v = c->h_pinned[8];
  f->info = (v == 0x7f7f7f7f) ? 0 : v;
  if (info) *info = f->info;
  return rs;
}

extern "C" int lu_fact_ipiv(lu_fact f, int* dIpiv) {
  if (!f) return -1;
  if (!dIpiv) return -2;
  if (f->n == 0) return LU_OK;
  CU_TRY(cudaMemcpyAsync(dIpiv, f->ipiv, (size_t)f->n * sizeof(int), cudaMemcpyDeviceToDevice, f->ctx->stream));
  return LU_OK;
}

extern "C" int lu_fact_lu(lu_fact f, double* dLU, int ldlu) {
  if (!f) return -1;
  if (!dLU && f->n > 0) return -2;
  if (ldlu < f->n) return -3;
  if (f->n == 0) return LU_OK;
  if (f->prec == LU_F64)
    CU_TRY(launch_from_working<double>((const double*)f->W, f->ldw, dLU, ldlu, f->n, f->ctx->stream));
  else
    CU_TRY(launch_from_working<float>((const float*)f->W, f->ldw, dLU, ldlu, f->n, f->ctx->stream));
  return LU_OK;
}

// ------------------------------------------------------------------ solve
static int ensure_info(lu_fact f) {
  if (f->info < 0) {
    int info = 0;
    int rc = lu_fact_info(f, &info);
    if (rc) return rc;
  }
  return f->info > 0 ? LU_ESINGULAR : LU_OK;
}

static int solve_chunks(lu_fact f, int nrhs, const double* dB, int64_t ldb, double* dX, int64_t ldx) {
  lu_ctx c = f->ctx;
  SolveScratch ss = f->ss;
  ss.max_ctas = c->solve_ctas;
  for (int q0 = 0; q0 < nrhs; q0 += 32) {
    const int nr = (nrhs - q0) < 32 ? (nrhs - q0) : 32;
    if (f->prec == LU_F64) {
      CU_TRY(PHASE(c, PH_SOLVE, 2, launch_lu_solve<double>((const double*)f->W, f->ldw, f->rowid, f->n, nr,
                                                            dB + q0 * ldb, ldb, dX + q0 * ldx, ldx, ss,
                                                            c->d_status, c->stream)));
    } else {
      CU_TRY(PHASE(c, PH_SOLVE, 2, launch_lu_solve<float>((const float*)f->W, f->ldw, f->rowid, f->n, nr,
                                                           dB + q0 * ldb, ldb, dX + q0 * ldx, ldx, ss,
                                                           c->d_status, c->stream)));
    }
  }
  return LU_OK;
}

extern "C" int lu_solve(lu_fact f, int nrhs, double* dB, int ldb) {
  if (!f) return -1;
  if (nrhs < 0) return -2;
  if (!dB && nrhs > 0 && f->n > 0) return -3;
  if (ldb < (f->n > 1 ? f->n : 1)) return -4;
  if (f->n == 0 || nrhs == 0) return LU_OK;
  int rc = ensure_info(f);
  if (rc) return rc;
  return solve_chunks(f, nrhs, dB, ldb, dB, ldb);
}

// ------------------------------------------------------------------ residual / refinement
static double hpl_scaled(int n, double rn, double an, double xn, double bn) {
  const double eps = std::ldexp(1.0, -53);
  const double den = eps * (an * xn + bn) * (double)n;
  return den > 0 ? rn / den : (rn > 0 ? INFINITY : 0.0);
}

static int ensure_vec_ws(lu_fact f, int nrhs) {
  const size_t n = (size_t)f->n;
  const size_t need = 2 * n * nrhs * 8 + residual_partial_bytes(f->n, nrhs > 32 ? 32 : nrhs) + 4096;
  if (f->vec_ws_bytes >= need) return LU_OK;
  ffree(f, f->vec_ws);
  f->vec_ws = nullptr;
  f->vec_ws_bytes = 0;
  int rc = falloc(f, (void**)&f->vec_ws, need);
  if (rc) return rc;
  f->vec_ws_bytes = need;
  return LU_OK;
}

// norms of one chunk of <= 32 columns into c->h_norms (anorm computed by caller)
static int residual_chunk(lu_ctx c, int n, int nr, const double* dA, int64_t lda, const double* dX, int64_t ldx,
                          const double* dB, int64_t ldb, double* dR, int64_t ldr, double* partial) {
  double* norms = c->d_small + 4;
  CU_TRY(PHASE(c, PH_RESID, 2, launch_residual(dA, lda, dX, ldx, dB, ldb, dR, ldr, n, nr, partial, norms, c->stream)));
  CU_TRY(cudaMemcpyAsync(c->h_norms + 4, norms, (size_t)3 * nr * sizeof(double), cudaMemcpyDeviceToHost,
                         c->stream));
  return LU_OK;
}

// The refinement's residual R = B - A X for a chunk of more than 16
// right-hand sides on the tensor cores: the product A X in FP64 accuracy by error-free
// splitting (the split update's kernels, k = 256 columns of A at a time,
// each chunk's product exact before its one FP64 subtraction), in the
// transposed form R^T -= X^T A^T, so that both operands are read along their
// contiguous columns.  The FP64 CUDA-core residual does 2 n^2 nr FMAs on
// GB300's slow FP64 pipes; here that work goes to the BF16 tensor cores.
// The tensor-core product pads the chunk's right-hand sides to 128 rows, so
// its cost does not shrink with nr while the CUDA-core residual's does: they
// cost the same at about 16 (n = 32768: 33 and 32 ms), and with fewer the
// CUDA-core residual also keeps the device freer for other work (served).
static bool split_residual_applies(lu_fact f, int n, int nr) { return f->ctx->split_residual && nr > 16 && n >= 1024; }

static int residual_chunk_split(lu_fact f, int n, int nr, const double* dA, int64_t lda, const double* dX,
                                int64_t ldx, const double* dB, int64_t ldb, double* dR, int64_t ldr) {
  lu_ctx c = f->ctx;
  cudaStream_t st = c->stream;
  const size_t need = ozaki_ws_bytes(32, n, 256, c->dev.sm_count);
  if (f->res_ws_bytes < need) {
    ffree(f, f->res_ws);
    f->res_ws = nullptr;
    f->res_ws_bytes = 0;
    int rc = falloc(f, &f->res_ws, need);
    if (rc) return rc;
    f->res_ws_bytes = need;
  }
  double* norms = c->d_small + 4;
  CU_TRY(cudaMemcpy2DAsync(dR, (size_t)ldr * 8, dB, (size_t)ldb * 8, (size_t)n * 8, nr, cudaMemcpyDeviceToDevice, st));
  for (int kc = 0; kc < n; kc += 256) {
    const int k = (n - kc) < 256 ? (n - kc) : 256;
    CU_TRY(PHASE(c, PH_RESID, 2, ozaki_split(dX + kc, ldx, dA + (int64_t)kc * lda, lda, nr, n, k, f->res_ws,
                                             c->d_status, st)));
    CU_TRY(PHASE(c, PH_RESID, 1, ozaki_gemm(dR, ldr, f->res_ws, nr, n, k, 0, n, c->d_status, c->dev, st)));
  }
  CU_TRY(PHASE(c, PH_RESID, 1, launch_colmax3(dR, ldr, dX, ldx, dB, ldb, n, nr, norms, st)));
  CU_TRY(cudaMemcpyAsync(c->h_norms + 4, norms, (size_t)3 * nr * sizeof(double), cudaMemcpyDeviceToHost, st));
  return LU_OK;
}

extern "C" int lu_refine(lu_fact f, const double* dA, int lda, const double* dB, int ldb, double* dX, int ldx,
                         int nrhs, double tol, int max_iter, int* iters, double* scaled_resid) {
  if (!f) return -1;
  const int n = f->n;
  if (!dA && n > 0) return -2;
  if (lda < (n > 1 ? n : 1)) return -3;
  if (!dB && n > 0 && nrhs > 0) return -4;
  if (ldb < (n > 1 ? n : 1)) return -5;
  if (!dX && n > 0 && nrhs > 0) return -6;
  if (ldx < (n > 1 ? n : 1)) return -7;
  if (nrhs < 0) return -8;
  if (!(tol > 0)) return -9;
  if (max_iter < 0) return -10;
  if (iters) *iters = 0;
  if (scaled_resid) *scaled_resid = 0.0;
  if (n == 0 || nrhs == 0) return LU_OK;
  int rc = ensure_info(f);
  if (rc) return rc;
  rc = ensure_vec_ws(f, nrhs);
  if (rc) return rc;
  lu_ctx c = f->ctx;
  cudaStream_t st = c->stream;
  double* R = f->vec_ws;
  double* D = R + (size_t)n * nrhs;
  double* partial = D + (size_t)n * nrhs;
  // ||A||_inf once
  CU_TRY(PHASE(c, PH_RESID, 2, launch_norm_inf(dA, lda, n, partial, c->d_small, st)));
  CU_TRY(cudaMemcpyAsync(c->h_norms, c->d_small, sizeof(double), cudaMemcpyDeviceToHost, st));
  // x0 = solve(b)
  rc = solve_chunks(f, nrhs, dB, ldb, dX, ldx);
  if (rc) return rc;
  int it = 0;
  double worst = 0.0;
  int result = LU_OK;
  while (true) {
    // r = b - A x per chunk, norms -> host
    worst = 0.0;
    int nactive = 0;
    for (int q0 = 0; q0 < nrhs; q0 += 32) {
      const int nr = (nrhs - q0) < 32 ? (nrhs - q0) : 32;
      if (split_residual_applies(f, n, nr))
        rc = residual_chunk_split(f, n, nr, dA, lda, dX + (int64_t)q0 * ldx, ldx, dB + (int64_t)q0 * ldb, ldb,
                                  R + (size_t)q0 * n, n);
      else
        rc = residual_chunk(c, n, nr, dA, lda, dX + (int64_t)q0 * ldx, ldx, dB + (int64_t)q0 * ldb, ldb,
                            R + (size_t)q0 * n, n, partial);
      if (rc) return rc;
      rc = read_status(c);  // synchronizes
      if (rc) return rc;
      const double an = c->h_norms[0];
      for (int q = 0; q < nr; ++q) {
        const double s = hpl_scaled(n, c->h_norms[4 + q], an, c->h_norms[4 + nr + q], c->h_norms[4 + 2 * nr + q]);
        if (!(s < tol)) ++nactive;
        c->h_pinned[16 + (q0 + q) % 32] = !(s < tol);
        if (!(s <= worst)) worst = s;
      }
      if (it < max_iter) {
        CU_TRY(cudaMemcpyAsync(c->d_active + 0, c->h_pinned + 16, (size_t)nr * sizeof(int), cudaMemcpyHostToDevice,
                               st));
        // d = solve(r) and x += d for the active columns of this chunk
        bool any = false;
        for (int q = 0; q < nr; ++q) any = any || c->h_pinned[16 + q];
        if (any) {
          rc = solve_chunks(f, nr, R + (size_t)q0 * n, n, D, n);
          if (rc) return rc;
          CU_TRY(PHASE(c, PH_OTHER, 1, launch_add_update(dX + (int64_t)q0 * ldx, ldx, D, n, n, nr, c->d_active, st)));
          CU_TRY(ctx_wait(c, st));  // h_pinned is reused by the next chunk
        }
      }
    }
    if (nactive == 0) break;
    if (it >= max_iter) {
      result = LU_ENOTCONV;
      break;
    }
    ++it;
  }
  if (iters) *iters = it;
  if (scaled_resid) *scaled_resid = worst;
  return result;
}

// ||r||, ||A||, ||x||, ||b|| (infinity norms, r = b - A x in FP64) per column
// into norms[4 q .. 4 q + 3].
static int residual_norms(lu_ctx c, int n, int nrhs, const double* dA, int lda, const double* dX, int ldx,
                          const double* dB, int ldb, double* norms) {
  const size_t need = residual_partial_bytes(n, nrhs > 32 ? 32 : nrhs) + 256;
  void* ws = nullptr;
  int rc = dalloc(c, &ws, need);
  if (rc) return rc;
  double* partial = (double*)ws;
  rc = LU_OK;
  if (launch_norm_inf(dA, lda, n, partial, c->d_small, c->stream) != cudaSuccess ||
      cudaMemcpyAsync(c->h_norms, c->d_small, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess)
    rc = LU_ECUDA;
  for (int q0 = 0; q0 < nrhs && rc == LU_OK; q0 += 32) {
    const int nr = (nrhs - q0) < 32 ? (nrhs - q0) : 32;
    rc = residual_chunk(c, n, nr, dA, lda, dX + (int64_t)q0 * ldx, ldx, dB + (int64_t)q0 * ldb, ldb, nullptr, 0,
                        partial);
    if (rc) break;
    rc = read_status(c);
    if (rc) break;
    for (int q = 0; q < nr; ++q) {
      double* o = norms + 4 * (size_t)(q0 + q);
      o[0] = c->h_norms[4 + q];
      o[1] = c->h_norms[0];
      o[2] = c->h_norms[4 + nr + q];
      o[3] = c->h_norms[4 + 2 * nr + q];
    }
  }
  dfree(c, ws);
  return rc;
}

extern "C" int lu_scaled_residual(lu_ctx c, int n, int nrhs, const double* dA, int lda, const double* dX, int ldx,
                                  const double* dB, int ldb, double* out) {
  if (!c) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (!out) return -10;
  if (n == 0 || nrhs == 0) return LU_OK;
  double* norms = new (std::nothrow) double[4 * (size_t)nrhs];
  if (!norms) return LU_ENOMEM;
  const int rc = residual_norms(c, n, nrhs, dA, lda, dX, ldx, dB, ldb, norms);
  if (rc == LU_OK)
    for (int q = 0; q < nrhs; ++q)
      out[q] = hpl_scaled(n, norms[4 * q], norms[4 * q + 1], norms[4 * q + 2], norms[4 * q + 3]);
  delete[] norms;
  return rc;
}

extern "C" int lu_residual_norms(lu_ctx c, int n, int nrhs, const double* dA, int lda, const double* dX, int ldx,
                                 const double* dB, int ldb, double* out) {
  if (!c) return -1;
  if (n < 0) return -2;
  if (nrhs < 0) return -3;
  if (!out) return -10;
  if (n == 0 || nrhs == 0) return LU_OK;
  return residual_norms(c, n, nrhs, dA, lda, dX, ldx, dB, ldb, out);
}

// ------------------------------------------------------------------ step-level entry points
static int ensure_step_ws(lu_ctx c, size_t bytes) {
  if (c->step_ws_bytes >= bytes) return LU_OK;
  dfree(c, c->step_ws);  // stream-ordered: work already enqueued keeps it until done
  c->step_ws = nullptr;
  c->step_ws_bytes = 0;
  int rc = dalloc(c, &c->step_ws, bytes);
  if (rc) return rc;
  c->step_ws_bytes = bytes;
  return LU_OK;
}

extern "C" int lu_step_panel(lu_ctx c, lu_prec prec, int m, int w, void* dP, int ld, int* dIpiv, int* dInfo) {
  if (!c) return -1;
  if (prec < LU_F64 || prec > LU_F32) return -2;
  if (m < 1) return -3;
  if (w < 1 || w > m || w > 512) return -4;
  if (!dP) return -5;
  if (ld < w) return -6;
  if (!dIpiv) return -7;
  if (!dInfo) return -8;
  const int tsize = prec == LU_F64 ? 8 : 4;
  const int gmax = c->dev.sm_count;
  const size_t pbytes = panel_scratch_bytes(gmax, 32, w, tsize);
  int rc = ensure_step_ws(c, pbytes);
  if (rc) return rc;
  PanelScratch ps;
  panel_scratch_carve(&ps, c->step_ws, gmax, 32, w, tsize);
  CU_TRY(cudaMemsetAsync(dInfo, 0x7f, sizeof(int), c->stream));
  if (prec == LU_F64)
    CU_TRY(launch_panel<double>((double*)dP, ld, m, w, 0, dIpiv, dInfo, c->d_status, ps, c->dev, c->stream));
  else
    CU_TRY(launch_panel<float>((float*)dP, ld, m, w, 0, dIpiv, dInfo, c->d_status, ps, c->dev, c->stream));
  // info: sentinel -> 0
  CU_TRY(cudaMemcpyAsync(c->h_pinned + 9, dInfo, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CU_TRY(cudaStreamSynchronize(c->stream));
  if (c->h_pinned[9] == 0x7f7f7f7f) CU_TRY(cudaMemsetAsync(dInfo, 0, sizeof(int), c->stream));
  return LU_OK;
}

extern "C" int lu_step_trsm(lu_ctx c, lu_prec prec, int w, int N, const void* dL, int ldl, void* dX, int ldx) {
  if (!c) return -1;
  if (prec < LU_F64 || prec > LU_F32) return -2;
  if (w < 1 || w > 512) return -3;
  if (N < 0) return -4;
  if (!dL) return -5;
  if (!dX && N > 0) return -7;
  if (ldl != ldx) return -6;  // the kernel shares one row stride
  if (prec == LU_F64)
    CU_TRY(launch_trsm_lower<double>((const double*)dL, (double*)dX, ldx, w, N, c->stream));
  else if (prec == LU_F32)
    CU_TRY(launch_trsm_lower<float>((const float*)dL, (float*)dX, ldx, w, N, c->stream));
  else
    CU_TRY(launch_trsm_inv((const float*)dL, (float*)dX, ldx, w, N, 0, nullptr, 0, nullptr, c->stream));
  return LU_OK;
}

extern "C" int lu_step_gemm(lu_ctx c, lu_prec prec, int m, int n, int k, void* dC, int ldc, const void* dA, int lda,
                            const void* dB, int ldb) {
  if (!c) return -1;
  if (prec < LU_F64 || prec > LU_F32) return -2;
  if (m < 0) return -3;
  if (n < 0) return -4;
  if (k < 0) return -5;
  if (m == 0 || n == 0 || k == 0) return LU_OK;
  if (prec == LU_F64) {
    CU_TRY(launch_gemm_simt<double>((double*)dC, ldc, (const double*)dA, lda, (const double*)dB, ldb, m, n, k,
                                    c->stream));
    return LU_OK;
  }
  if (prec == LU_F32) {
    CU_TRY(launch_gemm_simt<float>((float*)dC, ldc, (const float*)dA, lda, (const float*)dB, ldb, m, n, k, c->stream));
    return LU_OK;
  }
  // tensor-core path: the cast kernel reads A (m x k) and B (k x n) with one
  // row stride, so the operands are first packed into one strided buffer
  if (lda != ldb) return -9;
  const int kpad = round_up(k, 64);
  const size_t abytes = ((size_t)m * kpad * 2 + 1023) / 1024 * 1024;
  const size_t bbytes = ((size_t)n * kpad * 2 + 1023) / 1024 * 1024;
  int rc = ensure_step_ws(c, abytes + bbytes);
  if (rc) return rc;
  void* aop = c->step_ws;
  void* bop = (char*)c->step_ws + abytes;
  const int kind = prec == LU_BF16 ? 1 : 2;
  CU_TRY(launch_cast_operands(kind, (const float*)dA, (const float*)dB, lda, m, n, k, aop, bop, kpad, c->d_status,
                              c->stream));
  CU_TRY(tc_gemm_run(kind, (float*)dC, ldc, aop, bop, m, n, kpad, c->d_status, c->dev, c->stream));
  return LU_OK;
}

extern "C" int lu_step_wait_probe(lu_ctx c, int kind) {
  if (!c) return -1;
  if (kind < 0 || kind > 2) return -2;
  int rc = ensure_step_ws(c, 256);
  if (rc) return rc;
  CU_TRY(launch_wait_probe(kind, c->step_ws, c->d_status, c->stream));
  c->launches += 1;
  return read_status(c);
}

extern "C" int lu_step_gemm_ozaki(lu_ctx c, int m, int n, int k, double* dC, int ldc, const double* dA, int lda,
                                  const double* dB, int ldb) {
  if (!c) return -1;
  if (m < 0) return -2;
  if (n < 0) return -3;
  if (k < 1 || k > 256) return -4;
  if (m == 0 || n == 0) return LU_OK;
  if (!dC) return -5;
  if (ldc < n) return -6;
  if (!dA) return -7;
  if (lda < k) return -8;
  if (!dB) return -9;
  if (ldb < n) return -10;
  int rc = ensure_step_ws(c, ozaki_ws_bytes(m, n, k, c->dev.sm_count));
  if (rc) return rc;
  CU_TRY(ozaki_split(dA, lda, dB, ldb, m, n, k, c->step_ws, c->d_status, c->stream));
  CU_TRY(ozaki_gemm(dC, ldc, c->step_ws, m, n, k, 0, n, c->d_status, c->dev, c->stream));
  c->launches += 3;
  return LU_OK;
}

// ------------------------------------------------------------------ context accessors (batched / server files)
cudaStream_t gb_ctx_stream(lu_ctx c) { return c->stream; }
int gb_ctx_sm_count(lu_ctx c) { return c->dev.sm_count; }
int* gb_ctx_status(lu_ctx c) { return c->d_status; }
void gb_ctx_count_launches(lu_ctx c, long long k) { c->launches += k; }
void* gb_ctx_alloc(lu_ctx c, size_t bytes) {
  void* p = nullptr;
  return dalloc(c, &p, bytes) == LU_OK ? p : nullptr;
}
void gb_ctx_free(lu_ctx c, void* p) { dfree(c, p); }

// Bytes lu_factor (+ lu_refine's workspace for nrhs columns) allocates; the
// server's admission counts requests with it.
size_t gb_fact_bytes(int n, int nrhs, lu_prec prec, int nb, int sm_count) {
  const int nn = n > 0 ? n : 1;
  if (nb == 0) nb = default_nb(n, prec, false);
  nb = nb < nn ? nb : nn;
  const int tsize = prec == LU_F64 ? 8 : 4;
  const size_t ldw = (size_t)round_up(nn, 64);
  size_t b = ldw * nn * tsize + (size_t)(2 * nn + 64) * sizeof(int) + panel_scratch_bytes(sm_count, 32, nb, tsize) +
             solve_scratch_bytes(nn, tsize);
  if (prec != LU_F64) b += solve_dinv_bytes(nn, tsize);
  if (prec != LU_F64 && n > nb)  // diagonal-pivot check
    b += 4 * sizeof(int) + (size_t)nn * nb * tsize + (size_t)round_up(nb, 32) * 32 * tsize;
  if (prec == LU_BF16 || prec == LU_FP16) b += (size_t)2 * nn * round_up(nb, 64) * 2 + 1024;
  const int nr = nrhs > 32 ? 32 : (nrhs < 1 ? 1 : nrhs);
  b += 2 * (size_t)nn * nrhs * 8 + residual_partial_bytes(nn, nr) + 4096;
  if (nrhs > 16 && nn >= 1024) b += ozaki_ws_bytes(32, nn, 256, sm_count);  // the split residual
  return b;
}

// Move a factorization to another context (its stream, status word and
// pinned buffers).  The caller guarantees that no work on the old context
// still uses it.
void gb_fact_rebind(lu_fact f, lu_ctx c) { f->ctx = c; }

// A context that shares the device with others (the server's slots):
//  - no lookahead: the other requests fill the SMs that the lookahead would
//    give the next panel, and its extra launches and stream waits only
//    lengthen each request (the results are the same bit for bit either way);
//  - triangular solves on solve_ctas persistent CTAs: a solve's CTAs wait on
//    the blocks before theirs, and one CTA per block would hold most SMs
//    waiting for the length of the solve;
//  - trailing updates on gemm_ctas persistent CTAs (0: every SM);
//  - host waits asleep on a blocking event instead of spinning.
void gb_ctx_set_shared(lu_ctx c, int solve_ctas, int gemm_ctas) {
  c->lookahead = false;
  c->solve_ctas = solve_ctas;
  c->gemm_ctas = gemm_ctas;
  if (c->ev_block == nullptr) cudaEventCreateWithFlags(&c->ev_block, cudaEventBlockingSync | cudaEventDisableTiming);
}
void gb_ctx_wait(lu_ctx c) { ctx_wait(c, c->stream); }

extern "C" int lu_default_nb(int n, lu_prec prec, int flags) {
  if (n < 0) return -1;
  if (prec < LU_F64 || prec > LU_F32) return -2;
  const int nb = default_nb(n, prec, (flags & LU_FACTOR_OZAKI) != 0);
  return n > 0 && nb > n ? n : nb;
}

extern "C" size_t lu_fact_bytes(int n, int nrhs, lu_prec prec, int nb) {
  if (n < 1 || nrhs < 0 || prec < LU_F64 || prec > LU_F32 || nb < 0 || nb > 512) return 0;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return gb_fact_bytes(n, nrhs, prec, nb, sms);
}
