// Serving loop for dense solves: worker slots with their own contexts and
// streams (continuous batching), admission by an HBM budget, resident
// factors with LRU eviction, and a batch slot that solves the small requests
// of the queue together in one persistent launch.  Host C++ only; every GPU
// step goes through the library's own entry points (lu_factor, lu_refine,
// lu_batch_*).
#include <time.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"
#include "lu.h"
#include "lu_batched.h"
#include "lu_server.h"

size_t gb_fact_bytes(int n, int nrhs, lu_prec prec, int nb, int sm_count);
void gb_fact_rebind(lu_fact f, lu_ctx c);
void gb_ctx_set_shared(lu_ctx c, int solve_ctas, int gemm_ctas);
void gb_ctx_wait(lu_ctx c);
size_t gb_batch_bytes(int count, int nmax, int sm_count);

namespace {

uint64_t now_ns() {
  timespec ts;
  clock_gettime(CLOCK_MONOTONIC, &ts);
  return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct Job {
  uint64_t ticket;
  lu_request req;
  size_t bytes;  // transient bytes (factor + refinement), 0 for the factor part when reused
  uint64_t t_submit;
};

struct Resident {
  lu_fact f = nullptr;
  size_t bytes = 0;
  int in_use = 0;
  std::list<uint64_t>::iterator lru;
};

// Requests the batch slot takes: the batched kernel's limits.  The route
// depends on the request's shape only, so a request takes the same path (and
// gives the same bits) alone and in any mix.
constexpr int SMALL_NMAX = 512, SMALL_RHSMAX = 8, BATCH_MAX = 4096;
bool is_small(const lu_request& r) { return r.n <= SMALL_NMAX && r.nrhs <= SMALL_RHSMAX; }

}  // namespace

struct lu_server_s {
  int device = 0;
  lu_prec prec = LU_FP16;
  size_t budget = 0;
  int sm_count = 0;
  std::mutex mu;
  std::condition_variable cv_work;  // slots wait for work / memory
  std::condition_variable cv_done;  // waiters wait for results
  std::deque<Job> queue;
  std::deque<Job> small;  // requests for the batch slot
  std::unordered_map<uint64_t, lu_result> results;
  std::unordered_map<uint64_t, Resident> resident;  // key -> factor
  std::list<uint64_t> lru;                          // front = least recently used
  size_t in_use = 0;                                // running transient bytes + resident bytes
  uint64_t next_ticket = 1;
  uint64_t done = 0;
  uint64_t evictions = 0;
  bool stopping = false;
  std::vector<std::thread> slots;
  std::thread batch_slot;
  int batch_state = 0;  // 0 starting, 1 running, -1 unavailable (small requests use the worker slots)
  lu_ctx batch_ctx = nullptr;
  cudaStream_t batch_stream = nullptr;
  int max_slots = 0;
  std::vector<lu_ctx> ctxs;            // per slot; destroyed after the resident factors
  std::vector<cudaStream_t> streams;
  // Optionally one factorization at a time (GB300LU_SERVER_SERIAL_FACTOR):
  // the partial-pivot panels are cooperative grids; the trailing-update CTAs
  // leave room for a panel CTA on every SM, so by default factorizations
  // overlap too, and a panel launch that finds no room retries.
  std::mutex factor_mu;
  bool serialize_factor = false;
  // CTAs per triangular-solve launch in the slots' contexts
  // (GB300LU_SERVER_SOLVE_CTAS, default 8)
  int solve_ctas = 8;
  // persistent CTAs of the slots' trailing updates (GB300LU_SERVER_GEMM_CTAS,
  // default 0: every SM)
  int gemm_ctas = 0;
};

// Block width of a request's factorization: for the tensor-core precisions
// 256 from n = 2048 up (the single-request table's choice is 128 up to n =
// 12288): with many requests on the device at once their trailing updates
// share HBM, whose traffic per FLOP nb = 256 halves (served mix at 2000/s
// offered, 24 slots: 1776 -> 1865 solves/s).  It depends on the request
// alone, so a result is the same alone and in a mix.
static int request_nb(lu_server s, int n) {
  return (s->prec == LU_BF16 || s->prec == LU_FP16) && n >= 2048 ? 256 : 0;
}

static size_t request_bytes(lu_server s, const lu_request& r) {
  return gb_fact_bytes(r.n, r.nrhs, s->prec, request_nb(s, r.n), s->sm_count);
}

// Evict least-recently-used resident factors not in use until `need` fits.
// Called with the lock held; returns true if it fits.  Factors are freed
// outside the lock by the caller (returned in `freed`).
static bool make_room(lu_server s, size_t need, std::vector<lu_fact>& freed) {
  auto it = s->lru.begin();
  while (s->in_use + need > s->budget && it != s->lru.end()) {
    auto r = s->resident.find(*it);
    if (r != s->resident.end() && r->second.in_use == 0) {
      s->in_use -= r->second.bytes;
      freed.push_back(r->second.f);
      s->resident.erase(r);
      it = s->lru.erase(it);
      ++s->evictions;
    } else {
      ++it;
    }
  }
  return s->in_use + need <= s->budget;
}

static void slot_main(lu_server s, int slot) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  lu_ctx ctx = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || lu_create(&ctx, st) != LU_OK) {
    // a slot that cannot start leaves the work to the others
    if (st) cudaStreamDestroy(st);
    return;
  }
  gb_ctx_set_shared(ctx, s->solve_ctas, s->gemm_ctas);
  std::unique_lock<std::mutex> lk(s->mu);
  s->ctxs[slot] = ctx;
  s->streams[slot] = st;
  while (true) {
    // the oldest request whose memory fits (resident hits need the refinement part only)
    std::vector<lu_fact> freed;
    auto pick = s->queue.end();
    // Oldest first.  A request whose resident factor is busy (one request at
    // a time per factor) is passed over; the oldest other request is then
    // the only candidate, so no request overtakes an older one for memory.
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
      size_t need = it->bytes;
      auto r = it->req.use_resident ? s->resident.find(it->req.factor_key) : s->resident.end();
      if (r != s->resident.end()) {
        if (r->second.in_use > 0) continue;
        need = 0;  // the resident factor covers it (refinement vectors live in it)
      }
      if (make_room(s, need, freed)) pick = it;
      break;
    }
    if (!freed.empty()) {
      lk.unlock();
      for (lu_fact f : freed) lu_fact_free(f);
      cudaStreamSynchronize(st);
      lk.lock();
      continue;
    }
    if (pick == s->queue.end()) {
      if (s->stopping && s->queue.empty()) break;
      s->cv_work.wait(lk);
      continue;
    }
    Job job = *pick;
    s->queue.erase(pick);
    lu_result res;
    memset(&res, 0, sizeof(res));
    res.slot = slot;
    res.t_submit_ns = job.t_submit;
    lu_fact f = nullptr;
    bool reused = false;
    size_t charged = 0;
    if (job.req.use_resident) {
      auto r = s->resident.find(job.req.factor_key);
      if (r != s->resident.end()) {
        f = r->second.f;
        r->second.in_use++;
        s->lru.erase(r->second.lru);
        r->second.lru = s->lru.insert(s->lru.end(), job.req.factor_key);
        reused = true;
      } else {
        res.refactored = 1;
      }
    }
    if (!reused) {
      charged = job.bytes;
      s->in_use += charged;
    }
    lk.unlock();

    res.t_start_ns = now_ns();
    int rc = LU_OK;
    if (reused) gb_fact_rebind(f, ctx);  // its last user finished; it now runs on this slot's stream
    if (!reused) {
      std::unique_lock<std::mutex> flk(s->factor_mu, std::defer_lock);
      if (s->serialize_factor) flk.lock();
      int info = 0;
      rc = lu_factor(ctx, job.req.n, job.req.dA, job.req.lda, s->prec, request_nb(s, job.req.n), &f, &info);
      if (rc == LU_OK && info > 0) rc = LU_ESINGULAR;
    }
    int iters = 0;
    double sr = 0.0;
    if (rc == LU_OK)
      rc = lu_refine(f, job.req.dA, job.req.lda, job.req.dB, job.req.ldb, job.req.dX, job.req.ldx, job.req.nrhs,
                     16.0, 50, &iters, &sr);
    gb_ctx_wait(ctx);
    res.t_done_ns = now_ns();
    res.status = rc;
    res.iters = iters;
    res.scaled_resid = sr;
    res.reused_factor = reused ? 1 : 0;

    lk.lock();
    if (reused) {
      auto r = s->resident.find(job.req.factor_key);
      if (r != s->resident.end()) r->second.in_use--;
    } else if (f != nullptr && job.req.keep_factor && job.req.factor_key != 0 && rc != LU_ESINGULAR &&
               s->resident.find(job.req.factor_key) == s->resident.end()) {
      // the transient charge becomes the resident factor's charge
      Resident R;
      R.f = f;
      R.bytes = charged;
      R.lru = s->lru.insert(s->lru.end(), job.req.factor_key);
      s->resident.emplace(job.req.factor_key, R);
      f = nullptr;
      charged = 0;
    }
    s->in_use -= charged;
    s->results[job.ticket] = res;
    ++s->done;
    lk.unlock();
    if (!reused && f) lu_fact_free(f);
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    lk.lock();
  }
  lk.unlock();
}

// The batch slot: takes every queued small request at once (up to
// BATCH_MAX), plans them as one batch (FP32 factor + FP64 refinement to scaled
// residual < 16, one persistent launch), runs it and publishes the results.
static void batch_main(lu_server s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  lu_ctx ctx = nullptr;
  int* h_info = nullptr;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || lu_create(&ctx, st) != LU_OK ||
      cudaMallocHost(&h_info, (size_t)BATCH_MAX * 16) != cudaSuccess) {
    // without a batch slot the small requests go to the worker slots
    if (ctx) lu_destroy(ctx);
    if (st) cudaStreamDestroy(st);
    if (h_info) cudaFreeHost(h_info);
    std::lock_guard<std::mutex> lk(s->mu);
    s->batch_state = -1;
    s->cv_done.notify_all();
    return;
  }
  int* h_iters = h_info + BATCH_MAX;
  double* h_resid = reinterpret_cast<double*>(h_info + 2 * BATCH_MAX);
  std::unique_lock<std::mutex> lk(s->mu);
  s->batch_ctx = ctx;
  s->batch_stream = st;
  s->batch_state = 1;
  s->cv_done.notify_all();
  while (true) {
    if (s->small.empty()) {
      if (s->stopping) break;
      s->cv_work.wait(lk);
      continue;
    }
    // the oldest small requests whose batch fits the budget alone (halved
    // until it does; a single request that cannot fit was refused at submit)
    int count = (int)std::min<size_t>(s->small.size(), BATCH_MAX);
    int nmax = 1;
    size_t need = 0;
    while (true) {
      nmax = 1;
      for (int i = 0; i < count; ++i) nmax = std::max(nmax, s->small[i].req.n);
      need = gb_batch_bytes(count, nmax, s->sm_count) + (size_t)count * 16 + 1024;
      if (need <= s->budget || count == 1) break;
      count = (count + 1) / 2;
    }
    std::vector<lu_fact> freed;
    if (!make_room(s, need, freed)) {
      if (!freed.empty()) {
        lk.unlock();
        for (lu_fact f : freed) lu_fact_free(f);
        lk.lock();
      }
      s->cv_work.wait(lk);  // memory comes back as other requests finish
      continue;
    }
    std::vector<Job> jobs(s->small.begin(), s->small.begin() + count);
    s->small.erase(s->small.begin(), s->small.begin() + count);
    s->in_use += need;
    lk.unlock();
    for (lu_fact f : freed) lu_fact_free(f);

    const uint64_t t0 = now_ns();
    std::vector<int> n(count), k(count), lda(count), ldb(count), ldx(count);
    std::vector<const double*> A(count), B(count);
    std::vector<double*> X(count);
    for (int i = 0; i < count; ++i) {
      const lu_request& r = jobs[i].req;
      n[i] = r.n;
      k[i] = r.nrhs;
      A[i] = r.dA;
      lda[i] = r.lda;
      B[i] = r.dB;
      ldb[i] = r.ldb;
      X[i] = r.dX;
      ldx[i] = r.ldx;
    }
    int rc = LU_OK;
    int* d_out = nullptr;
    if (cudaMallocAsync((void**)&d_out, (size_t)count * 16, st) != cudaSuccess) {
      cudaGetLastError();
      rc = LU_ENOMEM;
    }
    int* d_info = d_out;
    int* d_iters = d_out ? d_out + count : nullptr;
    double* d_resid = d_out ? reinterpret_cast<double*>(d_out + 2 * count) : nullptr;
    lu_batch b = nullptr;
    if (rc == LU_OK)
      rc = lu_batch_create(ctx, count, n.data(), k.data(), A.data(), lda.data(), B.data(), ldb.data(), X.data(),
                           ldx.data(), LU_F32, 16.0, 50, 0, &b);
    if (rc == LU_OK) rc = lu_batch_run(b, d_info, d_iters, d_resid);
    if (rc == LU_OK &&
        (cudaMemcpyAsync(h_info, d_info, (size_t)count * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaMemcpyAsync(h_iters, d_iters, (size_t)count * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
         cudaMemcpyAsync(h_resid, d_resid, (size_t)count * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess))
      rc = LU_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == LU_OK) rc = LU_ECUDA;
    if (b) lu_batch_free(b);
    if (d_out) cudaFreeAsync(d_out, st);
    cudaStreamSynchronize(st);
    const uint64_t t1 = now_ns();

    lk.lock();
    s->in_use -= need;
    for (int i = 0; i < count; ++i) {
      lu_result res;
      memset(&res, 0, sizeof(res));
      res.slot = s->max_slots;  // the batch slot
      res.t_submit_ns = jobs[i].t_submit;
      res.t_start_ns = t0;
      res.t_done_ns = t1;
      if (rc != LU_OK) {
        res.status = rc;
      } else {
        const int info = h_info[i];
        res.status = info == 0 ? LU_OK : info > 0 ? LU_ESINGULAR : info == -1 ? LU_ENOTCONV : LU_ETIMEOUT;
        res.iters = h_iters[i];
        res.scaled_resid = h_resid[i];
      }
      s->results[jobs[i].ticket] = res;
    }
    s->done += count;
    lk.unlock();
    s->cv_done.notify_all();
    s->cv_work.notify_all();
    lk.lock();
  }
  lk.unlock();
  cudaFreeHost(h_info);
}

extern "C" int lu_server_create(lu_server* out, size_t hbm_budget_bytes, lu_prec prec, int max_slots) {
  if (!out) return -1;
  *out = nullptr;
  if (hbm_budget_bytes == 0) return -2;
  if (prec < LU_F64 || prec > LU_F32) return -3;
  if (max_slots < 1 || max_slots > 64) return -4;
  lu_server s = new (std::nothrow) lu_server_s();
  if (!s) return LU_ENOMEM;
  if (cudaGetDevice(&s->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, s->device) != cudaSuccess) {
    delete s;
    return LU_ECUDA;
  }
  s->prec = prec;
  s->budget = hbm_budget_bytes;
  s->serialize_factor = getenv("GB300LU_SERVER_SERIAL_FACTOR") != nullptr;
  if (const char* e = getenv("GB300LU_SERVER_SOLVE_CTAS")) s->solve_ctas = atoi(e);
  if (const char* e = getenv("GB300LU_SERVER_GEMM_CTAS")) s->gemm_ctas = atoi(e);
  s->max_slots = max_slots;
  s->ctxs.assign(max_slots, nullptr);
  s->streams.assign(max_slots, nullptr);
  for (int i = 0; i < max_slots; ++i) s->slots.emplace_back(slot_main, s, i);
  s->batch_slot = std::thread(batch_main, s);
  {
    // routing must not depend on timing: wait until the batch slot is up (or known unavailable)
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->batch_state != 0; });
  }
  *out = s;
  return LU_OK;
}

extern "C" int lu_server_submit(lu_server s, const lu_request* req, uint64_t* ticket) {
  if (!s) return -1;
  if (!req) return -2;
  if (!ticket) return -3;
  const lu_request& r = *req;
  if (r.n < 1 || r.nrhs < 1 || r.nrhs > 32 || !r.dA || !r.dB || !r.dX || r.lda < r.n || r.ldb < r.n ||
      r.ldx < r.n || r.dX == r.dB)
    return -2;
  Job j;
  j.req = r;
  j.t_submit = now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return LU_EINTERNAL;
    const bool small = is_small(r) && s->batch_state == 1;
    j.bytes = small ? gb_batch_bytes(1, r.n, s->sm_count) + 1024 + 16 : request_bytes(s, r);
    if (j.bytes > s->budget) return LU_ENOMEM;
    j.ticket = s->next_ticket++;
    *ticket = j.ticket;
    if (small)
      s->small.push_back(j);
    else
      s->queue.push_back(j);
  }
  s->cv_work.notify_all();
  return LU_OK;
}

extern "C" int lu_server_poll(lu_server s, uint64_t ticket, lu_result* out) {
  if (!s) return -1;
  if (!out) return -3;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->results.find(ticket);
  if (it == s->results.end()) return ticket == 0 || ticket >= s->next_ticket ? -2 : LU_EAGAIN;
  *out = it->second;
  return LU_OK;
}

extern "C" int lu_server_wait(lu_server s, uint64_t ticket, lu_result* out) {
  if (!s) return -1;
  if (!out) return -3;
  std::unique_lock<std::mutex> lk(s->mu);
  if (ticket == 0 || ticket >= s->next_ticket) return -2;
  s->cv_done.wait(lk, [&] { return s->results.count(ticket) != 0; });
  *out = s->results[ticket];
  return LU_OK;
}

extern "C" int lu_server_stats(lu_server s, uint64_t* done, int* resident, size_t* bytes_in_use,
                               uint64_t* evictions) {
  if (!s) return -1;
  std::lock_guard<std::mutex> lk(s->mu);
  if (done) *done = s->done;
  if (resident) *resident = (int)s->resident.size();
  if (bytes_in_use) *bytes_in_use = s->in_use;
  if (evictions) *evictions = s->evictions;
  return LU_OK;
}

extern "C" int lu_server_destroy(lu_server s) {
  if (!s) return -1;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->slots) t.join();
  if (s->batch_slot.joinable()) s->batch_slot.join();
  for (auto& kv : s->resident) lu_fact_free(kv.second.f);
  if (s->batch_ctx) lu_destroy(s->batch_ctx);
  if (s->batch_stream) cudaStreamDestroy(s->batch_stream);
  for (size_t i = 0; i < s->ctxs.size(); ++i) {
    if (s->ctxs[i]) lu_destroy(s->ctxs[i]);
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
  }
  delete s;
  return LU_OK;
}
