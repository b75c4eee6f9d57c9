// Serving loop for dense solves: worker slots with their own contexts and
// streams (continuous batching), admission by an HBM budget, resident
// factors with LRU eviction.  Host C++ only; every GPU step goes through the
// library's own entry points (lu_factor, lu_refine).
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
#include "lu_server.h"

size_t gb_fact_bytes(int n, int nrhs, lu_prec prec, int nb, int sm_count);
void gb_fact_rebind(lu_fact f, lu_ctx c);

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
  std::unordered_map<uint64_t, lu_result> results;
  std::unordered_map<uint64_t, Resident> resident;  // key -> factor
  std::list<uint64_t> lru;                          // front = least recently used
  size_t in_use = 0;                                // running transient bytes + resident bytes
  uint64_t next_ticket = 1;
  uint64_t done = 0;
  uint64_t evictions = 0;
  bool stopping = false;
  std::vector<std::thread> slots;
  std::vector<lu_ctx> ctxs;            // per slot; destroyed after the resident factors
  std::vector<cudaStream_t> streams;
  // Optionally one factorization at a time (GB300LU_SERVER_SERIAL_FACTOR):
  // the partial-pivot panels are cooperative grids; the trailing-update CTAs
  // leave room for a panel CTA on every SM, so by default factorizations
  // overlap too, and a panel launch that finds no room retries.
  std::mutex factor_mu;
  bool serialize_factor = false;
};

static size_t request_bytes(lu_server s, const lu_request& r) {
  return gb_fact_bytes(r.n, r.nrhs, s->prec, 0, s->sm_count);
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
      rc = lu_factor(ctx, job.req.n, job.req.dA, job.req.lda, s->prec, 0, &f, &info);  // synchronizes
      if (rc == LU_OK && info > 0) rc = LU_ESINGULAR;
    }
    int iters = 0;
    double sr = 0.0;
    if (rc == LU_OK)
      rc = lu_refine(f, job.req.dA, job.req.lda, job.req.dB, job.req.ldb, job.req.dX, job.req.ldx, job.req.nrhs,
                     16.0, 50, &iters, &sr);
    cudaStreamSynchronize(st);
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
  s->ctxs.assign(max_slots, nullptr);
  s->streams.assign(max_slots, nullptr);
  for (int i = 0; i < max_slots; ++i) s->slots.emplace_back(slot_main, s, i);
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
  j.bytes = request_bytes(s, r);
  j.t_submit = now_ns();
  if (j.bytes > s->budget) return LU_ENOMEM;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return LU_EINTERNAL;
    j.ticket = s->next_ticket++;
    *ticket = j.ticket;
    s->queue.push_back(j);
  }
  s->cv_work.notify_one();
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
  for (auto& kv : s->resident) lu_fact_free(kv.second.f);
  for (size_t i = 0; i < s->ctxs.size(); ++i) {
    if (s->ctxs[i]) lu_destroy(s->ctxs[i]);
    if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
  }
  delete s;
  return LU_OK;
}
