// server.cu -- a serving runtime over resident indices: requests (a batch of
// queries for one index and one k) are admitted against a device-memory
// budget, their queries copied to the device as they arrive (copy stream),
// queued, and a worker thread runs the queued requests of one (index, k) as
// ONE search-plan replay (CUDA graph) of up to max_batch queries, then copies
// every request's results straight to its host buffers and completes it.
// Latency is counted from submission to results on the host.
//
// Device memory: the plans (one per (index, k), made on first use) and a
// staging pool of `mem_budget` bytes holding each admitted request's queries
// until its batch has run. A request whose staging does not fit the free
// pool is refused with RABITQ_EBUSY (the caller retries or drops it); the
// refusals are counted.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cstring>

#include "internal.h"

using namespace rbq;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t ticket = 0;
  int32_t slot = 0, k = 0;
  int64_t nq = 0;
  int64_t* out_ids = nullptr;  // host, nq x k
  float* out_dist = nullptr;
  size_t off = 0, bytes = 0;   // staging range in the pool
  cudaEvent_t copied = nullptr;
  Clock::time_point t_submit;
  double latency_us = 0;
  int status = RABITQ_OK;
  bool done = false;
};

// First-fit allocator over [0, cap) in 256-byte units.
struct Pool {
  size_t cap = 0;
  std::map<size_t, size_t> free_;  // offset -> size
  void init(size_t c) {
    cap = c;
    free_.clear();
    if (c) free_[0] = c;
  }
  bool take(size_t bytes, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t at = it->first + bytes;
      free_.erase(it);
      if (rest) free_[at] = rest;
      return true;
    }
    return false;
  }
  void give(size_t off, size_t bytes) {
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
};

struct Slot {
  const rabitq_index* X = nullptr;
  const rabitq_predictor* pr = nullptr;
  int32_t nprobe = 0, bq = 4;
  float eps0 = 1.9f;
  std::map<int32_t, rabitq_plan*> plans;  // by k
};

}  // namespace

struct rabitq_server {
  rabitq_server_opts o{};
  int device = 0;
  std::deque<Slot> slots;  // stable references: the worker holds one during a batch
  unsigned char* pool_mem = nullptr;
  Pool pool;
  cudaStream_t copy_s = nullptr, run_s = nullptr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Req>> queue;
  std::map<int64_t, std::shared_ptr<Req>> all;
  int64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  rabitq_server_stats st{};
  int worker_status = RABITQ_OK;
};

namespace {

size_t req_bytes(const rabitq_index* X, int64_t nq) {
  return (sizeof(float) * (size_t)nq * X->d + 255) / 256 * 256;
}

// Run one batch: requests of one (slot, k), queries staged in the pool.
int run_batch(rabitq_server* S, Slot& sl, int32_t k, std::vector<std::shared_ptr<Req>>& batch,
              int64_t total) {
  RBQ_CUDA(cudaSetDevice(S->device));
  rabitq_plan*& plan = sl.plans[k];
  if (!plan) {
    rabitq_search_opts so;
    rabitq_search_opts_default(&so);
    RBQ_CHECK(rabitq_plan_create(sl.X, sl.pr, S->o.max_batch, k, sl.nprobe, sl.bq, sl.eps0, &so,
                                 &plan));
  }
  float* q = nullptr;
  int64_t* ids = nullptr;
  float* dist = nullptr;
  RBQ_CHECK(rabitq_plan_buffers(plan, &q, &ids, &dist, nullptr));
  const int d = sl.X->d;
  int64_t at = 0;
  for (auto& r : batch) {
    RBQ_CUDA(cudaStreamWaitEvent(S->run_s, r->copied, 0));
    RBQ_CUDA(cudaMemcpyAsync(q + at * d, S->pool_mem + r->off, sizeof(float) * r->nq * d,
                             cudaMemcpyDeviceToDevice, S->run_s));
    at += r->nq;
  }
  // batch sizes rounded up to a multiple of 16 (fewer graphs to capture);
  // the extra rows hold earlier queries and their results are not read
  const int64_t run_nq = std::min<int64_t>((total + 15) / 16 * 16, S->o.max_batch);
  RBQ_CHECK(rabitq_plan_run(plan, run_nq, S->run_s));
  at = 0;
  for (auto& r : batch) {
    RBQ_CUDA(cudaMemcpyAsync(r->out_ids, ids + at * k, sizeof(int64_t) * r->nq * k,
                             cudaMemcpyDeviceToHost, S->run_s));
    RBQ_CUDA(cudaMemcpyAsync(r->out_dist, dist + at * k, sizeof(float) * r->nq * k,
                             cudaMemcpyDeviceToHost, S->run_s));
    at += r->nq;
  }
  return rabitq_plan_sync(plan, S->run_s);  // waits for the results on the host
}

void worker_main(rabitq_server* S) {
  cudaSetDevice(S->device);
  for (;;) {
    std::vector<std::shared_ptr<Req>> batch;
    int64_t total = 0;
    Slot* sl = nullptr;  // stays valid: the slot deque only grows at its end
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_work.wait(lk, [S] { return S->stop || !S->queue.empty(); });
      if (S->stop && S->queue.empty()) return;
      if (S->o.batch_window_us > 0 && (int64_t)S->queue.size() < 2) {
        // give a lone request a short window to gather company
        S->cv_work.wait_for(lk, std::chrono::microseconds((int64_t)S->o.batch_window_us),
                            [S] { return S->stop || S->queue.size() >= 2; });
      }
      // the oldest request, then every queued request of the same (index,
      // k) that still fits the batch, in arrival order
      const int32_t slot = S->queue.front()->slot, k = S->queue.front()->k;
      sl = &S->slots[slot];
      for (auto it = S->queue.begin(); it != S->queue.end();) {
        Req& r = **it;
        if (r.slot == slot && r.k == k && total + r.nq <= S->o.max_batch) {
          total += r.nq;
          batch.push_back(*it);
          it = S->queue.erase(it);
        } else {
          ++it;
        }
      }
    }
    const int st = run_batch(S, *sl, batch.front()->k, batch, total);
    const auto now = Clock::now();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->st.batches += 1;
      S->st.batched_requests += (int64_t)batch.size();
      S->st.batched_queries += total;
      for (auto& r : batch) {
        r->status = st;
        r->latency_us = std::chrono::duration<double, std::micro>(now - r->t_submit).count();
        r->done = true;
        S->pool.give(r->off, r->bytes);
        S->st.in_flight_bytes -= (int64_t)r->bytes;
        cudaEventDestroy(r->copied);
        r->copied = nullptr;
      }
      if (st == RABITQ_ECUDA) S->worker_status = st;  // the device context is gone
    }
    S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" {

void rabitq_server_opts_default(rabitq_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->max_batch = 256;
  o->mem_budget = int64_t(64) << 20;
  o->batch_window_us = 0.0f;
}

int rabitq_server_create(const rabitq_server_opts* opts, rabitq_server** out) {
  set_error("");
  if (!out) return fail(RABITQ_EINVAL, "rabitq_server_create: out is null");
  *out = nullptr;
  rabitq_server_opts o;
  rabitq_server_opts_default(&o);
  if (opts) o = *opts;
  if (o.max_batch < 1 || o.max_batch > (1 << 20))
    return fail(RABITQ_EINVAL, "rabitq_server_create: need 1 <= max_batch <= 2^20");
  if (o.mem_budget < 4096) return fail(RABITQ_EINVAL, "rabitq_server_create: mem_budget < 4096");
  if (!(o.batch_window_us >= 0.0f) || o.batch_window_us > 1e6f)
    return fail(RABITQ_EINVAL, "rabitq_server_create: batch_window_us must be in [0, 1e6]");
  auto S = std::make_unique<rabitq_server>();
  S->o = o;
  RBQ_CUDA(cudaGetDevice(&S->device));
  const size_t cap = (size_t)o.mem_budget / 256 * 256;
  if (cudaMalloc(&S->pool_mem, cap) != cudaSuccess) {
    cudaGetLastError();
    return fail(RABITQ_ENOMEM, "rabitq_server_create: staging pool allocation failed");
  }
  S->pool.init(cap);
  if (cudaStreamCreateWithFlags(&S->copy_s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->run_s, cudaStreamNonBlocking) != cudaSuccess) {
    if (S->copy_s) cudaStreamDestroy(S->copy_s);
    cudaFree(S->pool_mem);
    return fail(RABITQ_ECUDA, "rabitq_server_create: stream creation failed");
  }
  rabitq_server* raw = S.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return RABITQ_OK;
}

int rabitq_server_add_index(rabitq_server* S, const rabitq_index* X,
                            const rabitq_predictor* pr, int32_t nprobe, int32_t bq, float eps0,
                            int32_t* slot) {
  set_error("");
  if (!S || !X || !slot) return fail(RABITQ_EINVAL, "rabitq_server_add_index: null argument");
  RBQ_CHECK(check_device(S->device, "rabitq_server_add_index"));
  RBQ_CHECK(check_device(X->device, "rabitq_server_add_index (index)"));
  if (pr && pr->K != X->K)
    return fail(RABITQ_EINVAL, "rabitq_server_add_index: predictor made for another bucket count");
  if (!pr && (nprobe < 1 || nprobe > X->K || nprobe > 16384))
    return fail(RABITQ_EINVAL, "rabitq_server_add_index: need 1 <= nprobe <= min(K, 16384)");
  if (bq < 1 || bq > 8) return fail(RABITQ_EINVAL, "rabitq_server_add_index: need 1 <= bq <= 8");
  if (!(eps0 >= 0.0f) || !(eps0 < __builtin_inff()))
    return fail(RABITQ_EINVAL, "rabitq_server_add_index: eps0 must be finite and >= 0");
  std::lock_guard<std::mutex> lk(S->mu);
  Slot sl;
  sl.X = X;
  sl.pr = pr;
  sl.nprobe = pr ? pr->nprobe_max : nprobe;
  sl.bq = bq;
  sl.eps0 = eps0;
  S->slots.push_back(sl);
  *slot = (int32_t)S->slots.size() - 1;
  return RABITQ_OK;
}

int rabitq_server_submit(rabitq_server* S, int32_t slot, const float* queries, int64_t nq,
                         int32_t k, int64_t* out_ids, float* out_dist, int64_t* ticket) {
  set_error("");
  if (!S || !queries || !out_ids || !out_dist || !ticket)
    return fail(RABITQ_EINVAL, "rabitq_server_submit: null argument");
  *ticket = 0;
  if (nq < 1 || nq > S->o.max_batch)
    return fail(RABITQ_EINVAL, "rabitq_server_submit: need 1 <= nq <= max_batch");
  if (k < 1 || k > 1024) return fail(RABITQ_EINVAL, "rabitq_server_submit: need 1 <= k <= 1024");
  auto r = std::make_shared<Req>();
  r->t_submit = Clock::now();
  int d = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (slot < 0 || slot >= (int32_t)S->slots.size())
      return fail(RABITQ_EINVAL, "rabitq_server_submit: unknown index slot");
    if (S->worker_status != RABITQ_OK)
      return fail(S->worker_status, "rabitq_server_submit: the server failed earlier");
    const rabitq_index* X = S->slots[slot].X;
    d = X->d;  // (the slot list is read under the lock: add_index may grow it)
    r->bytes = req_bytes(X, nq);
    // admission: the request's queries must fit the free staging memory
    if (!S->pool.take(r->bytes, &r->off)) {
      S->st.refused += 1;
      return fail(RABITQ_EBUSY, "rabitq_server_submit: device staging budget exhausted (retry)");
    }
    S->st.in_flight_bytes += (int64_t)r->bytes;
    if (S->st.in_flight_bytes > S->st.peak_in_flight_bytes)
      S->st.peak_in_flight_bytes = S->st.in_flight_bytes;
    r->ticket = S->next_ticket++;
    r->slot = slot;
    r->k = k;
    r->nq = nq;
    r->out_ids = out_ids;
    r->out_dist = out_dist;
    S->st.admitted += 1;
  }
  cudaError_t e = cudaEventCreateWithFlags(&r->copied, cudaEventDisableTiming);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S->pool_mem + r->off, queries, sizeof(float) * nq * d,
                        cudaMemcpyHostToDevice, S->copy_s);
  if (e == cudaSuccess) e = cudaEventRecord(r->copied, S->copy_s);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(S->mu);
    S->pool.give(r->off, r->bytes);
    S->st.in_flight_bytes -= (int64_t)r->bytes;
    if (r->copied) cudaEventDestroy(r->copied);
    return fail(RABITQ_ECUDA, std::string("rabitq_server_submit: ") + cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->queue.push_back(r);
    S->all[r->ticket] = r;
    *ticket = r->ticket;
  }
  S->cv_work.notify_one();
  return RABITQ_OK;
}

int rabitq_server_wait(rabitq_server* S, int64_t ticket, double timeout_s, double* latency_us) {
  set_error("");
  if (!S) return fail(RABITQ_EINVAL, "rabitq_server_wait: server is null");
  if (!(timeout_s >= 0.0)) return fail(RABITQ_EINVAL, "rabitq_server_wait: timeout_s < 0");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(RABITQ_EINVAL, "rabitq_server_wait: unknown ticket");
  std::shared_ptr<Req> r = it->second;
  const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                      [&r] { return r->done; });
  if (!ok) return fail(RABITQ_ETIMEOUT, "rabitq_server_wait: not done within the timeout");
  S->all.erase(ticket);
  if (latency_us) *latency_us = r->latency_us;
  if (r->status != RABITQ_OK) return fail(r->status, "rabitq_server_wait: the request's batch failed");
  return RABITQ_OK;
}

int rabitq_server_get_stats(rabitq_server* S, rabitq_server_stats* out) {
  if (!S || !out) return fail(RABITQ_EINVAL, "rabitq_server_get_stats: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  return RABITQ_OK;
}

void rabitq_server_free(rabitq_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->device);
  cudaStreamSynchronize(S->copy_s);
  cudaStreamSynchronize(S->run_s);
  for (auto& sl : S->slots)
    for (auto& kv : sl.plans) rabitq_plan_free(kv.second);
  for (auto& kv : S->all)
    if (kv.second->copied) cudaEventDestroy(kv.second->copied);
  cudaStreamDestroy(S->copy_s);
  cudaStreamDestroy(S->run_s);
  cudaFree(S->pool_mem);
  delete S;
}

}  // extern "C"
