// Serving runtime: continuous batching of spectrum requests over resident plans.
//
// Requests (N, L, P_zeta, map, seed) arrive through sigw_submit from any thread.  max_slots worker threads
// each take the oldest admissible request together with queued requests of the same size class (N, L), up to
// the plans' max_batch, and run them as one batch (sigw_generate_batch + sigw_spectrum) on a plan from a shared
// pool.  Every plan owns its CUDA stream, so the slots' batches overlap on the device.
//
// Admission by device memory: a new plan may be created only if its footprint fits the budget together with
// the plans already resident.  Only the oldest queued request may evict idle plans (least-recently-used first)
// to make room, and only when the eviction frees enough.  A later request may create a plan only in budget that
// is free without eviction and that the oldest request does not need (its footprint stays reserved while it has
// no plan of its size class), otherwise it must reuse an idle plan.  While the oldest request cannot be admitted
// even by evicting every idle plan, no later request starts, so finishing plans stay idle until the oldest
// request can evict them: the head of the queue cannot starve, whichever slot (general or express) looks first.  A request whose plan alone exceeds the budget is refused at
// submission (SIGW_EBUSY).
// Plans run on streams whose priority falls with the lattice size (smaller lattices first), so short requests
// are not held behind the thread blocks of long ones when they share the device.
// Express slots (sigw_server_set_express) are extra workers that take only requests of small lattices (N at most
// a given size), so short requests do not wait behind batches of large ones for a free general slot; they use
// the same pool, budget and admission rule, applied among the requests they may take.
// Latency of a request = completion time - submission time.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/sigw.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  uint64_t ticket = 0;
  int N = 0;
  double L = 0;
  sigw_pzeta pz{};
  sigw_ngmap map{};
  uint64_t seed = 0;
  Clock::time_point arrival;
  int state = 0;  // 0 queued, 1 running, 2 done
  sigw_status status = SIGW_OK;
  std::vector<double> omega;
  double latency = 0.0;
  int batch_size = 0;
};

struct PoolPlan {
  sigw_plan plan = nullptr;
  cudaStream_t stream = nullptr;  // created by the server with a priority by lattice size
  int N = 0;
  double L = 0;
  size_t bytes = 0;
  bool busy = false;
  bool creating = false;
  uint64_t last_use = 0;
};

}  // namespace

struct sigw_server_s {
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Req*> queue;
  std::unordered_map<uint64_t, Req*> reqs;
  std::vector<PoolPlan*> pool;
  std::vector<std::thread> workers;
  size_t budget = 0, in_use = 0;
  sigw_opts opts{};
  int dev = 0;
  bool stop = false;
  uint64_t next_ticket = 1, tick = 0;
  uint64_t n_submitted = 0, n_completed = 0, n_failed = 0, n_batches = 0, n_plans_created = 0, n_evicted = 0;
  uint64_t n_express_batches = 0;
  size_t peak_in_use = 0;
  int express_slots = 0;
};

namespace {

size_t footprint_of(const sigw_server_s* s, int N) {
  size_t b = 0;
  if (sigw_plan_footprint(N, &s->opts, &b) != SIGW_OK) return (size_t)-1;
  return b;
}

PoolPlan* idle_plan(sigw_server_s* s, int N, double L) {
  for (PoolPlan* p : s->pool)
    if (!p->busy && !p->creating && p->N == N && p->L == L) return p;
  return nullptr;
}

// Whether any plan (idle, busy or being created) of size class (N, L) is in the pool.
bool any_plan(sigw_server_s* s, int N, double L) {
  for (PoolPlan* p : s->pool)
    if (p->N == N && p->L == L) return true;
  return false;
}

struct Doomed {
  sigw_plan plan;
  cudaStream_t stream;
};

void destroy_all(std::vector<Doomed>& v) {
  for (Doomed& d : v) {
    if (d.plan) sigw_plan_destroy(d.plan);
    if (d.stream) cudaStreamDestroy(d.stream);
  }
  v.clear();
}

// Stream priority for a lattice size: the device's greatest priority for the smallest lattices.
int priority_for(int N) {
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  // numerically lower is higher priority; N <= 64 greatest, each doubling one step lower
  int p = greatest;
  for (int n = 64; n < N && p < least; n *= 2) ++p;
  return p;
}

// Evict idle plans (least recently used first) until `need` more bytes fit.  Called with the lock held;
// returns false, evicting nothing, if even evicting every idle plan would not make room.
bool make_room(sigw_server_s* s, size_t need, std::vector<Doomed>* to_destroy) {
  size_t idle = 0;
  for (PoolPlan* p : s->pool)
    if (!p->busy && !p->creating) idle += p->bytes;
  if (s->in_use - idle + need > s->budget) return false;
  while (s->in_use + need > s->budget) {
    PoolPlan* lru = nullptr;
    for (PoolPlan* p : s->pool)
      if (!p->busy && !p->creating && (!lru || p->last_use < lru->last_use)) lru = p;
    if (!lru) return false;
    to_destroy->push_back({lru->plan, lru->stream});
    s->in_use -= lru->bytes;
    s->pool.erase(std::find(s->pool.begin(), s->pool.end(), lru));
    delete lru;
    s->n_evicted++;
  }
  return true;
}

void finish(sigw_server_s* s, std::vector<Req*>& batch, sigw_status st, const double* omega_all, int ns) {
  const auto now = Clock::now();
  for (size_t i = 0; i < batch.size(); ++i) {
    Req* r = batch[i];
    r->status = st;
    if (st == SIGW_OK) r->omega.assign(omega_all + i * ns, omega_all + (i + 1) * ns);
    r->latency = std::chrono::duration<double>(now - r->arrival).count();
    r->batch_size = (int)batch.size();
    r->state = 2;
    if (st == SIGW_OK) s->n_completed++; else s->n_failed++;
  }
}

// max_N = 0: a general slot (any request); otherwise an express slot (requests with N <= max_N only).
void worker_main(sigw_server_s* s, int max_N) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    if (s->stop) break;
    // pick the oldest admissible request this slot may take
    PoolPlan* use = nullptr;
    Req* head = nullptr;
    bool create = false;
    size_t need = 0;
    std::vector<Doomed> destroy;
    // Budget the oldest queued request keeps reserved: its footprint while no plan of its size class exists.
    // If even evicting every idle plan would not make room for it, it is blocked: no later request may start
    // (idle plans then stay idle until enough of them can be evicted for the oldest one).
    size_t reserve = 0;
    bool blocked = false;
    if (!s->queue.empty() && !any_plan(s, s->queue.front()->N, s->queue.front()->L)) {
      reserve = footprint_of(s, s->queue.front()->N);
      size_t idle = 0;
      for (PoolPlan* p : s->pool)
        if (!p->busy && !p->creating) idle += p->bytes;
      blocked = s->in_use - idle + reserve > s->budget;
    }
    for (size_t qi = 0; qi < s->queue.size(); ++qi) {
      Req* r = s->queue[qi];
      if (qi > 0 && blocked) break;
      if (max_N > 0 && r->N > max_N) continue;
      if ((use = idle_plan(s, r->N, r->L))) {
        head = r;
        break;
      }
      need = footprint_of(s, r->N);
      if (qi == 0) {  // the oldest request may evict idle plans
        if (make_room(s, need, &destroy)) {
          head = r;
          create = true;
          break;
        }
      } else if (s->in_use + need + reserve <= s->budget) {  // the rest only in free, unreserved budget
        head = r;
        create = true;
        break;
      }
    }
    if (!head) {
      if (!destroy.empty()) {
        lk.unlock();
        destroy_all(destroy);
        lk.lock();
      }
      s->cv.wait(lk);
      continue;
    }
    if (create) {
      use = new PoolPlan();
      use->N = head->N;
      use->L = head->L;
      use->bytes = need;
      use->creating = true;
      s->in_use += need;
      s->peak_in_use = std::max(s->peak_in_use, s->in_use);
      s->pool.push_back(use);
    }
    use->busy = true;
    // the batch: head plus queued requests of the same size class, in arrival order
    std::vector<Req*> batch;
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)batch.size() < s->opts.max_batch;) {
      if ((*it)->N == head->N && (*it)->L == head->L) {
        batch.push_back(*it);
        (*it)->state = 1;
        it = s->queue.erase(it);
      } else {
        ++it;
      }
    }
    s->n_batches++;
    if (max_N > 0) s->n_express_batches++;
    lk.unlock();
    destroy_all(destroy);
    sigw_status st = SIGW_OK;
    if (create) {
      sigw_plan np = nullptr;
      cudaStream_t ps = nullptr;
      if (cudaStreamCreateWithPriority(&ps, cudaStreamNonBlocking, priority_for(head->N)) != cudaSuccess) {
        (void)cudaGetLastError();
        ps = nullptr;
        st = SIGW_ECUDA;
      }
      if (st == SIGW_OK) st = sigw_plan_create(head->N, head->L, &s->opts, ps, &np);
      lk.lock();
      use->creating = false;
      if (st == SIGW_OK) {
        use->plan = np;
        use->stream = ps;
        s->n_plans_created++;
      } else {
        if (ps) cudaStreamDestroy(ps);
        s->in_use -= use->bytes;
        s->pool.erase(std::find(s->pool.begin(), s->pool.end(), use));
        delete use;
        use = nullptr;
      }
      lk.unlock();
    }
    const int ns = head->N / 2;
    std::vector<double> omega((size_t)batch.size() * ns, 0.0);
    if (st == SIGW_OK) {
      std::vector<sigw_pzeta> pz;
      std::vector<sigw_ngmap> mp;
      std::vector<uint64_t> seeds;
      for (Req* r : batch) {
        pz.push_back(r->pz);
        mp.push_back(r->map);
        seeds.push_back(r->seed);
      }
      st = sigw_generate_batch(use->plan, pz.data(), mp.data(), seeds.data(), (int)batch.size(), nullptr);
      if (st == SIGW_OK) st = sigw_spectrum(use->plan, nullptr, 0, omega.data(), nullptr, nullptr, nullptr);
    }
    lk.lock();
    finish(s, batch, st, omega.data(), ns);
    if (use) {
      use->busy = false;
      use->last_use = ++s->tick;
    }
    s->cv.notify_all();
  }
}

}  // namespace

extern "C" {

sigw_status sigw_server_create(size_t hbm_budget_bytes, int max_slots, const sigw_opts* opts, sigw_server* out) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0) return SIGW_EINVAL;
  *out = nullptr;
  sigw_server s = new (std::nothrow) sigw_server_s();
  if (!s) return SIGW_ENOMEM;
  if (opts) s->opts = *opts; else sigw_opts_default(&s->opts);
  size_t probe = 0;
  if (sigw_plan_footprint(8, &s->opts, &probe) != SIGW_OK) {
    delete s;
    return SIGW_EINVAL;
  }
  s->budget = hbm_budget_bytes;
  if (cudaGetDevice(&s->dev) != cudaSuccess) {
    (void)cudaGetLastError();
    delete s;
    return SIGW_ECUDA;
  }
  for (int i = 0; i < max_slots; ++i) s->workers.emplace_back(worker_main, s, 0);
  *out = s;
  return SIGW_OK;
}

sigw_status sigw_submit(sigw_server s, int N, double L, const sigw_pzeta* pz, const sigw_ngmap* map, uint64_t seed,
                        uint64_t* ticket) {
  if (!s || !pz || !map || !ticket || !(L > 0) || N < 8 || N > 512 || (N & (N - 1))) return SIGW_EINVAL;
  if (!(pz->A >= 0) || !(pz->sigma > 0) || !(pz->kstar > 0) || map->kind < 0 || map->kind > 3) return SIGW_EINVAL;
  const size_t need = footprint_of(s, N);
  std::lock_guard<std::mutex> lk(s->mu);
  if (need > s->budget) return SIGW_EBUSY;
  Req* r = new (std::nothrow) Req();
  if (!r) return SIGW_ENOMEM;
  r->ticket = s->next_ticket++;
  r->N = N;
  r->L = L;
  r->pz = *pz;
  r->map = *map;
  r->seed = seed;
  r->arrival = Clock::now();
  s->reqs[r->ticket] = r;
  s->queue.push_back(r);
  s->n_submitted++;
  *ticket = r->ticket;
  s->cv.notify_all();
  return SIGW_OK;
}

sigw_status sigw_server_set_express(sigw_server s, int slots, int max_N) {
  if (!s || slots < 1 || slots > 16 || max_N < 8 || max_N > 512) return SIGW_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->express_slots > 0 || s->stop) return SIGW_ESTATE;
  s->express_slots = slots;
  for (int i = 0; i < slots; ++i) s->workers.emplace_back(worker_main, s, max_N);
  return SIGW_OK;
}

static sigw_status take_result(sigw_server s, Req* r, double* omega, double* latency_s) {
  const sigw_status st = r->status;
  if (omega && st == SIGW_OK) std::memcpy(omega, r->omega.data(), sizeof(double) * r->omega.size());
  if (latency_s) *latency_s = r->latency;
  s->reqs.erase(r->ticket);
  delete r;
  return st;
}

sigw_status sigw_poll(sigw_server s, uint64_t ticket, double* omega, double* latency_s) {
  if (!s) return SIGW_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return SIGW_EINVAL;
  if (it->second->state != 2) return SIGW_ENOTREADY;
  return take_result(s, it->second, omega, latency_s);
}

sigw_status sigw_wait(sigw_server s, uint64_t ticket, double timeout_s, double* omega, double* latency_s) {
  if (!s) return SIGW_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto deadline = Clock::now() + std::chrono::duration<double>(timeout_s < 0 ? 0 : timeout_s);
  while (true) {
    // Look the ticket up again after every wake: another thread may have taken (and freed) the result.
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return SIGW_EINVAL;
    Req* r = it->second;
    if (r->state == 2) return take_result(s, r, omega, latency_s);
    if (s->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
      auto again = s->reqs.find(ticket);
      if (again == s->reqs.end()) return SIGW_EINVAL;
      if (again->second->state == 2) return take_result(s, again->second, omega, latency_s);
      return SIGW_ETIMEOUT;
    }
  }
}

sigw_status sigw_server_stats_read(sigw_server s, sigw_server_stats* out) {
  if (!s || !out) return SIGW_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->n_submitted;
  out->completed = s->n_completed;
  out->failed = s->n_failed;
  out->queued = s->queue.size();
  out->batches = s->n_batches;
  out->plans_created = s->n_plans_created;
  out->plans_evicted = s->n_evicted;
  out->plans_resident = s->pool.size();
  out->hbm_in_use = s->in_use;
  out->hbm_peak = s->peak_in_use;
  out->hbm_budget = s->budget;
  out->express_batches = s->n_express_batches;
  return SIGW_OK;
}

sigw_status sigw_server_destroy(sigw_server s) {
  if (!s) return SIGW_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  for (std::thread& t : s->workers) t.join();
  for (PoolPlan* p : s->pool) {
    if (p->plan) sigw_plan_destroy(p->plan);
    if (p->stream) cudaStreamDestroy(p->stream);
    delete p;
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return SIGW_OK;
}

}  // extern "C"
