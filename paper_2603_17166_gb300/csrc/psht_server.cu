// Request server (psht_server_* of include/psht.h): worker threads with one CUDA stream each, a
// plan cache keyed by the caller's point-set name and the transform parameters, and admission
// against a device-memory budget.  Host code only; every transform runs through the plan API.
#include <cuda_runtime.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "psht_internal.h"

namespace psht {
namespace {

using Clock = std::chrono::steady_clock;
double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// The point count is part of the key: a cached plan writes (synthesis) or reads (adjoint) exactly
// its own npts values, so a request that reuses a points_key with another count gets its own plan
// instead of a plan sized for a different buffer.
struct PlanKey {
  uint64_t points;
  int64_t npts;
  int spin, lmax;
  double eps;
  uint32_t flags;
  bool operator<(const PlanKey& o) const {
    return std::tie(points, npts, spin, lmax, eps, flags) < std::tie(o.points, o.npts, o.spin, o.lmax, o.eps, o.flags);
  }
};

struct CachedPlan {
  psht_plan* plan = nullptr;  // null while a worker creates it
  size_t bytes = 0;           // reserved estimate until created, then the plan's own figure
  bool busy = false;          // a worker holds it (creating or executing)
  uint64_t last_use = 0;
  int precision = 0;
};

struct Job {
  int64_t ticket;
  psht_request req;
  Clock::time_point t_submit;
  size_t est = 0;  // device bytes of its plan, once estimated
};

struct Done {
  bool finished = false;
  psht_result res{};
};

}  // namespace

struct Server {
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job> queue;
  std::map<PlanKey, CachedPlan> cache;
  std::map<int64_t, Done> done;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  bool stopping = false;
  int64_t next_ticket = 1;
  uint64_t use_clock = 0;
  size_t in_use = 0, peak = 0;
  psht_server_stats stats{};

  static PlanKey key_of(const psht_request& r) {
    return PlanKey{r.points_key, r.npts, r.spin, r.lmax, r.eps, r.flags};
  }

  // Evict least-recently-used idle plans until `need` more bytes fit; false (evicting nothing) if
  // even evicting every idle plan would not make room.  Called with mu held; the evicted plans are
  // returned for destruction outside the lock.
  bool make_room(size_t need, std::vector<psht_plan*>& doomed) {
    if (in_use + need <= budget) return true;
    size_t idle = 0;
    for (auto& kv : cache)
      if (!kv.second.busy && kv.second.plan) idle += kv.second.bytes;
    if (in_use - idle + need > budget) return false;
    while (in_use + need > budget) {
      auto victim = cache.end();
      for (auto it = cache.begin(); it != cache.end(); ++it)
        if (!it->second.busy && it->second.plan &&
            (victim == cache.end() || it->second.last_use < victim->second.last_use))
          victim = it;
      in_use -= victim->second.bytes;
      doomed.push_back(victim->second.plan);
      cache.erase(victim);
      ++stats.evictions;
    }
    return true;
  }

  void finish(const Job& j, const psht_result& r) {
    std::lock_guard<std::mutex> g(mu);
    Done& d = done[j.ticket];
    d.res = r;
    d.finished = true;
    ++stats.completed;
    if (r.status != PSHT_OK) ++stats.failed;
    cv_done.notify_all();
    cv_work.notify_all();
  }

  static void set_message(psht_result& r, int rc) {
    r.message[0] = '\0';
    if (rc != PSHT_OK) {
      strncpy(r.message, psht_last_error(), sizeof(r.message) - 1);
      r.message[sizeof(r.message) - 1] = '\0';
    }
  }

  void fail(const Job& j, int rc, int w) {
    psht_result res{};
    res.status = rc;
    res.worker = w;
    res.total_ms = ms_between(j.t_submit, Clock::now());
    set_message(res, rc);
    finish(j, res);
  }

  // Worker loop.  Scans the queue in arrival order for the first job that can start: its plan
  // cached and idle, or not cached and admissible.  Once one new plan does not fit, later jobs
  // may only use cached plans, so that a large request is not starved by smaller ones behind it.
  void worker(int w) {
    cudaSetDevice(device);
    cudaStream_t st = streams[w];
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      bool acted = false, hold_new = false;
      for (size_t i = 0; i < queue.size() && !acted; ++i) {
        Job& q = queue[i];
        const PlanKey k = key_of(q.req);
        auto c = cache.find(k);
        if (c != cache.end()) {
          if (c->second.busy) continue;
          c->second.busy = true;
          c->second.last_use = ++use_clock;
          const Job job = q;
          queue.erase(queue.begin() + i);
          lk.unlock();
          run(w, st, job, true, 0);
          lk.lock();
          acted = true;
          break;
        }
        if (hold_new) continue;
        if (q.est == 0) {  // size of the new plan: one device reduction, done without the lock
          const psht_request r = q.req;
          const int64_t t = q.ticket;
          lk.unlock();
          size_t b = 0;
          int rc = psht_plan_estimate_points(r.spin, r.lmax, r.theta, r.phi, r.npts, r.eps, r.flags, st, &b);
          if (rc == PSHT_OK && b > budget) rc = PSHT_ENOMEM;
          lk.lock();
          for (auto it = queue.begin(); it != queue.end(); ++it) {
            if (it->ticket != t) continue;
            if (rc != PSHT_OK) {
              const Job bad = *it;
              queue.erase(it);
              lk.unlock();
              fail(bad, rc, w);
              lk.lock();
            } else {
              it->est = b;
            }
            break;
          }
          acted = true;  // the queue may have changed meanwhile: rescan
          break;
        }
        std::vector<psht_plan*> doomed;
        if (!make_room(q.est, doomed)) {
          hold_new = true;
          continue;
        }
        CachedPlan cp;
        cp.bytes = q.est;
        cp.busy = true;
        cp.last_use = ++use_clock;
        cache[k] = cp;
        in_use += q.est;
        peak = std::max(peak, in_use);
        const Job job = q;
        queue.erase(queue.begin() + i);
        lk.unlock();
        for (psht_plan* p : doomed) psht_plan_destroy(p);
        run(w, st, job, false, job.est);
        lk.lock();
        acted = true;
      }
      if (acted) continue;
      if (stopping && queue.empty()) return;
      cv_work.wait(lk);
    }
  }

  // Move every queued job with the same plan key and operation as `first` (up to kMaxBatch in all)
  // out of the queue: they run as one batch on the plan (psht_plan_*_batch).  Called with mu held.
  static constexpr int kMaxBatch = 8;
  int max_batch = kMaxBatch;  // psht_server_set_batch_limit
  std::vector<Job> take_batch(const Job& first) {
    std::vector<Job> b{first};
    const PlanKey k = key_of(first.req);
    for (auto it = queue.begin(); it != queue.end() && (int)b.size() < max_batch;) {
      if (it->req.op == first.req.op && !(key_of(it->req) < k) && !(k < key_of(it->req))) {
        b.push_back(*it);
        it = queue.erase(it);
      } else {
        ++it;
      }
    }
    return b;
  }

  void run(int w, cudaStream_t st, const Job& job, bool cached, size_t est) {
    const psht_request& r = job.req;
    const PlanKey k = key_of(r);
    psht_result res{};
    res.worker = w;
    res.plan_cached = cached ? 1 : 0;
    const Clock::time_point t0 = Clock::now();
    psht_plan* plan = nullptr;
    int rc = PSHT_OK;
    {
      std::lock_guard<std::mutex> g(mu);
      plan = cache[k].plan;
      if (cached) ++stats.cache_hits;
    }
    if (!plan) {
      rc = psht_plan_create(r.spin, r.lmax, r.theta, r.phi, r.npts, r.eps, r.flags, st, &plan);
      std::lock_guard<std::mutex> g(mu);
      CachedPlan& cp = cache[k];
      if (rc == PSHT_OK) {
        psht_info inf;
        psht_plan_info(plan, &inf);
        in_use = in_use - est + inf.device_bytes;
        cp.bytes = inf.device_bytes;
        cp.plan = plan;
        cp.precision = inf.precision;
        peak = std::max(peak, in_use);
        ++stats.plans_created;
      } else {
        in_use -= est;
        cache.erase(k);
      }
    }
    const Clock::time_point t1 = Clock::now();
    res.plan_ms = cached ? 0.0 : ms_between(t0, t1);
    // the requests queued for the same plan and operation join this one (continuous batching: they
    // arrived while the plan was busy or being built)
    std::vector<Job> batch{job};
    if (rc == PSHT_OK) {
      std::lock_guard<std::mutex> g(mu);
      batch = take_batch(job);
      stats.batches += 1;
      if (batch.size() > 1) stats.batched_requests += (int64_t)batch.size();
    }
    const int n = (int)batch.size();
    if (rc == PSHT_OK) {
      std::vector<const void*> ia(n), ib(n);
      std::vector<void*> oa(n), ob(n);
      bool any_b = false;
      for (int i = 0; i < n; ++i) {
        const psht_request& q = batch[i].req;
        ia[i] = q.in_a;
        ib[i] = q.in_b;
        oa[i] = q.out_a;
        ob[i] = q.out_b;
        any_b = any_b || (r.op == PSHT_OP_SYNTHESIS ? q.in_b != nullptr : q.out_b != nullptr);
      }
      if (n == 1)
        rc = (r.op == PSHT_OP_SYNTHESIS) ? psht_plan_synthesis(plan, r.in_a, r.in_b, r.out_a, st)
             : (r.op == PSHT_OP_ADJOINT) ? psht_plan_adjoint(plan, r.in_a, r.out_a, r.out_b, st)
                                         : PSHT_EINVAL;
      else
        rc = (r.op == PSHT_OP_SYNTHESIS)
                 ? psht_plan_synthesis_batch(plan, n, ia.data(), any_b ? ib.data() : nullptr, oa.data(), st)
                 : psht_plan_adjoint_batch(plan, n, ia.data(), oa.data(), any_b ? ob.data() : nullptr, st);
      if (rc == PSHT_OK && cudaStreamSynchronize(st) != cudaSuccess) rc = PSHT_ECUDA;
    }
    const Clock::time_point t2 = Clock::now();
    res.exec_ms = ms_between(t1, t2);
    res.status = rc;
    res.batch = n;
    set_message(res, rc);
    {
      std::lock_guard<std::mutex> g(mu);
      auto c = cache.find(k);
      if (c != cache.end()) {
        c->second.busy = false;
        res.precision = c->second.precision;
        if (rc == PSHT_OK && plan) {  // a first batched call adds the plan's batch buffers
          psht_info inf;
          psht_plan_info(plan, &inf);
          if (inf.device_bytes > c->second.bytes) {
            in_use += inf.device_bytes - c->second.bytes;
            c->second.bytes = inf.device_bytes;
            peak = std::max(peak, in_use);
          }
        }
      }
    }
    for (const Job& j : batch) {
      psht_result rj = res;
      rj.queue_ms = ms_between(j.t_submit, t0);
      rj.total_ms = ms_between(j.t_submit, t2);
      finish(j, rj);
    }
  }
};

}  // namespace psht

using psht::Server;

extern "C" {

struct psht_server {
  Server* s;
};

int psht_server_create(int nstreams, size_t budget_bytes, psht_server** out) {
  if (!out || nstreams < 1 || nstreams > 64) {
    psht::set_error("psht_server_create: out must not be NULL and nstreams must lie in [1, 64]");
    return PSHT_EINVAL;
  }
  *out = nullptr;
  auto* s = new Server();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    psht::set_error("psht_server_create: no current CUDA device");
    delete s;
    return PSHT_ECUDA;
  }
  size_t fr = 0, tot = 0;
  if (budget_bytes == 0) {
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      psht::set_error("psht_server_create: cudaMemGetInfo failed");
      delete s;
      return PSHT_ECUDA;
    }
    budget_bytes = (size_t)(0.8 * (double)fr);
  }
  s->budget = budget_bytes;
  s->stats.budget = budget_bytes;
  s->streams.resize(nstreams);
  for (int i = 0; i < nstreams; ++i) {
    if (cudaStreamCreateWithFlags(&s->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaStreamDestroy(s->streams[j]);
      psht::set_error("psht_server_create: cudaStreamCreate failed");
      delete s;
      return PSHT_ECUDA;
    }
  }
  for (int i = 0; i < nstreams; ++i) s->workers.emplace_back([s, i] { s->worker(i); });
  *out = new psht_server{s};
  return PSHT_OK;
}

int psht_server_set_batch_limit(psht_server* server, int max_batch) {
  if (!server || max_batch < 1 || max_batch > Server::kMaxBatch) {
    psht::set_error("psht_server_set_batch_limit: server must not be NULL and max_batch must lie in [1, 8]");
    return PSHT_EINVAL;
  }
  std::lock_guard<std::mutex> g(server->s->mu);
  server->s->max_batch = max_batch;
  return PSHT_OK;
}

int psht_server_submit(psht_server* server, const psht_request* request, int64_t* ticket) {
  if (!server || !request || !ticket) {
    psht::set_error("psht_server_submit: server, request and ticket must not be NULL");
    return PSHT_EINVAL;
  }
  if (request->op != PSHT_OP_SYNTHESIS && request->op != PSHT_OP_ADJOINT) {
    psht::set_error("psht_server_submit: op must be PSHT_OP_SYNTHESIS or PSHT_OP_ADJOINT");
    return PSHT_EINVAL;
  }
  Server* s = server->s;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stopping) {
    psht::set_error("psht_server_submit: the server is stopping");
    return PSHT_EINVAL;
  }
  psht::Job j;
  j.ticket = s->next_ticket++;
  j.req = *request;
  j.t_submit = psht::Clock::now();
  s->done[j.ticket] = psht::Done{};
  s->queue.push_back(j);
  ++s->stats.submitted;
  *ticket = j.ticket;
  s->cv_work.notify_one();
  return PSHT_OK;
}

int psht_server_wait(psht_server* server, int64_t ticket, psht_result* result) {
  if (!server) {
    psht::set_error("psht_server_wait: server must not be NULL");
    return PSHT_EINVAL;
  }
  Server* s = server->s;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it == s->done.end()) {
    psht::set_error("psht_server_wait: unknown ticket (or already waited)");
    return PSHT_EINVAL;
  }
  s->cv_done.wait(lk, [&] { return s->done[ticket].finished; });
  const psht_result r = s->done[ticket].res;
  s->done.erase(ticket);
  if (result) *result = r;
  return PSHT_OK;
}

int psht_server_get_stats(psht_server* server, psht_server_stats* stats) {
  if (!server || !stats) {
    psht::set_error("psht_server_get_stats: server and stats must not be NULL");
    return PSHT_EINVAL;
  }
  Server* s = server->s;
  std::lock_guard<std::mutex> g(s->mu);
  *stats = s->stats;
  stats->bytes_in_use = s->in_use;
  stats->bytes_peak = s->peak;
  return PSHT_OK;
}

int psht_server_destroy(psht_server* server) {
  if (!server) return PSHT_OK;
  Server* s = server->s;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stopping = true;
    s->cv_work.notify_all();
  }
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->cache)
    if (kv.second.plan) psht_plan_destroy(kv.second.plan);
  for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
  delete s;
  delete server;
  return PSHT_OK;
}

}  // extern "C"
