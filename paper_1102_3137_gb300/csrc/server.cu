// Serving loop: continuous batching of Dyson solves from IDMFT clients.
//
// The self-consistency loop of inhomogeneous DMFT calls the Dyson solver once
// per iteration with a fresh self-energy (Sec. 3: every iteration needs all
// frequencies again).  A server takes such requests from many clients:
//   - requests queue in arrival order; a worker thread admits the head of the
//     queue as soon as device memory (a budget of plan bytes) and a stream
//     slot allow, so requests that arrive while others run start right away
//     and their work overlaps on the GPU;
//   - while the head waits for memory, a later request whose plan is resident
//     and idle (it needs no memory) is admitted in its place, a bounded number
//     of times per head, so one large request does not hold up small ones;
//   - plans (factors, Lanczos bases, workspace) stay resident on the device
//     and are reused by later requests with the same geometry; idle plans are
//     evicted, least recently used first, when a new geometry needs room (and
//     only when evicting them makes room);
//   - each admitted request runs its whole batched solve (one captured graph
//     per chunk of at most the plan's max_freqs frequencies) on its own
//     stream; queued requests of the same geometry with the same V and start
//     vector join it as further frequencies (one fused launch sequence for
//     requests of uneven K, up to the plan's capacity); completion is detected
//     with events, and the latency from submission to completion is recorded
//     per request.
// A request's result does not depend on what else runs: every frequency is
// computed by its own thread-block cluster with fixed-order reductions.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dyson.h"
#include "dyson_common.cuh"
#include "host_internal.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

std::string geom_key(const dyson_geometry& g) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%d|%d,%d,%d|%.17g|%.17g|%d|%d|%d|%.17g|%d|%.17g|%d|%d|%.17g|%d|%d|%d", g.dim,
                g.L[0], g.L[1], g.dim == 3 ? g.L[2] : 1, g.t, g.mu, g.p, g.k_max, g.precision,
                g.krylov_tol, g.krylov_maxit, g.refine_tol, g.refine_max, g.max_freqs, g.eta,
                g.block_size > 1 ? g.block_size : 1, g.precond, g.freq_groups);
  return buf;
}

struct PlanSlot {
  std::string key;
  dyson_plan plan = nullptr;
  size_t bytes = 0;
  bool busy = false;
  double last_use = 0;
};

enum { Q_QUEUED = 0, Q_RUNNING = 1, Q_DONE = 2, Q_FAILED = 3 };

struct Req {
  dyson_request r;
  std::string key;
  int state = Q_QUEUED;
  int rc = DYSON_OK;
  std::string err;
  double t_submit = 0, t_start = 0, t_done = 0;
  PlanSlot* slot = nullptr;
  int stream = -1;
  int bypassed = 0;                        // later requests admitted while this one waited
};

// Backfill: while the request at the head of the queue waits for memory, a later
// request whose plan is resident and idle (it needs no memory) may run; at most
// BACKFILL_PER_HEAD times per head request, so the head is not starved, and only
// among the first BACKFILL_WINDOW queued requests.
constexpr int BACKFILL_PER_HEAD = 64;
constexpr size_t BACKFILL_WINDOW = 256;
// Fusion: queued requests with the admitted request's geometry, the same V and the
// same start vector(s) join its solve as further frequency segments, up to the
// plan's frequency capacity and FUSE_MAX requests per solve.
constexpr int FUSE_MAX = 32;

}  // namespace

struct dyson_server_s {
  int device = 0;
  size_t budget = 0;
  int max_inflight = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Req> reqs;
  std::vector<PlanSlot*> plans;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<uint64_t> stream_owner;      // ticket running on each stream, 0 = free
  std::vector<std::vector<uint64_t>> stream_group;   // every ticket of that stream's (fused) solve
  size_t used = 0;                         // bytes of all live plans
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  // statistics
  uint64_t completed = 0, admitted = 0, plans_created = 0, plans_evicted = 0, fused = 0;
  size_t peak_used = 0;
  int peak_running = 0;
};

namespace {

int running_count(dyson_server_s* s) {
  int n = 0;
  for (uint64_t t : s->stream_owner) n += t != 0;
  return n;
}

// Called with the lock held.  Returns a plan slot for the request's geometry,
// reusing an idle resident plan or creating one within the memory budget, or
// nullptr if it has to wait for memory.  Sets *rc on a hard error.
PlanSlot* acquire_plan(dyson_server_s* s, Req& q, std::unique_lock<std::mutex>& lk, int* rc,
                       std::string* err) {
  for (PlanSlot* ps : s->plans)
    if (!ps->busy && ps->key == q.key) {
      ps->busy = true;
      return ps;
    }
  size_t need = 0;
  int e = dyson_plan_footprint(&q.r.geom, &need);
  if (e) {
    *rc = e;
    *err = dyson_last_error();
    return nullptr;
  }
  // evict idle plans, least recently used first, until the new one fits; when
  // even evicting every idle plan would not make room, evict nothing and wait
  size_t idle = 0;
  for (PlanSlot* ps : s->plans)
    if (!ps->busy) idle += ps->bytes;
  if (s->used - idle + need > s->budget) return nullptr;
  while (s->used + need > s->budget) {
    PlanSlot* victim = nullptr;
    for (PlanSlot* ps : s->plans)
      if (!ps->busy && (!victim || ps->last_use < victim->last_use)) victim = ps;
    if (!victim) return nullptr;                 // wait for running requests to finish
    s->plans.erase(std::find(s->plans.begin(), s->plans.end(), victim));
    s->used -= victim->bytes;
    s->plans_evicted++;
    dyson_plan p = victim->plan;
    delete victim;
    lk.unlock();
    dyson_plan_destroy(p);
    lk.lock();
  }
  PlanSlot* ps = new PlanSlot();
  ps->key = q.key;
  ps->busy = true;
  ps->bytes = need;
  s->used += need;                               // reserve before creating
  s->plans.push_back(ps);
  lk.unlock();
  dyson_plan plan = nullptr;
  e = dyson_plan_create(&q.r.geom, &plan);
  std::string msg = e ? dyson_last_error() : "";
  lk.lock();
  if (e) {
    s->plans.erase(std::find(s->plans.begin(), s->plans.end(), ps));
    s->used -= need;
    delete ps;
    *rc = e;
    *err = msg;
    return nullptr;
  }
  ps->plan = plan;
  ps->bytes = dyson_internal_plan_bytes(plan);
  s->plans_created++;
  return ps;
}

void worker_main(dyson_server_s* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    // ---- completions
    for (size_t k = 0; k < s->streams.size(); ++k) {
      uint64_t t = s->stream_owner[k];
      if (!t) continue;
      cudaError_t q = cudaEventQuery(s->events[k]);
      if (q == cudaErrorNotReady) continue;
      const double td = now_s();
      for (uint64_t tg : s->stream_group[k]) {
        Req& r = s->reqs[tg];
        r.t_done = td;
        if (q == cudaSuccess) {
          r.state = Q_DONE;
        } else {
          r.state = Q_FAILED;
          r.rc = DYSON_E_CUDA;
          r.err = std::string("request failed on the device: ") + cudaGetErrorString(q);
        }
        s->completed++;
      }
      Req& r = s->reqs[t];
      r.slot->busy = false;
      r.slot->last_use = td;
      s->stream_owner[k] = 0;
      s->stream_group[k].clear();
      s->cv_done.notify_all();
    }
    if (s->stop && s->queue.empty() && running_count(s) == 0) break;
    // ---- admissions, in arrival order (with backfill, see BACKFILL_PER_HEAD)
    while (!s->queue.empty() && running_count(s) < s->max_inflight) {
      uint64_t t = s->queue.front();
      Req& head = s->reqs[t];
      int rc = DYSON_OK;
      std::string err;
      PlanSlot* ps = acquire_plan(s, head, lk, &rc, &err);
      if (!ps && rc) {                            // cannot be served at all
        head.state = Q_FAILED;
        head.rc = rc;
        head.err = err;
        s->queue.pop_front();
        s->cv_done.notify_all();
        continue;
      }
      if (ps) {
        s->queue.pop_front();
      } else {                                    // the head waits for memory
        if (s->queue.front() != t || head.bypassed >= BACKFILL_PER_HEAD) break;
        for (size_t j = 1; j < s->queue.size() && j <= BACKFILL_WINDOW && !ps; ++j) {
          Req& c = s->reqs[s->queue[j]];
          for (PlanSlot* cand : s->plans)
            if (!cand->busy && cand->key == c.key) {
              ps = cand;
              break;
            }
          if (ps) {
            ps->busy = true;
            t = s->queue[j];
            s->queue.erase(s->queue.begin() + (long)j);
            head.bypassed++;
          }
        }
        if (!ps) break;                           // nothing can run without memory: wait
      }
      Req& q = s->reqs[t];
      int k = 0;
      while (s->stream_owner[k]) ++k;
      s->stream_owner[k] = t;
      s->stream_group[k].assign(1, t);
      const double t0 = now_s();
      q.slot = ps;
      q.stream = k;
      q.state = Q_RUNNING;
      q.t_start = t0;
      s->admitted++;
      const dyson_request r = q.r;
      const int cap = r.geom.max_freqs;
      const size_t N = (size_t)r.geom.L[0] * r.geom.L[1] * (r.geom.dim == 3 ? r.geom.L[2] : 1);
      const size_t nq1 = N * (size_t)(r.geom.block_size > 1 ? r.geom.block_size : 1);
      // fusion: queued requests of this geometry with the same V and start vector(s)
      // join this solve while the frequencies fit the plan
      std::vector<SolveSeg> segs(1, SolveSeg{r.K, r.omega, r.sigma, r.diagG, r.status});
      int Ktot = r.K;
      for (size_t jq = 0; jq < s->queue.size() && (int)segs.size() < FUSE_MAX && Ktot < cap;) {
        Req& c = s->reqs[s->queue[jq]];
        const bool same = c.key == q.key && Ktot + c.r.K <= cap &&
                          (c.r.V == r.V || !std::memcmp(c.r.V, r.V, N * sizeof(double))) &&
                          (c.r.q1 == r.q1 || !std::memcmp(c.r.q1, r.q1, nq1 * sizeof(double)));
        if (!same) {
          ++jq;
          continue;
        }
        const uint64_t tc = s->queue[jq];
        s->queue.erase(s->queue.begin() + (long)jq);
        c.slot = ps;
        c.stream = k;
        c.state = Q_RUNNING;
        c.t_start = t0;
        s->admitted++;
        s->stream_group[k].push_back(tc);
        segs.push_back(SolveSeg{c.r.K, c.r.omega, c.r.sigma, c.r.diagG, c.r.status});
        Ktot += c.r.K;
      }
      if (segs.size() > 1) s->fused += segs.size();
      const int run = running_count(s);
      if (run > s->peak_running) s->peak_running = run;
      if (s->used > s->peak_used) s->peak_used = s->used;
      cudaStream_t st = s->streams[k];
      cudaEvent_t ev = s->events[k];
      lk.unlock();
      int e = DYSON_OK;
      if (segs.size() > 1) {
        e = dyson_internal_solve_enqueue_segs(ps->plan, (int)segs.size(), segs.data(), r.V, r.q1, DYSON_MEM_HOST,
                                              st);
      } else {
        // a request with more frequencies than its plan holds runs as consecutive
        // chunks of max_freqs on the same plan and stream (frequencies are independent)
        for (int k0 = 0; k0 < r.K && !e; k0 += cap) {
          const int kc = r.K - k0 < cap ? r.K - k0 : cap;
          e = dyson_internal_solve_enqueue(ps->plan, kc, r.omega + k0, r.V, r.sigma + 2 * (size_t)k0 * N, r.q1,
                                           r.diagG + 2 * (size_t)k0 * N, r.status ? r.status + k0 : nullptr,
                                           DYSON_MEM_HOST, st);
        }
      }
      std::string msg = e ? dyson_last_error() : "";
      if (!e) {
        cudaError_t ce = cudaEventRecord(ev, st);
        if (ce != cudaSuccess) {
          e = DYSON_E_CUDA;
          msg = cudaGetErrorString(ce);
        }
      }
      lk.lock();
      if (e) {
        const double td = now_s();
        for (uint64_t tg : s->stream_group[k]) {
          Req& qq = s->reqs[tg];
          qq.state = Q_FAILED;
          qq.rc = e;
          qq.err = msg;
          qq.t_done = td;
        }
        ps->busy = false;
        s->stream_owner[k] = 0;
        s->stream_group[k].clear();
        s->cv_done.notify_all();
      }
    }
    if (running_count(s) > 0)
      s->cv_work.wait_for(lk, std::chrono::microseconds(50));
    else
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
  }
}

int srv_fail(int code, const std::string& msg) { return dyson_internal_fail(code, msg); }

}  // namespace

extern "C" {

int dyson_server_create(size_t hbm_budget, int max_inflight, dyson_server* out) {
  if (!out) return srv_fail(DYSON_E_BAD_ARG, "out is NULL");
  if (hbm_budget == 0) return srv_fail(DYSON_E_BAD_ARG, "hbm_budget must be > 0");
  if (max_inflight < 1 || max_inflight > 64) return srv_fail(DYSON_E_BAD_ARG, "max_inflight must be in 1..64");
  dyson_server_s* s = new dyson_server_s();
  s->budget = hbm_budget;
  s->max_inflight = max_inflight;
  cudaGetDevice(&s->device);
  s->streams.resize(max_inflight);
  s->events.resize(max_inflight);
  s->stream_owner.assign(max_inflight, 0);
  s->stream_group.assign(max_inflight, {});
  for (int k = 0; k < max_inflight; ++k) {
    cudaError_t e = cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->events[k], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (int j = 0; j < k; ++j) {
        cudaStreamDestroy(s->streams[j]);
        cudaEventDestroy(s->events[j]);
      }
      delete s;
      return srv_fail(DYSON_E_CUDA, std::string("server streams: ") + cudaGetErrorString(e));
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return DYSON_OK;
}

int dyson_server_destroy(dyson_server s) {
  if (!s) return DYSON_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->worker.join();
  cudaSetDevice(s->device);
  for (PlanSlot* ps : s->plans) {
    dyson_plan_destroy(ps->plan);
    delete ps;
  }
  for (size_t k = 0; k < s->streams.size(); ++k) {
    cudaStreamDestroy(s->streams[k]);
    cudaEventDestroy(s->events[k]);
  }
  delete s;
  return DYSON_OK;
}

int dyson_submit(dyson_server s, const dyson_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return srv_fail(DYSON_E_BAD_ARG, "NULL server, request or ticket");
  if (r->K < 1 || r->geom.max_freqs < 1)
    return srv_fail(DYSON_E_BAD_ARG, "request K and geom.max_freqs must be >= 1");
  if (!r->omega || !r->V || !r->sigma || !r->q1 || !r->diagG)
    return srv_fail(DYSON_E_BAD_ARG, "request buffers must not be NULL");
  size_t need = 0;
  int rc = dyson_plan_footprint(&r->geom, &need);
  if (rc) return rc;
  if (need > s->budget)
    return srv_fail(DYSON_E_BUDGET, "request needs " + std::to_string(need) +
                                        " device bytes, more than the server budget " +
                                        std::to_string(s->budget));
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return srv_fail(DYSON_E_BAD_ARG, "server is shutting down");
    const uint64_t t = s->next_ticket++;
    Req& q = s->reqs[t];
    q.r = *r;
    // several requests already share the GPU: frequency groups inside one solve would
    // only add graph branches, so the server runs each solve as one batch by default
    if (q.r.geom.freq_groups == 0) q.r.geom.freq_groups = 1;
    q.key = geom_key(q.r.geom);
    q.t_submit = now_s();
    s->queue.push_back(t);
    *ticket = t;
  }
  s->cv_work.notify_all();
  return DYSON_OK;
}

int dyson_poll(dyson_server s, uint64_t ticket, int* done) {
  if (!s || !done) return srv_fail(DYSON_E_BAD_ARG, "NULL server or done");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return srv_fail(DYSON_E_NOT_FOUND, "unknown ticket");
  *done = (it->second.state == Q_DONE || it->second.state == Q_FAILED) ? 1 : 0;
  if (it->second.state == Q_FAILED) return srv_fail(it->second.rc, it->second.err);
  return DYSON_OK;
}

int dyson_wait(dyson_server s, uint64_t ticket, double* latency_ms, double* run_ms) {
  if (!s) return srv_fail(DYSON_E_BAD_ARG, "NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return srv_fail(DYSON_E_NOT_FOUND, "unknown ticket");
  s->cv_done.wait(lk, [&] {
    const int st = s->reqs[ticket].state;
    return st == Q_DONE || st == Q_FAILED;
  });
  Req q = s->reqs[ticket];
  s->reqs.erase(ticket);
  lk.unlock();
  if (latency_ms) *latency_ms = (q.t_done - q.t_submit) * 1e3;
  if (run_ms) *run_ms = (q.t_done - q.t_start) * 1e3;
  if (q.state == Q_FAILED) return srv_fail(q.rc, q.err);
  return DYSON_OK;
}

int dyson_server_stats(dyson_server s, dyson_server_stats_t* out) {
  if (!s || !out) return srv_fail(DYSON_E_BAD_ARG, "NULL server or stats");
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int)s->queue.size();
  out->running = running_count(s);
  out->resident_plans = (int)s->plans.size();
  out->bytes_in_use = s->used;
  out->peak_bytes = s->peak_used;
  out->peak_running = s->peak_running;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->plans_created = s->plans_created;
  out->plans_evicted = s->plans_evicted;
  out->fused = s->fused;
  return DYSON_OK;
}

}  // extern "C"
