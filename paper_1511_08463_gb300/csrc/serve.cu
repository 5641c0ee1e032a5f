// Host runtime for many simulations on one GPU: the concurrent batch call and the serving loop.
//
// Both run whole load steps (Algorithm 2 or 3 for one pf_load) of different sims at the same time
// from several host threads, each thread driving its own non-blocking CUDA stream, so that the
// latency-bound small kernels of small meshes overlap on the device.  A load step is the unit
// of scheduling: a step is host-synchronous (its convergence tests read scalars back), and any
// thread may run the next step of any sim once the previous one has returned.
//
// Serving (continuous batching): jobs -- a mesh, a material, a list of load steps and solver
// options -- arrive over time.  A job is admitted, in arrival order, as soon as its workspace
// (pf_workspace_bytes) fits in the free part of a caller-owned device arena; its state then
// stays resident until its last step.  Workers take the next step of the admitted job that has
// waited longest (round robin), so jobs admitted while others run share the device with them.
// Results do not depend on the mix: every kernel and reduction of a step is deterministic and
// independent of what else runs.
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "arena.hpp"
#include "solver.hpp"

using namespace pf;

using pf::ArenaAlloc;
using pf::ARENA_ALIGN;
using pf::round_up;

namespace {

pf_status fail(pf_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error_message(buf);
  return st;
}
#define CU(call)                                                                    \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      return fail(PF_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

inline pf_status worse(pf_status a, pf_status b) { return a > b ? a : b; }

struct Job {
  int64_t id = 0;
  pf_job d{};
  std::vector<pf_load> loads;
  double arrival = 0.0;  // server clock, seconds
  size_t bytes = 0, off = 0;
  pf_sim* sim = nullptr;
  int next = 0;
  double ready_at = 0.0;
  pf_status status = PF_OK;
  bool done = false;
  double admitted = -1.0, finished = -1.0;
};

}  // namespace

struct pf_server {
  pf_ctx* ctx = nullptr;
  char* arena = nullptr;
  ArenaAlloc alloc;
  std::mutex mu;
  std::condition_variable cv;       // work may be available
  std::condition_variable done_cv;  // a job finished
  std::deque<Job*> pending;         // not yet admitted, by arrival time
  std::deque<Job*> ready;           // admitted, next step not running
  std::map<int64_t, std::unique_ptr<Job>> jobs;
  int64_t next_id = 0;
  int64_t unfinished = 0;
  int active = 0, max_active = 0;
  int64_t steps_done = 0, jobs_done = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void finish_locked(Job* j, double t) {
    if (j->bytes) alloc.release(j->off, j->bytes);
    j->done = true;
    j->finished = t;
    --unfinished;
    ++jobs_done;
    done_cv.notify_all();
    cv.notify_all();  // freed memory may admit the next job
  }
  void worker(int w);
};

void pf_server::worker(int w) {
  cudaSetDevice(ctx->device);
  cudaStream_t st = streams[w];
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // 1. admission: the earliest arrived job, if its workspace fits now
    if (!pending.empty()) {
      Job* j = pending.front();
      size_t off = 0;
      if (j->arrival <= now() && alloc.alloc(j->bytes, &off)) {
        pending.pop_front();
        j->off = off;
        ++active;
        max_active = std::max(max_active, active);
        lk.unlock();
        pf_sim* sim = nullptr;
        pf_status e = create_sim(ctx, &j->d.mesh, arena + off, j->bytes, st, &sim);
        if (e == PF_OK) e = pf_set_material(sim, &j->d.material);
        const double t = now();
        lk.lock();
        j->admitted = t;
        j->ready_at = j->arrival;
        if (e != PF_OK) {
          if (sim) pf_destroy(sim);
          j->status = e;
          --active;
          finish_locked(j, t);
        } else {
          j->sim = sim;
          ready.push_back(j);
          cv.notify_one();
        }
        continue;
      }
    }
    // 2. the next load step of the job that has waited longest
    if (!ready.empty()) {
      Job* j = ready.front();
      ready.pop_front();
      const int k = j->next;
      lk.unlock();
      pf_step_report rep{};
      pf_status e = pf_load_step(j->sim, &j->loads[k], &j->d.opts, st, &rep);
      const double t_end = now();
      if (j->d.reports) j->d.reports[k] = rep;
      if (j->d.step_latency) j->d.step_latency[k] = t_end - j->ready_at;
      const bool fatal = e != PF_OK && e != PF_ENOTCONV;
      const bool last = fatal || k + 1 == (int)j->loads.size();
      if (last) {
        pf_status e2 = fields_to_host(j->sim, st, j->d.u_out, j->d.alpha_out, nullptr);
        if (e2 != PF_OK) e = worse(e, e2);
        pf_destroy(j->sim);
        j->sim = nullptr;
      }
      lk.lock();
      j->status = worse(j->status, e);
      j->next = k + 1;
      j->ready_at = t_end;
      ++steps_done;
      if (last) {
        --active;
        finish_locked(j, t_end);
      } else {
        ready.push_back(j);
      }
      continue;
    }
    if (stop && unfinished == 0) break;
    // 3. nothing to do: sleep until the next arrival or a notification
    if (!pending.empty() && pending.front()->arrival > now()) {
      const double dt = pending.front()->arrival - now();
      cv.wait_for(lk, std::chrono::duration<double>(std::max(dt, 0.0)));
    } else {
      cv.wait(lk);
    }
  }
}

namespace {

// Concurrent pf_solve_batch: up to o->batch_workers host threads (default 8), largest meshes
// first, each thread on its own stream forked from and joined back into the caller's stream.
pf_status solve_batch(pf_ctx* ctx, pf_sim* const* sims, const pf_load* loads, int n,
                      const pf_solver_opts* o, cudaStream_t caller, pf_step_report* reps) {
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return sims[a]->lv[0].g.n > sims[b]->lv[0].g.n; });
  const int W = std::max(1, std::min(n, o->batch_workers > 0 ? o->batch_workers : 8));
  CU(cudaSetDevice(ctx->device));
  cudaEvent_t fork;
  CU(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  CU(cudaEventRecord(fork, caller));
  std::vector<cudaStream_t> st(W, nullptr);
  std::vector<cudaEvent_t> join(W, nullptr);
  pf_status setup = PF_OK;
  for (int w = 0; w < W && setup == PF_OK; ++w) {
    if (cudaStreamCreateWithFlags(&st[w], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&join[w], cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamWaitEvent(st[w], fork, 0) != cudaSuccess)
      setup = fail(PF_ECUDA, "batch: stream setup failed");
  }
  std::vector<pf_status> res(n, PF_OK);
  if (setup == PF_OK) {
    std::atomic<int> next{0};
    auto run = [&](int w) {
      cudaSetDevice(ctx->device);
      for (int k = next++; k < n; k = next++) {
        const int i = order[k];
        pf_step_report r{};
        res[i] = pf_load_step(sims[i], &loads[i], o, st[w], &r);
        if (reps) reps[i] = r;
      }
      cudaEventRecord(join[w], st[w]);
    };
    std::vector<std::thread> th;
    for (int w = 1; w < W; ++w) th.emplace_back(run, w);
    run(0);
    for (auto& t : th) t.join();
    for (int w = 0; w < W; ++w) cudaStreamWaitEvent(caller, join[w], 0);
  }
  for (int w = 0; w < W; ++w) {
    if (join[w]) cudaEventDestroy(join[w]);
    if (st[w]) cudaStreamDestroy(st[w]);
  }
  cudaEventDestroy(fork);
  if (setup != PF_OK) return setup;
  pf_status worst = PF_OK;
  for (int i = 0; i < n; ++i) worst = worse(worst, res[i]);
  return worst;
}

}  // namespace

extern "C" {

pf_status pf_solve_batch(pf_ctx* ctx, pf_sim* const* sims, const pf_load* loads, int n,
                         const pf_solver_opts* o, void* stream, pf_step_report* reps) {
  if (!ctx || !o || n < 0 || (n > 0 && (!sims || !loads))) return fail(PF_EINVAL, "null argument");
  for (int i = 0; i < n; ++i) {
    if (!sims[i]) return fail(PF_EINVAL, "batch: sim %d is null", i);
    if (sims[i]->ctx != ctx) return fail(PF_EINVAL, "batch: sim %d belongs to another context", i);
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) return fail(PF_EINVAL, "batch: sim %d appears twice", i);
  }
  if (n == 0) return PF_OK;
  return solve_batch(ctx, sims, loads, n, o, static_cast<cudaStream_t>(stream), reps);
}

pf_status pf_server_create(pf_ctx* ctx, void* arena, size_t arena_bytes, int n_workers,
                           pf_server** out) {
  if (!ctx || !arena || !out) return fail(PF_EINVAL, "null argument");
  if (reinterpret_cast<uintptr_t>(arena) % ARENA_ALIGN)
    return fail(PF_EINVAL, "arena not %zu-byte aligned", ARENA_ALIGN);
  if (n_workers < 1 || n_workers > 256) return fail(PF_EINVAL, "n_workers must be in [1, 256]");
  CU(cudaSetDevice(ctx->device));
  std::unique_ptr<pf_server> s(new (std::nothrow) pf_server);
  if (!s) return fail(PF_ENOMEM, "host allocation failed");
  s->ctx = ctx;
  s->arena = static_cast<char*>(arena);
  s->alloc.init(arena_bytes / ARENA_ALIGN * ARENA_ALIGN);
  s->streams.assign(n_workers, nullptr);
  for (int w = 0; w < n_workers; ++w)
    if (cudaStreamCreateWithFlags(&s->streams[w], cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams)
        if (x) cudaStreamDestroy(x);
      return fail(PF_ECUDA, "server: stream creation failed");
    }
  ctx->add_user();
  pf_server* raw = s.get();
  for (int w = 0; w < n_workers; ++w) s->workers.emplace_back([raw, w] { raw->worker(w); });
  *out = s.release();
  return PF_OK;
}

double pf_server_now(const pf_server* s) { return s ? s->now() : 0.0; }

pf_status pf_server_submit(pf_server* s, const pf_job* job, int64_t* id) {
  if (!s || !job || !id) return fail(PF_EINVAL, "null argument");
  if (job->n_loads < 1 || !job->loads) return fail(PF_EINVAL, "job needs at least one load step");
  const size_t bytes = pf_workspace_bytes(&job->mesh, job->opts.precision);
  if (bytes == 0) return fail(PF_EINVAL, "invalid mesh descriptor");
  if (round_up(bytes) > s->alloc.size())
    return fail(PF_ENOMEM, "job needs %zu bytes, arena holds %zu", bytes, s->alloc.size());
  std::unique_ptr<Job> j(new (std::nothrow) Job);
  if (!j) return fail(PF_ENOMEM, "host allocation failed");
  j->d = *job;
  j->loads.assign(job->loads, job->loads + job->n_loads);
  j->bytes = bytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail(PF_EINVAL, "server is shutting down");
  j->arrival = job->arrival >= 0.0 ? job->arrival : s->now();
  j->id = s->next_id++;
  Job* p = j.get();
  s->jobs[j->id] = std::move(j);
  // keep pending ordered by arrival (stable for equal times)
  auto pos = std::upper_bound(s->pending.begin(), s->pending.end(), p,
                              [](const Job* a, const Job* b) { return a->arrival < b->arrival; });
  s->pending.insert(pos, p);
  ++s->unfinished;
  *id = p->id;
  s->cv.notify_all();
  return PF_OK;
}

pf_status pf_server_wait(pf_server* s, int64_t id, pf_job_info* info) {
  if (!s) return fail(PF_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(id);
  if (it == s->jobs.end()) return fail(PF_EINVAL, "unknown job %lld", (long long)id);
  Job* j = it->second.get();
  s->done_cv.wait(lk, [j] { return j->done; });
  if (info) {
    info->status = j->status;
    info->steps_done = j->next;
    info->arrival = j->arrival;
    info->admitted = j->admitted;
    info->finished = j->finished;
    info->footprint = j->bytes;
  }
  return PF_OK;
}

pf_status pf_server_drain(pf_server* s) {
  if (!s) return fail(PF_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  s->done_cv.wait(lk, [s] { return s->unfinished == 0; });
  return PF_OK;
}

pf_status pf_server_get_stats(pf_server* s, pf_server_stats* out) {
  if (!s || !out) return fail(PF_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->jobs_done = s->jobs_done;
  out->steps_done = s->steps_done;
  out->arena_bytes = s->alloc.size();
  out->arena_peak = s->alloc.peak();
  out->max_active = s->max_active;
  out->workers = (int32_t)s->workers.size();
  return PF_OK;
}

void pf_server_destroy(pf_server* s) {
  if (!s) return;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->done_cv.wait(lk, [s] { return s->unfinished == 0; });
    s->stop = true;
    s->cv.notify_all();
  }
  for (auto& t : s->workers) t.join();
  for (cudaStream_t x : s->streams)
    if (x) cudaStreamDestroy(x);
  pf_ctx* ctx = s->ctx;
  delete s;
  ctx->drop_user();
}

}  // extern "C"
