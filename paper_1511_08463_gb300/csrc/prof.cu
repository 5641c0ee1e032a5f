// Launch counting and per-class CUDA-event timing (see prof.hpp).
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "pf.h"
#include "prof.hpp"

namespace pf {
namespace {

struct Pending {
  int id;
  double bytes;
  cudaEvent_t a, b;
};

// Counters are atomic so that sims driven from several host threads count correctly; the event
// timing path (used by single-threaded measurement runs) takes a lock.
struct State {
  std::atomic<int64_t> launches{0};
  std::atomic<int64_t> per_class_launches[KC_COUNT] = {};
  std::atomic<bool> on{false};
  std::atomic<int> target{-1};  // -1: all classes
  std::mutex mu;                // guards pool, pending and the timing sums
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  int64_t timed_launches[KC_COUNT] = {};
  double ms[KC_COUNT] = {};
  double bytes[KC_COUNT] = {};
};
State g;
// per host thread: the launch currently bracketed and whether this thread is capturing a graph
thread_local cudaEvent_t t_open_a = nullptr;
thread_local int t_open_id = -1;
thread_local bool t_capturing = false;
thread_local int64_t t_captured = 0;  // launches recorded into a graph by this thread

cudaEvent_t take_event() {
  if (g.pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = g.pool.back();
  g.pool.pop_back();
  return e;
}

void harvest() {
  for (Pending& p : g.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      g.ms[p.id] += ms;
      g.bytes[p.id] += p.bytes;
      g.timed_launches[p.id] += 1;
    }
    g.pool.push_back(p.a);
    g.pool.push_back(p.b);
  }
  g.pending.clear();
}

const char* BASE_NAMES[KC_BASE_COUNT] = {
    "elastic_apply", "elastic_masked", "elastic_resb", "elastic_resid", "elastic_cheb",
    "damage_apply", "damage_masked", "damage_resb", "damage_cheb", "damage_grad", "damage_trial",
    "vector", "reduce", "transfer", "setup", "coarse_solve", "tail_vcycle",
    "elastic_resid_df", "damage_grad_df", "damage_trial_df",
    "elastic_cheb_z", "damage_cheb_z", "elastic_resb_z", "damage_resb_z", "damage_q", "damage_q_df"};

}  // namespace

void prof_pre(int id, cudaStream_t s) {
  if (t_capturing) {  // not a launch yet: counted each time the graph replays it
    ++t_captured;
    return;
  }
  g.launches.fetch_add(1, std::memory_order_relaxed);
  if (id >= 0 && id < KC_COUNT) g.per_class_launches[id].fetch_add(1, std::memory_order_relaxed);
  if (g.on.load(std::memory_order_relaxed) && !t_capturing) {
    const int tg = g.target.load(std::memory_order_relaxed);
    if (tg < 0 || tg == id) {
      std::lock_guard<std::mutex> lk(g.mu);
      t_open_a = take_event();
      t_open_id = id;
      if (t_open_a) cudaEventRecord(t_open_a, s);
    }
  }
}

void prof_post(int id, double bytes, cudaStream_t s) {
  if (t_open_a && t_open_id == id) {
    std::lock_guard<std::mutex> lk(g.mu);
    cudaEvent_t b = take_event();
    if (b) {
      cudaEventRecord(b, s);
      g.pending.push_back(Pending{id, bytes, t_open_a, b});
    } else {
      g.pool.push_back(t_open_a);
    }
    t_open_a = nullptr;
    t_open_id = -1;
    if (g.pending.size() >= 8192) harvest();
  }
}

namespace {
thread_local std::string t_failed_launch;
}
void prof_note_launch(const char* expr) {
  if (t_failed_launch.empty() && cudaPeekAtLastError() != cudaSuccess) t_failed_launch = expr;
}
const char* prof_failed_launch() { return t_failed_launch.c_str(); }

void prof_add_launches(int64_t n) { g.launches.fetch_add(n, std::memory_order_relaxed); }
void prof_set_capturing(bool on) {
  t_capturing = on;
  if (on) t_captured = 0;
}
int64_t prof_captured() { return t_captured; }
int64_t prof_launches() { return g.launches.load(); }

const char* kclass_name(int id) {
  static thread_local std::string s;
  if (id < 0 || id >= KC_COUNT) return "";
  const int base = id % KC_BASE_COUNT, var = id / KC_BASE_COUNT;
  s = BASE_NAMES[base];
  s += var >= KC_LEVELS ? "_f64_l" : "_f32_l";
  s += std::to_string(var % KC_LEVELS);
  return s.c_str();
}

}  // namespace pf

extern "C" {

pf_status pf_prof_enable(int on, int kernel_class) {
  std::lock_guard<std::mutex> lk(pf::g.mu);
  pf::harvest();
  pf::g.on = on != 0;
  pf::g.target = kernel_class;
  return PF_OK;
}

pf_status pf_prof_reset(void) {
  std::lock_guard<std::mutex> lk(pf::g.mu);
  pf::harvest();
  memset(pf::g.timed_launches, 0, sizeof pf::g.timed_launches);
  memset(pf::g.ms, 0, sizeof pf::g.ms);
  memset(pf::g.bytes, 0, sizeof pf::g.bytes);
  for (auto& c : pf::g.per_class_launches) c = 0;
  pf::g.launches = 0;
  return PF_OK;
}

int64_t pf_launch_count(void) { return pf::g.launches.load(); }

int pf_prof_class_count(void) { return pf::KC_COUNT; }

pf_status pf_prof_get(int kernel_class, const char** name, int64_t* launches, int64_t* timed,
                      double* ms, double* bytes) {
  if (kernel_class < 0 || kernel_class >= pf::KC_COUNT) return PF_EINVAL;
  std::lock_guard<std::mutex> lk(pf::g.mu);
  pf::harvest();
  if (name) *name = pf::kclass_name(kernel_class);
  if (launches) *launches = pf::g.per_class_launches[kernel_class];
  if (timed) *timed = pf::g.timed_launches[kernel_class];
  if (ms) *ms = pf::g.ms[kernel_class];
  if (bytes) *bytes = pf::g.bytes[kernel_class];
  return PF_OK;
}

}  // extern "C"
