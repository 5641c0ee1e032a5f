// Launch counting and per-class CUDA-event timing (see prof.hpp).
#include <string.h>

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

struct State {
  int64_t launches = 0;
  int64_t per_class_launches[KC_COUNT] = {};
  bool on = false;
  int target = -1;  // -1: all classes
  std::vector<cudaEvent_t> pool;
  std::vector<Pending> pending;
  cudaEvent_t open_a = nullptr;
  bool capturing = false;
  int open_id = -1;
  int64_t timed_launches[KC_COUNT] = {};
  double ms[KC_COUNT] = {};
  double bytes[KC_COUNT] = {};
};
State g;

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
    "vector", "reduce", "transfer", "setup", "coarse_solve"};

}  // namespace

void prof_pre(int id, cudaStream_t s) {
  g.launches++;
  if (id >= 0 && id < KC_COUNT) g.per_class_launches[id]++;
  if (g.on && !g.capturing && (g.target < 0 || g.target == id)) {
    g.open_a = take_event();
    g.open_id = id;
    if (g.open_a) cudaEventRecord(g.open_a, s);
  }
}

void prof_post(int id, double bytes, cudaStream_t s) {
  if (g.open_a && g.open_id == id) {
    cudaEvent_t b = take_event();
    if (b) {
      cudaEventRecord(b, s);
      g.pending.push_back(Pending{id, bytes, g.open_a, b});
    } else {
      g.pool.push_back(g.open_a);
    }
    g.open_a = nullptr;
    g.open_id = -1;
    if (g.pending.size() >= 8192) harvest();
  }
}

void prof_add_launches(int64_t n) { g.launches += n; }
void prof_set_capturing(bool on) { g.capturing = on; }
int64_t prof_launches() { return g.launches; }

const char* kclass_name(int id) {
  static thread_local std::string s;
  if (id < 0 || id >= KC_COUNT) return "";
  int base = id % KC_BASE_COUNT, var = id / KC_BASE_COUNT;
  s = BASE_NAMES[base];
  s += (var & 2) ? "_f64" : "_f32";
  s += (var & 1) ? "_coarse" : "_l0";
  return s.c_str();
}

}  // namespace pf

extern "C" {

pf_status pf_prof_enable(int on, int kernel_class) {
  pf::harvest();
  pf::g.on = on != 0;
  pf::g.target = kernel_class;
  return PF_OK;
}

pf_status pf_prof_reset(void) {
  pf::harvest();
  memset(pf::g.timed_launches, 0, sizeof pf::g.timed_launches);
  memset(pf::g.ms, 0, sizeof pf::g.ms);
  memset(pf::g.bytes, 0, sizeof pf::g.bytes);
  memset(pf::g.per_class_launches, 0, sizeof pf::g.per_class_launches);
  pf::g.launches = 0;
  return PF_OK;
}

int64_t pf_launch_count(void) { return pf::g.launches; }

int pf_prof_class_count(void) { return pf::KC_COUNT; }

pf_status pf_prof_get(int kernel_class, const char** name, int64_t* launches, int64_t* timed,
                      double* ms, double* bytes) {
  if (kernel_class < 0 || kernel_class >= pf::KC_COUNT) return PF_EINVAL;
  pf::harvest();
  if (name) *name = pf::kclass_name(kernel_class);
  if (launches) *launches = pf::g.per_class_launches[kernel_class];
  if (timed) *timed = pf::g.timed_launches[kernel_class];
  if (ms) *ms = pf::g.ms[kernel_class];
  if (bytes) *bytes = pf::g.bytes[kernel_class];
  return PF_OK;
}

}  // extern "C"
