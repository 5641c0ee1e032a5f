// Launch accounting and optional CUDA-event timing of kernel classes.
//
// Every kernel launch of the library goes through PF_LAUNCH, which counts it and, when timing
// is enabled for its class, brackets it with two events recorded on the launching stream.  The
// algorithmic bytes of each launch (compulsory reads and writes of the operator on its grid) are
// accumulated beside the measured time so achieved bandwidth can be computed per class.
// Process-wide state.  Launch counts are exact from any number of host threads; event timing
// is thread-safe but meant for single-threaded measurement runs (concurrent work on other
// streams would inflate the bracketed times).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pf {

enum KernelClass : int {
  KC_EL_APPLY = 0, KC_EL_MASKED, KC_EL_RESB, KC_EL_RESID, KC_EL_CHEB,
  KC_DM_APPLY, KC_DM_MASKED, KC_DM_RESB, KC_DM_CHEB, KC_DM_GRAD, KC_DM_TRIAL,
  KC_VECTOR, KC_REDUCE, KC_TRANSFER, KC_SETUP, KC_COARSE, KC_TAIL,
  KC_EL_RESID_DF, KC_DM_GRAD_DF, KC_DM_TRIAL_DF,  // FP64 in/out, double-float arithmetic
  // smoothing from zero: the first (pointwise) Chebyshev step formed inside the second one's
  // launch, or inside the residual's when it is the only pre-smoothing step
  KC_EL_CHEB_Z, KC_DM_CHEB_Z, KC_EL_RESB_Z, KC_DM_RESB_Z,
  KC_DM_Q, KC_DM_Q_DF,  // element energy densities of the damage operator: FP64, double-float
  KC_BASE_COUNT
};
// class id = base + KC_BASE_COUNT * (precision * KC_LEVELS + multigrid level), so that one class
// is one kernel at one problem size (deeper levels than KC_LEVELS - 1 share the last class)
constexpr int KC_LEVELS = 10;
constexpr int KC_COUNT = KC_BASE_COUNT * 2 * KC_LEVELS;

inline int kclass(int base, bool fp64, int level) {
  level = level < 0 ? 0 : (level >= KC_LEVELS ? KC_LEVELS - 1 : level);
  return base + KC_BASE_COUNT * ((fp64 ? KC_LEVELS : 0) + level);
}

void prof_pre(int id, cudaStream_t s);
// launches replayed by graphs are added here; while capturing, event timing is suspended
void prof_add_launches(int64_t n);
void prof_set_capturing(bool on);
// kernels this thread recorded since prof_set_capturing(true)
int64_t prof_captured();
int64_t prof_launches();
void prof_post(int id, double bytes, cudaStream_t s);
const char* kclass_name(int id);
// a launch that failed records its expression (this thread; read by the error reporting)
void prof_note_launch(const char* expr);
const char* prof_failed_launch();

}  // namespace pf

#define PF_LAUNCH(ID, BYTES, STREAM, ...)      \
  do {                                         \
    ::pf::prof_pre((ID), (STREAM));            \
    __VA_ARGS__;                               \
    ::pf::prof_note_launch(#__VA_ARGS__);      \
    ::pf::prof_post((ID), (BYTES), (STREAM));  \
  } while (0)
