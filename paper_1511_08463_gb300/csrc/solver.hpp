// Host-side data structures of libpf: the sim, its multigrid hierarchy and work buffers.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "kernels.cuh"

// One per GPU.  Owns a pool of small pinned host buffers (one per live sim, for scalar
// read-back), grown in chunks and released only with the context, so that creating and
// destroying sims never calls cudaFreeHost (which may synchronize the device) while other
// sims run.  Sims and servers hold a reference: pf_ctx_destroy frees the context once the last
// of them is gone, whatever the order in which the caller releases them.
struct pf_ctx {
  int device = 0;
  std::mutex mu;
  std::vector<double*> chunks;      // cudaMallocHost blocks
  std::vector<double*> free_slots;  // 64-double slots not in use
  int users = 0;                    // live sims and servers
  bool closed = false;              // pf_ctx_destroy was called
  double* take_slot();              // also registers a user
  void give_slot(double* p);        // also unregisters it; may free the context
  void add_user();
  void drop_user();                 // may free the context
};

namespace pf {

template <class T>
struct LevelBuf {
  T* coefE = nullptr;   // elastic abar per element
  T* dinvE = nullptr;   // inverse l1 diagonal (2n)
  T* wD = nullptr;      // damage mass weight per element
  T* dinvD = nullptr;   // (n)
  T *b = nullptr, *x = nullptr, *r = nullptr, *xt = nullptr, *d = nullptr, *dt = nullptr;  // 2n
  T *AE = nullptr, *AD = nullptr, *diagE = nullptr, *diagD = nullptr;  // coarsest dense
  T *AEi = nullptr, *ADi = nullptr;  // coarsest explicit inverses
};

struct Level {
  Grid g;
  LevelBuf<double> f64;
  LevelBuf<float> f32;
  bool dense = false;  // coarsest level solved by dense Cholesky
  uint8_t* exclD = nullptr;  // damage: active-set mask of this coarse level (level 0 uses the sim's)
  template <class T>
  LevelBuf<T>& buf();
};
template <>
inline LevelBuf<double>& Level::buf<double>() { return f64; }
template <>
inline LevelBuf<float>& Level::buf<float>() { return f32; }

template <class T>
struct Krylov {
  T *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *Ap = nullptr;
};

// scalar slots in device memory
enum Slot {
  S_RR = 0, S_RZ0 = 1, S_RZ1 = 2, S_PAP = 3, S_RES = 4, S_DU = 5,   // S_DU: 2 values
  S_OMEGA = 8, S_DALPHA = 9, S_PHI = 10,                            // S_PHI: 2 values
  S_EN = 12,                                                         // 2 values
  S_TMP = 16, S_TOL2 = 20, S_IT = 21, S_MAXIT = 22, S_COUNT = 32
};

// shared with other translation units of the library
void set_error_message(const char* msg);
pf_status describe_mesh(const pf_mesh_desc* d, Grid* g);      // validate + level-0 grid
pf_status describe_material(const pf_material* m, Mat* out);  // validate + kernel constants
// stream-ordered variants of pf_create_mesh and pf_get_fields (no device-wide synchronization)
pf_status create_sim(pf_ctx* ctx, const pf_mesh_desc* d, void* ws, size_t ws_bytes,
                     cudaStream_t st, pf_sim** out);
pf_status fields_to_host(pf_sim* s, cudaStream_t st, double* u, double* alpha, double* alpha_prev);

}  // namespace pf

struct pf_sim {
  pf_ctx* ctx = nullptr;
  pf_mesh_desc desc;
  pf::Mat m;
  bool have_material = false;
  pf_material mat_in;
  std::vector<pf::Level> lv;
  pf::LiftData lift;
  double t = 0.0, dT = 0.0;
  bool thermal = false;  // eigenstrain table valid and nonzero
  // resident state (FP64)
  double *u = nullptr, *alpha = nullptr, *alpha_prev = nullptr;
  float* alpha32 = nullptr;
  // FP64 work
  double *xu = nullptr, *r64 = nullptr, *q = nullptr, *eig = nullptr;
  double *xrs = nullptr, *F = nullptr, *Phi = nullptr, *rhs = nullptr, *drs = nullptr;
  double *xtr = nullptr, *Ftr = nullptr, *Phitr = nullptr, *rhstr = nullptr;
  double *tmpa = nullptr, *tmpb = nullptr;
  uint8_t *act = nullptr, *acttr = nullptr;
  float* tmp32 = nullptr;
  // Newton (ORAM-N): FP32 copies of the state, 12 work vectors of 3n floats ([u | alpha]),
  // FP64 step start and direction
  float *u32 = nullptr, *eig32 = nullptr;
  float* nv[12] = {};
  double *nu0 = nullptr, *na0 = nullptr, *ndu = nullptr, *nda = nullptr;
  pf::Krylov<double> k64;
  pf::Krylov<float> k32;
  // reductions
  double* part = nullptr;
  unsigned* ticket = nullptr;
  double* scal = nullptr;
  // per-step tolerance scales
  double r_scale = 0.0, phi_scale = 0.0;
  // MG state validity
  bool elastic_ready64 = false, elastic_ready32 = false, damage_ready64 = false,
       damage_ready32 = false;
  // xu holds the u-subproblem minimizer for the current alpha and load
  bool xu_valid = false;
  int xu_precision = -1;
  size_t ws_used = 0;
  std::atomic<bool> busy{false};  // a load step is running (PF_EBUSY for a second caller)
  // CUDA graphs holding one whole PCG solve each (device-side while loop), per operator
  // (elastic, damage) and precision (FP32, FP64); rebuilt if the smoothing degree or the number of
  // levels in use changes
  bool use_graphs = true;
  cudaGraph_t cg_graph[2][2] = {};
  cudaGraphExec_t cg_exec[2][2] = {};
  int cg_body_kernels[2][2] = {};
  int cg_deg[2][2] = {};
  int cg_nl[2][2] = {};
  // multigrid levels used by the solves (pf_solver_opts.mg_levels_max; all by default)
  int nl_active = 1;
  // single-block tail of the FP32 V-cycle (pf_solver_opts.mg_tail): first level per operator
  // (-1: none; -2: not computed yet) and its shared-memory bytes
  bool use_tail = true;
  int cdeg = 2;  // Chebyshev steps per smoothing on levels >= 1 (pf_solver_opts.mg_coarse_degree)
  int tail_first[2] = {-2, -2};
  int cg_tail[2][2] = {};
  int cg_tiles[2][2] = {};  // tile configuration the graph was captured with
  int tile_fine = 0, tile_coarse = 0;  // FP32 stencil tile heights (0: default)
  // the FP64-data kernels (physical residual, damage gradient and trial point) compute in
  // double-float: set for PF_MIXED solves, whose refinement only needs ~14 digits
  bool df = false;
  double* host = nullptr;  // pinned read-back slot from the context's pool
  ~pf_sim() {
    if (host && ctx) ctx->give_slot(host);
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        if (cg_exec[a][b]) cudaGraphExecDestroy(cg_exec[a][b]);
        if (cg_graph[a][b]) cudaGraphDestroy(cg_graph[a][b]);
      }
  }
};
