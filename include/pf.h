/*
 * pf.h -- C ABI of the GB300 phase-field fracture solver library (libpf.so).
 *
 * The library solves, one quasi-static load step at a time, the regularized fracture problem of
 * Farrell & Maurini, "Linear and nonlinear solvers for variational phase-field models of brittle
 * fracture": find a stationary point of
 *
 *   E(u, a) = int 1/2 a(a) A0 eps_eff(u):eps_eff(u) + Gc/c_w (w(a)/ell + ell |grad a|^2)
 *
 * (Section 1.1, eq. regenergy; thermal eigenstrain of eq. energytshock) over u in C_ubar and
 * alpha in D_alpha_prev = { alpha_prev <= alpha <= 1 } (Section 1.1), with P1 triangles on a
 * structured rectangle (Section 1.2, finite-element discretization).  Nonlinear solvers:
 * alternate minimization (Algorithm 1), its over-relaxation ORAM (Algorithm 2) and ORAM composed
 * with active-set Newton (Algorithm 3, Algorithm 4).  The linear subproblems (Section 3) are
 * solved matrix-free by preconditioned CG with a geometric multigrid V-cycle.
 *
 * Conventions for every function:
 *  - returns pf_status; never throws or aborts across the ABI.  On failure pf_last_error()
 *    returns a thread-local message describing the last error of the calling thread.
 *  - "device pointer" arguments are CUDA global-memory addresses on the sim's device; "host
 *    pointer" arguments are ordinary CPU memory.  The caller owns every buffer it passes.
 *  - stream arguments are cudaStream_t values passed as void* (NULL = legacy default stream).
 *  - every function taking a pf_sim claims that sim for the duration of the call: a second call
 *    on the same sim from another thread while it runs returns PF_EBUSY and does nothing.
 *    pf_destroy, which cannot report this, must not overlap any other call on its sim.
 *  - node order: the (nx+1)(ny+1) vertex grid row-major (x fastest), then, for crossed meshes,
 *    the nx*ny cell-centre grid row-major.  u is interleaved (u_x, u_y) per node.
 *  - doubled grid units: vertex (i, j) sits at (2i, 2j), the centre of cell (i, j) at
 *    (2i+1, 2j+1); pins and damage boxes are given in these integer units.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pf_status {
  PF_OK = 0,
  PF_EINVAL = 1,    /* invalid argument or unsupported configuration */
  PF_ENOMEM = 2,    /* workspace too small */
  PF_ENOTCONV = 3,  /* iteration cap reached; the last iterate is kept and stays valid */
  PF_ENUMERIC = 4,  /* NaN/Inf or breakdown detected in a reduction */
  PF_ETIMEOUT = 5,  /* a bounded device wait gave up */
  PF_ECUDA = 6,     /* a CUDA runtime call failed */
  PF_EBUSY = 7      /* the sim is in use by another call */
} pf_status;

enum { PF_MESH_RIGHT = 0, PF_MESH_CROSSED = 1 };
enum { PF_AT1 = 1, PF_AT2 = 2 };
enum { PF_PLANE_STRAIN = 0, PF_PLANE_STRESS = 1 };
enum { PF_FP64 = 0, PF_MIXED = 1 };
enum { PF_ALGO_AM = 0, PF_ALGO_ORAM = 1, PF_ALGO_ORAM_N = 2 };
enum { PF_EDGE_LEFT = 0, PF_EDGE_RIGHT = 1, PF_EDGE_BOTTOM = 2, PF_EDGE_TOP = 3 };
enum { PF_COMP_UX = 0, PF_COMP_UY = 1, PF_COMP_ALPHA = 2 };

#define PF_MAX_PINS 8
#define PF_MAX_BOXES 8

/* Structured triangulation of [x0, x0+lx] x [y0, y0+ly] with nx x ny cells.
 * kind = PF_MESH_RIGHT: each cell cut by its lower-left -> upper-right diagonal;
 * kind = PF_MESH_CROSSED: each cell cut by both diagonals (extra centre node).
 * Dirichlet data (the set C_ubar and the damage data of D_alpha, Section 1.1):
 *   fixed[edge][comp] != 0 prescribes the component on that edge; the value is t*load for
 *   displacement components (t = load amplitude of the step) and load for the damage.  Two
 *   edges meeting at a corner must agree on a component they both prescribe.
 *   pins: single prescribed nodes (doubled units), same value rule.
 * boxes: nodes with box[k][0] <= X2 <= box[k][1] and box[k][2] <= Y2 <= box[k][3] start with
 *   alpha = alpha_prev = box_value[k] (a pre-existing crack when 1).
 * mode_I != 0: moving-crack boundary data (Section 4.1, eq. surfingloading): the prescribed value
 *   of displacement component c on a fixed edge or pin is load * u_bar_c(x - x_tip(t), y -
 *   mode_I_param[3]) with x_tip(t) = mode_I_param[1] + mode_I_param[2] * t, instead of t * load;
 *   u_bar = K/(2 mu) sqrt(r/(2 pi)) (kappa - cos theta) (cos(theta/2), sin(theta/2)) is the
 *   asymptotic Mode-I displacement with K = mode_I_param[0], (r, theta) polar around the tip
 *   (theta in (-pi, pi]), kappa = (3 - nu)/(1 + nu) in plane stress and 3 - 4 nu in plane
 *   strain, mu and nu from the sim's material.  Node coordinates are x0 + lx X2 / (2 nx),
 *   y0 + ly Y2 / (2 ny). */
typedef struct pf_mesh_desc {
  int32_t kind, nx, ny;
  double x0, y0, lx, ly;
  uint8_t fixed[4][3];
  double load[4][3];
  int32_t n_pins;
  int32_t pin_x2[PF_MAX_PINS], pin_y2[PF_MAX_PINS], pin_comp[PF_MAX_PINS];
  double pin_load[PF_MAX_PINS];
  int32_t n_boxes;
  int32_t box[PF_MAX_BOXES][4];
  double box_value[PF_MAX_BOXES];
  int32_t mode_I;
  double mode_I_param[4];  /* K_I, tip abscissa at t = 0, tip speed, crack-line ordinate */
} pf_mesh_desc;

/* Material (Section 1.1 and Section 4): Young's modulus E, Poisson ratio nu, toughness Gc,
 * internal length ell, residual stiffness k_ell in a(alpha) = (1-alpha)^2 + k_ell, damage model
 * (PF_AT1: w = alpha, PF_AT2: w = alpha^2), plane strain/stress, thermal expansion beta and the
 * penetration length pen = 2 sqrt(kappa t) of T = -dT erfc(x2 / pen) (eq. tempfielderfc; x2
 * measured from the bottom edge y = y0, T evaluated at element centroids). */
typedef struct pf_material {
  double E, nu, Gc, ell, k_ell;
  int32_t model, plane;
  double beta, pen;
} pf_material;

/* One quasi-static load step: displacement amplitude t and thermal shock amplitude dT. */
typedef struct pf_load {
  double t, dT;
} pf_load;

/* Solver options.  Defaults from pf_default_opts().  Tolerances:
 *   am_tol: stop ORAM when max|alpha^k - alpha^{k-1}| <= am_tol (the damage-change criterion
 *           of Section 1.2) and max|u^k - u^{k-1}| <= am_tol * max|u^k| (the same test on the
 *           displacement, so that a step whose damage does not move still solves for u).
 *   u_rtol: u-subproblem FP64 residual <= u_rtol * (largest residual seen in the load step).
 *   inner_rtol: relative tolerance of each inner FP32 CG solve (PF_MIXED).
 *   rs_rtol: damage subproblem ||Phi||_2 <= rs_rtol * max(largest ||Phi||_2 seen in the load
 *           step, size of the terms summed into E_alpha) (Algorithm 4 termination; the term size,
 *           sqrt(n) (8/3) |T| (2 c3 + c2) with c3 = Gc/(c_w ell), c2 = 2 Gc/(c_w ell) for AT2, is
 *           the scale at a load at the AT1 threshold, where the linear term cancels).
 *   am_forcing, am_forcing_max: inexact subproblem solves.  In AM iteration k the two
 *           tolerances above are raised to f_k = min(am_forcing_max, am_forcing * dalpha_{k-1})
 *           (dalpha_0 = infinity), so the subproblems are solved loosely while the damage moves
 *           a lot and to u_rtol / rs_rtol as the iteration converges; the am_tol test is
 *           then accepted only in an iteration whose predecessor already met it (so its
 *           tolerances were at most am_forcing * am_tol).  0 (default): exact solves. 
 *   alpha_cg_rtol: relative tolerance of the reduced Newton solves inside Algorithm 4.
 *   zeta: zero tolerance of the active set (eq. reducedis).
 *   switch_tol: ORAM-N switches to Newton when ||Phi^k|| / ||Phi^0|| <= switch_tol (Alg. 3).
 *   newton_rtol: ORAM-N stops when ||Phi|| <= newton_rtol * ||Phi|| at the start of the step. */
typedef struct pf_solver_opts {
  int32_t algo, precision;
  double omega;
  double am_tol;
  int32_t am_maxit;
  double u_rtol, inner_rtol;
  int32_t cg_maxit;
  double rs_rtol;
  int32_t rs_maxit;
  double alpha_cg_rtol, zeta;
  int32_t mg_levels_max;   /* multigrid levels used (0 = all the mesh allows; 1 = CG with the
                            * l1-Jacobi Chebyshev smoother as preconditioner).  A coarsest level in
                            * use that is not the mesh's coarsest (dense solve) is smoothed with
                            * 8 * mg_degree steps. */
  int32_t mg_degree;       /* Chebyshev smoothing steps per pre/post smoothing (1..16) */
  double switch_tol, newton_rtol;
  int32_t newton_maxit, minres_maxit;
  double minres_rtol;
  int32_t use_graphs;      /* 1 (default): each PCG solve runs as one CUDA graph with a device-side
                            * loop; 0: host-driven iterations */
  int32_t batch_workers;   /* host threads (one stream each) of pf_solve_batch; default 8 */
  double am_forcing, am_forcing_max;
  int32_t mg_tail;         /* 1 (default): in FP32 V-cycles, the coarse levels that fit in one
                            * SM's shared memory run as a single thread block; 0: one grid per
                            * step on every level */
  int32_t mg_coarse_degree; /* Chebyshev steps per smoothing on the coarse levels (0 (default):
                             * mg_degree; at most 16) */
  int32_t omega_rule;      /* damage over-relaxation step (Algorithm 2): 0 (default) the
                            * recursive midpoint rule of Section 2.1 (omega, (1+omega)/2, ... until
                            * the update stays in the box); 1: always omega, then projection onto
                            * the box [alpha_prev, 1] */
  int32_t omega_auto;      /* 1: automated omega (no counterpart in the paper, which leaves it
                            * open in Section 2.2): every 5 iterations of a load step, with rho the
                            * contraction of max|alpha^k - alpha^{k-1}| over them, mu^2 =
                            * (rho + omega - 1)^2 / (rho omega^2) and omega <- 2 / (1 + sqrt(1 -
                            * mu^2)) clamped to [1, omega_max] (the optimum of two-block SOR).
                            * Each load step starts from `omega`.  0 (default): fixed omega. */
  double omega_max;        /* upper bound of the automated omega (default 1.9) */
  int32_t autotune;        /* 1: pf_load_step takes the smoother degrees and FP32 stencil tile
                            * heights that pf_autotune found for this mesh (kind, nx, ny) and
                            * precision, running pf_autotune first if none is cached; they replace
                            * mg_degree, mg_coarse_degree and the two tile heights below.
                            * 0 (default): as given. */
  int32_t tile_rows_fine, tile_rows_coarse;  /* stencil tile height (vertex rows per thread
                            * block of 32 columns) of the FP32 operator kernels on the finest
                            * level and on the coarser levels: 4, 8 or 16 (0 (default): 8).  Only
                            * the speed depends on them. */
} pf_solver_opts;

/* Per-step report (all counts summed over the step).  phi_start / phi_norm: ||Phi||_2 of the
 * full optimality system (eq. kkt: E_u on free dofs, MCP residual of E_alpha on [alpha_prev, 1])
 * after the Dirichlet lift at the start of the step and at its end. */
typedef struct pf_step_report {
  int32_t status, am_iters, rs_iters, newton_iters;
  int64_t cg_iters_u, cg_iters_alpha, krylov_iters_newton, outer_refinements;
  double dalpha_inf, du_rel, phi_norm, phi_start, omega_bar_min;
  double energy[3]; /* elastic, surface, total */
  double seconds;
  int64_t u_solves_reused; /* AM iterations whose u-subproblem had the same alpha and load as the
                              previous one, so its minimizer was reused instead of re-solved */
  int64_t u_notconv;       /* u-subproblem solves that stopped at their iteration cap */
  int64_t newton_steepest; /* ORAM-N Newton iterations whose accepted step came from the
                              steepest-descent fallback of Algorithm 4 */
  int64_t alpha_notconv;   /* damage-subproblem solves (Algorithm 4) that stopped at their
                              iteration cap or with a failed line search; the stopping test of
                              the load step is accepted only after an iteration whose two
                              subproblems both converged */
  double omega_final;      /* relaxation parameter in use at the end of the step */
} pf_step_report;

typedef struct pf_ctx pf_ctx;
typedef struct pf_sim pf_sim;

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* pf_last_error(void);

/* Library version string. */
const char* pf_version(void);

/* Fill *o with defaults (ORAM, omega = 1, FP64, am_tol 1e-6, ...). */
pf_status pf_default_opts(pf_solver_opts* o);

/* Create a context bound to CUDA device `device` (makes it current on this thread).  The
 * context owns a pool of small pinned host buffers (one per live sim, for scalar read-back); no
 * device memory.  Sims and servers may be used from several host threads at once (one thread
 * per sim at a time). */
pf_status pf_ctx_create(int device, pf_ctx** out);
/* Release the context.  Sims and servers created from it stay valid: the context is freed when
 * the last of them is destroyed. */
void pf_ctx_destroy(pf_ctx* ctx);

/* Bytes of device workspace pf_create_mesh needs for this mesh (both precisions included; the
 * precision argument is accepted for forward compatibility and may be either PF_FP64 or
 * PF_MIXED).  Returns 0 if the descriptor is invalid. */
size_t pf_workspace_bytes(const pf_mesh_desc* d, int precision);

/* Build the mesh, its multigrid hierarchy and the initial state (u = 0; alpha = alpha_prev = 0
 * except inside the damage boxes, Section 4 pre-existing cracks) inside the caller-owned device
 * workspace `dev_workspace` (at least pf_workspace_bytes bytes, 256-byte aligned), which must
 * outlive the sim.  PF_ENOMEM if ws_bytes is too small; PF_EINVAL for invalid descriptors. */
pf_status pf_create_mesh(pf_ctx* ctx, const pf_mesh_desc* d, void* dev_workspace,
                         size_t ws_bytes, pf_sim** out);

/* Set the material (Section 4 constants).  PF_EINVAL if nu not in (-1, 0.5), ell <= 0,
 * k_ell < 0, E <= 0 or Gc <= 0.  Must be called before the first load step. */
pf_status pf_set_material(pf_sim* sim, const pf_material* m);

/* Solve one load step (Algorithm 1/2/3 according to o->algo) on `stream`, in place on the
 * resident state: alpha_prev <- alpha, Dirichlet data t*load written into u, then iterate to
 * convergence.  Blocks the host until the step finishes (convergence decisions are read back).
 * On PF_ENOTCONV the last iterate is kept and the state stays valid. rep may be NULL.
 * PF_EBUSY if another thread is using the same sim (different sims may run concurrently from
 * different threads, each on its own stream). */
pf_status pf_load_step(pf_sim* sim, const pf_load* L, const pf_solver_opts* o, void* stream,
                       pf_step_report* rep);

/* Energies (elastic, surface, total) of the resident state for the last load (FP64,
 * deterministic reduction).  Synchronous. */
pf_status pf_energy(pf_sim* sim, void* stream, double out[3]);

/* One load step for each of n sims (loads[i] for sims[i]) with shared options; per-sim reports
 * in reps[i] (may be NULL).  No counterpart in the paper (it solves one problem at a time): the
 * steps run concurrently from o->batch_workers host threads, each on its own non-blocking stream
 * forked from `stream` (work already queued there comes first) and joined back into it, largest
 * meshes first.  The sims must be distinct and belong to ctx (PF_EINVAL otherwise).  Each sim's
 * result is the same as from pf_load_step alone.  Blocks until all steps end; returns the worst
 * status. */
pf_status pf_solve_batch(pf_ctx* ctx, pf_sim* const* sims, const pf_load* loads, int n,
                         const pf_solver_opts* o, void* stream, pf_step_report* reps);

/* ---------------------------------------------------------------------------------------------
 * Serving: a request loop over many simulations (no counterpart in the paper, which runs one
 * simulation at a time).  Jobs arrive over time; each is admitted, in arrival order, once its
 * workspace (pf_workspace_bytes) fits in the free part of the caller-owned device arena, and its
 * u, alpha, alpha_prev stay resident there until its last load step.  n_workers host threads,
 * each with its own non-blocking CUDA stream, run load steps of the admitted jobs round robin
 * (continuous batching: a job admitted while others run shares the device with them).  A job's
 * results do not depend on which other jobs run beside it.
 * ------------------------------------------------------------------------------------------- */
typedef struct pf_server pf_server;

typedef struct pf_job {
  pf_mesh_desc mesh;
  pf_material material;
  const pf_load* loads;     /* n_loads steps; copied at submission */
  int32_t n_loads;
  pf_solver_opts opts;
  double arrival;           /* seconds on the server clock at which the job arrives; < 0: now */
  /* optional caller-owned host outputs, written before the job is reported done; they must stay
   * valid until then: final u (2*n_nodes) and alpha (n_nodes); per-step reports (n_loads); per-
   * step latency in seconds (n_loads): end of the step minus the moment it became ready (the
   * job's arrival for the first step, the end of the previous step otherwise), so queueing for
   * admission and for a worker is included. */
  double* u_out;
  double* alpha_out;
  pf_step_report* reports;
  double* step_latency;
} pf_job;

typedef struct pf_job_info {
  int32_t status;           /* worst status over the job's steps (PF_ENOMEM etc. if not admitted) */
  int32_t steps_done;
  double arrival, admitted, finished;  /* server clock, seconds */
  size_t footprint;         /* arena bytes held while admitted */
} pf_job_info;

typedef struct pf_server_stats {
  int64_t jobs_done, steps_done;
  size_t arena_bytes, arena_peak;
  int32_t max_active, workers;
} pf_server_stats;

/* Start a server on ctx's device.  arena: device memory of arena_bytes, 256-byte aligned,
 * caller-owned, outliving the server.  n_workers in [1, 256].  The server clock starts here. */
pf_status pf_server_create(pf_ctx* ctx, void* arena, size_t arena_bytes, int n_workers,
                           pf_server** out);
/* Seconds since pf_server_create. */
double pf_server_now(const pf_server* s);
/* Queue a job (thread-safe, any time).  PF_ENOMEM if its workspace exceeds the whole arena,
 * PF_EINVAL for an invalid mesh or no load steps.  *id identifies it in pf_server_wait. */
pf_status pf_server_submit(pf_server* s, const pf_job* job, int64_t* id);
/* Block until job `id` is done; info may be NULL. */
pf_status pf_server_wait(pf_server* s, int64_t id, pf_job_info* info);
/* Block until every submitted job is done. */
pf_status pf_server_drain(pf_server* s);
pf_status pf_server_get_stats(pf_server* s, pf_server_stats* out);
/* Wait for all submitted jobs, stop the workers and free the server (not the arena). */
void pf_server_destroy(pf_server* s);

/* Copy the resident state to / from host memory (FP64, node order above, u interleaved).  Any
 * pointer may be NULL to skip that field.  Synchronous.  pf_set_fields also sets the current
 * load used by the operator entry points below. */
pf_status pf_get_fields(pf_sim* sim, double* u, double* alpha, double* alpha_prev);
pf_status pf_set_fields(pf_sim* sim, const double* u, const double* alpha,
                        const double* alpha_prev);

/* Mesh sizes: nodes, elements and multigrid levels. */
pf_status pf_sim_info(const pf_sim* sim, int64_t* n_nodes, int64_t* n_elements, int32_t* levels);

/* Release the sim (not its workspace).  No other call on the sim may run at the same time. */
void pf_destroy(pf_sim* sim);

/* ---------------------------------------------------------------------------------------------
 * Operator entry points (single kernels or single subproblem solves on the resident state).
 * They exist so that each step of the method can be checked on its own.
 * ------------------------------------------------------------------------------------------ */

/* Set the current load (t, dT) and write the Dirichlet data t*load into u (the lift applied at
 * the start of every load step) without solving; alpha_prev is not touched. */
pf_status pf_set_load(pf_sim* sim, const pf_load* L);

/* y = K(alpha) x for the elasticity operator E_uu (Section 1.2, eq. elasticity) with the
 * resident alpha.  x, y: device pointers to 2*n_nodes values, double when precision ==
 * PF_FP64, float when PF_MIXED (then alpha is read from its FP32 copy), aligned to one (u_x, u_y)
 * pair (16 bytes for double, 8 for float; PF_EINVAL otherwise).  masked != 0 applies the
 * operator of the free dofs: x is read as 0 on prescribed dofs and y is 0 there. */
pf_status pf_op_elastic_apply(pf_sim* sim, int precision, int masked, const void* x, void* y,
                              void* stream);

/* r = -(E_u) = f - K(alpha) u on free dofs, 0 on prescribed dofs, for the resident u, alpha and
 * the current load (thermal load vector included).  r: device, 2*n_nodes doubles, 16-byte
 * aligned (PF_EINVAL otherwise).  *norm2 (host) receives ||r||^2.  precision PF_FP64: FP64
 * arithmetic (the plain FP64 path); PF_MIXED: the arithmetic the mixed path uses for its FP64
 * residuals, double-float (pairs of FP32 numbers, ~48 significand bits) on the same FP64 data. */
pf_status pf_op_elastic_residual(pf_sim* sim, int precision, double* r, double* norm2,
                                 void* stream);

/* Damage gradient E_alpha = H alpha + g0 at the resident u, alpha (Section 1.2 and eq.
 * helmholtz), its MCP Fischer-Burmeister residual Phi on the box [lower, upper] (Section 2.4)
 * and the active-set flags (eq. reducedis; 1 = active).  F, Phi: device, n_nodes doubles;
 * active: device, n_nodes bytes (may be NULL).  *phi_norm2 (host) receives ||Phi||^2.
 * precision: as for pf_op_elastic_residual (PF_MIXED: H alpha + g0 in double-float). */
pf_status pf_op_damage_gradient(pf_sim* sim, int precision, double* F, double* Phi,
                                uint8_t* active, double* phi_norm2, void* stream);

/* y = H(q(u)) x, the damage Hessian E_aa at the resident u (precision as above; n_nodes
 * values). */
pf_status pf_op_damage_apply(pf_sim* sim, int precision, const void* x, void* y, void* stream);

/* Off-diagonal block of the Newton Jacobian of the coupled system (Section 3.3, eq. offdiag),
 * B = E_u,alpha at the resident u, alpha and current load, in FP64: transpose == 0 gives
 * y = B x (x: n_nodes damage values, y: 2*n_nodes interleaved displacement values, 0 on
 * prescribed dofs); transpose == 1 gives y = B^T x (x: 2*n_nodes, prescribed dofs ignored; y:
 * n_nodes).  Device pointers, caller-owned.  Synchronous. */
pf_status pf_op_coupling_apply(pf_sim* sim, int transpose, const double* x, double* y,
                               void* stream);

/* Solve the u-subproblem of Algorithm 1 at the resident alpha and current load, in place
 * (u <- minimizer; Section 3.1 solver: PCG + multigrid).  rep may be NULL. */
pf_status pf_op_u_solve(pf_sim* sim, const pf_solver_opts* o, void* stream, pf_step_report* rep);

/* Solve the alpha-subproblem of Algorithm 1 (box-constrained, Algorithm 4 with PCG + multigrid
 * on the inactive set, Section 3.2) at the resident u, in place, with bounds
 * [alpha_prev, 1] and the damage Dirichlet data.  rep may be NULL. */
pf_status pf_op_alpha_solve(pf_sim* sim, const pf_solver_opts* o, void* stream,
                            pf_step_report* rep);

/* ||Phi||_2 of the full optimality system (eq. kkt: E_u on free dofs, MCP residual of
 * E_alpha) at the resident state and current load.  Synchronous. */
pf_status pf_op_full_residual(pf_sim* sim, double* phi_norm, void* stream);

/* Energies (elastic, surface, total) of caller-given fields, like pf_energy, but without any
 * device memory allocation and without a sim.  No counterpart in the paper: it exists for callers
 * that cannot let a library call cudaMalloc/cudaFree -- for example an application whose memory
 * pool already owns all free device memory, or code that must not trigger the implicit device
 * synchronization those calls may perform.
 * d, m, L: host descriptors as for pf_create_mesh / pf_set_material / pf_load_step (the thermal
 * eigenstrain uses L->dT). u (2*n_nodes doubles, interleaved) and alpha (n_nodes doubles):
 * device pointers owned by the caller, node order as above.  out: host, 3 doubles.
 * Scratch: a fixed 328 KB array compiled into the library, held on every device that loads it
 * until the process exits.  Limit: at most 8192 cell rows (ny); larger meshes return PF_EINVAL
 * with a message.  The first call on a device looks up the array's device address and keeps it
 * (a cudaDeviceReset of that device invalidates it: do not use the library on a device after
 * resetting it).  All calls on a device share the array and reuse its previous contents, so
 * calls that overlap on the GPU race; serialize them.  Synchronous: every call waits for its
 * stream, so it cannot be recorded into a CUDA graph by stream capture. */
pf_status pf_energy_noalloc(const pf_mesh_desc* d, const pf_material* m, const pf_load* L,
                            const double* u, const double* alpha, double out[3], void* stream);

/* ---------------------------------------------------------------------------------------------
 * Autotuner (no counterpart in the paper).  Picks, for the sim's mesh and o->precision, the
 * Chebyshev smoothing steps per level (mg_degree on the finest level, mg_coarse_degree below) and
 * the stencil tile height of the FP32 operator kernels (4, 8 or 16 rows of 32 vertices per
 * thread block, one height for the finest level and one for the coarser levels), by timing on
 * `stream` whole preconditioned-CG solves of the elasticity operator at the sim's current damage
 * field (right-hand side K(alpha) v with v the resident displacement on the free dofs, or a fixed
 * pseudo-random field while it is zero; to o->inner_rtol in PF_MIXED, 1e-8 in PF_FP64): the
 * default first, then the other 11 degree pairs of (1-4) x (1-3) at the default tiles, then the
 * 8 other tile pairs at the best degrees (PF_MIXED only).  The fastest configuration is kept in a
 * process-wide cache keyed by (kind, nx, ny, precision) and applied to the sim; the resident
 * fields are not changed.  out may be NULL.  Synchronous.
 * ------------------------------------------------------------------------------------------- */
typedef struct pf_tune_report {
  int32_t mg_degree, mg_coarse_degree, tile_rows_fine, tile_rows_coarse, trials;
  int32_t iters_best, iters_default;
  double ms_best, ms_default;  /* one solve: the chosen and the default configuration */
} pf_tune_report;
pf_status pf_autotune(pf_sim* sim, const pf_solver_opts* o, void* stream, pf_tune_report* out);

/* ---------------------------------------------------------------------------------------------
 * Launch accounting and kernel timing (tracing support; process-wide).  Every kernel the
 * library launches is counted, exactly, from any number of host threads (a kernel inside a
 * CUDA graph counts once per replay).  With timing enabled, each launch of the
 * selected kernel class (-1 = every class) is bracketed by two CUDA events recorded on the
 * launching stream; the measured time and the launch's algorithmic bytes (compulsory reads and
 * writes of the operator on its grid) are accumulated per class.  Timing is meant for single-
 * threaded runs: work of other threads on other streams would overlap the bracketed launches.
 * ------------------------------------------------------------------------------------------ */
pf_status pf_prof_enable(int on, int kernel_class);
pf_status pf_prof_reset(void);
int64_t pf_launch_count(void);
int pf_prof_class_count(void);
/* name: static string valid until the next call on this thread; launches: all launches of the
 * class since the last reset; timed: launches that were timed; ms: summed event time; bytes:
 * summed algorithmic bytes of the timed launches.  PF_EINVAL for an unknown class. */
pf_status pf_prof_get(int kernel_class, const char** name, int64_t* launches, int64_t* timed,
                      double* ms, double* bytes);

#ifdef __cplusplus
}
#endif

#endif /* PF_H */
