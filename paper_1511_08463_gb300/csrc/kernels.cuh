// Host-side launchers of the libpf kernels (definitions in ops_*.cu and kernels_misc.cu).
#pragma once
#include "prof.hpp"
#include "stencil.cuh"

namespace pf {

// ---- stencil operators (ops_elastic.cu, ops_damage.cu) ----------------------------------------
template <class T>
void launch_elastic(cudaStream_t s, const Grid& g, const Mat& m, int coef, int mode, bool eigen,
                    bool dot, const ElasticArgs<T>& a);
template <class T>
void launch_damage(cudaStream_t s, const Grid& g, const Mat& m, int mode, bool dot,
                   const DamageArgs<T>& a);

// ---- pointwise vector kernels (kernels_misc.cu) -----------------------------------------------
template <class T>
void vec_fill(cudaStream_t s, T* y, T v, size_t n);
template <class TO, class TI>
void vec_convert(cudaStream_t s, TO* y, const TI* x, size_t n);
void vec_add_f32_to_f64(cudaStream_t s, double* x, const float* d, size_t n);
template <class T>
void vec_add(cudaStream_t s, T* x, const T* d, size_t n);  // x += d
template <class T>
void vec_mul(cudaStream_t s, T* z, const T* a, const T* b, size_t n);  // z = a .* b
template <class T>
void vec_dot(cudaStream_t s, const T* x, const T* y, size_t n, RedSlot slot);
// CG: a = *rz / *pAp; x += a p; r -= a Ap; out = r.r
template <class T>
void cg_update_xr(cudaStream_t s, T* x, T* r, const T* p, const T* Ap, size_t n,
                  const double* rz, const double* pAp, RedSlot slot);
// CG: p = z + (*rz_new / *rz_old) p   (rz_old == nullptr: p = z)
template <class T>
void cg_update_p(cudaStream_t s, T* p, const T* z, size_t n, const double* rz_new,
                 const double* rz_old);

// end of a graph-resident CG iteration: rz_old <- rz_new, it += 1, keep looping while
// rr > tol2 and it < maxit (sets the while-condition of the graph)
void cg_control(cudaStream_t s, cudaGraphConditionalHandle h, double* rz_new, double* rz_old,
                const double* rr, const double* tol2, double* it, const double* maxit);
// u <- u + omega (xt - u); reductions: max |du|, max |u_new|
void relax_u(cudaStream_t s, double* u, const double* xt, double omega, size_t n2, RedSlot slot);
// max feasible step along alpha + w (at - alpha) in [lo, hi]: out = -min ratio (MAX reduction)
void omega_star(cudaStream_t s, const Grid& g, const double* alpha, const double* at,
                const double* lo, RedSlot slot);
// alpha <- clip(alpha + w (at - alpha)); alpha32 = float(alpha); out = max |dalpha|
void relax_alpha(cudaStream_t s, const Grid& g, double* alpha, const double* at, const double* lo,
                 double w, float* alpha32, RedSlot slot);
// u[fixed dofs] = t * load
struct LiftData {
  double load[4][3];
  double pin_load[PF_MAX_PINS];
  // moving Mode-I crack data (pf_mesh_desc.mode_I): the value is load * u_bar(x - xt0 - v t,
  // y - yl) with u_bar = K/(2 mu) sqrt(r/(2 pi)) (kappa - cos theta) (cos, sin)(theta/2)
  int mode_I;
  double K, xt0, v, yl, mu, kappa;
  double x0, y0, lx, ly;
};
void lift_u(cudaStream_t s, const Grid& g, double* u, double t, const LiftData& ld);
// u <- u on free dofs, masked copy helpers
template <class T>
void mask_fixed(cudaStream_t s, const Grid& g, T* v, int ncomp);  // zero prescribed components
// y_i = a deterministic pseudo-random value in [-1/2, 1/2) from (i, seed) (integer hash)
template <class T>
void vec_hash_fill(cudaStream_t s, T* y, size_t n, unsigned seed);

// ---- element-wise kernels -----------------------------------------------------------------------
template <class T>
void elastic_coef(cudaStream_t s, const Grid& g, const Mat& m, const T* alpha, T* coef);
// q_T = A0 eps_eff : eps_eff (FP64); w64 = q + c2, w32 = float(q + c2)
void damage_q(cudaStream_t s, const Grid& g, const Mat& m, const double* u, const double* eig,
              double* q, double* w64, float* w32, bool df = false);  // df: double-float arithmetic
// energies: out[0] elastic, out[1] surface
void energy(cudaStream_t s, const Grid& g, const Mat& m, const double* u, const double* alpha,
            const double* eig, RedSlot slot);
// coarse element coefficient = mean of its four children
template <class T>
void coarsen_coef(cudaStream_t s, const Grid& gf, const Grid& gc, const T* cf, T* cc);
// inverse l1 diagonal: elastic (2 per node) or damage (1 per node)
template <class T>
void l1_dinv_elastic(cudaStream_t s, const Grid& g, const Mat& m, const T* coef, T* dinv);
template <class T>
void l1_dinv_damage(cudaStream_t s, const Grid& g, const Mat& m, const T* w, T* dinv);

// ---- multigrid transfer -------------------------------------------------------------------------
// bc = P^T rf on the coarse grid (comp_base: 0 elastic (2 comps), 2 damage (1 comp)); coarse
// prescribed components set to 0.
// level: index of the fine level (launch accounting)
template <class T>
void restrict_res(cudaStream_t s, const Grid& gf, const Grid& gc, int ncomp, int comp_base,
                  const T* rf, T* bc, const uint8_t* excl_c, int level);  // excl_c may be null

// ---- coarsest level dense solve -----------------------------------------------------------------
template <class T>
void coarse_assemble(cudaStream_t s, const Grid& g, const Mat& m, int physics, const T* coef,
                     T* A, T* diag0, const uint8_t* excl);  // excl (may be null): identity rows
// coarse active-set mask from the fine one (coincident nodes)
void mask_restrict(cudaStream_t s, const Grid& gf, const Grid& gc, const uint8_t* ef, uint8_t* ec);
template <class T>
void coarse_factor(cudaStream_t s, int n, T* A, const T* diag0);
template <class T>
void coarse_invert(cudaStream_t s, int n, const T* L, T* Ainv);  // explicit inverse from L
// ---- the coarse end of a V-cycle in one thread block (tail.cu) ---------------------------------
constexpr int MAX_TAIL = 8;          // levels the single-block kernel can hold
constexpr int TAIL_THREADS = 1024;
constexpr int TAIL_MAX_NODES = 1200;  // largest level a tail starts on, unless it holds them all
struct TailLevel {
  Grid g;
  Consts<float> cs;
  const float* coef;     // elastic abar_T or damage weight w_T per element (device)
  const float* dinv;     // inverse l1 diagonal (device)
  const uint8_t* excl;   // damage: excluded nodes (device); elastic: null
  int ox, oxn, ob, od, odi, oc, oe;  // shared-memory offsets, in floats (oe: flag bytes)
};
constexpr int MAX_CHEB = 16;  // Chebyshev steps per smoothing (pf_solver_opts degrees)
struct TailArgs {
  int nl, deg;                       // levels in the tail (ending in the dense solve); steps
  int deg0;                          // smoothing steps on the tail's first level
  int first_level;                   // hierarchy index of that level (launch accounting)
  int orec;                          // shared-memory offset of the element records, in floats
  int dense_slices;                  // column ranges of the dense solve (its partial sums use
                                     // the record area: dense_slices * n floats)
  const float* Ainv;                 // coarsest inverse (dense)
  const float* b_in;                 // right-hand side on the tail's first level (device)
  const float* rf;                   // if set, b_in is not read: the right-hand side is the
  Grid gf;                           // restriction of this residual on the finer grid gf
  float* x_out;                      // V-cycle result on that level (device)
  float cheb_cd[MAX_CHEB], cheb_cr[MAX_CHEB];  // coefficients of Chebyshev step k, as the
                                               // grid-wide smoother rounds them
  TailLevel L[MAX_TAIL];
};
size_t tail_smem_limit();  // dynamic shared memory available to the tail kernel (0: none)
void tail_vcycle(cudaStream_t s, int ncomp, const TailArgs& a, size_t smem);

// Both steps: in shared memory when the packed factor fits, else the two kernels above.
// A (n x n, row-major, overwritten), diag0 (pivot floor), Ainv (n x n).
constexpr int COARSE_WARPS = 8;  // columns of the inverse per block
template <class T>
void coarse_factor_invert(cudaStream_t s, int n, T* A, const T* diag0, T* Ainv);
template <class T>
void coarse_solve(cudaStream_t s, int n, const T* Ainv, const T* b, T* x);  // x = Ainv b

// ---- misc for the damage solve ------------------------------------------------------------------
// steepest-descent fallback of Algorithm 4: v = -pb qb Phi, dg = (pa - pb qa) Phi
void merit_parts(cudaStream_t s, const Grid& g, const double* x, const double* F,
                 const double* lo, double* v, double* dg);
// d_i = bound_i - x_i on active components (act 1: lower, 2: upper); other entries unchanged
void snap_active(cudaStream_t s, const Grid& g, const uint8_t* act, const double* x, const double* lo,
                 double* d);
// d = -(dg + Hv)
void merit_direction(cudaStream_t s, size_t n, const double* dg, const double* Hv, double* d);

// ---- Newton (ORAM-N) helpers (ops_newton.cu) ---------------------------------------------------
template <class T>
void launch_coupling(cudaStream_t s, const Grid& g, const Mat& m, bool transpose,
                     const CouplingArgs<T>& a);
template <class T>
void vec_lincomb(cudaStream_t s, T* z, T a, const T* x, T b, const T* y, T c, size_t n);
void newton_trial(cudaStream_t s, const Grid& g, double* u, const double* u0, const double* du,
                  double* alpha, const double* a0, const double* da, const double* lo, float* a32,
                  double mu);

}  // namespace pf
