// Pointwise, element-wise, transfer and coarse-solve kernels of libpf.
#include <math.h>

#include "kernels.cuh"
#include "mg_core.cuh"

namespace pf {

static inline unsigned nblocks(size_t n, int bs = RED_THREADS) {
  size_t b = (n + bs - 1) / bs;
  return (unsigned)(b < 1 ? 1 : b);
}
// Reduction kernels use a grid-stride loop over at most RED_GRID_CAP blocks (4 per SM): every
// block adds one ticket atomic and one partial that the last block sums, so a grid sized to the
// vector would spend more time in that serial tail than in streaming the vector.
constexpr size_t RED_GRID_CAP = 4 * 152;
static_assert(RED_GRID_CAP <= MAX_RED_BLOCKS, "partial buffers hold MAX_RED_BLOCKS blocks");
static inline unsigned rblocks(size_t n) {
  size_t b = (n + RED_THREADS - 1) / RED_THREADS;
  if (b > RED_GRID_CAP) b = RED_GRID_CAP;
  return (unsigned)(b < 1 ? 1 : b);
}
// float vectors are streamed as float4 when both operands are 16-byte aligned
template <class T>
__device__ __forceinline__ bool vec4_ok(const void* a, const void* b) {
  return sizeof(T) == 4 && ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 15) == 0;
}

// ---------------------------------------------------------------------------------------------
// pointwise vectors
// ---------------------------------------------------------------------------------------------
template <class T>
__global__ void k_fill(T* y, T v, size_t n) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = v;
}
template <class T>
void vec_fill(cudaStream_t s, T* y, T v, size_t n) {
  PF_LAUNCH(kclass(KC_VECTOR, sizeof(T) == 8, 0), double(n) * sizeof(T), s, pdl_launch(k_fill<T>, nblocks(n), RED_THREADS, 0, s, y, v, n));
}
template void vec_fill<double>(cudaStream_t, double*, double, size_t);
template void vec_fill<float>(cudaStream_t, float*, float, size_t);

template <class TO, class TI>
__global__ void k_convert(TO* y, const TI* x, size_t n) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) y[i] = TO(x[i]);
}
template <class TO, class TI>
void vec_convert(cudaStream_t s, TO* y, const TI* x, size_t n) {
  PF_LAUNCH(kclass(KC_VECTOR, false, 0), double(n) * (sizeof(TO) + sizeof(TI)), s, pdl_launch(k_convert<TO, TI>, nblocks(n), RED_THREADS, 0, s, y, x, n));
}
template void vec_convert<float, double>(cudaStream_t, float*, const double*, size_t);
template void vec_convert<double, float>(cudaStream_t, double*, const float*, size_t);
template void vec_convert<double, double>(cudaStream_t, double*, const double*, size_t);

__global__ void k_add_f32_to_f64(double* x, const float* d, size_t n) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += (double)d[i];
}
void vec_add_f32_to_f64(cudaStream_t s, double* x, const float* d, size_t n) {
  PF_LAUNCH(kclass(KC_VECTOR, true, 0), double(n) * 20.0, s, pdl_launch(k_add_f32_to_f64, nblocks(n), RED_THREADS, 0, s, x, d, n));
}

template <class T>
__global__ void k_add(T* x, const T* d, size_t n) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
}
template <class T>
void vec_add(cudaStream_t s, T* x, const T* d, size_t n) {
  PF_LAUNCH(kclass(KC_VECTOR, sizeof(T) == 8, 0), 3.0 * n * sizeof(T), s, pdl_launch(k_add<T>, nblocks(n), RED_THREADS, 0, s, x, d, n));
}
template void vec_add<double>(cudaStream_t, double*, const double*, size_t);
template void vec_add<float>(cudaStream_t, float*, const float*, size_t);

template <class T>
__global__ void k_mul(T* z, const T* a, const T* b, size_t n) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) z[i] = a[i] * b[i];
}
template <class T>
void vec_mul(cudaStream_t s, T* z, const T* a, const T* b, size_t n) {
  PF_LAUNCH(kclass(KC_VECTOR, sizeof(T) == 8, 0), 3.0 * n * sizeof(T), s, pdl_launch(k_mul<T>, nblocks(n), RED_THREADS, 0, s, z, a, b, n));
}
template void vec_mul<double>(cudaStream_t, double*, const double*, const double*, size_t);
template void vec_mul<float>(cudaStream_t, float*, const float*, const float*, size_t);

template <class T>
__global__ void k_dot(const T* x, const T* y, size_t n, RedSlot slot) {
  pdl_enter();
  T v[1] = {T(0)};
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  size_t done = 0;
  if constexpr (sizeof(T) == 4) {
    if (vec4_ok<T>(x, y)) {
      const float4* x4 = reinterpret_cast<const float4*>(x);
      const float4* y4 = reinterpret_cast<const float4*>(y);
      for (size_t i = t0; i < n / 4; i += st) {
        const float4 a = x4[i], b = y4[i];
        v[0] += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
      }
      done = n / 4 * 4;
    }
  }
  for (size_t i = done + t0; i < n; i += st) v[0] += x[i] * y[i];
  block_reduce_finalize<1, false, T>(v, slot);
}
template <class T>
void vec_dot(cudaStream_t s, const T* x, const T* y, size_t n, RedSlot slot) {
  PF_LAUNCH(kclass(KC_REDUCE, sizeof(T) == 8, 0), 2.0 * n * sizeof(T), s, pdl_launch(k_dot<T>, rblocks(n), RED_THREADS, 0, s, x, y, n, slot));
}
template void vec_dot<double>(cudaStream_t, const double*, const double*, size_t, RedSlot);
template void vec_dot<float>(cudaStream_t, const float*, const float*, size_t, RedSlot);

template <class T>
__global__ void k_cg_xr(T* x, T* r, const T* p, const T* Ap, size_t n, const double* rz,
                        const double* pAp, RedSlot slot) {
  pdl_enter();
  __shared__ T sa;  // step length computed once per block
  if (threadIdx.x == 0) sa = T(*rz / *pAp);
  __syncthreads();
  const T at = sa;
  T v[1] = {T(0)};
  const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, st = (size_t)gridDim.x * blockDim.x;
  size_t done = 0;
  if constexpr (sizeof(T) == 4) {
    if (vec4_ok<T>(x, r) && vec4_ok<T>(p, Ap)) {
      float4* x4 = reinterpret_cast<float4*>(x);
      float4* r4 = reinterpret_cast<float4*>(r);
      const float4* p4 = reinterpret_cast<const float4*>(p);
      const float4* a4 = reinterpret_cast<const float4*>(Ap);
      for (size_t i = t0; i < n / 4; i += st) {
        float4 xv = x4[i], rv = r4[i];
        const float4 pv = p4[i], av = a4[i];
        xv.x += at * pv.x; xv.y += at * pv.y; xv.z += at * pv.z; xv.w += at * pv.w;
        rv.x -= at * av.x; rv.y -= at * av.y; rv.z -= at * av.z; rv.w -= at * av.w;
        x4[i] = xv;
        r4[i] = rv;
        v[0] += rv.x * rv.x + rv.y * rv.y + rv.z * rv.z + rv.w * rv.w;
      }
      done = n / 4 * 4;
    }
  }
  for (size_t i = done + t0; i < n; i += st) {
    x[i] += at * p[i];
    T ri = r[i] - at * Ap[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  block_reduce_finalize<1, false, T>(v, slot);
}
template <class T>
void cg_update_xr(cudaStream_t s, T* x, T* r, const T* p, const T* Ap, size_t n, const double* rz,
                  const double* pAp, RedSlot slot) {
  PF_LAUNCH(kclass(KC_REDUCE, sizeof(T) == 8, 0), 6.0 * n * sizeof(T), s, pdl_launch(k_cg_xr<T>, rblocks(n), RED_THREADS, 0, s, x, r, p, Ap, n, rz, pAp, slot));
}
template void cg_update_xr<double>(cudaStream_t, double*, double*, const double*, const double*,
                                   size_t, const double*, const double*, RedSlot);
template void cg_update_xr<float>(cudaStream_t, float*, float*, const float*, const float*, size_t,
                                  const double*, const double*, RedSlot);

template <class T>
__global__ void k_cg_p(T* p, const T* z, size_t n, const double* rz_new, const double* rz_old) {
  pdl_enter();
  __shared__ T sb;  // conjugation coefficient computed once per block
  // beta = 0 (first iteration: *rz_old == 0, or no old value given) means p = z, and p is not
  // read (it may hold stale values)
  if (threadIdx.x == 0) sb = (rz_old && *rz_old != 0.0) ? T(*rz_new / *rz_old) : T(0);
  __syncthreads();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  p[i] = sb != T(0) ? z[i] + sb * p[i] : z[i];
}
template <class T>
void cg_update_p(cudaStream_t s, T* p, const T* z, size_t n, const double* rz_new,
                 const double* rz_old) {
  PF_LAUNCH(kclass(KC_VECTOR, sizeof(T) == 8, 0), 3.0 * n * sizeof(T), s, pdl_launch(k_cg_p<T>, nblocks(n), RED_THREADS, 0, s, p, z, n, rz_new, rz_old));
}
template void cg_update_p<double>(cudaStream_t, double*, const double*, size_t, const double*,
                                  const double*);
template void cg_update_p<float>(cudaStream_t, float*, const float*, size_t, const double*,
                                 const double*);

// End of one graph-resident CG iteration: rz_old <- rz_new, count the iteration and decide on
// the device whether the while-loop of the graph runs again.
__global__ void k_cg_control(cudaGraphConditionalHandle h, double* rz_new, double* rz_old,
                             const double* rr, const double* tol2, double* it, const double* maxit) {
  pdl_enter();
  *rz_old = *rz_new;
  double k = *it + 1.0;
  *it = k;
  double r = *rr;
  bool go = (r > *tol2) && (k < *maxit) && (r == r);
  cudaGraphSetConditional(h, go ? 1u : 0u);
}
void cg_control(cudaStream_t s, cudaGraphConditionalHandle h, double* rz_new, double* rz_old,
                const double* rr, const double* tol2, double* it, const double* maxit) {
  PF_LAUNCH(kclass(KC_REDUCE, false, false), 0.0, s,
            pdl_launch(k_cg_control, 1, 1, 0, s, h, rz_new, rz_old, rr, tol2, it, maxit));
}

// over-relaxation of u (Algorithm 2): prescribed dofs have xt == u, so they do not move
__global__ void k_relax_u(double* u, const double* xt, double omega, size_t n2, RedSlot slot) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n2;
       i += (size_t)gridDim.x * blockDim.x) {
    double uo = u[i];
    double un = uo + omega * (xt[i] - uo);
    u[i] = un;
    v[0] = fmax(v[0], fabs(un - uo));
    v[1] = fmax(v[1], fabs(un));
  }
  block_reduce_finalize<2, true>(v, slot);
}
void relax_u(cudaStream_t s, double* u, const double* xt, double omega, size_t n2, RedSlot slot) {
  PF_LAUNCH(kclass(KC_REDUCE, false, false), 0.0, s, pdl_launch(k_relax_u, rblocks(n2), RED_THREADS, 0, s, u, xt, omega, n2, slot));
}

__device__ __forceinline__ double upper_of(const Grid& g, int node, double lo) {
  int X2, Y2;
  node_coords(g, node, X2, Y2);
  return is_fixed(g, X2, Y2, 2) ? lo : 1.0;
}

// largest w with lo <= alpha + w (at - alpha) <= hi at every node: out[0] = -w*
__global__ void k_omega_star(Grid g, const double* alpha, const double* at, const double* lo,
                             RedSlot slot) {
  pdl_enter();
  double v[1] = {-INFINITY};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    double a = alpha[i], d = at[i] - a;
    double l = lo[i], h = upper_of(g, i, l);
    double r = INFINITY;
    if (d > 0.0) r = (h - a) / d;
    else if (d < 0.0) r = (l - a) / d;
    v[0] = fmax(v[0], -r);
  }
  block_reduce_finalize<1, true>(v, slot);
}
void omega_star(cudaStream_t s, const Grid& g, const double* alpha, const double* at,
                const double* lo, RedSlot slot) {
  PF_LAUNCH(kclass(KC_REDUCE, false, false), 0.0, s, pdl_launch(k_omega_star, rblocks(g.n), RED_THREADS, 0, s, g, alpha, at, lo, slot));
}

__global__ void k_relax_alpha(Grid g, double* alpha, const double* at, const double* lo, double w,
                              float* alpha32, RedSlot slot) {
  pdl_enter();
  double v[1] = {0.0};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x) {
    double a = alpha[i];
    double l = lo[i], h = upper_of(g, i, l);
    double an = fmin(fmax(a + w * (at[i] - a), l), h);
    alpha[i] = an;
    if (alpha32) alpha32[i] = (float)an;
    v[0] = fmax(v[0], fabs(an - a));
  }
  block_reduce_finalize<1, true>(v, slot);
}
void relax_alpha(cudaStream_t s, const Grid& g, double* alpha, const double* at, const double* lo,
                 double w, float* alpha32, RedSlot slot) {
  PF_LAUNCH(kclass(KC_REDUCE, false, false), 0.0, s, pdl_launch(k_relax_alpha, rblocks(g.n), RED_THREADS, 0, s, g, alpha, at, lo, w, alpha32, slot));
}

// Value of prescribed displacement component c at doubled coordinates (X2, Y2): t * g, or
// g * u_bar_c for the moving Mode-I crack of Section 4.1 (eq. surfingloading).
__device__ double lift_value(const Grid& g, const LiftData& ld, int X2, int Y2, int c, double t,
                             double gload) {
  if (!ld.mode_I) return t * gload;
  const double x = ld.x0 + ld.lx * (double)X2 / (2.0 * g.nx);
  const double y = ld.y0 + ld.ly * (double)Y2 / (2.0 * g.ny);
  const double dx = x - (ld.xt0 + ld.v * t), dy = y - ld.yl;
  const double r = hypot(dx, dy), th = atan2(dy, dx);
  const double amp = ld.K / (2.0 * ld.mu) * sqrt(r / (2.0 * M_PI)) * (ld.kappa - cos(th));
  return gload * (c == 0 ? amp * cos(0.5 * th) : amp * sin(0.5 * th));
}

__global__ void k_lift(Grid g, double* u, double t, LiftData ld) {
  pdl_enter();
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nv) return;  // only vertices lie on edges; pins checked below for all nodes
  int X2, Y2;
  node_coords(g, node, X2, Y2);
  for (int c = 0; c < 2; ++c) {
    if (X2 == 0 && g.fixed[0][c]) u[2 * node + c] = lift_value(g, ld, X2, Y2, c, t, ld.load[0][c]);
    if (X2 == 2 * g.nx && g.fixed[1][c]) u[2 * node + c] = lift_value(g, ld, X2, Y2, c, t, ld.load[1][c]);
    if (Y2 == 0 && g.fixed[2][c]) u[2 * node + c] = lift_value(g, ld, X2, Y2, c, t, ld.load[2][c]);
    if (Y2 == 2 * g.ny && g.fixed[3][c]) u[2 * node + c] = lift_value(g, ld, X2, Y2, c, t, ld.load[3][c]);
  }
}
__global__ void k_lift_pins(Grid g, double* u, double t, LiftData ld) {
  pdl_enter();
  for (int k = 0; k < g.npins; ++k) {
    if (g.pin_comp[k] > 1) continue;
    int X2 = g.pin_x2[k], Y2 = g.pin_y2[k], node;
    if ((X2 & 1) == 0) node = (Y2 / 2) * (g.nx + 1) + X2 / 2;
    else node = g.nv + (Y2 / 2) * g.nx + X2 / 2;
    u[2 * node + g.pin_comp[k]] = lift_value(g, ld, X2, Y2, g.pin_comp[k], t, ld.pin_load[k]);
  }
}
void lift_u(cudaStream_t s, const Grid& g, double* u, double t, const LiftData& ld) {
  PF_LAUNCH(kclass(KC_VECTOR, false, false), 0.0, s, pdl_launch(k_lift, nblocks(g.nv), RED_THREADS, 0, s, g, u, t, ld));
  if (g.npins > 0) PF_LAUNCH(kclass(KC_VECTOR, false, false), 0.0, s, pdl_launch(k_lift_pins, 1, 1, 0, s, g, u, t, ld));
}

template <class T>
__global__ void k_mask_fixed(Grid g, T* v, int ncomp) {
  pdl_enter();
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n) return;
  int X2, Y2;
  node_coords(g, node, X2, Y2);
  if (ncomp == 2) {
    if (is_fixed(g, X2, Y2, 0)) v[2 * node] = T(0);
    if (is_fixed(g, X2, Y2, 1)) v[2 * node + 1] = T(0);
  } else {
    if (is_fixed(g, X2, Y2, 2)) v[node] = T(0);
  }
}
template <class T>
void mask_fixed(cudaStream_t s, const Grid& g, T* v, int ncomp) {
  PF_LAUNCH(kclass(KC_VECTOR, false, false), 0.0, s, pdl_launch(k_mask_fixed<T>, nblocks(g.n), RED_THREADS, 0, s, g, v, ncomp));
}
template void mask_fixed<double>(cudaStream_t, const Grid&, double*, int);
template void mask_fixed<float>(cudaStream_t, const Grid&, float*, int);

// integer hash (a xorshift-multiply mix) of the index and a seed, scaled to [-1/2, 1/2)
template <class T>
__global__ void k_hash_fill(T* y, size_t n, unsigned seed) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  unsigned h = (unsigned)i * 0x9E3779B1u ^ seed;
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  y[i] = T(double(h) * (1.0 / 4294967296.0) - 0.5);
}
template <class T>
void vec_hash_fill(cudaStream_t s, T* y, size_t n, unsigned seed) {
  PF_LAUNCH(kclass(KC_VECTOR, sizeof(T) == 8, 0), double(n) * sizeof(T), s,
            pdl_launch(k_hash_fill<T>, nblocks(n), RED_THREADS, 0, s, y, n, seed));
}
template void vec_hash_fill<double>(cudaStream_t, double*, size_t, unsigned);
template void vec_hash_fill<float>(cudaStream_t, float*, size_t, unsigned);

// ---------------------------------------------------------------------------------------------
// element-wise kernels: one thread per cell
// ---------------------------------------------------------------------------------------------

template <class T>
__global__ void k_elastic_coef(Grid g, Mat m, const T* alpha, T* coef) {
  pdl_enter();
  int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= g.ncell) return;
  int cj = cell / g.nx, ci = cell - cj * g.nx;
  int NE = elems_per_cell(g.kind);
  for (int t = 0; t < NE; ++t) {
    int n0, n1, n2;
    cell_nodes(g, ci, cj, t, n0, n1, n2);
    coef[cell * NE + t] = abar3<T>(alpha[n0], alpha[n1], alpha[n2], T(m.k_ell));
  }
}
template <class T>
void elastic_coef(cudaStream_t s, const Grid& g, const Mat& m, const T* alpha, T* coef) {
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s, pdl_launch(k_elastic_coef<T>, nblocks(g.ncell), RED_THREADS, 0, s, g, m, alpha, coef));
}
template void elastic_coef<double>(cudaStream_t, const Grid&, const Mat&, const double*, double*);
template void elastic_coef<float>(cudaStream_t, const Grid&, const Mat&, const float*, float*);

__device__ __forceinline__ void strain_of(const Grid& g, int t, const double* u, int n0, int n1,
                                          int n2, double& exx, double& eyy, double& gxy) {
  int nn[3] = {n0, n1, n2};
  double sx = 0, sy = 0, s1 = 0, s2 = 0;
  for (int k = 0; k < 3; ++k) {
    double ux = u[2 * nn[k]], uy = u[2 * nn[k] + 1];
    int cx = gxr(g.kind, t, k), cy = gyr(g.kind, t, k);
    sx += cx * ux;
    sy += cy * uy;
    s1 += cy * ux;
    s2 += cx * uy;
  }
  exx = g.ihx * sx;
  eyy = g.ihy * sy;
  gxy = g.ihy * s1 + g.ihx * s2;
}

__global__ void k_damage_q(Grid g, Mat m, const double* u, const double* eig, double* q,
                           double* w64, float* w32) {
  pdl_enter();
  int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= g.ncell) return;
  int cj = cell / g.nx, ci = cell - cj * g.nx;
  int NE = elems_per_cell(g.kind);
  for (int t = 0; t < NE; ++t) {
    int n0, n1, n2;
    cell_nodes(g, ci, cj, t, n0, n1, n2);
    double exx, eyy, gxy;
    strain_of(g, t, u, n0, n1, n2, exx, eyy, gxy);
    if (eig) {
      double e0 = eig[cj * NE + t];
      exx -= e0;
      eyy -= e0;
    }
    double qq = m.lam2mu * (exx * exx + eyy * eyy) + 2.0 * m.lam * exx * eyy + m.mu * gxy * gxy;
    q[cell * NE + t] = qq;
    if (w64) w64[cell * NE + t] = qq + m.c2;
    if (w32) w32[cell * NE + t] = (float)(qq + m.c2);
  }
}
// The same energy densities in double-float arithmetic on the FP64 data (the mixed path): strains
// from the gradient tables (exact additions for their +-1 weights), then q = (lambda + 2 mu)
// (exx^2 + eyy^2) + 2 lambda exx eyy + mu gxy^2, written as FP64.
template <int KIND, int t>
__device__ __forceinline__ void q_elem_df(const Consts<dfloat>& cs, dfloat lam2, dfloat c2,
                                          const dfloat (&ux)[3], const dfloat (&uy)[3], dfloat e0,
                                          bool eigen, double* q, double* w64, float* w32, int e) {
  constexpr int a0 = gx(KIND, t, 0), a1 = gx(KIND, t, 1), a2 = gx(KIND, t, 2);
  constexpr int b0 = gy(KIND, t, 0), b1 = gy(KIND, t, 1), b2 = gy(KIND, t, 2);
  dfloat exx = cs.ihx * gsum<a0, a1, a2>(ux[0], ux[1], ux[2]);
  dfloat eyy = cs.ihy * gsum<b0, b1, b2>(uy[0], uy[1], uy[2]);
  const dfloat gxy = cs.ihy * gsum<b0, b1, b2>(ux[0], ux[1], ux[2]) +
                     cs.ihx * gsum<a0, a1, a2>(uy[0], uy[1], uy[2]);
  if (eigen) {
    exx -= e0;
    eyy -= e0;
  }
  const dfloat qq = cs.lam2mu * (exx * exx + eyy * eyy) + lam2 * (exx * eyy) + cs.mu * (gxy * gxy);
  q[e] = double(qq);
  if (w64 || w32) {
    const double w = double(qq + c2);
    if (w64) w64[e] = w;
    if (w32) w32[e] = (float)w;
  }
}
template <int KIND>
__global__ void k_damage_q_df(Grid g, Consts<dfloat> cs, dfloat lam2, dfloat c2, const double* u,
                              const double* eig, double* q, double* w64, float* w32) {
  pdl_enter();
  const int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= g.ncell) return;
  constexpr int NE = elems_per_cell(KIND);
  const int cj = cell / g.nx, ci = cell - cj * g.nx;
  const int v00 = cj * (g.nx + 1) + ci, v10 = v00 + 1, v01 = v00 + g.nx + 1, v11 = v01 + 1;
  auto ld = [&](int node, dfloat& x, dfloat& y) {
    const double2 v = *reinterpret_cast<const double2*>(u + 2 * (size_t)node);
    x = dfloat(v.x);
    y = dfloat(v.y);
  };
  dfloat x00, y00, x10, y10, x01, y01, x11, y11;
  ld(v00, x00, y00);
  ld(v10, x10, y10);
  ld(v01, x01, y01);
  ld(v11, x11, y11);
  const int e = cell * NE;
  auto e0 = [&](int t) { return eig ? dfloat(eig[cj * NE + t]) : dfloat(0); };
  const bool eg = eig != nullptr;
  if constexpr (KIND == CROSSED) {
    dfloat xc, yc;
    ld(g.nv + cell, xc, yc);
    q_elem_df<KIND, 0>(cs, lam2, c2, {x00, x10, xc}, {y00, y10, yc}, e0(0), eg, q, w64, w32, e);
    q_elem_df<KIND, 1>(cs, lam2, c2, {x10, x11, xc}, {y10, y11, yc}, e0(1), eg, q, w64, w32, e + 1);
    q_elem_df<KIND, 2>(cs, lam2, c2, {x11, x01, xc}, {y11, y01, yc}, e0(2), eg, q, w64, w32, e + 2);
    q_elem_df<KIND, 3>(cs, lam2, c2, {x01, x00, xc}, {y01, y00, yc}, e0(3), eg, q, w64, w32, e + 3);
  } else {
    q_elem_df<KIND, 0>(cs, lam2, c2, {x00, x10, x11}, {y00, y10, y11}, e0(0), eg, q, w64, w32, e);
    q_elem_df<KIND, 1>(cs, lam2, c2, {x00, x11, x01}, {y00, y11, y01}, e0(1), eg, q, w64, w32, e + 1);
  }
}

void damage_q(cudaStream_t s, const Grid& g, const Mat& m, const double* u, const double* eig,
              double* q, double* w64, float* w32, bool df) {
  if (df) {
    const Consts<dfloat> cs = make_consts<dfloat>(g, m);
    const dfloat lam2(2.0 * m.lam), c2(m.c2);
    if (g.kind == CROSSED)
      PF_LAUNCH(kclass(KC_DM_Q_DF, true, 0), 0.0, s, pdl_launch(k_damage_q_df<CROSSED>, nblocks(g.ncell), RED_THREADS, 0, s, g, cs, lam2, c2, u, eig, q, w64, w32));
    else
      PF_LAUNCH(kclass(KC_DM_Q_DF, true, 0), 0.0, s, pdl_launch(k_damage_q_df<RIGHT>, nblocks(g.ncell), RED_THREADS, 0, s, g, cs, lam2, c2, u, eig, q, w64, w32));
    return;
  }
  PF_LAUNCH(kclass(KC_DM_Q, true, 0), 0.0, s, pdl_launch(k_damage_q, nblocks(g.ncell), RED_THREADS, 0, s, g, m, u, eig, q, w64, w32));
}

__global__ void k_energy(Grid g, Mat m, const double* u, const double* alpha, const double* eig,
                         RedSlot slot) {
  pdl_enter();
  double v[2] = {0.0, 0.0};
  int NE = elems_per_cell(g.kind);
  for (int cell = blockIdx.x * blockDim.x + threadIdx.x; cell < g.ncell;
       cell += gridDim.x * blockDim.x) {
    int cj = cell / g.nx, ci = cell - cj * g.nx;
    for (int t = 0; t < NE; ++t) {
      int n0, n1, n2;
      cell_nodes(g, ci, cj, t, n0, n1, n2);
      double exx, eyy, gxy;
      strain_of(g, t, u, n0, n1, n2, exx, eyy, gxy);
      if (eig) {
        double e0 = eig[cj * NE + t];
        exx -= e0;
        eyy -= e0;
      }
      double qq = m.lam2mu * (exx * exx + eyy * eyy) + 2.0 * m.lam * exx * eyy + m.mu * gxy * gxy;
      double a0 = alpha[n0], a1 = alpha[n1], a2 = alpha[n2];
      double ab = abar3<double>(a0, a1, a2, m.k_ell);
      v[0] += 0.5 * ab * qq * g.area;
      double wbar;
      if (m.model == PF_AT1) wbar = (a0 + a1 + a2) * (1.0 / 3.0);
      else wbar = (a0 * a0 + a1 * a1 + a2 * a2 + a0 * a1 + a1 * a2 + a2 * a0) * (1.0 / 6.0);
      double gax = g.ihx * (gxr(g.kind, t, 0) * a0 + gxr(g.kind, t, 1) * a1 + gxr(g.kind, t, 2) * a2);
      double gay = g.ihy * (gyr(g.kind, t, 0) * a0 + gyr(g.kind, t, 1) * a1 + gyr(g.kind, t, 2) * a2);
      v[1] += m.gc_cw * (wbar / m.ell + m.ell * (gax * gax + gay * gay)) * g.area;
    }
  }
  block_reduce_finalize<2, false>(v, slot);
}
void energy(cudaStream_t s, const Grid& g, const Mat& m, const double* u, const double* alpha,
            const double* eig, RedSlot slot) {
  PF_LAUNCH(kclass(KC_REDUCE, false, false), 0.0, s, pdl_launch(k_energy, rblocks(g.ncell), RED_THREADS, 0, s, g, m, u, alpha, eig, slot));
}

// children of coarse element t of coarse cell (I, J): fine cells and fine element types
//  RIGHT   t0 (lower): (2I,2J).0, (2I+1,2J).0, (2I+1,2J).1, (2I+1,2J+1).0
//          t1 (upper): (2I,2J).1, (2I,2J+1).0, (2I,2J+1).1, (2I+1,2J+1).1
//  CROSSED t0 (bottom): BL.0, BL.1, BR.0, BR.3     t1 (right): BR.1, BR.2, TR.1, TR.0
//          t2 (top):    TR.2, TR.3, TL.2, TL.1     t3 (left):  TL.3, TL.0, BL.3, BL.2
template <class T>
__global__ void k_coarsen(Grid gf, Grid gc, const T* cf, T* cc) {
  pdl_enter();
  int cell = blockIdx.x * blockDim.x + threadIdx.x;
  if (cell >= gc.ncell) return;
  int J = cell / gc.nx, I = cell - J * gc.nx;
  int NE = elems_per_cell(gc.kind);
  auto F = [&](int di, int dj, int t) -> T {
    return cf[((2 * J + dj) * gf.nx + (2 * I + di)) * NE + t];
  };
  if (gc.kind == RIGHT) {
    cc[cell * 2 + 0] = (F(0, 0, 0) + F(1, 0, 0) + F(1, 0, 1) + F(1, 1, 0)) * T(0.25);
    cc[cell * 2 + 1] = (F(0, 0, 1) + F(0, 1, 0) + F(0, 1, 1) + F(1, 1, 1)) * T(0.25);
  } else {
    cc[cell * 4 + 0] = (F(0, 0, 0) + F(0, 0, 1) + F(1, 0, 0) + F(1, 0, 3)) * T(0.25);
    cc[cell * 4 + 1] = (F(1, 0, 1) + F(1, 0, 2) + F(1, 1, 1) + F(1, 1, 0)) * T(0.25);
    cc[cell * 4 + 2] = (F(1, 1, 2) + F(1, 1, 3) + F(0, 1, 2) + F(0, 1, 1)) * T(0.25);
    cc[cell * 4 + 3] = (F(0, 1, 3) + F(0, 1, 0) + F(0, 0, 3) + F(0, 0, 2)) * T(0.25);
  }
}
template <class T>
void coarsen_coef(cudaStream_t s, const Grid& gf, const Grid& gc, const T* cf, T* cc) {
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s, pdl_launch(k_coarsen<T>, nblocks(gc.ncell), RED_THREADS, 0, s, gf, gc, cf, cc));
}
template void coarsen_coef<double>(cudaStream_t, const Grid&, const Grid&, const double*, double*);
template void coarsen_coef<float>(cudaStream_t, const Grid&, const Grid&, const float*, float*);

// l1 row sums of the assembled element matrices: D_ii = sum_T sum_j |K_T(i, j)|, so that the
// spectrum of D^{-1} K lies in (0, 1].
template <class T>
__global__ void k_l1_elastic(Grid g, Consts<T> cs, const T* coef, T* dinv) {
  pdl_enter();
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n) return;
  int cells[8], ts[8], ks[8];
  int cnt = node_elements(g, node, cells, ts, ks);
  int NE = elems_per_cell(g.kind);
  T dx = T(0), dy = T(0);
  for (int e = 0; e < cnt; ++e) {
    int t = ts[e], k = ks[e];
    T w = coef[cells[e] * NE + t] * cs.area;
    T gkx = T(gxr(g.kind, t, k)) * cs.ihx, gky = T(gyr(g.kind, t, k)) * cs.ihy;
    T sx = T(0), sy = T(0);
    for (int l = 0; l < 3; ++l) {
      T glx = T(gxr(g.kind, t, l)) * cs.ihx, gly = T(gyr(g.kind, t, l)) * cs.ihy;
      sx += fabs(gkx * glx * cs.lam2mu + gky * gly * cs.mu) + fabs(gkx * gly * cs.lam + gky * glx * cs.mu);
      sy += fabs(gky * glx * cs.lam + gkx * gly * cs.mu) + fabs(gky * gly * cs.lam2mu + gkx * glx * cs.mu);
    }
    dx += w * sx;
    dy += w * sy;
  }
  int X2, Y2;
  node_coords(g, node, X2, Y2);
  dinv[2 * node] = (is_fixed(g, X2, Y2, 0) || dx <= T(0)) ? T(0) : T(1) / dx;
  dinv[2 * node + 1] = (is_fixed(g, X2, Y2, 1) || dy <= T(0)) ? T(0) : T(1) / dy;
}
template <class T>
void l1_dinv_elastic(cudaStream_t s, const Grid& g, const Mat& m, const T* coef, T* dinv) {
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s, pdl_launch(k_l1_elastic<T>, nblocks(g.n), RED_THREADS, 0, s, g, make_consts<T>(g, m), coef, dinv));
}
template void l1_dinv_elastic<double>(cudaStream_t, const Grid&, const Mat&, const double*, double*);
template void l1_dinv_elastic<float>(cudaStream_t, const Grid&, const Mat&, const float*, float*);

template <class T>
__global__ void k_l1_damage(Grid g, Consts<T> cs, const T* w, T* dinv) {
  pdl_enter();
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n) return;
  int cells[8], ts[8], ks[8];
  int cnt = node_elements(g, node, cells, ts, ks);
  int NE = elems_per_cell(g.kind);
  T dd = T(0);
  for (int e = 0; e < cnt; ++e) {
    int t = ts[e], k = ks[e];
    T me = w[cells[e] * NE + t] * cs.area * T(1.0 / 12.0);
    T gkx = T(gxr(g.kind, t, k)) * cs.ihx, gky = T(gyr(g.kind, t, k)) * cs.ihy;
    for (int l = 0; l < 3; ++l) {
      T glx = T(gxr(g.kind, t, l)) * cs.ihx, gly = T(gyr(g.kind, t, l)) * cs.ihy;
      dd += fabs(me * (l == k ? T(2) : T(1)) + cs.c1 * cs.area * (gkx * glx + gky * gly));
    }
  }
  int X2, Y2;
  node_coords(g, node, X2, Y2);
  dinv[node] = (is_fixed(g, X2, Y2, 2) || dd <= T(0)) ? T(0) : T(1) / dd;
}
template <class T>
void l1_dinv_damage(cudaStream_t s, const Grid& g, const Mat& m, const T* w, T* dinv) {
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s, pdl_launch(k_l1_damage<T>, nblocks(g.n), RED_THREADS, 0, s, g, make_consts<T>(g, m), w, dinv));
}
template void l1_dinv_damage<double>(cudaStream_t, const Grid&, const Mat&, const double*, double*);
template void l1_dinv_damage<float>(cudaStream_t, const Grid&, const Mat&, const float*, float*);

// ---------------------------------------------------------------------------------------------
// multigrid transfer (P1 nodal interpolation between nested structured meshes)
// ---------------------------------------------------------------------------------------------
template <class T>
__global__ void k_restrict(Grid gf, Grid gc, int ncomp, int comp_base, const T* rf, T* bc,
                           const uint8_t* excl_c) {
  pdl_enter();
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= gc.n) return;
  restrict_node(gf, gc, ncomp, comp_base, rf, bc, excl_c, node);
}
template <class T>
void restrict_res(cudaStream_t s, const Grid& gf, const Grid& gc, int ncomp, int comp_base,
                  const T* rf, T* bc, const uint8_t* excl_c, int level) {
  // read the fine residual, write the coarse right-hand side (+ coarse mask bytes)
  const double bytes = double(ncomp) * sizeof(T) * (gf.n + gc.n) + (excl_c ? double(gc.n) : 0.0);
  PF_LAUNCH(kclass(KC_TRANSFER, sizeof(T) == 8, level), bytes, s,
            pdl_launch(k_restrict<T>, nblocks(gc.n), RED_THREADS, 0, s, gf, gc, ncomp, comp_base, rf, bc, excl_c));
}
template void restrict_res<double>(cudaStream_t, const Grid&, const Grid&, int, int, const double*,
                                   double*, const uint8_t*, int);
template void restrict_res<float>(cudaStream_t, const Grid&, const Grid&, int, int, const float*,
                                  float*, const uint8_t*, int);


// ---------------------------------------------------------------------------------------------
// coarsest level: dense assembly, Cholesky and triangular solves in one thread block
// ---------------------------------------------------------------------------------------------
template <class T>
__global__ void k_coarse_assemble(Grid g, Mat m, int physics, const T* coef, T* A, T* diag0,
                                  const uint8_t* excl) {
  pdl_enter();
  // block = column j, threads = rows i
  const int ncomp = physics == 0 ? 2 : 1;
  const int nd = g.n * ncomp;
  int col = blockIdx.x;
  int nj = col / ncomp, cjc = col % ncomp;
  int X2j, Y2j;
  node_coords(g, nj, X2j, Y2j);
  bool fj = is_fixed(g, X2j, Y2j, physics == 0 ? cjc : 2) || (excl && excl[nj]);
  int NE = elems_per_cell(g.kind);
  for (int row = threadIdx.x; row < nd; row += blockDim.x) {
    int ni = row / ncomp, cic = row % ncomp;
    int X2i, Y2i;
    node_coords(g, ni, X2i, Y2i);
    bool fi = is_fixed(g, X2i, Y2i, physics == 0 ? cic : 2) || (excl && excl[ni]);
    double acc = 0.0;
    if (fi || fj) {
      acc = (row == col) ? 1.0 : 0.0;
    } else {
      for (int cell = 0; cell < g.ncell; ++cell) {
        int cj = cell / g.nx, ci = cell - cj * g.nx;
        for (int t = 0; t < NE; ++t) {
          int nn[3];
          cell_nodes(g, ci, cj, t, nn[0], nn[1], nn[2]);
          int ki = -1, kj = -1;
          for (int k = 0; k < 3; ++k) {
            if (nn[k] == ni) ki = k;
            if (nn[k] == nj) kj = k;
          }
          if (ki < 0 || kj < 0) continue;
          double w = double(coef[cell * NE + t]) * g.area;
          double gix = gxr(g.kind, t, ki) * g.ihx, giy = gyr(g.kind, t, ki) * g.ihy;
          double gjx = gxr(g.kind, t, kj) * g.ihx, gjy = gyr(g.kind, t, kj) * g.ihy;
          if (physics == 0) {
            double v;
            if (cic == 0 && cjc == 0) v = gix * gjx * m.lam2mu + giy * gjy * m.mu;
            else if (cic == 0 && cjc == 1) v = gix * gjy * m.lam + giy * gjx * m.mu;
            else if (cic == 1 && cjc == 0) v = giy * gjx * m.lam + gix * gjy * m.mu;
            else v = giy * gjy * m.lam2mu + gix * gjx * m.mu;
            acc += w * v;
          } else {
            acc += w * (ki == kj ? 2.0 : 1.0) / 12.0 + m.c1 * g.area * (gix * gjx + giy * gjy);
          }
        }
      }
    }
    A[(size_t)row * nd + col] = T(acc);
    if (row == col) diag0[row] = T(acc);
  }
}
template <class T>
void coarse_assemble(cudaStream_t s, const Grid& g, const Mat& m, int physics, const T* coef, T* A,
                     T* diag0, const uint8_t* excl) {
  int nd = g.n * (physics == 0 ? 2 : 1);
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s, pdl_launch(k_coarse_assemble<T>, nd, 256, 0, s, g, m, physics, coef, A, diag0, excl));
}
template void coarse_assemble<double>(cudaStream_t, const Grid&, const Mat&, int, const double*,
                                      double*, double*, const uint8_t*);
template void coarse_assemble<float>(cudaStream_t, const Grid&, const Mat&, int, const float*,
                                     float*, float*, const uint8_t*);

// Active-set mask of a coarse level: a coarse node is excluded iff the fine node at the same
// position is excluded (coarse vertex (I,J) = fine vertex (2I,2J); coarse centre (I,J) = fine
// vertex (2I+1, 2J+1)).
__global__ void k_mask_restrict(Grid gf, Grid gc, const uint8_t* ef, uint8_t* ec) {
  pdl_enter();
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= gc.n) return;
  int X2, Y2;
  node_coords(gc, node, X2, Y2);
  ec[node] = ef[Y2 * (gf.nx + 1) + X2];  // the fine vertex (X2, Y2) coincides with this node
}
void mask_restrict(cudaStream_t s, const Grid& gf, const Grid& gc, const uint8_t* ef, uint8_t* ec) {
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s,
            pdl_launch(k_mask_restrict, nblocks(gc.n), RED_THREADS, 0, s, gf, gc, ef, ec));
}

// In-place Cholesky A = L L^T (lower triangle); a pivot that is not positive relative to the
// original diagonal is replaced by that diagonal (a regularized factorization, acceptable for a
// preconditioner when the coarse operator is singular).
template <class T>
__global__ void k_coarse_factor(int n, T* A, const T* diag0) {
  pdl_enter();
  __shared__ T piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      T d = A[(size_t)k * n + k];
      T ref = diag0[k] > T(0) ? diag0[k] : T(1);
      if (!(d > T(1e-10) * ref)) d = ref;
      piv = sqrt(d);
      A[(size_t)k * n + k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(size_t)i * n + k] /= piv;
    __syncthreads();
    int m = n - k - 1;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      int i = k + 1 + idx / m, j = k + 1 + idx % m;
      if (j <= i) A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
    }
    __syncthreads();
  }
}
template <class T>
void coarse_factor(cudaStream_t s, int n, T* A, const T* diag0) {
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s, pdl_launch(k_coarse_factor<T>, 1, 1024, 0, s, n, A, diag0));
}
template void coarse_factor<double>(cudaStream_t, int, double*, const double*);
template void coarse_factor<float>(cudaStream_t, int, float*, const float*);

// Column j of A^{-1} from the Cholesky factor (one block per column; set-up time only).
template <class T>
__global__ void k_coarse_invert(int n, const T* L, T* Ainv) {
  pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  T* y = reinterpret_cast<T*>(smem_raw);
  const int j = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y[i] = (i == j) ? T(1) : T(0);
  __syncthreads();
  for (int k = 0; k < n; ++k) {  // forward: L y = e_j
    if (threadIdx.x == 0) y[k] /= L[(size_t)k * n + k];
    __syncthreads();
    T yk = y[k];
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) y[i] -= L[(size_t)i * n + k] * yk;
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {  // backward: L^T x = y
    if (threadIdx.x == 0) y[k] /= L[(size_t)k * n + k];
    __syncthreads();
    T yk = y[k];
    for (int i = threadIdx.x; i < k; i += blockDim.x) y[i] -= L[(size_t)k * n + i] * yk;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Ainv[(size_t)j * n + i] = y[i];
}
template <class T>
void coarse_invert(cudaStream_t s, int n, const T* L, T* Ainv) {
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s, pdl_launch(k_coarse_invert<T>, n, 128, n * sizeof(T), s, n, L, Ainv));
}
template void coarse_invert<double>(cudaStream_t, int, const double*, double*);
template void coarse_invert<float>(cudaStream_t, int, const float*, float*);

// ---- coarsest level, shared-memory path --------------------------------------------------------
// The packed lower triangle (row i holds L[i][0..i] at i(i+1)/2) of the coarsest operator fits
// in one SM's shared memory (n <= 320 in FP32): the factorization runs there with one block,
// and the inverse with one warp per column against a shared-memory copy of the factor.
__device__ __forceinline__ int packed(int i, int j) { return i * (i + 1) / 2 + j; }

template <class T>
size_t coarse_smem_bytes(int n) {
  return (size_t)n * (n + 1) / 2 * sizeof(T) + (size_t)COARSE_WARPS * n * sizeof(T);
}

// Same pivot rule and the same operations, in the same order per entry, as k_coarse_factor;
// the packed factor is written back over the first n(n+1)/2 entries of A.
template <class T>
__global__ void __launch_bounds__(1024) k_coarse_factor_smem(int n, T* A, const T* diag0) {
  pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  T* L = reinterpret_cast<T*>(smem_raw);
  T* colk = L + (size_t)n * (n + 1) / 2;  // column k below the diagonal
  __shared__ T piv;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j <= i; j += 32) L[packed(i, j)] = A[(size_t)i * n + j];
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      T d = L[packed(k, k)];
      T ref = diag0[k] > T(0) ? diag0[k] : T(1);
      if (!(d > T(1e-10) * ref)) d = ref;
      piv = sqrt(d);
      L[packed(k, k)] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + tid; i < n; i += nt) {
      const T v = L[packed(i, k)] / piv;
      L[packed(i, k)] = v;
      colk[i] = v;
    }
    __syncthreads();
    for (int i = k + 1 + warp; i < n; i += nw) {
      const T lik = colk[i];
      T* row = L + packed(i, 0);
      for (int j = k + 1 + lane; j <= i; j += 32) row[j] -= lik * colk[j];
    }
    __syncthreads();
  }
  const int np = n * (n + 1) / 2;
  for (int t = tid; t < np; t += nt) A[t] = L[t];
}

// Column j of A^{-1} = L^{-T} L^{-1} e_j: forward substitution by rows (dot products along row
// i of L), backward substitution by columns of L^T (row k of L scattered into y).
template <class T>
__global__ void __launch_bounds__(32 * COARSE_WARPS) k_coarse_invert_smem(int n, const T* Lp, T* Ainv) {
  pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  T* L = reinterpret_cast<T*>(smem_raw);
  const int np = n * (n + 1) / 2;
  for (int t = threadIdx.x; t < np; t += blockDim.x) L[t] = Lp[t];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T* y = L + np + (size_t)warp * n;
  const int j = blockIdx.x * COARSE_WARPS + warp;
  __syncthreads();
  if (j >= n) return;
  for (int i = lane; i < n; i += 32) y[i] = T(0);
  __syncwarp();
  for (int i = j; i < n; ++i) {  // forward: L y = e_j (y_i = 0 for i < j)
    const T* row = L + packed(i, 0);
    T acc = T(0);
    for (int k = j + lane; k < i; k += 32) acc += row[k] * y[k];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) y[i] = ((i == j ? T(1) : T(0)) - acc) / row[i];
    __syncwarp();
  }
  for (int k = n - 1; k >= 0; --k) {  // backward: L^T x = y, x overwrites y
    const T* row = L + packed(k, 0);
    const T xk = y[k] / row[k];
    __syncwarp();
    if (lane == 0) y[k] = xk;
    for (int i = lane; i < k; i += 32) y[i] -= row[i] * xk;
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) Ainv[(size_t)j * n + i] = y[i];
}

// Largest dynamic shared memory both kernels can be given (opt-in limit minus their static
// shared memory), raised to that once per process and instantiation; 0 if that fails.
template <class T>
size_t coarse_smem_limit() {
  static size_t limit = [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return size_t(0);
    cudaFuncAttributes fa, fb;
    if (cudaFuncGetAttributes(&fa, k_coarse_factor_smem<T>) != cudaSuccess ||
        cudaFuncGetAttributes(&fb, k_coarse_invert_smem<T>) != cudaSuccess)
      return size_t(0);
    const size_t st = fa.sharedSizeBytes > fb.sharedSizeBytes ? fa.sharedSizeBytes : fb.sharedSizeBytes;
    if ((size_t)optin <= st) return size_t(0);
    const int lim = optin - (int)st;
    if (cudaFuncSetAttribute(k_coarse_factor_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess ||
        cudaFuncSetAttribute(k_coarse_invert_smem<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess)
      return size_t(0);
    return (size_t)lim;
  }();
  return limit;
}

template <class T>
void coarse_factor_invert(cudaStream_t s, int n, T* A, const T* diag0, T* Ainv) {
  const size_t smem = coarse_smem_bytes<T>(n);
  if (smem > coarse_smem_limit<T>()) {  // does not fit (FP64 elastic): global-memory kernels
    coarse_factor<T>(s, n, A, diag0);
    coarse_invert<T>(s, n, A, Ainv);
    return;
  }
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s,
            pdl_launch(k_coarse_factor_smem<T>, 1, 1024, smem, s, n, A, diag0));
  PF_LAUNCH(kclass(KC_SETUP, false, false), 0.0, s,
            pdl_launch(k_coarse_invert_smem<T>, (n + COARSE_WARPS - 1) / COARSE_WARPS,
                       32 * COARSE_WARPS, smem, s, n, (const T*)A, Ainv));
}
template void coarse_factor_invert<double>(cudaStream_t, int, double*, const double*, double*);
template void coarse_factor_invert<float>(cudaStream_t, int, float*, const float*, float*);

// x = A^{-1} b with the stored symmetric inverse: thread i reads column i (coalesced).
template <class T>
__global__ void k_coarse_solve(int n, const T* Ainv, const T* b, T* x) {
  pdl_enter();
  extern __shared__ unsigned char smem_raw[];
  T* bs = reinterpret_cast<T*>(smem_raw);
  for (int i = threadIdx.x; i < n; i += blockDim.x) bs[i] = b[i];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T acc = T(0);
    for (int j = 0; j < n; ++j) acc += Ainv[(size_t)j * n + i] * bs[j];
    x[i] = acc;
  }
}
template <class T>
void coarse_solve(cudaStream_t s, int n, const T* Ainv, const T* b, T* x) {
  int threads = n < 1024 ? ((n + 31) / 32) * 32 : 1024;
  PF_LAUNCH(kclass(KC_COARSE, false, false), 0.0, s, pdl_launch(k_coarse_solve<T>, 1, threads, n * sizeof(T), s, n, Ainv, b, x));
}
template void coarse_solve<double>(cudaStream_t, int, const double*, const double*, double*);
template void coarse_solve<float>(cudaStream_t, int, const float*, const float*, float*);

// Active components are within the zero tolerance of their bound (eq. reducedis): the step puts
// them on it, d_i = bound_i - x_i; inactive components keep the reduced Newton step.
__global__ void k_snap_active(Grid g, const uint8_t* act, const double* x, const double* lo, double* d) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const uint8_t a = act[i];
  if (a == 1) d[i] = lo[i] - x[i];
  else if (a == 2) d[i] = upper_of(g, i, lo[i]) - x[i];
}
void snap_active(cudaStream_t s, const Grid& g, const uint8_t* act, const double* x, const double* lo,
                 double* d) {
  PF_LAUNCH(kclass(KC_VECTOR, false, false), 0.0, s,
            pdl_launch(k_snap_active, nblocks(g.n), RED_THREADS, 0, s, g, act, x, lo, d));
}

// ---------------------------------------------------------------------------------------------
// steepest-descent direction of ||Phi||^2 / 2 (Algorithm 4 fallback)
// Phi_i = phi(x - l, psi), psi = phi(h - x, -F): dPhi/dx = pa - pb qa on the diagonal and
// -pb qb H off it, with (pa, pb) = grad phi at (x - l, psi), (qa, qb) = grad phi at (h - x, -F).
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void dphi(double a, double b, double& da, double& db) {
  double r = sqrt(a * a + b * b);
  if (r > 0.0) {
    da = a / r - 1.0;
    db = b / r - 1.0;
  } else {
    da = db = 1.0 / sqrt(2.0) - 1.0;
  }
}
__global__ void k_merit_parts(Grid g, const double* x, const double* F, const double* lo, double* v,
                              double* dg) {
  pdl_enter();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  double l = lo[i], h = upper_of(g, i, l);
  double xi = x[i], Fi = F[i];
  double psi = phi_fb(h - xi, -Fi);
  double ph = phi_fb(xi - l, psi);
  double pa, pb, qa, qb;
  dphi(xi - l, psi, pa, pb);
  dphi(h - xi, -Fi, qa, qb);
  v[i] = -pb * qb * ph;
  dg[i] = (pa - pb * qa) * ph;
}
void merit_parts(cudaStream_t s, const Grid& g, const double* x, const double* F,
                 const double* lo, double* v, double* dg) {
  PF_LAUNCH(kclass(KC_VECTOR, false, false), 0.0, s, pdl_launch(k_merit_parts, nblocks(g.n), RED_THREADS, 0, s, g, x, F, lo, v, dg));
}
__global__ void k_merit_dir(size_t n, const double* dg, const double* Hv, double* d) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) d[i] = -(dg[i] + Hv[i]);
}
void merit_direction(cudaStream_t s, size_t n, const double* dg, const double* Hv, double* d) {
  PF_LAUNCH(kclass(KC_VECTOR, false, false), 0.0, s, pdl_launch(k_merit_dir, nblocks(n), RED_THREADS, 0, s, n, dg, Hv, d));
}

}  // namespace pf
