// Host driver of libpf: hierarchy set-up, Krylov solvers, the reduced-space active-set damage
// solve (Algorithm 4), over-relaxed alternate minimization (Algorithms 1-2) and the C ABI.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <cstdarg>
#include <type_traits>
#include <new>
#include <string>

#include "solver.hpp"

using namespace pf;

// ---------------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------------
static thread_local std::string g_err;
static pf_status fail(pf_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}
namespace pf {
void set_error_message(const char* msg) { g_err = msg; }
}  // namespace pf
// PF_DEBUG=1 in the environment prints one line per damage-solve iteration on stderr
static bool debug_enabled() {
  static const bool on = getenv("PF_DEBUG") && getenv("PF_DEBUG")[0] == '1';
  return on;
}
// PF_TRACE=1 prints one line per alternate-minimization iteration on stderr (damage change,
// relative displacement change, omega_bar, cumulative Krylov counts)
static bool trace_enabled() {
  static const bool on = getenv("PF_TRACE") && getenv("PF_TRACE")[0] == '1';
  return on;
}
#define CU(call)                                                                       \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess)                                                             \
      return fail(PF_ECUDA, "%s failed: %s (%s:%d)%s%.160s", #call, cudaGetErrorString(e_), \
                  __FILE__, __LINE__, *prof_failed_launch() ? "; first failed launch: " : "", \
                  prof_failed_launch());                                               \
  } while (0)
#define TRY(expr)                    \
  do {                               \
    pf_status s_ = (expr);           \
    if (s_ != PF_OK) return s_;      \
  } while (0)

// Exclusive use of a sim for the duration of one entry point: a second caller on the same sim
// gets PF_EBUSY instead of racing on its fields, reduction slots and work buffers.
struct SimClaim {
  pf_sim* s;
  bool ok;
  explicit SimClaim(pf_sim* sim) : s(sim) {
    bool idle = false;
    ok = s->busy.compare_exchange_strong(idle, true);
  }
  ~SimClaim() {
    if (ok) s->busy = false;
  }
};
#define CLAIM(sim)                                             \
  SimClaim claim_(sim);                                        \
  if (!claim_.ok) return fail(PF_EBUSY, "sim busy")


// ---------------------------------------------------------------------------------------------
// workspace arena
// ---------------------------------------------------------------------------------------------
namespace {
struct Arena {
  char* base;
  size_t cap, off = 0;
  bool dry;
  template <class T>
  T* take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off += n * sizeof(T);
    return p;
  }
};

constexpr int COARSE_TARGET_NODES = 128;
constexpr int MAX_DENSE_DOFS = 320;

bool pin_maps(int X2, int Y2, int kind) {
  // a node of this level is also a node of the next coarser level
  if ((X2 & 1) || (Y2 & 1)) return false;
  int cx = X2 / 2, cy = Y2 / 2;
  if ((cx & 1) != (cy & 1)) return false;
  if ((cx & 1) && kind != CROSSED) return false;
  return true;
}

Grid make_grid(const pf_mesh_desc& d, int level) {
  Grid g;
  memset(&g, 0, sizeof g);
  int f = 1 << level;
  g.kind = d.kind == PF_MESH_CROSSED ? CROSSED : RIGHT;
  g.nx = d.nx / f;
  g.ny = d.ny / f;
  g.nv = (g.nx + 1) * (g.ny + 1);
  g.ncell = g.nx * g.ny;
  g.n = g.nv + (g.kind == CROSSED ? g.ncell : 0);
  g.nelem = g.ncell * elems_per_cell(g.kind);
  g.hx = d.lx / g.nx;
  g.hy = d.ly / g.ny;
  g.ihx = 1.0 / g.hx;
  g.ihy = 1.0 / g.hy;
  g.area = g.hx * g.hy / (g.kind == CROSSED ? 4.0 : 2.0);
  for (int e = 0; e < 4; ++e)
    for (int c = 0; c < 3; ++c) g.fixed[e][c] = d.fixed[e][c] ? 1 : 0;
  g.npins = d.n_pins;
  for (int k = 0; k < d.n_pins; ++k) {
    g.pin_x2[k] = d.pin_x2[k] / f;
    g.pin_y2[k] = d.pin_y2[k] / f;
    g.pin_comp[k] = d.pin_comp[k];
    if (g.pin_x2[k] > 0 && g.pin_x2[k] < 2 * g.nx && g.pin_y2[k] > 0 && g.pin_y2[k] < 2 * g.ny)
      g.interior_pins = 1;
  }
  return g;
}

pf_status validate(const pf_mesh_desc* d) {
  if (!d) return fail(PF_EINVAL, "null mesh descriptor");
  if (d->kind != PF_MESH_RIGHT && d->kind != PF_MESH_CROSSED)
    return fail(PF_EINVAL, "unknown mesh kind %d", d->kind);
  if (d->nx < 1 || d->ny < 1 || d->nx > 65536 || d->ny > 65536)
    return fail(PF_EINVAL, "mesh size %d x %d out of range", d->nx, d->ny);
  if (!(d->lx > 0) || !(d->ly > 0)) return fail(PF_EINVAL, "domain size must be positive");
  if (2.0 * (double(d->nx) + 1.0) * (double(d->ny) + 1.0) > 2147483647.0)
    return fail(PF_EINVAL, "mesh %d x %d has too many nodes", d->nx, d->ny);
  if (d->n_pins < 0 || d->n_pins > PF_MAX_PINS) return fail(PF_EINVAL, "bad pin count");
  if (d->n_boxes < 0 || d->n_boxes > PF_MAX_BOXES) return fail(PF_EINVAL, "bad box count");
  if (d->mode_I != 0 && d->mode_I != 1) return fail(PF_EINVAL, "mode_I must be 0 or 1");
  if (d->mode_I && !(d->mode_I_param[0] == d->mode_I_param[0] && d->mode_I_param[1] ==
                     d->mode_I_param[1] && d->mode_I_param[2] == d->mode_I_param[2] &&
                     d->mode_I_param[3] == d->mode_I_param[3]))
    return fail(PF_EINVAL, "mode_I parameters must be finite numbers");
  for (int k = 0; k < d->n_pins; ++k) {
    int X2 = d->pin_x2[k], Y2 = d->pin_y2[k];
    bool vert = !(X2 & 1) && !(Y2 & 1), cen = (X2 & 1) && (Y2 & 1);
    if (X2 < 0 || Y2 < 0 || X2 > 2 * d->nx || Y2 > 2 * d->ny || !(vert || (cen && d->kind == PF_MESH_CROSSED)))
      return fail(PF_EINVAL, "pin %d is not a node", k);
    if (d->pin_comp[k] < 0 || d->pin_comp[k] > 2) return fail(PF_EINVAL, "pin %d: bad component", k);
  }
  // corner agreement: edges sharing a corner and prescribing the same component
  const int pairs[4][2] = {{0, 2}, {0, 3}, {1, 2}, {1, 3}};
  for (auto& pr : pairs)
    for (int c = 0; c < 3; ++c)
      if (d->fixed[pr[0]][c] && d->fixed[pr[1]][c] && d->load[pr[0]][c] != d->load[pr[1]][c])
        return fail(PF_EINVAL, "edges %d and %d prescribe different values at a corner", pr[0], pr[1]);
  return PF_OK;
}

int count_levels(const pf_mesh_desc& d) {
  int L = 1;
  int nx = d.nx, ny = d.ny;
  int kind = d.kind == PF_MESH_CROSSED ? CROSSED : RIGHT;
  while (true) {
    int nn = (nx + 1) * (ny + 1) + (kind == CROSSED ? nx * ny : 0);
    if (nn <= COARSE_TARGET_NODES) break;
    if ((nx & 1) || (ny & 1) || nx < 2 || ny < 2) break;
    bool ok = true;
    int f = 1 << (L - 1);
    for (int k = 0; k < d.n_pins; ++k)
      if (!pin_maps(d.pin_x2[k] / f, d.pin_y2[k] / f, kind)) ok = false;
    if (!ok) break;
    nx /= 2;
    ny /= 2;
    ++L;
  }
  return L;
}

template <class T>
void take_level(Arena& a, Level& L, bool coarsest) {
  const Grid& g = L.g;
  LevelBuf<T>& B = L.buf<T>();
  B.coefE = a.take<T>(g.nelem);
  B.wD = a.take<T>(g.nelem);
  B.dinvE = a.take<T>(2 * (size_t)g.n);
  B.dinvD = a.take<T>(g.n);
  B.b = a.take<T>(2 * (size_t)g.n);
  B.x = a.take<T>(2 * (size_t)g.n);
  B.r = a.take<T>(2 * (size_t)g.n);
  B.xt = a.take<T>(2 * (size_t)g.n);
  B.d = a.take<T>(2 * (size_t)g.n);
  B.dt = a.take<T>(2 * (size_t)g.n);
  if (coarsest && L.dense) {
    size_t ne = 2 * (size_t)g.n, nd = g.n;
    B.AE = a.take<T>(ne * ne);
    B.AD = a.take<T>(nd * nd);
    B.diagE = a.take<T>(ne);
    B.diagD = a.take<T>(nd);
    B.AEi = a.take<T>(ne * ne);
    B.ADi = a.take<T>(nd * nd);
  }
}

template <class T>
void take_krylov(Arena& a, Krylov<T>& k, size_t n2) {
  k.x = a.take<T>(n2);
  k.r = a.take<T>(n2);
  k.z = a.take<T>(n2);
  k.p = a.take<T>(n2);
  k.Ap = a.take<T>(n2);
}

void layout(pf_sim& s, Arena& a) {
  const pf_mesh_desc& d = s.desc;
  int L = count_levels(d);
  s.lv.resize(L);
  for (int l = 0; l < L; ++l) s.lv[l].g = make_grid(d, l);
  Level& lc = s.lv[L - 1];
  lc.dense = L > 1 && 2 * lc.g.n <= MAX_DENSE_DOFS;
  const Grid& g = s.lv[0].g;
  size_t n = g.n, n2 = 2 * n;
  s.u = a.take<double>(n2);
  s.alpha = a.take<double>(n);
  s.alpha_prev = a.take<double>(n);
  s.alpha32 = a.take<float>(n);
  s.xu = a.take<double>(n2);
  s.r64 = a.take<double>(n2);
  s.q = a.take<double>(g.nelem);
  s.eig = a.take<double>((size_t)g.ny * elems_per_cell(g.kind));
  s.xrs = a.take<double>(n);
  s.F = a.take<double>(n);
  s.Phi = a.take<double>(n);
  s.rhs = a.take<double>(n);
  s.drs = a.take<double>(n);
  s.xtr = a.take<double>(n);
  s.Ftr = a.take<double>(n);
  s.Phitr = a.take<double>(n);
  s.rhstr = a.take<double>(n);
  s.tmpa = a.take<double>(n2);
  s.tmpb = a.take<double>(n2);
  s.act = a.take<uint8_t>(n);
  s.acttr = a.take<uint8_t>(n);
  s.tmp32 = a.take<float>(n2);
  s.u32 = a.take<float>(n2);
  s.eig32 = a.take<float>((size_t)g.ny * elems_per_cell(g.kind));
  for (int k = 0; k < 12; ++k) s.nv[k] = a.take<float>(3 * n);
  s.nu0 = a.take<double>(n2);
  s.na0 = a.take<double>(n);
  s.ndu = a.take<double>(n2);
  s.nda = a.take<double>(n);
  take_krylov(a, s.k64, n2);
  take_krylov(a, s.k32, n2);
  for (int l = 0; l < L; ++l) {
    take_level<double>(a, s.lv[l], l == L - 1);
    take_level<float>(a, s.lv[l], l == L - 1);
    if (l > 0) s.lv[l].exclD = a.take<uint8_t>(s.lv[l].g.n);
  }
  size_t nb = ((size_t)(g.nx + 1 + TX - 1) / TX) * ((g.ny + 1 + TY_MIN - 1) / TY_MIN);
  nb = std::max<size_t>(nb, MAX_RED_BLOCKS);
  s.part = a.take<double>(nb * 4);
  s.ticket = a.take<unsigned>(64);
  s.scal = a.take<double>(S_COUNT);
  s.ws_used = a.off;
}

inline RedSlot slot(pf_sim& s, int k) { return RedSlot{s.part, s.ticket, s.scal + k}; }

}  // namespace

double* pf_ctx::take_slot() {
  std::lock_guard<std::mutex> lk(mu);
  if (free_slots.empty()) {
    constexpr int SLOTS = 64, SLOT_DOUBLES = 64;
    double* p = nullptr;
    if (cudaMallocHost(&p, SLOTS * SLOT_DOUBLES * sizeof(double)) != cudaSuccess) return nullptr;
    chunks.push_back(p);
    for (int k = SLOTS - 1; k >= 0; --k) free_slots.push_back(p + k * SLOT_DOUBLES);
  }
  double* p = free_slots.back();
  free_slots.pop_back();
  ++users;
  return p;
}

static void free_ctx(pf_ctx* c) {
  for (double* p : c->chunks) cudaFreeHost(p);
  delete c;
}

void pf_ctx::give_slot(double* p) {
  bool last;
  {
    std::lock_guard<std::mutex> lk(mu);
    free_slots.push_back(p);
    last = --users == 0 && closed;
  }
  if (last) free_ctx(this);
}

void pf_ctx::add_user() {
  std::lock_guard<std::mutex> lk(mu);
  ++users;
}

void pf_ctx::drop_user() {
  bool last;
  {
    std::lock_guard<std::mutex> lk(mu);
    last = --users == 0 && closed;
  }
  if (last) free_ctx(this);
}

namespace {

pf_status read_scalars(pf_sim& s, cudaStream_t st, int k, int cnt, double* out) {
  CU(cudaMemcpyAsync(s.host, s.scal + k, cnt * sizeof(double), cudaMemcpyDeviceToHost, st));
  CU(cudaStreamSynchronize(st));
  CU(cudaGetLastError());
  for (int i = 0; i < cnt; ++i) out[i] = s.host[i];
  return PF_OK;
}

// ---------------------------------------------------------------------------------------------
// operators on level 0 and the multigrid hierarchy
// ---------------------------------------------------------------------------------------------
enum Physics { ELASTIC = 0, DAMAGE = 1 };

template <class T>
const T* alpha_of(pf_sim& s);
template <>
const double* alpha_of<double>(pf_sim& s) { return s.alpha; }
template <>
const float* alpha_of<float>(pf_sim& s) { return s.alpha32; }

template <class T>
Krylov<T>& kry(pf_sim& s);
template <>
Krylov<double>& kry<double>(pf_sim& s) { return s.k64; }
template <>
Krylov<float>& kry<float>(pf_sim& s) { return s.k32; }

// y = A x on level l (masked operator of the free/inactive set), optional fused x.y
// The multigrid and Krylov operators read the per-element coefficient abar_T stored by the
// set-up on every level, level 0 included (the stencil is issue-bound, and recomputing abar_T
// from the nodal damage in every element of every sweep costs more instructions than the
// coefficient's bytes); the FP64 physical residual computes abar_T from alpha itself.
template <class T>
void apply_op(pf_sim& s, cudaStream_t st, int phys, int l, const T* x, T* y, bool dot, int sl) {
  Level& L = s.lv[l];
  if (phys == ELASTIC) {
    ElasticArgs<T> a{};
    a.x = x;
    a.alpha = alpha_of<T>(s);
    a.coef = L.buf<T>().coefE;
    a.y = y;
    a.slot = slot(s, sl);
    a.coarse = l;
    launch_elastic<T>(st, L.g, s.m, COEF_ELEM, M_MASKED, false, dot, a);
  } else {
    DamageArgs<T> a{};
    a.x = x;
    a.w = L.buf<T>().wD;
    a.excl = l == 0 ? s.act : L.exclD;
    a.y = y;
    a.slot = slot(s, sl);
    a.coarse = l;
    launch_damage<T>(st, L.g, s.m, M_MASKED, dot, a);
  }
}

// r = b - A x.  x0 > 0: x is not read but is the single Chebyshev step from zero, x0 D^-1 b,
// formed on the fly and written to x.
template <class T>
void residual_op(pf_sim& s, cudaStream_t st, int phys, int l, const T* b, T* x, T* r,
                 double x0 = 0.0) {
  Level& L = s.lv[l];
  if (phys == ELASTIC) {
    ElasticArgs<T> a{};
    if (x0 > 0.0) {
      a.x0b = 1;
      a.c0 = T(x0);
      a.dinv = L.buf<T>().dinvE;
      a.dout = x;
    } else {
      a.x = x;
    }
    a.alpha = alpha_of<T>(s);
    a.coef = L.buf<T>().coefE;
    a.b = b;
    a.y = r;
    a.coarse = l;
    launch_elastic<T>(st, L.g, s.m, COEF_ELEM, M_RESB, false, false, a);
  } else {
    DamageArgs<T> a{};
    if (x0 > 0.0) {
      a.x0b = 1;
      a.c0 = T(x0);
      a.dinv = L.buf<T>().dinvD;
      a.dout = x;
    } else {
      a.x = x;
    }
    a.w = L.buf<T>().wD;
    a.excl = l == 0 ? s.act : L.exclD;
    a.b = b;
    a.y = r;
    a.coarse = l;
    launch_damage<T>(st, L.g, s.m, M_RESB, false, a);
  }
}

template <class T>
void cheb_step(pf_sim& s, cudaStream_t st, int phys, int l, const T* b, const T* x, const T* d,
               T* xo, T* dout, double cd, double cr, const T* xc = nullptr, int dot_slot = -1,
               double x0 = 0.0) {
  Level& L = s.lv[l];
  const bool dot = dot_slot >= 0;
  if (phys == ELASTIC) {
    ElasticArgs<T> a{};
    if (xc) {
      a.xc = xc;
      a.gc = s.lv[l + 1].g;
    }
    a.x = x;
    a.x0b = x0 > 0.0;
    a.c0 = T(x0);
    a.alpha = alpha_of<T>(s);
    a.coef = L.buf<T>().coefE;
    a.b = b;
    a.d = d;
    a.dinv = L.buf<T>().dinvE;
    a.cd = T(cd);
    a.cr = T(cr);
    a.y = xo;
    a.dout = dout;
    a.coarse = l;
    if (dot) a.slot = slot(s, dot_slot);
    launch_elastic<T>(st, L.g, s.m, COEF_ELEM, M_CHEB, false, dot, a);
  } else {
    DamageArgs<T> a{};
    if (xc) {
      a.xc = xc;
      a.gc = s.lv[l + 1].g;
    }
    a.x = x;
    a.x0b = x0 > 0.0;
    a.c0 = T(x0);
    a.w = L.buf<T>().wD;
    a.excl = l == 0 ? s.act : L.exclD;
    a.b = b;
    a.d = d;
    a.dinv = L.buf<T>().dinvD;
    a.cd = T(cd);
    a.cr = T(cr);
    a.y = xo;
    a.dout = dout;
    a.coarse = l;
    if (dot) a.slot = slot(s, dot_slot);
    launch_damage<T>(st, L.g, s.m, M_CHEB, dot, a);
  }
}

// Coefficients of the first `steps` Chebyshev steps on D_l1^{-1} A over [lmin, lmax] = [0.1, 1]
// (l1 scaling bounds the spectrum by 1): d_k = cd[k] d_{k-1} + cr[k] D^-1 (b - A x_{k-1}).
static void cheb_coefs(int steps, double* cd, double* cr) {
  const double lmax = 1.0, lmin = 0.1;
  const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  for (int k = 0; k < steps; ++k) {
    if (k == 0) {
      cd[k] = 0.0;
      cr[k] = 1.0 / theta;
    } else {
      const double rn = 1.0 / (2.0 * sigma - rho);
      cd[k] = rn * rho;
      cr[k] = 2.0 * rn / delta;
      rho = rn;
    }
  }
}

// Chebyshev smoothing on D_l1^{-1} A over [lmin, lmax] = [0.1, 1] (l1 scaling bounds the
// spectrum by 1).  Starts from x (x0 == nullptr: from zero); result written to x.
// xc (optional, not with from_zero): the coarse-grid correction, prolongated into x by the first
// step as it reads x (x + P xc), which saves the separate prolongation launch.
// dot_slot >= 0: the last step also reduces b . x_new into that scalar slot
template <class T>
void smooth(pf_sim& s, cudaStream_t st, int phys, int l, const T* b, T* x, bool from_zero,
            int steps, const T* xc = nullptr, int dot_slot = -1) {
  LevelBuf<T>& B = s.lv[l].buf<T>();
  const int nc = phys == ELASTIC ? 2 : 1;
  const size_t nd = (size_t)nc * s.lv[l].g.n;
  double cdk[8 * MAX_CHEB], crk[8 * MAX_CHEB];  // up to the 8 * degree steps of a coarsest level
  cheb_coefs(steps, cdk, crk);
  // From zero the first step is pointwise, x = d = c0 D^-1 b: alone it is a launch that reads no
  // x (no fill needed); followed by more steps, the second forms it from b and dinv as it stages
  // its nodes, so it takes no launch of its own.  The first output buffer is chosen so that the
  // last step writes into x.
  const int k0 = from_zero && steps >= 2 ? 1 : 0;
  T* other = B.xt;
  T *cx = from_zero ? nullptr : x, *cd_ = nullptr, *nd_ = B.d;
  T* nx_ = from_zero ? (((steps - k0) & 1) ? x : other) : other;
  for (int k = k0; k < steps; ++k) {
    cheb_step<T>(s, st, phys, l, b, cx, cd_, nx_, nd_, cdk[k], crk[k], k == 0 ? xc : nullptr,
                 k == steps - 1 ? dot_slot : -1, k0 == 1 && k == 1 ? crk[0] : 0.0);
    // rotate buffers: new x becomes current; the old current x buffer is free for the next step
    T* ox = cx;
    cx = nx_;
    nx_ = ox ? ox : (cx == x ? other : x);
    T* od = cd_ ? cd_ : B.dt;
    cd_ = nd_;
    nd_ = od;
  }
  if (cx != x) cudaMemcpyAsync(x, cx, nd * sizeof(T), cudaMemcpyDeviceToDevice, st);
}

// Level from which the rest of an FP32 V-cycle runs in the single-block kernel (tail.cu),
// provided the hierarchy ends in a dense solve, all levels are in use and the tail spans at
// least two levels: level 0 if the whole hierarchy fits in one block's shared memory (the
// V-cycle becomes one launch), else the first level of at most TAIL_MAX_NODES nodes (a larger
// level keeps one SM busy for longer than its grid-wide launches take).  -1: no tail.
// shared-memory floats of one tail level: x, x_new, b, d, dinv (nc per node), coefficients per
// element, then one flag byte per node (+ one exclusion byte per node for the damage operator)
size_t tail_level_floats(const Grid& g, int nc) {
  return 5 * (size_t)nc * g.n + g.nelem + ((size_t)(nc == 1 ? 2 : 1) * g.n + 3) / 4;
}

int tail_first(pf_sim& s, int phys) {
  const int nlev = (int)s.lv.size();
  if (!s.use_tail || s.nl_active != nlev || nlev < 2 || !s.lv[nlev - 1].dense) return -1;
  if (s.tail_first[phys] != -2) return s.tail_first[phys];
  const size_t limit = tail_smem_limit();
  const int nc = phys == ELASTIC ? 2 : 1;
  const int nrc = phys == ELASTIC ? 3 : 4;  // element record components
  int best = -1;
  size_t acc = 0;
  int small = -1;  // first level of at most TAIL_MAX_NODES nodes that fits
  for (int l = nlev - 1; l >= 0 && nlev - l <= MAX_TAIL; --l) {
    const Grid& g = s.lv[l].g;
    acc += tail_level_floats(g, nc) * sizeof(float);
    // records of the largest (this) level
    if (acc + (size_t)nrc * g.nelem * sizeof(float) > limit) break;
    best = l;
    if (g.n <= TAIL_MAX_NODES) small = l;
  }
  if (best != 0) best = small;
  if (best > nlev - 2) best = -1;
  s.tail_first[phys] = best;
  return best;
}

void launch_tail(pf_sim& s, cudaStream_t st, int phys, const float* b, float* x, int deg,
                 const float* rf) {
  const int nlev = (int)s.lv.size(), l0 = s.tail_first[phys];
  const int nc = phys == ELASTIC ? 2 : 1;
  TailArgs a{};
  a.nl = nlev - l0;
  a.deg = s.cdeg;
  a.deg0 = l0 == 0 ? deg : s.cdeg;
  a.first_level = l0;
  double cdk[MAX_CHEB], crk[MAX_CHEB];
  cheb_coefs(MAX_CHEB, cdk, crk);
  for (int k = 0; k < MAX_CHEB; ++k) {
    a.cheb_cd[k] = float(cdk[k]);
    a.cheb_cr[k] = float(crk[k]);
  }
  const Level& Lc = s.lv[nlev - 1];
  a.Ainv = phys == ELASTIC ? Lc.f32.AEi : Lc.f32.ADi;
  a.b_in = b;
  a.x_out = x;
  if (rf) {  // right-hand side restricted from the finer level's residual by the kernel
    a.rf = rf;
    a.gf = s.lv[l0 - 1].g;
  }
  int off = 0;
  for (int k = 0; k < a.nl; ++k) {
    const Level& L = s.lv[l0 + k];
    TailLevel& t = a.L[k];
    t.g = L.g;
    t.cs = make_consts<float>(L.g, s.m);
    t.coef = phys == ELASTIC ? L.f32.coefE : L.f32.wD;
    t.dinv = phys == ELASTIC ? L.f32.dinvE : L.f32.dinvD;
    t.excl = phys == DAMAGE ? (l0 + k == 0 ? s.act : L.exclD) : nullptr;
    const int nd = nc * L.g.n;
    t.ox = off;
    t.oxn = t.ox + nd;
    t.ob = t.oxn + nd;
    t.od = t.ob + nd;
    t.odi = t.od + nd;
    t.oc = t.odi + nd;
    t.oe = t.oc + L.g.nelem;
    off += (int)tail_level_floats(L.g, nc);
  }
  a.orec = off;  // records of the largest level (the first)
  const int nrec = (phys == ELASTIC ? 3 : 4) * s.lv[l0].g.nelem;
  const int nd = nc * s.lv[nlev - 1].g.n, np = (nd + 1) / 2;
  a.dense_slices = std::max(1, std::min(TAIL_THREADS / np, nrec / nd));
  off += std::max(nrec, a.dense_slices * nd);
  tail_vcycle(st, nc, a, (size_t)off * sizeof(float));
}

// Returns true if dot_slot received b . x from the last level-0 smoothing step (false when the
// single-block tail ran this level or no slot was asked for).
// rf (levels below the finest): b is not formed yet; it is the restriction P^T rf of the finer
// level's residual.  The single-block tail forms it as it loads the level; otherwise it is
// formed into b (this level's right-hand side buffer) by the restriction kernel first.
template <class T>
bool vcycle(pf_sim& s, cudaStream_t st, int phys, int l, const T* b, T* x, int deg,
            int dot_slot = -1, const T* rf = nullptr) {
  const int nc = phys == ELASTIC ? 2 : 1;
  if constexpr (std::is_same<T, float>::value) {
    if (l == tail_first(s, phys)) {
      launch_tail(s, st, phys, b, x, deg, rf);
      return false;
    }
  }
  Level& L = s.lv[l];
  LevelBuf<T>& B = L.buf<T>();
  const int nlev = s.nl_active;  // levels in use (mg_levels_max)
  const int dl = l == 0 ? deg : s.cdeg;  // smoothing steps on this level
  if (rf) {
    const Level& F = s.lv[l - 1];
    restrict_res<T>(st, F.g, L.g, nc, phys == ELASTIC ? 0 : 2, rf, const_cast<T*>(b),
                    phys == DAMAGE ? L.exclD : nullptr, l - 1);
    rf = nullptr;
  }
  if (l == nlev - 1) {
    if (L.dense && nlev > 1) {
      coarse_solve<T>(st, nc * L.g.n, phys == ELASTIC ? B.AEi : B.ADi, b, x);
      return false;
    }
    smooth<T>(s, st, phys, l, b, x, true, nlev > 1 ? 8 * s.cdeg : deg, nullptr, dot_slot);
    return dot_slot >= 0;
  }
  Level& C = s.lv[l + 1];
  LevelBuf<T>& BC = C.buf<T>();
  if (dl == 1) {  // the one pre-smoothing step from zero is pointwise: formed by the residual
    double c0, r0;
    cheb_coefs(1, &c0, &r0);
    residual_op<T>(s, st, phys, l, b, x, B.r, r0);
  } else {
    smooth<T>(s, st, phys, l, b, x, true, dl);
    residual_op<T>(s, st, phys, l, b, x, B.r);
  }
  vcycle<T>(s, st, phys, l + 1, BC.b, BC.x, deg, -1, B.r);
  // prolongation x += P x_c fused into the first post-smoothing step
  smooth<T>(s, st, phys, l, b, x, false, dl, BC.x, dot_slot);
  return dot_slot >= 0;
}

// z = M r; with dot_slot >= 0, also r . z into that slot, computed by the preconditioner's last
// level-0 kernel when it can (returns true) -- otherwise the caller reduces it itself
template <class T>
bool precond(pf_sim& s, cudaStream_t st, int phys, const T* r, T* z, int deg, int dot_slot = -1) {
  if (s.nl_active == 1) {
    // single level: Chebyshev smoother alone
    smooth<T>(s, st, phys, 0, r, z, true, deg, nullptr, dot_slot);
    return dot_slot >= 0;
  }
  return vcycle<T>(s, st, phys, 0, r, z, deg, dot_slot);
}
// z = M r and r . z into the slot, fused when the preconditioner allows it
template <class T>
void precond_dot(pf_sim& s, cudaStream_t st, int phys, const T* r, T* z, int deg, size_t nd,
                 int dot_slot) {
  if (!precond<T>(s, st, phys, r, z, deg, dot_slot)) vec_dot<T>(st, r, z, nd, slot(s, dot_slot));
}

// set up the coefficients, l1 diagonals and the coarsest factorization of one operator
template <class T>
void setup_elastic(pf_sim& s, cudaStream_t st) {
  const int nlev = (int)s.lv.size();
  elastic_coef<T>(st, s.lv[0].g, s.m, alpha_of<T>(s), s.lv[0].buf<T>().coefE);
  for (int l = 1; l < nlev; ++l)
    coarsen_coef<T>(st, s.lv[l - 1].g, s.lv[l].g, s.lv[l - 1].buf<T>().coefE, s.lv[l].buf<T>().coefE);
  for (int l = 0; l < nlev; ++l)
    l1_dinv_elastic<T>(st, s.lv[l].g, s.m, s.lv[l].buf<T>().coefE, s.lv[l].buf<T>().dinvE);
  Level& Lc = s.lv[nlev - 1];
  if (Lc.dense && nlev > 1) {
    LevelBuf<T>& B = Lc.buf<T>();
    coarse_assemble<T>(st, Lc.g, s.m, ELASTIC, B.coefE, B.AE, B.diagE, nullptr);
    coarse_factor_invert<T>(st, 2 * Lc.g.n, B.AE, B.diagE, B.AEi);
  }
}

template <class T>
void setup_damage(pf_sim& s, cudaStream_t st) {
  const int nlev = (int)s.lv.size();
  for (int l = 1; l < nlev; ++l)
    coarsen_coef<T>(st, s.lv[l - 1].g, s.lv[l].g, s.lv[l - 1].buf<T>().wD, s.lv[l].buf<T>().wD);
  for (int l = 0; l < nlev; ++l)
    l1_dinv_damage<T>(st, s.lv[l].g, s.m, s.lv[l].buf<T>().wD, s.lv[l].buf<T>().dinvD);
}

// The active set changed: coarse-level masks (a coarse node is excluded iff its coincident fine
// node is) and the coarsest level's dense inverse of the masked operator.
template <class T>
void damage_masks(pf_sim& s, cudaStream_t st) {
  const int nlev = (int)s.lv.size();
  for (int l = 1; l < nlev; ++l)
    mask_restrict(st, s.lv[l - 1].g, s.lv[l].g, l == 1 ? s.act : s.lv[l - 1].exclD, s.lv[l].exclD);
  Level& Lc = s.lv[nlev - 1];
  if (Lc.dense && nlev > 1) {
    LevelBuf<T>& B = Lc.buf<T>();
    coarse_assemble<T>(st, Lc.g, s.m, DAMAGE, B.wD, B.AD, B.diagD, Lc.exclD);
    coarse_factor_invert<T>(st, Lc.g.n, B.AD, B.diagD, B.ADi);
  }
}

// Preconditioned CG for A_ff x = b (x starts at 0).  Stops when ||r|| <= rtol ||b||.
// Host-driven loop: one read-back of ||r||^2 per iteration.
template <class T>
pf_status pcg_host(pf_sim& s, cudaStream_t st, int phys, const T* b, int maxit, double rtol,
                   int deg, int64_t* iters, double* relres) {
  Krylov<T>& K = kry<T>(s);
  const int nc = phys == ELASTIC ? 2 : 1;
  const size_t nd = (size_t)nc * s.lv[0].g.n;
  vec_fill<T>(st, K.x, T(0), nd);
  CU(cudaMemcpyAsync(K.r, b, nd * sizeof(T), cudaMemcpyDeviceToDevice, st));
  vec_dot<T>(st, K.r, K.r, nd, slot(s, S_RR));
  double rr0;
  TRY(read_scalars(s, st, S_RR, 1, &rr0));
  if (!(rr0 == rr0) || isinf(rr0)) return fail(PF_ENUMERIC, "CG: right-hand side is not finite");
  if (relres) *relres = 0.0;
  if (rr0 == 0.0) return PF_OK;
  const double tol2 = rtol * rtol * rr0;
  precond_dot<T>(s, st, phys, K.r, K.z, deg, nd, S_RZ0);
  cg_update_p<T>(st, K.p, K.z, nd, nullptr, nullptr);
  int cur = 0;
  double rr = rr0;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    apply_op<T>(s, st, phys, 0, K.p, K.Ap, true, S_PAP);
    cg_update_xr<T>(st, K.x, K.r, K.p, K.Ap, nd, s.scal + (cur ? S_RZ1 : S_RZ0), s.scal + S_PAP,
                    slot(s, S_RR));
    TRY(read_scalars(s, st, S_RR, 1, &rr));
    if (!(rr == rr)) return fail(PF_ENUMERIC, "CG breakdown (NaN residual)");
    if (rr <= tol2) break;
    precond_dot<T>(s, st, phys, K.r, K.z, deg, nd, cur ? S_RZ0 : S_RZ1);
    cg_update_p<T>(st, K.p, K.z, nd, s.scal + (cur ? S_RZ0 : S_RZ1), s.scal + (cur ? S_RZ1 : S_RZ0));
    cur ^= 1;
  }
  if (iters) *iters += std::min(it, maxit);
  if (relres) *relres = sqrt(rr / rr0);
  if (it > maxit) return fail(PF_ENOTCONV, "CG did not converge in %d iterations (rel. res. %.3e)",
                              maxit, sqrt(rr / rr0));
  return PF_OK;
}

// One CG iteration body, in the order: z = M r; rz_new = r.z; p = z + (rz_new/rz_old) p;
// Ap, pAp; x += a p, r -= a Ap, rr; control (rz_old <- rz_new, loop while rr > tol2).
template <class T>
pf_status build_cg_graph(pf_sim& s, int phys, int deg) {
  const int pi = sizeof(T) == 8 ? 1 : 0;
  const int degkey = deg * 1000 + s.cdeg;
  if (s.cg_exec[phys][pi] && s.cg_deg[phys][pi] == degkey && s.cg_nl[phys][pi] == s.nl_active &&
      s.cg_tail[phys][pi] == (int)s.use_tail && s.cg_tiles[phys][pi] == s.tile_fine * 100 + s.tile_coarse)
    return PF_OK;
  if (s.cg_exec[phys][pi]) {
    cudaGraphExecDestroy(s.cg_exec[phys][pi]);
    cudaGraphDestroy(s.cg_graph[phys][pi]);
    s.cg_exec[phys][pi] = nullptr;
    s.cg_graph[phys][pi] = nullptr;
  }
  Krylov<T>& K = kry<T>(s);
  const size_t nd = (size_t)(phys == ELASTIC ? 2 : 1) * s.lv[0].g.n;
  // the graph and the capture stream are released on every early return
  struct Owned {
    cudaGraph_t g = nullptr;
    cudaStream_t cs = nullptr;
    ~Owned() {
      if (cs) cudaStreamDestroy(cs);
      if (g) cudaGraphDestroy(g);
    }
  } own;
  cudaGraph_t g;
  CU(cudaGraphCreate(&g, 0));
  own.g = g;
  cudaGraphConditionalHandle h;
  CU(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  CU(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t cs;
  CU(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  own.cs = cs;
  CU(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  prof_set_capturing(true);
  precond_dot<T>(s, cs, phys, K.r, K.z, deg, nd, S_RZ1);
  cg_update_p<T>(cs, K.p, K.z, nd, s.scal + S_RZ1, s.scal + S_RZ0);
  apply_op<T>(s, cs, phys, 0, K.p, K.Ap, true, S_PAP);
  cg_update_xr<T>(cs, K.x, K.r, K.p, K.Ap, nd, s.scal + S_RZ1, s.scal + S_PAP, slot(s, S_RR));
  cg_control(cs, h, s.scal + S_RZ1, s.scal + S_RZ0, s.scal + S_RR, s.scal + S_TOL2, s.scal + S_IT,
             s.scal + S_MAXIT);
  const int64_t nk = prof_captured();
  prof_set_capturing(false);
  cudaGraph_t captured;
  cudaError_t e1 = cudaStreamEndCapture(cs, &captured);
  cudaError_t e2 = cudaStreamDestroy(cs);
  own.cs = nullptr;
  if (e1 != cudaSuccess || e2 != cudaSuccess)
    return fail(PF_ECUDA, "CG graph capture failed: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
  cudaGraphExec_t ex;
  cudaError_t e3 = cudaGraphInstantiate(&ex, g, 0);
  if (e3 != cudaSuccess)
    return fail(PF_ECUDA, "CG graph instantiation failed: %s", cudaGetErrorString(e3));
  own.g = nullptr;  // kept by the sim
  s.cg_graph[phys][pi] = g;
  s.cg_exec[phys][pi] = ex;
  s.cg_body_kernels[phys][pi] = (int)nk;
  s.cg_deg[phys][pi] = degkey;
  s.cg_nl[phys][pi] = s.nl_active;
  s.cg_tail[phys][pi] = (int)s.use_tail;
  s.cg_tiles[phys][pi] = s.tile_fine * 100 + s.tile_coarse;
  return PF_OK;
}

// Same solve as pcg_host with the whole iteration loop inside one CUDA graph launch.
template <class T>
pf_status pcg_graph(pf_sim& s, cudaStream_t st, int phys, const T* b, int maxit, double rtol,
                    int deg, int64_t* iters, double* relres) {
  Krylov<T>& K = kry<T>(s);
  const size_t nd = (size_t)(phys == ELASTIC ? 2 : 1) * s.lv[0].g.n;
  const int pi = sizeof(T) == 8 ? 1 : 0;
  TRY(build_cg_graph<T>(s, phys, deg));
  vec_fill<T>(st, K.x, T(0), nd);
  CU(cudaMemcpyAsync(K.r, b, nd * sizeof(T), cudaMemcpyDeviceToDevice, st));
  vec_dot<T>(st, K.r, K.r, nd, slot(s, S_RR));
  double rr0;
  TRY(read_scalars(s, st, S_RR, 1, &rr0));
  if (!(rr0 == rr0) || isinf(rr0)) return fail(PF_ENUMERIC, "CG: right-hand side is not finite");
  if (relres) *relres = 0.0;
  if (rr0 == 0.0) return PF_OK;
  const double tol2 = rtol * rtol * rr0;
  double* hb = s.host;
  hb[0] = tol2;
  hb[1] = 0.0;
  hb[2] = double(maxit);
  CU(cudaMemcpyAsync(s.scal + S_TOL2, hb, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
  CU(cudaMemsetAsync(s.scal + S_RZ0, 0, sizeof(double), st));
  CU(cudaGraphLaunch(s.cg_exec[phys][pi], st));
  double rr, it;
  TRY(read_scalars(s, st, S_RR, 1, &rr));
  TRY(read_scalars(s, st, S_IT, 1, &it));
  prof_add_launches((int64_t)it * s.cg_body_kernels[phys][pi]);
  if (!(rr == rr)) return fail(PF_ENUMERIC, "CG breakdown (NaN residual)");
  if (iters) *iters += (int64_t)it;
  if (relres) *relres = sqrt(rr / rr0);
  if (rr > tol2) return fail(PF_ENOTCONV, "CG did not converge in %d iterations (rel. res. %.3e)",
                             maxit, sqrt(rr / rr0));
  return PF_OK;
}

template <class T>
pf_status pcg(pf_sim& s, cudaStream_t st, int phys, const T* b, int maxit, double rtol, int deg,
              int64_t* iters, double* relres) {
  if (s.use_graphs) return pcg_graph<T>(s, st, phys, b, maxit, rtol, deg, iters, relres);
  return pcg_host<T>(s, st, phys, b, maxit, rtol, deg, iters, relres);
}

// ---------------------------------------------------------------------------------------------
// load, eigenstrain, physical residual
// ---------------------------------------------------------------------------------------------
pf_status set_load(pf_sim& s, double t, double dT, cudaStream_t st) {
  s.t = t;
  s.dT = dT;
  const Grid& g = s.lv[0].g;
  s.lift.mu = s.m.mu;  // material constants of the Mode-I boundary field
  s.lift.kappa = s.mat_in.plane == PF_PLANE_STRESS ? (3.0 - s.mat_in.nu) / (1.0 + s.mat_in.nu)
                                                   : 3.0 - 4.0 * s.mat_in.nu;
  lift_u(st, g, s.u, t, s.lift);
  s.thermal = s.m.model && s.mat_in.beta != 0.0 && dT != 0.0;
  if (s.thermal) {
    int NE = elems_per_cell(g.kind);
    std::vector<double> tab((size_t)g.ny * NE);
    for (int j = 0; j < g.ny; ++j)
      for (int t2 = 0; t2 < NE; ++t2) {
        double y = (j + centroid_fy(g.kind, t2)) * g.hy;
        tab[(size_t)j * NE + t2] = s.mat_in.beta * (-dT * erfc(y / s.mat_in.pen));
      }
    CU(cudaMemcpyAsync(s.eig, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    vec_convert<float, double>(st, s.eig32, s.eig, tab.size());
    CU(cudaStreamSynchronize(st));
  }
  CU(cudaGetLastError());
  s.elastic_ready64 = s.elastic_ready32 = s.xu_valid = false;
  return PF_OK;
}

// r = f - K(alpha) u on free dofs (FP64); returns ||r||
pf_status physical_residual(pf_sim& s, cudaStream_t st, const double* u, double* r, double* nrm) {
  ElasticArgs<double> a{};
  a.x = u;
  a.alpha = s.alpha;
  a.eig = s.eig;
  a.y = r;
  a.slot = slot(s, S_RES);
  a.df = s.df;
  launch_elastic<double>(st, s.lv[0].g, s.m, COEF_ALPHA, M_RESID, s.thermal, false, a);
  double v;
  TRY(read_scalars(s, st, S_RES, 1, &v));
  *nrm = sqrt(v);
  return PF_OK;
}

// ---------------------------------------------------------------------------------------------
// u-subproblem: FP64 residual with FP64 PCG (PF_FP64) or FP32 PCG (PF_MIXED) corrections
// ---------------------------------------------------------------------------------------------
pf_status u_solve(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, pf_step_report* rep) {
  const Grid& g = s.lv[0].g;
  const size_t n2 = 2 * (size_t)g.n;
  const bool mixed = o.precision == PF_MIXED;
  if (mixed ? !s.elastic_ready32 : !s.elastic_ready64) {
    if (mixed) setup_elastic<float>(s, st);
    else setup_elastic<double>(s, st);
    (mixed ? s.elastic_ready32 : s.elastic_ready64) = true;
  }
  CU(cudaMemcpyAsync(s.xu, s.u, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double rn;
  TRY(physical_residual(s, st, s.xu, s.r64, &rn));
  s.r_scale = std::max(s.r_scale, rn);
  const double tol = o.u_rtol * s.r_scale;
  for (int outer = 0; outer < 60; ++outer) {
    if (rn <= tol || rn == 0.0) return PF_OK;
    if (!(rn == rn)) return fail(PF_ENUMERIC, "u-subproblem residual is NaN");
    if (rep) rep->outer_refinements++;
    if (!mixed) {
      double rel = std::max(tol / rn, 1e-15);
      pf_status stt = pcg<double>(s, st, ELASTIC, s.r64, o.cg_maxit, rel, o.mg_degree,
                                  rep ? &rep->cg_iters_u : nullptr, nullptr);
      if (stt != PF_OK && stt != PF_ENOTCONV) return stt;
      vec_add<double>(st, s.xu, s.k64.x, n2);
    } else {
      vec_convert<float, double>(st, s.tmp32, s.r64, n2);
      // do not reduce the residual further than the outer target needs
      const double rel = std::min(0.5, std::max(o.inner_rtol, 0.5 * tol / rn));
      pf_status stt = pcg<float>(s, st, ELASTIC, s.tmp32, o.cg_maxit, rel, o.mg_degree,
                                 rep ? &rep->cg_iters_u : nullptr, nullptr);
      if (stt != PF_OK && stt != PF_ENOTCONV) return stt;
      vec_add_f32_to_f64(st, s.xu, s.k32.x, n2);
    }
    TRY(physical_residual(s, st, s.xu, s.r64, &rn));
  }
  if (rn <= tol || rn == 0.0) return PF_OK;
  return fail(PF_ENOTCONV, "u-subproblem: residual %.3e above tolerance %.3e", rn, tol);
}

// ---------------------------------------------------------------------------------------------
// damage subproblem: Algorithm 4 on the box [alpha_prev, 1]
// ---------------------------------------------------------------------------------------------
// out[0] = ||Phi||^2, out[1] = ||F_N||^2
pf_status grad_at(pf_sim& s, cudaStream_t st, const double* x, double zeta, double* F, double* Phi,
                  double* rhs, uint8_t* act, double out[2]) {
  DamageArgs<double> a{};
  a.x = x;
  a.w = s.q;
  a.lo = s.alpha_prev;
  a.zeta = zeta;
  a.y = F;
  a.dout = Phi;
  a.rhs = rhs;
  a.act = act;
  a.slot = slot(s, S_PHI);
  a.df = s.df;
  launch_damage<double>(st, s.lv[0].g, s.m, M_GRAD, false, a);
  return read_scalars(s, st, S_PHI, 2, out);
}

pf_status trial_at(pf_sim& s, cudaStream_t st, const double* x, const double* d, double mu,
                   double zeta, double out[2]) {
  DamageArgs<double> a{};
  a.x = x;
  a.d = d;
  a.cd = mu;
  a.w = s.q;
  a.lo = s.alpha_prev;
  a.zeta = zeta;
  a.y = s.Ftr;
  a.dout = s.Phitr;
  a.rhs = s.rhstr;
  a.act = s.acttr;
  a.xt = s.xtr;
  a.slot = slot(s, S_PHI);
  a.df = s.df;
  launch_damage<double>(st, s.lv[0].g, s.m, M_TRIAL, false, a);
  return read_scalars(s, st, S_PHI, 2, out);
}

void damage_prepare(pf_sim& s, cudaStream_t st, bool mixed) {
  const Grid& g = s.lv[0].g;
  damage_q(st, g, s.m, s.u, s.thermal ? s.eig : nullptr, s.q, s.lv[0].f64.wD,
           mixed ? s.lv[0].f32.wD : nullptr, s.df);
  if (mixed) setup_damage<float>(s, st);
  else setup_damage<double>(s, st);
}

pf_status alpha_solve(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, pf_step_report* rep) {
  const Grid& g = s.lv[0].g;
  const size_t n = g.n;
  const bool mixed = o.precision == PF_MIXED;
  damage_prepare(s, st, mixed);
  CU(cudaMemcpyAsync(s.xrs, s.alpha, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double v[2];
  TRY(grad_at(s, st, s.xrs, o.zeta, s.F, s.Phi, s.rhs, s.act, v));
  double phi2 = v[0];
  double phi0 = sqrt(phi2);
  s.phi_scale = std::max(s.phi_scale, phi0);
  // relative to the largest ||Phi|| of the load step, and to the size of the gradient's terms:
  // at a load at the AT1 damage threshold the linear term (c3 - q_T) |T| / 3 cancels, and what is
  // left of F is the error the u-subproblem's tolerance leaves in q (its largest ||Phi|| is then
  // no scale).  The terms' size per node is about (c3 + q_T + c2) |T| / 3 over the node's (up
  // to 8) elements, with q_T ~ c3 at the threshold.
  const double term = 8.0 * g.area * (2.0 * s.m.c3 + s.m.c2) / 3.0;
  const double tol = o.rs_rtol * std::max(s.phi_scale, sqrt(double(n)) * term);
  const double c_armijo = 1e-4;
  int it = 0;
  for (;;) {
    double phi = sqrt(phi2);
    if (!(phi == phi)) return fail(PF_ENUMERIC, "damage residual is NaN");
    if (phi <= tol || phi2 == 0.0) break;
    if (it >= o.rs_maxit) {
      if (rep) rep->rs_iters += it;
      return fail(PF_ENOTCONV, "damage solve: %d iterations, ||Phi|| %.3e > %.3e", it, phi, tol);
    }
    ++it;
    // reduced Newton step on the inactive set: H_NN d_N = -F_N, d_A = 0 (eq. reducednewton)
    if (mixed) damage_masks<float>(s, st);
    else damage_masks<double>(s, st);
    // inexact Newton: solve only as accurately as the termination test of Algorithm 4 needs
    const double cg_rel = std::min(0.5, std::max(o.alpha_cg_rtol, 0.5 * tol / phi));
    int64_t cg_its = 0;
    double cg_res = 0.0;
    if (!mixed) {
      pf_status stt = pcg<double>(s, st, DAMAGE, s.rhs, o.cg_maxit, cg_rel, o.mg_degree,
                                  &cg_its, &cg_res);
      if (stt != PF_OK && stt != PF_ENOTCONV) return stt;
      CU(cudaMemcpyAsync(s.drs, s.k64.x, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else {
      vec_convert<float, double>(st, s.tmp32, s.rhs, n);
      pf_status stt = pcg<float>(s, st, DAMAGE, s.tmp32, o.cg_maxit, cg_rel, o.mg_degree,
                                 &cg_its, &cg_res);
      if (stt != PF_OK && stt != PF_ENOTCONV) return stt;
      vec_convert<double, float>(st, s.drs, s.k32.x, n);
    }
    snap_active(st, g, s.act, s.xrs, s.alpha_prev, s.drs);
    // projected line search on ||Phi||^2; steepest descent of the merit function if it fails
    bool accepted = false;
    for (int dir = 0; dir < 2 && !accepted; ++dir) {
      if (dir == 1) {
        merit_parts(st, g, s.xrs, s.F, s.alpha_prev, s.tmpa, s.tmpb);
        DamageArgs<double> a{};
        a.x = s.tmpa;
        a.w = s.lv[0].f64.wD;
        a.y = s.tmpa + n;
        launch_damage<double>(st, g, s.m, M_APPLY, false, a);
        merit_direction(st, n, s.tmpb, s.tmpa + n, s.drs);
      }
      for (double mu = 1.0; mu >= 0x1p-20; mu *= 0.5) {
        double w[2];
        TRY(trial_at(s, st, s.xrs, s.drs, mu, o.zeta, w));
        if (w[0] <= (1.0 - 2.0 * c_armijo * mu) * phi2) {
          std::swap(s.xrs, s.xtr);
          std::swap(s.F, s.Ftr);
          std::swap(s.Phi, s.Phitr);
          std::swap(s.rhs, s.rhstr);
          // the active flags stay in place: CUDA graphs of the damage PCG read this buffer
          CU(cudaMemcpyAsync(s.act, s.acttr, n, cudaMemcpyDeviceToDevice, st));
          phi2 = w[0];
          v[1] = w[1];
          accepted = true;
          break;
        }
      }
    }
    if (rep) rep->cg_iters_alpha += cg_its;
    if (debug_enabled())
      fprintf(stderr, "[pf] rs %d phi %.4e -> %.4e tol %.2e |F_N| %.3e cg %lld (rel %.1e, reached %.1e) %s\n",
              it, phi, sqrt(phi2), tol, sqrt(v[1]), (long long)cg_its, cg_rel, cg_res,
              accepted ? "accepted" : "line search failed");
    if (!accepted) {
      if (rep) rep->rs_iters += it;
      return fail(PF_ENOTCONV, "damage solve: line search failed at ||Phi|| %.3e", phi);
    }
  }
  if (rep) rep->rs_iters += it;
  return PF_OK;
}

// first candidate of omega, (1+omega)/2, ... not above the largest feasible step (Section 2.1)
double choose_omega_bar(double omega, double wstar) {
  if (omega <= 1.0) return omega;
  double w = omega;
  for (int k = 0; k <= 30; ++k) {
    if (w <= wstar) return w;
    w = 0.5 * (1.0 + w);
  }
  return 1.0;
}

pf_status energy_now(pf_sim& s, cudaStream_t st, double out[3]) {
  energy(st, s.lv[0].g, s.m, s.u, s.alpha, s.thermal ? s.eig : nullptr, slot(s, S_EN));
  double v[2];
  TRY(read_scalars(s, st, S_EN, 2, v));
  out[0] = v[0];
  out[1] = v[1];
  out[2] = v[0] + v[1];
  return PF_OK;
}

pf_status full_residual(pf_sim& s, cudaStream_t st, double zeta, double* nrm) {
  double rn;
  TRY(physical_residual(s, st, s.u, s.r64, &rn));
  damage_q(st, s.lv[0].g, s.m, s.u, s.thermal ? s.eig : nullptr, s.q, nullptr, nullptr, s.df);
  double v[2];
  TRY(grad_at(s, st, s.alpha, zeta, s.Ftr, s.Phitr, s.rhstr, s.acttr, v));
  *nrm = sqrt(rn * rn + v[0]);
  return PF_OK;
}

pf_status begin_step(pf_sim& s, cudaStream_t st, const pf_load& L) {
  const size_t n = s.lv[0].g.n;
  CU(cudaMemcpyAsync(s.alpha_prev, s.alpha, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  TRY(set_load(s, L.t, L.dT, st));
  s.r_scale = 0.0;
  s.phi_scale = 0.0;
  return PF_OK;
}

// One pass of the loop of Algorithm 2 (Algorithm 1 when omega = 1): returns the damage change
// max|alpha^k - alpha^{k-1}| and the relative displacement change.
pf_status oram_iteration(pf_sim& s, cudaStream_t st, const pf_solver_opts& oin,
                         pf_step_report* rep, double omega, double da_prev, double* da_out,
                         double* durel_out, bool* sub_ok) {
  const Grid& g = s.lv[0].g;
  const size_t n2 = 2 * (size_t)g.n;
  // inexact subproblem solves: tolerances follow the last damage change
  pf_solver_opts o = oin;
  if (oin.am_forcing > 0.0) {
    const double f = std::min(oin.am_forcing_max, oin.am_forcing * da_prev);
    o.u_rtol = std::max(oin.u_rtol, f);
    o.rs_rtol = std::max(oin.rs_rtol, f);
  }
  // u-subproblem (Algorithm 2, first line of the loop).  If neither alpha nor the load has
  // changed since the last solve, K(alpha) and the right-hand side are bitwise the same and
  // so is the minimizer u~: it is reused.
  if (!(s.xu_valid && s.xu_precision == o.precision)) {
    pf_status st1 = u_solve(s, st, o, rep);
    if (st1 != PF_OK && st1 != PF_ENOTCONV) return st1;
    s.xu_valid = st1 == PF_OK;
    s.xu_precision = o.precision;
    if (st1 == PF_ENOTCONV) {
      *sub_ok = false;
      if (rep) rep->u_notconv++;
    }
  } else if (rep) {
    rep->u_solves_reused++;
  }
  relax_u(st, s.u, s.xu, omega, n2, slot(s, S_DU));
  double du[2];
  TRY(read_scalars(s, st, S_DU, 2, du));
  pf_status st2 = alpha_solve(s, st, o, rep);
  if (st2 != PF_OK && st2 != PF_ENOTCONV) return st2;
  if (st2 == PF_ENOTCONV) {
    *sub_ok = false;
    if (rep) rep->alpha_notconv++;
  }
  omega_star(st, g, s.alpha, s.xrs, s.alpha_prev, slot(s, S_OMEGA));
  double ms;
  TRY(read_scalars(s, st, S_OMEGA, 1, &ms));
  double wbar = oin.omega_rule == 1 ? omega : choose_omega_bar(omega, -ms);
  relax_alpha(st, g, s.alpha, s.xrs, s.alpha_prev, wbar, s.alpha32, slot(s, S_DALPHA));
  double da;
  TRY(read_scalars(s, st, S_DALPHA, 1, &da));
  if (da > 0.0) s.elastic_ready64 = s.elastic_ready32 = s.xu_valid = false;
  *da_out = da;
  *durel_out = du[1] > 0.0 ? du[0] / du[1] : du[0];
  if (rep) rep->omega_bar_min = std::min(rep->omega_bar_min, wbar);
  if (trace_enabled())
    fprintf(stderr, "[pf-am] da %.3e du %.3e wbar %.4f cg_u %lld cg_a %lld rs %d\n", da,
            *durel_out, wbar, rep ? (long long)rep->cg_iters_u : 0LL,
            rep ? (long long)rep->cg_iters_alpha : 0LL, rep ? rep->rs_iters : 0);
  return PF_OK;
}

// Automated omega: the optimum of two-block SOR, 2 / (1 + sqrt(1 - mu^2)), with the Jacobi
// eigenvalue mu^2 recovered from the contraction rho observed at the current omega through
// (rho + omega - 1)^2 = rho omega^2 mu^2; clamped to [1, omega_max].
constexpr int OMEGA_PERIOD = 5;
double omega_update(double rho, double omega, double omega_max) {
  if (!(rho > 0.0 && rho < 1.0)) return omega;
  const double mu2 = (rho + omega - 1.0) * (rho + omega - 1.0) / (rho * omega * omega);
  if (!(mu2 >= 0.0 && mu2 < 1.0)) return omega;
  return std::min(omega_max, std::max(1.0, 2.0 / (1.0 + sqrt(1.0 - mu2))));
}

pf_status oram_step(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, pf_step_report* rep) {
  double omega = o.algo == PF_ALGO_AM ? 1.0 : o.omega;
  const bool adapt = o.omega_auto && o.algo != PF_ALGO_AM;
  double da_prev = HUGE_VAL;
  double da_hist[OMEGA_PERIOD + 1] = {};  // da of iterations k - OMEGA_PERIOD .. k (ring)
  for (int k = 1; k <= o.am_maxit; ++k) {
    double da, durel;
    bool sub_ok = true;
    TRY(oram_iteration(s, st, o, rep, omega, da_prev, &da, &durel, &sub_ok));
    if (rep) rep->omega_final = omega;
    da_hist[k % (OMEGA_PERIOD + 1)] = da;
    if (adapt && k % OMEGA_PERIOD == 0 && k > OMEGA_PERIOD) {
      const double prev = da_hist[(k - OMEGA_PERIOD) % (OMEGA_PERIOD + 1)];
      if (prev > 0.0 && da > 0.0) omega = omega_update(pow(da / prev, 1.0 / OMEGA_PERIOD), omega,
                                                       o.omega_max);
    }
    // with inexact solves a small change may only mean a loose solve did not move the state:
    // the test counts only for an iteration run at (nearly) the exact tolerances, i.e. one
    // whose predecessor already met the damage-change criterion
    const bool exact = o.am_forcing <= 0.0 || da_prev <= o.am_tol;
    da_prev = da;
    if (rep) {
      rep->am_iters = k;
      rep->dalpha_inf = da;
      rep->du_rel = durel;
    }
    // the stopping test is accepted only after an iteration whose subproblems both converged
    if (exact && sub_ok && da <= o.am_tol && durel <= o.am_tol) return PF_OK;
  }
  return fail(PF_ENOTCONV, "alternate minimization: %d iterations, |dalpha| %.3e", o.am_maxit,
              rep ? rep->dalpha_inf : -1.0);
}

// ---------------------------------------------------------------------------------------------
// ORAM-N (Algorithm 3): ORAM until the optimality residual has dropped by switch_tol, then the
// reduced-space active-set Newton method (Algorithm 4) on the coupled system (u, alpha), whose
// reduced Jacobian J_NN = [[A, B], [B^T, C]] (Section 3.3, eq. inactjac) is solved by MINRES
// with the block preconditioner of eq. preconditioner (S ~ C), each inverse action approximated
// by two multigrid V-cycles.  The Krylov solve runs in FP32; residuals, line search and active
// set in FP64.
// ---------------------------------------------------------------------------------------------
inline float* upart(float* x) { return x; }
inline float* apart(pf_sim& s, float* x) { return x + 2 * (size_t)s.lv[0].g.n; }

// y = J_NN x: y_u = K x_u + B x_a, y_a = B^T x_u + H_NN x_a (masks: fixed u dofs, active alpha)
void jac_apply(pf_sim& s, cudaStream_t st, float* x, float* y) {
  const Grid& g = s.lv[0].g;
  apply_op<float>(s, st, ELASTIC, 0, upart(x), upart(y), false, S_TMP);
  apply_op<float>(s, st, DAMAGE, 0, apart(s, x), apart(s, y), false, S_TMP);
  CouplingArgs<float> b{};
  b.u = s.u32;
  b.alpha = s.alpha32;
  b.eig = s.thermal ? s.eig32 : nullptr;
  b.excl = s.act;
  b.accumulate = 1;
  b.x = apart(s, x);
  b.y = upart(y);
  launch_coupling<float>(st, g, s.m, false, b);
  b.x = upart(x);
  b.y = apart(s, y);
  launch_coupling<float>(st, g, s.m, true, b);
}

// two V-cycles of the operator's multigrid: x = V r; x += V (r - A x)
void two_vcycles(pf_sim& s, cudaStream_t st, int phys, float* r, float* x, float* t, float* e,
                 int deg) {
  const size_t nd = (size_t)(phys == ELASTIC ? 2 : 1) * s.lv[0].g.n;
  precond<float>(s, st, phys, r, x, deg);
  residual_op<float>(s, st, phys, 0, r, x, t);
  precond<float>(s, st, phys, t, e, deg);
  vec_add<float>(st, x, e, nd);
}

// z = P^{-1} r, eq. preconditioner: y1 = A^-1 r_u; z_a = C^-1 (r_a - B^T y1); z_u = A^-1 (r_u - B z_a)
void block_prec(pf_sim& s, cudaStream_t st, float* r, float* z, int deg) {
  const Grid& g = s.lv[0].g;
  const size_t n = g.n;
  float *y1 = s.nv[8], *t = s.nv[9], *e = s.nv[10], *w = s.nv[11];
  two_vcycles(s, st, ELASTIC, upart(r), upart(y1), upart(t), upart(e), deg);
  CouplingArgs<float> b{};
  b.u = s.u32;
  b.alpha = s.alpha32;
  b.eig = s.thermal ? s.eig32 : nullptr;
  b.excl = s.act;
  b.accumulate = 0;
  b.x = upart(y1);
  b.y = apart(s, w);
  launch_coupling<float>(st, g, s.m, true, b);                            // w_a = B^T y1
  vec_lincomb<float>(st, apart(s, w), 1.f, apart(s, r), -1.f, apart(s, w), 0.f, n);  // r_a - w_a
  two_vcycles(s, st, DAMAGE, apart(s, w), apart(s, z), apart(s, t), apart(s, e), deg);
  b.x = apart(s, z);
  b.y = upart(w);
  launch_coupling<float>(st, g, s.m, false, b);                           // w_u = B z_a
  vec_lincomb<float>(st, upart(w), 1.f, upart(r), -1.f, upart(w), 0.f, 2 * n);  // r_u - w_u
  two_vcycles(s, st, ELASTIC, upart(w), upart(z), upart(t), upart(e), deg);
}

pf_status dot3(pf_sim& s, cudaStream_t st, const float* x, const float* y, double* out) {
  vec_dot<float>(st, x, y, 3 * (size_t)s.lv[0].g.n, slot(s, S_TMP));
  return read_scalars(s, st, S_TMP, 1, out);
}

// Preconditioned MINRES (Paige & Saunders) for J_NN x = b from x = 0 (x may be b's storage);
// stops when the preconditioned residual estimate drops below rtol times its initial value.
pf_status minres(pf_sim& s, cudaStream_t st, float* b, float* x, double rtol, int maxit, int deg,
                 int64_t* its) {
  const size_t N = 3 * (size_t)s.lv[0].g.n;
  float *r1 = s.nv[0], *r2 = s.nv[1], *y = s.nv[2], *v = s.nv[3], *w = s.nv[4], *w1 = s.nv[5],
        *w2 = s.nv[6];
  CU(cudaMemcpyAsync(r1, b, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  vec_fill<float>(st, x, 0.f, N);  // after the copy: x may share storage with b
  vec_fill<float>(st, w, 0.f, N);
  vec_fill<float>(st, w2, 0.f, N);
  block_prec(s, st, r1, y, deg);
  double beta1;
  TRY(dot3(s, st, r1, y, &beta1));
  // a preconditioner that is not positive definite in FP32 (near-singular crack band) gives no
  // Newton direction: reported as non-convergence, so that the caller falls back
  if (!(beta1 >= 0.0)) return fail(PF_ENOTCONV, "MINRES: preconditioner not positive definite");
  beta1 = sqrt(beta1);
  if (beta1 == 0.0) return PF_OK;
  CU(cudaMemcpyAsync(r2, r1, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
  double oldb = 0.0, beta = beta1, dbar = 0.0, epsln = 0.0, phibar = beta1, cs = -1.0, sn = 0.0;
  int it = 0;
  for (it = 1; it <= maxit; ++it) {
    const double sc = 1.0 / beta;
    vec_lincomb<float>(st, v, float(sc), y, 0.f, nullptr, 0.f, N);  // v = y / beta
    jac_apply(s, st, v, y);                                        // y = J v
    if (it >= 2) vec_lincomb<float>(st, y, 1.f, y, float(-beta / oldb), r1, 0.f, N);
    double alfa;
    TRY(dot3(s, st, v, y, &alfa));
    vec_lincomb<float>(st, y, 1.f, y, float(-alfa / beta), r2, 0.f, N);
    std::swap(r1, r2);  // r1 <- r2, r2 <- y (copied below)
    CU(cudaMemcpyAsync(r2, y, N * sizeof(float), cudaMemcpyDeviceToDevice, st));
    block_prec(s, st, r2, y, deg);
    oldb = beta;
    double bb;
    TRY(dot3(s, st, r2, y, &bb));
    if (!(bb >= 0.0)) return fail(PF_ENOTCONV, "MINRES: preconditioner not positive definite");
    beta = sqrt(bb);
    const double oldeps = epsln;
    const double delta = cs * dbar + sn * alfa;
    const double gbar = sn * dbar - cs * alfa;
    epsln = sn * beta;
    dbar = -cs * beta;
    const double gamma = std::max(hypot(gbar, beta), 1e-300);
    cs = gbar / gamma;
    sn = beta / gamma;
    const double phi = cs * phibar;
    phibar = sn * phibar;
    // w = (v - oldeps w1 - delta w2) / gamma with (w1, w2) <- (w2, w)
    std::swap(w1, w2);
    std::swap(w2, w);
    vec_lincomb<float>(st, w, float(1.0 / gamma), v, float(-oldeps / gamma), w1, 0.f, N);
    vec_lincomb<float>(st, w, 1.f, w, float(-delta / gamma), w2, 0.f, N);
    vec_lincomb<float>(st, x, float(phi), w, 0.f, nullptr, 1.f, N);
    if (phibar <= rtol * beta1 || beta == 0.0) break;
  }
  if (its) *its += std::min(it, maxit);
  return PF_OK;
}

// ||Phi|| of the coupled optimality system at the resident state; leaves F, Phi, act, rhs of
// the damage part in the sim's main buffers and r64 = -E_u.
pf_status coupled_residual(pf_sim& s, cudaStream_t st, double zeta, double* nrm) {
  double rn;
  TRY(physical_residual(s, st, s.u, s.r64, &rn));
  damage_q(st, s.lv[0].g, s.m, s.u, s.thermal ? s.eig : nullptr, s.q, s.lv[0].f64.wD,
           s.lv[0].f32.wD, s.df);
  double v[2];
  TRY(grad_at(s, st, s.alpha, zeta, s.F, s.Phi, s.rhs, s.act, v));
  *nrm = sqrt(rn * rn + v[0]);
  return PF_OK;
}

// Steepest-descent direction of ||Phi||^2 / 2 for the coupled system (the fallback of Algorithm
// 4 when the Newton search fails), at the state whose residuals coupled_residual left in r64
// (= -E_u on free dofs) and F (= E_alpha).  With Phi_u = E_u and the nested Fischer-Burmeister
// Phi_alpha, a generalized Jacobian is G = D + R J (D, R diagonal: 0 and 1 on displacement dofs,
// pa - pb qa and -pb qb on damage nodes; J = [[K, B], [B^T, H]] the Hessian of the energy on free
// displacement dofs and all damage nodes).  J is symmetric, so G^T Phi = D Phi + J (R Phi).
// Writes -G^T Phi into (du, da).  FP64 throughout.
void coupled_merit_direction(pf_sim& s, cudaStream_t st, double* du, double* da) {
  const Grid& g = s.lv[0].g;
  const size_t n = g.n, n2 = 2 * n;
  double *vu = s.tmpa, *va = s.xtr, *dga = s.Phitr, *hva = s.Ftr;
  vec_lincomb<double>(st, vu, -1.0, s.r64, 0.0, nullptr, 0.0, n2);  // R Phi on u: Phi_u = E_u
  merit_parts(st, g, s.alpha, s.F, s.alpha_prev, va, dga);          // R Phi and D Phi on alpha
  ElasticArgs<double> ea{};
  ea.x = vu;
  ea.alpha = s.alpha;
  ea.y = du;
  launch_elastic<double>(st, g, s.m, COEF_ALPHA, M_MASKED, false, false, ea);  // K_ff vu
  CouplingArgs<double> b{};
  b.u = s.u;
  b.alpha = s.alpha;
  b.eig = s.thermal ? s.eig : nullptr;
  b.excl = nullptr;
  b.accumulate = 1;
  b.x = va;
  b.y = du;
  launch_coupling<double>(st, g, s.m, false, b);  // + B va
  b.accumulate = 0;
  b.x = vu;
  b.y = da;
  launch_coupling<double>(st, g, s.m, true, b);  // B^T vu
  DamageArgs<double> dm{};
  dm.x = va;
  dm.w = s.lv[0].f64.wD;
  dm.y = hva;
  launch_damage<double>(st, g, s.m, M_APPLY, false, dm);  // H va
  vec_lincomb<double>(st, da, -1.0, hva, -1.0, dga, -1.0, n);
  vec_lincomb<double>(st, du, -1.0, du, 0.0, nullptr, 0.0, n2);
}

// Algorithm 4 on the coupled system: reduced Newton steps with a projected line search on
// ||Phi||^2.  Returns PF_OK when ||Phi|| <= tol, PF_ENOTCONV otherwise (state = best point).
pf_status newton_solve(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, pf_step_report* rep,
                       double tol, double* phi_out) {
  const Grid& g = s.lv[0].g;
  const size_t n = g.n, n2 = 2 * n;
  double phi;
  TRY(coupled_residual(s, st, o.zeta, &phi));
  for (int it = 0; it < o.newton_maxit; ++it) {
    *phi_out = phi;
    if (phi <= tol) return PF_OK;
    if (rep) rep->newton_iters++;
    // operators at the current state (FP32 inner solves)
    vec_convert<float, double>(st, s.u32, s.u, n2);
    setup_elastic<float>(s, st);
    setup_damage<float>(s, st);
    damage_masks<float>(s, st);
    // right-hand side -F_N = [r64 ; rhs]; the solution overwrites it
    float* xs = s.nv[7];
    vec_convert<float, double>(st, xs, s.r64, n2);
    vec_convert<float, double>(st, xs + n2, s.rhs, n);
    int64_t kits = 0;
    const pf_status ms = minres(s, st, xs, xs, o.minres_rtol, o.minres_maxit, o.mg_degree, &kits);
    if (ms != PF_OK && ms != PF_ENOTCONV) return ms;
    const bool have_newton = ms == PF_OK;  // else only the steepest-descent direction is tried
    if (rep) rep->krylov_iters_newton += kits;
    double mu_acc = 0.0;
    vec_convert<double, float>(st, s.ndu, xs, n2);
    vec_convert<double, float>(st, s.nda, xs + n2, n);
    snap_active(st, g, s.act, s.alpha, s.alpha_prev, s.nda);
    // projected line search (alpha clipped to its box; u unbounded) along the Newton direction,
    // then, if it fails, along the steepest-descent direction of ||Phi||^2 / 2
    CU(cudaMemcpyAsync(s.nu0, s.u, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(s.na0, s.alpha, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    bool accepted = false;
    int dir_acc = -1;
    const double phi2 = phi * phi;
    for (int dir = have_newton ? 0 : 1; dir < 2 && !accepted; ++dir) {
      if (dir == 1) {
        // residuals at the iteration's starting point, then the merit gradient there
        CU(cudaMemcpyAsync(s.u, s.nu0, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(s.alpha, s.na0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        double p0;
        TRY(coupled_residual(s, st, o.zeta, &p0));
        coupled_merit_direction(s, st, s.ndu, s.nda);
      }
      for (double mu = 1.0; mu >= 0x1p-20; mu *= 0.5) {
        newton_trial(st, g, s.u, s.nu0, s.ndu, s.alpha, s.na0, s.nda, s.alpha_prev, s.alpha32, mu);
        double pt;
        TRY(coupled_residual(s, st, o.zeta, &pt));
        if (pt * pt <= (1.0 - 2.0 * 1e-4 * mu) * phi2) {
          phi = pt;
          accepted = true;
          mu_acc = mu;
          dir_acc = dir;
          break;
        }
      }
    }
    if (accepted && dir_acc == 1 && rep) rep->newton_steepest++;
    if (trace_enabled())
      fprintf(stderr, "[pf-newton] it %d phi %.4e -> %.4e minres %lld mu %g %s\n", it,
              sqrt(phi2), phi, (long long)kits, mu_acc,
              accepted ? (dir_acc == 0 ? "newton" : "steepest") : "failed");
    s.elastic_ready64 = s.elastic_ready32 = s.xu_valid = false;
    if (!accepted) {  // restore this Newton iteration's starting point
      CU(cudaMemcpyAsync(s.u, s.nu0, n2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      CU(cudaMemcpyAsync(s.alpha, s.na0, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      vec_convert<float, double>(st, s.alpha32, s.alpha, n);
      TRY(coupled_residual(s, st, o.zeta, &phi));
      *phi_out = phi;
      return PF_ENOTCONV;
    }
  }
  *phi_out = phi;
  return phi <= tol ? PF_OK : PF_ENOTCONV;
}

pf_status oramn_step(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, pf_step_report* rep) {
  double phi_start;
  TRY(coupled_residual(s, st, o.zeta, &phi_start));
  const double tol = o.newton_rtol * phi_start;
  if (rep) rep->phi_start = phi_start;
  int oram_its = 0;
  const int max_outer = 50;
  double phi = phi_start;
  for (int outer = 0; outer < max_outer; ++outer) {
    double phi0;
    TRY(coupled_residual(s, st, o.zeta, &phi0));
    phi = phi0;
    if (phi0 <= tol) break;
    double da_prev = HUGE_VAL;
    if (trace_enabled())
      fprintf(stderr, "[pf-oramn] outer %d phi0 %.4e tol %.4e oram_its %d\n", outer, phi0, tol,
              oram_its);
    while (phi / phi0 > o.switch_tol && phi > tol && oram_its < o.am_maxit) {
      double da, durel;
      bool sub_ok = true;
      TRY(oram_iteration(s, st, o, rep, o.omega, da_prev, &da, &durel, &sub_ok));
      da_prev = da;
      ++oram_its;
      if (rep) rep->am_iters = oram_its;
      TRY(coupled_residual(s, st, o.zeta, &phi));
    }
    if (phi <= tol) break;
    pf_status ns = newton_solve(s, st, o, rep, tol, &phi);
    if (ns == PF_OK) break;
    if (ns != PF_ENOTCONV) return ns;
    if (oram_its >= o.am_maxit) break;
  }
  if (rep) rep->phi_norm = phi;
  return phi <= tol ? PF_OK : PF_ENOTCONV;
}

// ---------------------------------------------------------------------------------------------
// autotuner: smoother degrees and FP32 stencil tile heights, timed on whole PCG solves
// ---------------------------------------------------------------------------------------------
struct TuneCfg {
  int deg, cdeg, tf, tc;
};
struct TuneKey {
  int kind, nx, ny, prec;
  bool operator<(const TuneKey& o) const {
    if (kind != o.kind) return kind < o.kind;
    if (nx != o.nx) return nx < o.nx;
    if (ny != o.ny) return ny < o.ny;
    return prec < o.prec;
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneCfg> g_tune;

TuneKey tune_key(const pf_sim& s, int precision) {
  return TuneKey{s.desc.kind, s.desc.nx, s.desc.ny, precision};
}

// stencil tile heights of the sim's levels: tile_fine on level 0, tile_coarse below
void apply_tiles(pf_sim& s) {
  for (size_t l = 0; l < s.lv.size(); ++l) s.lv[l].g.tile_rows = l == 0 ? s.tile_fine : s.tile_coarse;
}

// the per-call solver settings that pf_load_step derives from the options
void apply_opts(pf_sim& s, const pf_solver_opts& o) {
  s.df = o.precision == PF_MIXED;
  s.use_graphs = o.use_graphs != 0;
  s.nl_active = o.mg_levels_max > 0 ? std::min<int>(o.mg_levels_max, (int)s.lv.size())
                                    : (int)s.lv.size();
  s.use_tail = o.mg_tail != 0;
  s.cdeg = o.mg_coarse_degree > 0 ? o.mg_coarse_degree : o.mg_degree;
}

// mean time of two PCG solves of K(alpha) x = b under configuration c (after one untimed solve
// that also captures the solve's graph)
template <class T>
pf_status time_pcg(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, const TuneCfg& c,
                   const T* b, double rtol, double* ms, int* its) {
  s.cdeg = c.cdeg;
  s.tile_fine = c.tf;
  s.tile_coarse = c.tc;
  apply_tiles(s);
  int64_t it0 = 0, it1 = 0;
  pf_status e = pcg<T>(s, st, ELASTIC, b, o.cg_maxit, rtol, c.deg, &it0, nullptr);
  if (e != PF_OK && e != PF_ENOTCONV) return e;
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(PF_ECUDA, "cudaEventCreate failed");
  }
  cudaEventRecord(e0, st);
  for (int r = 0; r < 2 && (e == PF_OK || e == PF_ENOTCONV); ++r)
    e = pcg<T>(s, st, ELASTIC, b, o.cg_maxit, rtol, c.deg, &it1, nullptr);
  cudaEventRecord(e1, st);
  cudaError_t se = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (se != cudaSuccess) return fail(PF_ECUDA, "tuning solve: %s", cudaGetErrorString(se));
  if (e != PF_OK && e != PF_ENOTCONV) return e;
  // a configuration whose solve does not converge is never chosen
  *ms = e == PF_OK ? 0.5 * t : HUGE_VAL;
  *its = (int)(it1 / 2);
  return PF_OK;
}

template <class T>
pf_status tune_t(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, TuneCfg* best,
                 pf_tune_report* rep) {
  const Grid& g = s.lv[0].g;
  const size_t n2 = 2 * (size_t)g.n;
  const bool mixed = std::is_same<T, float>::value;
  setup_elastic<T>(s, st);
  (mixed ? s.elastic_ready32 : s.elastic_ready64) = true;
  T *v, *b;
  if constexpr (std::is_same<T, float>::value) {
    v = s.nv[0];
    b = s.tmp32;
  } else {
    v = s.tmpb;
    b = s.tmpa;
  }
  // solution of the test solve: the resident displacement (smooth, with the crack's jump) on
  // the free dofs, like the corrections the u-subproblems compute; a pseudo-random field if the
  // displacement is still zero
  vec_convert<T, double>(st, v, s.u, n2);
  mask_fixed<T>(st, g, v, 2);
  vec_dot<T>(st, v, v, n2, slot(s, S_TMP));
  double vv;
  TRY(read_scalars(s, st, S_TMP, 1, &vv));
  if (!(vv > 0.0)) {
    vec_hash_fill<T>(st, v, n2, 12345u);
    mask_fixed<T>(st, g, v, 2);
  }
  apply_op<T>(s, st, ELASTIC, 0, v, b, false, S_TMP);
  const double rtol = mixed ? o.inner_rtol : 1e-8;
  const TuneCfg dflt{o.mg_degree, o.mg_coarse_degree > 0 ? o.mg_coarse_degree : o.mg_degree, 0, 0};
  double ms_d;
  int it_d;
  TRY(time_pcg<T>(s, st, o, dflt, b, rtol, &ms_d, &it_d));
  TuneCfg cur = dflt;
  double ms_b = ms_d;
  int it_b = it_d, trials = 1;
  for (int d = 1; d <= 4; ++d)
    for (int cd = 1; cd <= 3; ++cd) {
      const TuneCfg c{d, cd, 0, 0};
      if (c.deg == dflt.deg && c.cdeg == dflt.cdeg) continue;
      double ms;
      int it;
      TRY(time_pcg<T>(s, st, o, c, b, rtol, &ms, &it));
      ++trials;
      if (ms < ms_b) {
        ms_b = ms;
        it_b = it;
        cur = c;
      }
    }
  if (mixed) {
    const int rows[3] = {TY_MIN, TY, 16};
    const TuneCfg base = cur;
    for (int a = 0; a < 3; ++a)
      for (int c2 = 0; c2 < 3; ++c2) {
        const TuneCfg c{base.deg, base.cdeg, rows[a] == TY ? 0 : rows[a], rows[c2] == TY ? 0 : rows[c2]};
        if (c.tf == 0 && c.tc == 0) continue;
        double ms;
        int it;
        TRY(time_pcg<T>(s, st, o, c, b, rtol, &ms, &it));
        ++trials;
        if (ms < ms_b) {
          ms_b = ms;
          it_b = it;
          cur = c;
        }
      }
  }
  *best = cur;
  if (rep) {
    rep->mg_degree = cur.deg;
    rep->mg_coarse_degree = cur.cdeg;
    rep->tile_rows_fine = cur.tf ? cur.tf : TY;
    rep->tile_rows_coarse = cur.tc ? cur.tc : TY;
    rep->trials = trials;
    rep->iters_best = it_b;
    rep->iters_default = it_d;
    rep->ms_best = ms_b;
    rep->ms_default = ms_d;
  }
  s.xu_valid = false;
  return PF_OK;
}

// tune, cache and apply (the sim's options must already be applied by apply_opts)
pf_status tune_sim(pf_sim& s, cudaStream_t st, const pf_solver_opts& o, TuneCfg* out,
                   pf_tune_report* rep) {
  TuneCfg c;
  if (o.precision == PF_MIXED) TRY(tune_t<float>(s, st, o, &c, rep));
  else TRY(tune_t<double>(s, st, o, &c, rep));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(s, o.precision)] = c;
  }
  s.cdeg = c.cdeg;
  s.tile_fine = c.tf;
  s.tile_coarse = c.tc;
  apply_tiles(s);
  *out = c;
  return PF_OK;
}

}  // namespace

namespace pf {
pf_status describe_mesh(const pf_mesh_desc* d, Grid* g) {
  pf_status st = validate(d);
  if (st != PF_OK) return st;
  *g = make_grid(*d, 0);
  return PF_OK;
}

// kernel constants of a material for callers without a sim (the same constants pf_set_material
// stores in a sim)
pf_status describe_material(const pf_material* mi, Mat* out) {
  if (!mi || !out) return fail(PF_EINVAL, "null argument");
  if (!(mi->E > 0) || !(mi->Gc > 0) || !(mi->ell > 0) || !(mi->k_ell >= 0) || !(mi->nu > -1.0) ||
      !(mi->nu < 0.5))
    return fail(PF_EINVAL, "invalid material constants");
  if (mi->model != PF_AT1 && mi->model != PF_AT2) return fail(PF_EINVAL, "unknown damage model");
  if (mi->plane != PF_PLANE_STRAIN && mi->plane != PF_PLANE_STRESS)
    return fail(PF_EINVAL, "unknown plane assumption");
  if (mi->beta != 0.0 && !(mi->pen > 0)) return fail(PF_EINVAL, "penetration length must be positive");
  Mat m{};
  double E = mi->E, nu = mi->nu;
  m.mu = E / (2.0 * (1.0 + nu));
  m.lam = mi->plane == PF_PLANE_STRAIN ? E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) : E * nu / (1.0 - nu * nu);
  m.lam2mu = m.lam + 2.0 * m.mu;
  m.k_ell = mi->k_ell;
  double cw = mi->model == PF_AT1 ? 8.0 / 3.0 : 2.0;  // c_w = 4 int_0^1 sqrt(w)
  m.c1 = 2.0 * mi->Gc * mi->ell / cw;
  m.c2 = mi->model == PF_AT2 ? 2.0 * mi->Gc / (cw * mi->ell) : 0.0;
  m.c3 = mi->model == PF_AT1 ? mi->Gc / (cw * mi->ell) : 0.0;
  m.gc_cw = mi->Gc / cw;
  m.ell = mi->ell;
  m.model = mi->model;
  *out = m;
  return PF_OK;
}
}  // namespace pf

// =============================================================================================
// C ABI
// =============================================================================================
namespace pf {
// Build a sim in caller-given workspace; every device operation is ordered on `st` and finished
// when this returns (no device-wide synchronization, so other streams keep running).
pf_status create_sim(pf_ctx* ctx, const pf_mesh_desc* d, void* ws, size_t ws_bytes,
                     cudaStream_t st, pf_sim** out) {
  if (!ctx || !out) return fail(PF_EINVAL, "null argument");
  TRY(validate(d));
  if (!ws) return fail(PF_EINVAL, "null workspace");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(PF_EINVAL, "workspace not 256-byte aligned");
  size_t need = pf_workspace_bytes(d, PF_FP64);
  if (ws_bytes < need) return fail(PF_ENOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, need);
  CU(cudaSetDevice(ctx->device));
  pf_sim* s = new (std::nothrow) pf_sim;
  if (!s) return fail(PF_ENOMEM, "host allocation failed");
  s->ctx = ctx;
  s->host = ctx->take_slot();
  if (!s->host) {
    delete s;
    return fail(PF_ECUDA, "cudaMallocHost failed");
  }
  s->desc = *d;
  Arena a{static_cast<char*>(ws), ws_bytes, 0, false};
  layout(*s, a);
  for (int e = 0; e < 4; ++e)
    for (int c = 0; c < 3; ++c) s->lift.load[e][c] = d->load[e][c];
  for (int k = 0; k < d->n_pins; ++k) s->lift.pin_load[k] = d->pin_load[k];
  s->lift.mode_I = d->mode_I;
  s->lift.K = d->mode_I_param[0];
  s->lift.xt0 = d->mode_I_param[1];
  s->lift.v = d->mode_I_param[2];
  s->lift.yl = d->mode_I_param[3];
  s->lift.x0 = d->x0;
  s->lift.y0 = d->y0;
  s->lift.lx = d->lx;
  s->lift.ly = d->ly;
  // initial state on the host: u = 0, alpha = alpha_prev from the damage boxes and the damage
  // Dirichlet data
  const Grid& g = s->lv[0].g;
  std::vector<double> al(g.n, 0.0);
  for (int node = 0; node < g.n; ++node) {
    int X2, Y2;
    if (node < g.nv) {
      int j = node / (g.nx + 1), i = node - j * (g.nx + 1);
      X2 = 2 * i;
      Y2 = 2 * j;
    } else {
      int c = node - g.nv, j = c / g.nx, i = c - j * g.nx;
      X2 = 2 * i + 1;
      Y2 = 2 * j + 1;
    }
    for (int b = 0; b < d->n_boxes; ++b)
      if (X2 >= d->box[b][0] && X2 <= d->box[b][1] && Y2 >= d->box[b][2] && Y2 <= d->box[b][3])
        al[node] = d->box_value[b];
    const int eX[4] = {0, 2 * g.nx, -1, -1}, eY[4] = {-1, -1, 0, 2 * g.ny};
    for (int e = 0; e < 4; ++e)
      if (d->fixed[e][2] && ((eX[e] >= 0 && X2 == eX[e]) || (eY[e] >= 0 && Y2 == eY[e])))
        al[node] = d->load[e][2];
    for (int k = 0; k < d->n_pins; ++k)
      if (d->pin_comp[k] == 2 && d->pin_x2[k] == X2 && d->pin_y2[k] == Y2) al[node] = d->pin_load[k];
  }
  std::vector<float> al32(al.begin(), al.end());
  const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
  cudaError_t e1 = cudaMemsetAsync(s->u, 0, 2 * (size_t)g.n * sizeof(double), st);
  cudaError_t e2 = cudaMemcpyAsync(s->alpha, al.data(), g.n * sizeof(double), h2d, st);
  cudaError_t e3 = cudaMemcpyAsync(s->alpha_prev, al.data(), g.n * sizeof(double), h2d, st);
  cudaError_t e4 = cudaMemcpyAsync(s->alpha32, al32.data(), g.n * sizeof(float), h2d, st);
  cudaError_t e5 = cudaMemsetAsync(s->ticket, 0, 64 * sizeof(unsigned), st);
  cudaError_t e6 =
      cudaMemsetAsync(s->eig, 0, (size_t)g.ny * elems_per_cell(g.kind) * sizeof(double), st);
  cudaError_t e7 = cudaStreamSynchronize(st);  // the host vectors above are read until here
  for (cudaError_t e : {e1, e2, e3, e4, e5, e6, e7})
    if (e != cudaSuccess) {
      delete s;
      return fail(PF_ECUDA, "initial state upload: %s", cudaGetErrorString(e));
    }
  *out = s;
  return PF_OK;
}

// Copy the resident fields to host memory, ordered on `st`; synchronous.
pf_status fields_to_host(pf_sim* s, cudaStream_t st, double* u, double* alpha,
                         double* alpha_prev) {
  const size_t n = s->lv[0].g.n;
  const cudaMemcpyKind d2h = cudaMemcpyDeviceToHost;
  if (u) CU(cudaMemcpyAsync(u, s->u, 2 * n * sizeof(double), d2h, st));
  if (alpha) CU(cudaMemcpyAsync(alpha, s->alpha, n * sizeof(double), d2h, st));
  if (alpha_prev) CU(cudaMemcpyAsync(alpha_prev, s->alpha_prev, n * sizeof(double), d2h, st));
  CU(cudaStreamSynchronize(st));
  return PF_OK;
}
}  // namespace pf

extern "C" {

const char* pf_last_error(void) { return g_err.c_str(); }
const char* pf_version(void) { return "libpf 0.1 (sm_103a)"; }

pf_status pf_default_opts(pf_solver_opts* o) {
  if (!o) return fail(PF_EINVAL, "null options");
  memset(o, 0, sizeof *o);
  o->algo = PF_ALGO_ORAM;
  o->precision = PF_FP64;
  o->omega = 1.0;
  o->am_tol = 1e-6;
  o->am_maxit = 20000;
  o->u_rtol = 1e-8;
  o->inner_rtol = 1e-4;
  o->cg_maxit = 2000;
  o->rs_rtol = 1e-8;
  o->rs_maxit = 100;
  o->alpha_cg_rtol = 1e-6;
  o->zeta = 1e-10;
  o->mg_levels_max = 0;
  o->mg_degree = 2;
  o->switch_tol = 1e-2;
  o->newton_rtol = 1e-8;
  o->newton_maxit = 30;
  o->minres_maxit = 500;
  o->minres_rtol = 1e-6;
  o->use_graphs = 1;
  o->batch_workers = 8;
  o->am_forcing = 0.0;
  o->am_forcing_max = 1e-3;
  o->mg_tail = 1;
  o->mg_coarse_degree = 0;
  o->omega_rule = 0;
  o->omega_auto = 0;
  o->omega_max = 1.9;
  o->autotune = 0;
  o->tile_rows_fine = o->tile_rows_coarse = 0;
  return PF_OK;
}

pf_status pf_ctx_create(int device, pf_ctx** out) {
  if (!out) return fail(PF_EINVAL, "null output");
  CU(cudaSetDevice(device));
  pf_ctx* c = new (std::nothrow) pf_ctx;
  if (!c) return fail(PF_ENOMEM, "host allocation failed");
  c->device = device;
  double* probe = c->take_slot();  // allocate the first chunk now so errors surface here
  if (!probe) {
    delete c;
    return fail(PF_ECUDA, "cudaMallocHost failed");
  }
  c->give_slot(probe);
  *out = c;
  return PF_OK;
}

void pf_ctx_destroy(pf_ctx* c) {
  if (!c) return;
  bool now;
  {
    std::lock_guard<std::mutex> lk(c->mu);
    c->closed = true;
    now = c->users == 0;
  }
  if (now) free_ctx(c);
}

size_t pf_workspace_bytes(const pf_mesh_desc* d, int precision) {
  (void)precision;
  if (validate(d) != PF_OK) return 0;
  pf_sim s;
  s.desc = *d;
  Arena a{nullptr, 0, 0, true};
  layout(s, a);
  return a.off + 256;
}

pf_status pf_create_mesh(pf_ctx* ctx, const pf_mesh_desc* d, void* ws, size_t ws_bytes,
                         pf_sim** out) {
  TRY(pf::create_sim(ctx, d, ws, ws_bytes, nullptr, out));
  CU(cudaDeviceSynchronize());
  return PF_OK;
}

pf_status pf_set_material(pf_sim* s, const pf_material* mi) {
  if (!s || !mi) return fail(PF_EINVAL, "null argument");
  CLAIM(s);
  if (!(mi->E > 0) || !(mi->Gc > 0) || !(mi->ell > 0) || !(mi->k_ell >= 0) || !(mi->nu > -1.0) ||
      !(mi->nu < 0.5))
    return fail(PF_EINVAL, "invalid material constants");
  if (mi->model != PF_AT1 && mi->model != PF_AT2) return fail(PF_EINVAL, "unknown damage model");
  if (mi->plane != PF_PLANE_STRAIN && mi->plane != PF_PLANE_STRESS)
    return fail(PF_EINVAL, "unknown plane assumption");
  if (mi->beta != 0.0 && !(mi->pen > 0)) return fail(PF_EINVAL, "penetration length must be positive");
  Mat m{};
  double E = mi->E, nu = mi->nu;
  m.mu = E / (2.0 * (1.0 + nu));
  m.lam = mi->plane == PF_PLANE_STRAIN ? E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu)) : E * nu / (1.0 - nu * nu);
  m.lam2mu = m.lam + 2.0 * m.mu;
  m.k_ell = mi->k_ell;
  double cw = mi->model == PF_AT1 ? 8.0 / 3.0 : 2.0;  // c_w = 4 int_0^1 sqrt(w)
  m.c1 = 2.0 * mi->Gc * mi->ell / cw;
  m.c2 = mi->model == PF_AT2 ? 2.0 * mi->Gc / (cw * mi->ell) : 0.0;
  m.c3 = mi->model == PF_AT1 ? mi->Gc / (cw * mi->ell) : 0.0;
  m.gc_cw = mi->Gc / cw;
  m.ell = mi->ell;
  m.model = mi->model;
  s->m = m;
  s->mat_in = *mi;
  s->have_material = true;
  s->elastic_ready64 = s->elastic_ready32 = s->xu_valid = false;
  return PF_OK;
}



static pf_status check_opts(const pf_solver_opts* o) {
  if (!o) return fail(PF_EINVAL, "null options");
  if (o->algo < PF_ALGO_AM || o->algo > PF_ALGO_ORAM_N) return fail(PF_EINVAL, "unknown algorithm");
  if (o->precision != PF_FP64 && o->precision != PF_MIXED) return fail(PF_EINVAL, "unknown precision");
  if (!(o->omega > 0.0 && o->omega < 2.0)) return fail(PF_EINVAL, "omega must lie in (0, 2)");
  if (o->am_maxit < 1 || o->cg_maxit < 1 || o->rs_maxit < 1 || o->mg_degree < 1)
    return fail(PF_EINVAL, "iteration limits must be positive");
  if (o->mg_degree > MAX_CHEB || o->mg_coarse_degree > MAX_CHEB)
    return fail(PF_EINVAL, "Chebyshev degrees must not exceed 16");
  if (!(o->am_forcing >= 0.0) || !(o->am_forcing_max >= 0.0))
    return fail(PF_EINVAL, "am_forcing and am_forcing_max must be >= 0");
  if (o->omega_rule != 0 && o->omega_rule != 1) return fail(PF_EINVAL, "omega_rule must be 0 or 1");
  if (o->omega_auto != 0 && o->omega_auto != 1) return fail(PF_EINVAL, "omega_auto must be 0 or 1");
  if (o->autotune != 0 && o->autotune != 1) return fail(PF_EINVAL, "autotune must be 0 or 1");
  for (int tr : {o->tile_rows_fine, o->tile_rows_coarse})
    if (tr != 0 && tr != TY_MIN && tr != TY && tr != 16)
      return fail(PF_EINVAL, "tile heights must be 0, 4, 8 or 16");
  if (o->omega_auto && !(o->omega_max >= 1.0 && o->omega_max < 2.0))
    return fail(PF_EINVAL, "omega_max must lie in [1, 2)");
  if (o->algo == PF_ALGO_ORAM_N &&
      (o->newton_maxit < 1 || o->minres_maxit < 1 || !(o->switch_tol > 0.0 && o->switch_tol < 1.0) ||
       !(o->newton_rtol > 0.0) || !(o->minres_rtol > 0.0 && o->minres_rtol < 1.0)))
    return fail(PF_EINVAL, "ORAM-N needs newton_maxit, minres_maxit >= 1, switch_tol and "
                           "minres_rtol in (0, 1), newton_rtol > 0");
  return PF_OK;
}

pf_status pf_load_step(pf_sim* s, const pf_load* L, const pf_solver_opts* o, void* stream,
                       pf_step_report* rep) {
  if (!s || !L) return fail(PF_EINVAL, "null argument");
  TRY(check_opts(o));
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  CLAIM(s);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaError_t e = cudaSetDevice(s->ctx->device); e != cudaSuccess)
    return fail(PF_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  auto t0 = std::chrono::steady_clock::now();
  pf_solver_opts oo = *o;
  apply_opts(*s, oo);
  s->tile_fine = o->tile_rows_fine == TY ? 0 : o->tile_rows_fine;
  s->tile_coarse = o->tile_rows_coarse == TY ? 0 : o->tile_rows_coarse;
  if (o->autotune) {  // the cached configuration for this mesh and precision, tuned on first use
    TuneCfg c;
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(tune_key(*s, o->precision));
      if (it != g_tune.end()) {
        c = it->second;
        have = true;
      }
    }
    if (!have) TRY(tune_sim(*s, st, oo, &c, nullptr));
    oo.mg_degree = c.deg;
    oo.mg_coarse_degree = c.cdeg;
    apply_opts(*s, oo);
    s->tile_fine = c.tf;
    s->tile_coarse = c.tc;
  }
  apply_tiles(*s);
  o = &oo;
  pf_step_report r{};
  r.omega_bar_min = o->omega;
  r.omega_final = o->algo == PF_ALGO_AM ? 1.0 : o->omega;
  pf_status status = begin_step(*s, st, *L);
  // ||Phi|| of the full optimality system (eq. kkt) at the start and the end of the step, so
  // that the residual a converged step leaves is visible (ORAM-N computes both itself)
  const bool am_algo = o->algo != PF_ALGO_ORAM_N;
  if (status == PF_OK && am_algo) status = full_residual(*s, st, o->zeta, &r.phi_start);
  if (status == PF_OK)
    status = o->algo == PF_ALGO_ORAM_N ? oramn_step(*s, st, *o, &r) : oram_step(*s, st, *o, &r);
  if ((status == PF_OK || status == PF_ENOTCONV) && am_algo) {
    pf_status e1 = full_residual(*s, st, o->zeta, &r.phi_norm);
    if (e1 != PF_OK) status = e1;
  }
  if (status == PF_OK || status == PF_ENOTCONV) {
    pf_status e2 = energy_now(*s, st, r.energy);
    if (e2 != PF_OK) status = e2;
  }
  r.status = status;
  r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (rep) *rep = r;
  return status;
}

pf_status pf_autotune(pf_sim* s, const pf_solver_opts* o, void* stream, pf_tune_report* out) {
  if (!s) return fail(PF_EINVAL, "null sim");
  TRY(check_opts(o));
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  CLAIM(s);
  CU(cudaSetDevice(s->ctx->device));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  apply_opts(*s, *o);
  TuneCfg c;
  pf_tune_report r{};
  TRY(tune_sim(*s, st, *o, &c, &r));
  if (out) *out = r;
  return PF_OK;
}

pf_status pf_energy(pf_sim* s, void* stream, double out[3]) {
  if (!s || !out) return fail(PF_EINVAL, "null argument");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  CU(cudaSetDevice(s->ctx->device));
  return energy_now(*s, static_cast<cudaStream_t>(stream), out);
}

pf_status pf_get_fields(pf_sim* s, double* u, double* alpha, double* alpha_prev) {
  if (!s) return fail(PF_EINVAL, "null sim");
  CLAIM(s);
  CU(cudaSetDevice(s->ctx->device));
  CU(cudaDeviceSynchronize());
  size_t n = s->lv[0].g.n;
  if (u) CU(cudaMemcpy(u, s->u, 2 * n * sizeof(double), cudaMemcpyDeviceToHost));
  if (alpha) CU(cudaMemcpy(alpha, s->alpha, n * sizeof(double), cudaMemcpyDeviceToHost));
  if (alpha_prev) CU(cudaMemcpy(alpha_prev, s->alpha_prev, n * sizeof(double), cudaMemcpyDeviceToHost));
  return PF_OK;
}

pf_status pf_set_fields(pf_sim* s, const double* u, const double* alpha, const double* alpha_prev) {
  if (!s) return fail(PF_EINVAL, "null sim");
  CLAIM(s);
  CU(cudaSetDevice(s->ctx->device));
  size_t n = s->lv[0].g.n;
  if (u) CU(cudaMemcpy(s->u, u, 2 * n * sizeof(double), cudaMemcpyHostToDevice));
  if (alpha) {
    CU(cudaMemcpy(s->alpha, alpha, n * sizeof(double), cudaMemcpyHostToDevice));
    vec_convert<float, double>(0, s->alpha32, s->alpha, n);
  }
  if (alpha_prev) CU(cudaMemcpy(s->alpha_prev, alpha_prev, n * sizeof(double), cudaMemcpyHostToDevice));
  CU(cudaDeviceSynchronize());
  s->elastic_ready64 = s->elastic_ready32 = s->xu_valid = false;
  return PF_OK;
}

pf_status pf_sim_info(const pf_sim* s, int64_t* n_nodes, int64_t* n_elements, int32_t* levels) {
  if (!s) return fail(PF_EINVAL, "null sim");
  if (n_nodes) *n_nodes = s->lv[0].g.n;
  if (n_elements) *n_elements = s->lv[0].g.nelem;
  if (levels) *levels = (int32_t)s->lv.size();
  return PF_OK;
}

void pf_destroy(pf_sim* s) { delete s; }

pf_status pf_set_load(pf_sim* s, const pf_load* L) {
  if (!s || !L) return fail(PF_EINVAL, "null argument");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  CU(cudaSetDevice(s->ctx->device));
  TRY(set_load(*s, L->t, L->dT, 0));
  CU(cudaDeviceSynchronize());
  return PF_OK;
}

pf_status pf_op_elastic_apply(pf_sim* s, int precision, int masked, const void* x, void* y,
                              void* stream) {
  if (!s || !x || !y) return fail(PF_EINVAL, "null argument");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CU(cudaSetDevice(s->ctx->device));
  const int mode = masked ? M_MASKED : M_APPLY;
  // the operator reads and writes (u_x, u_y) pairs as one vector access
  const uintptr_t pair = precision == PF_FP64 ? 16 : 8;
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y)) % pair)
    return fail(PF_EINVAL, "x and y must be aligned to %d bytes", (int)pair);
  if (precision == PF_FP64) {
    ElasticArgs<double> a{};
    a.x = static_cast<const double*>(x);
    a.alpha = s->alpha;
    a.y = static_cast<double*>(y);
    launch_elastic<double>(st, s->lv[0].g, s->m, COEF_ALPHA, mode, false, false, a);
  } else if (precision == PF_MIXED) {
    ElasticArgs<float> a{};
    a.x = static_cast<const float*>(x);
    a.alpha = s->alpha32;
    a.y = static_cast<float*>(y);
    launch_elastic<float>(st, s->lv[0].g, s->m, COEF_ALPHA, mode, false, false, a);
  } else {
    return fail(PF_EINVAL, "unknown precision");
  }
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return PF_OK;
}

pf_status pf_op_elastic_residual(pf_sim* s, int precision, double* r, double* norm2,
                                 void* stream) {
  if (!s || !r) return fail(PF_EINVAL, "null argument");
  if (precision != PF_FP64 && precision != PF_MIXED) return fail(PF_EINVAL, "unknown precision");
  if (reinterpret_cast<uintptr_t>(r) % 16) return fail(PF_EINVAL, "r must be 16-byte aligned");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  CU(cudaSetDevice(s->ctx->device));
  double nrm;
  s->df = precision == PF_MIXED;
  TRY(physical_residual(*s, static_cast<cudaStream_t>(stream), s->u, r, &nrm));
  if (norm2) *norm2 = nrm * nrm;
  return PF_OK;
}

pf_status pf_op_damage_gradient(pf_sim* s, int precision, double* F, double* Phi,
                                uint8_t* active, double* phi_norm2, void* stream) {
  if (!s || !F || !Phi) return fail(PF_EINVAL, "null argument");
  if (precision != PF_FP64 && precision != PF_MIXED) return fail(PF_EINVAL, "unknown precision");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CU(cudaSetDevice(s->ctx->device));
  s->df = precision == PF_MIXED;
  damage_q(st, s->lv[0].g, s->m, s->u, s->thermal ? s->eig : nullptr, s->q, nullptr, nullptr,
           s->df);
  double v[2];
  TRY(grad_at(*s, st, s->alpha, 1e-10, F, Phi, s->rhstr, active ? active : s->acttr, v));
  if (phi_norm2) *phi_norm2 = v[0];
  return PF_OK;
}

pf_status pf_op_damage_apply(pf_sim* s, int precision, const void* x, void* y, void* stream) {
  if (!s || !x || !y) return fail(PF_EINVAL, "null argument");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CU(cudaSetDevice(s->ctx->device));
  const Grid& g = s->lv[0].g;
  damage_q(st, g, s->m, s->u, s->thermal ? s->eig : nullptr, s->q, s->lv[0].f64.wD, s->lv[0].f32.wD,
           precision == PF_MIXED);
  if (precision == PF_FP64) {
    DamageArgs<double> a{};
    a.x = static_cast<const double*>(x);
    a.w = s->lv[0].f64.wD;
    a.y = static_cast<double*>(y);
    launch_damage<double>(st, g, s->m, M_APPLY, false, a);
  } else if (precision == PF_MIXED) {
    DamageArgs<float> a{};
    a.x = static_cast<const float*>(x);
    a.w = s->lv[0].f32.wD;
    a.y = static_cast<float*>(y);
    launch_damage<float>(st, g, s->m, M_APPLY, false, a);
  } else {
    return fail(PF_EINVAL, "unknown precision");
  }
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return PF_OK;
}

pf_status pf_op_coupling_apply(pf_sim* s, int transpose, const double* x, double* y,
                               void* stream) {
  if (!s || !x || !y) return fail(PF_EINVAL, "null argument");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  if (transpose != 0 && transpose != 1) return fail(PF_EINVAL, "transpose must be 0 or 1");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CU(cudaSetDevice(s->ctx->device));
  CouplingArgs<double> b{};
  b.u = s->u;
  b.alpha = s->alpha;
  b.eig = s->thermal ? s->eig : nullptr;
  b.x = x;
  b.y = y;
  launch_coupling<double>(st, s->lv[0].g, s->m, transpose == 1, b);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(st));
  return PF_OK;
}

pf_status pf_op_u_solve(pf_sim* s, const pf_solver_opts* o, void* stream, pf_step_report* rep) {
  if (!s) return fail(PF_EINVAL, "null sim");
  CLAIM(s);
  TRY(check_opts(o));
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CU(cudaSetDevice(s->ctx->device));
  s->r_scale = 0.0;
  s->df = o->precision == PF_MIXED;
  s->use_graphs = o->use_graphs != 0;
  s->nl_active = o->mg_levels_max > 0 ? std::min<int>(o->mg_levels_max, (int)s->lv.size())
                                      : (int)s->lv.size();
  s->use_tail = o->mg_tail != 0;
  s->cdeg = o->mg_coarse_degree > 0 ? o->mg_coarse_degree : o->mg_degree;
  s->elastic_ready64 = s->elastic_ready32 = s->xu_valid = false;
  pf_step_report r{};
  pf_status status = u_solve(*s, st, *o, &r);
  if (status == PF_OK || status == PF_ENOTCONV)
    CU(cudaMemcpyAsync(s->u, s->xu, 2 * (size_t)s->lv[0].g.n * sizeof(double),
                       cudaMemcpyDeviceToDevice, st));
  CU(cudaStreamSynchronize(st));
  if (rep) *rep = r;
  return status;
}

pf_status pf_op_alpha_solve(pf_sim* s, const pf_solver_opts* o, void* stream, pf_step_report* rep) {
  if (!s) return fail(PF_EINVAL, "null sim");
  CLAIM(s);
  TRY(check_opts(o));
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  CU(cudaSetDevice(s->ctx->device));
  s->phi_scale = 0.0;
  s->df = o->precision == PF_MIXED;
  s->use_graphs = o->use_graphs != 0;
  s->nl_active = o->mg_levels_max > 0 ? std::min<int>(o->mg_levels_max, (int)s->lv.size())
                                      : (int)s->lv.size();
  s->use_tail = o->mg_tail != 0;
  s->cdeg = o->mg_coarse_degree > 0 ? o->mg_coarse_degree : o->mg_degree;
  pf_step_report r{};
  pf_status status = alpha_solve(*s, st, *o, &r);
  if (status == PF_OK || status == PF_ENOTCONV) {
    const size_t n = s->lv[0].g.n;
    CU(cudaMemcpyAsync(s->alpha, s->xrs, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    vec_convert<float, double>(st, s->alpha32, s->alpha, n);
    s->elastic_ready64 = s->elastic_ready32 = s->xu_valid = false;
  }
  CU(cudaStreamSynchronize(st));
  if (rep) *rep = r;
  return status;
}

pf_status pf_op_full_residual(pf_sim* s, double* phi_norm, void* stream) {
  if (!s || !phi_norm) return fail(PF_EINVAL, "null argument");
  CLAIM(s);
  if (!s->have_material) return fail(PF_EINVAL, "material not set");
  CU(cudaSetDevice(s->ctx->device));
  return full_residual(*s, static_cast<cudaStream_t>(stream), 1e-10, phi_norm);
}

}  // extern "C"
