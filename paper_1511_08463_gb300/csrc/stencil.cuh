// Matrix-free P1 operators on structured triangulations, in cell-tiled stencil form.
//
// One thread block owns a tile of TX x TY vertices (and, on crossed meshes, the TX x TY cell
// centres with the same indices).  It stages the node values of the tile plus a one-node halo in
// shared memory, computes one record per element of the (TX+1) x (TY+1) cells that touch the
// tile (each element exactly once per block, no atomics), and every thread then gathers the
// contributions of the elements around its vertex (6 on right meshes, 8 on crossed meshes) and
// its centre (4) in a fixed order, so results are bitwise reproducible.
//
// Operators (Section 1.2 second derivatives, P1 exact integration):
//   ElasticOp: K(alpha) u = sum_T w_T B_T^T A0 (B_T u_T - eps0_T), w_T = abar_T |T|,
//              abar_T = (1/|T|) int_T (1 - alpha_h)^2 + k_ell (eq. elasticity; eigenstrain of
//              eq. energytshock for the physical residual).
//   DamageOp:  H p = sum_T (w_T M_T + c1 L_T) p_T with w_T = q_T + c2 (eq. helmholtz), and for
//              the gradient E_alpha = H alpha + g0, g0_T = (c3 - q_T) |T| / 3 per node.
#pragma once
#include <type_traits>

#include "dfloat.cuh"
#include "mg_core.cuh"

namespace pf {

enum Mode : int {
  M_APPLY = 0,   // y = A x
  M_MASKED = 1,  // y = A_ff x_f on free dofs (x read as 0 on excluded dofs), 0 on excluded dofs
  M_RESB = 2,    // r = b - A_ff x_f on free dofs, 0 on excluded dofs
  M_RESID = 3,   // elastic physical residual r = f - K u on free dofs (u unmasked), 0 elsewhere
  M_CHEB = 4,    // Chebyshev step: d' = cd d + cr dinv (b - A x); x' = x + d' (free dofs);
                 // x == null reads x = 0 (first step from zero)
  M_GRAD = 5,    // damage: F = H x + g0, Phi, active flags, rhs = -F on the inactive set
  M_TRIAL = 6    // damage: same as M_GRAD at x_t = clip(x + mu d, lo, hi); writes x_t
};

// Kernel constants in the operator's own precision, prepared on the host so that FP32 kernels
// perform no per-element FP64 conversions (FP64 throughput is ~1/58 of FP32 on this part).
template <class T>
struct Consts {
  T ihx, ihy, area, lam, mu, lam2mu, k_ell, c1, c2, c3;
};
template <class T>
inline Consts<T> make_consts(const Grid& g, const Mat& m) {
  return Consts<T>{T(g.ihx), T(g.ihy), T(g.area), T(m.lam), T(m.mu), T(m.lam2mu), T(m.k_ell),
                   T(m.c1), T(m.c2), T(m.c3)};
}

// ----------------------------------------------------------------------------------------------
// generic tile kernel
// ----------------------------------------------------------------------------------------------
// FP32 elasticity and damage operators are compiled for full occupancy (2048 threads per SM, at
// most 32 registers per thread), the double-float ones for half (at most 64 registers)
template <class Op, int TYV = TY>
__global__ void __launch_bounds__(TX* TYV, Op::FULL_OCC ? 2048 / (TX * TYV)
                                                        : (Op::HALF_OCC ? 1024 / (TX * TYV) : 1))
    stencil_kernel(Op op) {
  pdl_enter();
  using V = typename Op::V;
  using R = typename Op::R;
  using ET = typename Op::ET;
  constexpr int KIND = Op::KIND;
  constexpr int NE = elems_per_cell(KIND);
  constexpr int NRC = Op::NRC;
  constexpr int NC = KIND == CROSSED ? TYV + 1 : 1;
  __shared__ V sv[TYV + 2][TX + 2];
  __shared__ V sc[NC][TX + 1];
  // element records stored component-major: consecutive cells -> consecutive words, so both the
  // record writes and the gathers are free of shared-memory bank conflicts.  (A record-major
  // layout with one 16-byte word per FP32 record needs fewer instructions but four shared-memory
  // wavefronts per warp access instead of three; it measured slower.)
  constexpr bool VEC4 = false;
  __shared__ typename std::conditional<VEC4, float4, ET>::type
      se[VEC4 ? 1 : NRC][NE][TYV + 1][TX + 1];
  const Grid& g = op.g;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TYV;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int tid = tx + ty * TX;

  for (int s = tid; s < (TX + 2) * (TYV + 2); s += TX * TYV) {
    int li = s % (TX + 2), lj = s / (TX + 2);
    int gi = i0 - 1 + li, gj = j0 - 1 + lj;
    bool in = gi >= 0 && gi <= g.nx && gj >= 0 && gj <= g.ny;
    sv[lj][li] = in ? op.load(gj * (g.nx + 1) + gi, 2 * gi, 2 * gj) : Op::zero();
  }
  if constexpr (KIND == CROSSED) {
    for (int s = tid; s < (TX + 1) * (TYV + 1); s += TX * TYV) {
      int li = s % (TX + 1), lj = s / (TX + 1);
      int gi = i0 - 1 + li, gj = j0 - 1 + lj;
      bool in = gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny;
      sc[lj][li] = in ? op.load(g.nv + gj * g.nx + gi, 2 * gi + 1, 2 * gj + 1) : Op::zero();
    }
  }
  __syncthreads();
  auto put = [&](int t, int lj, int li, const R& r) {
    if constexpr (VEC4) {
      se[0][t][lj][li] = make_float4(r.c[0], r.c[1], r.c[2], NRC == 4 ? r.c[NRC - 1] : 0.f);
    } else {
#pragma unroll
      for (int c = 0; c < NRC; ++c) se[c][t][lj][li] = r.c[c];
    }
  };
  for (int s = tid; s < (TX + 1) * (TYV + 1); s += TX * TYV) {
    int li = s % (TX + 1), lj = s / (TX + 1);
    int ci = i0 - 1 + li, cj = j0 - 1 + lj;
    bool valid = ci >= 0 && ci < g.nx && cj >= 0 && cj < g.ny;
    V v00 = sv[lj][li], v10 = sv[lj][li + 1], v01 = sv[lj + 1][li], v11 = sv[lj + 1][li + 1];
    int cell = cj * g.nx + ci;
    const typename Op::Cell cd = op.cell(valid, cell);  // the cell's coefficients, one load
    if constexpr (KIND == CROSSED) {
      V c = sc[lj][li];
      put(0, lj, li, op.template element<0>(valid, cell, cj, cd, v00, v10, c));
      put(1, lj, li, op.template element<1>(valid, cell, cj, cd, v10, v11, c));
      put(2, lj, li, op.template element<2>(valid, cell, cj, cd, v11, v01, c));
      put(3, lj, li, op.template element<3>(valid, cell, cj, cd, v01, v00, c));
    } else {
      put(0, lj, li, op.template element<0>(valid, cell, cj, cd, v00, v10, v11));
      put(1, lj, li, op.template element<1>(valid, cell, cj, cd, v00, v11, v01));
    }
  }
  __syncthreads();
  auto get = [&](int t, int lj, int li) {
    R r;
    if constexpr (VEC4) {
      const float4 v = se[0][t][lj][li];
      r.c[0] = v.x;
      r.c[1] = v.y;
      r.c[2] = v.z;
      if constexpr (NRC == 4) r.c[NRC - 1] = v.w;
    } else {
#pragma unroll
      for (int c = 0; c < NRC; ++c) r.c[c] = se[c][t][lj][li];
    }
    return r;
  };

  constexpr int NRA = Op::NR > 0 ? Op::NR : 1;
  using RT = typename Op::RT;
  RT red[NRA];
#pragma unroll
  for (int q = 0; q < NRA; ++q) red[q] = RT(0);

  const int i = i0 + tx, j = j0 + ty;
  if (i <= g.nx && j <= g.ny) {
    typename Op::Acc a = Op::acc0();
    if constexpr (KIND == CROSSED) {
      op.template add<0, 0>(a, get(0, ty + 1, tx + 1));  // cell (i, j): vertex is v00
      op.template add<3, 1>(a, get(3, ty + 1, tx + 1));
      op.template add<0, 1>(a, get(0, ty + 1, tx));      // cell (i-1, j): v10
      op.template add<1, 0>(a, get(1, ty + 1, tx));
      op.template add<1, 1>(a, get(1, ty, tx));          // cell (i-1, j-1): v11
      op.template add<2, 0>(a, get(2, ty, tx));
      op.template add<2, 1>(a, get(2, ty, tx + 1));      // cell (i, j-1): v01
      op.template add<3, 0>(a, get(3, ty, tx + 1));
    } else {
      op.template add<0, 0>(a, get(0, ty + 1, tx + 1));  // cell (i, j): v00
      op.template add<1, 0>(a, get(1, ty + 1, tx + 1));
      op.template add<0, 1>(a, get(0, ty + 1, tx));      // cell (i-1, j): v10
      op.template add<0, 2>(a, get(0, ty, tx));          // cell (i-1, j-1): v11
      op.template add<1, 1>(a, get(1, ty, tx));
      op.template add<1, 2>(a, get(1, ty, tx + 1));      // cell (i, j-1): v01
    }
    op.store(j * (g.nx + 1) + i, 2 * i, 2 * j, sv[ty + 1][tx + 1], a, red);
  }
  if constexpr (KIND == CROSSED) {
    if (i < g.nx && j < g.ny) {
      typename Op::Acc a = Op::acc0();
      op.template add<0, 2>(a, get(0, ty + 1, tx + 1));
      op.template add<1, 2>(a, get(1, ty + 1, tx + 1));
      op.template add<2, 2>(a, get(2, ty + 1, tx + 1));
      op.template add<3, 2>(a, get(3, ty + 1, tx + 1));
      op.store(g.nv + j * g.nx + i, 2 * i + 1, 2 * j + 1, sc[ty + 1][tx + 1], a, red);
    }
  }
  if constexpr (Op::NR > 0) block_reduce_finalize<Op::NR, Op::RED_MAX, RT>(red, op.args.slot);
}

// ----------------------------------------------------------------------------------------------
// elasticity operator K(alpha) (2 dofs per node, interleaved)
// ----------------------------------------------------------------------------------------------
// (u_x, u_y) of one node as a single 8-byte (float) or 16-byte (double) access; every interleaved
// vector of the library starts on a 256-byte boundary, and the entry points that take caller
// vectors check their alignment.
template <class T>
struct Pair {
  T x, y;
};
template <class T>
__device__ __forceinline__ Pair<T> ld_pair(const T* p, int node) {
  if constexpr (sizeof(T) == 4) {
    const float2 v = *reinterpret_cast<const float2*>(p + 2 * (size_t)node);
    return Pair<T>{v.x, v.y};
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p + 2 * (size_t)node);
    return Pair<T>{v.x, v.y};
  }
}
template <class T>
__device__ __forceinline__ void st_pair(T* p, int node, T x, T y) {
  if constexpr (sizeof(T) == 4)
    *reinterpret_cast<float2*>(p + 2 * (size_t)node) = make_float2(x, y);
  else
    *reinterpret_cast<double2*>(p + 2 * (size_t)node) = make_double2(x, y);
}

// COEF_ALPHA: abar_T from the three nodal damage values; COEF_ELEM: abar_T read per element.
enum { COEF_ALPHA = 0, COEF_ELEM = 1 };

template <class T>
struct ElasticArgs {
  const T* x;         // input displacement (2n)
  const T* alpha;     // COEF_ALPHA: nodal damage (n)
  const T* coef;      // COEF_ELEM: abar per element
  const double* eig;  // EIGEN: eps0 = beta T per (cell row, element)
  const T* b;         // M_RESB, M_CHEB right-hand side
  const T* d;         // M_CHEB previous update
  const T* dinv;      // M_CHEB inverse diagonal (2n)
  const T* xc;        // M_CHEB: if set, x is read as x + P xc (prolongation from grid gc fused
  Grid gc;            // into the first post-smoothing step)
  T cd, cr;           // M_CHEB coefficients
  int x0b;            // M_CHEB, M_RESB: x is the first Chebyshev step from zero, c0 D^-1 b (0 on
  T c0;               // prescribed dofs), formed from b and dinv as it is read; M_CHEB takes it
                      // as the previous update too, M_RESB writes it to dout
  T* y;               // output (2n); M_CHEB: new x
  T* dout;            // M_CHEB: new d; M_RESB with x0b: the first step's x
  RedSlot slot;
  int coarse;         // launch accounting: multigrid level (0 = finest)
  int df;             // M_RESID with T = double: 1 computes in double-float (the mixed path)
};

// Arithmetic helpers shared by the operators.  For float and double they are the plain
// expressions; for double-float they leave out zero terms and use exact additions for the
// integer weights +-1, +-2 of the gradient tables instead of general products.
template <class C>
__device__ __forceinline__ C to_c(double v) { return C(v); }
template <class C>
__device__ __forceinline__ C to_c(float v) { return C(v); }
template <int c, class C>
__device__ __forceinline__ C imul(C v) {
  if constexpr (std::is_same<C, dfloat>::value) {
    static_assert(c >= -2 && c <= 2, "gradient weights are small integers");
    if constexpr (c == 0) return C(0);
    else if constexpr (c == 1) return v;
    else if constexpr (c == -1) return -v;
    else if constexpr (c == 2) return v + v;
    else return -(v + v);
  } else {
    return C(c) * v;
  }
}
template <int a, int b, int c, class C>
__device__ __forceinline__ C gsum(C x, C y, C z) {
  if constexpr (std::is_same<C, dfloat>::value) {
    C s = C(0);
    bool h = false;
    if constexpr (a != 0) {
      s = imul<a>(x);
      h = true;
    }
    if constexpr (b != 0) {
      s = h ? s + imul<b>(y) : imul<b>(y);
      h = true;
    }
    if constexpr (c != 0) s = h ? s + imul<c>(z) : imul<c>(z);
    return s;
  } else {
    return C(a) * x + C(b) * y + C(c) * z;
  }
}
// The NE per-element coefficients of a cell (cell-major arrays), as the arithmetic type: one
// 16- or 8-byte load for FP32 (the arrays start on 256-byte boundaries)
template <class C, int NE, class T>
__device__ __forceinline__ void load_cell_coefs(const T* p, int cell, C (&w)[NE]) {
  if constexpr (std::is_same<T, float>::value && NE == 4) {
    const float4 v = reinterpret_cast<const float4*>(p)[cell];
    w[0] = to_c<C>(v.x);
    w[1] = to_c<C>(v.y);
    w[2] = to_c<C>(v.z);
    w[3] = to_c<C>(v.w);
  } else if constexpr (std::is_same<T, float>::value && NE == 2) {
    const float2 v = reinterpret_cast<const float2*>(p)[cell];
    w[0] = to_c<C>(v.x);
    w[1] = to_c<C>(v.y);
  } else {
#pragma unroll
    for (int t = 0; t < NE; ++t) w[t] = to_c<C>(p[cell * NE + t]);
  }
}

// storage value of a computed one
template <class T, class C>
__device__ __forceinline__ T to_t(C v) {
  if constexpr (std::is_same<C, dfloat>::value) return T(double(v));
  else return T(v);
}

// C: the arithmetic type; dfloat for the FP64 physical residual of the mixed path (inputs and
// outputs stay FP64, T = double)
template <class T, int KIND_, int COEF, int MODE, bool EIGEN, bool DOT, class C = T>
struct ElasticOp {
  using Scalar = T;
  static constexpr bool FULL_OCC = sizeof(T) == 4;
  static constexpr bool HALF_OCC = std::is_same<C, dfloat>::value;
  static constexpr int KIND = KIND_;
  static constexpr int NR = (MODE == M_RESID || DOT) ? 1 : 0;
  static constexpr bool RED_MAX = false;
  // per-thread partial sums in the operator's precision (FP64 for double-float)
  using RT = typename std::conditional<std::is_same<C, dfloat>::value, double, C>::type;
  static constexpr int NE_ = elems_per_cell(KIND_);
  // a staged node: displacement, and the damage when the coefficient is computed from it
  struct VA {
    C ux, uy, a;
  };
  struct __align__(2 * sizeof(C)) VE {
    C ux, uy;
  };
  using V = typename std::conditional<COEF == COEF_ALPHA, VA, VE>::type;
  // per-cell data of the records loop: the stored element coefficients (COEF_ELEM)
  struct Cell {
    C w[COEF == COEF_ELEM ? NE_ : 1];
  };
  using ET = C;
  static constexpr int NRC = 3;
  struct R {
    C c[3];  // w A0 eps: sxx, syy, sxy
  };
  struct Acc {
    C ax, bx, ay, by;
  };
  Grid g;
  Mat m;
  Consts<C> cs;
  ElasticArgs<T> args;

  __device__ static V zero() {
    V v{};
    return v;
  }
  __device__ static Acc acc0() { return Acc{C(0), C(0), C(0), C(0)}; }

  __device__ Cell cell(bool valid, int c) const {
    Cell d{};
    if constexpr (COEF == COEF_ELEM)
      if (valid) load_cell_coefs<C>(args.coef, c, d.w);
    return d;
  }

  __device__ V load(int node, int X2, int Y2) const {
    V v;
    v.ux = v.uy = C(0);  // M_CHEB without x: smoothing from zero
    if (args.x) {
      const Pair<T> u = ld_pair(args.x, node);
      v.ux = to_c<C>(u.x);
      v.uy = to_c<C>(u.y);
    }
    if constexpr (MODE == M_CHEB || MODE == M_RESB) {
      if (args.x0b) {  // the step from zero, rounded as the M_CHEB store rounds it
        const Pair<T> b = ld_pair(args.b, node), di = ld_pair(args.dinv, node);
        v.ux = args.c0 * di.x * b.x;
        v.uy = args.c0 * di.y * b.y;
      }
    }
    if constexpr (MODE == M_CHEB) {
      if (args.xc) {
        int ca, cb;
        prolong_nodes(g, args.gc, node, X2, Y2, ca, cb);
        const Pair<T> pa = ld_pair(args.xc, ca), pb = ld_pair(args.xc, cb);
        v.ux += to_c<C>(T(0.5) * (pa.x + pb.x));
        v.uy += to_c<C>(T(0.5) * (pa.y + pb.y));
      }
    }
    if (MODE != M_APPLY && MODE != M_RESID) {
      if (is_fixed(g, X2, Y2, 0)) v.ux = C(0);
      if (is_fixed(g, X2, Y2, 1)) v.uy = C(0);
    }
    if constexpr (COEF == COEF_ALPHA) v.a = to_c<C>(args.alpha[node]);
    return v;
  }

  // one element with its own scalar coefficient load (callers whose coefficient array carries
  // no alignment guarantee, e.g. the single-block tail's shared-memory copy)
  template <int t>
  __device__ R element(bool valid, int cell, int cj, const V& n0, const V& n1, const V& n2) const {
    Cell d{};
    if constexpr (COEF == COEF_ELEM)
      if (valid) d.w[t] = to_c<C>(args.coef[cell * NE_ + t]);
    return element<t>(valid, cell, cj, d, n0, n1, n2);
  }
  template <int t>
  __device__ R element(bool valid, int cell, int cj, const Cell& cd, const V& n0, const V& n1,
                       const V& n2) const {
    if (!valid) return R{{C(0), C(0), C(0)}};
    constexpr int NE = elems_per_cell(KIND);
    constexpr int a0 = gx(KIND, t, 0), a1 = gx(KIND, t, 1), a2 = gx(KIND, t, 2);
    constexpr int b0 = gy(KIND, t, 0), b1 = gy(KIND, t, 1), b2 = gy(KIND, t, 2);
    C w;
    if constexpr (COEF == COEF_ALPHA)
      w = abar3<C>(n0.a, n1.a, n2.a, cs.k_ell) * cs.area;
    else
      w = cd.w[t] * cs.area;
    (void)NE;
    const C ihx = cs.ihx, ihy = cs.ihy;
    C sx = gsum<a0, a1, a2>(n0.ux, n1.ux, n2.ux);
    C sy = gsum<b0, b1, b2>(n0.uy, n1.uy, n2.uy);
    C s1 = gsum<b0, b1, b2>(n0.ux, n1.ux, n2.ux);
    C s2 = gsum<a0, a1, a2>(n0.uy, n1.uy, n2.uy);
    C exx = ihx * sx, eyy = ihy * sy, gxy = ihy * s1 + ihx * s2;
    if (EIGEN) {
      C e0 = to_c<C>(args.eig[cj * NE + t]);
      exx -= e0;
      eyy -= e0;
    }
    const C lam = cs.lam, l2m = cs.lam2mu, mu = cs.mu;
    return R{{w * (l2m * exx + lam * eyy), w * (lam * exx + l2m * eyy), w * mu * gxy}};
  }

  template <int t, int k>
  __device__ void add(Acc& a, const R& r) const {
    constexpr int cx = gx(KIND, t, k), cy = gy(KIND, t, k);
    if (cx != 0) {
      a.ax += imul<cx>(r.c[0]);
      a.ay += imul<cx>(r.c[2]);
    }
    if (cy != 0) {
      a.bx += imul<cy>(r.c[2]);
      a.by += imul<cy>(r.c[1]);
    }
  }

  __device__ void store(int node, int X2, int Y2, const V& own, const Acc& a,
                        RT (&red)[NR > 0 ? NR : 1]) const {
    C fx = cs.ihx * a.ax + cs.ihy * a.bx;
    C fy = cs.ihx * a.ay + cs.ihy * a.by;
    bool f0 = false, f1 = false;
    if (MODE != M_APPLY) {
      f0 = is_fixed(g, X2, Y2, 0);
      f1 = is_fixed(g, X2, Y2, 1);
    }
    if constexpr (MODE == M_RESID) {
      const T rx = f0 ? T(0) : to_t<T>(-fx), ry = f1 ? T(0) : to_t<T>(-fy);
      st_pair(args.y, node, rx, ry);
      red[0] += RT(rx) * RT(rx) + RT(ry) * RT(ry);
    } else {
      static_assert(std::is_same<C, T>::value, "only the physical residual runs in double-float");
      if (MODE == M_APPLY || MODE == M_MASKED) {
        T yx = f0 ? T(0) : fx, yy = f1 ? T(0) : fy;
        st_pair(args.y, node, yx, yy);
        if (DOT) red[0] += own.ux * yx + own.uy * yy;
      } else if (MODE == M_RESB) {
        const Pair<T> b = ld_pair(args.b, node);
        T rx = f0 ? T(0) : b.x - fx, ry = f1 ? T(0) : b.y - fy;
        st_pair(args.y, node, rx, ry);
        if (args.x0b) st_pair(args.dout, node, own.ux, own.uy);
        if (DOT) red[0] += rx * rx + ry * ry;
      } else if (MODE == M_CHEB) {
        const Pair<T> b = ld_pair(args.b, node), di = ld_pair(args.dinv, node);
        const Pair<T> p = args.d ? ld_pair(args.d, node)
                                 : (args.x0b ? Pair<T>{own.ux, own.uy} : Pair<T>{T(0), T(0)});
        T rx = b.x - fx, ry = b.y - fy;
        T dx = f0 ? T(0) : args.cd * p.x + args.cr * di.x * rx;
        T dy = f1 ? T(0) : args.cd * p.y + args.cr * di.y * ry;
        st_pair(args.dout, node, dx, dy);
        const T yx = own.ux + dx, yy = own.uy + dy;
        st_pair(args.y, node, yx, yy);
        // the preconditioner's last step: r.z of the CG, with b = r and the new x = z
        if (DOT) red[0] += b.x * yx + b.y * yy;
      }
    }
  }
};

// ----------------------------------------------------------------------------------------------
// damage Hessian H(q) (1 dof per node); gradient / MCP residual / active set in FP64
// ----------------------------------------------------------------------------------------------
template <class T>
struct DamageArgs {
  const T* x;           // input field (n)
  const T* w;           // per-element mass weight; M_GRAD/M_TRIAL: q_T (weight q + c2)
  const uint8_t* excl;  // M_MASKED/M_RESB/M_CHEB: 1 = excluded (active or fixed) node
  const T* b;           // M_RESB, M_CHEB
  const T* d;           // M_CHEB previous update; M_TRIAL direction
  const T* dinv;        // M_CHEB
  const T* xc;          // M_CHEB: if set, x is read as x + P xc (grid gc), see ElasticArgs
  Grid gc;
  const double* lo;     // M_GRAD/M_TRIAL: lower bound alpha_prev
  T cd, cr;             // M_CHEB coefficients; M_TRIAL: cd = step mu
  int x0b;              // M_CHEB, M_RESB: x is the first Chebyshev step from zero, c0 D^-1 b (0 on
  T c0;                 // excluded nodes), as in ElasticArgs
  double zeta;
  T* y;                 // output: M_APPLY..M_CHEB result; M_GRAD/M_TRIAL: F
  T* dout;              // M_CHEB new d; M_GRAD/M_TRIAL: Phi; M_RESB with x0b: the first step's x
  T* rhs;               // M_GRAD/M_TRIAL: -F on the inactive set, 0 elsewhere
  T* xt;                // M_TRIAL: trial point
  uint8_t* act;         // M_GRAD/M_TRIAL: active flags written
  RedSlot slot;
  int coarse;           // launch accounting: multigrid level (0 = finest)
  int df;               // M_GRAD/M_TRIAL: 1 computes H x + g0 in double-float (the mixed path)
};

// C: the arithmetic type; dfloat for the FP64 damage gradient / trial point of the mixed path
// (inputs and outputs stay FP64, T = double)
template <class T, int KIND_, int MODE, bool DOT, class C = T>
struct DamageOp {
  using Scalar = T;
  static constexpr bool FULL_OCC = sizeof(T) == 4;
  static constexpr bool HALF_OCC = std::is_same<C, dfloat>::value;
  static constexpr int KIND = KIND_;
  static constexpr int NR = (MODE == M_GRAD || MODE == M_TRIAL) ? 2 : (DOT ? 1 : 0);
  static constexpr bool RED_MAX = false;
  static constexpr bool DF = std::is_same<C, dfloat>::value;
  using RT = typename std::conditional<DF, double, C>::type;
  struct V {
    C p;
  };
  static constexpr int NE_ = elems_per_cell(KIND_);
  struct Cell {  // the cell's element weights
    C w[NE_];
  };
  using ET = C;
  static constexpr int NRC = 4;
  struct R {
    C c[4];  // P, M, X, Y
  };
  struct Acc {
    C P, M, X, Y;
  };
  Grid g;
  Mat m;
  Consts<C> cs;
  DamageArgs<T> args;

  __device__ static V zero() { return V{C(0)}; }
  __device__ static Acc acc0() { return Acc{C(0), C(0), C(0), C(0)}; }

  __device__ Cell cell(bool valid, int c) const {
    Cell d{};
    if (valid) load_cell_coefs<C>(args.w, c, d.w);
    return d;
  }

  __device__ double upper(int X2, int Y2, double l) const {
    return is_fixed(g, X2, Y2, 2) ? l : 1.0;
  }
  // the line-search point of M_TRIAL in FP64: clip(x + mu d) to the node's box
  __device__ double trial_value(int node, int X2, int Y2) const {
    double l = args.lo[node], h = upper(X2, Y2, l);
    double z = double(args.x[node]) + double(args.cd) * double(args.d[node]);
    return fmin(fmax(z, l), h);
  }

  __device__ V load(int node, int X2, int Y2) const {
    V v;
    if (MODE == M_TRIAL) {
      v.p = to_c<C>(T(trial_value(node, X2, Y2)));
    } else {
      v.p = args.x ? to_c<C>(args.x[node]) : C(0);  // M_CHEB without x: smoothing from zero
      if constexpr (MODE == M_CHEB || MODE == M_RESB) {
        if (args.x0b) v.p = args.c0 * args.dinv[node] * args.b[node];  // the step from zero
      }
      if constexpr (MODE == M_CHEB) {
        if (args.xc) {
          int ca, cb;
          prolong_nodes(g, args.gc, node, X2, Y2, ca, cb);
          v.p += to_c<C>(T(0.5) * (args.xc[ca] + args.xc[cb]));
        }
      }
      if ((MODE == M_MASKED || MODE == M_RESB || MODE == M_CHEB) && args.excl && args.excl[node]) v.p = C(0);
    }
    return v;
  }

  // one element with its own scalar weight load (callers whose weight array carries no alignment
  // guarantee, e.g. the single-block tail's shared-memory copy)
  template <int t>
  __device__ R element(bool valid, int cell, int cj, const V& n0, const V& n1, const V& n2) const {
    Cell d{};
    if (valid) d.w[t] = to_c<C>(args.w[cell * NE_ + t]);
    return element<t>(valid, cell, cj, d, n0, n1, n2);
  }
  template <int t>
  __device__ R element(bool valid, int cell, int cj, const Cell& cd, const V& n0, const V& n1,
                       const V& n2) const {
    if (!valid) return R{{C(0), C(0), C(0), C(0)}};
    constexpr int a0 = gx(KIND, t, 0), a1 = gx(KIND, t, 1), a2 = gx(KIND, t, 2);
    constexpr int b0 = gy(KIND, t, 0), b1 = gy(KIND, t, 1), b2 = gy(KIND, t, 2);
    const C area = cs.area;
    C wt = cd.w[t];
    C qT = wt;
    if (MODE == M_GRAD || MODE == M_TRIAL) wt = wt + cs.c2;
    C me = wt * area * C(1.0 / 12.0);
    C S = n0.p + n1.p + n2.p;
    C gpx = cs.ihx * gsum<a0, a1, a2>(n0.p, n1.p, n2.p);
    C gpy = cs.ihy * gsum<b0, b1, b2>(n0.p, n1.p, n2.p);
    C c1a = cs.c1 * area;
    C P = me * S;
    if (MODE == M_GRAD || MODE == M_TRIAL) P += (cs.c3 - qT) * area * C(1.0 / 3.0);
    return R{{P, me, c1a * cs.ihx * gpx, c1a * cs.ihy * gpy}};
  }

  template <int t, int k>
  __device__ void add(Acc& a, const R& r) const {
    constexpr int cx = gx(KIND, t, k), cy = gy(KIND, t, k);
    a.P += r.c[0];
    a.M += r.c[1];
    if (cx != 0) a.X += imul<cx>(r.c[2]);
    if (cy != 0) a.Y += imul<cy>(r.c[3]);
  }

  __device__ void store(int node, int X2, int Y2, const V& own, const Acc& a,
                        RT (&red)[NR > 0 ? NR : 1]) const {
    C f = a.P + a.M * own.p + a.X + a.Y;
    if constexpr (MODE == M_GRAD || MODE == M_TRIAL) {  // T = double
      // the node's own value exactly as FP64 (a double-float copy keeps 48 bits)
      double xv;
      if constexpr (DF) xv = MODE == M_TRIAL ? trial_value(node, X2, Y2) : double(args.x[node]);
      else xv = double(own.p);
      const double F = to_t<double>(f);
      double l = args.lo[node], h = upper(X2, Y2, l);
      double ph;
      bool fpos, fneg;
      if constexpr (DF) {
        // the nested Fischer-Burmeister function in double-float; the distances to the bounds
        // are exact FP64 differences, F the double-float sum itself
        const dfloat a = dfloat(xv - l), b = dfloat(h - xv), mf = -f;
        const dfloat psi = df_sqrt(b * b + mf * mf) - b - mf;
        ph = double(df_sqrt(a * a + psi * psi) - a - psi);
        fpos = df_positive(f);
        fneg = df_negative(f);
      } else {
        ph = mcp_phi(xv, F, l, h);
        fpos = F > 0.0;
        fneg = F < 0.0;
      }
      // eq. reducedis with both bounds; a single-point box counts as lower-active
      const bool lower = (h - l <= args.zeta) || (xv <= l + args.zeta && fpos);
      const bool upper = !lower && (xv >= h - args.zeta && fneg);
      const bool active = lower || upper;
      args.y[node] = T(F);
      args.dout[node] = T(ph);
      args.rhs[node] = active ? T(0) : T(-F);
      args.act[node] = lower ? 1 : (upper ? 2 : 0);
      if (MODE == M_TRIAL) args.xt[node] = T(xv);
      red[0] += RT(ph * ph);
      red[1] += active ? RT(0) : RT(F * F);
    } else {
      static_assert(!DF, "only the gradient and the trial point run in double-float");
      if (MODE == M_APPLY) {
        args.y[node] = f;
        if (DOT) red[0] += own.p * f;
      } else if (MODE == M_MASKED) {
        T v = (args.excl && args.excl[node]) ? T(0) : f;
        args.y[node] = v;
        if (DOT) red[0] += own.p * v;
      } else if (MODE == M_RESB) {
        T r = (args.excl && args.excl[node]) ? T(0) : args.b[node] - f;
        args.y[node] = r;
        if (args.x0b) args.dout[node] = own.p;
        if (DOT) red[0] += r * r;
      } else if (MODE == M_CHEB) {
        T dp = args.d ? args.d[node] : (args.x0b ? own.p : T(0));
        const T bn = args.b[node];
        T dn = (args.excl && args.excl[node]) ? T(0) : args.cd * dp + args.cr * args.dinv[node] * (bn - f);
        args.dout[node] = dn;
        args.y[node] = own.p + dn;
        if (DOT) red[0] += bn * (own.p + dn);  // r.z of the CG (see ElasticOp)
      }
    }
  }
};

// ----------------------------------------------------------------------------------------------
// coupling block E_ua of the Newton Jacobian (Section 1.2 eq. offdiag, Section 3.3 block B):
//   B_ij = int a'(alpha_h) A0 eps_eff(u) : eps(phi_i) phi_j,  a'(alpha) = -2 (1 - alpha),
// per element  int_T a'(alpha_h) phi_j = -2 |T| (1/3 - (alpha_j + S_alpha) / 12)  (P1 mass matrix).
//   CouplingOp<T, K, false>: y_u (+)= B x_alpha  (x_alpha read as 0 on excluded alpha nodes;
//                            y_u zero on prescribed displacement dofs)
//   CouplingOp<T, K, true>:  y_a (+)= B^T x_u    (x_u read as 0 on prescribed dofs; y_a zero on
//                            excluded alpha nodes)
// ----------------------------------------------------------------------------------------------
template <class T>
struct CouplingArgs {
  const T* x;         // input: x_alpha (n) or x_u (2n)
  const T* u;         // state displacement (2n)
  const T* alpha;     // state damage (n)
  const T* eig;       // eps0 per (cell row, element) or null
  const uint8_t* excl;  // alpha exclusion mask (active set), may be null
  T* y;               // output (2n for B, n for B^T)
  int accumulate;     // 1: y += result
  RedSlot slot;
  int coarse;
};

template <class T, int KIND_, bool TRANSPOSE>
struct CouplingOp {
  using Scalar = T;
  static constexpr bool FULL_OCC = false;
  static constexpr bool HALF_OCC = false;
  static constexpr int KIND = KIND_;
  static constexpr int NR = 0;
  static constexpr bool RED_MAX = false;
  using RT = T;
  using ET = T;
  static constexpr int NRC = TRANSPOSE ? 2 : 3;
  struct V {
    T x0, x1, ux, uy, a;  // input (x0 = x_alpha or x_u,x; x1 = x_u,y), state u, alpha
  };
  struct R {
    T c[NRC];
  };
  struct Acc {
    T c[4];
  };
  Grid g;
  Mat m;
  Consts<T> cs;
  CouplingArgs<T> args;

  __device__ static V zero() { return V{T(0), T(0), T(0), T(0), T(0)}; }
  __device__ static Acc acc0() { return Acc{{T(0), T(0), T(0), T(0)}}; }

  __device__ V load(int node, int X2, int Y2) const {
    V v;
    if (TRANSPOSE) {
      v.x0 = is_fixed(g, X2, Y2, 0) ? T(0) : args.x[2 * node];
      v.x1 = is_fixed(g, X2, Y2, 1) ? T(0) : args.x[2 * node + 1];
    } else {
      v.x0 = (args.excl && args.excl[node]) ? T(0) : args.x[node];
      v.x1 = T(0);
    }
    v.ux = args.u[2 * node];
    v.uy = args.u[2 * node + 1];
    v.a = args.alpha[node];
    return v;
  }

  struct Cell {};
  __device__ Cell cell(bool, int) const { return Cell{}; }
  template <int t>
  __device__ R element(bool valid, int cell, int cj, const Cell&, const V& n0, const V& n1,
                       const V& n2) const {
    return element<t>(valid, cell, cj, n0, n1, n2);
  }

  template <int t>
  __device__ R element(bool valid, int cell, int cj, const V& n0, const V& n1, const V& n2) const {
    R r;
    if (!valid) {
#pragma unroll
      for (int c = 0; c < NRC; ++c) r.c[c] = T(0);
      return r;
    }
    constexpr int NE = elems_per_cell(KIND);
    const T ihx = cs.ihx, ihy = cs.ihy;
    // stress of the state: sigma = A0 (eps(u) - eps0)
    T exx = ihx * (T(gx(KIND, t, 0)) * n0.ux + T(gx(KIND, t, 1)) * n1.ux + T(gx(KIND, t, 2)) * n2.ux);
    T eyy = ihy * (T(gy(KIND, t, 0)) * n0.uy + T(gy(KIND, t, 1)) * n1.uy + T(gy(KIND, t, 2)) * n2.uy);
    T gxy = ihy * (T(gy(KIND, t, 0)) * n0.ux + T(gy(KIND, t, 1)) * n1.ux + T(gy(KIND, t, 2)) * n2.ux) +
            ihx * (T(gx(KIND, t, 0)) * n0.uy + T(gx(KIND, t, 1)) * n1.uy + T(gx(KIND, t, 2)) * n2.uy);
    if (args.eig) {
      T e0 = args.eig[cj * NE + t];
      exx -= e0;
      eyy -= e0;
    }
    const T sxx = cs.lam2mu * exx + cs.lam * eyy, syy = cs.lam * exx + cs.lam2mu * eyy,
            sxy = cs.mu * gxy;
    const T Sa = n0.a + n1.a + n2.a;
    const T area = cs.area;
    if (!TRANSPOSE) {
      // s_T = sum_j int_T a'(alpha_h) phi_j x_alpha,j
      const T w0 = T(-2) * area * (T(1.0 / 3.0) - (n0.a + Sa) * T(1.0 / 12.0));
      const T w1 = T(-2) * area * (T(1.0 / 3.0) - (n1.a + Sa) * T(1.0 / 12.0));
      const T w2 = T(-2) * area * (T(1.0 / 3.0) - (n2.a + Sa) * T(1.0 / 12.0));
      const T sT = w0 * n0.x0 + w1 * n1.x0 + w2 * n2.x0;
      r.c[0] = sT * sxx;
      r.c[1] = sT * syy;
      r.c[2] = sT * sxy;
    } else {
      // e_T = sigma : eps(x_u); node j receives -2|T| (1/3 - (alpha_j + S_a)/12) e_T
      T dxx = ihx * (T(gx(KIND, t, 0)) * n0.x0 + T(gx(KIND, t, 1)) * n1.x0 + T(gx(KIND, t, 2)) * n2.x0);
      T dyy = ihy * (T(gy(KIND, t, 0)) * n0.x1 + T(gy(KIND, t, 1)) * n1.x1 + T(gy(KIND, t, 2)) * n2.x1);
      T dxy = ihy * (T(gy(KIND, t, 0)) * n0.x0 + T(gy(KIND, t, 1)) * n1.x0 + T(gy(KIND, t, 2)) * n2.x0) +
              ihx * (T(gx(KIND, t, 0)) * n0.x1 + T(gx(KIND, t, 1)) * n1.x1 + T(gx(KIND, t, 2)) * n2.x1);
      const T eT = sxx * dxx + syy * dyy + sxy * dxy;
      r.c[0] = T(-2) * area * eT * (T(1.0 / 3.0) - Sa * T(1.0 / 12.0));  // node-independent part
      r.c[1] = T(2) * area * eT * T(1.0 / 12.0);                         // times alpha_j
    }
    return r;
  }

  template <int t, int k>
  __device__ void add(Acc& a, const R& r) const {
    if (!TRANSPOSE) {
      constexpr int cx = gx(KIND, t, k), cy = gy(KIND, t, k);
      if (cx != 0) {
        a.c[0] += T(cx) * r.c[0];
        a.c[2] += T(cx) * r.c[2];
      }
      if (cy != 0) {
        a.c[1] += T(cy) * r.c[2];
        a.c[3] += T(cy) * r.c[1];
      }
    } else {
      a.c[0] += r.c[0];
      a.c[1] += r.c[1];
    }
  }

  __device__ void store(int node, int X2, int Y2, const V& own, const Acc& a,
                        RT (&red)[1]) const {
    if (!TRANSPOSE) {
      T fx = cs.ihx * a.c[0] + cs.ihy * a.c[1];
      T fy = cs.ihx * a.c[2] + cs.ihy * a.c[3];
      if (is_fixed(g, X2, Y2, 0)) fx = T(0);
      if (is_fixed(g, X2, Y2, 1)) fy = T(0);
      if (args.accumulate) {
        fx += args.y[2 * node];
        fy += args.y[2 * node + 1];
      }
      args.y[2 * node] = fx;
      args.y[2 * node + 1] = fy;
    } else {
      T f = a.c[0] + a.c[1] * own.a;
      if (args.excl && args.excl[node]) f = T(0);
      if (args.accumulate) f += args.y[node];
      args.y[node] = f;
    }
  }
};

}  // namespace pf
