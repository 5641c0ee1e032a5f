// Launchers of the damage stencil operator H(q) and the damage gradient / MCP residual
// (Section 1.2, eq. helmholtz; Section 2.4).
#include "kernels.cuh"

namespace pf {

template <class T>
static double damage_bytes(const Grid& g, int mode, const DamageArgs<T>& a) {
  const double t = sizeof(T);
  double node = 0.0;
  switch (mode) {
    case M_APPLY: node = 2 * t; break;
    case M_MASKED: node = 2 * t; break;
    case M_RESB: node = (a.x0b ? 4 : 3) * t; break;  // x, b, r (x0b: b, dinv, r, x written)
    case M_CHEB: node = ((a.x ? 1 : 0) + (a.d ? 1 : 0) + 4) * t; break;  // b, dinv, y, d' (+ x, d)
    case M_GRAD: node = 5 * t + 1; break;
    case M_TRIAL: node = 7 * t + 1; break;
  }
  if (a.excl) node += 1;
  const double xc = (mode == M_CHEB && a.xc) ? double(a.gc.n) * t : 0.0;  // fused prolongation
  return double(g.n) * node + double(g.nelem) * t + xc;
}

template <class Op, int TYV>
static void launch_tile(cudaStream_t s, const Op& op, int id, double bytes) {
  dim3 block(TX, TYV);
  dim3 grid((op.g.nx + 1 + TX - 1) / TX, (op.g.ny + 1 + TYV - 1) / TYV);
  PF_LAUNCH(id, bytes, s, pdl_launch(stencil_kernel<Op, TYV>, grid, block, 0, s, op));
}
// FP32 operators run with the level's tile height (TY_MIN, TY or 16 rows, Grid::tile_rows);
// FP64 operators always with TY
template <class Op>
static void launch_op(cudaStream_t s, const Op& op, int id, double bytes) {
  if constexpr (sizeof(typename Op::Scalar) == 4) {
    if (op.g.tile_rows == TY_MIN) return launch_tile<Op, TY_MIN>(s, op, id, bytes);
    if (op.g.tile_rows == 16) return launch_tile<Op, 16>(s, op, id, bytes);
  }
  launch_tile<Op, TY>(s, op, id, bytes);
}

template <class T, int K, int M, bool D>
static void go(cudaStream_t s, const Grid& g, const Mat& m, const DamageArgs<T>& a) {
  if constexpr (std::is_same<T, double>::value && (M == M_GRAD || M == M_TRIAL)) {
    if (a.df) {  // the mixed path's gradient / trial point: FP64 data, double-float arithmetic
      DamageOp<T, K, M, D, dfloat> op;
      op.g = g;
      op.m = m;
      op.cs = make_consts<dfloat>(g, m);
      op.args = a;
      launch_op(s, op, kclass(M == M_GRAD ? KC_DM_GRAD_DF : KC_DM_TRIAL_DF, true, a.coarse),
                damage_bytes<T>(g, M, a));
      return;
    }
  }
  const int base = M == M_APPLY ? KC_DM_APPLY : M == M_MASKED ? KC_DM_MASKED
                 : M == M_RESB ? (a.x0b ? KC_DM_RESB_Z : KC_DM_RESB)
                 : M == M_CHEB ? (a.x0b ? KC_DM_CHEB_Z : KC_DM_CHEB) : M == M_GRAD ? KC_DM_GRAD : KC_DM_TRIAL;
  DamageOp<T, K, M, D> op;
  op.g = g;
  op.m = m;
  op.cs = make_consts<T>(g, m);
  op.args = a;
  launch_op(s, op, kclass(base, sizeof(T) == 8, a.coarse), damage_bytes<T>(g, M, a));
}

template <class T, int K>
static void dispatch(cudaStream_t s, const Grid& g, const Mat& m, int mode, bool dot,
                     const DamageArgs<T>& a) {
  switch (mode) {
    case M_APPLY: return go<T, K, M_APPLY, false>(s, g, m, a);
    case M_MASKED:
      return dot ? go<T, K, M_MASKED, true>(s, g, m, a) : go<T, K, M_MASKED, false>(s, g, m, a);
    case M_RESB: return go<T, K, M_RESB, false>(s, g, m, a);
    case M_CHEB:
      return dot ? go<T, K, M_CHEB, true>(s, g, m, a) : go<T, K, M_CHEB, false>(s, g, m, a);
  }
  if constexpr (sizeof(T) == 8) {
    if (mode == M_GRAD) return go<T, K, M_GRAD, false>(s, g, m, a);
    if (mode == M_TRIAL) return go<T, K, M_TRIAL, false>(s, g, m, a);
  }
}

template <class T>
void launch_damage(cudaStream_t s, const Grid& g, const Mat& m, int mode, bool dot,
                   const DamageArgs<T>& a) {
  if (g.kind == CROSSED)
    dispatch<T, CROSSED>(s, g, m, mode, dot, a);
  else
    dispatch<T, RIGHT>(s, g, m, mode, dot, a);
}

template void launch_damage<double>(cudaStream_t, const Grid&, const Mat&, int, bool,
                                    const DamageArgs<double>&);
template void launch_damage<float>(cudaStream_t, const Grid&, const Mat&, int, bool,
                                   const DamageArgs<float>&);

}  // namespace pf
