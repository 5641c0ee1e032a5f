// Launchers of the elasticity stencil operator K(alpha) (Section 1.2, eq. elasticity).
#include "kernels.cuh"

namespace pf {

// algorithmic bytes of one launch: compulsory reads and writes of the operator on its grid
template <class T>
static double elastic_bytes(const Grid& g, int coef, int mode, const ElasticArgs<T>& a) {
  const double t = sizeof(T);
  double node = 0.0;
  switch (mode) {
    case M_APPLY:
    case M_MASKED: node = 4 * t; break;
    case M_RESB: node = (a.x0b ? 8 : 6) * t; break;  // x, b, r (x0b: b, dinv, r, x written)
    case M_RESID: node = 4 * t; break;
    case M_CHEB: node = ((a.x ? 2 : 0) + (a.d ? 2 : 0) + 8) * t; break;  // b, dinv, y, d' (+ x, d)
  }
  double coefb = coef == COEF_ALPHA ? double(g.n) * t : double(g.nelem) * t;
  if (mode == M_CHEB && a.xc) coefb += 2.0 * a.gc.n * t;  // fused prolongation: coarse x
  return double(g.n) * node + coefb;
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

template <class T, int K, int C, int M, bool E, bool D>
static void go(cudaStream_t s, const Grid& g, const Mat& m, const ElasticArgs<T>& a) {
  if constexpr (std::is_same<T, double>::value && M == M_RESID) {
    if (a.df) {  // the mixed path's physical residual: FP64 data, double-float arithmetic
      ElasticOp<T, K, C, M, E, D, dfloat> op;
      op.g = g;
      op.m = m;
      op.cs = make_consts<dfloat>(g, m);
      op.args = a;
      launch_op(s, op, kclass(KC_EL_RESID_DF, true, a.coarse), elastic_bytes<T>(g, C, M, a));
      return;
    }
  }
  const int base = M == M_APPLY ? KC_EL_APPLY : M == M_MASKED ? KC_EL_MASKED
                 : M == M_RESB ? (a.x0b ? KC_EL_RESB_Z : KC_EL_RESB)
                 : M == M_RESID ? KC_EL_RESID : (a.x0b ? KC_EL_CHEB_Z : KC_EL_CHEB);
  ElasticOp<T, K, C, M, E, D> op;
  op.g = g;
  op.m = m;
  op.cs = make_consts<T>(g, m);
  op.args = a;
  launch_op(s, op, kclass(base, sizeof(T) == 8, a.coarse), elastic_bytes<T>(g, C, M, a));
}

template <class T, int K>
static void dispatch(cudaStream_t s, const Grid& g, const Mat& m, int coef, int mode, bool eigen,
                     bool dot, const ElasticArgs<T>& a) {
  if (coef == COEF_ALPHA) {
    switch (mode) {
      case M_APPLY: return go<T, K, COEF_ALPHA, M_APPLY, false, false>(s, g, m, a);
      case M_MASKED:
        return dot ? go<T, K, COEF_ALPHA, M_MASKED, false, true>(s, g, m, a)
                   : go<T, K, COEF_ALPHA, M_MASKED, false, false>(s, g, m, a);
      case M_RESB: return go<T, K, COEF_ALPHA, M_RESB, false, false>(s, g, m, a);
      case M_RESID:
        return eigen ? go<T, K, COEF_ALPHA, M_RESID, true, false>(s, g, m, a)
                     : go<T, K, COEF_ALPHA, M_RESID, false, false>(s, g, m, a);
      case M_CHEB: return go<T, K, COEF_ALPHA, M_CHEB, false, false>(s, g, m, a);
    }
  } else {
    switch (mode) {
      case M_APPLY: return go<T, K, COEF_ELEM, M_APPLY, false, false>(s, g, m, a);
      case M_MASKED:
        return dot ? go<T, K, COEF_ELEM, M_MASKED, false, true>(s, g, m, a)
                   : go<T, K, COEF_ELEM, M_MASKED, false, false>(s, g, m, a);
      case M_RESB: return go<T, K, COEF_ELEM, M_RESB, false, false>(s, g, m, a);
      case M_CHEB:
        return dot ? go<T, K, COEF_ELEM, M_CHEB, false, true>(s, g, m, a)
                   : go<T, K, COEF_ELEM, M_CHEB, false, false>(s, g, m, a);
    }
  }
}

template <class T>
void launch_elastic(cudaStream_t s, const Grid& g, const Mat& m, int coef, int mode, bool eigen,
                    bool dot, const ElasticArgs<T>& a) {
  if (g.kind == CROSSED)
    dispatch<T, CROSSED>(s, g, m, coef, mode, eigen, dot, a);
  else
    dispatch<T, RIGHT>(s, g, m, coef, mode, eigen, dot, a);
}

template void launch_elastic<double>(cudaStream_t, const Grid&, const Mat&, int, int, bool, bool,
                                     const ElasticArgs<double>&);
template void launch_elastic<float>(cudaStream_t, const Grid&, const Mat&, int, int, bool, bool,
                                    const ElasticArgs<float>&);

}  // namespace pf
