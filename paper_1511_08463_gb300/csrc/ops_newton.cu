// Launchers of the coupling block of the Newton Jacobian (Section 3.3, eq. offdiag) and the
// small vector kernels of MINRES.
#include "kernels.cuh"

namespace pf {

template <class Op>
static void launch_op(cudaStream_t s, const Op& op, int id, double bytes) {
  dim3 block(TX, TY);
  dim3 grid((op.g.nx + 1 + TX - 1) / TX, (op.g.ny + 1 + TY - 1) / TY);
  PF_LAUNCH(id, bytes, s, pdl_launch(stencil_kernel<Op>, grid, block, 0, s, op));
}

template <class T, int K, bool TR>
static void go(cudaStream_t s, const Grid& g, const Mat& m, const CouplingArgs<T>& a) {
  CouplingOp<T, K, TR> op;
  op.g = g;
  op.m = m;
  op.cs = make_consts<T>(g, m);
  op.args = a;
  const double t = sizeof(T);
  const double bytes = double(g.n) * t * (TR ? 2 + 3 + 1 : 1 + 3 + 2) + (a.accumulate ? double(g.n) * t : 0.0);
  launch_op(s, op, kclass(KC_VECTOR, sizeof(T) == 8, false), bytes);
}

template <class T>
void launch_coupling(cudaStream_t s, const Grid& g, const Mat& m, bool transpose,
                     const CouplingArgs<T>& a) {
  if (g.kind == CROSSED)
    transpose ? go<T, CROSSED, true>(s, g, m, a) : go<T, CROSSED, false>(s, g, m, a);
  else
    transpose ? go<T, RIGHT, true>(s, g, m, a) : go<T, RIGHT, false>(s, g, m, a);
}
template void launch_coupling<double>(cudaStream_t, const Grid&, const Mat&, bool,
                                      const CouplingArgs<double>&);
template void launch_coupling<float>(cudaStream_t, const Grid&, const Mat&, bool,
                                     const CouplingArgs<float>&);

// z = a x + b y + c z (c == 0: z not read); scalars from the host
template <class T>
__global__ void k_lincomb(T* z, T a, const T* x, T b, const T* y, T c, size_t n) {
  pdl_enter();
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T v = a * x[i];
  if (y) v += b * y[i];
  if (c != T(0)) v += c * z[i];
  z[i] = v;
}
template <class T>
void vec_lincomb(cudaStream_t s, T* z, T a, const T* x, T b, const T* y, T c, size_t n) {
  if (n == 0) return;
  PF_LAUNCH(kclass(KC_VECTOR, sizeof(T) == 8, false), 3.0 * n * sizeof(T), s,
            pdl_launch(k_lincomb<T>, (unsigned)((n + 255) / 256), 256, 0, s, z, a, x, b, y, c, n));
}
template void vec_lincomb<double>(cudaStream_t, double*, double, const double*, double,
                                  const double*, double, size_t);
template void vec_lincomb<float>(cudaStream_t, float*, float, const float*, float, const float*,
                                 float, size_t);

// Newton trial point: u = u0 + mu du on free dofs; alpha = clip(alpha0 + mu dalpha, lo, hi); alpha32 copy
__global__ void k_newton_trial(Grid g, double* u, const double* u0, const double* du, double* alpha,
                               const double* a0, const double* da, const double* lo, float* a32,
                               double mu) {
  pdl_enter();
  int node = blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.n) return;
  int X2, Y2;
  node_coords(g, node, X2, Y2);
  // prescribed displacement components keep their lifted values
  for (int c = 0; c < 2; ++c)
    u[2 * node + c] = u0[2 * node + c] + (is_fixed(g, X2, Y2, c) ? 0.0 : mu * du[2 * node + c]);
  const double l = lo[node], h = is_fixed(g, X2, Y2, 2) ? l : 1.0;
  const double an = fmin(fmax(a0[node] + mu * da[node], l), h);
  alpha[node] = an;
  a32[node] = (float)an;
}
void newton_trial(cudaStream_t s, const Grid& g, double* u, const double* u0, const double* du,
                  double* alpha, const double* a0, const double* da, const double* lo, float* a32,
                  double mu) {
  PF_LAUNCH(kclass(KC_VECTOR, true, false), 0.0, s,
            pdl_launch(k_newton_trial, (unsigned)((g.n + 255) / 256), 256, 0, s, g, u, u0, du, alpha, a0, da,
                                                                         lo, a32, mu));
}

}  // namespace pf
