// Per-node building blocks of the P1 operators and multigrid transfers on the structured meshes,
// shared by the grid-wide kernels and the single-block coarse-level kernel.
#pragma once
#include "pf_core.cuh"

namespace pf {

__device__ __forceinline__ void cell_nodes(const Grid& g, int ci, int cj, int t, int& n0, int& n1,
                                           int& n2) {
  int v00 = cj * (g.nx + 1) + ci, v10 = v00 + 1, v01 = v00 + g.nx + 1, v11 = v01 + 1;
  if (g.kind == CROSSED) {
    int c = g.nv + cj * g.nx + ci;
    if (t == 0) { n0 = v00; n1 = v10; n2 = c; }
    else if (t == 1) { n0 = v10; n1 = v11; n2 = c; }
    else if (t == 2) { n0 = v11; n1 = v01; n2 = c; }
    else { n0 = v01; n1 = v00; n2 = c; }
  } else {
    if (t == 0) { n0 = v00; n1 = v10; n2 = v11; }
    else { n0 = v00; n1 = v11; n2 = v01; }
  }
}

__device__ __forceinline__ int gxr(int kind, int t, int k) { return gx(kind, t, k); }
__device__ __forceinline__ int gyr(int kind, int t, int k) { return gy(kind, t, k); }

// element (cell offset, element type, local index) lists around a node
__device__ __forceinline__ int node_elements(const Grid& g, int node, int* cells, int* ts,
                                             int* ks) {
  int cnt = 0;
  auto push = [&](int ci, int cj, int t, int k) {
    if (ci >= 0 && ci < g.nx && cj >= 0 && cj < g.ny) {
      cells[cnt] = cj * g.nx + ci;
      ts[cnt] = t;
      ks[cnt] = k;
      ++cnt;
    }
  };
  if (node < g.nv) {
    int j = node / (g.nx + 1), i = node - j * (g.nx + 1);
    if (g.kind == CROSSED) {
      push(i, j, 0, 0); push(i, j, 3, 1);
      push(i - 1, j, 0, 1); push(i - 1, j, 1, 0);
      push(i - 1, j - 1, 1, 1); push(i - 1, j - 1, 2, 0);
      push(i, j - 1, 2, 1); push(i, j - 1, 3, 0);
    } else {
      push(i, j, 0, 0); push(i, j, 1, 0);
      push(i - 1, j, 0, 1);
      push(i - 1, j - 1, 0, 2); push(i - 1, j - 1, 1, 1);
      push(i, j - 1, 1, 2);
    }
  } else {
    int c = node - g.nv, j = c / g.nx, i = c - j * g.nx;
    for (int t = 0; t < 4; ++t) push(i, j, t, 2);
  }
  return cnt;
}

template <class T>
__device__ __forceinline__ T fget(const Grid& gf, const T* v, bool centre, int i, int j, int c,
                                  int ncomp) {
  if (!centre) {
    if (i < 0 || i > gf.nx || j < 0 || j > gf.ny) return T(0);
    return v[(j * (gf.nx + 1) + i) * ncomp + c];
  }
  if (i < 0 || i >= gf.nx || j < 0 || j >= gf.ny) return T(0);
  return v[(gf.nv + j * gf.nx + i) * ncomp + c];
}

// (P^T r_f)(node), component c, at coarse doubled coordinates (X2, Y2): P1 interpolation
// weights 1 at the coincident fine vertex and 1/2 at its fine neighbours.
template <class T>
__device__ __forceinline__ T restrict_value(const Grid& gf, int ncomp, const T* rf, int X2, int Y2,
                                            int c) {
  T acc;
  if ((X2 & 1) == 0) {  // coarse vertex (I, J) = fine vertex (2I, 2J)
    int i = X2, j = Y2;  // fine vertex indices 2I, 2J
    acc = fget(gf, rf, false, i, j, c, ncomp);
    T h = fget(gf, rf, false, i - 1, j, c, ncomp) + fget(gf, rf, false, i + 1, j, c, ncomp) +
          fget(gf, rf, false, i, j - 1, c, ncomp) + fget(gf, rf, false, i, j + 1, c, ncomp);
    if (gf.kind == RIGHT) {
      h += fget(gf, rf, false, i + 1, j + 1, c, ncomp) + fget(gf, rf, false, i - 1, j - 1, c, ncomp);
    } else {
      h += fget(gf, rf, true, i, j, c, ncomp) + fget(gf, rf, true, i - 1, j, c, ncomp) +
           fget(gf, rf, true, i, j - 1, c, ncomp) + fget(gf, rf, true, i - 1, j - 1, c, ncomp);
    }
    acc += T(0.5) * h;
  } else {  // coarse centre (I, J) = fine vertex (2I+1, 2J+1)
    int I = X2 / 2, J = Y2 / 2;
    acc = fget(gf, rf, false, 2 * I + 1, 2 * J + 1, c, ncomp);
    T h = fget(gf, rf, true, 2 * I, 2 * J, c, ncomp) + fget(gf, rf, true, 2 * I + 1, 2 * J, c, ncomp) +
          fget(gf, rf, true, 2 * I, 2 * J + 1, c, ncomp) +
          fget(gf, rf, true, 2 * I + 1, 2 * J + 1, c, ncomp);
    acc += T(0.5) * h;
  }
  return acc;
}

// b_c(node) = (P^T r_f)(node) for every component; zero on prescribed and excluded coarse dofs.
template <class T>
__device__ __forceinline__ void restrict_node(const Grid& gf, const Grid& gc, int ncomp,
                                              int comp_base, const T* rf, T* bc,
                                              const uint8_t* excl_c, int node) {
  int X2, Y2;
  node_coords(gc, node, X2, Y2);
  for (int c = 0; c < ncomp; ++c) {
    T acc = restrict_value(gf, ncomp, rf, X2, Y2, c);
    if (is_fixed(gc, X2, Y2, comp_base + c) || (excl_c && excl_c[node])) acc = T(0);
    bc[node * ncomp + c] = acc;
  }
}

template <class T>
__device__ __forceinline__ T cget(const Grid& gc, const T* v, bool centre, int I, int J, int c,
                                  int ncomp) {
  if (!centre) return v[(J * (gc.nx + 1) + I) * ncomp + c];
  return v[(gc.nv + J * gc.nx + I) * ncomp + c];
}

// (P x_c)(node), component c: P1 interpolation from the nested coarse grid (weight 1 at a
// coincident coarse node, 1/2 at the two coarse nodes of the coarse edge the fine node bisects).
template <class T>
__device__ __forceinline__ T prolong_value(const Grid& gf, const Grid& gc, int ncomp, const T* xc,
                                           int node, int X2, int Y2, int c) {
  if (node < gf.nv) {
    int i = X2 / 2, j = Y2 / 2, I = i >> 1, J = j >> 1, pi = i & 1, pj = j & 1;
    if (!pi && !pj) return cget(gc, xc, false, I, J, c, ncomp);
    if (pi && !pj) return T(0.5) * (cget(gc, xc, false, I, J, c, ncomp) + cget(gc, xc, false, I + 1, J, c, ncomp));
    if (!pi && pj) return T(0.5) * (cget(gc, xc, false, I, J, c, ncomp) + cget(gc, xc, false, I, J + 1, c, ncomp));
    if (gf.kind == RIGHT)
      return T(0.5) * (cget(gc, xc, false, I, J, c, ncomp) + cget(gc, xc, false, I + 1, J + 1, c, ncomp));
    return cget(gc, xc, true, I, J, c, ncomp);
  }
  int cc = node - gf.nv, j = cc / gf.nx, i = cc - j * gf.nx;
  int I = i >> 1, J = j >> 1, pi = i & 1, pj = j & 1;
  return T(0.5) * (cget(gc, xc, false, I + pi, J + pj, c, ncomp) + cget(gc, xc, true, I, J, c, ncomp));
}

// The same interpolation as prolong_value, as the mean of two coarse nodes (a == b at a fine node
// that coincides with a coarse one): (P x_c)(node) = (x_c[a] + x_c[b]) / 2, with no branch on
// the node's parity, so that all components can be read with one access per coarse node.
__device__ __forceinline__ void prolong_nodes(const Grid& gf, const Grid& gc, int node, int X2,
                                              int Y2, int& a, int& b) {
  if (node < gf.nv) {
    const int i = X2 / 2, j = Y2 / 2, I = i >> 1, J = j >> 1, pi = i & 1, pj = j & 1;
    if (gf.kind == CROSSED && pi && pj) {  // fine vertex at a coarse cell centre
      a = b = gc.nv + J * gc.nx + I;
    } else {
      a = J * (gc.nx + 1) + I;
      b = (J + pj) * (gc.nx + 1) + I + pi;
    }
  } else {
    const int cc = node - gf.nv, j = cc / gf.nx, i = cc - j * gf.nx;
    const int I = i >> 1, J = j >> 1;
    a = (J + (j & 1)) * (gc.nx + 1) + I + (i & 1);
    b = gc.nv + J * gc.nx + I;
  }
}

// x_f(node) += (P x_c)(node) (P1 interpolation), except on prescribed and excluded fine dofs.
template <class T>
__device__ __forceinline__ void prolong_node(const Grid& gf, const Grid& gc, int ncomp,
                                             int comp_base, const T* xc, T* xf,
                                             const uint8_t* excl, int node) {
  int X2, Y2;
  node_coords(gf, node, X2, Y2);
  bool ex = excl && excl[node];
  for (int c = 0; c < ncomp; ++c) {
    T v = prolong_value(gf, gc, ncomp, xc, node, X2, Y2, c);
    if (ex || is_fixed(gf, X2, Y2, comp_base + c)) v = T(0);
    xf[node * ncomp + c] += v;
  }
}

}  // namespace pf
