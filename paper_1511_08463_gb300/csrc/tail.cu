// The coarse end of the multigrid V-cycle in one thread block.
//
// Below a few thousand nodes every level of the hierarchy is latency-bound: each smoothing step,
// residual and transfer launched as its own grid costs several microseconds of launch and
// memory latency for a few microseconds' worth of arithmetic.  From the first level whose data
// (and that of all coarser levels) fits in one SM's shared memory, this kernel runs the rest of
// the V-cycle -- Chebyshev pre-smoothing, residual, restriction down to the coarsest level, the
// dense coarsest solve, then prolongation and post-smoothing back up -- with block barriers
// between the steps instead of kernel boundaries.  Same operations as the grid-wide path (the
// l1-Jacobi Chebyshev smoother on [0.1, 1], P1 transfers, masks for prescribed and active dofs,
// coarsest solve with the stored inverse, the Chebyshev coefficients the host computed for it);
// operators are applied in gather form per node, so sums run in a different order than in the
// tiled kernels.  Given the finer level's residual, the kernel forms its own right-hand side by
// restriction as it loads the level.  FP32 only.
#include "kernels.cuh"
#include "mg_core.cuh"

namespace pf {

namespace {

// Operator of the tail: the tiled kernels' own element and gather code (ElasticOp / DamageOp with
// per-element coefficients), applied to a whole level held in shared memory.
template <int KIND, int NC>
struct TailOp;
template <int KIND>
struct TailOp<KIND, 2> {
  using Op = ElasticOp<float, KIND, COEF_ELEM, M_APPLY, false, false>;
  static __device__ typename Op::V val(const float* x, int node) {
    return typename Op::V{x[2 * node], x[2 * node + 1]};
  }
  static __device__ void result(const Op& op, const typename Op::Acc& a, const typename Op::V&,
                                float* f) {
    f[0] = op.cs.ihx * a.ax + op.cs.ihy * a.bx;
    f[1] = op.cs.ihx * a.ay + op.cs.ihy * a.by;
  }
  static __device__ Op make(const TailLevel& L, const float* coef) {
    Op op;
    op.g = L.g;
    op.cs = L.cs;
    op.args = ElasticArgs<float>{};
    op.args.coef = coef;
    return op;
  }
};
template <int KIND>
struct TailOp<KIND, 1> {
  using Op = DamageOp<float, KIND, M_APPLY, false>;
  static __device__ typename Op::V val(const float* x, int node) { return typename Op::V{x[node]}; }
  static __device__ void result(const Op&, const typename Op::Acc& a, const typename Op::V& own,
                                float* f) {
    f[0] = a.P + a.M * own.p + a.X + a.Y;
  }
  static __device__ Op make(const TailLevel& L, const float* coef) {
    Op op;
    op.g = L.g;
    op.cs = L.cs;
    op.args = DamageArgs<float>{};
    op.args.w = coef;
    return op;
  }
};

struct TailBufs {
  float *x, *xn, *b, *d, *dinv, *coef;
  uint8_t* excl;  // damage: excluded nodes (restriction / prolongation masks); elastic: null
  uint8_t* fz;    // per node: bit c set if component c takes no update (prescribed or excluded)
};

__device__ __forceinline__ TailBufs bufs(float* sm, const TailLevel& L) {
  TailBufs B;
  B.x = sm + L.ox;
  B.xn = sm + L.oxn;
  B.b = sm + L.ob;
  B.d = sm + L.od;
  B.dinv = sm + L.odi;
  B.coef = sm + L.oc;
  B.fz = reinterpret_cast<uint8_t*>(sm + L.oe);
  B.excl = L.excl ? B.fz + L.g.n : nullptr;
  return B;
}

// f = A x on every node of the level, handed node by node to `use(node, own, f)`.  Pass 1: one
// record per element into rec (component-major); pass 2: each node gathers the records of its
// elements in the tiled kernel's order.  Ends with the block barrier after pass 2.
template <int KIND, int NC, class Use>
__device__ void apply_level(const TailLevel& L, const float* coef, const float* x, float* rec,
                            Use use) {
  using TO = TailOp<KIND, NC>;
  using Op = typename TO::Op;
  using R = typename Op::R;
  constexpr int NE = elems_per_cell(KIND);
  constexpr int NRC = Op::NRC;
  const Op op = TO::make(L, coef);
  const Grid& g = L.g;
  const int ne = g.nelem;
  for (int c = threadIdx.x; c < g.ncell; c += blockDim.x) {
    const int cj = c / g.nx, ci = c - cj * g.nx;
    const int v00 = cj * (g.nx + 1) + ci;
    const auto a00 = TO::val(x, v00), a10 = TO::val(x, v00 + 1);
    const auto a01 = TO::val(x, v00 + g.nx + 1), a11 = TO::val(x, v00 + g.nx + 2);
    R r[NE];
    if constexpr (KIND == CROSSED) {
      const auto ac = TO::val(x, g.nv + c);
      r[0] = op.template element<0>(true, c, cj, a00, a10, ac);
      r[1] = op.template element<1>(true, c, cj, a10, a11, ac);
      r[2] = op.template element<2>(true, c, cj, a11, a01, ac);
      r[3] = op.template element<3>(true, c, cj, a01, a00, ac);
    } else {
      r[0] = op.template element<0>(true, c, cj, a00, a10, a11);
      r[1] = op.template element<1>(true, c, cj, a00, a11, a01);
    }
#pragma unroll
    for (int t = 0; t < NE; ++t)
#pragma unroll
      for (int q = 0; q < NRC; ++q) rec[q * ne + c * NE + t] = r[t].c[q];
  }
  __syncthreads();
  auto get = [&](int ci, int cj, int t) {
    R r;
    const int e = (cj * g.nx + ci) * NE + t;
#pragma unroll
    for (int q = 0; q < NRC; ++q) r.c[q] = rec[q * ne + e];
    return r;
  };
  for (int node = threadIdx.x; node < g.n; node += blockDim.x) {
    typename Op::Acc a = Op::acc0();
    if (node < g.nv) {
      const int j = node / (g.nx + 1), i = node - j * (g.nx + 1);
      const bool cR = i < g.nx, cL = i > 0, cU = j < g.ny, cD = j > 0;
      if constexpr (KIND == CROSSED) {
        if (cR && cU) { op.template add<0, 0>(a, get(i, j, 0)); op.template add<3, 1>(a, get(i, j, 3)); }
        if (cL && cU) { op.template add<0, 1>(a, get(i - 1, j, 0)); op.template add<1, 0>(a, get(i - 1, j, 1)); }
        if (cL && cD) { op.template add<1, 1>(a, get(i - 1, j - 1, 1)); op.template add<2, 0>(a, get(i - 1, j - 1, 2)); }
        if (cR && cD) { op.template add<2, 1>(a, get(i, j - 1, 2)); op.template add<3, 0>(a, get(i, j - 1, 3)); }
      } else {
        if (cR && cU) { op.template add<0, 0>(a, get(i, j, 0)); op.template add<1, 0>(a, get(i, j, 1)); }
        if (cL && cU) op.template add<0, 1>(a, get(i - 1, j, 0));
        if (cL && cD) { op.template add<0, 2>(a, get(i - 1, j - 1, 0)); op.template add<1, 1>(a, get(i - 1, j - 1, 1)); }
        if (cR && cD) op.template add<1, 2>(a, get(i, j - 1, 1));
      }
    } else if constexpr (KIND == CROSSED) {
      const int c = node - g.nv, j = c / g.nx, i = c - j * g.nx;
      op.template add<0, 2>(a, get(i, j, 0));
      op.template add<1, 2>(a, get(i, j, 1));
      op.template add<2, 2>(a, get(i, j, 2));
      op.template add<3, 2>(a, get(i, j, 3));
    }
    const auto own = TO::val(x, node);
    float f[NC];
    TO::result(op, a, own, f);
    use(node, f);
  }
  __syncthreads();
}

// `steps` Chebyshev steps on D_l1^{-1} A over [0.1, 1] with the grid-wide smoother's recurrence
// coefficients (computed once on the host) and update; the new iterate goes to xn and the
// buffers are swapped, as the grid-wide path rotates them.
template <int KIND, int NC>
__device__ void smooth(const TailArgs& a, const TailLevel& L, TailBufs& B, float* rec,
                       bool from_zero, int steps) {
  const int nd = NC * L.g.n;
  int k0 = 0;
  if (from_zero && steps > 0) {  // the first step from zero is pointwise: x = d = c0 D^-1 b
    const float c0 = a.cheb_cr[0];
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
      const int node = i / NC, c = i - node * NC;
      const float v = (B.fz[node] >> c) & 1 ? 0.f : c0 * B.dinv[i] * B.b[i];
      B.d[i] = v;
      B.x[i] = v;
    }
    __syncthreads();
    k0 = 1;
  }
  for (int k = k0; k < steps; ++k) {
    const float cd = a.cheb_cd[k], cr = a.cheb_cr[k];
    const bool first = k == 0;
    apply_level<KIND, NC>(L, B.coef, B.x, rec, [&](int node, const float* f) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int i = NC * node + c;
        const float dp = first ? 0.f : B.d[i];
        const float dn = (B.fz[node] >> c) & 1 ? 0.f : cd * dp + cr * B.dinv[i] * (B.b[i] - f[c]);
        B.d[i] = dn;
        B.xn[i] = B.x[i] + dn;
      }
    });
    float* t = B.x;
    B.x = B.xn;
    B.xn = t;
  }
}

template <int KIND, int NC>
__global__ void __launch_bounds__(TAIL_THREADS) k_tail_vcycle(TailArgs a) {
  pdl_enter();
  extern __shared__ float sm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  float* rec = sm + a.orec;
  TailBufs B[MAX_TAIL];
  for (int l = 0; l < a.nl; ++l) {
    const TailLevel& L = a.L[l];
    B[l] = bufs(sm, L);
    const int nd = NC * L.g.n;
    for (int i = tid; i < nd; i += nt) B[l].dinv[i] = L.dinv[i];
    for (int i = tid; i < L.g.nelem; i += nt) B[l].coef[i] = L.coef[i];
    for (int node = tid; node < L.g.n; node += nt) {
      int X2, Y2;
      node_coords(L.g, node, X2, Y2);
      uint8_t f = 0;
      if (NC == 2) {
        f = (is_fixed(L.g, X2, Y2, 0) ? 1 : 0) | (is_fixed(L.g, X2, Y2, 1) ? 2 : 0);
      } else {
        const bool ex = L.excl[node] != 0;
        B[l].excl[node] = ex ? 1 : 0;
        f = (ex || is_fixed(L.g, X2, Y2, 2)) ? 1 : 0;
      }
      B[l].fz[node] = f;
    }
  }
  if (a.rf) {
    for (int node = tid; node < a.L[0].g.n; node += nt)
      restrict_node(a.gf, a.L[0].g, NC, NC == 2 ? 0 : 2, a.rf, B[0].b, a.L[0].excl, node);
  } else {
    for (int i = tid; i < NC * a.L[0].g.n; i += nt) B[0].b[i] = a.b_in[i];
  }
  __syncthreads();
  const int comp_base = NC == 2 ? 0 : 2;
  for (int l = 0; l + 1 < a.nl; ++l) {  // down: pre-smooth, residual, restrict
    const TailLevel& L = a.L[l];
    smooth<KIND, NC>(a, L, B[l], rec, true, l == 0 ? a.deg0 : a.deg);
    TailBufs& Bl = B[l];
    apply_level<KIND, NC>(L, Bl.coef, Bl.x, rec, [&](int node, const float* f) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int i = NC * node + c;
        Bl.xn[i] = (Bl.fz[node] >> c) & 1 ? 0.f : Bl.b[i] - f[c];
      }
    });
    const TailLevel& C = a.L[l + 1];
    for (int node = tid; node < C.g.n; node += nt)
      restrict_node(L.g, C.g, NC, comp_base, Bl.xn, B[l + 1].b, B[l + 1].excl, node);
    __syncthreads();
  }
  const int lc = a.nl - 1;  // coarsest level of the tail
  {  // dense coarsest solve x = Ainv b with the stored inverse: each thread takes a pair of
     // outputs over one of dense_slices column ranges (many independent loads in flight across
     // the block instead of one long chain per output), then the slices are summed in order
    const int n = NC * a.L[lc].g.n, np = (n + 1) >> 1, S = a.dense_slices;
    const float* bc = B[lc].b;
    for (int t = tid; t < np * S; t += nt) {
      const int ip = t % np, sl = t / np, i = 2 * ip;
      const int j0 = sl * n / S, j1 = (sl + 1) * n / S;
      float s0 = 0.f, s1 = 0.f;
      if ((n & 1) == 0) {  // rows of even length: (i, i+1) is one aligned 8-byte load
#pragma unroll 8
        for (int j = j0; j < j1; ++j) {
          const float2 v = *reinterpret_cast<const float2*>(a.Ainv + (size_t)j * n + i);
          s0 += v.x * bc[j];
          s1 += v.y * bc[j];
        }
      } else {
#pragma unroll 8
        for (int j = j0; j < j1; ++j) {
          s0 += a.Ainv[(size_t)j * n + i] * bc[j];
          if (i + 1 < n) s1 += a.Ainv[(size_t)j * n + i + 1] * bc[j];
        }
      }
      rec[sl * n + i] = s0;
      if (i + 1 < n) rec[sl * n + i + 1] = s1;
    }
    __syncthreads();
    for (int i = tid; i < n; i += nt) {
      float acc = rec[i];
      for (int sl = 1; sl < S; ++sl) acc += rec[sl * n + i];
      B[lc].x[i] = acc;
    }
    __syncthreads();
  }
  for (int l = a.nl - 2; l >= 0; --l) {  // up: prolong, post-smooth
    const TailLevel& L = a.L[l];
    const TailLevel& C = a.L[l + 1];
    for (int node = tid; node < L.g.n; node += nt)
      prolong_node(L.g, C.g, NC, comp_base, B[l + 1].x, B[l].x, B[l].excl, node);
    __syncthreads();
    smooth<KIND, NC>(a, L, B[l], rec, false, l == 0 ? a.deg0 : a.deg);
  }
  for (int i = tid; i < NC * a.L[0].g.n; i += nt) a.x_out[i] = B[0].x[i];
}

}  // namespace

template <class F>
static bool raise_smem(F f, int lim) {
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) == cudaSuccess;
}

size_t tail_smem_limit() {
  static size_t limit = [] {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return size_t(0);
    size_t st = 0;
    const void* fs[4] = {(const void*)k_tail_vcycle<RIGHT, 1>, (const void*)k_tail_vcycle<RIGHT, 2>,
                         (const void*)k_tail_vcycle<CROSSED, 1>, (const void*)k_tail_vcycle<CROSSED, 2>};
    for (const void* f : fs) {
      cudaFuncAttributes fa;
      if (cudaFuncGetAttributes(&fa, f) != cudaSuccess) return size_t(0);
      st = fa.sharedSizeBytes > st ? fa.sharedSizeBytes : st;
    }
    if ((size_t)optin <= st) return size_t(0);
    const int lim = optin - (int)st;
    if (!raise_smem(k_tail_vcycle<RIGHT, 1>, lim) || !raise_smem(k_tail_vcycle<RIGHT, 2>, lim) ||
        !raise_smem(k_tail_vcycle<CROSSED, 1>, lim) || !raise_smem(k_tail_vcycle<CROSSED, 2>, lim))
      return size_t(0);
    return (size_t)lim;
  }();
  return limit;
}

void tail_vcycle(cudaStream_t s, int ncomp, const TailArgs& a, size_t smem) {
  const int id = kclass(KC_TAIL, false, a.first_level);
  const bool crossed = a.L[0].g.kind == CROSSED;
  if (crossed && ncomp == 2)
    PF_LAUNCH(id, 0.0, s, pdl_launch(k_tail_vcycle<CROSSED, 2>, 1, TAIL_THREADS, smem, s, a));
  else if (crossed)
    PF_LAUNCH(id, 0.0, s, pdl_launch(k_tail_vcycle<CROSSED, 1>, 1, TAIL_THREADS, smem, s, a));
  else if (ncomp == 2)
    PF_LAUNCH(id, 0.0, s, pdl_launch(k_tail_vcycle<RIGHT, 2>, 1, TAIL_THREADS, smem, s, a));
  else
    PF_LAUNCH(id, 0.0, s, pdl_launch(k_tail_vcycle<RIGHT, 1>, 1, TAIL_THREADS, smem, s, a));
}

}  // namespace pf
