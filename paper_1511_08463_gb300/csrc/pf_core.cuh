// Core definitions shared by the kernels and the host driver of libpf.
//
// Discretization (Section 1.2, P1 elements on simplicial meshes) of the regularized energy of
// Section 1.1 on a structured rectangle.  Two triangulations:
//   RIGHT:   cell (i,j) -> t0 = (v00, v10, v11), t1 = (v00, v11, v01)
//   CROSSED: cell (i,j) -> t0 = (v00, v10, c), t1 = (v10, v11, c), t2 = (v11, v01, c),
//            t3 = (v01, v00, c), c the centre node of the cell.
// On every element the P1 basis gradients are constant: grad phi_k = (GX[t][k] / hx,
// GY[t][k] / hy) with small integers GX, GY (tables below), and |T| = hx hy / 2 (RIGHT) or
// hx hy / 4 (CROSSED).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pf.h"

namespace pf {

// Programmatic dependent launch (PDL).  Every kernel of the library starts with pdl_enter():
// griddepcontrol.wait blocks until the kernel launched before it on the stream has completed
// and its memory is visible, and launch_dependents then lets the next kernel be launched and
// scheduled while this one runs.  Each kernel thus still sees all effects of its predecessor
// (stream order is kept), but the next launch's latency overlaps this kernel's execution --
// which matters for the many small kernels of the coarse multigrid levels.  Both instructions
// are no-ops for a kernel launched without the PDL attribute.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Launch `k` on `s` with the programmatic-stream-serialization attribute (errors are reported
// by cudaGetLastError, like a triple-chevron launch).
template <class... KArgs, class... Args>
inline void pdl_launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

constexpr int RIGHT = 0;
constexpr int CROSSED = 1;
constexpr int TX = 32;  // stencil tile: vertices per block in x
constexpr int TY = 8;   // stencil tile: vertices per block in y (default; FP32 multigrid kernels
                        // also come with TY_MIN and 16 rows, chosen per level by the autotuner)
constexpr int TY_MIN = 4;
constexpr int RED_THREADS = 256;
constexpr int MAX_RED_BLOCKS = 4096;

__host__ __device__ constexpr int elems_per_cell(int kind) { return kind == CROSSED ? 4 : 2; }

// Gradient integer tables.  gx(kind, t, k): x-component of grad phi_k on element t times hx.
__host__ __device__ constexpr int gx(int kind, int t, int k) {
  return kind == CROSSED
             ? (t == 0 ? (k == 0 ? -1 : k == 1 ? 1 : 0)
                : t == 1 ? (k == 0 ? 1 : k == 1 ? 1 : -2)
                : t == 2 ? (k == 0 ? 1 : k == 1 ? -1 : 0)
                         : (k == 0 ? -1 : k == 1 ? -1 : 2))
             : (t == 0 ? (k == 0 ? -1 : k == 1 ? 1 : 0) : (k == 0 ? 0 : k == 1 ? 1 : -1));
}
__host__ __device__ constexpr int gy(int kind, int t, int k) {
  return kind == CROSSED
             ? (t == 0 ? (k == 0 ? -1 : k == 1 ? -1 : 2)
                : t == 1 ? (k == 0 ? -1 : k == 1 ? 1 : 0)
                : t == 2 ? (k == 0 ? 1 : k == 1 ? 1 : -2)
                         : (k == 0 ? 1 : k == 1 ? -1 : 0))
             : (t == 0 ? (k == 0 ? 0 : k == 1 ? -1 : 1) : (k == 0 ? -1 : k == 1 ? 0 : 1));
}
// Centroid height of element t inside its cell, as a fraction of hy.
__host__ __device__ constexpr double centroid_fy(int kind, int t) {
  return kind == CROSSED ? (t == 0 ? 1.0 / 6.0 : t == 2 ? 5.0 / 6.0 : 0.5)
                         : (t == 0 ? 1.0 / 3.0 : 2.0 / 3.0);
}

// One level of the structured hierarchy, passed by value to kernels.
struct Grid {
  int kind, nx, ny;
  int nv, n;      // vertices, nodes
  int ncell;      // nx * ny
  int nelem;      // ncell * elems_per_cell
  double hx, hy, ihx, ihy, area;  // area of one element
  uint8_t fixed[4][3];             // [edge][comp] (edges: left, right, bottom, top)
  int npins;
  int pin_x2[PF_MAX_PINS], pin_y2[PF_MAX_PINS], pin_comp[PF_MAX_PINS];
  int interior_pins;  // 1 if some pin lies strictly inside the rectangle
  int tile_rows;      // stencil tile height of the FP32 kernels on this level (0: TY)
};

// Material constants in the form the kernels use.
struct Mat {
  double lam, mu, lam2mu;  // Lame constants (plane strain or the plane-stress lambda*)
  double k_ell;
  double c1;    // 2 Gc ell / c_w           (Laplacian coefficient of E_aa)
  double c2;    // 2 Gc / (c_w ell) for AT2 (mass coefficient of E_aa), 0 for AT1
  double c3;    // Gc / (c_w ell) for AT1   (linear term of E_alpha), 0 for AT2
  double gc_cw, ell;
  int model;
};

__device__ __forceinline__ bool is_fixed(const Grid& g, int X2, int Y2, int comp) {
  // interior nodes are free unless a pin sits off the boundary (rare): skip the pin loop
  if (!g.interior_pins && X2 > 0 && X2 < 2 * g.nx && Y2 > 0 && Y2 < 2 * g.ny) return false;
  bool f = (X2 == 0 && g.fixed[0][comp]) || (X2 == 2 * g.nx && g.fixed[1][comp]) ||
           (Y2 == 0 && g.fixed[2][comp]) || (Y2 == 2 * g.ny && g.fixed[3][comp]);
  for (int k = 0; k < g.npins; ++k)
    f = f || (g.pin_x2[k] == X2 && g.pin_y2[k] == Y2 && g.pin_comp[k] == comp);
  return f;
}

__device__ __forceinline__ void node_coords(const Grid& g, int node, int& X2, int& Y2) {
  if (node < g.nv) {
    int j = node / (g.nx + 1), i = node - j * (g.nx + 1);
    X2 = 2 * i;
    Y2 = 2 * j;
  } else {
    int c = node - g.nv;
    int j = c / g.nx, i = c - j * g.nx;
    X2 = 2 * i + 1;
    Y2 = 2 * j + 1;
  }
}

// abar(alpha) on one P1 element: (1/|T|) int_T (1 - alpha_h)^2 + k_ell, written with
// d = 1 - alpha so that fully damaged elements give exactly k_ell.
template <class T>
__device__ __forceinline__ T abar3(T a0, T a1, T a2, T k_ell) {
  T d0 = T(1) - a0, d1 = T(1) - a1, d2 = T(1) - a2;
  return (d0 * d0 + d1 * d1 + d2 * d2 + d0 * d1 + d1 * d2 + d2 * d0) * T(1.0 / 6.0) + k_ell;
}

// Fischer-Burmeister function (Section 2.4) and its nested MCP form on [lo, hi]:
// Phi = phi(x - lo, phi(hi - x, -F)).
__device__ __forceinline__ double phi_fb(double a, double b) { return sqrt(a * a + b * b) - a - b; }
__device__ __forceinline__ double mcp_phi(double x, double F, double lo, double hi) {
  return phi_fb(x - lo, phi_fb(hi - x, -F));
}

// ---- deterministic grid reductions ---------------------------------------------------------
// Each block writes its partial to part[blockIdx]; the last block to arrive (ticket) sums the
// partials in block order and writes *out.  No inter-block waiting.
struct RedSlot {
  double* part;      // >= gridDim.x * NV doubles
  unsigned* ticket;  // one counter, zero between launches
  double* out;       // NV doubles
};

template <int NV, bool MAX, class VT = double>
__device__ __forceinline__ void block_reduce_finalize(VT (&v)[NV], RedSlot slot) {
  __shared__ double red[NV][32];
  __shared__ bool last;
  int lane = threadIdx.x & 31, warp = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
  int tid = threadIdx.x + threadIdx.y * blockDim.x;
  int nthreads = blockDim.x * blockDim.y;
  lane = tid & 31;
  warp = tid >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    VT x = v[q];  // warp stage in the partials' own precision, then FP64 across warps
    for (int o = 16; o > 0; o >>= 1) {
      VT y = __shfl_down_sync(0xffffffffu, x, o);
      x = MAX ? (x > y ? x : y) : x + y;
    }
    if (lane == 0) red[q][warp] = double(x);
  }
  __syncthreads();
  int nwarps = (nthreads + 31) >> 5;
  if (tid == 0) {
    int bid = blockIdx.x + blockIdx.y * gridDim.x;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double x = red[q][0];
      for (int w = 1; w < nwarps; ++w) x = MAX ? fmax(x, red[q][w]) : x + red[q][w];
      slot.part[bid * NV + q] = x;
    }
    __threadfence();
    unsigned nb = gridDim.x * gridDim.y;
    unsigned t = atomicAdd(slot.ticket, 1u);
    last = (t == nb - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    unsigned nb = gridDim.x * gridDim.y;
    // each thread sums a strided subset in fixed order, then a fixed-order tree; the partials
    // are read from L2 eight at a time (all in flight together) and added in the same order
    for (int q = 0; q < NV; ++q) {
      double x = MAX ? -INFINITY : 0.0;
      unsigned b = tid;
      for (; b + 7u * nthreads < nb; b += 8u * nthreads) {
        double y[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) y[u] = __ldcg(slot.part + (size_t)(b + u * nthreads) * NV + q);
#pragma unroll
        for (int u = 0; u < 8; ++u) x = MAX ? fmax(x, y[u]) : x + y[u];
      }
      for (; b < nb; b += nthreads) {
        const double y = __ldcg(slot.part + (size_t)b * NV + q);
        x = MAX ? fmax(x, y) : x + y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        double y = __shfl_down_sync(0xffffffffu, x, o);
        x = MAX ? fmax(x, y) : x + y;
      }
      __syncthreads();
      if (lane == 0) red[q][warp] = x;
      __syncthreads();
      if (tid == 0) {
        double s = red[q][0];
        for (int w = 1; w < nwarps; ++w) s = MAX ? fmax(s, red[q][w]) : s + red[q][w];
        slot.out[q] = s;
      }
    }
    if (tid == 0) *slot.ticket = 0u;
  }
}

}  // namespace pf
