// Energy evaluation that performs no device memory allocation (pf_energy_noalloc).
//
// Who needs it: callers that cannot let a library call cudaMalloc or cudaFree.  Examples are an
// application that has handed the whole device to its own memory pool (a framework's caching
// allocator holding every free byte), and code running where an implicit device-wide
// synchronization is not acceptable (cudaMalloc/cudaFree may synchronize the device).  The
// regular pf_energy needs a sim, whose workspace the caller must provide; this variant takes
// the fields directly and keeps its reduction scratch in a fixed array compiled into the library.
//
// The scratch is the file-scope __device__ array below: every GPU that loads the library holds
// it (328 KB) until the process exits.  Every call on a device uses the same array, which
// keeps the previous call's contents, so calls whose work overlaps on the GPU (different streams
// or threads without ordering) race on it and must be serialized by the caller.
#include <math.h>

#include <mutex>

#include "solver.hpp"

namespace pf {
namespace {

constexpr int NOALLOC_MAX_ROWS = 8192;  // cell rows (ny) supported by the eigenstrain table
constexpr size_t PART_DOUBLES = size_t(MAX_RED_BLOCKS) * 2;  // reduction partials (2 sums)
constexpr size_t OUT_OFFSET = PART_DOUBLES;                  // 2 output sums
constexpr size_t TICKET_OFFSET = OUT_OFFSET + 32;            // one unsigned counter (256-B aligned)
constexpr size_t EIG_OFFSET = TICKET_OFFSET + 32;            // eigenstrain table (rows x 4)
constexpr size_t SCRATCH_DOUBLES = EIG_OFFSET + size_t(NOALLOC_MAX_ROWS) * 4;

static __device__ __align__(256) double g_noalloc_scratch[SCRATCH_DOUBLES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
double* g_dev_ptr[MAX_DEVICES] = {};

// Device address of the scratch array for the current device (looked up once per device; the
// host-side name g_noalloc_scratch is only a stand-in and must never be passed to a kernel).
// A cudaDeviceReset of the device unloads the module, so the cached address is then stale: the
// library must not be used on a device after it has been reset.
pf_status scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error_message(cudaGetErrorString(e));
    return PF_ECUDA;
  }
  if (dev < 0 || dev >= MAX_DEVICES) {
    set_error_message("pf_energy_noalloc: device index out of range");
    return PF_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error_message("pf_energy_noalloc: cudaGetSymbolAddress of the scratch array failed");
      return PF_ECUDA;
    }
    g_dev_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_dev_ptr[dev];
  return PF_OK;
}

// beta T at element centroids per (cell row, element type), T = -dT erfc(y / pen)
__global__ void k_eig_rows(double* eig, int ny, int kind, double hy, double beta, double dT,
                           double pen) {
  pdl_enter();
  int NE = elems_per_cell(kind);
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ny * NE) return;
  int j = idx / NE, t = idx - j * NE;
  double y = (j + centroid_fy(kind, t)) * hy;
  eig[idx] = beta * (-dT * erfc(y / pen));
}

}  // namespace
}  // namespace pf

extern "C" pf_status pf_energy_noalloc(const pf_mesh_desc* d, const pf_material* mi,
                                       const pf_load* L, const double* u, const double* alpha,
                                       double out[3], void* stream) {
  using namespace pf;
  if (!d || !mi || !L || !u || !alpha || !out) {
    set_error_message("pf_energy_noalloc: null argument");
    return PF_EINVAL;
  }
  Grid g;
  pf_status st = describe_mesh(d, &g);
  if (st != PF_OK) return st;
  if (g.ny > NOALLOC_MAX_ROWS) {
    set_error_message("pf_energy_noalloc: the mesh has more than 8192 cell rows (ny), the "
                      "maximum of the fixed scratch array");
    return PF_EINVAL;
  }
  Mat m;
  st = describe_material(mi, &m);
  if (st != PF_OK) return st;
  double* scr = nullptr;
  st = scratch_address(&scr);
  if (st != PF_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned* ticket = reinterpret_cast<unsigned*>(scr + TICKET_OFFSET);
  // the ticket must start at zero; the previous call may have been interrupted
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned), s);
  const bool thermal = mi->beta != 0.0 && L->dT != 0.0;
  double* eig = scr + EIG_OFFSET;
  if (e == cudaSuccess && thermal) {
    const int cnt = g.ny * elems_per_cell(g.kind);
    PF_LAUNCH(kclass(KC_SETUP, true, 0), 8.0 * cnt, s,
              pdl_launch(k_eig_rows, dim3((cnt + 255) / 256), dim3(256), 0, s, eig, g.ny, g.kind,
                         g.hy, mi->beta, L->dT, mi->pen));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    energy(s, g, m, u, alpha, thermal ? eig : nullptr, RedSlot{scr, ticket, scr + OUT_OFFSET});
    e = cudaGetLastError();
  }
  double host[2] = {0.0, 0.0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, scr + OUT_OFFSET, 2 * sizeof(double),
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error_message(cudaGetErrorString(e));
    return PF_ECUDA;
  }
  out[0] = host[0];
  out[1] = host[1];
  out[2] = host[0] + host[1];
  return PF_OK;
}
