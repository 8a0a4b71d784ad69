// Pair search that allocates nothing: the cell lists and neighbour lists live in a
// fixed device array of this library instead of caller-provided scratch.
//
// It serves callers that cannot hand over device memory and must not allocate any:
// code without access to a CUDA allocator (a plug-in or callback inside a larger
// application that is handed only its input and output buffers), or code that must
// not pay the implicit device synchronisation cudaMalloc/cudaFree may cause.  The
// caller still owns the inputs (centres) and the output (pair list).  The call reads
// the pair count back and synchronises its stream, so it cannot itself be captured.
//
// Costs and rules of the shared array:
//   - kStaticScratchBytes (16 MiB) of device memory is reserved on every GPU that
//     loads this library, for the life of the process.
//   - One array per device serves every call: calls whose work overlaps on the GPU
//     (two streams, or two host threads without ordering) race on it and give wrong
//     results.  Order them on one stream or serialise them.
//   - The array keeps the contents of the last call; the per-cell counters and the
//     status word are cleared on the caller's stream at the start of each call.
//   - The first call on each device looks up the array's device address (with that
//     device current) and caches it; make that first call before any stream capture.
//     The cached address belongs to the device's context: after cudaDeviceReset the
//     library must be loaded again before this entry point is used.
#include <cstdint>
#include <mutex>
#include <string>

#include "ibmlbm.h"
#include "common.cuh"
#include "launch.h"
#include "pair_grid.h"

using namespace ibmlbm;

namespace {

constexpr size_t kStaticScratchBytes = 16u << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_pair_scratch[kStaticScratchBytes];

int static_fail(int code, const std::string& msg) {
  set_last_error(msg);  // reported by ibm_lbm_last_error()
  return code;
}

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};

// device address of g_pair_scratch on the current device (looked up once per device)
int scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(IBMLBM_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return static_fail(IBMLBM_ERR_UNSUPPORTED, "device ordinal beyond 63");
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pair_scratch);
    if (e != cudaSuccess || !p)
      return static_fail(IBMLBM_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return IBMLBM_OK;
}

}  // namespace

extern "C" int ibm_lbm_pair_search_static(int32_t dim, const int32_t* n_nodes, const int32_t* periodic,
                                          double diameter, double zeta, int32_t n, const double* d_X,
                                          int32_t max_neighbors, int32_t* d_pairs, int64_t cap,
                                          int64_t* h_count, void* stream) {
  if (dim != 2 && dim != 3) return static_fail(IBMLBM_ERR_INVALID_ARG, "dim must be 2 or 3");
  if (!n_nodes || !h_count) return static_fail(IBMLBM_ERR_INVALID_ARG, "n_nodes or count is NULL");
  if (n < 0) return static_fail(IBMLBM_ERR_INVALID_ARG, "n < 0");
  if (!(diameter > 0.0) || !(zeta > 0.0))
    return static_fail(IBMLBM_ERR_INVALID_ARG, "diameter and zeta must be > 0");
  if (max_neighbors < 0 || max_neighbors > 64)
    return static_fail(IBMLBM_ERR_INVALID_ARG, "max_neighbors must be in 0..64");
  *h_count = 0;
  PairArgs a{};
  a.wall_lo = -0.5;
  for (int k = 0; k < 3; ++k) {
    if (k < dim && n_nodes[k] < 1) return static_fail(IBMLBM_ERR_INVALID_ARG, "n_nodes must be >= 1");
    a.L[k] = k < dim ? (double)n_nodes[k] : 1.0;
    a.g.per[k] = (k < dim && periodic) ? (periodic[k] ? 1 : 0) : 0;
  }
  // the cells of ibm_lbm_pair_search and of a run (pair_grid.h)
  cell_grid(dim, a.L, a.g.per, diameter + zeta, a.nc, a.H);
  if (n == 0) return IBMLBM_OK;
  if (!d_X || (cap > 0 && !d_pairs)) return static_fail(IBMLBM_ERR_INVALID_ARG, "X or pairs is NULL");
  const int kmax = max_neighbors ? max_neighbors : 32;
  const PairScratch ps = pair_scratch(n, kmax, a.nc);
  if (!ps.ok || ps.total > kStaticScratchBytes)
    return static_fail(IBMLBM_ERR_CAPACITY,
                       "problem needs " + (ps.ok ? std::to_string(ps.total) : std::string("more than 2^64")) +
                           " bytes of scratch, above the fixed " + std::to_string(kStaticScratchBytes) +
                           "; use ibm_lbm_pair_search");
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc) return rc;
  char* sc = static_cast<char*>(base);
  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  a.g.nx = (int)a.L[0];
  a.g.ny = (int)a.L[1];
  a.g.nz = (int)a.L[2];
  a.D = dim;
  a.n = n;
  a.diam = diameter;
  a.zeta = zeta;
  a.thr2 = (diameter + zeta) * (diameter + zeta);
  a.kmax = kmax;
  a.X = d_X;
  a.cell_count = reinterpret_cast<int*>(sc + ps.cell_count);
  a.cell_ids = reinterpret_cast<int*>(sc + ps.cell_ids);
  a.cell_cap = ps.cell_cap;
  a.nbr = reinterpret_cast<int*>(sc + ps.nbr);
  a.nbr_count = reinterpret_cast<int*>(sc + ps.nbr_count);
  a.gt_count = reinterpret_cast<int*>(sc + ps.gt);
  a.status = reinterpret_cast<uint32_t*>(sc + ps.status);
  a.Fc = nullptr;
#define STATIC_TRY(expr)                                                                      \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return static_fail(IBMLBM_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)
  // the status word must start at zero (the cell counters are cleared by
  // launch_pair_cells); everything else is written before it is read
  STATIC_TRY(cudaMemsetAsync(a.status, 0, sizeof(uint32_t), s));
  STATIC_TRY(launch_pair_cells(a, s));
  STATIC_TRY(launch_pair_contacts(a, s));
  STATIC_TRY(launch_pair_compact(a, d_pairs, cap, s));
  int total = 0;
  uint32_t st = 0;
  STATIC_TRY(cudaMemcpyAsync(&total, a.gt_count + n, sizeof(int), cudaMemcpyDeviceToHost, s));
  STATIC_TRY(cudaMemcpyAsync(&st, a.status, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  STATIC_TRY(cudaStreamSynchronize(s));
#undef STATIC_TRY
  *h_count = total;
  if (st & ST_CAPACITY) return static_fail(IBMLBM_ERR_CAPACITY, "a particle has more than max_neighbors partners");
  if (total > cap) return static_fail(IBMLBM_ERR_CAPACITY, "more pairs than cap");
  return IBMLBM_OK;
}
