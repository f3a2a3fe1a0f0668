// Allocation-free variant of the nucleon two-point contraction.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being
// captured, applications whose device memory is owned by a custom or framework pool
// allocator that forbids side allocations, and hosts that pre-plan every byte of device
// memory before a long run.  For them this file keeps the contraction's per-site scratch
// (two doubles per 4D site) in a fixed array linked into the library instead of a
// context workspace.  The array costs every GPU that loads the library
// NOALLOC_MAX_SITES * 16 bytes (8 MiB) until the process exits.
#include "mdwf.h"
#include "mdwf_kernels.h"

#include <mutex>
#include <string>

namespace mdwf {
bool ctx_geom(const mdwf_ctx* c, Geom* g);
void nucleon_mats(NucMats* m);
}  // namespace mdwf

using namespace mdwf;

namespace {

constexpr long long NOALLOC_MAX_SITES = 1LL << 19;   // 524288 4D sites, e.g. 32^3 x 16

// per-site partial correlator values, re/im interleaved; shared by every call
__device__ __align__(256) double g_nucleon_scratch[2 * NOALLOC_MAX_SITES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mutex;
void* g_scratch_addr[MAX_DEVICES] = {};
thread_local std::string g_err;

}  // namespace

extern "C" {

const char* mdwf_noalloc_last_error(void) { return g_err.c_str(); }

int mdwf_contract_nucleon_noalloc(const mdwf_ctx* ctx, const double* u1, const double* d, const double* u2,
                                  double* corr, void* stream) {
  if (!ctx || !u1 || !d || !u2 || !corr) {
    g_err = "null pointer";
    return MDWF_ERR_ARG;
  }
  Geom g;
  if (!ctx_geom(ctx, &g)) {
    g_err = "invalid context";
    return MDWF_ERR_ARG;
  }
  const long long V = 2 * g.vh;
  if (V > NOALLOC_MAX_SITES) {
    g_err = "lattice has " + std::to_string(V) + " sites; the allocation-free contraction holds at most " +
            std::to_string(NOALLOC_MAX_SITES) + " (use mdwf_contract_nucleon)";
    return MDWF_ERR_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    g_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return MDWF_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    // set-up once per device, with that device current: the host-side name of the array is
    // not a device address, so the kernel gets the address the runtime reports for it
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_nucleon_scratch);
      if (e != cudaSuccess || !p) {
        g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return MDWF_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    }
    scratch = g_scratch_addr[dev];
  }
  NucMats m;
  nucleon_mats(&m);
  // every scratch entry the sums read is written earlier in the same call: nothing to clear
  e = launch_nucleon(g, m, u1, d, u2, (double*)scratch, corr, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    g_err = std::string("launch_nucleon: ") + cudaGetErrorString(e);
    return MDWF_ERR_CUDA;
  }
  return MDWF_SUCCESS;
}

}  // extern "C"
