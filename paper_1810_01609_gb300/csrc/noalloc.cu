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
int ctx_device(const mdwf_ctx* c);
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
  // the propagators are device buffers of the context's device; the scratch array used
  // is the current device's copy, so the two must be the same device
  if (dev != ctx_device(ctx)) {
    g_err = "the context was created on device " + std::to_string(ctx_device(ctx)) + " but device " +
            std::to_string(dev) + " is current";
    return MDWF_ERR_ARG;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
  if (e != cudaSuccess) {
    g_err = std::string("cudaStreamIsCapturing: ") + cudaGetErrorString(e);
    return MDWF_ERR_CUDA;
  }
  void* scratch = nullptr;
  {
    // The host-side name of the array is not a device address: the kernel gets the
    // address the runtime reports for it, looked up with this device current.  Outside
    // stream capture it is looked up on every call (cheap once the module is loaded, and
    // correct again after a device reset reloads the module); during capture the address
    // from this device's last uncaptured call is used.
    std::lock_guard<std::mutex> lock(g_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_nucleon_scratch);
      if (e != cudaSuccess || !p) {
        g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return MDWF_ERR_CUDA;
      }
      g_scratch_addr[dev] = p;
    } else if (!g_scratch_addr[dev]) {
      g_err = "the first call on a device must come before any stream capture";
      return MDWF_ERR_STATE;
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
