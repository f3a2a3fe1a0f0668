// Tensor-core hop for half-precision storage (F16 / BF16): placeholder until the
// mma-based kernel lands; the generic CUDA-core hop serves every precision meanwhile.
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"

namespace mdwf {
bool hop_tc_supported(int, const HopParams&, bool) { return false; }
cudaError_t launch_hop_tc(int, bool, bool, const HopParams&, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace mdwf
