// BF16-storage instantiations of the bulk-staged CUDA-core hop kernel (see dslash_impl.cuh).
#include "dslash_impl.cuh"

namespace mdwf {
template cudaError_t launch_hop_bulk_prec<BF16>(const HopParams&, bool, bool, bool, int, size_t, cudaStream_t);
}  // namespace mdwf
