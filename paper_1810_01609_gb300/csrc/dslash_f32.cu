// F32-storage instantiations of the CUDA-core hop kernels (see dslash_impl.cuh).
#include "dslash_impl.cuh"

namespace mdwf {
template cudaError_t launch_hop_prec<F32>(const HopParams&, bool, bool, bool, bool, bool, int, size_t, cudaStream_t);
}  // namespace mdwf
