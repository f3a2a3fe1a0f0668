// Dispatch of the CUDA-core hop kernels (dslash_impl.cuh) over storage precisions; each
// precision's instantiations live in their own translation unit (dslash_<prec>.cu) so the
// build compiles them in parallel.
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"
#include "mdwf_epi.cuh"

namespace mdwf {

template <int P>
cudaError_t launch_hop_prec(const HopParams& p, bool dag, bool r12, bool epi, bool occ, int threads, size_t smem,
                            cudaStream_t st);

size_t hop_smem_bytes(int prec, const HopParams& p, bool epi) {
  const size_t csz = prec == F64 ? 8 : 4;
  const size_t links = (size_t)p.ns * 8 * (prec == F64 ? 18 : 20) * csz;
  const size_t nbr = (size_t)((p.ns * 8 + 3) & ~3) * 4;
  const size_t pre = (links + nbr + 15) & ~(size_t)15;
  if (!epi) return pre;
  const int threads = p.ns * p.in.nrhs * p.in.Ls;
  return pre + epi_smem_bytes(csz, p.ns, p.in.nrhs, p.in.Ls, p.has_center, threads);
}

cudaError_t launch_hop(int prec, bool dag, bool r12, bool epi, bool occ, const HopParams& p, cudaStream_t st) {
  const int threads = p.ns * p.in.nrhs * p.in.Ls;
  const size_t smem = hop_smem_bytes(prec, p, epi);
  switch (prec) {
    case F64: return launch_hop_prec<F64>(p, dag, r12, epi, occ, threads, smem, st);
    case F32: return launch_hop_prec<F32>(p, dag, r12, epi, occ, threads, smem, st);
    case F16: return launch_hop_prec<F16>(p, dag, r12, epi, occ, threads, smem, st);
    case BF16: return launch_hop_prec<BF16>(p, dag, r12, epi, occ, threads, smem, st);
    case I16: return launch_hop_prec<I16>(p, dag, r12, epi, occ, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mdwf
