// Dispatch of the CUDA-core hop kernels (dslash_impl.cuh) over storage precisions; each
// precision's instantiations live in their own translation units (dslash_<prec>.cu for the
// single-column kernel, dslash2_<prec>.cu for the paired-column one, dslash3_<prec>.cu for
// the bulk-staged one) so the
// build compiles them in parallel.
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"
#include "mdwf_epi.cuh"

namespace mdwf {

template <int P>
cudaError_t launch_hop_prec(const HopParams& p, bool dag, bool r12, bool epi, bool occ, bool emu, int threads,
                            size_t smem, cudaStream_t st);
template <int P>
cudaError_t launch_hop2_prec(const HopParams& p, bool dag, bool r12, bool epi, int threads, size_t smem,
                             cudaStream_t st);

template <int P>
cudaError_t launch_hop_bulk_prec(const HopParams& p, bool dag, bool r12, bool epi, int threads, size_t smem,
                                 cudaStream_t st);

bool hop_bulk_supported(int prec, const HopParams& p) {
  // the bulk copies need 16-byte aligned rows: the field's base and 48 W bytes per row
  return (prec == F16 || prec == BF16 || prec == I16) && ((uintptr_t)p.in.data & 15) == 0;
}

bool hop_pair_supported(int prec, const HopParams& p) {
  return prec != F64 && ((p.in.nrhs * p.in.Ls) & 1) == 0;
}

int hop_threads(const HopParams& p, bool pair) {
  const int t = p.ns * p.in.nrhs * p.in.Ls;
  return pair ? t / 2 : t;
}

size_t hop_smem_bytes(int prec, const HopParams& p, bool epi, bool pair, bool bulk) {
  const size_t csz = prec == F64 ? 8 : 4;
  if (bulk) {
    const size_t pre = (size_t)bulk_layout(p.ns, p.in.nrhs * p.in.Ls).epi;
    return epi ? pre + epi_smem_bytes(csz, p.ns, p.in.nrhs, p.in.Ls, p.has_center, hop_threads(p, false)) : pre;
  }
  // staged links: 18 float2 per link for the paired kernel, else 18 (F64) or 20 reals;
  // 16 bytes per site of bank offset
  const size_t links = pair ? (size_t)p.ns * (8 * 18 + 2) * 8 : (size_t)p.ns * (8 * (prec == F64 ? 18 : 20) * csz + 16);
  const size_t nbr = (size_t)((p.ns * 8 + 3) & ~3) * 4;
  const size_t pre = (links + nbr + 15) & ~(size_t)15;
  if (!epi) return pre;
  return pre + epi_smem_bytes(csz, p.ns, p.in.nrhs, p.in.Ls, p.has_center, hop_threads(p, pair));
}

cudaError_t launch_hop(int prec, bool dag, bool r12, bool epi, bool occ, bool pair, bool emu, bool bulk,
                       const HopParams& p, cudaStream_t st) {
  if (emu && prec != F64) return cudaErrorInvalidValue;
  const int threads = hop_threads(p, pair);
  const size_t smem = hop_smem_bytes(prec, p, epi, pair, bulk);
  if (bulk) {
    if (!hop_bulk_supported(prec, p)) return cudaErrorInvalidValue;
    switch (prec) {
      case F16: return launch_hop_bulk_prec<F16>(p, dag, r12, epi, threads, smem, st);
      case BF16: return launch_hop_bulk_prec<BF16>(p, dag, r12, epi, threads, smem, st);
      case I16: return launch_hop_bulk_prec<I16>(p, dag, r12, epi, threads, smem, st);
    }
    return cudaErrorInvalidValue;
  }
  if (pair) {
    if (!hop_pair_supported(prec, p)) return cudaErrorInvalidValue;
    switch (prec) {
      case F32: return launch_hop2_prec<F32>(p, dag, r12, epi, threads, smem, st);
      case F16: return launch_hop2_prec<F16>(p, dag, r12, epi, threads, smem, st);
      case BF16: return launch_hop2_prec<BF16>(p, dag, r12, epi, threads, smem, st);
      case I16: return launch_hop2_prec<I16>(p, dag, r12, epi, threads, smem, st);
    }
    return cudaErrorInvalidValue;
  }
  switch (prec) {
    case F64: return launch_hop_prec<F64>(p, dag, r12, epi, occ, emu, threads, smem, st);
    case F32: return launch_hop_prec<F32>(p, dag, r12, epi, occ, emu, threads, smem, st);
    case F16: return launch_hop_prec<F16>(p, dag, r12, epi, occ, emu, threads, smem, st);
    case BF16: return launch_hop_prec<BF16>(p, dag, r12, epi, occ, emu, threads, smem, st);
    case I16: return launch_hop_prec<I16>(p, dag, r12, epi, occ, emu, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mdwf
