// Faces of a T-partitioned lattice (Sec. "Current State of the Art": the radius-one
// stencil is decomposed over GPUs and the faces exchanged while the interior computes).
//
// A hop across the partition boundary in t needs, for each site of the neighbouring
// partition's first (or last) timeslice, the neighbour's spin-projected half spinor
// (1 - sig gamma_4) psi: 12 reals per face site and column, 2x less than the spinor.  This
// kernel forms them with the hop kernels' own projection (load_proj), so a face holds
// exactly the reals the receiving kernel would have formed from the field itself (and the
// F16 / int16 scale): the partitioned operator is bit-identical to the undecomposed one.
#include "dslash_impl.cuh"

namespace mdwf {

namespace {

template <int P, int SIG>
__global__ void pack_face_kernel(const __grid_constant__ FaceParams p) {
  using C = typename PT<P>::C;
  const long long W = p.in.W();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.slice_vh * W) return;
  const long long f = i / W;
  const int col = (int)(i - f * W);
  C h[12];
  const C nrm = load_proj<P, 3, SIG>(p.in, (unsigned)(p.first + f), col, h);
  C* dst = (C*)p.face + i * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) dst[k] = h[k];
  if constexpr (PT<P>::NORM) p.norm[i] = nrm;
}

template <int P>
cudaError_t launch_pf(int sig, const FaceParams& p, cudaStream_t st) {
  const long long n = p.slice_vh * p.in.W();
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (sig > 0) pack_face_kernel<P, 1><<<blocks, 128, 0, st>>>(p);
  else pack_face_kernel<P, -1><<<blocks, 128, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_pack_face(int prec, int sig, const FaceParams& p, cudaStream_t st) {
  switch (prec) {
    case F64: return launch_pf<F64>(sig, p, st);
    case F32: return launch_pf<F32>(sig, p, st);
    case F16: return launch_pf<F16>(sig, p, st);
    case BF16: return launch_pf<BF16>(sig, p, st);
    case I16: return launch_pf<I16>(sig, p, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mdwf
