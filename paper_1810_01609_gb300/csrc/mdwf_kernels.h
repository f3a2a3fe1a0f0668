// Launch interfaces of the libmdwf kernels (host side).
#pragma once
#include "mdwf_impl.cuh"

namespace mdwf {

// ---------------------------------------------------------------- hop (dslash.cu, dslash_tc.cu)
struct HopParams {
  const void* gauge;  // gauge field of the output parity (precision of the kernel)
  int gs;             // reals per link in that layout
  Field in;           // input half (parity 1 - pout)
  Field out;          // output half (parity pout)
  Field center;       // optional centre term (parity pout)
  Field raxpy;        // axpy target r (parity pout): r -= alpha * result
  int pout;
  Geom g;
  int ns;             // 4D sites per CTA
  double t_bc;
  // epilogue: out = fin( cc * cop(center) + hc * post(hop) )
  SChain post;
  double hc;
  int has_center;
  SChain cop;
  double cc;
  int norm_pre;       // reduce |cc*cop(center) + hc*post(hop)|^2 (before fin)
  SChain fin;
  int axpy_r;         // r -= alpha[rhs] * out and reduce |r|^2 instead of storing out
  double mf;
  float hcf, ccf, mff;   // hc, cc, mf rounded once for the 32-bit kernels
  Red red;
  int* status;        // device flag: nonzero once a bounded device-side wait gave up
  // sites of the output half this launch covers: x_cb in [x_begin, x_end)
  long long x_begin, x_end;
  // T-partitioned lattice: face_mode 1 takes the backward t term (direction 7) of every
  // site from `face` (the lower neighbour's last timeslice), 2 the forward t term
  // (direction 3) from the upper neighbour's first timeslice.  A face holds, per face site
  // f and column, the 12 projected reals the kernel would form (compute type) and, for
  // F16, the neighbour's norm.  bc_lo / bc_hi: the local first / last timeslice is the
  // global one (where the time boundary phase applies).
  int face_mode;
  const void* face;
  const float* face_norm;
  long long face_base;  // checkerboard index of the face's timeslice in the local lattice
  int bc_lo, bc_hi;
};

// pair: the paired-column kernel (32-bit compute types, nrhs * Ls even, ns * nrhs * Ls / 2
// threads); occ: the occupancy-bounded build of a fused single-column 32-bit kernel; emu:
// the emulated-FP64 (double-float) hop loop of the FP64 kernel; bulk: the single-column
// kernel with its neighbour rows staged in shared memory by bulk copies (16-bit storage)
size_t hop_smem_bytes(int prec, const HopParams& p, bool epi, bool pair = false, bool bulk = false);
int hop_threads(const HopParams& p, bool pair);
bool hop_pair_supported(int prec, const HopParams& p);
bool hop_bulk_supported(int prec, const HopParams& p);
cudaError_t launch_hop(int prec, bool dag, bool r12, bool epi, bool occ, bool pair, bool emu, bool bulk,
                       const HopParams& p, cudaStream_t st);

// one face of a T-partitioned lattice (partition.cu): for every site f of the local
// timeslice starting at checkerboard index `first` (slice_vh sites) and every column, the
// 12 reals of (1 - sig gamma_4) in projected as the hop kernels project them, in the
// compute type, at face[(f * W + col) * 12]; F16 / int16 also the site's scale at norm[f * W + col]
struct FaceParams {
  Field in;
  long long slice_vh, first;
  void* face;
  float* norm;
};
cudaError_t launch_pack_face(int prec, int sig, const FaceParams& p, cudaStream_t st);

// tcgen05 tensor-core hop for F16 / BF16 storage (dslash_umma.cu); p.ns = 4D sites per CTA
bool hop_tc_supported(int prec, const HopParams& p, bool r12);
size_t hop_tc_smem_bytes(const HopParams& p);
int hop_tc_tmem_cols(const HopParams& p);        // tensor-memory columns one CTA allocates
cudaError_t launch_hop_tc(int prec, bool dag, bool r12, bool epi, const HopParams& p, cudaStream_t st);

// ---------------------------------------------------------------- s-local kernels (slocal.cu)
struct SLParams {
  Field a, b, c, d;     // operands (meaning per kernel)
  Field x;              // solution accumulator (cg_update: its own precision)
  int ns;               // 4D sites per CTA
  long long vh;
  SChain chain;
  double ca, cb;        // scalars
  double mf;
  float caf, cbf, mff;  // the same rounded once for the 32-bit kernels
  Red red;
};

// out(a) = ca * chain(in(b)) [+ cb * c]   (c optional: c.data == nullptr)
cudaError_t launch_chain(int prec, const SLParams& p, cudaStream_t st);
// a = ca * b + cb * c (b/c may alias a); optional |a|^2 reduction; a.data == nullptr: no store
cudaError_t launch_axpby(int prec, const SLParams& p, cudaStream_t st);
// x += alpha p ; p = r + beta p ; phat = chain(p)   (a = p, b = r, c = phat; x separate;
// c.data == nullptr: no phat)
cudaError_t launch_cg_update(int prec_x, int prec, const SLParams& p, cudaStream_t st);
// Re <b, c> per rhs into red.out (RED_STORE)
cudaError_t launch_dot(int prec, const SLParams& p, cudaStream_t st);
// a[rhs] += red.out[rhs] * b[rhs]
cudaError_t launch_rhs_axpy(int prec, const SLParams& p, cudaStream_t st);
// a(prec_out) (+)= b(prec_in); ca = 1 accumulate, 0 overwrite; cb != 0: zero b afterwards
cudaError_t launch_convert(int prec_out, int prec_in, const SLParams& p, cudaStream_t st);

// ---------------------------------------------------------------- layout / physics (pack.cu)
struct PackParams {
  Geom g;
  int Ls, nrhs;
  const double* user;   // user 5D field (device)
  double* user_out;
  void* data[2];        // internal halves (parity 0, 1)
  float* norm[2];
};
cudaError_t launch_pack(int prec, const PackParams& p, cudaStream_t st);
cudaError_t launch_unpack(int prec, const PackParams& p, cudaStream_t st);

struct GaugeParams {
  Geom g;
  const double* user;   // user links (device)
  double* out64[2];     // internal F64 gauge per parity
  int gs;               // stride of the F64 layout (18 or 12)
  double t_bc;
  double* err;          // su3 check max error (device, may be null)
  // T-partitioned lattice: `user` holds T + 1 timeslices, the first being the lower
  // neighbour's last one (only its t links are read, for the backward links at t = 0);
  // bc_lo / bc_hi: the local first / last timeslice is the global one (phase t_bc)
  int ghost;
  int bc_lo, bc_hi;
};
cudaError_t launch_gauge_load(const GaugeParams& p, cudaStream_t st);
cudaError_t launch_gauge_convert(int prec, const double* in64, void* out, long long nlinks,
                                 int gs_in, int gs_out, int nreal, cudaStream_t st);

struct SrcParams {
  Geom g;
  int Ls, nrhs;
  const double* in;
  double* out;
};
// 4D -> 5D wall embedding P (b at s=0) in user layouts
cudaError_t launch_embed_wall(const SrcParams& p, cudaStream_t st);
// 5D -> 4D projection q = P_- y_0 + P_+ y_{Ls-1}
cudaError_t launch_project4d(const SrcParams& p, cudaStream_t st);
// gamma_3 gamma_5 on the spin index of 4D fields
cudaError_t launch_fh_source(const SrcParams& p, cudaStream_t st);
// nucleon 2-pt: per-site values then per-timeslice fixed-order sums
struct NucMats {          // row-major 4x4 complex spin matrices
  double car[16], cai[16];  // C gamma_5
  double cbr[16], cbi[16];  // gamma_4 (C gamma_5)^+ gamma_4
  double pr[16], pi[16];    // (1 + gamma_4)/2
};
// the spin matrices above in the library's chiral basis (host; one definition shared by
// the regular and the allocation-free contraction)
void nucleon_mats(NucMats* m);
cudaError_t launch_nucleon(const Geom& g, const NucMats& m, const double* u1, const double* d,
                           const double* u2, double* site_tmp, double* corr, cudaStream_t st);

}  // namespace mdwf
