// Tensor-core Wilson hop for half-precision storage (F16 + per-site norm, BF16), fused
// with the s-direction epilogue of mdwf_epi.cuh.  The SU(3) products of the stencil
// (Sec. "Current State of the Art": a radius-one stencil with small dense blocks) run as
// warp-level mma.sync.m16n8k8 (f16/bf16 inputs, FP32 accumulation) on sm_103a.
//
// Mapping.  One warp owns one 4D site x and loops over its W = nrhs * Ls columns (5D
// sites) in tiles of 8.  For direction d (mu = d & 3, forward for d < 4), with
// sig = +1 for (1 - gamma_mu) and -1 for (1 + gamma_mu):
//   rows (16)  = (column c in the tile, slot j in {0,1}); slot j holds the half spinor
//                h_j = psi_j - sig (X_mu psi_d)_j of the neighbour column, which is
//                psi_j + kappa * psi_{partner(j)} with kappa in {+-1, +-i}, formed in
//                f16x2 straight from the stored chunk (one 16-byte load = one colour,
//                4 spins) without conversion;
//   K (8)      = input colour (re, im), 3 used;
//   N (8)      = output colour (re, im), 3 used;
//   B          = U_d embedded as a real 6x6 matrix, built once per site per direction.
// The MMA result (U_d h)_j is scaled in FP32 by the neighbour's per-site norm (rows
// differ per column) and accumulated: upper spin j += it, and lower spin
// (j or 1-j, by mu) += zeta * it with zeta = -sig X_mu^+ entry in {+-1, +-i}; the two
// lower contributions of a column are joined with one shuffle at the end of the tile.
// Every multiply of two stored values is exact in FP32 and sums are FP32, so the
// arithmetic matches an FP32 evaluation of the half-precision inputs up to the rounding
// of the f16x2 projection.
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"
#include "mdwf_epi.cuh"

namespace mdwf {

template <int P> struct TC;
template <> struct TC<F16> {
  using H2 = __half2;
  static __device__ __forceinline__ uint32_t h2(float a, float b) {
    H2 v = __floats2half2_rn(a, b);
    return *(uint32_t*)&v;
  }
};
template <> struct TC<BF16> {
  using H2 = __nv_bfloat162;
  static __device__ __forceinline__ uint32_t h2(float a, float b) {
    H2 v = __floats2bfloat162_rn(a, b);
    return *(uint32_t*)&v;
  }
};

template <int P>
__device__ __forceinline__ void mma16n8k8(float d[4], uint32_t a0, uint32_t a1, uint32_t b) {
  if constexpr (P == F16) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%7,%7,%7};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(b), "f"(0.0f));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5}, {%6}, {%7,%7,%7,%7};\n"
        : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
        : "r"(a0), "r"(a1), "r"(b), "f"(0.0f));
  }
}

__device__ __forceinline__ uint32_t swap_halves(uint32_t v) { return (v >> 16) | (v << 16); }

template <typename H2>
__device__ __forceinline__ uint32_t hfma2u(uint32_t a, uint32_t m, uint32_t c) {
  H2 r = __hfma2(*(const H2*)&a, *(const H2*)&m, *(const H2*)&c);
  return *(uint32_t*)&r;
}

// Per-lane constants of one direction mu for slot j.
struct DirConst {
  uint32_t mf, mb;   // f16x2 multipliers of the partner spin for sig = +1 (forward) / -1
  float zf, zb;      // lower-spin coefficient magnitude*sign for sig = +1 / -1
};

// Loads of one direction for the two rows of a lane (columns colA, colB of the tile).
struct DirLoad {
  uint4 qa, qb;
  float na, nb;
};

template <int P>
__device__ __forceinline__ void tc_load(DirLoad& L, const uint4* __restrict__ chunks, const float* __restrict__ norms,
                                        int nbr, int W, int WN, int t, int colA, int colB, bool vA, bool vB) {
  const uint4* pc = chunks + ((long long)nbr * 3 + t) * W;
  L.qa = make_uint4(0, 0, 0, 0);
  L.qb = make_uint4(0, 0, 0, 0);
  L.na = 0.f;
  L.nb = 0.f;
  if (vA) {
    L.qa = __ldg(pc + colA);
    L.na = (P == F16) ? __ldg(norms + (long long)nbr * WN + colA) : 1.f;
  }
  if (vB) {
    L.qb = __ldg(pc + colB);
    L.nb = (P == F16) ? __ldg(norms + (long long)nbr * WN + colB) : 1.f;
  }
}

// One direction: project the two rows, mma, accumulate.
template <int P, int MU, bool FWD, bool DAG>
__device__ __forceinline__ void tc_dir(const DirLoad& L, int j, uint32_t bfrag, const DirConst& k, float up[2][2],
                                       float lo_s[2][2], float lo_w[2][2]) {
  using H2 = typename TC<P>::H2;
  constexpr int SIG = (FWD != DAG) ? 1 : -1;   // (1 - sig gamma_mu)
  const uint4 qa = L.qa, qb = L.qb;
  const float na = L.na, nb = L.nb;
  // slot j of spin pair: psi_j and its partner (3-j for x,y ; 2+j for z,t)
  const uint32_t sa = j ? qa.y : qa.x, sb = j ? qb.y : qb.x;
  uint32_t pa, pb;
  if (MU <= 1) { pa = j ? qa.z : qa.w; pb = j ? qb.z : qb.w; }
  else { pa = j ? qa.w : qa.z; pb = j ? qb.w : qb.z; }
  if (MU == 0 || MU == 2) { pa = swap_halves(pa); pb = swap_halves(pb); }   // factor i
  const uint32_t m = SIG > 0 ? k.mf : k.mb;
  const uint32_t a0 = hfma2u<H2>(pa, m, sa);
  const uint32_t a1 = hfma2u<H2>(pb, m, sb);
  float d[4];
  mma16n8k8<P>(d, a0, a1, bfrag);
  // upper spin j
  up[0][0] = fmaf(na, d[0], up[0][0]); up[0][1] = fmaf(na, d[1], up[0][1]);
  up[1][0] = fmaf(nb, d[2], up[1][0]); up[1][1] = fmaf(nb, d[3], up[1][1]);
  // lower spin: x,y -> spin 1-j (swap), z,t -> spin j (same); zeta real (y,t) or imaginary (x,z)
  const float z = SIG > 0 ? k.zf : k.zb;
  const float wa = z * na, wb = z * nb;
  float(*lo)[2] = (MU <= 1) ? lo_w : lo_s;
  if (MU == 0 || MU == 2) {  // zeta = z i : (re, im) -> (-z im, z re)
    lo[0][0] = fmaf(-wa, d[1], lo[0][0]); lo[0][1] = fmaf(wa, d[0], lo[0][1]);
    lo[1][0] = fmaf(-wb, d[3], lo[1][0]); lo[1][1] = fmaf(wb, d[2], lo[1][1]);
  } else {
    lo[0][0] = fmaf(wa, d[0], lo[0][0]); lo[0][1] = fmaf(wa, d[1], lo[0][1]);
    lo[1][0] = fmaf(wb, d[2], lo[1][0]); lo[1][1] = fmaf(wb, d[3], lo[1][1]);
  }
}

template <int P, bool DAG>
__global__ void __launch_bounds__(256) hop_tc_kernel(const __grid_constant__ HopParams p) {
  using H2 = typename TC<P>::H2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.in.Ls, nrhs = p.in.nrhs, W = Ls * nrhs, LsP = Ls + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ns = blockDim.x >> 5;
  const int g = lane >> 2, t = lane & 3, j = g & 1;
  const int ngrp = ns * nrhs;
  float* tileH = (float*)smem_raw;
  float* tileC = tileH + ngrp * 24 * LsP;
  const size_t toff = ((size_t)ngrp * 24 * LsP * sizeof(float) * (p.has_center ? 2 : 1) + 15) & ~(size_t)15;
  double* redsm = (double*)(smem_raw + toff);
  const long long x_cb = (long long)blockIdx.x * ns + warp;

  if (x_cb < p.g.vh) {
    int c[4];
    cb_coords(p.g, x_cb, p.pout, c);
    int nbr[8];
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      nbr[mu] = (int)nbr_cb(p.g, c, mu, +1);
      nbr[4 + mu] = (int)nbr_cb(p.g, c, mu, -1);
    }
    // B fragments: lane (g, t) holds (k = 2t, 2t+1 ; n = g) of U_d embedded as real 6x6:
    // output re: (Re U[c][t], -Im U[c][t]) ; output im: (Im U[c][t], Re U[c][t]), c = g/2
    uint32_t bfr[8];
    const uint32_t* gl = (const uint32_t*)((const __half*)p.gauge + x_cb * 8 * p.gs);
#pragma unroll
    for (int d = 0; d < 8; d++) {
      uint32_t u = 0;
      if (g < 6 && t < 3) u = __ldg(gl + (d * p.gs) / 2 + (g >> 1) * 3 + t);
      bfr[d] = (g < 6 && t < 3) ? (j ? swap_halves(u) : (u ^ 0x80000000u)) : 0u;
    }
    // per-lane projection / reconstruction constants (see header): kappa for slot j,
    // half2 multiplier of the (possibly swapped) partner for sig = +1 / -1
    DirConst kc[4];
    {
      // kappa: x: -i, -i ; y: -1, +1 ; z: -i, +i ; t: -1, -1  ->  h = psi_j + sig kappa psi_p
      // for an i-factor the partner is swapped (im, re) and multiplied by (-s, +s) * sig*kappa_i
      const float kx = -1.f, ky = j ? 1.f : -1.f, kz = j ? 1.f : -1.f, kt = -1.f;
      kc[0].mf = TC<P>::h2(-kx, kx);
      kc[0].mb = TC<P>::h2(kx, -kx);
      kc[1].mf = TC<P>::h2(ky, ky);
      kc[1].mb = TC<P>::h2(-ky, -ky);
      kc[2].mf = TC<P>::h2(-kz, kz);
      kc[2].mb = TC<P>::h2(kz, -kz);
      kc[3].mf = TC<P>::h2(kt, kt);
      kc[3].mb = TC<P>::h2(-kt, -kt);
      // zeta = -sig X_mu^+ entry feeding the lower spin: x: sig i ; y: sig (j ? 1 : -1) ;
      // z: sig (j ? -i : i) ; t: -sig
      kc[0].zf = 1.f; kc[0].zb = -1.f;
      kc[1].zf = j ? 1.f : -1.f; kc[1].zb = -kc[1].zf;
      kc[2].zf = j ? -1.f : 1.f; kc[2].zb = -kc[2].zf;
      kc[3].zf = -1.f; kc[3].zb = 1.f;
    }
    const uint4* chunks = (const uint4*)p.in.data;
    const float* norms = p.in.norm;
    const int WN = W;
    const int nct = (W + 7) >> 3;
    for (int tile = 0; tile < nct; tile++) {
      const int colA = tile * 8 + (g >> 1), colB = colA + 4;
      const bool vA = colA < W && t < 3, vB = colB < W && t < 3;
      float up[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, ls[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, lw[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
      // all eight directions' loads first, so one memory latency covers the tile
      DirLoad L[8];
#pragma unroll
      for (int d = 0; d < 8; d++) tc_load<P>(L[d], chunks, norms, nbr[d], W, WN, t, colA, colB, vA, vB);
      tc_dir<P, 0, true, DAG>(L[0], j, bfr[0], kc[0], up, ls, lw);
      tc_dir<P, 0, false, DAG>(L[4], j, bfr[4], kc[0], up, ls, lw);
      tc_dir<P, 1, true, DAG>(L[1], j, bfr[1], kc[1], up, ls, lw);
      tc_dir<P, 1, false, DAG>(L[5], j, bfr[5], kc[1], up, ls, lw);
      tc_dir<P, 2, true, DAG>(L[2], j, bfr[2], kc[2], up, ls, lw);
      tc_dir<P, 2, false, DAG>(L[6], j, bfr[6], kc[2], up, ls, lw);
      tc_dir<P, 3, true, DAG>(L[3], j, bfr[3], kc[3], up, ls, lw);
      tc_dir<P, 3, false, DAG>(L[7], j, bfr[7], kc[3], up, ls, lw);
      // lower spin 2+j of a column = own "same" part + partner slot's "swap" part
      float lo[2][2];
#pragma unroll
      for (int rw = 0; rw < 2; rw++)
#pragma unroll
        for (int q = 0; q < 2; q++) lo[rw][q] = ls[rw][q] + __shfl_xor_sync(0xffffffffu, lw[rw][q], 4);
#pragma unroll
      for (int rw = 0; rw < 2; rw++) {
        const int col = rw ? colB : colA;
        if (col < W && t < 3) {
          const int r = col / Ls, s = col - r * Ls, grp = warp * nrhs + r;
          float* th = tileH + grp * 24 * LsP + s;
          th[(2 * (t * 4 + j)) * LsP] = up[rw][0];
          th[(2 * (t * 4 + j) + 1) * LsP] = up[rw][1];
          th[(2 * (t * 4 + 2 + j)) * LsP] = lo[rw][0];
          th[(2 * (t * 4 + 2 + j) + 1) * LsP] = lo[rw][1];
        }
      }
    }
  }
  __syncthreads();
  hop_epilogue<P>(p, tileH, tileC, redsm, ns);
}

bool hop_tc_supported(int prec, const HopParams& p, bool r12) {
  if (r12 || (prec != F16 && prec != BF16)) return false;
  if (p.gs != 24) return false;
  if (p.g.vh >= (1LL << 31) / 8) return false;
  return true;
}

template <int P, bool DAG>
static cudaError_t go_tc(const HopParams& p, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(hop_tc_kernel<P, DAG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int threads = p.ns * 32;
  const size_t smem = epi_smem_bytes(4, p.ns, p.in.nrhs, p.in.Ls, p.has_center, threads);
  const long long blocks = (p.g.vh + p.ns - 1) / p.ns;
  hop_tc_kernel<P, DAG><<<(unsigned)blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

size_t hop_tc_smem_bytes(const HopParams& p) {
  return epi_smem_bytes(4, p.ns, p.in.nrhs, p.in.Ls, p.has_center, p.ns * 32);
}

cudaError_t launch_hop_tc(int prec, bool dag, bool /*epi*/, const HopParams& p, cudaStream_t st) {
  if (prec == F16) return dag ? go_tc<F16, true>(p, st) : go_tc<F16, false>(p, st);
  if (prec == BF16) return dag ? go_tc<BF16, true>(p, st) : go_tc<BF16, false>(p, st);
  return cudaErrorNotSupported;
}

}  // namespace mdwf
