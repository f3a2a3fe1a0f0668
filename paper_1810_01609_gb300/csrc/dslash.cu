// Wilson hopping term of the Moebius domain-wall operator (Sec. "Current State of the
// Art": a radius-one stencil on L^3 x T x L5 x Nc x Ns), fused with the s-direction
// operators (M5 / M5^-1 / D5), the CG axpy and FP64-accumulated norms.
//
//   H psi(x) = sum_mu (1 - sig gamma_mu) U_mu(x) psi(x+mu) + (1 + sig gamma_mu) U_mu(x-mu)^+ psi(x-mu)
//   sig = +1 for H, -1 for H^+ = gamma5 H gamma5.
//
// Chiral basis gamma_mu = [[0, X_mu], [X_mu^+, 0]], X_k = i sigma_k, X_t = 1:
// (1 - sig gamma_mu) psi = (h, -sig X_mu^+ h) with the half spinor h = psi_u - sig X_mu psi_d,
// so each direction multiplies one SU(3) matrix into two colour vectors.
//
// Thread layout: a CTA owns ns whole 4D sites; thread (site_l, r, s) computes the hop of
// one 5D site of one right-hand side, so link loads are shared by the nrhs * Ls threads of
// a site through L1.  The epilogue stages the hop result in shared memory, where one
// thread per (site, rhs, real component) applies the s-direction chains in place.
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"
#include "mdwf_epi.cuh"

namespace mdwf {

template <typename C>
struct cplx { C re, im; };

// psi[24] ordered [colour][spin][re,im]
#define PRE(sp, co) psi[2 * ((co) * 4 + (sp))]
#define PIM(sp, co) psi[2 * ((co) * 4 + (sp)) + 1]
#define ARE(sp, co) acc[2 * ((co) * 4 + (sp))]
#define AIM(sp, co) acc[2 * ((co) * 4 + (sp)) + 1]

template <int MU, int SIG, typename C>
__device__ __forceinline__ void hop_dir(const C psi[24], const C U[18], C acc[24]) {
  const C sg = (C)SIG;
  cplx<C> h0[3], h1[3];
#pragma unroll
  for (int co = 0; co < 3; co++) {
    if (MU == 0) {         // h0 = p0 - s i p3 ; h1 = p1 - s i p2
      h0[co] = {PRE(0, co) + sg * PIM(3, co), PIM(0, co) - sg * PRE(3, co)};
      h1[co] = {PRE(1, co) + sg * PIM(2, co), PIM(1, co) - sg * PRE(2, co)};
    } else if (MU == 1) {  // h0 = p0 - s p3 ; h1 = p1 + s p2
      h0[co] = {PRE(0, co) - sg * PRE(3, co), PIM(0, co) - sg * PIM(3, co)};
      h1[co] = {PRE(1, co) + sg * PRE(2, co), PIM(1, co) + sg * PIM(2, co)};
    } else if (MU == 2) {  // h0 = p0 - s i p2 ; h1 = p1 + s i p3
      h0[co] = {PRE(0, co) + sg * PIM(2, co), PIM(0, co) - sg * PRE(2, co)};
      h1[co] = {PRE(1, co) - sg * PIM(3, co), PIM(1, co) + sg * PRE(3, co)};
    } else {               // h0 = p0 - s p2 ; h1 = p1 - s p3
      h0[co] = {PRE(0, co) - sg * PRE(2, co), PIM(0, co) - sg * PIM(2, co)};
      h1[co] = {PRE(1, co) - sg * PRE(3, co), PIM(1, co) - sg * PIM(3, co)};
    }
  }
#pragma unroll
  for (int a = 0; a < 3; a++) {
    cplx<C> u0 = {0, 0}, u1 = {0, 0};
#pragma unroll
    for (int b = 0; b < 3; b++) {
      const C ur = U[2 * (3 * a + b)], ui = U[2 * (3 * a + b) + 1];
      u0.re += ur * h0[b].re - ui * h0[b].im;
      u0.im += ur * h0[b].im + ui * h0[b].re;
      u1.re += ur * h1[b].re - ui * h1[b].im;
      u1.im += ur * h1[b].im + ui * h1[b].re;
    }
    ARE(0, a) += u0.re; AIM(0, a) += u0.im;
    ARE(1, a) += u1.re; AIM(1, a) += u1.im;
    if (MU == 0) {         // lower0 = s i Uh1 ; lower1 = s i Uh0
      ARE(2, a) -= sg * u1.im; AIM(2, a) += sg * u1.re;
      ARE(3, a) -= sg * u0.im; AIM(3, a) += sg * u0.re;
    } else if (MU == 1) {  // lower0 = s Uh1 ; lower1 = -s Uh0
      ARE(2, a) += sg * u1.re; AIM(2, a) += sg * u1.im;
      ARE(3, a) -= sg * u0.re; AIM(3, a) -= sg * u0.im;
    } else if (MU == 2) {  // lower0 = s i Uh0 ; lower1 = -s i Uh1
      ARE(2, a) -= sg * u0.im; AIM(2, a) += sg * u0.re;
      ARE(3, a) += sg * u1.im; AIM(3, a) -= sg * u1.re;
    } else {               // lower0 = -s Uh0 ; lower1 = -s Uh1
      ARE(2, a) -= sg * u0.re; AIM(2, a) -= sg * u0.im;
      ARE(3, a) -= sg * u1.re; AIM(3, a) -= sg * u1.im;
    }
  }
}

// Load one link (18 reals, row-major [a][b] complex) in compute precision.
template <int P, bool R12>
__device__ __forceinline__ void load_link(const void* base, long long off, typename PT<P>::C U[18],
                                          bool flip) {
  using C = typename PT<P>::C;
  constexpr int NR = R12 ? 12 : 18;
  if constexpr (P == F64) {
    const double2* g = (const double2*)((const double*)base + off);
#pragma unroll
    for (int i = 0; i < NR / 2; i++) { double2 q = __ldg(g + i); U[2 * i] = q.x; U[2 * i + 1] = q.y; }
  } else if constexpr (P == F32) {
    const float4* g = (const float4*)((const float*)base + off);
    constexpr int NQ = R12 ? 3 : 5;
    float t[20];
#pragma unroll
    for (int i = 0; i < NQ; i++) { float4 q = __ldg(g + i); t[4 * i] = q.x; t[4 * i + 1] = q.y; t[4 * i + 2] = q.z; t[4 * i + 3] = q.w; }
#pragma unroll
    for (int i = 0; i < NR; i++) U[i] = t[i];
  } else {
    using G = typename PT<P>::G;
    const uint4* g = (const uint4*)((const G*)base + off);
    constexpr int NQ = R12 ? 2 : 3;
    uint32_t t[12];
#pragma unroll
    for (int i = 0; i < NQ; i++) { uint4 q = __ldg(g + i); t[4 * i] = q.x; t[4 * i + 1] = q.y; t[4 * i + 2] = q.z; t[4 * i + 3] = q.w; }
#pragma unroll
    for (int i = 0; i < NR / 2; i++) {
      float2 f;
      if constexpr (P == F16) f = __half22float2(*(const __half2*)&t[i]);
      else f = __bfloat1622float2(*(const __nv_bfloat162*)&t[i]);
      U[2 * i] = f.x; U[2 * i + 1] = f.y;
    }
  }
  if constexpr (R12) {
    // row2 = conj(row0 x row1), times the boundary phase the stored rows carry
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;
      const C ar = U[2 * i], ai = U[2 * i + 1], br = U[6 + 2 * j], bi = U[6 + 2 * j + 1];
      const C cr = U[2 * j], ci = U[2 * j + 1], dr = U[6 + 2 * i], di = U[6 + 2 * i + 1];
      C re = (ar * br - ai * bi) - (cr * dr - ci * di);
      C im = (ar * bi + ai * br) - (cr * di + ci * dr);
      U[12 + 2 * k] = flip ? -re : re;
      U[12 + 2 * k + 1] = flip ? im : -im;
    }
  }
}

template <int P, bool DAG, bool R12, bool EPI>
__global__ void __launch_bounds__(MAXTHREADS)
hop_kernel(const __grid_constant__ HopParams p) {
  using C = typename PT<P>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.in.Ls, nrhs = p.in.nrhs;
  const int W = Ls * nrhs;
  const int tid = threadIdx.x;
  const int site_l = tid / W;
  const int col = tid - site_l * W;
  const long long x_cb = (long long)blockIdx.x * p.ns + site_l;
  const bool active = x_cb < p.g.vh;
  constexpr int SF = DAG ? -1 : 1;

  C acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = 0;

  if (active) {
    int c[4];
    cb_coords(p.g, x_cb, p.pout, c);
    const long long gbase = x_cb * 8 * p.gs;
    C U[18], psi[24];
    // forward links carry the boundary phase on t at T-1, backward ones on t at 0
#define HOP_MU(MU)                                                                   \
    {                                                                                \
      load_site<P>(p.in, nbr_cb(p.g, c, MU, +1), col, psi);                          \
      load_link<P, R12>(p.gauge, gbase + (MU) * p.gs, U,                             \
                        R12 && MU == 3 && c[3] == p.g.T - 1 && p.t_bc < 0);          \
      hop_dir<MU, SF>(psi, U, acc);                                                  \
      load_site<P>(p.in, nbr_cb(p.g, c, MU, -1), col, psi);                          \
      load_link<P, R12>(p.gauge, gbase + (4 + MU) * p.gs, U,                         \
                        R12 && MU == 3 && c[3] == 0 && p.t_bc < 0);                  \
      hop_dir<MU, -SF>(psi, U, acc);                                                 \
    }
    HOP_MU(0) HOP_MU(1) HOP_MU(2) HOP_MU(3)
#undef HOP_MU
  }

  if constexpr (!EPI) {
    if (active) store_site<P>(p.out, x_cb, col, acc);
    return;
  } else {
    const int LsP = Ls + 1;
    const int ngrp = p.ns * nrhs;
    C* tileH = (C*)smem_raw;
    C* tileC = tileH + ngrp * 24 * LsP;
    const size_t toff = ((size_t)ngrp * 24 * LsP * sizeof(C) * (p.has_center ? 2 : 1) + 15) & ~(size_t)15;
    double* redsm = (double*)(smem_raw + toff);
    const int r = col / Ls, s = col - r * Ls;
    const int grp = site_l * nrhs + r;
    if (active) {
#pragma unroll
      for (int k = 0; k < 24; k++) tileH[(grp * 24 + k) * LsP + s] = acc[k];
    }
    __syncthreads();
    hop_epilogue<P>(p, tileH, tileC, redsm, p.ns);
  }
}

template <int P, bool DAG, bool R12, bool EPI>
static cudaError_t launch_one(const HopParams& p, int threads, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(hop_kernel<P, DAG, R12, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long blocks = (p.g.vh + p.ns - 1) / p.ns;
  hop_kernel<P, DAG, R12, EPI><<<(unsigned)blocks, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int P>
static cudaError_t launch_p(const HopParams& p, bool dag, bool r12, bool epi, int threads,
                            size_t smem, cudaStream_t st) {
  if (dag) {
    if (r12) return epi ? launch_one<P, true, true, true>(p, threads, smem, st) : launch_one<P, true, true, false>(p, threads, smem, st);
    return epi ? launch_one<P, true, false, true>(p, threads, smem, st) : launch_one<P, true, false, false>(p, threads, smem, st);
  }
  if (r12) return epi ? launch_one<P, false, true, true>(p, threads, smem, st) : launch_one<P, false, true, false>(p, threads, smem, st);
  return epi ? launch_one<P, false, false, true>(p, threads, smem, st) : launch_one<P, false, false, false>(p, threads, smem, st);
}

size_t hop_smem_bytes(int prec, const HopParams& p, bool epi) {
  if (!epi) return 0;
  const int threads = p.ns * p.in.nrhs * p.in.Ls;
  return epi_smem_bytes(prec == F64 ? 8 : 4, p.ns, p.in.nrhs, p.in.Ls, p.has_center, threads);
}

cudaError_t launch_hop(int prec, bool dag, bool r12, bool epi, const HopParams& p, cudaStream_t st) {
  const int threads = p.ns * p.in.nrhs * p.in.Ls;
  const size_t smem = hop_smem_bytes(prec, p, epi);
  switch (prec) {
    case F64: return launch_p<F64>(p, dag, r12, epi, threads, smem, st);
    case F32: return launch_p<F32>(p, dag, r12, epi, threads, smem, st);
    case F16: return launch_p<F16>(p, dag, r12, epi, threads, smem, st);
    case BF16: return launch_p<BF16>(p, dag, r12, epi, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace mdwf
