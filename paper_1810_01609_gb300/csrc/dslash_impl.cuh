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
#pragma once
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"
#include "mdwf_epi.cuh"
#include "mdwf_df.cuh"
#include <type_traits>

namespace mdwf {

template <typename C>
struct cplx { C re, im; };

// psi[24] ordered [colour][spin][re,im]
#define PRE(sp, co) psi[2 * ((co) * 4 + (sp))]
#define PIM(sp, co) psi[2 * ((co) * 4 + (sp)) + 1]
#define ARE(sp, co) acc[2 * ((co) * 4 + (sp))]
#define AIM(sp, co) acc[2 * ((co) * 4 + (sp)) + 1]

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
      else if constexpr (P == I16) { f = i16x2_to_float2(t[i]); f.x *= I16_INV; f.y *= I16_INV; }
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

// Explicitly rounded arithmetic on one value (float, double) or on a pair of columns
// (float2, the packed FP32 instructions of sm_100+): the compiler makes no contraction
// choices, so the single-column and the paired-column kernels perform the same roundings
// in the same order and agree bit for bit.
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ double vmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double vneg(double a) { return -a; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

// SU(3) on a projected half spinor h (2 slots x 3 colours, complex) and reconstruction:
// upper spins += n U h, lower spins += -sig n X_mu^+ U h, n the neighbour's storage scale.
// V is the compute type, or float2 for two columns at once (U then holds every real twice).
// Per output real: re = ((ur0 hr0 - ui0 hi0) + ur1 hr1 - ui1 hi1) + ..., one rounding per
// product-add in this order.
template <int MU, int SIG, typename V>
__device__ __forceinline__ void su3_recon(const V h[12], const V* U, V acc[24], const V n) {
  const V sg = SIG > 0 ? n : vneg(n);
  const V nsg = vneg(sg);
#pragma unroll
  for (int a = 0; a < 3; a++) {
    V u0r, u0i, u1r, u1i;
    {
      const V ur = U[6 * a], ui = U[6 * a + 1], mui = vneg(ui);
      u0r = vfma(mui, h[1], vmul(ur, h[0])); u0i = vfma(ui, h[0], vmul(ur, h[1]));
      u1r = vfma(mui, h[7], vmul(ur, h[6])); u1i = vfma(ui, h[6], vmul(ur, h[7]));
    }
#pragma unroll
    for (int b = 1; b < 3; b++) {
      const V ur = U[2 * (3 * a + b)], ui = U[2 * (3 * a + b) + 1], mui = vneg(ui);
      u0r = vfma(mui, h[2 * b + 1], vfma(ur, h[2 * b], u0r));
      u0i = vfma(ui, h[2 * b], vfma(ur, h[2 * b + 1], u0i));
      u1r = vfma(mui, h[6 + 2 * b + 1], vfma(ur, h[6 + 2 * b], u1r));
      u1i = vfma(ui, h[6 + 2 * b], vfma(ur, h[6 + 2 * b + 1], u1i));
    }
    ARE(0, a) = vfma(n, u0r, ARE(0, a)); AIM(0, a) = vfma(n, u0i, AIM(0, a));
    ARE(1, a) = vfma(n, u1r, ARE(1, a)); AIM(1, a) = vfma(n, u1i, AIM(1, a));
    if (MU == 0) {         // lower0 = s i Uh1 ; lower1 = s i Uh0
      ARE(2, a) = vfma(nsg, u1i, ARE(2, a)); AIM(2, a) = vfma(sg, u1r, AIM(2, a));
      ARE(3, a) = vfma(nsg, u0i, ARE(3, a)); AIM(3, a) = vfma(sg, u0r, AIM(3, a));
    } else if (MU == 1) {  // lower0 = s Uh1 ; lower1 = -s Uh0
      ARE(2, a) = vfma(sg, u1r, ARE(2, a)); AIM(2, a) = vfma(sg, u1i, AIM(2, a));
      ARE(3, a) = vfma(nsg, u0r, ARE(3, a)); AIM(3, a) = vfma(nsg, u0i, AIM(3, a));
    } else if (MU == 2) {  // lower0 = s i Uh0 ; lower1 = -s i Uh1
      ARE(2, a) = vfma(nsg, u0i, ARE(2, a)); AIM(2, a) = vfma(sg, u0r, AIM(2, a));
      ARE(3, a) = vfma(sg, u1i, ARE(3, a)); AIM(3, a) = vfma(nsg, u1r, AIM(3, a));
    } else {               // lower0 = -s Uh0 ; lower1 = -s Uh1
      ARE(2, a) = vfma(nsg, u0r, ARE(2, a)); AIM(2, a) = vfma(nsg, u0i, AIM(2, a));
      ARE(3, a) = vfma(nsg, u1r, ARE(3, a)); AIM(3, a) = vfma(nsg, u1i, AIM(3, a));
    }
  }
}

template <int P>
__device__ __forceinline__ auto mk2(float a, float b) {
  if constexpr (P == F16) return __floats2half2_rn(a, b);
  else return __floats2bfloat162_rn(a, b);
}

// A neighbour column of a 16-bit field as stored: its three 16-byte chunks (one colour's
// four spins each) and its scale (F16 / int16 norm, 1 for BF16).  Loading and projecting
// are separate steps so that a hop loop can load the next direction's column while it
// computes the current one.
struct Raw16 { uint4 q[3]; float n; };

template <int P>
__device__ __forceinline__ void raw_load16(const Field& f, unsigned nbr, int col, Raw16& r) {
  const uint4* d = (const uint4*)f.data;
  const unsigned W = (unsigned)f.W();
#pragma unroll
  for (int c = 0; c < 3; c++) r.q[c] = __ldg(d + (nbr * 3 + c) * W + col);
  r.n = 1.0f;
  if constexpr (P == F16 || P == I16) r.n = __ldg(f.norm + nbr * W + col);
}

// Projected half spinor h (slot j, colour c at h[6j + 2c]) of a raw 16-bit column; returns
// the scale folded into the accumulation.  F16 / BF16 project in 16-bit pairs (one
// rounding of the pair sum, then exact conversion); int16 converts its exact integers and
// projects in FP32, its scale being norm / 32767.
template <int P, int MU, int SIG>
__device__ __forceinline__ float proj16(const Raw16& r, float h[12]) {
  if constexpr (P == I16) {
    float psi[24];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const uint32_t w[4] = {r.q[c].x, r.q[c].y, r.q[c].z, r.q[c].w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float2 fv = i16x2_to_float2(w[j]);
        psi[8 * c + 2 * j] = fv.x; psi[8 * c + 2 * j + 1] = fv.y;
      }
    }
    const float sg = (float)SIG;
#pragma unroll
    for (int co = 0; co < 3; co++) {
      float* h0 = h + 2 * co;
      float* h1 = h + 6 + 2 * co;
      if (MU == 0) {
        h0[0] = PRE(0, co) + sg * PIM(3, co); h0[1] = PIM(0, co) - sg * PRE(3, co);
        h1[0] = PRE(1, co) + sg * PIM(2, co); h1[1] = PIM(1, co) - sg * PRE(2, co);
      } else if (MU == 1) {
        h0[0] = PRE(0, co) - sg * PRE(3, co); h0[1] = PIM(0, co) - sg * PIM(3, co);
        h1[0] = PRE(1, co) + sg * PRE(2, co); h1[1] = PIM(1, co) + sg * PIM(2, co);
      } else if (MU == 2) {
        h0[0] = PRE(0, co) + sg * PIM(2, co); h0[1] = PIM(0, co) - sg * PRE(2, co);
        h1[0] = PRE(1, co) - sg * PIM(3, co); h1[1] = PIM(1, co) + sg * PRE(3, co);
      } else {
        h0[0] = PRE(0, co) - sg * PRE(2, co); h0[1] = PIM(0, co) - sg * PIM(2, co);
        h1[0] = PRE(1, co) - sg * PRE(3, co); h1[1] = PIM(1, co) - sg * PIM(3, co);
      }
    }
    return r.n * I16_INV;
  } else {
    using H2 = typename std::conditional<P == F16, __half2, __nv_bfloat162>::type;
    const H2 ps = mk2<P>((float)SIG, (float)SIG);
#pragma unroll
    for (int co = 0; co < 3; co++) {
      const uint4 q = r.q[co];
      const H2 w0 = *(const H2*)&q.x, w1 = *(const H2*)&q.y, w2 = *(const H2*)&q.z, w3 = *(const H2*)&q.w;
      H2 r0, r1;
      if (MU == 0 || MU == 2) {
        // i * w = (-w.im, w.re): h0 = w0 - s i wA, h1 = w1 -+ s i wB
        const H2 iA = MU == 0 ? __lowhigh2highlow(w3) : __lowhigh2highlow(w2);
        const H2 iB = MU == 0 ? __lowhigh2highlow(w2) : __lowhigh2highlow(w3);
        // -s i wA = s (wA.im, -wA.re) = iA * (s, -s)
        const H2 m0 = mk2<P>((float)SIG, (float)-SIG);
        r0 = __hfma2(iA, m0, w0);
        r1 = MU == 0 ? __hfma2(iB, m0, w1) : __hfma2(iB, __hneg2(m0), w1);
      } else if (MU == 1) {
        r0 = __hfma2(w3, __hneg2(ps), w0);
        r1 = __hfma2(w2, ps, w1);
      } else {
        r0 = __hfma2(w2, __hneg2(ps), w0);
        r1 = __hfma2(w3, __hneg2(ps), w1);
      }
      float2 f0, f1;
      if constexpr (P == F16) { f0 = __half22float2(r0); f1 = __half22float2(r1); }
      else { f0 = __bfloat1622float2(r0); f1 = __bfloat1622float2(r1); }
      h[2 * co] = f0.x; h[2 * co + 1] = f0.y;
      h[6 + 2 * co] = f1.x; h[6 + 2 * co + 1] = f1.y;
    }
    return r.n;
  }
}

// Neighbour column -> projected half spinor h in the compute precision; returns the scale
// folded into the accumulation (1 for FP64 / FP32 / BF16).
template <int P, int MU, int SIG>
__device__ __forceinline__ typename PT<P>::C load_proj(const Field& f, unsigned nbr, int col, typename PT<P>::C h[12]) {
  using C = typename PT<P>::C;
  if constexpr (P == F64 || P == F32) {
    C psi[24];
    load_site<P>(f, nbr, col, psi);
    const C sg = (C)SIG;
#pragma unroll
    for (int co = 0; co < 3; co++) {
      C* h0 = h + 2 * co;
      C* h1 = h + 6 + 2 * co;
      if (MU == 0) {
        h0[0] = PRE(0, co) + sg * PIM(3, co); h0[1] = PIM(0, co) - sg * PRE(3, co);
        h1[0] = PRE(1, co) + sg * PIM(2, co); h1[1] = PIM(1, co) - sg * PRE(2, co);
      } else if (MU == 1) {
        h0[0] = PRE(0, co) - sg * PRE(3, co); h0[1] = PIM(0, co) - sg * PIM(3, co);
        h1[0] = PRE(1, co) + sg * PRE(2, co); h1[1] = PIM(1, co) + sg * PIM(2, co);
      } else if (MU == 2) {
        h0[0] = PRE(0, co) + sg * PIM(2, co); h0[1] = PIM(0, co) - sg * PRE(2, co);
        h1[0] = PRE(1, co) - sg * PIM(3, co); h1[1] = PIM(1, co) + sg * PRE(3, co);
      } else {
        h0[0] = PRE(0, co) - sg * PRE(2, co); h0[1] = PIM(0, co) - sg * PIM(2, co);
        h1[0] = PRE(1, co) - sg * PRE(3, co); h1[1] = PIM(1, co) - sg * PIM(3, co);
      }
    }
    return (C)1;
  } else {
    Raw16 r;
    raw_load16<P>(f, nbr, col, r);
    return proj16<P, MU, SIG>(r, h);
  }
}

// The projected half spinor of a neighbour across the partition boundary, read from the
// face the neighbouring partition packed (pack_face_kernel: the same 12 reals load_proj
// forms, and for F16 / int16 the neighbour's scale as load_proj returns it).  nbr is the neighbour's index in the local
// lattice with periodic wrap, i.e. face_base + the face site.
template <int P>
__device__ __forceinline__ typename PT<P>::C load_face(const HopParams& p, unsigned nbr, int col,
                                                       typename PT<P>::C h[12]) {
  using C = typename PT<P>::C;
  const long long W = p.in.W();
  const long long f = ((long long)nbr - p.face_base) * W + col;
  const C* src = (const C*)p.face + f * 12;
#pragma unroll
  for (int k = 0; k < 12; k++) h[k] = src[k];
  if constexpr (PT<P>::NORM) return p.face_norm[f];
  return (C)1;
}

// ---------------------------------------------------------------- emulated FP64 hop
// FP64 storage, double-float arithmetic (mdwf_df.cuh): the neighbour's reals and the links
// are split into float pairs, projected with TwoSum, multiplied and accumulated over all
// eight directions as compensated sums, and rounded to double once per output real.

// neighbour column -> projected half spinor (slot j, colour c at h[6j + 2c]) in double-float
template <int MU, int SIG>
__device__ __forceinline__ void load_proj_emu(const Field& f, unsigned nbr, int col, dfl h[12]) {
  const double2* d = (const double2*)f.data;
  const long long W = f.W();
  constexpr int S = SIG;
#pragma unroll
  for (int co = 0; co < 3; co++) {
    dfl re[4], im[4];
#pragma unroll
    for (int sp = 0; sp < 4; sp++) {
      const double2 q = __ldg(d + ((long long)nbr * 12 + co * 4 + sp) * W + col);
      re[sp] = split_f64(q.x); im[sp] = split_f64(q.y);
    }
    dfl* h0 = h + 2 * co;
    dfl* h1 = h + 6 + 2 * co;
    if (MU == 0) {         // h0 = p0 - s i p3 ; h1 = p1 - s i p2
      h0[0] = dadd<S>(re[0], im[3]); h0[1] = dadd<-S>(im[0], re[3]);
      h1[0] = dadd<S>(re[1], im[2]); h1[1] = dadd<-S>(im[1], re[2]);
    } else if (MU == 1) {  // h0 = p0 - s p3 ; h1 = p1 + s p2
      h0[0] = dadd<-S>(re[0], re[3]); h0[1] = dadd<-S>(im[0], im[3]);
      h1[0] = dadd<S>(re[1], re[2]); h1[1] = dadd<S>(im[1], im[2]);
    } else if (MU == 2) {  // h0 = p0 - s i p2 ; h1 = p1 + s i p3
      h0[0] = dadd<S>(re[0], im[2]); h0[1] = dadd<-S>(im[0], re[2]);
      h1[0] = dadd<-S>(re[1], im[3]); h1[1] = dadd<S>(im[1], re[3]);
    } else {               // h0 = p0 - s p2 ; h1 = p1 - s p3
      h0[0] = dadd<-S>(re[0], re[2]); h0[1] = dadd<-S>(im[0], im[2]);
      h1[0] = dadd<-S>(re[1], re[3]); h1[1] = dadd<-S>(im[1], im[3]);
    }
  }
}

// a face's projected half spinor (FP64, packed by pack_face_kernel) in double-float
__device__ __forceinline__ void load_face_emu(const HopParams& p, unsigned nbr, int col, dfl h[12]) {
  double t[12];
  load_face<F64>(p, nbr, col, t);
#pragma unroll
  for (int k = 0; k < 12; k++) h[k] = split_f64(t[k]);
}

// SU(3) on h and reconstruction, compensated: u = U h per colour row, then the upper spins
// += u and the lower ones += -sig X_mu^+ u
template <int MU, int SIG>
__device__ __forceinline__ void su3_recon_emu(const dfl h[12], const dfl* U, dacc acc[24]) {
  constexpr int S = SIG;
#pragma unroll
  for (int a = 0; a < 3; a++) {
    dacc u0r, u0i, u1r, u1i;
    {
      const dfl ur = U[6 * a], ui = U[6 * a + 1];
      u0r = dprod<1>(ur, h[0]); dfma<-1>(u0r, ui, h[1]);
      u0i = dprod<1>(ur, h[1]); dfma<1>(u0i, ui, h[0]);
      u1r = dprod<1>(ur, h[6]); dfma<-1>(u1r, ui, h[7]);
      u1i = dprod<1>(ur, h[7]); dfma<1>(u1i, ui, h[6]);
    }
#pragma unroll
    for (int b = 1; b < 3; b++) {
      const dfl ur = U[2 * (3 * a + b)], ui = U[2 * (3 * a + b) + 1];
      dfma<1>(u0r, ur, h[2 * b]); dfma<-1>(u0r, ui, h[2 * b + 1]);
      dfma<1>(u0i, ur, h[2 * b + 1]); dfma<1>(u0i, ui, h[2 * b]);
      dfma<1>(u1r, ur, h[6 + 2 * b]); dfma<-1>(u1r, ui, h[6 + 2 * b + 1]);
      dfma<1>(u1i, ur, h[6 + 2 * b + 1]); dfma<1>(u1i, ui, h[6 + 2 * b]);
    }
    dacc_add<1>(ARE(0, a), u0r); dacc_add<1>(AIM(0, a), u0i);
    dacc_add<1>(ARE(1, a), u1r); dacc_add<1>(AIM(1, a), u1i);
    if (MU == 0) {         // lower0 = s i Uh1 ; lower1 = s i Uh0
      dacc_add<-S>(ARE(2, a), u1i); dacc_add<S>(AIM(2, a), u1r);
      dacc_add<-S>(ARE(3, a), u0i); dacc_add<S>(AIM(3, a), u0r);
    } else if (MU == 1) {  // lower0 = s Uh1 ; lower1 = -s Uh0
      dacc_add<S>(ARE(2, a), u1r); dacc_add<S>(AIM(2, a), u1i);
      dacc_add<-S>(ARE(3, a), u0r); dacc_add<-S>(AIM(3, a), u0i);
    } else if (MU == 2) {  // lower0 = s i Uh0 ; lower1 = -s i Uh1
      dacc_add<-S>(ARE(2, a), u0i); dacc_add<S>(AIM(2, a), u0r);
      dacc_add<S>(ARE(3, a), u1i); dacc_add<-S>(AIM(3, a), u1r);
    } else {               // lower0 = -s Uh0 ; lower1 = -s Uh1
      dacc_add<-S>(ARE(2, a), u0r); dacc_add<-S>(AIM(2, a), u0i);
      dacc_add<-S>(ARE(3, a), u1r); dacc_add<-S>(AIM(3, a), u1i);
    }
  }
}

// Link staging stride in shared memory (compute-precision reals per link, 16-byte rows)
template <typename C> __host__ __device__ constexpr int link_stride() { return sizeof(C) == 8 ? 18 : 20; }
// ... and per site: its 8 links plus 16 bytes, so that the sites sharing a warp (whose
// threads read their own site's link) start 4 banks apart instead of on the same bank
template <typename C> __host__ __device__ constexpr int site_link_stride() { return 8 * link_stride<C>() + 16 / (int)sizeof(C); }

// OCC: the occupancy-bounded build (at least 4 CTAs of MAXTHREADS per SM, i.e. at most 64
// registers, a few spilled); the autotuner picks it or the unbounded one per kernel and
// lattice (fused 32-bit kernels only)
// EMU (FP64 storage only): the emulated-FP64 hop loop; phase 0 stages the links as
// double-float pairs, the epilogue runs in FP64 on the rounded hop result
template <int P, bool DAG, bool R12, bool EPI, bool OCC, bool EMU = false>
__global__ void __launch_bounds__(MAXTHREADS, OCC ? 4 : 0)
hop_kernel(const __grid_constant__ HopParams p) {
  static_assert(!EMU || P == F64, "emulated FP64: FP64 storage only");
  using C = typename PT<P>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.in.Ls, nrhs = p.in.nrhs;
  const int W = Ls * nrhs;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int site_l = tid / W;
  const int col = tid - site_l * W;
  const long long site0 = p.x_begin + (long long)blockIdx.x * p.ns;
  const long long x_cb = site0 + site_l;
  const bool active = x_cb < p.x_end;
  constexpr int SF = DAG ? -1 : 1;
  constexpr int LSTR = link_stride<C>();
  constexpr int SSTR = site_link_stride<C>();
  // shared: links of the CTA's sites (compute precision), neighbour table, epilogue
  C* slink = (C*)smem_raw;
  unsigned* snbr = (unsigned*)(slink + p.ns * SSTR);
  unsigned char* epi_base = (unsigned char*)(snbr + ((p.ns * 8 + 3) & ~3));

  // phase 0: one thread per (site, direction) loads and converts the link, and finds the
  // neighbour; forward links carry the boundary phase on t at T-1, backward ones on t at 0
  for (int i = tid; i < p.ns * 8; i += nt) {
    const long long x = site0 + (i >> 3);
    if (x >= p.x_end) continue;
    const int d = i & 7, mu = d & 3;
    int c[4];
    cb_coords(p.g, x, p.pout, c);
    snbr[i] = (unsigned)nbr_cb(p.g, c, mu, d < 4 ? +1 : -1);
    C U[18];
    const bool flip = R12 && mu == 3 && p.t_bc < 0 &&
                      (d < 4 ? c[3] == p.g.T - 1 && p.bc_hi : c[3] == 0 && p.bc_lo);
    load_link<P, R12>(p.gauge, (x * 8 + d) * p.gs, U, flip);
    if constexpr (EMU) {
      dfl* dl = (dfl*)(slink + (i >> 3) * SSTR + (i & 7) * LSTR);   // 18 pairs in the 18 doubles' space
#pragma unroll
      for (int k = 0; k < 18; k++) dl[k] = split_f64(U[k]);
    } else {
#pragma unroll
      for (int k = 0; k < 18; k++) slink[(i >> 3) * SSTR + (i & 7) * LSTR + k] = U[k];
    }
  }
  __syncthreads();

  C acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = 0;
  if constexpr (EMU) {
    if (active) {
      const unsigned* nb = snbr + site_l * 8;
      const dfl* lk = (const dfl*)(slink + site_l * SSTR);
      dacc da[24];
#pragma unroll
      for (int i = 0; i < 24; i++) da[i] = {0.0f, 0.0f};
      dfl h[12];
#define HOPE_D(D, MU, SIG)                                                                \
      { if (((D) == 7 && p.face_mode == 1) || ((D) == 3 && p.face_mode == 2)) load_face_emu(p, nb[D], col, h); \
        else load_proj_emu<MU, SIG>(p.in, nb[D], col, h);                                  \
        su3_recon_emu<MU, SIG>(h, lk + (D) * LSTR, da); }
      HOPE_D(0, 0, SF) HOPE_D(4, 0, -SF) HOPE_D(1, 1, SF) HOPE_D(5, 1, -SF)
      HOPE_D(2, 2, SF) HOPE_D(6, 2, -SF) HOPE_D(3, 3, SF) HOPE_D(7, 3, -SF)
#undef HOPE_D
#pragma unroll
      for (int i = 0; i < 24; i++) acc[i] = dfl_to_f64(da[i].s, da[i].e);
    }
  } else if (active) {
    const unsigned* nb = snbr + site_l * 8;
    const C* lk = slink + site_l * SSTR;
    C h[12];
#define HOP_D(D, MU, SIG)                                                                 \
    { const C nrm = ((D) == 7 && p.face_mode == 1) || ((D) == 3 && p.face_mode == 2)       \
                        ? load_face<P>(p, nb[D], col, h) : load_proj<P, MU, SIG>(p.in, nb[D], col, h); \
      su3_recon<MU, SIG>(h, lk + (D) * LSTR, acc, nrm); }
    HOP_D(0, 0, SF) HOP_D(4, 0, -SF) HOP_D(1, 1, SF) HOP_D(5, 1, -SF)
    HOP_D(2, 2, SF) HOP_D(6, 2, -SF) HOP_D(3, 3, SF) HOP_D(7, 3, -SF)
#undef HOP_D
  }

  if constexpr (!EPI) {
    if (active) store_site<P>(p.out, x_cb, col, acc);
    return;
  } else {
    const int GS = tile_gstr(Ls);
    const int ngrp = p.ns * nrhs;
    C* tileH = (C*)epi_base;
    const size_t toff = ((size_t)ngrp * GS * sizeof(C) + 15) & ~(size_t)15;
    double* redsm = (double*)(epi_base + toff);
    const int r = col / Ls, s = col - r * Ls;
    const int grp = site_l * nrhs + r;
    if (active) {
      C* dst = tileH + grp * GS + s * TSTR;
      if constexpr (sizeof(C) == 4) {
#pragma unroll
        for (int k = 0; k < 24; k += 4) *(float4*)(dst + k) = make_float4(acc[k], acc[k + 1], acc[k + 2], acc[k + 3]);
      } else {
#pragma unroll
        for (int k = 0; k < 24; k += 2) *(double2*)(dst + k) = make_double2(acc[k], acc[k + 1]);
      }
    }
    __syncthreads();
    hop_epilogue<P>(p, tileH, redsm, p.ns);
  }
}

// Paired-column variant for the 32-bit compute types: thread (site_l, c) computes columns
// c and c + W/2 of its site (W = nrhs * Ls even) on float2 = (column c, column c + W/2)
// with the packed FP32 instructions, so one instruction stream carries two 5D sites and
// each staged link real, loaded once as a duplicated pair, serves both.  Same roundings
// in the same order as hop_kernel: the two kernels agree bit for bit.
template <int P, bool DAG, bool R12, bool EPI>
__global__ void __launch_bounds__(MAXTHREADS)
hop2_kernel(const __grid_constant__ HopParams p) {
  using C = float;
  static_assert(P != F64, "paired columns: 32-bit compute types only");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.in.Ls, nrhs = p.in.nrhs;
  const int W = Ls * nrhs, W2 = W >> 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int site_l = tid / W2;
  const int colA = tid - site_l * W2, colB = colA + W2;
  const long long site0 = p.x_begin + (long long)blockIdx.x * p.ns;
  const long long x_cb = site0 + site_l;
  const bool active = x_cb < p.x_end;
  constexpr int SF = DAG ? -1 : 1;
  // shared: links as duplicated pairs (18 float2 = 144 bytes per link), neighbour table,
  // epilogue
  constexpr int SSTR2 = 8 * 18 + 2;   // float2 per site: 8 links + 16 bytes (bank offset)
  float2* slink = (float2*)smem_raw;
  unsigned* snbr = (unsigned*)(slink + p.ns * SSTR2);
  unsigned char* epi_base = (unsigned char*)(snbr + ((p.ns * 8 + 3) & ~3));

  for (int i = tid; i < p.ns * 8; i += nt) {
    const long long x = site0 + (i >> 3);
    if (x >= p.x_end) continue;
    const int d = i & 7, mu = d & 3;
    int c[4];
    cb_coords(p.g, x, p.pout, c);
    snbr[i] = (unsigned)nbr_cb(p.g, c, mu, d < 4 ? +1 : -1);
    C U[18];
    const bool flip = R12 && mu == 3 && p.t_bc < 0 &&
                      (d < 4 ? c[3] == p.g.T - 1 && p.bc_hi : c[3] == 0 && p.bc_lo);
    load_link<P, R12>(p.gauge, (x * 8 + d) * p.gs, U, flip);
    float4* dst = (float4*)(slink + (i >> 3) * SSTR2 + (i & 7) * 18);
#pragma unroll
    for (int k = 0; k < 18; k += 2) dst[k >> 1] = make_float4(U[k], U[k], U[k + 1], U[k + 1]);
  }
  __syncthreads();

  float2 acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = make_float2(0.0f, 0.0f);
  if (active) {
    const unsigned* nb = snbr + site_l * 8;
    const float2* lk = slink + site_l * SSTR2;
    C hA[12], hB[12];
    float2 h[12];
#define HOP2_D(D, MU, SIG)                                                                \
    { const bool fc = ((D) == 7 && p.face_mode == 1) || ((D) == 3 && p.face_mode == 2);    \
      const C nA = fc ? load_face<P>(p, nb[D], colA, hA) : load_proj<P, MU, SIG>(p.in, nb[D], colA, hA); \
      const C nB = fc ? load_face<P>(p, nb[D], colB, hB) : load_proj<P, MU, SIG>(p.in, nb[D], colB, hB); \
      _Pragma("unroll") for (int k = 0; k < 12; k++) h[k] = make_float2(hA[k], hB[k]);     \
      su3_recon<MU, SIG>(h, lk + (D) * 18, acc, make_float2(nA, nB)); }
    HOP2_D(0, 0, SF) HOP2_D(4, 0, -SF) HOP2_D(1, 1, SF) HOP2_D(5, 1, -SF)
    HOP2_D(2, 2, SF) HOP2_D(6, 2, -SF) HOP2_D(3, 3, SF) HOP2_D(7, 3, -SF)
#undef HOP2_D
  }

  if constexpr (!EPI) {
    if (active) {
      C v[24];
#pragma unroll
      for (int k = 0; k < 24; k++) v[k] = acc[k].x;
      store_site<P>(p.out, x_cb, colA, v);
#pragma unroll
      for (int k = 0; k < 24; k++) v[k] = acc[k].y;
      store_site<P>(p.out, x_cb, colB, v);
    }
    return;
  } else {
    const int GS = tile_gstr(Ls);
    const int ngrp = p.ns * nrhs;
    C* tileH = (C*)epi_base;
    const size_t toff = ((size_t)ngrp * GS * sizeof(C) + 15) & ~(size_t)15;
    double* redsm = (double*)(epi_base + toff);
    if (active) {
      const int rA = colA / Ls, sA = colA - rA * Ls, rB = colB / Ls, sB = colB - rB * Ls;
      C* dA = tileH + (site_l * nrhs + rA) * GS + sA * TSTR;
      C* dB = tileH + (site_l * nrhs + rB) * GS + sB * TSTR;
#pragma unroll
      for (int k = 0; k < 24; k += 4) {
        *(float4*)(dA + k) = make_float4(acc[k].x, acc[k + 1].x, acc[k + 2].x, acc[k + 3].x);
        *(float4*)(dB + k) = make_float4(acc[k].y, acc[k + 1].y, acc[k + 2].y, acc[k + 3].y);
      }
    }
    __syncthreads();
    hop_epilogue<P>(p, tileH, redsm, p.ns);
  }
}

template <int P, bool DAG, bool R12, bool EPI>
static cudaError_t launch_pair(const HopParams& p, int threads, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(hop2_kernel<P, DAG, R12, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long blocks = (p.x_end - p.x_begin + p.ns - 1) / p.ns;
  HopParams q = p;
  q.hcf = (float)p.hc; q.ccf = (float)p.cc; q.mff = (float)p.mf;
  hop2_kernel<P, DAG, R12, EPI><<<(unsigned)blocks, threads, smem, st>>>(q);
  return cudaGetLastError();
}

// all (dagger, 12-real links, epilogue) variants of the paired-column kernel of one
// 32-bit storage precision
template <int P>
cudaError_t launch_hop2_prec(const HopParams& p, bool dag, bool r12, bool epi, int threads, size_t smem,
                             cudaStream_t st) {
  if (dag) {
    if (r12) return epi ? launch_pair<P, true, true, true>(p, threads, smem, st) : launch_pair<P, true, true, false>(p, threads, smem, st);
    return epi ? launch_pair<P, true, false, true>(p, threads, smem, st) : launch_pair<P, true, false, false>(p, threads, smem, st);
  }
  if (r12) return epi ? launch_pair<P, false, true, true>(p, threads, smem, st) : launch_pair<P, false, true, false>(p, threads, smem, st);
  return epi ? launch_pair<P, false, false, true>(p, threads, smem, st) : launch_pair<P, false, false, false>(p, threads, smem, st);
}

// ---------------------------------------------------------------- bulk-staged hop
// 16-bit storage: after phase 0 the CTA issues one asynchronous bulk copy (the TMA engine,
// cp.async.bulk) per (site, direction) of the neighbour's whole row -- its 3 chunks
// of every column, 48 W contiguous bytes -- into shared memory, all completing on one
// mbarrier; the threads load their neighbours' scales meanwhile, wait once (bounded), and
// run the hop loop from shared memory.  Same arithmetic as hop_kernel (bit-identical).

constexpr int BULK_WAIT_SPINS = 1 << 24;   // bounded mbarrier wait (about a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bulk_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < BULK_WAIT_SPINS; it++) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
    if (it >= 8) __nanosleep(64);
  }
  return false;
}

template <int P, bool DAG, bool R12, bool EPI>
__global__ void __launch_bounds__(MAXTHREADS)
hop_bulk_kernel(const __grid_constant__ HopParams p) {
  static_assert(P == F16 || P == BF16 || P == I16, "bulk-staged hop: 16-bit storage only");
  using C = float;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int Ls = p.in.Ls, nrhs = p.in.nrhs;
  const int W = Ls * nrhs;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int site_l = tid / W;
  const int col = tid - site_l * W;
  const long long site0 = p.x_begin + (long long)blockIdx.x * p.ns;
  const long long x_cb = site0 + site_l;
  const bool active = x_cb < p.x_end;
  const int nact = (int)min((long long)p.ns, p.x_end - site0);
  constexpr int SF = DAG ? -1 : 1;
  constexpr int LSTR = 20;
  constexpr int SSTR = site_link_stride<C>();
  const BulkLayout BL = bulk_layout(p.ns, W);
  C* slink = (C*)smem_raw;
  unsigned* snbr = (unsigned*)(smem_raw + BL.nbr);
  uint64_t* bar = (uint64_t*)(smem_raw + BL.bar);
  unsigned char* rows = smem_raw + BL.rows;
  unsigned char* epi_base = smem_raw + BL.epi;
  const uint32_t rb = 48u * (uint32_t)W;   // bytes of one neighbour row

  // one arrival (thread 0, with the transaction count of all the rows) completes the
  // barrier's phase 0 once every row has landed
  const uint32_t bar_a = smem_u32(bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar_a),
                 "r"((uint32_t)nact * 8u * rb)
                 : "memory");
  }
  for (int i = tid; i < p.ns * 8; i += nt) {
    const long long x = site0 + (i >> 3);
    if (x >= p.x_end) continue;
    const int d = i & 7, mu = d & 3;
    int c[4];
    cb_coords(p.g, x, p.pout, c);
    snbr[i] = (unsigned)nbr_cb(p.g, c, mu, d < 4 ? +1 : -1);
    C U[18];
    const bool flip = R12 && mu == 3 && p.t_bc < 0 &&
                      (d < 4 ? c[3] == p.g.T - 1 && p.bc_hi : c[3] == 0 && p.bc_lo);
    load_link<P, R12>(p.gauge, (x * 8 + d) * p.gs, U, flip);
#pragma unroll
    for (int k = 0; k < 18; k++) slink[(i >> 3) * SSTR + (i & 7) * LSTR + k] = U[k];
  }
  __syncthreads();

  // the neighbour rows, one bulk copy each (every row of the CTA's active sites, whatever
  // the thread count)
  {
    const unsigned char* src = (const unsigned char*)p.in.data;
    for (int i = tid; i < nact * 8; i += nt)
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                       smem_u32(rows + (size_t)i * rb)),
                   "l"(src + (size_t)snbr[i] * rb), "r"(rb), "r"(bar_a)
                   : "memory");
  }
  // the scales of this thread's eight neighbour columns, while the rows arrive
  const unsigned* nb = snbr + site_l * 8;
  float nsc[8];
#pragma unroll
  for (int d = 0; d < 8; d++) nsc[d] = 1.0f;
  if constexpr (P == F16 || P == I16) {
    if (active) {
#pragma unroll
      for (int d = 0; d < 8; d++) nsc[d] = __ldg(p.in.norm + (long long)nb[d] * W + col);
    }
  }
  if (!bulk_wait(bar_a, 0)) {
    if (tid == 0 && p.status) atomicOr(p.status, 1);
    bulk_wait(bar_a, 0);   // a second bounded wait before the rows' memory can be left
  }

  C acc[24];
#pragma unroll
  for (int i = 0; i < 24; i++) acc[i] = 0;
  if (active) {
    const C* lk = slink + site_l * SSTR;
    const unsigned char* myrows = rows + (size_t)site_l * 8 * rb + (size_t)col * 16;
    C h[12];
#define HOPB_D(D, MU, SIG)                                                                \
    { C nrm;                                                                              \
      if (((D) == 7 && p.face_mode == 1) || ((D) == 3 && p.face_mode == 2)) {             \
        nrm = load_face<P>(p, nb[D], col, h);                                             \
      } else {                                                                            \
        Raw16 r;                                                                          \
        _Pragma("unroll") for (int c = 0; c < 3; c++)                                     \
            r.q[c] = *(const uint4*)(myrows + (size_t)(D) * rb + (size_t)c * W * 16);      \
        r.n = nsc[D];                                                                     \
        nrm = proj16<P, MU, SIG>(r, h);                                                   \
      }                                                                                   \
      su3_recon<MU, SIG>(h, lk + (D) * LSTR, acc, nrm); }
    HOPB_D(0, 0, SF) HOPB_D(4, 0, -SF) HOPB_D(1, 1, SF) HOPB_D(5, 1, -SF)
    HOPB_D(2, 2, SF) HOPB_D(6, 2, -SF) HOPB_D(3, 3, SF) HOPB_D(7, 3, -SF)
#undef HOPB_D
  }

  if constexpr (!EPI) {
    if (active) store_site<P>(p.out, x_cb, col, acc);
    return;
  } else {
    const int GS = tile_gstr(Ls);
    const int ngrp = p.ns * nrhs;
    C* tileH = (C*)epi_base;
    const size_t toff = ((size_t)ngrp * GS * sizeof(C) + 15) & ~(size_t)15;
    double* redsm = (double*)(epi_base + toff);
    const int r = col / Ls, s = col - r * Ls;
    const int grp = site_l * nrhs + r;
    if (active) {
      C* dst = tileH + grp * GS + s * TSTR;
#pragma unroll
      for (int k = 0; k < 24; k += 4) *(float4*)(dst + k) = make_float4(acc[k], acc[k + 1], acc[k + 2], acc[k + 3]);
    }
    __syncthreads();
    hop_epilogue<P>(p, tileH, redsm, p.ns);
  }
}

template <int P, bool DAG, bool R12, bool EPI>
static cudaError_t launch_bulk(const HopParams& p, int threads, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(hop_bulk_kernel<P, DAG, R12, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long blocks = (p.x_end - p.x_begin + p.ns - 1) / p.ns;
  HopParams q = p;
  q.hcf = (float)p.hc; q.ccf = (float)p.cc; q.mff = (float)p.mf;
  hop_bulk_kernel<P, DAG, R12, EPI><<<(unsigned)blocks, threads, smem, st>>>(q);
  return cudaGetLastError();
}

// all (dagger, 12-real links, epilogue) variants of the bulk-staged kernel of one 16-bit
// storage precision
template <int P>
cudaError_t launch_hop_bulk_prec(const HopParams& p, bool dag, bool r12, bool epi, int threads, size_t smem,
                                 cudaStream_t st) {
  if (dag) {
    if (r12) return epi ? launch_bulk<P, true, true, true>(p, threads, smem, st) : launch_bulk<P, true, true, false>(p, threads, smem, st);
    return epi ? launch_bulk<P, true, false, true>(p, threads, smem, st) : launch_bulk<P, true, false, false>(p, threads, smem, st);
  }
  if (r12) return epi ? launch_bulk<P, false, true, true>(p, threads, smem, st) : launch_bulk<P, false, true, false>(p, threads, smem, st);
  return epi ? launch_bulk<P, false, false, true>(p, threads, smem, st) : launch_bulk<P, false, false, false>(p, threads, smem, st);
}

template <int P, bool DAG, bool R12, bool EPI, bool OCC = false, bool EMU = false>
static cudaError_t launch_one(const HopParams& p, int threads, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(hop_kernel<P, DAG, R12, EPI, OCC, EMU>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long blocks = (p.x_end - p.x_begin + p.ns - 1) / p.ns;
  HopParams q = p;   // scalars rounded once for the 32-bit kernels
  q.hcf = (float)p.hc; q.ccf = (float)p.cc; q.mff = (float)p.mf;
  hop_kernel<P, DAG, R12, EPI, OCC, EMU><<<(unsigned)blocks, threads, smem, st>>>(q);
  return cudaGetLastError();
}

// the emulated-FP64 variants (FP64 storage)
template <bool DAG, bool R12>
static cudaError_t launch_emu(const HopParams& p, bool epi, int threads, size_t smem, cudaStream_t st) {
  return epi ? launch_one<F64, DAG, R12, true, false, true>(p, threads, smem, st)
             : launch_one<F64, DAG, R12, false, false, true>(p, threads, smem, st);
}

template <int P, bool DAG, bool R12>
static cudaError_t launch_epi(const HopParams& p, bool occ, int threads, size_t smem, cudaStream_t st) {
  if constexpr (P != F64) {
    if (occ) return launch_one<P, DAG, R12, true, true>(p, threads, smem, st);
  }
  return launch_one<P, DAG, R12, true>(p, threads, smem, st);
}

// all (dagger, 12-real links, epilogue, occupancy-bounded; FP64: emulated) variants of one
// storage precision
template <int P>
cudaError_t launch_hop_prec(const HopParams& p, bool dag, bool r12, bool epi, bool occ, bool emu, int threads,
                            size_t smem, cudaStream_t st) {
  if constexpr (P == F64) {
    if (emu) {
      if (dag) return r12 ? launch_emu<true, true>(p, epi, threads, smem, st) : launch_emu<true, false>(p, epi, threads, smem, st);
      return r12 ? launch_emu<false, true>(p, epi, threads, smem, st) : launch_emu<false, false>(p, epi, threads, smem, st);
    }
  }
  if (dag) {
    if (r12) return epi ? launch_epi<P, true, true>(p, occ, threads, smem, st) : launch_one<P, true, true, false>(p, threads, smem, st);
    return epi ? launch_epi<P, true, false>(p, occ, threads, smem, st) : launch_one<P, true, false, false>(p, threads, smem, st);
  }
  if (r12) return epi ? launch_epi<P, false, true>(p, occ, threads, smem, st) : launch_one<P, false, true, false>(p, threads, smem, st);
  return epi ? launch_epi<P, false, false>(p, occ, threads, smem, st) : launch_one<P, false, false, false>(p, threads, smem, st);
}

}  // namespace mdwf
