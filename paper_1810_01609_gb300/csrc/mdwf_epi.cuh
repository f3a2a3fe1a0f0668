// Shared epilogue of the fused hop kernels.  On entry tileH holds the hop result of every
// 5D site of the CTA's ns 4D sites, laid out [grp = site_l * nrhs + r][s][24 reals]
// (strides tile_gstr(Ls) and TSTR);
// the epilogue computes   out = fin( cc * cop(center) + hc * post(hop) )
// (post/cop/fin: s-direction chains of D5, A5, A5^-1 and adjoints), optionally reduces
// |out|^2 before fin, and either stores out or does r -= alpha out with |r|^2.
// post and fin run as column passes over the tile (one thread per (site, rhs, real
// component), all s in registers); cop (always empty or one bidiagonal op) only needs the
// slices s +- 1 and runs in the per-site pass, the centre read straight from global memory
// (no second tile: the epilogue's shared memory is the hop tile alone).
#pragma once
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"

namespace mdwf {

// Chunk k of the 24 reals of site (x_cb, col), in the compute type (F16 scaled by nrm).
// Chunks follow the storage: F64 one complex (2 reals), F32 two spins of one colour (4),
// F16 / BF16 all four spins of one colour (8); reals are [colour][spin][re, im].
template <int P>
__device__ __forceinline__ void load_chunk(const Field& f, long long x_cb, int col, int k, float nrm,
                                           typename PT<P>::C* out) {
  const long long W = f.W();
  if constexpr (P == F64) {
    const double2 q = __ldg((const double2*)f.data + (x_cb * 12 + k) * W + col);
    out[0] = q.x; out[1] = q.y;
  } else if constexpr (P == F32) {
    const float4 q = __ldg((const float4*)f.data + (x_cb * 6 + k) * W + col);
    out[0] = q.x; out[1] = q.y; out[2] = q.z; out[3] = q.w;
  } else {
    const uint4 q = __ldg((const uint4*)f.data + (x_cb * 3 + k) * W + col);
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int j = 0; j < 4; j++) {
      float2 v;
      if constexpr (P == F16) v = __half22float2(*(const __half2*)&w[j]);
      else if constexpr (P == I16) v = i16x2_to_float2(w[j]);
      else v = __bfloat1622float2(*(const __nv_bfloat162*)&w[j]);
      out[2 * j] = v.x * nrm; out[2 * j + 1] = v.y * nrm;
    }
  }
}

// s-neighbours of a bidiagonal op a + b S at slice s: S = B takes the upper spins (P_-) from
// s+1 and the lower ones (P_+) from s-1, S = B^+ the reverse; across the wall the value is
// -mf times the other end.  Returns the slices and the coefficients b (or -b mf).
template <typename C>
struct SNbr { int su, sl; C fu, fl; };
template <typename C>
__device__ __forceinline__ SNbr<C> s_nbr(const SOp& o, int s, int Ls, C mf) {
  const C b = sop_b<C>(o);
  const int sp = s + 1 < Ls ? s + 1 : 0, sm = s > 0 ? s - 1 : Ls - 1;
  const C fp = s + 1 < Ls ? b : -b * mf, fm = s > 0 ? b : -b * mf;
  SNbr<C> n;
  if (!o.dag) { n.su = sp; n.fu = fp; n.sl = sm; n.fl = fm; }
  else { n.su = sm; n.fu = fm; n.sl = sp; n.fl = fp; }
  return n;
}

// 16-bit pair j of a stored chunk as floats
template <int P>
__device__ __forceinline__ float2 pair16(const uint4& q, int j) {
  const uint32_t w = j == 0 ? q.x : j == 1 ? q.y : j == 2 ? q.z : q.w;
  if constexpr (P == F16) return __half22float2(*(const __half2*)&w);
  else if constexpr (P == I16) return i16x2_to_float2(w);
  else return __bfloat1622float2(*(const __nv_bfloat162*)&w);
}

// v = cc cop(center) + hc v at (x_cb, rhs r, slice s), chunk by chunk (few live
// registers); cop is empty or one bidiagonal op
template <int P>
__device__ __forceinline__ void center_combine(const HopParams& p, long long x_cb, int r, int s,
                                               typename PT<P>::C v[24]) {
  using C = typename PT<P>::C;
  const Field& f = p.center;
  const int Ls = f.Ls;
  const long long W = f.W();
  const int col = r * Ls + s;
  const C hc = pick<C>(p.hcf, p.hc), cc = pick<C>(p.ccf, p.cc);
  const SOp& o = p.cop.op[0];
  const bool bid = o.kind != SOP_NONE;
  const C a = bid ? sop_a<C>(o) : (C)1;
  SNbr<C> n = {s, s, (C)0, (C)0};
  if (bid) n = s_nbr<C>(o, s, Ls, pick<C>(p.mff, p.mf));
  const int cu = r * Ls + n.su, cl = r * Ls + n.sl;
  if constexpr (P == F64 || P == F32) {
    constexpr int NC = PT<P>::NC, CW = 24 / NC;
#pragma unroll
    for (int k = 0; k < NC; k++) {
      C own[CW], nb[CW];
      load_chunk<P>(f, x_cb, col, k, 1.0f, own);
      if (bid) {
        const bool upper = CW == 4 ? (k & 1) == 0 : (k & 3) < 2;
        load_chunk<P>(f, x_cb, upper ? cu : cl, k, 1.0f, nb);
        const C fc = upper ? n.fu : n.fl;
#pragma unroll
        for (int j = 0; j < CW; j++) own[j] = a * own[j] + fc * nb[j];
      }
#pragma unroll
      for (int j = 0; j < CW; j++) v[CW * k + j] = cc * own[j] + hc * v[CW * k + j];
    }
  } else {
    float n0 = 1.0f, nu = 1.0f, nl = 1.0f;
    if constexpr (P == F16 || P == I16) {
      const float u = P == I16 ? I16_INV : 1.0f;   // fixed-point unit
      n0 = __ldg(f.norm + x_cb * W + col) * u;
      if (bid) { nu = __ldg(f.norm + x_cb * W + cu) * n.fu * u; nl = __ldg(f.norm + x_cb * W + cl) * n.fl * u; }
    } else {
      nu = n.fu; nl = n.fl;
    }
    const float ca = cc * a * n0;
    const uint4* d = (const uint4*)f.data;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const uint4 q0 = __ldg(d + (x_cb * 3 + k) * W + col);
      uint4 qu = make_uint4(0, 0, 0, 0), ql = make_uint4(0, 0, 0, 0);
      if (bid) { qu = __ldg(d + (x_cb * 3 + k) * W + cu); ql = __ldg(d + (x_cb * 3 + k) * W + cl); }
#pragma unroll
      for (int j = 0; j < 4; j++) {
        const float2 w0 = pair16<P>(q0, j);
        float re = ca * w0.x, im = ca * w0.y;
        if (bid) {
          // spins 0, 1 (j < 2) from slice su, spins 2, 3 from slice sl
          const float2 w1 = pair16<P>(j < 2 ? qu : ql, j);
          const float m = cc * (j < 2 ? nu : nl);
          re += m * w1.x; im += m * w1.y;
        }
        v[8 * k + 2 * j] = re + hc * v[8 * k + 2 * j];
        v[8 * k + 2 * j + 1] = im + hc * v[8 * k + 2 * j + 1];
      }
    }
  }
}

// Store v (or r -= alpha v, returning |r|^2 of the site)
template <int P>
__device__ __forceinline__ double epi_output(const HopParams& p, long long x, int col, int r,
                                             const typename PT<P>::C v[24]) {
  using C = typename PT<P>::C;
  if (p.axpy_r) {
    C rv[24];
    load_site<P>(p.raxpy, x, col, rv);
    const C a = pick<C>(p.red.cg[r].alpha_f, p.red.cg[r].alpha);
    C n = 0;
#pragma unroll
    for (int k = 0; k < 24; k++) { rv[k] -= a * v[k]; n += rv[k] * rv[k]; }
    store_site<P>(p.raxpy, x, col, rv);
    return (double)n;
  }
  store_site<P>(p.out, x, col, v);
  return 0.0;
}

template <int P>
__device__ __forceinline__ void hop_epilogue(const HopParams& p, typename PT<P>::C* tileH, double* redsm, int ns) {
  using C = typename PT<P>::C;
  const int Ls = p.in.Ls, nrhs = p.in.nrhs, W = Ls * nrhs;
  const int GS = tile_gstr(Ls);
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long site0 = p.x_begin + (long long)blockIdx.x * ns;
  const int nsites = ns * W;
  const C mf = pick<C>(p.mff, p.mf), hc = pick<C>(p.hcf, p.hc), cc = pick<C>(p.ccf, p.cc);
  const bool has_post = p.post.op[0].kind != SOP_NONE;
  const bool has_fin = p.fin.op[0].kind != SOP_NONE;
  const int nitems = ns * nrhs * 24;
  // column items chirality-major (all upper-spin columns, then all lower-spin ones): the
  // two chiralities walk s in opposite directions, so a warp stays on one code path
  const int nhalf = ns * nrhs * 12;
  if (has_post) {
    for (int it2 = tid; it2 < nitems; it2 += nt) {
      const int lowerh = it2 >= nhalf;
      const int j = lowerh ? it2 - nhalf : it2;
      const int g = j / 12, q = j - g * 12;                         // q: colour (q / 4), spin pair, re/im
      const int comp = 8 * (q >> 2) + 4 * lowerh + (q & 3);
      if (site0 + (nrhs == 1 ? g : g / nrhs) >= p.x_end) continue;
      chain_apply_fast(p.post, comp, tileH + g * GS + comp, TSTR, Ls, mf);
    }
    __syncthreads();
  }
  // site pass: hc post(hop) + cc cop(center), |.|^2, then fin (column pass) or output
  const float inv_w = 1.0f / (float)W, inv_ls = 1.0f / (float)Ls;
  for (int i = tid; i < nsites; i += nt) {
    const int site_l = div_small(i, inv_w), col = i - site_l * W;
    const int r = div_small(col, inv_ls), s = col - r * Ls, grp = site_l * nrhs + r;
    const long long x = site0 + site_l;
    double part = 0.0;
    if (x < p.x_end) {
      C v[24];
      C* row = tileH + grp * GS + s * TSTR;
#pragma unroll
      for (int k = 0; k < 24; k++) v[k] = row[k];
      if (p.has_center) {
        center_combine<P>(p, x, r, s, v);
      } else if (p.hc != 1.0) {
#pragma unroll
        for (int k = 0; k < 24; k++) v[k] *= hc;
      }
      if (p.norm_pre) {
        C n = 0;
#pragma unroll
        for (int k = 0; k < 24; k++) n += v[k] * v[k];
        part = (double)n;
      }
      if (has_fin) {
#pragma unroll
        for (int k = 0; k < 24; k++) row[k] = v[k];
      } else {
        const double pr = epi_output<P>(p, x, col, r, v);
        if (p.axpy_r) part = pr;
      }
    }
    if (p.norm_pre || (p.axpy_r && !has_fin)) redsm[i] = part;
  }
  if (has_fin) {
    __syncthreads();
    for (int it2 = tid; it2 < nitems; it2 += nt) {
      const int lowerh = it2 >= nhalf;
      const int j = lowerh ? it2 - nhalf : it2;
      const int g = j / 12, q = j - g * 12;
      const int comp = 8 * (q >> 2) + 4 * lowerh + (q & 3);
      if (site0 + (nrhs == 1 ? g : g / nrhs) >= p.x_end) continue;
      chain_apply_fast(p.fin, comp, tileH + g * GS + comp, TSTR, Ls, mf);
    }
    __syncthreads();
    for (int i = tid; i < nsites; i += nt) {
      const int site_l = div_small(i, inv_w), col = i - site_l * W;
      const int r = div_small(col, inv_ls), s = col - r * Ls, grp = site_l * nrhs + r;
      const long long x = site0 + site_l;
      double part = 0.0;
      if (x < p.x_end) {
        C v[24];
#pragma unroll
        for (int k = 0; k < 24; k++) v[k] = tileH[grp * GS + s * TSTR + k];
        part = epi_output<P>(p, x, col, r, v);
      }
      if (p.axpy_r) redsm[i] = part;
    }
  }
  if (p.red.mode != RED_NONE) block_grid_reduce_sm(p.red, redsm, Ls, ns);
}

// shared memory of the fused epilogue: tile(s) + reduction scratch
__host__ __device__ inline size_t epi_smem_bytes(size_t csz, int ns, int nrhs, int Ls, bool center, int threads) {
  const size_t tile = (size_t)ns * nrhs * tile_gstr(Ls) * csz;
  const size_t nsites = (size_t)ns * nrhs * Ls;
  const size_t red = ((nsites > (size_t)threads ? nsites : (size_t)threads) + (size_t)ns * nrhs) * sizeof(double);
  (void)center;   // the centre is read per site from global memory, not staged
  return ((tile + 15) & ~(size_t)15) + red + 16;
}

}  // namespace mdwf
