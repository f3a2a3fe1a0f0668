// Shared epilogue of the fused hop kernels.  On entry tileH holds the hop result of every
// 5D site of the CTA's ns 4D sites, laid out [grp = site_l * nrhs + r][s][24 reals]
// (strides tile_gstr(Ls) and TSTR);
// the epilogue computes   out = fin( cc * cop(center) + hc * post(hop) )
// (post/cop/fin: s-direction chains of D5, A5, A5^-1 and adjoints), optionally reduces
// |out|^2 before fin, and either stores out or does r -= alpha out with |r|^2.
#pragma once
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"

namespace mdwf {

template <int P>
__device__ __forceinline__ void hop_epilogue(const HopParams& p, typename PT<P>::C* tileH,
                                             typename PT<P>::C* tileC, double* redsm, int ns) {
  using C = typename PT<P>::C;
  const int Ls = p.in.Ls, nrhs = p.in.nrhs, W = Ls * nrhs;
  const int GS = tile_gstr(Ls);
  const int tid = threadIdx.x, nt = blockDim.x;
  const long long site0 = (long long)blockIdx.x * ns;
  const int nsites = ns * W;
  const C mf = (C)p.mf;
  if (p.has_center) {
    for (int i = tid; i < nsites; i += nt) {
      const int site_l = i / W, col = i - site_l * W;
      if (site0 + site_l >= p.g.vh) continue;
      const int r = col / Ls, s = col - r * Ls, grp = site_l * nrhs + r;
      C v[24];
      load_site<P>(p.center, site0 + site_l, col, v);
#pragma unroll
      for (int k = 0; k < 24; k++) tileC[grp * GS + s * TSTR + k] = v[k];
    }
    __syncthreads();
  }
  const int nitems = ns * nrhs * 24;
  const C hc = (C)p.hc, cc = (C)p.cc;
  // items chirality-major (all upper-spin columns, then all lower-spin ones): the two
  // chiralities walk s in opposite directions, so a warp stays on one code path
  const int nhalf = ns * nrhs * 12;
  for (int it2 = tid; it2 < nitems; it2 += nt) {
    const int lowerh = it2 >= nhalf;
    const int j = lowerh ? it2 - nhalf : it2;
    const int g = j / 12, q = j - g * 12;                         // q: colour (q / 4), spin pair, re/im
    const int comp = 8 * (q >> 2) + 4 * lowerh + (q & 3);
    if (site0 + (nrhs == 1 ? g : g / nrhs) >= p.g.vh) continue;
    C* h = tileH + g * GS + comp;
    if (p.post.op[0].kind != SOP_NONE) chain_apply_fast(p.post, comp, h, TSTR, Ls, mf);
    if (p.has_center) {
      C* cv = tileC + g * GS + comp;
      if (p.cop.op[0].kind != SOP_NONE) chain_apply_fast(p.cop, comp, cv, TSTR, Ls, mf);
      for (int ss = 0; ss < Ls; ss++) h[ss * TSTR] = cc * cv[ss * TSTR] + hc * h[ss * TSTR];
    } else if (p.hc != 1.0) {
      for (int ss = 0; ss < Ls; ss++) h[ss * TSTR] = hc * h[ss * TSTR];
    }
  }
  __syncthreads();
  if (p.norm_pre) {
    for (int i = tid; i < nsites; i += nt) {
      const int site_l = i / W, col = i - site_l * W;
      const int r = col / Ls, s = col - r * Ls, grp = site_l * nrhs + r;
      C n = 0;
      if (site0 + site_l < p.g.vh) {
#pragma unroll
        for (int k = 0; k < 24; k++) { C v = tileH[grp * GS + s * TSTR + k]; n += v * v; }
      }
      redsm[i] = (double)n;
    }
  }
  if (p.fin.op[0].kind != SOP_NONE) {
    __syncthreads();
    for (int it2 = tid; it2 < nitems; it2 += nt) {
      const int lowerh = it2 >= nhalf;
      const int j = lowerh ? it2 - nhalf : it2;
      const int g = j / 12, q = j - g * 12;
      const int comp = 8 * (q >> 2) + 4 * lowerh + (q & 3);
      if (site0 + (nrhs == 1 ? g : g / nrhs) >= p.g.vh) continue;
      chain_apply_fast(p.fin, comp, tileH + g * GS + comp, TSTR, Ls, mf);
    }
    __syncthreads();
  }
  for (int i = tid; i < nsites; i += nt) {
    const int site_l = i / W, col = i - site_l * W;
    const int r = col / Ls, s = col - r * Ls, grp = site_l * nrhs + r;
    const long long x = site0 + site_l;
    double part = 0.0;
    if (x < p.g.vh) {
      C v[24];
#pragma unroll
      for (int k = 0; k < 24; k++) v[k] = tileH[grp * GS + s * TSTR + k];
      if (p.axpy_r) {
        C rv[24];
        load_site<P>(p.raxpy, x, col, rv);
        const C a = (C)p.red.cg[r].alpha;
        C n = 0;
#pragma unroll
        for (int k = 0; k < 24; k++) { rv[k] -= a * v[k]; n += rv[k] * rv[k]; }
        store_site<P>(p.raxpy, x, col, rv);
        part = (double)n;
      } else {
        store_site<P>(p.out, x, col, v);
      }
    }
    if (p.axpy_r) redsm[i] = part;
  }
  if (p.red.mode != RED_NONE) block_grid_reduce_sm(p.red, redsm, Ls, ns);
}

// shared memory of the fused epilogue: tile(s) + reduction scratch
__host__ __device__ inline size_t epi_smem_bytes(size_t csz, int ns, int nrhs, int Ls, bool center, int threads) {
  const size_t tile = (size_t)ns * nrhs * tile_gstr(Ls) * csz;
  const size_t nsites = (size_t)ns * nrhs * Ls;
  const size_t red = ((nsites > (size_t)threads ? nsites : (size_t)threads) + (size_t)ns * nrhs) * sizeof(double);
  return ((tile * (center ? 2 : 1) + 15) & ~(size_t)15) + red + 16;
}

}  // namespace mdwf
