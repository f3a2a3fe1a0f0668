// s-local kernels: the fifth-dimension operators D5 = b5 + c5 B, A5 = alpha + beta B and
// A5^-1 on whole 5D columns (Sec. "Current State of the Art": the small dense diagonal
// blocks of the domain-wall matrix), and the BLAS-1 steps of CG with FP64-accumulated,
// fixed-order reductions (Sec. "Performance Measurement Method": all reductions in
// double precision).
//
// Thread layout as in the hop kernels: a CTA owns ns 4D sites, thread (site_l, r, s).
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"
#include "mdwf_epi.cuh"

namespace mdwf {

// out = ca * chain(b) [+ cb * c]
template <int P>
__global__ void __launch_bounds__(MAXTHREADS) chain_kernel(const __grid_constant__ SLParams p) {
  using C = typename PT<P>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.b.Ls, nrhs = p.b.nrhs, W = Ls * nrhs, LsP = Ls + 1;
  const int tid = threadIdx.x, site_l = tid / W, col = tid - site_l * W;
  const long long x_cb = (long long)blockIdx.x * p.ns + site_l;
  const bool active = x_cb < p.vh;
  const int r = col / Ls, s = col - r * Ls, grp = site_l * nrhs + r;
  C* tile = (C*)smem_raw;
  if (active) {
    C v[24];
    load_site<P>(p.b, x_cb, col, v);
#pragma unroll
    for (int k = 0; k < 24; k++) tile[(grp * 24 + k) * LsP + s] = v[k];
  }
  __syncthreads();
  const int nitems = p.ns * nrhs * 24;
  for (int it = tid; it < nitems; it += blockDim.x) {
    if ((long long)blockIdx.x * p.ns + (it / 24) / nrhs >= p.vh) continue;
    chain_apply_fast(p.chain, it % 24, tile + it * LsP, 1, Ls, pick<C>(p.mff, p.mf));
  }
  __syncthreads();
  if (active) {
    C v[24];
    const C ca = pick<C>(p.caf, p.ca);
#pragma unroll
    for (int k = 0; k < 24; k++) v[k] = ca * tile[(grp * 24 + k) * LsP + s];
    if (p.c.data) {
      C w[24];
      load_site<P>(p.c, x_cb, col, w);
      const C cb = pick<C>(p.cbf, p.cb);
#pragma unroll
      for (int k = 0; k < 24; k++) v[k] += cb * w[k];
    }
    store_site<P>(p.a, x_cb, col, v);
  }
}

// a = ca * b + cb * c ; optional |a|^2
template <int P>
__global__ void __launch_bounds__(MAXTHREADS) axpby_kernel(const __grid_constant__ SLParams p) {
  using C = typename PT<P>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.b.Ls, nrhs = p.b.nrhs, W = Ls * nrhs;
  const int tid = threadIdx.x, site_l = tid / W, col = tid - site_l * W;
  const long long x_cb = (long long)blockIdx.x * p.ns + site_l;
  double part = 0.0;
  if (x_cb < p.vh) {
    C v[24];
    load_site<P>(p.b, x_cb, col, v);
    const C ca = pick<C>(p.caf, p.ca);
#pragma unroll
    for (int k = 0; k < 24; k++) v[k] *= ca;
    if (p.c.data) {
      C w[24];
      load_site<P>(p.c, x_cb, col, w);
      const C cb = pick<C>(p.cbf, p.cb);
#pragma unroll
      for (int k = 0; k < 24; k++) v[k] += cb * w[k];
    }
    if (p.red.mode != RED_NONE) {
      C n = 0;
#pragma unroll
      for (int k = 0; k < 24; k++) n += v[k] * v[k];
      part = (double)n;
    }
    if (p.a.data) store_site<P>(p.a, x_cb, col, v);
  }
  if (p.red.mode != RED_NONE) block_grid_reduce(p.red, part, (double*)smem_raw, Ls, p.ns);
}

// CG step: x += alpha p ; p = r + beta p ; phat = chain(p).   a = p, b = r, c = phat.
// A chain of one bidiagonal op (the left form's phat = D5 p) is applied per site from the
// new p of the slices s +- 1 (one 16-byte-row tile, one barrier); other chains run as
// column passes over the tile.
template <int PX, int P>
__global__ void __launch_bounds__(MAXTHREADS) cg_update_kernel(const __grid_constant__ SLParams p) {
  using C = typename PT<P>::C;
  using CX = typename PT<PX>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.a.Ls, nrhs = p.a.nrhs, W = Ls * nrhs, LsP = Ls + 1;
  const int tid = threadIdx.x, site_l = tid / W, col = tid - site_l * W;
  const long long x_cb = (long long)blockIdx.x * p.ns + site_l;
  const bool active = x_cb < p.vh;
  const int r = col / Ls, s = col - r * Ls, grp = site_l * nrhs + r;
  C* tile = (C*)smem_raw;
  if constexpr (sizeof(C) == 4) {
    const SOp& o = p.chain.op[0];
    if (p.c.data != nullptr && o.kind == SOP_BIDIAG && p.chain.op[1].kind == SOP_NONE) {
      // tile rows [grp][s][TSTR]: the new p of every 5D site of the CTA
      C pv[24];
      if (active) {
        const double alpha = p.red.cg[r].alpha;
        C rv[24];
        load_site<P>(p.a, x_cb, col, pv);
        if (pick<CX>(p.red.cg[r].alpha_f, alpha) != (CX)0) {
          CX xv[24];
          load_site<PX>(p.x, x_cb, col, xv);
          const CX ax = pick<CX>(p.red.cg[r].alpha_f, alpha);
#pragma unroll
          for (int k = 0; k < 24; k++) xv[k] += ax * (CX)pv[k];
          store_site<PX>(p.x, x_cb, col, xv);
        }
        load_site<P>(p.b, x_cb, col, rv);
        const C bt = pick<C>(p.red.cg[r].beta_f, p.red.cg[r].beta);
#pragma unroll
        for (int k = 0; k < 24; k++) pv[k] = rv[k] + bt * pv[k];
        store_site<P>(p.a, x_cb, col, pv);
        C* row = tile + (grp * Ls + s) * TSTR;
#pragma unroll
        for (int k = 0; k < 24; k += 4) *(float4*)(row + k) = make_float4(pv[k], pv[k + 1], pv[k + 2], pv[k + 3]);
      }
      __syncthreads();
      if (active) {
        // upper spins (0, 1) of each colour from slice su, lower ones (2, 3) from sl
        const SNbr<C> n = s_nbr<C>(o, s, Ls, pick<C>(p.mff, p.mf));
        const C a = sop_a<C>(o);
        const C* ru = tile + (grp * Ls + n.su) * TSTR;
        const C* rl = tile + (grp * Ls + n.sl) * TSTR;
        C v[24];
#pragma unroll
        for (int c = 0; c < 3; c++) {
          const float4 u = *(const float4*)(ru + 8 * c);
          const float4 l = *(const float4*)(rl + 8 * c + 4);
          v[8 * c + 0] = a * pv[8 * c + 0] + n.fu * u.x;
          v[8 * c + 1] = a * pv[8 * c + 1] + n.fu * u.y;
          v[8 * c + 2] = a * pv[8 * c + 2] + n.fu * u.z;
          v[8 * c + 3] = a * pv[8 * c + 3] + n.fu * u.w;
          v[8 * c + 4] = a * pv[8 * c + 4] + n.fl * l.x;
          v[8 * c + 5] = a * pv[8 * c + 5] + n.fl * l.y;
          v[8 * c + 6] = a * pv[8 * c + 6] + n.fl * l.z;
          v[8 * c + 7] = a * pv[8 * c + 7] + n.fl * l.w;
        }
        store_site<P>(p.c, x_cb, col, v);
      }
      return;
    }
  }
  if (active) {
    const double alpha = p.red.cg[r].alpha;
    C pv[24], rv[24];
    load_site<P>(p.a, x_cb, col, pv);
    if (pick<CX>(p.red.cg[r].alpha_f, alpha) != (CX)0) {
      CX xv[24];
      load_site<PX>(p.x, x_cb, col, xv);
      const CX ax = pick<CX>(p.red.cg[r].alpha_f, alpha);
#pragma unroll
      for (int k = 0; k < 24; k++) xv[k] += ax * (CX)pv[k];
      store_site<PX>(p.x, x_cb, col, xv);
    }
    load_site<P>(p.b, x_cb, col, rv);
    const C bt = pick<C>(p.red.cg[r].beta_f, p.red.cg[r].beta);
#pragma unroll
    for (int k = 0; k < 24; k++) { pv[k] = rv[k] + bt * pv[k]; tile[(grp * 24 + k) * LsP + s] = pv[k]; }
    store_site<P>(p.a, x_cb, col, pv);
  }
  if (p.c.data == nullptr) return;   // no phat wanted (the form applies no pre-chain to p)
  __syncthreads();
  const int nitems = p.ns * nrhs * 24;
  for (int it = tid; it < nitems; it += blockDim.x) {
    if ((long long)blockIdx.x * p.ns + (it / 24) / nrhs >= p.vh) continue;
    chain_apply_fast(p.chain, it % 24, tile + it * LsP, 1, Ls, pick<C>(p.mff, p.mf));
  }
  __syncthreads();
  if (active) {
    C v[24];
#pragma unroll
    for (int k = 0; k < 24; k++) v[k] = tile[(grp * 24 + k) * LsP + s];
    store_site<P>(p.c, x_cb, col, v);
  }
}

// a(PO) = [a +] b(PI); optionally b = 0
template <int PO, int PI>
__global__ void __launch_bounds__(MAXTHREADS) convert_kernel(const __grid_constant__ SLParams p) {
  using CO = typename PT<PO>::C;
  using CI = typename PT<PI>::C;
  const int Ls = p.b.Ls, nrhs = p.b.nrhs, W = Ls * nrhs;
  const int tid = threadIdx.x, site_l = tid / W, col = tid - site_l * W;
  const long long x_cb = (long long)blockIdx.x * p.ns + site_l;
  if (x_cb >= p.vh) return;
  CI v[24];
  load_site<PI>(p.b, x_cb, col, v);
  CO o[24];
  if (p.ca != 0.0) {
    load_site<PO>(p.a, x_cb, col, o);
#pragma unroll
    for (int k = 0; k < 24; k++) o[k] += (CO)v[k];
  } else {
#pragma unroll
    for (int k = 0; k < 24; k++) o[k] = (CO)v[k];
  }
  store_site<PO>(p.a, x_cb, col, o);
  if (p.cb != 0.0) {
    CI z[24];
#pragma unroll
    for (int k = 0; k < 24; k++) z[k] = 0;
    store_site<PI>(p.b, x_cb, col, z);
  }
}

// Re <b, c> per right-hand side (FP64 accumulated)
template <int P>
__global__ void __launch_bounds__(MAXTHREADS) dot_kernel(const __grid_constant__ SLParams p) {
  using C = typename PT<P>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.b.Ls, nrhs = p.b.nrhs, W = Ls * nrhs;
  const int tid = threadIdx.x, site_l = tid / W, col = tid - site_l * W;
  const long long x_cb = (long long)blockIdx.x * p.ns + site_l;
  double part = 0.0;
  if (x_cb < p.vh) {
    C u[24], v[24];
    load_site<P>(p.b, x_cb, col, u);
    load_site<P>(p.c, x_cb, col, v);
    C n = 0;
#pragma unroll
    for (int k = 0; k < 24; k++) n += u[k] * v[k];
    part = (double)n;
  }
  block_grid_reduce(p.red, part, (double*)smem_raw, Ls, p.ns);
}

// a[rhs] += coef[rhs] * b[rhs], coef read from device memory (p.red.out)
template <int P>
__global__ void __launch_bounds__(MAXTHREADS) rhs_axpy_kernel(const __grid_constant__ SLParams p) {
  using C = typename PT<P>::C;
  const int Ls = p.b.Ls, nrhs = p.b.nrhs, W = Ls * nrhs;
  const int tid = threadIdx.x, site_l = tid / W, col = tid - site_l * W;
  const long long x_cb = (long long)blockIdx.x * p.ns + site_l;
  if (x_cb >= p.vh) return;
  const C cf = (C)p.red.out[col / Ls];
  C u[24], v[24];
  load_site<P>(p.a, x_cb, col, u);
  load_site<P>(p.b, x_cb, col, v);
#pragma unroll
  for (int k = 0; k < 24; k++) u[k] += cf * v[k];
  store_site<P>(p.a, x_cb, col, u);
}

template <typename K>
static cudaError_t go(K kern, const SLParams& p, int W, size_t smem, cudaStream_t st) {
  static_assert(sizeof(SLParams) < 4000, "param size");
  const long long blocks = (p.vh + p.ns - 1) / p.ns;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  SLParams q = p;   // scalars rounded once for the 32-bit kernels
  q.caf = (float)p.ca; q.cbf = (float)p.cb; q.mff = (float)p.mf;
  kern<<<(unsigned)blocks, p.ns * W, smem, st>>>(q);
  return cudaGetLastError();
}

static size_t tile_bytes(int prec, const Field& f, int ns) {
  // column tile [grp][24][Ls + 1], or (cg_update, one bidiagonal op) 16-byte rows [grp][s][TSTR]
  const size_t col = (size_t)ns * f.nrhs * 24 * (f.Ls + 1) * (prec == F64 ? 8 : 4);
  const size_t rows = (size_t)ns * f.nrhs * f.Ls * TSTR * 4;
  return col > rows ? col : rows;
}

cudaError_t launch_chain(int prec, const SLParams& p, cudaStream_t st) {
  const int W = p.b.nrhs * p.b.Ls;
  const size_t smem = tile_bytes(prec, p.b, p.ns);
  switch (prec) {
    case F64: return go(chain_kernel<F64>, p, W, smem, st);
    case F32: return go(chain_kernel<F32>, p, W, smem, st);
    case F16: return go(chain_kernel<F16>, p, W, smem, st);
    case BF16: return go(chain_kernel<BF16>, p, W, smem, st);
    case I16: return go(chain_kernel<I16>, p, W, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_axpby(int prec, const SLParams& p, cudaStream_t st) {
  const int W = p.b.nrhs * p.b.Ls;
  const size_t smem = 2 * (size_t)p.ns * W * sizeof(double) + 16;
  switch (prec) {
    case F64: return go(axpby_kernel<F64>, p, W, smem, st);
    case F32: return go(axpby_kernel<F32>, p, W, smem, st);
    case F16: return go(axpby_kernel<F16>, p, W, smem, st);
    case BF16: return go(axpby_kernel<BF16>, p, W, smem, st);
    case I16: return go(axpby_kernel<I16>, p, W, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_cg_update(int prec_x, int prec, const SLParams& p, cudaStream_t st) {
  const int W = p.a.nrhs * p.a.Ls;
  const size_t smem = tile_bytes(prec, p.a, p.ns);
  if (prec == F64 && prec_x == F64) return go(cg_update_kernel<F64, F64>, p, W, smem, st);
  if (prec_x == F32) {
    switch (prec) {
      case F32: return go(cg_update_kernel<F32, F32>, p, W, smem, st);
      case F16: return go(cg_update_kernel<F32, F16>, p, W, smem, st);
      case BF16: return go(cg_update_kernel<F32, BF16>, p, W, smem, st);
      case I16: return go(cg_update_kernel<F32, I16>, p, W, smem, st);
    }
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_dot(int prec, const SLParams& p, cudaStream_t st) {
  const int W = p.b.nrhs * p.b.Ls;
  const size_t smem = 2 * (size_t)p.ns * W * sizeof(double) + 16;
  switch (prec) {
    case F64: return go(dot_kernel<F64>, p, W, smem, st);
    case F32: return go(dot_kernel<F32>, p, W, smem, st);
    case F16: return go(dot_kernel<F16>, p, W, smem, st);
    case BF16: return go(dot_kernel<BF16>, p, W, smem, st);
    case I16: return go(dot_kernel<I16>, p, W, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_rhs_axpy(int prec, const SLParams& p, cudaStream_t st) {
  const int W = p.b.nrhs * p.b.Ls;
  switch (prec) {
    case F64: return go(rhs_axpy_kernel<F64>, p, W, 0, st);
    case F32: return go(rhs_axpy_kernel<F32>, p, W, 0, st);
    case F16: return go(rhs_axpy_kernel<F16>, p, W, 0, st);
    case BF16: return go(rhs_axpy_kernel<BF16>, p, W, 0, st);
    case I16: return go(rhs_axpy_kernel<I16>, p, W, 0, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_convert(int po, int pi, const SLParams& p, cudaStream_t st) {
  const int W = p.b.nrhs * p.b.Ls;
#define CV(A, B) if (po == A && pi == B) return go(convert_kernel<A, B>, p, W, 0, st);
  CV(F64, F64) CV(F64, F32) CV(F64, F16) CV(F64, BF16)
  CV(F32, F64) CV(F16, F64) CV(BF16, F64) CV(F32, F32) CV(F16, F32) CV(BF16, F32)
  CV(F64, I16) CV(I16, F64) CV(I16, F32)
#undef CV
  return cudaErrorInvalidValue;
}

}  // namespace mdwf
