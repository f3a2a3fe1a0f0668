// Tensor-core Wilson hop for half-precision storage (F16 + per-site norm, BF16), fused
// with the s-direction epilogue of mdwf_epi.cuh (Sec. "Current State of the Art": a
// radius-one stencil with small dense diagonal blocks).  sm_103a warp-level
// mma.sync.m16n8k16 with FP32 accumulation carries the SU(3) products.
//
// Phase 1 (one thread per 5D site of the CTA): for each of the 8 directions the
// neighbour column is loaded once (3 x 16 bytes = 4 spins of each colour), projected with
// (1 - sig gamma_mu) in 16-bit pairs -- upper spins h = psi_u - sig X_mu psi_d, lower spins
// -sig X_mu^+ h -- and scaled by norm_d / ref, ref = the largest of the 8 neighbour norms
// of that column, so that all 8 directions can share one accumulator.  The four spin rows
// [re,im of 3 colours, 0, 0] (16 bytes each) go to shared memory in ldmatrix row order.
// Phase 2 (warps): a task is 4 columns x 4 spins = 16 rows of one site; for each
// forward/backward pair of directions one ldmatrix.x4 gives the A fragment
// (K = 2 directions x 8) and one mma adds U_mu(x) and U_mu(x-mu)^+ (B, built once per
// site as real 6x6 blocks, K = input colour re/im, N = output colour re/im).  The FP32
// result times ref is the hop of those 5D sites; the shared epilogue takes it from there.
// Products of 16-bit inputs are exact in FP32 and sums are FP32; the extra rounding over
// an FP32 evaluation is that of the 16-bit projection and of the norm ratio.
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

template <int P>
__device__ __forceinline__ void mma16n8k16(float d[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  if constexpr (P == F16) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void* smem_row) {
  const unsigned addr = (unsigned)__cvta_generic_to_shared(smem_row);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(addr));
}

// x -> i x on an f16x2 / bf16x2 complex (re low, im high): (-im, re)
__device__ __forceinline__ uint32_t times_i(uint32_t v) { return swap_halves(v) ^ 0x00008000u; }
__device__ __forceinline__ uint32_t neg2(uint32_t v) { return v ^ 0x80008000u; }

// Phase-1 work of one direction for one 5D site: project (1 - sig gamma_mu) psi of the
// neighbour column in 16-bit pairs, scale by ratio = norm_d / ref and write the four spin
// rows [colour re,im x 3, 0, 0] of 16 bytes each.
template <int P, int MU, int SIG>
__device__ __forceinline__ void stage_dir(const uint4 q[3], uint32_t ratio, uint4* rows) {
  using H2 = typename TC<P>::H2;
  // per-colour constants of h_j = psi_j + sig*kappa_j psi_partner
  const uint32_t one_pm = TC<P>::h2((float)SIG, (float)-SIG);   // (sig, -sig)
  const uint32_t mp_pm = TC<P>::h2((float)-SIG, (float)SIG);    // (-sig, sig)
  const uint32_t s_neg = TC<P>::h2((float)-SIG, (float)-SIG);   // (-sig, -sig)
  const uint32_t s_pos = TC<P>::h2((float)SIG, (float)SIG);     // (sig, sig)
  uint32_t v[4][3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const uint32_t w0 = (&q[c].x)[0], w1 = (&q[c].x)[1], w2 = (&q[c].x)[2], w3 = (&q[c].x)[3];
    uint32_t h0, h1;
    if (MU == 0) {        // h0 = w0 - sig i w3 ; h1 = w1 - sig i w2
      h0 = hfma2u<H2>(swap_halves(w3), one_pm, w0);
      h1 = hfma2u<H2>(swap_halves(w2), one_pm, w1);
    } else if (MU == 1) { // h0 = w0 - sig w3 ; h1 = w1 + sig w2
      h0 = hfma2u<H2>(w3, s_neg, w0);
      h1 = hfma2u<H2>(w2, s_pos, w1);
    } else if (MU == 2) { // h0 = w0 - sig i w2 ; h1 = w1 + sig i w3
      h0 = hfma2u<H2>(swap_halves(w2), one_pm, w0);
      h1 = hfma2u<H2>(swap_halves(w3), mp_pm, w1);
    } else {              // h0 = w0 - sig w2 ; h1 = w1 - sig w3
      h0 = hfma2u<H2>(w2, s_neg, w0);
      h1 = hfma2u<H2>(w3, s_neg, w1);
    }
    if (P == F16) {
      H2 a = __hmul2(*(const H2*)&h0, *(const H2*)&ratio);
      H2 b = __hmul2(*(const H2*)&h1, *(const H2*)&ratio);
      h0 = *(uint32_t*)&a;
      h1 = *(uint32_t*)&b;
    }
    // lower spins = -sig X_mu^+ h
    uint32_t l0, l1;
    if (MU == 0) {        // l0 = sig i h1 ; l1 = sig i h0
      l0 = times_i(h1); l1 = times_i(h0);
      if (SIG < 0) { l0 = neg2(l0); l1 = neg2(l1); }
    } else if (MU == 1) { // l0 = sig h1 ; l1 = -sig h0
      l0 = SIG > 0 ? h1 : neg2(h1); l1 = SIG > 0 ? neg2(h0) : h0;
    } else if (MU == 2) { // l0 = sig i h0 ; l1 = -sig i h1
      l0 = times_i(h0); l1 = times_i(h1);
      if (SIG > 0) l1 = neg2(l1); else l0 = neg2(l0);
    } else {              // l0 = -sig h0 ; l1 = -sig h1
      l0 = SIG > 0 ? neg2(h0) : h0; l1 = SIG > 0 ? neg2(h1) : h1;
    }
    v[0][c] = h0; v[1][c] = h1; v[2][c] = l0; v[3][c] = l1;
  }
#pragma unroll
  for (int k = 0; k < 4; k++) rows[k] = make_uint4(v[k][0], v[k][1], v[k][2], 0u);
}

// Shared memory carve of the mma hop: A rows, per-column scale, neighbour table, epilogue.
struct MmaSmem {
  size_t a_off, ref_off, nbr_off, tile_off, red_off, total;
};
__host__ __device__ inline MmaSmem mma_smem(int ns, int nrhs, int Ls, bool center, int threads) {
  MmaSmem m;
  const size_t W = (size_t)nrhs * Ls;
  m.a_off = 0;
  m.ref_off = m.a_off + (size_t)ns * 8 * W * 4 * 16;
  m.nbr_off = m.ref_off + ((ns * W * 4 + 15) & ~(size_t)15);
  m.tile_off = m.nbr_off + ((size_t)ns * 8 * 4 + 15) / 16 * 16;
  const size_t tile = (size_t)ns * nrhs * tile_gstr(Ls) * 4;
  (void)center;
  m.red_off = m.tile_off + ((tile + 15) & ~(size_t)15);
  const size_t nsites = (size_t)ns * W;
  m.total = m.red_off + ((nsites > (size_t)threads ? nsites : (size_t)threads) + (size_t)ns * nrhs) * 8 + 16;
  return m;
}

template <int P, bool DAG>
__global__ void __launch_bounds__(256) hop_mma_kernel(const __grid_constant__ HopParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Ls = p.in.Ls, nrhs = p.in.nrhs, W = Ls * nrhs, GS = tile_gstr(Ls);
  const int ns = p.ns, nt = blockDim.x, tid = threadIdx.x;
  const long long site0 = (long long)blockIdx.x * ns;
  const MmaSmem L = mma_smem(ns, nrhs, Ls, p.has_center, nt);
  uint4* Abuf = (uint4*)(smem_raw + L.a_off);
  float* ref = (float*)(smem_raw + L.ref_off);
  int* nbrs = (int*)(smem_raw + L.nbr_off);
  float* tileH = (float*)(smem_raw + L.tile_off);
  double* redsm = (double*)(smem_raw + L.red_off);

  // phase 0: neighbour table of the CTA's sites
  for (int i = tid; i < ns * 8; i += nt) {
    const long long x = site0 + i / 8;
    if (x >= p.g.vh) continue;
    int c[4];
    cb_coords(p.g, x, p.pout, c);
    const int d = i & 7;
    nbrs[i] = (int)nbr_cb(p.g, c, d & 3, d < 4 ? +1 : -1);
  }
  __syncthreads();

  // phase 1: one thread per 5D site stages the 8 directions' projected rows
  const uint4* chunks = (const uint4*)p.in.data;
  for (int i = tid; i < ns * W; i += nt) {
    const int site_l = i / W, col = i - site_l * W;
    if (site0 + site_l >= p.g.vh) continue;
    const int* nb = nbrs + site_l * 8;
    float nv[8];
    float mx = 0.f;
#pragma unroll
    for (int d = 0; d < 8; d++) {
      nv[d] = (P == F16) ? __ldg(p.in.norm + (long long)nb[d] * W + col) : 1.f;
      mx = fmaxf(mx, nv[d]);
    }
    ref[i] = mx;
    const float inv = mx > 0.f ? 1.f / mx : 0.f;
    uint4* rows = Abuf + ((size_t)site_l * 8 * W + col) * 4;
#define STAGE(D, MU, SIG)                                                                 \
    {                                                                                     \
      const uint4* pc = chunks + (long long)nb[D] * 3 * W + col;                          \
      uint4 q[3] = {__ldg(pc), __ldg(pc + W), __ldg(pc + 2 * W)};                         \
      const uint32_t ratio = TC<P>::h2(nv[D] * inv, nv[D] * inv);                         \
      stage_dir<P, MU, SIG>(q, ratio, rows + (size_t)(D) * W * 4);                        \
    }
    constexpr int SF = DAG ? -1 : 1;
    STAGE(0, 0, SF) STAGE(1, 1, SF) STAGE(2, 2, SF) STAGE(3, 3, SF)
    STAGE(4, 0, -SF) STAGE(5, 1, -SF) STAGE(6, 2, -SF) STAGE(7, 3, -SF)
#undef STAGE
  }
  __syncthreads();

  // phase 2: a warp takes whole sites; per 4-column tile: 16 rows = 4 columns x 4 spins,
  // K = 2 directions (forward/backward of one mu) per mma
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int ntile = (W + 3) >> 2;
  const int m = lane >> 3, rr = lane & 7;            // ldmatrix: matrix m, row rr
  const int rho = (m & 1) * 8 + rr;                  // row within the tile
  for (int site_l = warp; site_l < ns; site_l += nwarps) {
    const long long x = site0 + site_l;
    if (x >= p.g.vh) continue;
    // B: lane (g, t) holds (k = 2t, 2t+1 ; n = g) of U_d as a real 6x6 block:
    // output re: (Re U[c][t], -Im U[c][t]), output im: (Im U[c][t], Re U[c][t]), c = g/2
    uint32_t bfr[8];
    {
      const uint32_t* gl = (const uint32_t*)((const __half*)p.gauge + x * 8 * p.gs);
#pragma unroll
      for (int d = 0; d < 8; d++) {
        uint32_t u = 0;
        if (g < 6 && t < 3) u = __ldg(gl + (d * p.gs) / 2 + (g >> 1) * 3 + t);
        bfr[d] = (g < 6 && t < 3) ? ((g & 1) ? swap_halves(u) : (u ^ 0x80000000u)) : 0u;
      }
    }
    const uint4* abase_site = Abuf + (size_t)site_l * 8 * W * 4;
    const float* ref_site = ref + site_l * W;
    // output rows of this lane: column 2*rw + g/4 of the tile, spin g%4; track (rhs, s)
    int oc[2] = {g >> 2, 2 + (g >> 2)};
    int orr[2], os[2];
#pragma unroll
    for (int rw = 0; rw < 2; rw++) { orr[rw] = oc[rw] / Ls; os[rw] = oc[rw] - orr[rw] * Ls; }
    const int spin = g & 3;
    for (int tile = 0; tile < ntile; tile++) {
      int colr = tile * 4 + (rho >> 2);
      colr = colr < W ? colr : W - 1;   // rows past the last column read a valid row; unused
      const uint4* abase = abase_site + (size_t)colr * 4 + (rho & 3);
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int ks = 0; ks < 4; ks++) {
        const int dsel = (m >> 1) ? ks + 4 : ks;
        uint32_t a[4];
        ldsm_x4(a, abase + (size_t)dsel * W * 4);
        mma16n8k16<P>(acc, a, bfr[ks], bfr[ks + 4]);
      }
#pragma unroll
      for (int rw = 0; rw < 2; rw++) {
        const int col = tile * 4 + oc[rw];
        if (col < W && t < 3) {
          const float sc = ref_site[col];
          float* th = tileH + (site_l * nrhs + orr[rw]) * GS + os[rw] * TSTR + 2 * (t * 4 + spin);
          th[0] = acc[2 * rw] * sc;
          th[1] = acc[2 * rw + 1] * sc;
        }
        os[rw] += 4;
        while (os[rw] >= Ls) { os[rw] -= Ls; orr[rw]++; }
      }
    }
  }
  __syncthreads();
  hop_epilogue<P>(p, tileH, redsm, ns);
}

bool hop_tc_supported(int prec, const HopParams& p, bool r12) {
  if (r12 || (prec != F16 && prec != BF16)) return false;
  if (p.gs != 24) return false;
  if (p.g.vh * 3 * (long long)p.in.nrhs * p.in.Ls >= (1LL << 31)) return false;
  return true;
}

static int tc_threads(const HopParams& p) {
  const int W = p.in.nrhs * p.in.Ls;
  int t = ((p.ns * W + 31) / 32) * 32;
  return t < 64 ? 64 : (t > 256 ? 256 : t);
}

size_t hop_tc_smem_bytes(const HopParams& p) {
  return mma_smem(p.ns, p.in.nrhs, p.in.Ls, p.has_center, tc_threads(p)).total;
}

template <int P, bool DAG>
static cudaError_t go_tc(const HopParams& p, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(hop_mma_kernel<P, DAG>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int threads = tc_threads(p);
  const size_t smem = hop_tc_smem_bytes(p);
  const long long blocks = (p.g.vh + p.ns - 1) / p.ns;
  HopParams q = p;   // scalars rounded once for the 32-bit kernels
  q.hcf = (float)p.hc; q.ccf = (float)p.cc; q.mff = (float)p.mf;
  hop_mma_kernel<P, DAG><<<(unsigned)blocks, threads, smem, st>>>(q);
  return cudaGetLastError();
}

cudaError_t launch_hop_tc(int prec, bool dag, bool /*epi*/, const HopParams& p, cudaStream_t st) {
  if (prec == F16) return dag ? go_tc<F16, true>(p, st) : go_tc<F16, false>(p, st);
  if (prec == BF16) return dag ? go_tc<BF16, true>(p, st) : go_tc<BF16, false>(p, st);
  return cudaErrorNotSupported;
}

}  // namespace mdwf
