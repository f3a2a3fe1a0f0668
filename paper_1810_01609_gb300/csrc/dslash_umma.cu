// Wilson hop on the 5th-generation tensor cores (tcgen05, sm_103a) for 16-bit storage
// (F16 + per-site norm, BF16), fused with the s-direction epilogue of mdwf_epi.cuh.
//
// The hop of one 4D site x is a dense contraction (Sec. "Current State of the Art": a
// radius-one stencil whose blocks are small dense matrices):
//
//   out[o][n] = sum_k  A_x[o][k] * H_x[k][n]
//
//   n = (rhs, s)            the nrhs * Ls columns of the site (all share its links)
//   k = (dir d, slot j, colour b, re/im)   K = 8 x 12 = 96: the projected half spinor
//        h_{d,j} = (psi_u -/+ X_mu psi_d)_j of the neighbour in direction d
//   o = (colour a, spin sigma, re/im)      24 output reals in the site order
//   A_x[o][k] = real form of R_d (1 (x) U_d): the SU(3) link times the reconstruction of
//        the lower spins, entries +-Re U, +-Im U, or 0
//
// One CTA owns S 4D sites.  CUDA cores build A_x (from the 8 links, in 16 bits) and H_x
// (neighbour chunks projected with packed 16-bit FMAs; F16 neighbours rescaled by
// norm_d / max_d norm_d of their column so that all 8 directions share one product) in
// shared memory in the no-swizzle K-major core-matrix layout; one thread issues
// 6 tcgen05.mma (M = 64 rows, N = nrhs*Ls padded to 16, K = 16 each) per site with FP32
// accumulation in tensor memory; warps 0 and 1 move the accumulators to the epilogue
// tile (times max_d norm_d for F16) and the shared epilogue applies the s-direction chains,
// centre term, norms and reductions.  Products of 16-bit inputs are exact in FP32; the
// rounding beyond an FP32 evaluation is that of the 16-bit projection and norm ratio.
//
// Shared-memory operand layout (both operands K-major, no swizzle): a core matrix is 8
// rows x 16 bytes (8 elements along K) stored as 128 contiguous bytes; the 12 core
// matrices along K of one 8-row group are 144 bytes apart (leading byte offset) and 8-row
// groups 12 x 144 + 16 = 1744 bytes apart (stride byte offset).  The 16-byte gaps skew the
// shared-memory banks of core matrices, so the 16-byte stores of a warp that all write the
// same row of different core matrices spread over the banks.  Site j's A rows are rows
// 24j .. 24j+23 of one shared row sequence: the MMA's M - 24 extra rows read whatever
// follows (the next sites' rows, other buffers) and produce accumulator rows nobody reads.
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"
#include "mdwf_epi.cuh"

namespace mdwf {

namespace {

constexpr int UM_THREADS = 128;
constexpr int UM_M = 64;                  // MMA rows: accumulator row 16w + i in TMEM lane 32w + i
constexpr int UM_KCH = 12;                // K = 96 = 12 core matrices of 8 elements
constexpr int UM_LBO = 144;               // bytes between core matrices along K
constexpr int UM_GRP = UM_KCH * UM_LBO + 16;   // bytes between 8-row groups
constexpr int UM_KSTEP = 2 * UM_LBO;      // one MMA's K = 16: two core matrices
constexpr int UM_WAIT_SPINS = 1 << 24;    // bounded mbarrier waits (about a second)

__host__ __device__ inline int um_npad(int W) { return (W + 15) & ~15; }

struct UmLayout {
  int bar, nbr, nmax, a, b, tile, total, npad, tcols;
};

__host__ __device__ inline int um_tcols(int n) {
  int c = 32;
  while (c < n) c <<= 1;
  return c;
}

__host__ __device__ inline UmLayout um_layout(int S, int nrhs, int Ls) {
  UmLayout L;
  const int W = nrhs * Ls;
  L.npad = um_npad(W);
  L.tcols = um_tcols(S * L.npad);
  L.bar = 0;                                   // mbarrier (8 B) + TMEM address (4 B)
  L.nbr = 16;                                  // S * 8 neighbour indices, then S * 8 flags
  L.nmax = L.nbr + ((S * 8 * 5 + 15) & ~15);   // S * npad column scales (F16)
  L.a = (L.nmax + S * L.npad * 4 + 127) & ~127;
  L.b = L.a + 3 * S * UM_GRP;
  L.tile = L.b + S * (L.npad / 8) * UM_GRP;
  const size_t epi = epi_smem_bytes(4, S, nrhs, Ls, false, UM_THREADS);
  int end = L.tile + (int)epi;
  const int a_end = L.a + (3 * (S - 1) + UM_M / 8) * UM_GRP;   // rows the last site's MMA reads
  L.total = end > a_end ? end : a_end;
  return L;
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, leading / stride byte offsets, fixed 0b001 at
// bits 46-48, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)(UM_LBO >> 4) << 16;
  d |= (uint64_t)(UM_GRP >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, A and B both F16 or both BF16,
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24
template <int P>
__host__ __device__ constexpr uint32_t um_idesc(int N) {
  return (1u << 4) | ((P == BF16 ? 1u : 0u) << 7) | ((P == BF16 ? 1u : 0u) << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(UM_M >> 4) << 24);
}

__device__ __forceinline__ void um_mma(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool um_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < UM_WAIT_SPINS; it++) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase));
    if (done) return true;
    if (it >= 8) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void um_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// ------------------------------------------------------------------ 16-bit pair helpers
template <int P> struct H2T;
template <> struct H2T<F16> { using T = __half2; };
template <> struct H2T<BF16> { using T = __nv_bfloat162; };

template <int P>
__device__ __forceinline__ uint32_t pk(float a, float b) {
  if constexpr (P == F16) { __half2 v = __floats2half2_rn(a, b); return *(uint32_t*)&v; }
  else { __nv_bfloat162 v = __floats2bfloat162_rn(a, b); return *(uint32_t*)&v; }
}
template <int P>
__device__ __forceinline__ float2 unpk(uint32_t u) {
  if constexpr (P == F16) return __half22float2(*(const __half2*)&u);
  else return __bfloat1622float2(*(const __nv_bfloat162*)&u);
}
template <int P>
__device__ __forceinline__ uint32_t hfma(uint32_t a, uint32_t b, uint32_t c) {
  using H = typename H2T<P>::T;
  H r = __hfma2(*(const H*)&a, *(const H*)&b, *(const H*)&c);
  return *(uint32_t*)&r;
}
template <int P>
__device__ __forceinline__ uint32_t hmul(uint32_t a, uint32_t b) {
  using H = typename H2T<P>::T;
  H r = __hmul2(*(const H*)&a, *(const H*)&b);
  return *(uint32_t*)&r;
}
__device__ __forceinline__ uint32_t swp(uint32_t v) { return __byte_perm(v, 0, 0x1032); }

// Row a of link (x, d) as three 16-bit (re, im) pairs; 12-real links rebuild row 2 as
// conj(row0 x row1), negated at the time boundary when the stored rows carry the phase.
template <int P, bool R12>
__device__ __forceinline__ void link_row(const void* gauge, long long off, int a, bool flip, uint32_t row[3]) {
  const uint32_t* g = (const uint32_t*)((const uint16_t*)gauge + off);
  if (!R12 || a < 2) {
#pragma unroll
    for (int b = 0; b < 3; b++) row[b] = __ldg(g + 3 * a + b);
  } else {
    float2 r0[3], r1[3];
#pragma unroll
    for (int b = 0; b < 3; b++) { r0[b] = unpk<P>(__ldg(g + b)); r1[b] = unpk<P>(__ldg(g + 3 + b)); }
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;
      const float re = (r0[i].x * r1[j].x - r0[i].y * r1[j].y) - (r0[j].x * r1[i].x - r0[j].y * r1[i].y);
      const float im = (r0[i].x * r1[j].y + r0[i].y * r1[j].x) - (r0[j].x * r1[i].y + r0[j].y * r1[i].x);
      row[k] = flip ? pk<P>(-re, im) : pk<P>(re, -im);
    }
  }
}

// The 8 rows o = 8a + 2 sigma + reim of A_x for direction d (K entries 12d..12d+11: slot 0
// colours 0..2, slot 1 colours 0..2, each a (re, im) pair), from row a of the link; sg =
// +-1 is the sign of the direction's projector (1 - sg gamma_mu).  Upper spins sigma = 0, 1
// take U h of slot sigma; the lower spins take U h of one slot times +-1 or +-i:
//   mu:        0     1     2     3
//   sigma 2: (1,+i) (1,+1) (0,+i) (0,-1)      (slot, coefficient for sg = +1;
//   sigma 3: (0,+i) (0,-1) (1,-i) (1,-1)       sg = -1 negates the coefficient)
// A coefficient c times U h in real form: Re(c U h) and Im(c U h) are rows of the pairs
// P0 = (Re U, -Im U), P1 = (Im U, Re U) and their negatives N0, N1:
//   c = +1: (P0, P1), -1: (N0, N1), +i: (N1, P0), -i: (P1, N0)   for (re, im) rows.
template <int MU, int SG>
__device__ __forceinline__ void write_a_rows(unsigned char* A, int j, int d, int a, const uint32_t row[3]) {
  uint32_t P0[3], P1[3], N0[3], N1[3];
#pragma unroll
  for (int b = 0; b < 3; b++) {
    P0[b] = row[b] ^ 0x80000000u;
    P1[b] = swp(row[b]);
    N0[b] = P0[b] ^ 0x80008000u;
    N1[b] = P1[b] ^ 0x80008000u;
  }
  constexpr int l0_slot = MU < 2 ? 1 : 0, l1_slot = MU < 2 ? 0 : 1;
  constexpr int l0_code = MU == 0 ? 2 : MU == 1 ? 0 : MU == 2 ? 2 : 1;   // 0: +1, 1: -1, 2: +i, 3: -i
  constexpr int l1_code = MU == 0 ? 2 : MU == 1 ? 1 : MU == 2 ? 3 : 1;
  constexpr int flipc = SG < 0 ? 1 : 0;
  const int c0 = (12 * d) >> 3;        // core matrix of the direction's first K element
  unsigned char* grp = A + (3 * j + a) * UM_GRP;
#pragma unroll
  for (int sigma = 0; sigma < 4; sigma++) {
    const int slot = sigma == 0 ? 0 : sigma == 1 ? 1 : sigma == 2 ? l0_slot : l1_slot;
    const int code = sigma < 2 ? 0 : (sigma == 2 ? l0_code : l1_code) ^ flipc;   // compile-time
#pragma unroll
    for (int reim = 0; reim < 2; reim++) {
      // variant 0 P0, 1 P1, 2 N0, 3 N1 of the (code, reim) row, selected by value
      const int var = code == 0 ? reim : code == 1 ? 2 + reim : code == 2 ? (reim ? 0 : 3) : (reim ? 2 : 1);
      uint32_t v[6];
#pragma unroll
      for (int b = 0; b < 3; b++) {
        const uint32_t w = var == 0 ? P0[b] : var == 1 ? P1[b] : var == 2 ? N0[b] : N1[b];
        v[b] = slot == 0 ? w : 0u;
        v[3 + b] = slot == 1 ? w : 0u;
      }
      unsigned char* rowp = grp + (2 * sigma + reim) * 16;
      if ((d & 1) == 0) {              // chunk c0 elements 0..7, chunk c0+1 elements 0..3
        *(uint4*)(rowp + c0 * UM_LBO) = make_uint4(v[0], v[1], v[2], v[3]);
        *(uint2*)(rowp + (c0 + 1) * UM_LBO) = make_uint2(v[4], v[5]);
      } else {                         // chunk c0 elements 4..7, chunk c0+1 elements 0..7
        *(uint2*)(rowp + c0 * UM_LBO + 8) = make_uint2(v[0], v[1]);
        *(uint4*)(rowp + (c0 + 1) * UM_LBO) = make_uint4(v[2], v[3], v[4], v[5]);
      }
    }
  }
}

// Projected half spinor of one neighbour chunk set (colours 0..2, 4 spins each):
// h slot 0 / slot 1 of colour co as (re, im) pairs, (1 - sig gamma_mu) in the chiral basis.
template <int P, int MU, int SIG>
__device__ __forceinline__ void proj(const uint4 q[3], uint32_t h[6]) {
  const uint32_t ps = pk<P>((float)SIG, (float)SIG);
  const uint32_t ns = ps ^ 0x80008000u;
#pragma unroll
  for (int co = 0; co < 3; co++) {
    const uint32_t w0 = q[co].x, w1 = q[co].y, w2 = q[co].z, w3 = q[co].w;
    uint32_t r0, r1;
    if (MU == 0 || MU == 2) {
      // i * w = (-w.im, w.re); h0 = w0 - s i wA, h1 = w1 -+ s i wB, -s i wA = swap(wA) * (s, -s)
      const uint32_t iA = swp(MU == 0 ? w3 : w2), iB = swp(MU == 0 ? w2 : w3);
      const uint32_t m0 = pk<P>((float)SIG, (float)-SIG);
      r0 = hfma<P>(iA, m0, w0);
      r1 = MU == 0 ? hfma<P>(iB, m0, w1) : hfma<P>(iB, m0 ^ 0x80008000u, w1);
    } else if (MU == 1) {
      r0 = hfma<P>(w3, ns, w0);
      r1 = hfma<P>(w2, ps, w1);
    } else {
      r0 = hfma<P>(w2, ns, w0);
      r1 = hfma<P>(w3, ns, w1);
    }
    h[co] = r0;
    h[3 + co] = r1;
  }
}

// direction D's projected half spinor comes from the partition face in this launch
template <int D>
__device__ __forceinline__ bool from_face(const HopParams& p) {
  return (D == 7 && p.face_mode == 1) || (D == 3 && p.face_mode == 2);
}

template <int P, int D, int SF>
__device__ __forceinline__ void proj_dir(const HopParams& p, unsigned nbr, int col, uint32_t h[6]) {
  constexpr int MU = D & 3;
  constexpr int SIG = D < 4 ? SF : -SF;
  const Field& f = p.in;
  if ((D & 3) == 3 && from_face<D>(p)) {   // the 12 reals the neighbouring partition formed
    const float* src = (const float*)p.face + (((long long)nbr - p.face_base) * f.W() + col) * 12;
#pragma unroll
    for (int co = 0; co < 3; co++) {
      h[co] = pk<P>(src[2 * co], src[2 * co + 1]);
      h[3 + co] = pk<P>(src[6 + 2 * co], src[7 + 2 * co]);
    }
    return;
  }
  const uint4* dp = (const uint4*)f.data;
  const unsigned W = (unsigned)f.W();
  uint4 q[3];
#pragma unroll
  for (int co = 0; co < 3; co++) q[co] = __ldg(dp + (nbr * 3 + co) * W + col);
  proj<P, MU, SIG>(q, h);
}

// the F16 norm of neighbour d's column (from the face across a partition boundary)
template <int D>
__device__ __forceinline__ float nbr_norm(const HopParams& p, unsigned nbr, int col) {
  const long long W = p.in.W();
  if ((D & 3) == 3 && from_face<D>(p)) return p.face_norm[((long long)nbr - p.face_base) * W + col];
  return __ldg(p.in.norm + nbr * W + col);
}

template <int P, int PQ, int SF>
__device__ __forceinline__ void build_pair(const HopParams& p, const unsigned* nb, int col, float inv_nmax,
                                           unsigned char* Bcol) {
  uint32_t h0[6], h1[6];
  proj_dir<P, 2 * PQ, SF>(p, nb[2 * PQ], col, h0);
  proj_dir<P, 2 * PQ + 1, SF>(p, nb[2 * PQ + 1], col, h1);
  if constexpr (P == F16) {
    const float r0 = nbr_norm<2 * PQ>(p, nb[2 * PQ], col) * inv_nmax;
    const float r1 = nbr_norm<2 * PQ + 1>(p, nb[2 * PQ + 1], col) * inv_nmax;
    const uint32_t s0 = pk<P>(r0, r0), s1 = pk<P>(r1, r1);
#pragma unroll
    for (int i = 0; i < 6; i++) { h0[i] = hmul<P>(h0[i], s0); h1[i] = hmul<P>(h1[i], s1); }
  }
  *(uint4*)(Bcol + (3 * PQ) * UM_LBO) = make_uint4(h0[0], h0[1], h0[2], h0[3]);
  *(uint4*)(Bcol + (3 * PQ + 1) * UM_LBO) = make_uint4(h0[4], h0[5], h1[0], h1[1]);
  *(uint4*)(Bcol + (3 * PQ + 2) * UM_LBO) = make_uint4(h1[2], h1[3], h1[4], h1[5]);
}

template <int P, bool DAG, bool R12, bool EPI>
__global__ void __launch_bounds__(UM_THREADS, 4) hop_umma_kernel(const __grid_constant__ HopParams p) {
  using C = float;
  extern __shared__ __align__(1024) unsigned char smem[];
  const int Ls = p.in.Ls, nrhs = p.in.nrhs, W = Ls * nrhs;
  const int S = p.ns;
  const UmLayout L = um_layout(S, nrhs, Ls);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long site0 = p.x_begin + (long long)blockIdx.x * S;
  const int nact = (int)min((long long)S, p.x_end - site0);   // active sites of this CTA
  constexpr int SF = DAG ? -1 : 1;
  uint64_t* bar = (uint64_t*)(smem + L.bar);
  uint32_t* tslot = (uint32_t*)(smem + L.bar + 8);
  unsigned* snbr = (unsigned*)(smem + L.nbr);
  float* nmax = (float*)(smem + L.nmax);
  unsigned char* A = smem + L.a;
  unsigned char* B = smem + L.b;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(su32(tslot)),
                 "r"((uint32_t)L.tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 32) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }

  // phase 0: neighbour table (and the 12-real links' time-boundary flags), one thread
  // per (site, direction)
  unsigned char* sflip = smem + L.nbr + S * 8 * 4;
  for (int i = tid; i < nact * 8; i += UM_THREADS) {
    const int j = i >> 3, d = i & 7, mu = d & 3;
    int c[4];
    cb_coords(p.g, site0 + j, p.pout, c);
    snbr[i] = (unsigned)nbr_cb(p.g, c, mu, d < 4 ? +1 : -1);
    sflip[i] = R12 && mu == 3 && p.t_bc < 0 && (d < 4 ? c[3] == p.g.T - 1 && p.bc_hi : c[3] == 0 && p.bc_lo);
  }
  __syncthreads();

  // link matrices, one thread per (site, direction, colour row a): 8 rows of 12 entries
  for (int i = tid; i < nact * 24; i += UM_THREADS) {
    const int j = i / 24, r = i - j * 24, d = r / 3, a = r - d * 3;
    uint32_t row[3];
    link_row<P, R12>(p.gauge, ((site0 + j) * 8 + d) * p.gs, a, sflip[j * 8 + d] != 0, row);
    switch (d) {   // forward directions project with SF, backward ones with -SF
      case 0: write_a_rows<0, SF>(A, j, d, a, row); break;
      case 1: write_a_rows<1, SF>(A, j, d, a, row); break;
      case 2: write_a_rows<2, SF>(A, j, d, a, row); break;
      case 3: write_a_rows<3, SF>(A, j, d, a, row); break;
      case 4: write_a_rows<0, -SF>(A, j, d, a, row); break;
      case 5: write_a_rows<1, -SF>(A, j, d, a, row); break;
      case 6: write_a_rows<2, -SF>(A, j, d, a, row); break;
      default: write_a_rows<3, -SF>(A, j, d, a, row); break;
    }
  }

  // phase 1: projected neighbours (B operand), one thread per (site, direction pair, column)
  const float inv_w = 1.0f / (float)W;
  for (int i = tid; i < nact * 4 * W; i += UM_THREADS) {
    const int jq = div_small(i, inv_w), n = i - jq * W, j = jq >> 2, pq = jq & 3;
    const unsigned* nb = snbr + j * 8;
    float inv = 1.0f;
    if constexpr (P == F16) {
      float m = fmaxf(fmaxf(fmaxf(nbr_norm<0>(p, nb[0], n), nbr_norm<1>(p, nb[1], n)),
                            fmaxf(nbr_norm<2>(p, nb[2], n), nbr_norm<3>(p, nb[3], n))),
                      fmaxf(fmaxf(nbr_norm<4>(p, nb[4], n), nbr_norm<5>(p, nb[5], n)),
                            fmaxf(nbr_norm<6>(p, nb[6], n), nbr_norm<7>(p, nb[7], n))));
      inv = m > 0.0f ? 1.0f / m : 0.0f;
      if (pq == 0) nmax[j * L.npad + n] = m;
    }
    const int grow = j * L.npad + n;
    unsigned char* Bcol = B + (grow >> 3) * UM_GRP + (grow & 7) * 16;
    switch (pq) {
      case 0: build_pair<P, 0, SF>(p, nb, n, inv, Bcol); break;
      case 1: build_pair<P, 1, SF>(p, nb, n, inv, Bcol); break;
      case 2: build_pair<P, 2, SF>(p, nb, n, inv, Bcol); break;
      default: build_pair<P, 3, SF>(p, nb, n, inv, Bcol); break;
    }
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t bar_a = su32(bar);

  // phase 2: the contraction, 6 MMAs (K = 16 each) per site, issued by one thread, which
  // also waits for their completion (the other threads wait at the barrier)
  int* okflag = (int*)(smem + L.bar + 12);
  if (tid == 0) {
    const uint32_t idesc = um_idesc<P>(L.npad);
    const uint32_t a0 = su32(A), b0 = su32(B);
    for (int j = 0; j < nact; j++) {
#pragma unroll
      for (int ks = 0; ks < 6; ks++)
        um_mma(tbase + (uint32_t)(j * L.npad), sdesc(a0 + 3 * j * UM_GRP + ks * UM_KSTEP),
               sdesc(b0 + j * (L.npad / 8) * UM_GRP + ks * UM_KSTEP), idesc, ks > 0 ? 1u : 0u);
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar_a)
                 : "memory");
    bool ok = um_wait(bar_a, 0);
    if (!ok) {
      if (p.status) atomicOr(p.status, 1);
      ok = um_wait(bar_a, 0);   // a second bounded wait before the accumulators are read or released
    }
    *okflag = ok ? 1 : 0;
    fence_before();
  }
  __syncthreads();
  fence_after();

  // phase 3: accumulators -> epilogue tile.  With M = 64 accumulator row 16w + i sits in
  // TMEM lane 32w + i (i < 16), which only warp w may read: rows 0..15 go through warp 0,
  // rows 16..23 through warp 1.
  C* tileH = (C*)(smem + L.tile);
  const int GS = tile_gstr(Ls);
  if (warp < 2 && *okflag) {
    const int o = 16 * warp + lane;                  // accumulator row of this lane
    const bool mine = lane < (warp == 0 ? 16 : 8);
    const float inv_ls = 1.0f / (float)Ls;
    if (nrhs == 1 && W <= 16) {   // one right-hand side of Ls <= 16: column n is slice s, one load per site
      for (int j = 0; j < nact; j++) {
        float v[16];
        um_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(j * L.npad), v);
        if (mine) {
          C* dst = tileH + j * nrhs * GS + o;
          const float* sc = nmax + j * L.npad;
#pragma unroll
          for (int q = 0; q < 16; q++)
            if (q < W) dst[q * TSTR] = P == F16 ? v[q] * sc[q] : v[q];
        }
      }
    } else
    for (int j = 0; j < nact; j++) {
      for (int c0 = 0; c0 < W; c0 += 16) {
        float v[16];
        um_ld16(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)(j * L.npad + c0), v);
        if (mine) {
          int r = div_small(c0, inv_ls), s = c0 - r * Ls;   // column n = r Ls + s, walked in order
          C* dst = tileH + (j * nrhs + r) * GS + s * TSTR + o;
#pragma unroll
          for (int q = 0; q < 16; q++) {
            if (c0 + q < W) {
              float sc = 1.0f;
              if constexpr (P == F16) sc = nmax[j * L.npad + c0 + q];
              *dst = v[q] * sc;
            }
            dst += TSTR;
            if (++s == Ls) { s = 0; dst += GS - Ls * TSTR; }
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"((uint32_t)L.tcols));
  }

  if constexpr (!EPI) {
    for (int i = tid; i < nact * W; i += UM_THREADS) {
      const int j = i / W, n = i - j * W, r = n / Ls, s = n - r * Ls;
      C v[24];
      const C* row = tileH + (j * nrhs + r) * GS + s * TSTR;
#pragma unroll
      for (int k = 0; k < 24; k++) v[k] = row[k];
      store_site<P>(p.out, site0 + j, n, v);
    }
  } else {
    const size_t toff = ((size_t)S * nrhs * GS * sizeof(C) + 15) & ~(size_t)15;
    double* redsm = (double*)((unsigned char*)tileH + toff);
    hop_epilogue<P>(p, tileH, redsm, S);
  }
}

template <int P, bool DAG, bool R12, bool EPI>
cudaError_t launch_um(const HopParams& p, size_t smem, cudaStream_t st) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(hop_umma_kernel<P, DAG, R12, EPI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const long long blocks = (p.x_end - p.x_begin + p.ns - 1) / p.ns;
  HopParams q = p;
  q.hcf = (float)p.hc; q.ccf = (float)p.cc; q.mff = (float)p.mf;
  hop_umma_kernel<P, DAG, R12, EPI><<<(unsigned)blocks, UM_THREADS, smem, st>>>(q);
  return cudaGetLastError();
}

template <int P>
cudaError_t launch_um_prec(const HopParams& p, bool dag, bool r12, bool epi, size_t smem, cudaStream_t st) {
  if (dag) {
    if (r12) return epi ? launch_um<P, true, true, true>(p, smem, st) : launch_um<P, true, true, false>(p, smem, st);
    return epi ? launch_um<P, true, false, true>(p, smem, st) : launch_um<P, true, false, false>(p, smem, st);
  }
  if (r12) return epi ? launch_um<P, false, true, true>(p, smem, st) : launch_um<P, false, true, false>(p, smem, st);
  return epi ? launch_um<P, false, false, true>(p, smem, st) : launch_um<P, false, false, false>(p, smem, st);
}

}  // namespace

bool hop_tc_supported(int prec, const HopParams& p, bool r12) {
  (void)r12;
  const int W = p.in.nrhs * p.in.Ls;
  return (prec == F16 || prec == BF16) && W <= 256;
}

size_t hop_tc_smem_bytes(const HopParams& p) {
  return (size_t)um_layout(p.ns, p.in.nrhs, p.in.Ls).total;
}

int hop_tc_tmem_cols(const HopParams& p) { return um_layout(p.ns, p.in.nrhs, p.in.Ls).tcols; }

cudaError_t launch_hop_tc(int prec, bool dag, bool r12, bool epi, const HopParams& p, cudaStream_t st) {
  const size_t smem = hop_tc_smem_bytes(p);
  if (prec == F16) return launch_um_prec<F16>(p, dag, r12, epi, smem, st);
  if (prec == BF16) return launch_um_prec<BF16>(p, dag, r12, epi, smem, st);
  return cudaErrorInvalidValue;
}

}  // namespace mdwf
