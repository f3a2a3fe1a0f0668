// Internal definitions of libmdwf: precision traits, field and gauge layouts, lattice
// geometry, s-direction operators and deterministic FP64 reductions.
//
// Internal spinor layout (one parity half of a field; Ls-inner, site-blocked):
//   16-byte chunk (x_cb, c, r, s) at  (x_cb * NC + c) * W + (r * Ls + s),  W = nrhs * Ls
// so that the nrhs * Ls threads of one 4D site read consecutive chunks.  A site's 24
// reals are ordered [colour][spin][re,im]; an F16/BF16 chunk is one colour (4 spins).
// F16 keeps one float norm per 5D site at norm[x_cb * W + r * Ls + s].
//
// Internal gauge layout (per parity): link (x_cb, dir) at (x_cb * 8 + dir) * GS reals,
// dir 0..3 = U_mu(x), dir 4..7 = U_mu(x - mu)^+, boundary phase folded in (recon 18) or
// re-applied after rebuilding the third row (recon 12).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace mdwf {

enum Prec { F64 = 0, F32 = 1, F16 = 2, BF16 = 3, I16 = 4 };
constexpr int NPREC = 5;   // storage precisions (array extent for per-precision state)
constexpr int MAXLS = 32;
constexpr int MAXTHREADS = 256;  // threads per CTA of site-tiled kernels (NS * nrhs * Ls)

template <int P> struct PT;
template <> struct PT<F64> {
  using C = double; using S = double; using G = double;
  static constexpr int NC = 12; static constexpr bool NORM = false;
  static constexpr int GS18 = 18, GS12 = 12;
};
template <> struct PT<F32> {
  using C = float; using S = float; using G = float;
  static constexpr int NC = 6; static constexpr bool NORM = false;
  static constexpr int GS18 = 20, GS12 = 12;
};
template <> struct PT<F16> {
  using C = float; using S = __half; using G = __half;
  static constexpr int NC = 3; static constexpr bool NORM = true;
  static constexpr int GS18 = 24, GS12 = 16;
};
template <> struct PT<BF16> {
  using C = float; using S = __nv_bfloat16; using G = __nv_bfloat16;
  static constexpr int NC = 3; static constexpr bool NORM = false;
  static constexpr int GS18 = 24, GS12 = 16;
};
// 16-bit fixed point: a site's reals are q / 32767 times its norm, links q / 32767
template <> struct PT<I16> {
  using C = float; using S = int16_t; using G = int16_t;
  static constexpr int NC = 3; static constexpr bool NORM = true;
  static constexpr int GS18 = 24, GS12 = 16;
};
constexpr float I16_ONE = 32767.0f;
constexpr float I16_INV = 1.0f / 32767.0f;

// the two int16 of a 32-bit word as exact floats: x + 1.5 2^23 written into a float's
// mantissa (|x| < 2^22), minus 1.5 2^23
__device__ __forceinline__ float2 i16x2_to_float2(uint32_t w) {
  const int lo = (int)(int16_t)(w & 0xFFFFu), hi = (int)w >> 16;
  return make_float2(__int_as_float(0x4B400000 + lo) - 12582912.0f, __int_as_float(0x4B400000 + hi) - 12582912.0f);
}
__device__ __forceinline__ uint32_t float2_to_i16x2(float a, float b) {
  return ((uint32_t)(uint16_t)(int16_t)__float2int_rn(a)) | ((uint32_t)(uint16_t)(int16_t)__float2int_rn(b) << 16);
}

inline int prec_nc(int p) { return p == F64 ? 12 : p == F32 ? 6 : 3; }
inline bool prec_norm(int p) { return p == F16 || p == I16; }
inline int gauge_stride(int p, int recon) {
  if (recon == 12) return p == F64 || p == F32 ? 12 : 16;
  return p == F64 ? 18 : p == F32 ? 20 : 24;
}
inline size_t prec_gsize(int p) { return p == F64 ? 8 : p == F32 ? 4 : 2; }

// One parity half of an internal field.
struct Field {
  void* data;
  float* norm;     // F16 only
  int nrhs;
  int Ls;
  long long vh;    // 4D sites per parity
  __host__ __device__ long long W() const { return (long long)nrhs * Ls; }
};

// ---------------------------------------------------------------- conversions
template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// load the 24 reals of 5D site (x_cb, col = r*Ls+s) into v (compute type)
template <int P>
__device__ __forceinline__ void load_site(const Field& f, long long x_cb, int col,
                                          typename PT<P>::C v[24]) {
  const long long W = f.W();
  if constexpr (P == F64) {
    const double2* d = (const double2*)f.data;
#pragma unroll
    for (int c = 0; c < 12; c++) {
      double2 q = __ldg(d + (x_cb * 12 + c) * W + col);
      v[2 * c] = q.x; v[2 * c + 1] = q.y;
    }
  } else if constexpr (P == F32) {
    const float4* d = (const float4*)f.data;
#pragma unroll
    for (int c = 0; c < 6; c++) {
      float4 q = __ldg(d + (x_cb * 6 + c) * W + col);
      v[4 * c] = q.x; v[4 * c + 1] = q.y; v[4 * c + 2] = q.z; v[4 * c + 3] = q.w;
    }
  } else {
    const uint4* d = (const uint4*)f.data;
    float nrm = 1.0f;
    if constexpr (P == F16) nrm = __ldg(f.norm + x_cb * W + col);
    if constexpr (P == I16) nrm = __ldg(f.norm + x_cb * W + col) * I16_INV;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint4 q = __ldg(d + (x_cb * 3 + c) * W + col);
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; j++) {
        if constexpr (P == F16 || P == I16) {
          const float2 fv = P == F16 ? __half22float2(*(const __half2*)&w[j]) : i16x2_to_float2(w[j]);
          v[8 * c + 2 * j] = fv.x * nrm; v[8 * c + 2 * j + 1] = fv.y * nrm;
        } else {
          float2 fv = __bfloat1622float2(*(const __nv_bfloat162*)&w[j]);
          v[8 * c + 2 * j] = fv.x; v[8 * c + 2 * j + 1] = fv.y;
        }
      }
    }
  }
}

// store 24 reals; returns nothing.  F16 computes the per-site max-abs norm.
template <int P>
__device__ __forceinline__ void store_site(const Field& f, long long x_cb, int col,
                                           const typename PT<P>::C v[24]) {
  const long long W = f.W();
  if constexpr (P == F64) {
    double2* d = (double2*)f.data;
#pragma unroll
    for (int c = 0; c < 12; c++) d[(x_cb * 12 + c) * W + col] = make_double2(v[2 * c], v[2 * c + 1]);
  } else if constexpr (P == F32) {
    float4* d = (float4*)f.data;
#pragma unroll
    for (int c = 0; c < 6; c++)
      d[(x_cb * 6 + c) * W + col] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  } else {
    uint4* d = (uint4*)f.data;
    float scale = 1.0f;
    if constexpr (P == F16 || P == I16) {
      float m = 0.0f;
#pragma unroll
      for (int i = 0; i < 24; i++) m = fmaxf(m, fabsf(v[i]));
      // a site whose largest component is below the smallest normal float stores zero
      // (1/m would overflow); such entries are far below half-precision resolution of any
      // field they belong to
      if (!(m >= 1.17549435e-38f)) m = 0.0f;
      f.norm[x_cb * W + col] = m;
      scale = m > 0.0f ? (P == I16 ? I16_ONE : 1.0f) / m : 0.0f;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      uint32_t w[4];
#pragma unroll
      for (int j = 0; j < 4; j++) {
        if constexpr (P == F16) {
          __half2 h = __floats2half2_rn(v[8 * c + 2 * j] * scale, v[8 * c + 2 * j + 1] * scale);
          w[j] = *(uint32_t*)&h;
        } else if constexpr (P == I16) {
          w[j] = float2_to_i16x2(v[8 * c + 2 * j] * scale, v[8 * c + 2 * j + 1] * scale);
        } else {
          __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * c + 2 * j], v[8 * c + 2 * j + 1]);
          w[j] = *(uint32_t*)&h;
        }
      }
      d[(x_cb * 3 + c) * W + col] = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
}

// i / w for 0 <= i < 2^16, 1 <= w <= 2^10 without an integer division: the FP32 quotient
// of i + 1/2 lies at least 1/(2w) from an integer and has a relative error below 2^-23
// (checked exhaustively over that range).
__device__ __forceinline__ int div_small(int i, float inv_w) { return __float2int_rz(((float)i + 0.5f) * inv_w); }

// ---------------------------------------------------------------- geometry
// n / d for 0 <= n < 2^32 by a multiply-high (Granlund-Montgomery, round-up variant):
// m = floor(2^(32+l) / d) + 1 with l = ceil(log2 d) has m d - 2^(32+l) <= 2^l, so
// floor(n m / 2^(32+l)) = floor(n / d); m < 2^33 is kept as m_hi 2^32 + m_lo.
struct FastDiv {
  uint32_t m_lo, m_hi, l;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{0u, 1u, 0u};   // d = 1: m = 2^32
  if (d > 1) {
    uint32_t l = 0;
    while ((1ull << l) < d) l++;
    const unsigned long long m = ((1ull << (32 + l)) / d) + 1ull;
    f.m_lo = (uint32_t)m;
    f.m_hi = (uint32_t)(m >> 32);
    f.l = l;
  }
  return f;
}
__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv& f) {
  const uint32_t t = __umulhi(n, f.m_lo);
  return (uint32_t)(((unsigned long long)t + (f.m_hi ? n : 0u)) >> f.l);
}

struct Geom {
  int X, Y, Z, T, Xh;
  long long vh;      // < 2^31
  FastDiv fXh, fY, fZ;
};

__device__ __forceinline__ void cb_coords(const Geom& g, long long x_cb, int parity, int c[4]) {
  const uint32_t n = (uint32_t)x_cb;
  const uint32_t r1 = fdiv(n, g.fXh), r2 = fdiv(r1, g.fY), r3 = fdiv(r2, g.fZ);
  const int xh = (int)(n - r1 * (uint32_t)g.Xh);
  c[1] = (int)(r1 - r2 * (uint32_t)g.Y);
  c[2] = (int)(r2 - r3 * (uint32_t)g.Z);
  c[3] = (int)r3;
  c[0] = 2 * xh + ((parity + c[1] + c[2] + c[3]) & 1);
}

__device__ __forceinline__ long long cb_index(const Geom& g, const int c[4]) {
  return ((((long long)c[3] * g.Z + c[2]) * g.Y + c[1]) * g.X + c[0]) >> 1;
}

__device__ __forceinline__ long long nbr_cb(const Geom& g, const int c[4], int mu, int dir) {
  int n[4] = {c[0], c[1], c[2], c[3]};
  const int L = mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.T;
  int v = n[mu] + dir;
  n[mu] = v < 0 ? v + L : (v >= L ? v - L : v);
  return cb_index(g, n);
}

// ---------------------------------------------------------------- s-direction operators
// Each op acts on the Ls values of one real component of one (4D site, rhs).
// The spin pair decides the shift direction: B moves P_- (spins 0,1) from s+1 and P_+
// (spins 2,3) from s-1; B^+ swaps them.  "up" = takes s+1 with the wall -mf at Ls-1.
enum SOpKind { SOP_NONE = 0, SOP_BIDIAG = 1, SOP_INV = 2 };
struct SOp {
  int kind;      // SOP_NONE / SOP_BIDIAG (a + b S) / SOP_INV ((a + b S)^-1)
  int dag;       // use B^+ instead of B
  double a, b;   // coefficients
  double inv_a;  // 1/a
  double c0;     // 1 / (a (1 + mf rho^Ls)), rho = -b/a
  double w[MAXLS];  // w[k] = -mf rho^(k+1) c0, k = 0..Ls-2
  // the same rounded to FP32 on the host: the 32-bit kernels read these, so that no
  // double -> float conversion (an FP64-pipe instruction, scarce on GB300) runs per use
  float fa, fb, finv_a, fc0;
  float fw[MAXLS];
};

// coefficients in the compute type
template <typename C> __device__ __forceinline__ C sop_a(const SOp& o) { if constexpr (sizeof(C) == 4) return o.fa; else return (C)o.a; }
template <typename C> __device__ __forceinline__ C sop_b(const SOp& o) { if constexpr (sizeof(C) == 4) return o.fb; else return (C)o.b; }
template <typename C> __device__ __forceinline__ C sop_inv_a(const SOp& o) { if constexpr (sizeof(C) == 4) return o.finv_a; else return (C)o.inv_a; }
template <typename C> __device__ __forceinline__ C sop_c0(const SOp& o) { if constexpr (sizeof(C) == 4) return o.fc0; else return (C)o.c0; }
template <typename C> __device__ __forceinline__ C sop_w(const SOp& o, int j) { if constexpr (sizeof(C) == 4) return o.fw[j]; else return (C)o.w[j]; }

struct SChain {
  SOp op[2];
};

// In-place application of one op to the strided sequence y[s * st], s = 0..Ls-1.
template <typename C>
__device__ __forceinline__ void sop_apply(const SOp& o, bool up, C* y, int st, int Ls, C mf) {
  if (o.kind == SOP_BIDIAG) {
    const C a = sop_a<C>(o), b = sop_b<C>(o);
    if (up) {
      C y0 = y[0];
      for (int s = 0; s < Ls - 1; s++) y[s * st] = a * y[s * st] + b * y[(s + 1) * st];
      y[(Ls - 1) * st] = a * y[(Ls - 1) * st] - b * mf * y0;
    } else {
      C yl = y[(Ls - 1) * st];
      for (int s = Ls - 1; s > 0; s--) y[s * st] = a * y[s * st] + b * y[(s - 1) * st];
      y[0] = a * y[0] - b * mf * yl;
    }
  } else if (o.kind == SOP_INV) {
    // (a + b S)^-1 with S^Ls = -mf: the last (up) / first (down) entry from the closed
    // form sum, then a first-order recurrence back through the chain.
    const C inv_a = sop_inv_a<C>(o), b = sop_b<C>(o);
    if (up) {
      C acc = sop_c0<C>(o) * y[(Ls - 1) * st];
      for (int j = 0; j < Ls - 1; j++) acc += sop_w<C>(o, j) * y[j * st];
      y[(Ls - 1) * st] = acc;
      for (int s = Ls - 2; s >= 0; s--) {
        acc = (y[s * st] - b * acc) * inv_a;
        y[s * st] = acc;
      }
    } else {
      C acc = sop_c0<C>(o) * y[0];
      for (int j = 0; j < Ls - 1; j++) acc += sop_w<C>(o, j) * y[(Ls - 1 - j) * st];
      y[0] = acc;
      for (int s = 1; s < Ls; s++) {
        acc = (y[s * st] - b * acc) * inv_a;
        y[s * st] = acc;
      }
    }
  }
}

template <typename C>
__device__ __forceinline__ void chain_apply(const SChain& ch, int comp, C* y, int st, int Ls, C mf) {
  // comp = real index within the site [colour][spin][re/im] -> spin = (comp >> 1) & 3
  const bool lower = ((comp >> 1) & 3) >= 2;
#pragma unroll
  for (int i = 0; i < 2; i++) {
    if (ch.op[i].kind == SOP_NONE) continue;
    const bool up = (!lower) != (bool)ch.op[i].dag;  // B: P_- up; B^+: P_+ up
    sop_apply(ch.op[i], up, y, st, Ls, mf);
  }
}

// Compile-time-Ls version: the column lives in registers, every loop is unrolled.
template <typename C, int L>
__device__ __forceinline__ void sop_col(const SOp& o, bool up, C (&y)[L], C mf) {
  if (o.kind == SOP_BIDIAG) {
    const C a = sop_a<C>(o), b = sop_b<C>(o);
    if (up) {
      const C y0 = y[0];
#pragma unroll
      for (int s = 0; s < L - 1; s++) y[s] = a * y[s] + b * y[s + 1];
      y[L - 1] = a * y[L - 1] - b * mf * y0;
    } else {
      const C yl = y[L - 1];
#pragma unroll
      for (int s = L - 1; s > 0; s--) y[s] = a * y[s] + b * y[s - 1];
      y[0] = a * y[0] - b * mf * yl;
    }
  } else if (o.kind == SOP_INV) {
    const C inv_a = sop_inv_a<C>(o), b = sop_b<C>(o);
    if (up) {
      C acc = sop_c0<C>(o) * y[L - 1];
#pragma unroll
      for (int j = 0; j < L - 1; j++) acc += sop_w<C>(o, j) * y[j];
      y[L - 1] = acc;
#pragma unroll
      for (int s = L - 2; s >= 0; s--) { acc = (y[s] - b * acc) * inv_a; y[s] = acc; }
    } else {
      C acc = sop_c0<C>(o) * y[0];
#pragma unroll
      for (int j = 0; j < L - 1; j++) acc += sop_w<C>(o, j) * y[L - 1 - j];
      y[0] = acc;
#pragma unroll
      for (int s = 1; s < L; s++) { acc = (y[s] - b * acc) * inv_a; y[s] = acc; }
    }
  }
}

template <typename C, int L>
__device__ __forceinline__ void chain_col(const SChain& ch, bool lower, C* col, int st, C mf) {
  C y[L];
#pragma unroll
  for (int s = 0; s < L; s++) y[s] = col[s * st];
#pragma unroll
  for (int i = 0; i < 2; i++) {
    if (ch.op[i].kind == SOP_NONE) continue;
    sop_col<C, L>(ch.op[i], (!lower) != (bool)ch.op[i].dag, y, mf);
  }
#pragma unroll
  for (int s = 0; s < L; s++) col[s * st] = y[s];
}

// chain on one strided column in shared memory: unrolled register code for the common
// Ls = 8, 10, 12, 16 (few variants keep the kernels' code small), a loop otherwise
template <typename C>
__device__ __forceinline__ void chain_apply_fast(const SChain& ch, int comp, C* col, int st, int Ls, C mf) {
  const bool lower = ((comp >> 1) & 3) >= 2;
  switch (Ls) {
#define CASE_L(L) case L: chain_col<C, L>(ch, lower, col, st, mf); return;
    CASE_L(8) CASE_L(10) CASE_L(12) CASE_L(16)
#undef CASE_L
    default: chain_apply(ch, comp, col, st, Ls, mf);
  }
}

// Epilogue tile layout [grp = site * nrhs + rhs][s][component]: 24 components padded to
// TSTR per s (16-byte aligned rows, conflict-free 16-byte accesses), groups padded so
// that consecutive groups start 24 banks apart (conflict-free column walks).
constexpr int TSTR = 28;
__host__ __device__ inline int tile_gstr(int Ls) {
  const int base = Ls * TSTR;
  return base + ((24 - (base & 31)) & 31);
}

// Shared-memory layout of the bulk-staged hop kernel: links (20 floats each, 8 per site
// plus 4 floats of bank offset), neighbour table, mbarrier, the neighbour rows (48 W bytes
// each, 128-byte aligned), epilogue.
struct BulkLayout { int nbr, bar, rows, epi; };
__host__ __device__ inline BulkLayout bulk_layout(int ns, int W) {
  BulkLayout L;
  L.nbr = ns * (8 * 20 + 4) * 4;
  L.bar = (L.nbr + ((ns * 8 + 3) & ~3) * 4 + 15) & ~15;
  L.rows = (L.bar + 16 + 127) & ~127;
  L.epi = L.rows + ns * 8 * 48 * W;
  return L;
}

// ---------------------------------------------------------------- reductions
// Block partials -> last block sums them in a fixed order (deterministic) and runs a
// scalar program.  partials[block * nrhs + r], counter reset by the last block.
enum RedMode { RED_NONE = 0, RED_STORE = 1, RED_CG_ALPHA = 2, RED_CG_BETA = 3 };

struct CGScalars {   // per right-hand side
  double gamma;      // |r|^2 of the current iterate
  double qq;         // |M p|^2
  double alpha, beta;
  double stop2;      // iterated-residual threshold (squared)
  double maxr2;      // max |r|^2 since the last reliable update
  int active;        // 0 once converged: alpha = beta = 0 freeze the iterate
  int hit;           // gamma <= stop2 seen
  int breakdown;
  int pad;
  float alpha_f, beta_f;   // alpha, beta rounded once for the 32-bit kernels
  int pad2[2];
};

// a scalar in the compute type: the FP32 copy for 32-bit kernels (no per-thread
// double -> float conversion on the FP64 pipe), the double otherwise
template <typename C> __device__ __forceinline__ C pick(float f, double d) {
  if constexpr (sizeof(C) == 4) return f; else return (C)d;
}

struct Red {
  int mode;
  double* partials;   // [blocks][nrhs] block partials, then [groups][nrhs] group partials
  unsigned int* counter;   // [0]: groups finished; [1 + g]: blocks of group g finished
  double* out;        // RED_STORE: out[r]
  CGScalars* cg;      // RED_CG_*
  int nrhs;
};

constexpr int RED_GROUP = 128;   // blocks per first-level group of the grid reduction

// fixed-order sum over i < n of src[i * stride] by the whole block (sm: blockDim doubles)
__device__ inline double block_sum_strided(const double* src, int n, int stride, double* sm) {
  const int tid = threadIdx.x;
  double acc = 0.0;
  for (int b = tid; b < n; b += blockDim.x) acc += __ldcg(src + (long long)b * stride);
  sm[tid] = acc;
  __syncthreads();
  for (int w = blockDim.x; w > 1;) {
    const int h = (w + 1) >> 1;
    if (tid < w - h) sm[tid] += sm[tid + h];
    __syncthreads();
    w = h;
  }
  const double tot = sm[0];
  __syncthreads();
  return tot;
}

// Grid reduction of per-5D-site values sm[(site_l * nrhs + r) * Ls + s], i < ns * nrhs * Ls,
// already in shared memory (scratch must hold max(ns*nrhs*Ls, blockDim.x) + ns*nrhs doubles):
// fixed-order sums per (site, rhs), per rhs over the block; the last block of each group of
// RED_GROUP blocks sums its group's partials, the last group to finish sums the group
// partials and runs the scalar program.  Every sum runs in a fixed order, whichever block
// finishes last: the result is deterministic, and no block reads more than
// max(RED_GROUP, blocks / RED_GROUP) partials per right-hand side.
__device__ inline void block_grid_reduce_sm(const Red& red, double* sm, int Ls, int ns) {
  const int tid = threadIdx.x;
  const int nrhs = red.nrhs;
  const int ngrp = ns * nrhs;
  const int nitems = ngrp * Ls;
  double* sm2 = sm + (nitems > (int)blockDim.x ? nitems : (int)blockDim.x);
  __syncthreads();
  for (int gi = tid; gi < ngrp; gi += blockDim.x) {
    double acc = 0.0;
    for (int s = 0; s < Ls; s++) acc += sm[gi * Ls + s];
    sm2[gi] = acc;
  }
  __syncthreads();
  for (int r = tid; r < nrhs; r += blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < ns; i++) acc += sm2[i * nrhs + r];
    red.partials[(long long)blockIdx.x * nrhs + r] = acc;
  }
  const int nb = gridDim.x;
  const int g = blockIdx.x / RED_GROUP, ngroups = (nb + RED_GROUP - 1) / RED_GROUP;
  const int gsize = min(RED_GROUP, nb - g * RED_GROUP);
  double* gpart = red.partials + (long long)nb * nrhs;
  __shared__ unsigned int ticket;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(red.counter + 1 + g, 1u);
  __syncthreads();
  if (ticket != (unsigned)gsize - 1) return;
  __threadfence();
  // last block of group g: its group's partials, fixed order
  for (int r = 0; r < nrhs; r++) {
    const double tot = block_sum_strided(red.partials + ((long long)g * RED_GROUP) * nrhs + r, gsize, nrhs, sm);
    if (tid == 0) gpart[(long long)g * nrhs + r] = tot;
  }
  if (tid == 0) red.counter[1 + g] = 0u;
  __threadfence();
  __syncthreads();
  if (tid == 0) ticket = atomicAdd(red.counter, 1u);
  __syncthreads();
  if (ticket != (unsigned)ngroups - 1) return;
  __threadfence();
  // last group: the group partials, fixed order, and the scalar program
  for (int r = 0; r < nrhs; r++) {
    const double tot = block_sum_strided(gpart + r, ngroups, nrhs, sm);
    if (tid == 0) {
      if (red.mode == RED_STORE) {
        red.out[r] = tot;
      } else if (red.mode == RED_CG_ALPHA) {
        CGScalars& c = red.cg[r];
        c.qq = tot;
        if (!(tot == tot) || tot <= 0.0) {
          if (c.active && c.gamma > 0.0) c.breakdown = 1;
          c.alpha = 0.0;
        } else {
          c.alpha = c.active ? c.gamma / tot : 0.0;
        }
        c.alpha_f = (float)c.alpha;
      } else if (red.mode == RED_CG_BETA) {
        CGScalars& c = red.cg[r];
        if (c.active) {
          if (!(tot == tot)) c.breakdown = 1;
          c.beta = c.gamma > 0.0 ? tot / c.gamma : 0.0;
          c.gamma = tot;
          if (tot <= c.stop2) c.hit = 1;
        } else {
          c.beta = 0.0;
        }
        c.beta_f = (float)c.beta;
      }
    }
  }
  if (tid == 0) *red.counter = 0u;
}

// Per-thread value version for kernels whose threads are exactly the (site_l, r, s) sites.
__device__ inline void block_grid_reduce(const Red& red, double v, double* sm, int Ls, int ns) {
  sm[threadIdx.x] = v;
  block_grid_reduce_sm(red, sm, Ls, ns);
}

}  // namespace mdwf
