// Layout conversion and the physics steps around the solve:
//   * user <-> internal spinor layouts, with the F16 (+ per-site norm) / BF16 / F32
//     storage formats of the "double-half" inner solver (Sec. "Current State of the Art");
//   * gauge load into the per-parity SoA link layout (forward links and daggered backward
//     links, time boundary phase folded in) and the SU(3) check;
//   * 4D point-source injection / projection, the Feynman-Hellmann sequential source and
//     the nucleon two-point contraction (Sec. "Performance Measurement Method": the
//     propagators feed tensor contractions).
#include "mdwf_impl.cuh"
#include "mdwf_kernels.h"

#include <type_traits>

namespace mdwf {

__device__ __forceinline__ long long full_index(const Geom& g, const int c[4]) {
  return (((long long)c[3] * g.Z + c[2]) * g.Y + c[1]) * g.X + c[0];
}

// ---------------------------------------------------------------- pack / unpack
// thread per (parity, x_cb, r, s); user site has 12 complex ordered [spin][colour]
template <int P>
__global__ void pack_kernel(PackParams p) {
  const long long W = (long long)p.nrhs * p.Ls;
  const long long n = 2 * p.g.vh * W;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int col = (int)(i % W);
  const long long x_cb = (i / W) % p.g.vh;
  const int parity = (int)(i / (W * p.g.vh));
  const int r = col / p.Ls, s = col % p.Ls;
  int c[4];
  cb_coords(p.g, x_cb, parity, c);
  const long long V = 2 * p.g.vh;
  const double2* src = (const double2*)p.user + (((long long)r * p.Ls + s) * V + full_index(p.g, c)) * 12;
  double v[24];  // [colour][spin][re,im]
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int co = 0; co < 3; co++) {
      double2 z = src[sp * 3 + co];
      v[2 * (co * 4 + sp)] = z.x; v[2 * (co * 4 + sp) + 1] = z.y;
    }
  if constexpr (P == F64) {
    double2* d = (double2*)p.data[parity];
#pragma unroll
    for (int k = 0; k < 12; k++) d[(x_cb * 12 + k) * W + col] = make_double2(v[2 * k], v[2 * k + 1]);
  } else if constexpr (P == F32) {
    float4* d = (float4*)p.data[parity];
#pragma unroll
    for (int k = 0; k < 6; k++)
      d[(x_cb * 6 + k) * W + col] = make_float4(__double2float_rn(v[4 * k]), __double2float_rn(v[4 * k + 1]),
                                                __double2float_rn(v[4 * k + 2]), __double2float_rn(v[4 * k + 3]));
  } else {
    // F16: norm = float(max |v|), half = RNE(v / double(norm)); BF16: RNE(v);
    // I16: norm as F16, q = RNE(32767 v / double(norm)) (FP64 product, then quotient)
    double scale_div = 1.0;
    bool zero = false;
    if constexpr (P == F16 || P == I16) {
      double m = 0.0;
#pragma unroll
      for (int k = 0; k < 24; k++) m = fmax(m, fabs(v[k]));
      const float nf = __double2float_rn(m);
      p.norm[parity][x_cb * W + col] = nf;
      scale_div = (double)nf;
      zero = !(nf > 0.0f);
    }
    uint4* d = (uint4*)p.data[parity];
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint16_t h[8];
#pragma unroll
      for (int j = 0; j < 8; j++) {
        if constexpr (P == F16) {
          __half q = zero ? __float2half(0.0f) : __double2half(v[8 * k + j] / scale_div);
          h[j] = *(uint16_t*)&q;
        } else if constexpr (P == I16) {
          h[j] = zero ? (uint16_t)0 : (uint16_t)(int16_t)__double2int_rn(32767.0 * v[8 * k + j] / scale_div);
        } else {
          __nv_bfloat16 q = __double2bfloat16(v[8 * k + j]);
          h[j] = *(uint16_t*)&q;
        }
      }
      d[(x_cb * 3 + k) * W + col] = make_uint4(h[0] | ((uint32_t)h[1] << 16), h[2] | ((uint32_t)h[3] << 16),
                                               h[4] | ((uint32_t)h[5] << 16), h[6] | ((uint32_t)h[7] << 16));
    }
  }
}

template <int P>
__global__ void unpack_kernel(PackParams p) {
  const long long W = (long long)p.nrhs * p.Ls;
  const long long n = 2 * p.g.vh * W;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int col = (int)(i % W);
  const long long x_cb = (i / W) % p.g.vh;
  const int parity = (int)(i / (W * p.g.vh));
  const int r = col / p.Ls, s = col % p.Ls;
  int c[4];
  cb_coords(p.g, x_cb, parity, c);
  double v[24];
  if constexpr (P == F64) {
    const double2* d = (const double2*)p.data[parity];
#pragma unroll
    for (int k = 0; k < 12; k++) { double2 q = d[(x_cb * 12 + k) * W + col]; v[2 * k] = q.x; v[2 * k + 1] = q.y; }
  } else if constexpr (P == F32) {
    const float4* d = (const float4*)p.data[parity];
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 q = d[(x_cb * 6 + k) * W + col];
      v[4 * k] = q.x; v[4 * k + 1] = q.y; v[4 * k + 2] = q.z; v[4 * k + 3] = q.w;
    }
  } else {
    const uint4* d = (const uint4*)p.data[parity];
    double nrm = 1.0;
    if constexpr (P == F16) nrm = (double)p.norm[parity][x_cb * W + col];
    if constexpr (P == I16) nrm = (double)p.norm[parity][x_cb * W + col] / 32767.0;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      uint4 q = d[(x_cb * 3 + k) * W + col];
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 8; j++) {
        uint16_t b = (uint16_t)(w[j >> 1] >> (16 * (j & 1)));
        if constexpr (P == F16) v[8 * k + j] = (double)__half2float(*(__half*)&b) * nrm;
        else if constexpr (P == I16) v[8 * k + j] = (double)(int16_t)b * nrm;
        else v[8 * k + j] = (double)__bfloat162float(*(__nv_bfloat16*)&b);
      }
    }
  }
  const long long V = 2 * p.g.vh;
  double2* dst = (double2*)p.user_out + (((long long)r * p.Ls + s) * V + full_index(p.g, c)) * 12;
#pragma unroll
  for (int sp = 0; sp < 4; sp++)
#pragma unroll
    for (int co = 0; co < 3; co++)
      dst[sp * 3 + co] = make_double2(v[2 * (co * 4 + sp)], v[2 * (co * 4 + sp) + 1]);
}

template <typename K>
static cudaError_t go1d(K kern, long long n, const PackParams& p, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int T = 128;
  kern<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_pack(int prec, const PackParams& p, cudaStream_t st) {
  const long long n = 2 * p.g.vh * p.nrhs * p.Ls;
  switch (prec) {
    case F64: return go1d(pack_kernel<F64>, n, p, st);
    case F32: return go1d(pack_kernel<F32>, n, p, st);
    case F16: return go1d(pack_kernel<F16>, n, p, st);
    case BF16: return go1d(pack_kernel<BF16>, n, p, st);
    case I16: return go1d(pack_kernel<I16>, n, p, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_unpack(int prec, const PackParams& p, cudaStream_t st) {
  const long long n = 2 * p.g.vh * p.nrhs * p.Ls;
  switch (prec) {
    case F64: return go1d(unpack_kernel<F64>, n, p, st);
    case F32: return go1d(unpack_kernel<F32>, n, p, st);
    case F16: return go1d(unpack_kernel<F16>, n, p, st);
    case BF16: return go1d(unpack_kernel<BF16>, n, p, st);
    case I16: return go1d(unpack_kernel<I16>, n, p, st);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- gauge
__device__ __forceinline__ void atomic_max_pos(double* a, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax((unsigned long long*)a, (unsigned long long)__double_as_longlong(v));
}

// thread per (parity, x_cb, dir)
__global__ void gauge_load_kernel(GaugeParams p) {
  const long long n = 2 * p.g.vh * 8;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int dir = (int)(i % 8);
  const long long x_cb = (i / 8) % p.g.vh;
  const int parity = (int)(i / (8 * p.g.vh));
  const int mu = dir & 3;
  int c[4];
  cb_coords(p.g, x_cb, parity, c);
  int s[4] = {c[0], c[1], c[2], c[3]};
  double sign = 1.0;
  if (dir >= 4) {  // U_mu(x - mu)^+
    const int L = mu == 0 ? p.g.X : mu == 1 ? p.g.Y : mu == 2 ? p.g.Z : p.g.T;
    // with a ghost timeslice t - 1 = -1 is that slice (no wrap)
    s[mu] = (mu == 3 && p.ghost) ? s[mu] - 1 : (s[mu] - 1 + L) % L;
    if (mu == 3 && c[3] == 0 && p.bc_lo) sign = p.t_bc;
  } else if (mu == 3 && c[3] == p.g.T - 1 && p.bc_hi) {
    sign = p.t_bc;
  }
  if (p.ghost) s[3] += 1;   // user array index: the ghost slice comes first
  const double2* u = (const double2*)p.user + (full_index(p.g, s) * 4 + mu) * 9;
  double2 m[9];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int b = 0; b < 3; b++) {
      double2 z = u[a * 3 + b];
      if (dir >= 4) m[b * 3 + a] = make_double2(z.x, -z.y);  // dagger
      else m[a * 3 + b] = z;
    }
  double* out = p.out64[parity] + (x_cb * 8 + dir) * p.gs;
  const int nreal = p.gs;  // 18 or 12
  for (int k = 0; k < nreal / 2; k++) { out[2 * k] = sign * m[k].x; out[2 * k + 1] = sign * m[k].y; }
  if (p.err) {
    // |U U^+ - 1|_max and |det U - 1| of the unsigned link
    double e = 0.0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) {
        double re = 0.0, im = 0.0;
        for (int k = 0; k < 3; k++) {
          const double2 x = m[a * 3 + k], y = m[b * 3 + k];
          re += x.x * y.x + x.y * y.y;
          im += x.y * y.x - x.x * y.y;
        }
        e = fmax(e, fabs(re - (a == b ? 1.0 : 0.0)));
        e = fmax(e, fabs(im));
      }
    // det via cofactor expansion on row 0
    auto cm = [](double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); };
    double2 d = make_double2(0, 0);
    for (int k = 0; k < 3; k++) {
      const int i1 = (k + 1) % 3, i2 = (k + 2) % 3;
      double2 t1 = cm(m[3 + i1], m[6 + i2]), t2 = cm(m[3 + i2], m[6 + i1]);
      double2 cof = make_double2(t1.x - t2.x, t1.y - t2.y);
      double2 pr = cm(m[k], cof);
      d.x += pr.x; d.y += pr.y;
    }
    e = fmax(e, fabs(d.x - 1.0) + fabs(d.y));
    if (!(e == e)) e = 1e300;
    atomic_max_pos(p.err, e);
  }
}

cudaError_t launch_gauge_load(const GaugeParams& p, cudaStream_t st) {
  const long long n = 2 * p.g.vh * 8;
  gauge_load_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename G>
__global__ void gauge_convert_kernel(const double* in, G* out, long long nlinks, int gs_in, int gs_out, int nreal) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nlinks) return;
  for (int k = 0; k < gs_out; k++) {
    const double v = k < nreal ? in[i * gs_in + k] : 0.0;
    if constexpr (sizeof(G) == 8) out[i * gs_out + k] = v;
    else if constexpr (sizeof(G) == 4) out[i * gs_out + k] = (float)v;
    else if constexpr (std::is_same<G, int16_t>::value) out[i * gs_out + k] = (int16_t)__double2int_rn(32767.0 * v);
    else out[i * gs_out + k] = G(v);
  }
}

cudaError_t launch_gauge_convert(int prec, const double* in64, void* out, long long nlinks, int gs_in,
                                 int gs_out, int nreal, cudaStream_t st) {
  const unsigned b = (unsigned)((nlinks + 127) / 128);
  switch (prec) {
    case F64: gauge_convert_kernel<double><<<b, 128, 0, st>>>(in64, (double*)out, nlinks, gs_in, gs_out, nreal); break;
    case F32: gauge_convert_kernel<float><<<b, 128, 0, st>>>(in64, (float*)out, nlinks, gs_in, gs_out, nreal); break;
    case F16: gauge_convert_kernel<__half><<<b, 128, 0, st>>>(in64, (__half*)out, nlinks, gs_in, gs_out, nreal); break;
    case BF16: gauge_convert_kernel<__nv_bfloat16><<<b, 128, 0, st>>>(in64, (__nv_bfloat16*)out, nlinks, gs_in, gs_out, nreal); break;
    case I16: gauge_convert_kernel<int16_t><<<b, 128, 0, st>>>(in64, (int16_t*)out, nlinks, gs_in, gs_out, nreal); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- sources
// thread per (rhs, 4D site, spin-colour component)
__global__ void embed_wall_kernel(SrcParams p) {
  const long long V = 2 * p.g.vh;
  const long long n = (long long)p.nrhs * V * 12;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = (int)(i % 12);
  const long long x = (i / 12) % V;
  const int r = (int)(i / (12 * V));
  const int spin = k / 3;
  const double2 b = ((const double2*)p.in)[((long long)r * V + x) * 12 + k];
  double2* out = (double2*)p.out;
  for (int s = 0; s < p.Ls; s++) {
    // (P b_wall)_s: P_- b at s = 0, P_+ b at s = Ls-1
    const bool on = (spin < 2 && s == 0) || (spin >= 2 && s == p.Ls - 1);
    out[(((long long)r * p.Ls + s) * V + x) * 12 + k] = on ? b : make_double2(0.0, 0.0);
  }
}

__global__ void project4d_kernel(SrcParams p) {
  const long long V = 2 * p.g.vh;
  const long long n = (long long)p.nrhs * V * 12;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = (int)(i % 12);
  const long long x = (i / 12) % V;
  const int r = (int)(i / (12 * V));
  const int s = (k / 3) < 2 ? 0 : p.Ls - 1;   // q = P_- y_0 + P_+ y_{Ls-1}
  ((double2*)p.out)[((long long)r * V + x) * 12 + k] =
      ((const double2*)p.in)[(((long long)r * p.Ls + s) * V + x) * 12 + k];
}

// gamma_3 gamma_5 psi = (i psi_2, -i psi_3, i psi_0, -i psi_1) in the chiral basis
__global__ void fh_source_kernel(SrcParams p) {
  const long long V = 2 * p.g.vh;
  const long long n = (long long)p.nrhs * V * 12;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = (int)(i % 12);
  const long long base = i - k;
  const int spin = k / 3, co = k % 3;
  const int src_spin = (spin + 2) & 3;
  const double sg = (spin == 0 || spin == 2) ? 1.0 : -1.0;
  const double2 z = ((const double2*)p.in)[base + src_spin * 3 + co];
  ((double2*)p.out)[i] = make_double2(-sg * z.y, sg * z.x);  // sg * i * z
}

template <typename K>
static cudaError_t go_src(K kern, const SrcParams& p, cudaStream_t st) {
  const long long n = (long long)p.nrhs * 2 * p.g.vh * 12;
  if (n <= 0) return cudaSuccess;
  kern<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(p);
  return cudaGetLastError();
}
cudaError_t launch_embed_wall(const SrcParams& p, cudaStream_t st) { return go_src(embed_wall_kernel, p, st); }
cudaError_t launch_project4d(const SrcParams& p, cudaStream_t st) { return go_src(project4d_kernel, p, st); }
cudaError_t launch_fh_source(const SrcParams& p, cudaStream_t st) { return go_src(fh_source_kernel, p, st); }

// ---------------------------------------------------------------- nucleon 2-pt
// G_{g g'} = eps_abc eps_a'b'c' [ U1^{aa'}_{al al'} Dt^{bb'}_{al al'} U2^{cc'}_{g g'}
//                               - U1^{ac'}_{al g'} Dt^{bb'}_{al al'} U2^{ca'}_{g al'} ]
// Dt^{bb'} = CG5 D^{bb'} CG5bar, C(t) = sum_x Tr[P G(x)].  The 4x4 spin matrices CG5,
// CG5bar and P are built on the host from the library's gamma basis.
// Propagators are 12 columns [src_spin*3 + src_colour][t][z][y][x][spin][colour].
struct Cz { double re, im; };
__device__ __forceinline__ Cz cmul(Cz a, Cz b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ void cacc(Cz& a, Cz b) { a.re += b.re; a.im += b.im; }

__device__ __forceinline__ Cz prop(const double* S, long long V, long long x, int si, int ci, int sj, int cj) {
  const double2 z = __ldg((const double2*)S + ((long long)(sj * 3 + cj) * V + x) * 12 + si * 3 + ci);
  return {z.x, z.y};
}

__global__ void nucleon_site_kernel(Geom g, NucMats m, const double* u1, const double* dq, const double* u2,
                                    double* site) {
  const long long V = 2 * g.vh;
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= V) return;
  Cz tot = {0.0, 0.0};
  for (int b = 0; b < 3; b++)
    for (int bp = 0; bp < 3; bp++) {
      // Dt = CG5 D^{b b'} CG5bar
      Cz t1m[4][4], dt[4][4];
      for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
          Cz acc = {0, 0};
          for (int k = 0; k < 4; k++) cacc(acc, cmul(prop(dq, V, x, i, b, k, bp), Cz{m.cbr[k * 4 + j], m.cbi[k * 4 + j]}));
          t1m[i][j] = acc;
        }
      for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
          Cz acc = {0, 0};
          for (int k = 0; k < 4; k++) cacc(acc, cmul(Cz{m.car[i * 4 + k], m.cai[i * 4 + k]}, t1m[k][j]));
          dt[i][j] = acc;
        }
      // (a, c) and (a', c') run over the two orderings of the colours other than b, b'
      const int o1 = (b + 1) % 3, o2 = (b + 2) % 3, q1 = (bp + 1) % 3, q2 = (bp + 2) % 3;
      for (int pa = 0; pa < 2; pa++)
        for (int pq = 0; pq < 2; pq++) {
          const int a = pa ? o2 : o1, c = pa ? o1 : o2;   // eps_{a b c} = +1 for (b+1, b, b+2)?
          const int ap = pq ? q2 : q1, cp = pq ? q1 : q2;
          // eps_abc with (a,b,c): +1 for cyclic order of (0,1,2)
          const double ea = ((a - b + 3) % 3 == 2) ? 1.0 : -1.0;   // (b, c, a) cyclic <=> a = b + 2
          const double eb = ((ap - bp + 3) % 3 == 2) ? 1.0 : -1.0;
          const double es = ea * eb;
          // term 1
          Cz s1 = {0, 0}, tr2 = {0, 0};
          for (int i = 0; i < 4; i++)
            for (int j = 0; j < 4; j++) {
              cacc(s1, cmul(prop(u1, V, x, i, a, j, ap), dt[i][j]));
              cacc(tr2, cmul(Cz{m.pr[j * 4 + i], m.pi[j * 4 + i]}, prop(u2, V, x, i, c, j, cp)));
            }
          const Cz t1 = cmul(s1, tr2);
          // term 2: A_{al g} = sum_al' Dt_{al al'} U2^{ca'}_{g al'} ; B_{g' g} = sum_al U1^{ac'}_{al g'} A_{al g}
          Cz A[4][4];
          for (int i = 0; i < 4; i++)
            for (int gg = 0; gg < 4; gg++) {
              Cz acc = {0, 0};
              for (int j = 0; j < 4; j++) cacc(acc, cmul(dt[i][j], prop(u2, V, x, gg, c, j, ap)));
              A[i][gg] = acc;
            }
          Cz t2 = {0, 0};
          for (int gp = 0; gp < 4; gp++)
            for (int gg = 0; gg < 4; gg++) {
              const Cz pw = {m.pr[gp * 4 + gg], m.pi[gp * 4 + gg]};
              if (pw.re == 0.0 && pw.im == 0.0) continue;
              Cz bsum = {0, 0};
              for (int i = 0; i < 4; i++) cacc(bsum, cmul(prop(u1, V, x, i, a, gp, cp), A[i][gg]));
              cacc(t2, cmul(pw, bsum));
            }
          tot.re += es * (t1.re - t2.re);
          tot.im += es * (t1.im - t2.im);
        }
    }
  site[2 * x] = tot.re;
  site[2 * x + 1] = tot.im;
}

// one block per timeslice, fixed-order sums
__global__ void timeslice_sum_kernel(Geom g, const double* site, double* corr) {
  const long long V3 = (long long)g.X * g.Y * g.Z;
  const int t = blockIdx.x;
  __shared__ double sr[256], si[256];
  double ar = 0.0, ai = 0.0;
  for (long long i = threadIdx.x; i < V3; i += blockDim.x) {
    ar += site[2 * (t * V3 + i)];
    ai += site[2 * (t * V3 + i) + 1];
  }
  sr[threadIdx.x] = ar; si[threadIdx.x] = ai;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) { sr[threadIdx.x] += sr[threadIdx.x + w]; si[threadIdx.x] += si[threadIdx.x + w]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { corr[2 * t] = sr[0]; corr[2 * t + 1] = si[0]; }
}

cudaError_t launch_nucleon(const Geom& g, const NucMats& m, const double* u1, const double* d,
                           const double* u2, double* site_tmp, double* corr, cudaStream_t st) {
  const long long V = 2 * g.vh;
  nucleon_site_kernel<<<(unsigned)((V + 127) / 128), 128, 0, st>>>(g, m, u1, d, u2, site_tmp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  timeslice_sum_kernel<<<g.T, 256, 0, st>>>(g, site_tmp, corr);
  return cudaGetLastError();
}

}  // namespace mdwf
