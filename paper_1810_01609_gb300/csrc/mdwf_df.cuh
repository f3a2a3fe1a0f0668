// Double-float arithmetic for the emulated-FP64 hop: a real as the unevaluated sum hi + lo
// of two floats (Dekker's double-length representation, 1971), added with Knuth's TwoSum
// (TAOCP vol. 2, 4.2.2: s + e = a + b exactly) and multiplied with the FMA-based exact
// product (p + e = a b exactly); a sum of products is accumulated as in Ogita, Rump and
// Oishi's Dot2 (SIAM J. Sci. Comput. 26, 2005): the leading parts through TwoSum, every
// error term in a second float.  About 47 significant bits, on the FP32 pipe: GB300 runs
// FP64 at 1/64 of the FP32 rate, so the hop's SU(3) products cost several times less
// this way than in native FP64.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace mdwf {

struct dfl { float hi, lo; };   // hi + lo
struct dacc { float s, e; };    // running sum s with its accumulated error e

// A double as hi + lo by bit manipulation (no FP64 instruction): hi = x truncated to 24
// significant bits, lo = the rest truncated to 23 bits (|x - hi - lo| < 2^-46 |x|).
// |x| < 2^-126 gives +-0 (an absolute error below 1.2e-38); |x| >= 2^127, Inf and NaN give
// NaN, so that they still show up in the norms the solver checks.
__device__ __forceinline__ dfl split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int e = (int)((hw >> 20) & 0x7FFu);
  const unsigned sgn = hw & 0x80000000u;
  const unsigned top = ((hw & 0xFFFFFu) << 3) | (lw >> 29);
  dfl r;
  r.hi = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | top);
  // the low 29 mantissa bits: their top 23 as an exact float (2^23 + k - 2^23), times
  // 2^(e - 1069), the weight of bit 6 of the double's mantissa
  const float k = __fsub_rn(__uint_as_float(0x4B000000u | ((lw & 0x1FFFFFFFu) >> 6)), 8388608.0f);
  r.lo = __uint_as_float(__float_as_uint(__fmul_rn(k, __uint_as_float((unsigned)(e - 942) << 23))) ^ sgn);
  if (e < 943) r.lo = 0.0f;
  if (e < 897) r.hi = __uint_as_float(sgn);
  if (e > 1150) { r.hi = __uint_as_float(0x7FC00000u); r.lo = 0.0f; }
  return r;
}

__device__ __forceinline__ double dfl_to_f64(float hi, float lo) { return (double)hi + (double)lo; }

// s + e = a + b exactly (Knuth's TwoSum, no magnitude ordering needed)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a + S b (S = +-1)
template <int S>
__device__ __forceinline__ dfl dadd(dfl a, dfl b) {
  const float bh = S > 0 ? b.hi : -b.hi, bl = S > 0 ? b.lo : -b.lo;
  float s, e;
  two_sum(a.hi, bh, s, e);
  return {s, __fadd_rn(__fadd_rn(a.lo, bl), e)};
}

// acc = S x y (first term of a sum)
template <int S>
__device__ __forceinline__ dacc dprod(dfl x, dfl y) {
  const float xh = S > 0 ? x.hi : -x.hi, xl = S > 0 ? x.lo : -x.lo;
  const float p = __fmul_rn(xh, y.hi);
  const float pe = __fmaf_rn(xh, y.hi, -p);
  return {p, __fadd_rn(pe, __fmaf_rn(xh, y.lo, __fmul_rn(xl, y.hi)))};
}

// acc += S x y
template <int S>
__device__ __forceinline__ void dfma(dacc& a, dfl x, dfl y) {
  const float xh = S > 0 ? x.hi : -x.hi, xl = S > 0 ? x.lo : -x.lo;
  const float p = __fmul_rn(xh, y.hi);
  const float pe = __fmaf_rn(xh, y.hi, -p);
  const float c = __fmaf_rn(xh, y.lo, __fmul_rn(xl, y.hi));
  float s, se;
  two_sum(a.s, p, s, se);
  a.s = s;
  a.e = __fadd_rn(a.e, __fadd_rn(se, __fadd_rn(pe, c)));
}

// acc += S u
template <int S>
__device__ __forceinline__ void dacc_add(dacc& a, const dacc& u) {
  const float us = S > 0 ? u.s : -u.s, ue = S > 0 ? u.e : -u.e;
  float s, se;
  two_sum(a.s, us, s, se);
  a.s = s;
  a.e = __fadd_rn(a.e, __fadd_rn(se, ue));
}

}  // namespace mdwf
