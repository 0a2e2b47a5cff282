// Double-float ("double-single") arithmetic and storage.
//
// A real x is kept as an unevaluated sum hi + lo of two FP32 numbers.  Sums and
// products use the error-free transformations
//   TwoSum(a, b):  s = fl(a + b), e = (a + b) - s exactly   (Knuth, six adds)
//   TwoProd(a, b): p = fl(a * b), e = a * b - p exactly     (one FMA)
// and a dot product accumulates its products as Dot2 does (Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005)):
// the high parts are summed with TwoSum, every rounding error of a sum or a
// product, and the cross terms hi*lo + lo*hi, go into a running FP32 low part.
// Intermediate pairs are not renormalised (the low part may exceed half an ulp
// of the high part, which costs nothing in accuracy); a pair is renormalised
// with TwoSum when it is stored.  Accuracy: about 2^-48 relative to the
// magnitudes of the summed terms, from FP32 instructions only.  The explicit
// __fadd_rn / __fmul_rn / __fmaf_rn intrinsics keep the compiler from merging
// or reassociating the error-free steps.
//
// Storage of a complex number: one float4 (re.hi, re.lo, im.hi, im.lo).
//   spinor vector: element [rhs][comp][s*Vh + cb], 12 float4 per site
//   link field:    element [parity][mu][comp][cb], 9 float4 per link
#pragma once
#include "common.cuh"

namespace qcd {

constexpr int PDF = 3;  // precision tag of double-float storage (qcd_prec QCD_DF64)

struct F2 {
  float h, l;
};

struct DCx {
  F2 re, im;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
  return {s, e};
}

// a + b with the high parts summed exactly and the low parts added
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  F2 t = two_sum(a.h, b.h);
  return {t.h, __fadd_rn(t.l, __fadd_rn(a.l, b.l))};
}

__device__ __forceinline__ F2 df_neg(F2 a) { return {-a.h, -a.l}; }

// renormalised pair: |lo| <= ulp(hi) / 2
__device__ __forceinline__ F2 df_norm(F2 a) { return two_sum(a.h, a.l); }

// running dot product (s, l)
struct Dot {
  float s, l;
};

// acc = a * b
__device__ __forceinline__ Dot dot_first(F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return {p, e};
}

// acc += a * b
__device__ __forceinline__ void dot_add(Dot& acc, F2 a, F2 b) {
  const float p = __fmul_rn(a.h, b.h);
  const float pe = __fmaf_rn(a.h, b.h, -p);
  const F2 t = two_sum(acc.s, p);
  float l = __fmaf_rn(a.h, b.l, acc.l);
  l = __fmaf_rn(a.l, b.h, l);
  acc.l = __fadd_rn(l, __fadd_rn(pe, t.l));
  acc.s = t.h;
}

__device__ __forceinline__ F2 dot_value(const Dot& d) { return {d.s, d.l}; }

// ----------------------------------------------------------------------------- complex
__device__ __forceinline__ DCx dcx_add(const DCx& a, const DCx& b) {
  return {df_add(a.re, b.re), df_add(a.im, b.im)};
}
__device__ __forceinline__ DCx dcx_neg(const DCx& a) { return {df_neg(a.re), df_neg(a.im)}; }
__device__ __forceinline__ DCx dcx_mul_i(const DCx& a) { return {df_neg(a.im), a.re}; }
__device__ __forceinline__ DCx dcx_mul_mi(const DCx& a) { return {a.im, df_neg(a.re)}; }

// ----------------------------------------------------------------------------- conversions
// FP64 <-> double-float by integer operations on the IEEE bit patterns (a
// conversion through GB300's FP64 pipe, at 1/58 of the FP32 rate, costs three
// or four FP64 operations per real).  For 2^-100 <= |x| < 2^100:
//   hi = x rounded to 24 significant bits (mantissa rounded half up),
//   lo = fl32(x - hi), with x - hi formed exactly as an integer count of
//        units in the last place of x (|x - hi| <= 2^28 units);
// |x - (hi + lo)| <= 2^-48 |x|.  Zeros map to zeros; other values (tiny,
// huge, non-finite) take the FP64 conversions.
__device__ __forceinline__ F2 df_from_double(double x) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const unsigned long long mag = bits & 0x7fffffffffffffffull;
  const unsigned e = (unsigned)(mag >> 52);
  if (mag == 0) return {0.f, 0.f};
  if (e < 923u || e > 1122u) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};  // x - h is exact in FP64
  }
  const unsigned long long hm = (mag + (1ull << 28)) & ~((1ull << 29) - 1);
  const unsigned eh = (unsigned)(hm >> 52);  // e, or e + 1 after a carry out of the mantissa
  float hi = __uint_as_float(((eh - 896u) << 23) | (unsigned)((hm >> 29) & 0x7fffffull));
  const int r = (int)((long long)mag - (long long)hm);  // x - hi in units of 2^(e - 1075)
  // r * 2^(e - 1075) = (r * 2^(e - 1027)) * 2^-48, both factors normal FP32 numbers
  const float up = __uint_as_float((e - 900u) << 23);
  float lo = __fmul_rn(__fmul_rn(__int2float_rn(r), up), 3.5527136788005009e-15f);
  if (bits >> 63) {
    hi = -hi;
    lo = -lo;
  }
  return {hi, lo};
}

// FP32 -> FP64, exact, by bit manipulation for normal numbers and zero
__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0u && (u & 0x7fffffffu) == 0u) return 0.0;
  if (ef == 0u || ef == 255u) return (double)f;
  const unsigned long long d = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(ef + 896u) << 52) |
                               ((unsigned long long)(u & 0x7fffffu) << 29);
  return __longlong_as_double((long long)d);
}

__device__ __forceinline__ double df_to_double(F2 a) { return f32_to_f64(a.h) + f32_to_f64(a.l); }

__device__ __forceinline__ DCx dcx_load(const float4* p) {
  const float4 d = __ldg(p);
  return {{d.x, d.y}, {d.z, d.w}};
}
__device__ __forceinline__ float4 dcx_pack(const DCx& v) {
  return make_float4(v.re.h, v.re.l, v.im.h, v.im.l);
}

// ----------------------------------------------------------------------------- views
// Spinor view in the interface of the other precisions (load / store as
// double, for the pack / unpack kernels) plus raw double-float access.
template <>
struct SpinorView<PDF> {
  using R = double;
  float4* __restrict__ p;
  float* norm;  // unused
  long stride;
  __device__ __forceinline__ void load(long site, Cx<R> v[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float4 d = __ldg(p + k * stride + site);
      v[k] = {df_to_double({d.x, d.y}), df_to_double({d.z, d.w})};
    }
  }
  __device__ __forceinline__ void store(long site, const Cx<R> v[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const F2 a = df_from_double(v[k].re), b = df_from_double(v[k].im);
      p[k * stride + site] = make_float4(a.h, a.l, b.h, b.l);
    }
  }
  __device__ __forceinline__ void load_df(long site, DCx v[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = dcx_load(p + k * stride + site);
  }
  __device__ __forceinline__ void store_df(long site, const DCx v[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * stride + site] = dcx_pack(v[k]);
  }
  __device__ __forceinline__ SpinorView offset_rhs(int r) const {
    SpinorView o = *this;
    o.p += (long)r * 12 * stride;
    return o;
  }
};

struct LinkViewDF {
  const float4* __restrict__ p;
  long Vh;
  __device__ __forceinline__ void load(int parity, int mu, long cb, DCx u[9]) const {
    const float4* q = p + (long)(parity * 4 + mu) * 9 * Vh + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = dcx_load(q + k * Vh);
  }
};

}  // namespace qcd
