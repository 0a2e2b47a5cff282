// Device-side building blocks shared by the kernels of libqcd: complex
// arithmetic, the even-odd (checkerboard) site geometry, and typed views of
// the internal structure-of-arrays storage of spinors and links.
//
// Internal storage (private to the library):
//   spinor vector (one parity, `nrhs` right-hand sides, `ls` fifth-dimension
//   slices): component-major SoA, element [rhs][comp][s*Vh + cb]; a site holds
//   4 spins x 3 colours complex = 24 reals, stored as
//     F64: 12 x double2 (one complex each)
//     F32:  6 x float4  (two complex each)
//     F16:  3 x uint4   (eight binary16 each) plus one float scale per site
//   link field: element [parity][mu][comp][cb], U_mu(x) for x of that parity
//     F64: 9 x double2 (18 reals); F32: 9 x float2 (18) or 3 x float4 (12);
//     F16: 9 x half2 (18) or 3 x uint2 (12).  With 12 reals only rows 0,1 of
//     the SU(3) matrix are kept; row 2 = conj(row0 x row1).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace qcd {

// ----------------------------------------------------------------------------- launch order
// Programmatic dependent launch (sm_90 and later): a kernel launched with the
// programmatic-serialization attribute (launch_k in internal.h) may be scheduled
// while its predecessor in the stream finishes.  pdl_enter(), the first statement
// of such a kernel, waits until the predecessor grid has completed and its memory
// operations are visible, then allows the next kernel to begin launching.  Without
// a programmatic predecessor both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// ----------------------------------------------------------------------------- complex
template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cx(R a, R b) {
  return Cx<R>{a, b};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator+(Cx<R> a, Cx<R> b) {
  return {a.re + b.re, a.im + b.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a, Cx<R> b) {
  return {a.re - b.re, a.im - b.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator-(Cx<R> a) {
  return {-a.re, -a.im};
}
template <typename R>
__device__ __forceinline__ Cx<R> operator*(R s, Cx<R> a) {
  return {s * a.re, s * a.im};
}
// multiply by +i / -i
template <typename R>
__device__ __forceinline__ Cx<R> mul_i(Cx<R> a) {
  return {-a.im, a.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> mul_mi(Cx<R> a) {
  return {a.im, -a.re};
}
// acc + a*b
template <typename R>
__device__ __forceinline__ Cx<R> cmadd(Cx<R> a, Cx<R> b, Cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
  return acc;
}
// acc + conj(a)*b
template <typename R>
__device__ __forceinline__ Cx<R> cjmadd(Cx<R> a, Cx<R> b, Cx<R> acc) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
  return acc;
}
template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R>
__device__ __forceinline__ Cx<R> conjg(Cx<R> a) {
  return {a.re, -a.im};
}

// ----------------------------------------------------------------------------- division
// n / d for 0 <= n < 2^31 by a multiply-high and a shift (Granlund & Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, Thm 4.2 with
// N = 31): l = ceil(log2 d), m = ceil(2^(31+l) / d) < 2^32, n / d = (n m) >> (31 + l).
// d = 1 is flagged by s = -1.  Replaces the ~20-instruction runtime division in
// the index arithmetic of the stencils.
struct FastDiv {
  unsigned m;
  int s;  // l - 1
};

inline FastDiv make_fastdiv(unsigned d) {
  if (d <= 1) return {0u, -1};
  int l = 0;
  while ((1ull << l) < d) ++l;
  const unsigned long long m = ((1ull << (31 + l)) + d - 1) / d;
  return {(unsigned)m, l - 1};
}

__device__ __forceinline__ int fdiv(int n, FastDiv f) {
  return f.s < 0 ? n : (int)(__umulhi((unsigned)n, f.m) >> f.s);
}

// ----------------------------------------------------------------------------- geometry
// Lattice extents, boundary factors and the even-odd map.  Canonical site
// index i = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) & 1; within a parity
// the checkerboard index is cb = i >> 1 (Lx even).
struct Geom {
  int L[4];
  int apbc[4];  // 1 where the boundary factor is -1
  int V, Vh;
  FastDiv dL[3];  // division by L[0], L[1], L[2]
};

inline Geom make_geom(const int L[4], const int bc[4], long V, long Vh) {
  Geom g;
  for (int m = 0; m < 4; ++m) {
    g.L[m] = L[m];
    g.apbc[m] = bc[m] < 0;
  }
  g.V = (int)V;
  g.Vh = (int)Vh;
  for (int m = 0; m < 3; ++m) g.dL[m] = make_fastdiv((unsigned)L[m]);
  return g;
}

struct SiteCoords {
  int x[4];
  int i;  // canonical index
};

__device__ __forceinline__ SiteCoords cb_to_site(const Geom& g, int cb, int parity) {
  SiteCoords c;
  int i2 = 2 * cb;
  int r = fdiv(i2, g.dL[0]);
  int x0 = i2 - r * g.L[0];
  int r2 = fdiv(r, g.dL[1]);
  c.x[1] = r - r2 * g.L[1];
  c.x[3] = fdiv(r2, g.dL[2]);
  c.x[2] = r2 - c.x[3] * g.L[2];
  c.x[0] = x0 + ((parity + c.x[1] + c.x[2] + c.x[3]) & 1);
  c.i = c.x[0] + g.L[0] * (c.x[1] + g.L[1] * (c.x[2] + g.L[2] * c.x[3]));
  return c;
}

// canonical index of the neighbour x +- mu_hat; *wrap = 1 if the step crosses
// the lattice boundary.
__device__ __forceinline__ int neighbour_index(const Geom& g, const SiteCoords& c, int mu, int dir,
                                               int* wrap) {
  int stride = 1;
#pragma unroll
  for (int m = 0; m < 4; ++m)
    if (m < mu) stride *= g.L[m];
  int xm = c.x[mu];
  if (dir > 0) {
    *wrap = (xm == g.L[mu] - 1);
    return *wrap ? c.i - (g.L[mu] - 1) * stride : c.i + stride;
  } else {
    *wrap = (xm == 0);
    return *wrap ? c.i + (g.L[mu] - 1) * stride : c.i - stride;
  }
}

// ----------------------------------------------------------------------------- precision tags
enum Prec { P64 = 0, P32 = 1, P16 = 2 };

template <int P>
struct MathType {
  using type = float;
};
template <>
struct MathType<P64> {
  using type = double;
};

// ----------------------------------------------------------------------------- spinor views
// A view of one right-hand side / slice group of a spinor vector.  `stride` is
// the component stride (sites per component array = ls*Vh); `site` passed to
// load/store is s*Vh + cb.
template <int P>
struct SpinorView;

template <>
struct SpinorView<P64> {
  using R = double;
  double2* __restrict__ p;
  float* norm;  // unused
  long stride;
  __device__ __forceinline__ void load(long site, Cx<R> v[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      double2 d = __ldg(p + k * stride + site);
      v[k] = {d.x, d.y};
    }
  }
  __device__ __forceinline__ void store(long site, const Cx<R> v[12]) const {
#pragma unroll
    for (int k = 0; k < 12; ++k) p[k * stride + site] = make_double2(v[k].re, v[k].im);
  }
  __device__ __forceinline__ SpinorView offset_rhs(int r) const {
    SpinorView o = *this;
    o.p += (long)r * 12 * stride;
    return o;
  }
};

// FP32 and FP16 storage interleaves the two spins of each chiral half: spin
// pair q (q = 0, 1, 2: spins 0 and 1 of colour q; q = 3, 4, 5: spins 2 and 3 of
// colour q - 3) is one 16-byte unit (re_a, re_b, im_a, im_b).  load / store
// give the canonical order [spin * 3 + colour] (a renaming of registers);
// load_p / store_p give the pairs as two FP32 lanes, the operands of the packed
// FP32x2 arithmetic of the stencil.
struct P2 {
  float2 re, im;  // (spin a, spin b)
};

template <>
struct SpinorView<P32> {
  using R = float;
  float4* __restrict__ p;
  float* norm;  // unused
  long stride;
  __device__ __forceinline__ void load(long site, Cx<R> v[12]) const {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int b = q < 3 ? q : q + 3;  // canonical index of spin a
      float4 d = __ldg(p + q * stride + site);
      v[b] = {d.x, d.z};
      v[b + 3] = {d.y, d.w};
    }
  }
  __device__ __forceinline__ void store(long site, const Cx<R> v[12]) const {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int b = q < 3 ? q : q + 3;
      p[q * stride + site] = make_float4(v[b].re, v[b + 3].re, v[b].im, v[b + 3].im);
    }
  }
  __device__ __forceinline__ void load_p(long site, P2 w[6]) const {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      float4 d = __ldg(p + q * stride + site);
      w[q] = {make_float2(d.x, d.y), make_float2(d.z, d.w)};
    }
  }
  __device__ __forceinline__ void store_p(long site, const P2 w[6]) const {
#pragma unroll
    for (int q = 0; q < 6; ++q) p[q * stride + site] = make_float4(w[q].re.x, w[q].re.y, w[q].im.x, w[q].im.y);
  }
  // the pairs without their site scale (FP32 has none: *scale = 1)
  __device__ __forceinline__ void load_p_raw(long site, P2 w[6], float* scale) const {
    load_p(site, w);
    *scale = 1.f;
  }
  __device__ __forceinline__ SpinorView offset_rhs(int r) const {
    SpinorView o = *this;
    o.p += (long)r * 6 * stride;
    return o;
  }
};

// binary16 storage of psi/s with s = max |component| of the site (FP32),
// round-to-nearest-even on store; arithmetic is FP32.  uint4 k holds spin pairs
// q = 2k, 2k + 1 as half2 (re_a, re_b), half2 (im_a, im_b).
template <>
struct SpinorView<P16> {
  using R = float;
  uint4* __restrict__ p;
  float* __restrict__ norm;
  long stride;
  __device__ __forceinline__ void load(long site, Cx<R> v[12]) const {
    float s = __ldg(norm + site);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 d = __ldg(p + k * stride + site);
      const __half2* h = reinterpret_cast<const __half2*>(&d);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int q = 2 * k + j, b = q < 3 ? q : q + 3;
        const float2 re = __half22float2(h[2 * j]), im = __half22float2(h[2 * j + 1]);
        v[b] = {re.x * s, im.x * s};
        v[b + 3] = {re.y * s, im.y * s};
      }
    }
  }
  __device__ __forceinline__ void store(long site, const Cx<R> v[12]) const {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(v[k].re), fabsf(v[k].im)));
    float inv = (m > 0.f) ? 1.0f / m : 0.f;
    norm[site] = m;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 d;
      __half2* h = reinterpret_cast<__half2*>(&d);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int q = 2 * k + j, b = q < 3 ? q : q + 3;
        h[2 * j] = __floats2half2_rn(v[b].re * inv, v[b + 3].re * inv);
        h[2 * j + 1] = __floats2half2_rn(v[b].im * inv, v[b + 3].im * inv);
      }
      p[k * stride + site] = d;
    }
  }
  __device__ __forceinline__ void load_p(long site, P2 w[6]) const {
    const float s = __ldg(norm + site);
    const float2 s2 = make_float2(s, s);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 d = __ldg(p + k * stride + site);
      const __half2* h = reinterpret_cast<const __half2*>(&d);
#pragma unroll
      for (int j = 0; j < 2; ++j)
        w[2 * k + j] = {__fmul2_rn(__half22float2(h[2 * j]), s2), __fmul2_rn(__half22float2(h[2 * j + 1]), s2)};
    }
  }
  // the stored pairs psi/s and the site scale s (the caller applies s where it is cheapest)
  __device__ __forceinline__ void load_p_raw(long site, P2 w[6], float* scale) const {
    *scale = __ldg(norm + site);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 d = __ldg(p + k * stride + site);
      const __half2* h = reinterpret_cast<const __half2*>(&d);
#pragma unroll
      for (int j = 0; j < 2; ++j) w[2 * k + j] = {__half22float2(h[2 * j]), __half22float2(h[2 * j + 1])};
    }
  }
  __device__ __forceinline__ void store_p(long site, const P2 w[6]) const {
    P2 unused[6];
    store_p_rounded<false>(site, w, unused);
  }
  // the same, and with ROUNDED the values a later load returns (the stored halves
  // times the site scale) in wr
  template <bool ROUNDED>
  __device__ __forceinline__ void store_p_rounded(long site, const P2 w[6], P2 wr[6]) const {
    float m = 0.f;
#pragma unroll
    for (int q = 0; q < 6; ++q)
      m = fmaxf(m, fmaxf(fmaxf(fabsf(w[q].re.x), fabsf(w[q].re.y)), fmaxf(fabsf(w[q].im.x), fabsf(w[q].im.y))));
    float inv = (m > 0.f) ? 1.0f / m : 0.f;
    norm[site] = m;
    const float2 m2 = make_float2(m, m);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint4 d;
      __half2* h = reinterpret_cast<__half2*>(&d);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const P2& w2 = w[2 * k + j];
        h[2 * j] = __floats2half2_rn(w2.re.x * inv, w2.re.y * inv);
        h[2 * j + 1] = __floats2half2_rn(w2.im.x * inv, w2.im.y * inv);
        if constexpr (ROUNDED)
          wr[2 * k + j] = {__fmul2_rn(__half22float2(h[2 * j]), m2), __fmul2_rn(__half22float2(h[2 * j + 1]), m2)};
      }
      p[k * stride + site] = d;
    }
  }
  __device__ __forceinline__ SpinorView offset_rhs(int r) const {
    SpinorView o = *this;
    o.p += (long)r * 3 * stride;
    o.norm += (long)r * stride;
    return o;
  }
};

// ----------------------------------------------------------------------------- link views
template <int P, int RECON>
struct LinkView;

template <typename R>
__device__ __forceinline__ void reconstruct_row2(Cx<R> u[9]) {
  // row2 = conj(row0 x row1)
  u[6] = conjg(cmul(u[1], u[5]) - cmul(u[2], u[4]));
  u[7] = conjg(cmul(u[2], u[3]) - cmul(u[0], u[5]));
  u[8] = conjg(cmul(u[0], u[4]) - cmul(u[1], u[3]));
}

template <>
struct LinkView<P64, 18> {
  using R = double;
  const double2* __restrict__ p;
  long Vh;
  __device__ __forceinline__ void load(int parity, int mu, long cb, Cx<R> u[9]) const {
    const double2* q = p + (long)(parity * 4 + mu) * 9 * Vh + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      double2 d = __ldg(q + k * Vh);
      u[k] = {d.x, d.y};
    }
  }
};

template <>
struct LinkView<P32, 18> {
  using R = float;
  const float2* __restrict__ p;
  long Vh;
  __device__ __forceinline__ void load(int parity, int mu, long cb, Cx<R> u[9]) const {
    const float2* q = p + (long)(parity * 4 + mu) * 9 * Vh + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float2 d = __ldg(q + k * Vh);
      u[k] = {d.x, d.y};
    }
  }
};

template <>
struct LinkView<P32, 12> {
  using R = float;
  const float4* __restrict__ p;
  long Vh;
  __device__ __forceinline__ void load(int parity, int mu, long cb, Cx<R> u[9]) const {
    const float4* q = p + (long)(parity * 4 + mu) * 3 * Vh + cb;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float4 d = __ldg(q + k * Vh);
      u[2 * k] = {d.x, d.y};
      u[2 * k + 1] = {d.z, d.w};
    }
    reconstruct_row2(u);
  }
};

template <>
struct LinkView<P16, 18> {
  using R = float;
  const __half2* __restrict__ p;
  long Vh;
  __device__ __forceinline__ void load(int parity, int mu, long cb, Cx<R> u[9]) const {
    const __half2* q = p + (long)(parity * 4 + mu) * 9 * Vh + cb;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      float2 f = __half22float2(__ldg(q + k * Vh));
      u[k] = {f.x, f.y};
    }
  }
};

template <>
struct LinkView<P16, 12> {
  using R = float;
  const uint2* __restrict__ p;
  long Vh;
  __device__ __forceinline__ void load(int parity, int mu, long cb, Cx<R> u[9]) const {
    const uint2* q = p + (long)(parity * 4 + mu) * 3 * Vh + cb;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      uint2 d = __ldg(q + k * Vh);
      const __half2* h = reinterpret_cast<const __half2*>(&d);
      float2 f0 = __half22float2(h[0]), f1 = __half22float2(h[1]);
      u[2 * k] = {f0.x, f0.y};
      u[2 * k + 1] = {f1.x, f1.y};
    }
    reconstruct_row2(u);
  }
};

}  // namespace qcd

namespace qcd {

// ----------------------------------------------------------------------------- runtime-typed view
// A spinor vector whose storage precision is chosen at run time (BLAS and
// solver kernels mix precisions, e.g. an FP32 iterate added into an FP64 sum).
struct AnyView {
  int prec;  // 0 F64, 1 F32, 2 F16
  void* p;
  float* norm;
  long stride;  // sites per component array (ls * Vh)
};

template <typename R, int P>
__device__ __forceinline__ void any_load_p(const AnyView& v, int r, long site, Cx<R> out[12]) {
  SpinorView<P> s;
  s.p = (decltype(s.p))v.p;
  s.norm = v.norm;
  s.stride = v.stride;
  Cx<typename SpinorView<P>::R> t[12];
  s.offset_rhs(r).load(site, t);
#pragma unroll
  for (int k = 0; k < 12; ++k) out[k] = {(R)t[k].re, (R)t[k].im};
}

template <typename R, int P>
__device__ __forceinline__ void any_store_p(const AnyView& v, int r, long site, const Cx<R> in[12]) {
  SpinorView<P> s;
  s.p = (decltype(s.p))v.p;
  s.norm = v.norm;
  s.stride = v.stride;
  using T = typename SpinorView<P>::R;
  Cx<T> t[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) t[k] = {(T)in[k].re, (T)in[k].im};
  s.offset_rhs(r).store(site, t);
}

template <typename R>
__device__ __forceinline__ void any_load(const AnyView& v, int r, long site, Cx<R> out[12]) {
  if (v.prec == P64)
    any_load_p<R, P64>(v, r, site, out);
  else if (v.prec == P32)
    any_load_p<R, P32>(v, r, site, out);
  else
    any_load_p<R, P16>(v, r, site, out);
}

template <typename R>
__device__ __forceinline__ void any_store(const AnyView& v, int r, long site, const Cx<R> in[12]) {
  if (v.prec == P64)
    any_store_p<R, P64>(v, r, site, in);
  else if (v.prec == P32)
    any_store_p<R, P32>(v, r, site, in);
  else
    any_store_p<R, P16>(v, r, site, in);
}

// ----------------------------------------------------------------------------- block reduction
// Sum NR doubles over the block (warp shuffles, then shared memory); the
// result is valid in thread 0.  Deterministic for a fixed block size.
template <int NR>
__device__ __forceinline__ void block_sum(double v[NR]) {
  __shared__ double sh[32][NR];
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NR; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NR; ++k) sh[warp][k] = v[k];
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] = (lane < nw) ? sh[lane][k] : 0.0;
#pragma unroll
    for (int k = 0; k < NR; ++k)
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------- chiral basis
// gamma_mu = [[0, B_mu],[B_mu^dag, 0]] with B_x = -i sigma_1, B_y = -i sigma_2,
// B_z = -i sigma_3, B_t = 1 (upper spins 0,1; lower spins 2,3).
// (B l)_k for spin pair l = (l0, l1), colour c
template <int MU, typename R>
__device__ __forceinline__ void apply_B(const Cx<R> l0, const Cx<R> l1, Cx<R>& o0, Cx<R>& o1) {
  if (MU == 0) {  // -i sigma_1 = [[0,-i],[-i,0]]
    o0 = mul_mi(l1);
    o1 = mul_mi(l0);
  } else if (MU == 1) {  // -i sigma_2 = [[0,-1],[1,0]]
    o0 = -l1;
    o1 = l0;
  } else if (MU == 2) {  // -i sigma_3 = diag(-i, i)
    o0 = mul_mi(l0);
    o1 = mul_i(l1);
  } else {  // 1
    o0 = l0;
    o1 = l1;
  }
}

// (B^dag h)_k
template <int MU, typename R>
__device__ __forceinline__ void apply_Bdag(const Cx<R> h0, const Cx<R> h1, Cx<R>& o0, Cx<R>& o1) {
  if (MU == 0) {  // [[0,i],[i,0]]
    o0 = mul_i(h1);
    o1 = mul_i(h0);
  } else if (MU == 1) {  // [[0,1],[-1,0]]
    o0 = h1;
    o1 = -h0;
  } else if (MU == 2) {  // diag(i, -i)
    o0 = mul_i(h0);
    o1 = mul_mi(h1);
  } else {
    o0 = h0;
    o1 = h1;
  }
}

}  // namespace qcd
