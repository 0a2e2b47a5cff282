// Double-float (FP32 pair) Wilson hopping stencil and the vector operations on
// double-float fields.  These carry the outer steps of the mixed-precision
// solver (Sec. II C, last paragraph: the high-precision residual b - Mhat x
// and the preparation / reconstruction of the even-odd system) at about 48
// significant bits using only FP32 instructions; on GB300 an FP64 FMA costs
// as much issue time as 58 FP32 ones, so the IEEE-FP64 stencil is ALU-bound
// at 1.2 TFLOP/s while this one runs close to its memory traffic.
//
// The stencil computes the same sum as the FP32/FP64 one (Eq. (1) in hopping
// form, chiral-basis spin projection, 8 x (12 + 132) + 7 x 24 = 1320 real
// operations per output site), each operation replaced by its double-float
// counterpart (dfloat.cuh):
//   out(x) = [x1(x) + c2 x2(x)] + a * sum_mu [ (1 - gamma_mu) U_mu(x) in(x+mu)
//                                          + (1 + gamma_mu) U_mu(x-mu)^dag in(x-mu) ]
// (projectors exchanged for the adjoint).  The link-times-half-spinor
// products are Dot2 sums of six terms per output real.
#include <cstdio>
#include <string>
#include <vector>

#include "dfloat.cuh"
#include "internal.h"

namespace qcd {

namespace {

// ----------------------------------------------------------------------------- stencil
struct HopDfArgs {
  Geom g;
  int out_parity;
  int ls;
  FastDiv d_ls;
  int x1, x2;  // epilogue terms present
  F2 a, c2;
  LinkViewDF U;
  SpinorView<PDF> in, out, vx1, vx2;
  const int* stop;
};

// Spin structure of one hop direction, chosen at run time so that the eight
// directions share one copy of the code (the link multiplication dominates
// and is the same for all of them; a fully unrolled kernel is several times
// larger than the instruction cache and stalls on instruction fetch).
//
// Chiral basis: gamma_mu = [[0, B],[B^dag, 0]], B_x = -i sigma_1, B_y = -i sigma_2,
// B_z = -i sigma_3, B_t = 1.  Each B maps the lower spin pair l to
// (ph0 l_{p0}, ph1 l_{p1}) with phases ph in {+-1, +-i} and (p0, p1) = (1, 0) for x, y
// (off-diagonal) or (0, 1) for z, t.  With S = +-1 the projector sign and f the
// boundary factor of the hop:
//   h_s     = u_s + S ph_s l_{p_s}                       (s = 0, 1)
//   upper_s += f g_s,  lower_s += f S conj(ph_{p_s}) g_{p_s},  g = U h (U^dag for backward)
struct Phase {
  float r, i;  // r + i*i, one of them zero, the other +-1
};

__device__ __forceinline__ Phase conj_ph(Phase p) { return {p.r, -p.i}; }
__device__ __forceinline__ Phase scale_ph(Phase p, float s) { return {s * p.r, s * p.i}; }

// acc + p * x, p a phase (the products by 0 and +-1 are exact)
__device__ __forceinline__ DCx dcx_add_ph(const DCx& acc, Phase p, const DCx& x) {
  const F2 re = {__fmaf_rn(p.r, x.re.h, __fmul_rn(-p.i, x.im.h)), __fmaf_rn(p.r, x.re.l, __fmul_rn(-p.i, x.im.l))};
  const F2 im = {__fmaf_rn(p.r, x.im.h, __fmul_rn(p.i, x.re.h)), __fmaf_rn(p.r, x.im.l, __fmul_rn(p.i, x.re.l))};
  return {df_add(acc.re, re), df_add(acc.im, im)};
}

// acc + f * x, f = +-1
__device__ __forceinline__ DCx dcx_add_sign(const DCx& acc, float f, const DCx& x) {
  return {df_add(acc.re, {f * x.re.h, f * x.re.l}), df_add(acc.im, {f * x.im.h, f * x.im.l})};
}

// g = U h for both spins of h; every output real is a Dot2 sum of six products
__device__ __forceinline__ void link_mul_df(const DCx U[9], const DCx h[6], DCx g[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Dot re, im;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const DCx u = U[a * 3 + b];
        const DCx v = h[sp * 3 + b];
        // re += ur vr - ui vi,  im += ur vi + ui vr
        if (b == 0) {
          re = dot_first(u.re, v.re);
          im = dot_first(u.re, v.im);
        } else {
          dot_add(re, u.re, v.re);
          dot_add(im, u.re, v.im);
        }
        dot_add(re, df_neg(u.im), v.im);
        dot_add(im, u.im, v.re);
      }
      g[sp * 3 + a] = {dot_value(re), dot_value(im)};
    }
}

// Bring the neighbour spinor and the link of direction d into L1 ahead of
// their loads (prefetches hold no registers; a thread computes for about a
// thousand instructions per direction, which covers the DRAM latency).
__device__ __forceinline__ void prefetch_l1(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

__device__ __forceinline__ void prefetch_dir(const HopDfArgs& A, const SpinorView<PDF>& in, long soff,
                                             const SiteCoords& c, int cb, int d) {
  const int mu = d >> 1;
  const bool back = d & 1;
  int wrap;
  const int j = neighbour_index(A.g, c, mu, back ? -1 : +1, &wrap);
  const float4* base = in.p + soff + (j >> 1);
#pragma unroll
  for (int k = 0; k < 12; ++k) prefetch_l1(base + (long)k * in.stride);
  const long lcb = back ? (long)(j >> 1) : (long)cb;
  const int lpar = back ? 1 - A.out_parity : A.out_parity;
  const float4* qu = A.U.p + (long)(lpar * 4 + mu) * 9 * A.U.Vh + lcb;
#pragma unroll
  for (int k = 0; k < 9; ++k) prefetch_l1(qu + (long)k * A.U.Vh);
}

// one thread per (output site, slice); blockIdx.y = slice of all right-hand sides
template <int DAG>
__global__ void __launch_bounds__(128, 3) k_hop_df(HopDfArgs A) {
  if (A.stop && *A.stop) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= A.g.Vh) return;
  const int q = blockIdx.y;
  const int r = fdiv(q, A.d_ls), s = q - r * A.ls;
  const long soff = (long)s * A.g.Vh;
  const SpinorView<PDF> in = A.in.offset_rhs(r);
  const SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
  const float SF = DAG ? 1.f : -1.f;  // sign of gamma in the forward projector
  DCx acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll 1
  for (int d = 0; d < 8; ++d) {
    if (d < 7) prefetch_dir(A, in, soff, c, cb, d + 1);
    const int mu = d >> 1;
    const bool back = d & 1;
    int wrap;
    const int j = neighbour_index(A.g, c, mu, back ? -1 : +1, &wrap);
    const float f = (wrap && A.g.apbc[mu]) ? -1.f : 1.f;
    const float S = back ? -SF : SF;
    const bool swap = mu < 2;
    Phase ph0, ph1;
    if (mu == 0) {
      ph0 = {0.f, -1.f};
      ph1 = {0.f, -1.f};
    } else if (mu == 1) {
      ph0 = {-1.f, 0.f};
      ph1 = {1.f, 0.f};
    } else if (mu == 2) {
      ph0 = {0.f, -1.f};
      ph1 = {0.f, 1.f};
    } else {
      ph0 = {1.f, 0.f};
      ph1 = {1.f, 0.f};
    }
    // neighbour spinor with the lower pair stored as (l_{p0}, l_{p1})
    DCx psi[12];
    {
      const float4* base = in.p + soff + (j >> 1);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const int ck = (k < 6 || !swap) ? k : (k < 9 ? k + 3 : k - 3);
        psi[k] = dcx_load(base + (long)ck * in.stride);
      }
    }
    DCx h[6];
    const Phase c0 = scale_ph(ph0, S), c1 = scale_ph(ph1, S);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      h[cc] = dcx_add_ph(psi[cc], c0, psi[6 + cc]);
      h[3 + cc] = dcx_add_ph(psi[3 + cc], c1, psi[9 + cc]);
    }
    // U_mu(x) forward; U_mu(x - mu)^dag backward (transposed on load, imaginary parts negated)
    DCx U[9];
    {
      const long lcb = back ? (long)(j >> 1) : (long)cb;
      const int lpar = back ? 1 - A.out_parity : A.out_parity;
      const float4* qu = A.U.p + (long)(lpar * 4 + mu) * 9 * A.U.Vh + lcb;
      const float ci = back ? -1.f : 1.f;
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int ek = back ? (k % 3) * 3 + k / 3 : k;
        const DCx u = dcx_load(qu + (long)ek * A.U.Vh);
        U[k] = {u.re, {ci * u.im.h, ci * u.im.l}};
      }
    }
    DCx g[6];
    link_mul_df(U, h, g);
    const Phase q0 = scale_ph(conj_ph(swap ? ph1 : ph0), f * S);
    const Phase q1 = scale_ph(conj_ph(swap ? ph0 : ph1), f * S);
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      const DCx g0 = g[cc], g1 = g[3 + cc];
      acc[cc] = dcx_add_sign(acc[cc], f, g0);
      acc[3 + cc] = dcx_add_sign(acc[3 + cc], f, g1);
      acc[6 + cc] = dcx_add_ph(acc[6 + cc], q0, swap ? g1 : g0);
      acc[9 + cc] = dcx_add_ph(acc[9 + cc], q1, swap ? g0 : g1);
    }
  }
  const long site = soff + cb;
  DCx o[12];
  if (A.x1) {
    DCx v1[12];
    A.vx1.offset_rhs(r).load_df(site, v1);
    DCx v2[12];
    if (A.x2) A.vx2.offset_rhs(r).load_df(site, v2);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      Dot dr = {v1[k].re.h, v1[k].re.l}, di = {v1[k].im.h, v1[k].im.l};
      if (A.x2) {
        dot_add(dr, A.c2, v2[k].re);
        dot_add(di, A.c2, v2[k].im);
      }
      dot_add(dr, A.a, acc[k].re);
      dot_add(di, A.a, acc[k].im);
      o[k] = {df_norm(dot_value(dr)), df_norm(dot_value(di))};
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k)
      o[k] = {df_norm(dot_value(dot_first(A.a, acc[k].re))), df_norm(dot_value(dot_first(A.a, acc[k].im)))};
  }
  A.out.offset_rhs(r).store_df(site, o);
}

Geom df_geom(const Lattice& lat) { return make_geom(lat.L, lat.bc, lat.V, lat.Vh); }

SpinorView<PDF> dfview(const Field& f) {
  SpinorView<PDF> v;
  v.p = (float4*)f.data;
  v.norm = nullptr;
  v.stride = f.nsites();
  return v;
}

struct HopDfLaunch {
  HopDfArgs args;
  int dagger;
  int nslices;
  cudaStream_t st;
};

void run_df(void* ctx, const LaunchCfg& cfg) {
  auto* L = (HopDfLaunch*)ctx;
  dim3 grid((unsigned)((L->args.g.Vh + cfg.block - 1) / cfg.block), (unsigned)L->nslices);
  if (L->dagger)
    k_hop_df<1><<<grid, cfg.block, 0, L->st>>>(L->args);
  else
    k_hop_df<0><<<grid, cfg.block, 0, L->st>>>(L->args);
}

// ----------------------------------------------------------------------------- vector operations
constexpr int kThreads = 256;

unsigned grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  long cap = 8L * sm_count();
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

F2 df_scalar_host(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

// generic view of a standard-precision field (F64 / F32 / F16)
template <int P>
SpinorView<P> stdview(const Field& f) {
  SpinorView<P> v;
  v.p = (decltype(v.p))f.data;
  v.norm = f.norm;
  v.stride = f.nsites();
  return v;
}

// double-float <- F64 (exact split) / F32 / F16 (exact, lo = 0)
template <int P>
__global__ void k_to_df(SpinorView<P> src, SpinorView<PDF> dst, long n) {
  const int r = blockIdx.y;
  const SpinorView<P> s = src.offset_rhs(r);
  const SpinorView<PDF> d = dst.offset_rhs(r);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<typename SpinorView<P>::R> v[12];
    s.load(i, v);
    DCx o[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if constexpr (P == P64)
        o[k] = {df_from_double(v[k].re), df_from_double(v[k].im)};
      else
        o[k] = {{v[k].re, 0.f}, {v[k].im, 0.f}};
    }
    d.store_df(i, o);
  }
}

// F64 (hi + lo in FP64) / F32 / F16 (hi + lo rounded once in FP32) <- double-float
template <int P>
__global__ void k_from_df(SpinorView<PDF> src, SpinorView<P> dst, long n) {
  const int r = blockIdx.y;
  const SpinorView<PDF> s = src.offset_rhs(r);
  const SpinorView<P> d = dst.offset_rhs(r);
  using R = typename SpinorView<P>::R;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    DCx v[12];
    s.load_df(i, v);
    Cx<R> o[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if constexpr (P == P64)
        o[k] = {df_to_double(v[k].re), df_to_double(v[k].im)};
      else
        o[k] = {__fadd_rn(v[k].re.h, v[k].re.l), __fadd_rn(v[k].im.h, v[k].im.l)};
    }
    d.store(i, o);
  }
}

// y = a x + b y in double-float arithmetic; x double-float or FP32 / FP16 (lo = 0)
template <int PX>
__global__ void k_axpby_df(F2 a, SpinorView<PX> x, F2 b, SpinorView<PDF> y, long n) {
  const int r = blockIdx.y;
  const SpinorView<PX> xs = x.offset_rhs(r);
  const SpinorView<PDF> ys = y.offset_rhs(r);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    DCx vx[12], vy[12];
    if constexpr (PX == PDF) {
      xs.load_df(i, vx);
    } else {
      Cx<float> t[12];
      xs.load(i, t);
#pragma unroll
      for (int k = 0; k < 12; ++k) vx[k] = {{t[k].re, 0.f}, {t[k].im, 0.f}};
    }
    ys.load_df(i, vy);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      Dot dr = dot_first(b, vy[k].re), di = dot_first(b, vy[k].im);
      dot_add(dr, a, vx[k].re);
      dot_add(di, a, vx[k].im);
      vy[k] = {df_norm(dot_value(dr)), df_norm(dot_value(di))};
    }
    ys.store_df(i, vy);
  }
}

// y = a x + b y in FP64 with x double-float, y FP64
__global__ void k_axpby_df_f64(double a, SpinorView<PDF> x, double b, SpinorView<P64> y, long n) {
  const int r = blockIdx.y;
  const SpinorView<PDF> xs = x.offset_rhs(r);
  const SpinorView<P64> ys = y.offset_rhs(r);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<double> vx[12], vy[12];
    xs.load(i, vx);
    ys.load(i, vy);
#pragma unroll
    for (int k = 0; k < 12; ++k) vy[k] = {fma(a, vx[k].re, b * vy[k].re), fma(a, vx[k].im, b * vy[k].im)};
    ys.store(i, vy);
  }
}

// per-block partial sums of |x|^2: per-site sums of (hi + lo)^2 in FP32, across
// sites in FP64 (the norms steer the iteration; they need no 48-bit accuracy)
__global__ void k_norm2_df(SpinorView<PDF> x, long n, double* partial) {
  const int r = blockIdx.y;
  const SpinorView<PDF> xs = x.offset_rhs(r);
  double acc[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    DCx v[12];
    xs.load_df(i, v);
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float re = __fadd_rn(v[k].re.h, v[k].re.l), im = __fadd_rn(v[k].im.h, v[k].im.l);
      s = fmaf(re, re, fmaf(im, im, s));
    }
    acc[0] += (double)s;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partial[(long)r * gridDim.x + blockIdx.x] = acc[0];
}

// links: FP64 internal layout [parity][mu][comp][cb] (double2) -> float4 pairs
__global__ void k_links_df(const double2* __restrict__ U64, float4* Udf, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 u = U64[i];
    const F2 re = df_from_double(u.x), im = df_from_double(u.y);
    Udf[i] = make_float4(re.h, re.l, im.h, im.l);
  }
}

}  // namespace

void hop_df(const qcd_gauge* gh, const Field& in, Field& out, int out_parity, int dagger, double a,
            const Field* x1, const Field* x2, double c2, cudaStream_t st, const int* stop,
            bool allow_tuning) {
  if (in.prec != QCD_DF64 || out.prec != QCD_DF64 || (x1 && x1->prec != QCD_DF64) ||
      (x2 && x2->prec != QCD_DF64))
    raise(QCD_ERR_ARG, "hop_df: every operand must be double-float");
  if (x2 && !x1) raise(QCD_ERR_ARG, "hop_df: x2 needs x1");
  if (in.data == out.data || (x1 && x1->data == out.data) || (x2 && x2->data == out.data))
    raise(QCD_ERR_ARG, "hop: output aliases an input");
  if (!gh->Udf) raise(QCD_ERR_ARG, "hop_df: the handle has no double-float links");
  if (in.Vh == 0 || in.nrhs * in.ls == 0) return;
  HopDfLaunch L;
  HopDfArgs& A = L.args;
  A.g = df_geom(gh->lat);
  A.out_parity = out_parity;
  A.ls = in.ls;
  A.d_ls = make_fastdiv((unsigned)in.ls);
  A.x1 = x1 != nullptr;
  A.x2 = x2 != nullptr;
  A.a = df_scalar_host(a);
  A.c2 = df_scalar_host(c2);
  A.U.p = (const float4*)gh->Udf;
  A.U.Vh = gh->lat.Vh;
  A.in = dfview(in);
  A.out = dfview(out);
  A.vx1 = x1 ? dfview(*x1) : dfview(out);
  A.vx2 = x2 ? dfview(*x2) : dfview(out);
  A.stop = stop;
  L.dagger = dagger;
  L.nslices = in.ls * in.nrhs;
  L.st = st;
  if (L.nslices > 65535) raise(QCD_ERR_ARG, "hop_df: too many slices");
  std::vector<LaunchCfg> cands = {{128, 1}, {64, 1}};
  char key[128];
  snprintf(key, sizeof key, "hopdf L%dx%dx%dx%d ns%d x%d%d", gh->lat.L[0], gh->lat.L[1], gh->lat.L[2],
           gh->lat.L[3], L.nslices, A.x1, A.x2);
  LaunchCfg cfg = tune(key, cands, &run_df, &L, st, allow_tuning, stop);
  run_df(&L, cfg);
  QCD_LAUNCH_CK();
}

void links_to_df(qcd_gauge* g, cudaStream_t st) {
  const long n = 2L * 4 * 9 * g->lat.Vh;
  k_links_df<<<grid_for(n), kThreads, 0, st>>>((const double2*)g->U64, (float4*)g->Udf, n);
  QCD_LAUNCH_CK();
}

void df_copy(const Field& src, Field& dst, cudaStream_t st) {
  const long n = src.nsites();
  dim3 grid(grid_for(n), src.nrhs);
  if (dst.prec == QCD_DF64) {
    switch (src.prec) {
      case QCD_F64: k_to_df<P64><<<grid, kThreads, 0, st>>>(stdview<P64>(src), dfview(dst), n); break;
      case QCD_F32: k_to_df<P32><<<grid, kThreads, 0, st>>>(stdview<P32>(src), dfview(dst), n); break;
      case QCD_F16: k_to_df<P16><<<grid, kThreads, 0, st>>>(stdview<P16>(src), dfview(dst), n); break;
      default: raise(QCD_ERR_ARG, "df_copy: bad source precision");
    }
  } else {
    if (src.prec != QCD_DF64) raise(QCD_ERR_ARG, "df_copy: no double-float operand");
    switch (dst.prec) {
      case QCD_F64: k_from_df<P64><<<grid, kThreads, 0, st>>>(dfview(src), stdview<P64>(dst), n); break;
      case QCD_F32: k_from_df<P32><<<grid, kThreads, 0, st>>>(dfview(src), stdview<P32>(dst), n); break;
      case QCD_F16: k_from_df<P16><<<grid, kThreads, 0, st>>>(dfview(src), stdview<P16>(dst), n); break;
      default: raise(QCD_ERR_ARG, "df_copy: bad destination precision");
    }
  }
  QCD_LAUNCH_CK();
}

void df_axpby(double a, const Field& x, double b, Field& y, cudaStream_t st) {
  const long n = x.nsites();
  dim3 grid(grid_for(n), x.nrhs);
  if (y.prec == QCD_DF64) {
    const F2 fa = df_scalar_host(a), fb = df_scalar_host(b);
    switch (x.prec) {
      case QCD_DF64: k_axpby_df<PDF><<<grid, kThreads, 0, st>>>(fa, dfview(x), fb, dfview(y), n); break;
      case QCD_F32: k_axpby_df<P32><<<grid, kThreads, 0, st>>>(fa, stdview<P32>(x), fb, dfview(y), n); break;
      case QCD_F16: k_axpby_df<P16><<<grid, kThreads, 0, st>>>(fa, stdview<P16>(x), fb, dfview(y), n); break;
      default: raise(QCD_ERR_UNSUPPORTED, "axpby: FP64 x into a double-float y");
    }
  } else if (x.prec == QCD_DF64 && y.prec == QCD_F64) {
    k_axpby_df_f64<<<grid, kThreads, 0, st>>>(a, dfview(x), b, stdview<P64>(y), n);
  } else {
    raise(QCD_ERR_UNSUPPORTED, "axpby: unsupported double-float combination");
  }
  QCD_LAUNCH_CK();
}

void df_norm2_partials(const Field& x, double* partial, unsigned nb, cudaStream_t st) {
  k_norm2_df<<<dim3(nb, x.nrhs), kThreads, 0, st>>>(dfview(x), x.nsites(), partial);
  QCD_LAUNCH_CK();
}

unsigned df_norm2_blocks(long n) { return grid_for(n); }

}  // namespace qcd
