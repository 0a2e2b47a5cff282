// Fused domain-wall stencil: out = [x +] a * W H_{p,1-p} in, or with dagger
// [x +] a * W^T (H^dag)_{p,1-p} in, where H is the 4D Wilson hop on every
// fifth-dimension slice (Eq. (2)) and W = B A^-1 the inverse of the site-local
// block of D B^-1 (A^-1 for Shamir; see dwf.cu).
//
// The even-odd operator applies W right after a hop twice per application
// (Mhat = 1 - 1/4 W H_eo W H_oe).  Run as two kernels, the hop writes all Ls
// slices to HBM and the column kernel reads them back; here one block owns 32
// sites and all Ls slices of one right-hand side: it stages the sites' links
// in shared memory once (as the multi-slice stencil does), every thread row
// computes the hop for slices ty, ty + BY, ... into a shared-memory tile
// [s][24 reals][32 sites], the block runs the column passes of W on the tile
// (one thread per (site, complex component) column), and writes the result
// with the a / x epilogue.  HBM traffic: the links once per site, the input
// spinors (neighbour re-reads from L2), the output, and x.
#include <type_traits>

#include "common.cuh"
#include "dwf_col.cuh"
#include "internal.h"
#include "stencil.cuh"

namespace qcd {

namespace {

using namespace stencil;
using namespace dwcol;

constexpr int kFusedMaxLs = 32;  // tile of 32 sites x Ls slices x 96 B within 96 KB

// PK = 1: the hop with packed FP32x2 arithmetic (stencil.cuh); PK = 2: the same
// with the links staged as two rows
template <int P, int RECON, int BY, int PK>
__global__ void __launch_bounds__(32 * BY) k_dw_hop_w(HopArgs<P, RECON> A, ColCoef<float> c) {
  pdl_enter();
  using R = typename MathType<P>::type;
  static_assert(sizeof(R) == 4, "the fused stencil computes in FP32");
  if (A.stop && *A.stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* tile = reinterpret_cast<R*>(smraw);
  constexpr int cs = 24 * 32;  // stride between slices of the tile
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int r = blockIdx.y;
  const int cb = blockIdx.x * 32 + tx;
  const bool valid = cb < A.g.Vh;
  const int Ls = A.ls;
  const R sg = A.dagger ? R(1) : R(-1);
  if constexpr (PK) {
    using SM = typename std::conditional<PK == 2, SmLinks12, SmLinks<float>>::type;
    __shared__ SM sm;
    if constexpr (PK == 2)
      stage_links_sm12<P, RECON, BY>(A, sm, tx, ty, cb, valid);
    else
      stage_links_sm<P, RECON, BY>(A, sm, tx, ty, cb, valid);
    __syncthreads();
    const SpinorView<P> in = A.in.offset_rhs(r);
    for (int s = ty; s < Ls; s += BY) {
      P2 acc[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (valid) {
        const long soff = (long)s * A.g.Vh;
        hop_link_smp<P, RECON, 0>(A, sm, tx, sg, in, soff, acc);
        hop_link_smp<P, RECON, 1>(A, sm, tx, sg, in, soff, acc);
        hop_link_smp<P, RECON, 2>(A, sm, tx, sg, in, soff, acc);
        hop_link_smp<P, RECON, 3>(A, sm, tx, sg, in, soff, acc);
        hop_link_smp<P, RECON, 4>(A, sm, tx, sg, in, soff, acc);
        hop_link_smp<P, RECON, 5>(A, sm, tx, sg, in, soff, acc);
        hop_link_smp<P, RECON, 6>(A, sm, tx, sg, in, soff, acc);
        hop_link_smp<P, RECON, 7>(A, sm, tx, sg, in, soff, acc);
      }
      // spin pair q: canonical components b (lane x) and b + 3 (lane y)
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int b = q < 3 ? q : q + 3;
        tile[s * cs + (2 * b) * 32 + tx] = acc[q].re.x;
        tile[s * cs + (2 * b + 1) * 32 + tx] = acc[q].im.x;
        tile[s * cs + (2 * (b + 3)) * 32 + tx] = acc[q].re.y;
        tile[s * cs + (2 * (b + 3) + 1) * 32 + tx] = acc[q].im.y;
      }
    }
  } else {
    __shared__ SmLinks<R> sm;
    stage_links_sm<P, RECON, BY>(A, sm, tx, ty, cb, valid);
    __syncthreads();
    const SpinorView<P> in[1] = {A.in.offset_rhs(r)};
    for (int s = ty; s < Ls; s += BY) {
      Cx<R> acc[1][12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[0][k] = {R(0), R(0)};
      if (valid) {
        const long soff[1] = {(long)s * A.g.Vh};
        hop_link_sm<P, RECON, 1, 0>(A, sm, tx, sg, in, soff, 1, acc);
        hop_link_sm<P, RECON, 1, 1>(A, sm, tx, sg, in, soff, 1, acc);
        hop_link_sm<P, RECON, 1, 2>(A, sm, tx, sg, in, soff, 1, acc);
        hop_link_sm<P, RECON, 1, 3>(A, sm, tx, sg, in, soff, 1, acc);
        hop_link_sm<P, RECON, 1, 4>(A, sm, tx, sg, in, soff, 1, acc);
        hop_link_sm<P, RECON, 1, 5>(A, sm, tx, sg, in, soff, 1, acc);
        hop_link_sm<P, RECON, 1, 6>(A, sm, tx, sg, in, soff, 1, acc);
        hop_link_sm<P, RECON, 1, 7>(A, sm, tx, sg, in, soff, 1, acc);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        tile[s * cs + (2 * k) * 32 + tx] = acc[0][k].re;
        tile[s * cs + (2 * k + 1) * 32 + tx] = acc[0][k].im;
      }
    }
  }
  __syncthreads();
  for (int k = ty; k < 12; k += BY)
    if (Ls <= 16)  // the column of the inverse in registers
      col_apply<R, 16>(tile + (2 * k) * 32 + tx, tile + (2 * k + 1) * 32 + tx, cs, c, (k < 6) != (A.dagger != 0),
                       A.dagger);
    else
      col_apply(tile + (2 * k) * 32 + tx, tile + (2 * k + 1) * 32 + tx, cs, c, (k < 6) != (A.dagger != 0), A.dagger);
  __syncthreads();
  if (!valid) return;
  const R a = (R)A.a;
  const SpinorView<P> out = A.out.offset_rhs(r);
  for (int s = ty; s < Ls; s += BY) {
    const long site = (long)s * A.g.Vh + cb;
    Cx<R> o[12];
    if (A.xpay) {
      A.x.offset_rhs(r).load(site, o);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        o[k].re = fma(a, tile[s * cs + (2 * k) * 32 + tx], o[k].re);
        o[k].im = fma(a, tile[s * cs + (2 * k + 1) * 32 + tx], o[k].im);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k)
        o[k] = {a * tile[s * cs + (2 * k) * 32 + tx], a * tile[s * cs + (2 * k + 1) * 32 + tx]};
    }
    out.store(site, o);
  }
}

template <int P>
SpinorView<P> fview(const Field& f) {
  SpinorView<P> v;
  using T = decltype(v.p);
  v.p = (T)f.data;
  v.norm = f.norm;
  v.stride = f.nsites();
  return v;
}

template <int P, int RECON>
struct FusedLaunch {
  HopArgs<P, RECON> args;
  ColCoef<float> coef;
  size_t smem;
  unsigned nsb;
  int nrhs;
  cudaStream_t st;
};

template <int P, int RECON, int BY, int PK>
void launch_fused(FusedLaunch<P, RECON>* L) {
  static std::atomic<unsigned long long> attr_mask{0};
  if (first_use_on_device(attr_mask)) {
    QCD_CK(cudaFuncSetAttribute(k_dw_hop_w<P, RECON, BY, PK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kFusedMaxLs * 24 * 32 * (int)sizeof(float)));
  }
  launch_k(k_dw_hop_w<P, RECON, BY, PK>, dim3(L->nsb, (unsigned)L->nrhs), dim3(32, BY), L->smem, L->st, L->args,
                                                                                                  L->coef);
}

template <int P, int RECON>
void run_fused(void* ctx, const LaunchCfg& cfg) {
  auto* L = (FusedLaunch<P, RECON>*)ctx;
  switch (cfg.tile) {  // BY, + 100 for the packed arithmetic, + 200 for that with two-row links
    case 4: launch_fused<P, RECON, 4, 0>(L); break;
    case 16: launch_fused<P, RECON, 16, 0>(L); break;
    case 104: launch_fused<P, RECON, 4, 1>(L); break;
    case 108: launch_fused<P, RECON, 8, 1>(L); break;
    case 116: launch_fused<P, RECON, 16, 1>(L); break;
    case 204: launch_fused<P, RECON, 4, RECON == 12 ? 2 : 1>(L); break;  // two-row links need 12-real storage
    case 208: launch_fused<P, RECON, 8, RECON == 12 ? 2 : 1>(L); break;
    default: launch_fused<P, RECON, 8, 0>(L); break;
  }
}

template <int P, int RECON>
void fused_impl(const qcd_gauge* gh, const void* links, const DwParams& p, const Field& in, Field& out,
                int out_parity, int dagger, double a, const Field* x, cudaStream_t st, const int* stop) {
  FusedLaunch<P, RECON> L;
  HopArgs<P, RECON>& A = L.args;
  A.g = make_geom(gh->lat.L, gh->lat.bc, gh->lat.V, gh->lat.Vh);
  A.out_parity = out_parity;
  A.ls = in.ls;
  A.d_ls = make_fastdiv((unsigned)in.ls);
  A.nslices = in.ls * in.nrhs;
  A.ntiles = 1;
  A.d_ntiles = make_fastdiv(1u);
  A.dagger = dagger;
  A.xpay = x != nullptr;
  A.a = a;
  A.U.p = (decltype(A.U.p))links;
  A.U.Vh = gh->lat.Vh;
  A.in = fview<P>(in);
  A.out = fview<P>(out);
  A.x = x ? fview<P>(*x) : fview<P>(out);
  A.stop = stop;
  A.red = 0;
  A.partial = A.gpartial = nullptr;
  A.counters = A.npartial = nullptr;
  L.coef = make_coef<float>(p, w_spec(p));
  L.smem = (size_t)in.ls * 24 * 32 * sizeof(float);
  L.nsb = (unsigned)((gh->lat.Vh + 31) / 32);
  L.nrhs = in.nrhs;
  L.st = st;
  // the first candidate is the one used when no timing is allowed (tuning off): the
  // shape measured fastest at 16^3 x 32 x 16 for this link storage
  std::vector<LaunchCfg> cands;
  if (RECON == 12) cands = {{256, 208}, {128, 204}};
  for (const LaunchCfg& c : std::vector<LaunchCfg>{{256, 8}, {256, 108}, {128, 4}, {128, 104}, {512, 16}, {512, 116}})
    cands.push_back(c);
  char key[160];
  snprintf(key, sizeof key, "dwhopw p%d r%d L%dx%dx%dx%d ls%d nrhs%d xp%d mob%d", P, RECON, gh->lat.L[0],
           gh->lat.L[1], gh->lat.L[2], gh->lat.L[3], in.ls, in.nrhs, A.xpay, (int)p.mobius());
  LaunchCfg cfg = tune(key, cands, &run_fused<P, RECON>, &L, st, true, stop);  // not while captured or stopped
  run_fused<P, RECON>(&L, cfg);
  QCD_LAUNCH_CK();
}

}  // namespace

bool dw_hop_w_fusable(const DwParams& p, int prec) {
  return (prec == QCD_F32 || prec == QCD_F16) && p.Ls >= 1 && p.Ls <= kFusedMaxLs;
}

void dw_hop_w(const qcd_gauge* g, const DwParams& p, const Field& in, Field& out, int out_parity, int dagger,
              double a, const Field* x, cudaStream_t st, const int* stop) {
  if (in.prec != out.prec || (x && x->prec != out.prec))
    raise(QCD_ERR_ARG, "dw_hop_w: mixed precisions are not supported");
  if (!dw_hop_w_fusable(p, in.prec) || in.ls != p.Ls)
    raise(QCD_ERR_UNSUPPORTED, "the fused domain-wall stencil needs FP32 / FP16 fields and Ls <= %d", kFusedMaxLs);
  if (in.data == out.data || (x && x->data == out.data))
    raise(QCD_ERR_ARG, "dw_hop_w: output aliases an input");
  if (in.Vh == 0 || in.nrhs == 0) return;
  if (in.prec == QCD_F32) {
    if (g->lat.recon == 12)
      fused_impl<P32, 12>(g, g->U32, p, in, out, out_parity, dagger, a, x, st, stop);
    else
      fused_impl<P32, 18>(g, g->U32, p, in, out, out_parity, dagger, a, x, st, stop);
  } else {
    if (g->lat.recon == 12)
      fused_impl<P16, 12>(g, g->U16, p, in, out, out_parity, dagger, a, x, st, stop);
    else
      fused_impl<P16, 18>(g, g->U16, p, in, out, out_parity, dagger, a, x, st, stop);
  }
}

}  // namespace qcd
