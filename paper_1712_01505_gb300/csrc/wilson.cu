// Wilson hopping stencil (Eq. (1)) on one parity of the even-odd lattice:
//
//   out(x) = [x(x) +] a * sum_mu [ (1 - gamma_mu) U_mu(x) in(x+mu)
//                                + (1 + gamma_mu) U_mu(x-mu)^dag in(x-mu) ]
//
// for x of the output parity (the neighbours are all of the other parity).
// With `dagger` the projectors are exchanged, which gives H^dag.  The same
// kernel serves the domain-wall operator (the 4D hop acts identically on every
// fifth-dimension slice, Sec. II B 2) and several right-hand sides: a thread
// owns one output site and a tile of TILE slices, loads each link once and
// applies it to all slices of its tile (the links are "common in the 5th
// direction").
//
// Spin structure: in the chiral basis gamma_mu = [[0, B],[B^dag, 0]] with
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.  For a spinor
// (u, l) (upper / lower spin pairs) and sg = -1 for (1 - gamma), +1 for
// (1 + gamma):  (1 + sg gamma)(u, l) = (h, sg B^dag h) with h = u + sg B l.
// Only the half spinor h is multiplied by the link: 2 x 66 flops instead of
// 4 x 66.  Per output site and slice: 8 x (12 projection + 132 link) + 7 x 24
// accumulation = 1320 flops.
#include <climits>
#include <cstdio>
#include <string>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "stencil.cuh"

namespace qcd {

namespace {

using namespace stencil;

template <int P, int RECON, int TILE, int MU>
__device__ __forceinline__ void hop_dir(const HopArgs<P, RECON>& A, const SiteCoords& c, int cb,
                                        int q0, typename MathType<P>::type sg,
                                        Cx<typename MathType<P>::type> acc[TILE][12]) {
  using R = typename MathType<P>::type;
  const Geom& g = A.g;
  // forward: (1 + sg gamma) U_mu(x) in(x + mu)
  {
    int wrap;
    int j = neighbour_index(g, c, MU, +1, &wrap);
    long ncb = j >> 1;
    // boundary sign: folded into the accumulating FMAs in FP64 (ALU-bound,
    // saves instructions), applied to the half spinor in FP32/FP16 (memory-bound)
    const bool neg = wrap && g.apbc[MU];
    const R f = (P == P64 && neg) ? R(-1) : R(1);
    Cx<R> U[9];
    A.U.load(A.out_parity, MU, cb, U);
#pragma unroll
    for (int t = 0; t < TILE; ++t) {
      int q = q0 + t;
      if (TILE > 1 && q >= A.nslices) break;
      int r = fdiv(q, A.d_ls), s = q - r * A.ls;
      Cx<R> psi[12], h[6], gg[6];
      A.in.offset_rhs(r).load((long)s * g.Vh + ncb, psi);
      project<MU>(psi, sg, h);
      if (P != P64 && neg)
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = -h[k];
      link_mul<false>(U, h, gg);
      if constexpr (P == P64)
        reconstruct_add<MU>(gg, sg, f, acc[t]);
      else
        reconstruct_add<MU>(gg, sg, R(1), acc[t]);
    }
  }
  // backward: (1 - sg gamma) U_mu(x - mu)^dag in(x - mu)
  {
    int wrap;
    int j = neighbour_index(g, c, MU, -1, &wrap);
    long ncb = j >> 1;
    const bool neg = wrap && g.apbc[MU];
    const R f = (P == P64 && neg) ? R(-1) : R(1);
    Cx<R> U[9];
    A.U.load(1 - A.out_parity, MU, ncb, U);
#pragma unroll
    for (int t = 0; t < TILE; ++t) {
      int q = q0 + t;
      if (TILE > 1 && q >= A.nslices) break;
      int r = fdiv(q, A.d_ls), s = q - r * A.ls;
      Cx<R> psi[12], h[6], gg[6];
      A.in.offset_rhs(r).load((long)s * g.Vh + ncb, psi);
      project<MU>(psi, -sg, h);
      if (P != P64 && neg)
#pragma unroll
        for (int k = 0; k < 6; ++k) h[k] = -h[k];
      link_mul<true>(U, h, gg);
      if constexpr (P == P64)
        reconstruct_add<MU>(gg, -sg, f, acc[t]);
      else
        reconstruct_add<MU>(gg, -sg, R(1), acc[t]);
    }
  }
}

// ----------------------------------------------------------------------------- prefetch
// Register-free prefetches of the neighbour spinors and links of a direction,
// so that more of the stencil's DRAM traffic is in flight than the registers
// of the resident threads can hold.  PF = 0: none; PF = 1: into L1, one
// direction ahead of its loads; PF = 2: into L1, two directions ahead.
__device__ __forceinline__ void prefetch_line(const void* p) { asm volatile("prefetch.global.L1 [%0];" ::"l"(p)); }

template <int P>
__host__ __device__ constexpr int spinor_comps() {
  return P == P64 ? 12 : (P == P32 ? 6 : 3);
}
template <int P, int RECON>
__host__ __device__ constexpr int link_comps() {
  return (P == P64 || RECON == 18) ? 9 : 3;
}

template <int P, int RECON, int MU>
__device__ __forceinline__ void prefetch_dir(const HopArgs<P, RECON>& A, const SiteCoords& c, int cb, int q0) {
  const int r = q0 / A.ls, s = q0 - r * A.ls;
  const SpinorView<P> in = A.in.offset_rhs(r);
  int wrap;
  const long jf = neighbour_index(A.g, c, MU, +1, &wrap) >> 1;
  const long jb = neighbour_index(A.g, c, MU, -1, &wrap) >> 1;
  const long so = (long)s * A.g.Vh;
#pragma unroll
  for (int k = 0; k < spinor_comps<P>(); ++k) {
    prefetch_line(in.p + k * in.stride + so + jf);
    prefetch_line(in.p + k * in.stride + so + jb);
  }
  if (P == P16) {
    prefetch_line(in.norm + so + jf);
    prefetch_line(in.norm + so + jb);
  }
  constexpr int NL = link_comps<P, RECON>();
  const auto* qf = A.U.p + (long)(A.out_parity * 4 + MU) * NL * A.U.Vh + cb;
  const auto* qb = A.U.p + (long)((1 - A.out_parity) * 4 + MU) * NL * A.U.Vh + jb;
#pragma unroll
  for (int k = 0; k < NL; ++k) {
    prefetch_line(qf + k * A.U.Vh);
    prefetch_line(qb + k * A.U.Vh);
  }
}

template <int PF, int P, int RECON, int MU>
__device__ __forceinline__ void prefetch_before(const HopArgs<P, RECON>& A, const SiteCoords& c, int cb, int q0) {
  if constexpr (PF == 1 && MU < 3) prefetch_dir<P, RECON, MU + 1>(A, c, cb, q0);
  if constexpr (PF == 2 && MU == 0) prefetch_dir<P, RECON, 1>(A, c, cb, q0);
  if constexpr (PF == 2 && MU < 2) prefetch_dir<P, RECON, MU + 2>(A, c, cb, q0);
}

template <int P, int RECON, int TILE, int PF>
__device__ __forceinline__ void hop_tile(const HopArgs<P, RECON>& A) {
  using R = typename MathType<P>::type;
  if (A.stop && *A.stop) return;
  // block -> (site block, slice tile), tiles of one site block adjacent in
  // launch order so that they read the same links at about the same time
  int sblock = fdiv(blockIdx.x, A.d_ntiles);
  int tile = blockIdx.x - sblock * A.ntiles;
  int cb = sblock * blockDim.x + threadIdx.x;
  if (cb >= A.g.Vh) return;
  int q0 = tile * TILE;
  SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
  Cx<R> acc[TILE][12];
#pragma unroll
  for (int t = 0; t < TILE; ++t)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[t][k] = {R(0), R(0)};
  const R sg = A.dagger ? R(1) : R(-1);
  prefetch_before<PF, P, RECON, 0>(A, c, cb, q0);
  hop_dir<P, RECON, TILE, 0>(A, c, cb, q0, sg, acc);
  prefetch_before<PF, P, RECON, 1>(A, c, cb, q0);
  hop_dir<P, RECON, TILE, 1>(A, c, cb, q0, sg, acc);
  prefetch_before<PF, P, RECON, 2>(A, c, cb, q0);
  hop_dir<P, RECON, TILE, 2>(A, c, cb, q0, sg, acc);
  hop_dir<P, RECON, TILE, 3>(A, c, cb, q0, sg, acc);
  const R a = (R)A.a;
#pragma unroll
  for (int t = 0; t < TILE; ++t) {
    int q = q0 + t;
    if (TILE > 1 && q >= A.nslices) break;
    int r = fdiv(q, A.d_ls), s = q - r * A.ls;
    long site = (long)s * A.g.Vh + cb;
    Cx<R> o[12];
    if (A.xpay) {
      A.x.offset_rhs(r).load(site, o);
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = fmac(a, acc[t][k], o[k]);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = a * acc[t][k];
    }
    A.out.offset_rhs(r).store(site, o);
  }
}

template <int P, int RECON, int TILE, int PF>
__global__ void __launch_bounds__(256) k_hop(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_tile<P, RECON, TILE, PF>(A);
}

// one slice per thread in blocks of 64 with the registers bounded so that 14 blocks (28
// warps) fit on an SM
template <int P, int RECON, int PF>
__global__ void __launch_bounds__(64, 14) k_hop_occ(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_tile<P, RECON, 1, PF>(A);
}

// One (site, slice) per thread with the packed FP32x2 arithmetic of stencil.cuh
// and the links read from global memory (FP32 / FP16): the single-slice stencil
// for the precisions whose arithmetic, not HBM, bounds it (FP16: the site scale
// rides on the hop's boundary factor, the link multiply and the projection run
// two spins per instruction).  PF as in k_hop.
template <int P, int RECON, int PF>
__device__ __forceinline__ void hop_pk(const HopArgs<P, RECON>& A) {
  if (A.stop && *A.stop) return;
  const int sblock = fdiv(blockIdx.x, A.d_ntiles);
  const int q = blockIdx.x - sblock * A.ntiles;
  const int cb = sblock * blockDim.x + threadIdx.x;
  if (cb >= A.g.Vh) return;
  const SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
  const int r = fdiv(q, A.d_ls), s = q - r * A.ls;
  const SpinorView<P> in = A.in.offset_rhs(r);
  const long soff = (long)s * A.g.Vh;
  P2 acc[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) acc[k] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  const float sg = A.dagger ? 1.f : -1.f;
  prefetch_before<PF, P, RECON, 0>(A, c, cb, q);
  hop_link_gp<P, RECON, 0, false>(A, c, cb, sg, in, soff, acc);
  hop_link_gp<P, RECON, 0, true>(A, c, cb, sg, in, soff, acc);
  prefetch_before<PF, P, RECON, 1>(A, c, cb, q);
  hop_link_gp<P, RECON, 1, false>(A, c, cb, sg, in, soff, acc);
  hop_link_gp<P, RECON, 1, true>(A, c, cb, sg, in, soff, acc);
  prefetch_before<PF, P, RECON, 2>(A, c, cb, q);
  hop_link_gp<P, RECON, 2, false>(A, c, cb, sg, in, soff, acc);
  hop_link_gp<P, RECON, 2, true>(A, c, cb, sg, in, soff, acc);
  hop_link_gp<P, RECON, 3, false>(A, c, cb, sg, in, soff, acc);
  hop_link_gp<P, RECON, 3, true>(A, c, cb, sg, in, soff, acc);
  const long site = soff + cb;
  const float2 a2 = bc2((float)A.a);
  P2 o[6];
  if (A.xpay) {
    A.x.offset_rhs(r).load_p(site, o);
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = {fma2(a2, acc[k].re, o[k].re), fma2(a2, acc[k].im, o[k].im)};
  } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = {__fmul2_rn(a2, acc[k].re), __fmul2_rn(a2, acc[k].im)};
  }
  A.out.offset_rhs(r).store_p(site, o);
}

template <int P, int RECON, int PF>
__global__ void __launch_bounds__(256) k_hop_pk(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_pk<P, RECON, PF>(A);
}

// the same for blocks of 64 threads with the registers bounded so that 14 blocks (28
// warps) fit on an SM
template <int P, int RECON, int PF>
__global__ void __launch_bounds__(64, 14) k_hop_pk_occ(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_pk<P, RECON, PF>(A);
}

constexpr int kRedGroup = 64;

// The group sums of the single-slice stencils' fused inner products: v[3] per
// thread, summed per warp in R, per block in FP64 (one partial per block), then
// by the last block of each group of kRedGroup blocks in block order.
template <typename R, typename HA>
__device__ __forceinline__ void red_epilogue(const HA& A, R v[3]) {
  // warp sums in R
#pragma unroll
  for (int k = 0; k < 3; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  __shared__ double wsum[8][3];
  __shared__ int last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) wsum[warp][k] = (double)v[k];
  __syncthreads();
  const int ngroups = (gridDim.x + kRedGroup - 1) / kRedGroup;
  const int grp = blockIdx.x / kRedGroup;
  if (threadIdx.x == 0) {
    double b[3] = {0.0, 0.0, 0.0};
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
#pragma unroll
      for (int k = 0; k < 3; ++k) b[k] += wsum[w][k];
#pragma unroll
    for (int k = 0; k < 3; ++k) A.partial[(long)blockIdx.x * 4 + k] = b[k];
    __threadfence();
    const int members = min(kRedGroup, (int)gridDim.x - grp * kRedGroup);
    last = (atomicAdd(&A.counters[grp], 1) == members - 1);
    if (blockIdx.x == 0) *A.npartial = ngroups;
  }
  __syncthreads();
  if (last && warp == 0) {  // the group's last block: sum its members in order
    __threadfence();
    const int first = grp * kRedGroup;
    const int members = min(kRedGroup, (int)gridDim.x - first);
    double g[3] = {0.0, 0.0, 0.0};
    for (int m = lane; m < members; m += 32)
#pragma unroll
      for (int k = 0; k < 3; ++k) g[k] += __ldcg(&A.partial[(long)(first + m) * 4 + k]);  // L2, not a stale L1
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int o = 16; o > 0; o >>= 1) g[k] += __shfl_down_sync(0xffffffffu, g[k], o);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < 3; ++k) A.gpartial[(long)grp * 4 + k] = g[k];
      A.counters[grp] = 0;
    }
  }
}

// Single right-hand side, out = x + a H in, with a BiCGStab inner product
// formed in the epilogue from the values just stored (FP32 / FP64 storage,
// so the stored and the computed values agree): RED = 1 gives (rt, out),
// RED = 2 gives (out, x) and |out|^2.  Sums within a warp in R (FP64 adds
// on 1M threads would cost GB300's slow FP64 pipe tens of microseconds),
// across warps and blocks in FP64: one partial per block, then the last
// block of each group of 64 blocks sums the group (fixed order, so the result
// does not depend on block scheduling).
template <int P, int RECON, int RED, int PF>
__device__ __forceinline__ void hop_red(const HopArgs<P, RECON>& A) {
  using R = typename MathType<P>::type;
  if (A.stop && *A.stop) return;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  R v[3] = {R(0), R(0), R(0)};
  if (cb < A.g.Vh) {
    SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
    Cx<R> acc[1][12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[0][k] = {R(0), R(0)};
    const R sg = A.dagger ? R(1) : R(-1);
    prefetch_before<PF, P, RECON, 0>(A, c, cb, 0);
    hop_dir<P, RECON, 1, 0>(A, c, cb, 0, sg, acc);
    prefetch_before<PF, P, RECON, 1>(A, c, cb, 0);
    hop_dir<P, RECON, 1, 1>(A, c, cb, 0, sg, acc);
    prefetch_before<PF, P, RECON, 2>(A, c, cb, 0);
    hop_dir<P, RECON, 1, 2>(A, c, cb, 0, sg, acc);
    hop_dir<P, RECON, 1, 3>(A, c, cb, 0, sg, acc);
    const R a = (R)A.a;
    Cx<R> xs[12], o[12];
    A.x.load(cb, xs);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = fmac(a, acc[0][k], xs[k]);
    A.out.store(cb, o);
    Cx<R> d = {R(0), R(0)};
    if (RED == 1) {
      Cx<R> w[12];
      A.rt.load(cb, w);
#pragma unroll
      for (int k = 0; k < 12; ++k) d = cjmadd(w[k], o[k], d);
    } else {
      R oo = R(0);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        d = cjmadd(o[k], xs[k], d);
        oo = fma(o[k].re, o[k].re, fma(o[k].im, o[k].im, oo));
      }
      v[2] = oo;
    }
    v[0] = d.re;
    v[1] = d.im;
  }
  red_epilogue<R>(A, v);
}

template <int P, int RECON, int RED, int PF>
__global__ void __launch_bounds__(256) k_hop_red(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_red<P, RECON, RED, PF>(A);
}

template <int P, int RECON, int RED, int PF>
__global__ void __launch_bounds__(64, 14) k_hop_red_occ(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_red<P, RECON, RED, PF>(A);
}

// The packed single-slice stencil (k_hop_pk) with the inner products of
// k_hop_red in its epilogue, for FP16 storage: the sums use the values as stored
// (the FP16 halves times the site scale, for out as for rt and x), so they are
// the inner products of the fields the next kernels read.  SPT sites per thread; the _occ
// kernel: blocks of 64 threads with the registers bounded for 14 blocks (28 warps) per SM.
template <int P, int RECON, int RED, int SPT>
__device__ __forceinline__ void hop_pk_red(const HopArgs<P, RECON>& A) {
  static_assert(P == P16, "the packed stencil with fused inner products is the FP16 one");
  if (A.stop && *A.stop) return;
  float v[3] = {0.f, 0.f, 0.f};
#pragma unroll 1
  for (int it = 0; it < SPT; ++it) {  // SPT sites per thread: one reduction epilogue per SPT blocks' worth
    const int cb = (blockIdx.x * SPT + it) * blockDim.x + threadIdx.x;
    if (cb >= A.g.Vh) break;
    const SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
    P2 acc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const float sg = A.dagger ? 1.f : -1.f;
    hop_link_gp<P, RECON, 0, false>(A, c, cb, sg, A.in, 0, acc);
    hop_link_gp<P, RECON, 0, true>(A, c, cb, sg, A.in, 0, acc);
    hop_link_gp<P, RECON, 1, false>(A, c, cb, sg, A.in, 0, acc);
    hop_link_gp<P, RECON, 1, true>(A, c, cb, sg, A.in, 0, acc);
    hop_link_gp<P, RECON, 2, false>(A, c, cb, sg, A.in, 0, acc);
    hop_link_gp<P, RECON, 2, true>(A, c, cb, sg, A.in, 0, acc);
    hop_link_gp<P, RECON, 3, false>(A, c, cb, sg, A.in, 0, acc);
    hop_link_gp<P, RECON, 3, true>(A, c, cb, sg, A.in, 0, acc);
    const float2 a2 = bc2((float)A.a);
    P2 xs[6], o[6], orr[6];
    A.x.load_p(cb, xs);
#pragma unroll
    for (int k = 0; k < 6; ++k) o[k] = {fma2(a2, acc[k].re, xs[k].re), fma2(a2, acc[k].im, xs[k].im)};
    A.out.template store_p_rounded<true>(cb, o, orr);
    float2 dr = make_float2(0.f, 0.f), di = dr, dj = dr;
    if constexpr (RED == 1) {  // (rt, out) = sum conj(rt) out
      P2 w[6];
      A.rt.load_p(cb, w);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        dr = fma2(w[q].re, orr[q].re, dr);
        dr = fma2(w[q].im, orr[q].im, dr);
        di = fma2(w[q].re, orr[q].im, di);
        dj = fma2(w[q].im, orr[q].re, dj);
      }
    } else {  // (out, x) = sum conj(out) x, |out|^2
      float2 oo = make_float2(0.f, 0.f);
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        dr = fma2(orr[q].re, xs[q].re, dr);
        dr = fma2(orr[q].im, xs[q].im, dr);
        di = fma2(orr[q].re, xs[q].im, di);
        dj = fma2(orr[q].im, xs[q].re, dj);
        oo = fma2(orr[q].re, orr[q].re, oo);
        oo = fma2(orr[q].im, orr[q].im, oo);
      }
      v[2] += oo.x + oo.y;
    }
    v[0] += dr.x + dr.y;
    v[1] += (di.x + di.y) - (dj.x + dj.y);
  }
  red_epilogue<float>(A, v);
}

template <int P, int RECON, int RED, int SPT>
__global__ void __launch_bounds__(256) k_hop_pk_red(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_pk_red<P, RECON, RED, SPT>(A);
}

template <int P, int RECON, int RED, int SPT>
__global__ void __launch_bounds__(64, 14) k_hop_pk_red_occ(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_pk_red<P, RECON, RED, SPT>(A);
}

// RED (with TS = 1, several right-hand sides): the BiCGStab inner products of
// the k_hop_red kernel per right-hand side.  A warp is 32 sites of one slice, so
// it reduces in registers and lane 0 writes partial[(q * nsb + site block) * 4
// + k] (nsb = ceil(Vh / 32)); k_red_rows then sums each slice's partials in order.
template <int P, int RECON, int BY, int TS, int RED>
__device__ __forceinline__ void hop_sm(const HopArgs<P, RECON>& A) {
  static_assert(RED == 0 || TS == 1, "fused reductions need one slice per thread");
  using R = typename MathType<P>::type;
  if (A.stop && *A.stop) return;
  __shared__ SmLinks<R> sm;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sblock = fdiv(blockIdx.x, A.d_ntiles);
  const int stile = blockIdx.x - sblock * A.ntiles;
  const int cb = sblock * 32 + tx;
  const bool valid = cb < A.g.Vh;
  stage_links_sm<P, RECON, BY>(A, sm, tx, ty, cb, valid);
  __syncthreads();
  const int q0 = (stile * BY + ty) * TS;
  if (q0 >= A.nslices) return;      // a whole warp (one row of slices)
  if (!valid && RED == 0) return;  // sites past Vh: with RED they add zero to the warp's sum
  const int nt = min(TS, A.nslices - q0);
  SpinorView<P> in[TS];
  long soff[TS];
#pragma unroll
  for (int t = 0; t < TS; ++t) {
    const int q = min(q0 + t, A.nslices - 1);
    const int r = fdiv(q, A.d_ls), s = q - r * A.ls;
    in[t] = A.in.offset_rhs(r);
    soff[t] = (long)s * A.g.Vh;
  }
  Cx<R> acc[TS][12];
#pragma unroll
  for (int t = 0; t < TS; ++t)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[t][k] = {R(0), R(0)};
  R red[3] = {R(0), R(0), R(0)};
  if (valid) {
  const R sg = A.dagger ? R(1) : R(-1);
  hop_link_sm<P, RECON, TS, 0>(A, sm, tx, sg, in, soff, nt, acc);
  hop_link_sm<P, RECON, TS, 1>(A, sm, tx, sg, in, soff, nt, acc);
  hop_link_sm<P, RECON, TS, 2>(A, sm, tx, sg, in, soff, nt, acc);
  hop_link_sm<P, RECON, TS, 3>(A, sm, tx, sg, in, soff, nt, acc);
  hop_link_sm<P, RECON, TS, 4>(A, sm, tx, sg, in, soff, nt, acc);
  hop_link_sm<P, RECON, TS, 5>(A, sm, tx, sg, in, soff, nt, acc);
  hop_link_sm<P, RECON, TS, 6>(A, sm, tx, sg, in, soff, nt, acc);
  hop_link_sm<P, RECON, TS, 7>(A, sm, tx, sg, in, soff, nt, acc);
  const R a = (R)A.a;
#pragma unroll
  for (int t = 0; t < TS; ++t) {
    if (TS > 1 && t >= nt) break;
    const int q = q0 + t;
    const int r = fdiv(q, A.d_ls);
    const long site = soff[t] + cb;
    Cx<R> o[12];
    if (A.xpay) {
      A.x.offset_rhs(r).load(site, o);
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = fmac(a, acc[t][k], o[k]);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = a * acc[t][k];
    }
    A.out.offset_rhs(r).store(site, o);
    if constexpr (RED == 1) {  // (rt, out)
      Cx<R> w[12], d = {R(0), R(0)};
      A.rt.offset_rhs(r).load(site, w);
#pragma unroll
      for (int k = 0; k < 12; ++k) d = cjmadd(w[k], o[k], d);
      red[0] = d.re;
      red[1] = d.im;
    } else if constexpr (RED == 2) {  // (out, x), |out|^2
      Cx<R> xs[12], d = {R(0), R(0)};
      A.x.offset_rhs(r).load(site, xs);
      R oo = R(0);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        d = cjmadd(o[k], xs[k], d);
        oo = fma(o[k].re, o[k].re, fma(o[k].im, o[k].im, oo));
      }
      red[0] = d.re;
      red[1] = d.im;
      red[2] = oo;
    }
  }
  }  // valid
  if constexpr (RED != 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int o = 16; o > 0; o >>= 1) red[k] += __shfl_down_sync(0xffffffffu, red[k], o);
    if (tx == 0) {
      const long nsb = (A.g.Vh + 31) / 32;
#pragma unroll
      for (int k = 0; k < 3; ++k) A.partial[((long)q0 * nsb + sblock) * 4 + k] = (double)red[k];
    }
  }
}

// The shared-memory kernel with packed FP32x2 arithmetic (stencil.cuh): one
// slice per thread, spinors loaded as spin pairs; RED as in hop_sm.
// L12 = 1: links staged as two rows (SmLinks12), row 2 rebuilt per use
template <int P, int RECON, int BY, int RED, int L12>
__device__ __forceinline__ void hop_smp(const HopArgs<P, RECON>& A) {
  if (A.stop && *A.stop) return;
  using SM = typename std::conditional<L12 != 0, SmLinks12, SmLinks<float>>::type;
  __shared__ SM sm;
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int sblock = fdiv(blockIdx.x, A.d_ntiles);
  const int stile = blockIdx.x - sblock * A.ntiles;
  const int cb = sblock * 32 + tx;
  const bool valid = cb < A.g.Vh;
  if constexpr (L12 != 0)
    stage_links_sm12<P, RECON, BY>(A, sm, tx, ty, cb, valid);
  else
    stage_links_sm<P, RECON, BY>(A, sm, tx, ty, cb, valid);
  __syncthreads();
  const int q0 = stile * BY + ty;
  if (q0 >= A.nslices) return;      // a whole warp (one row of slices)
  if (!valid && RED == 0) return;  // sites past Vh: with RED they add zero to the warp's sum
  const int r = fdiv(q0, A.d_ls), s = q0 - r * A.ls;
  const SpinorView<P> in = A.in.offset_rhs(r);
  const long soff = (long)s * A.g.Vh;
  float red[3] = {0.f, 0.f, 0.f};
  if (valid) {
    P2 acc[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) acc[q] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const float sg = A.dagger ? 1.f : -1.f;
    hop_link_smp<P, RECON, 0>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 1>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 2>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 3>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 4>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 5>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 6>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 7>(A, sm, tx, sg, in, soff, acc);
    const long site = soff + cb;
    const float2 a2 = bc2((float)A.a);
    P2 o[6];
    if (A.xpay) {
      A.x.offset_rhs(r).load_p(site, o);
#pragma unroll
      for (int q = 0; q < 6; ++q) o[q] = {fma2(a2, acc[q].re, o[q].re), fma2(a2, acc[q].im, o[q].im)};
    } else {
#pragma unroll
      for (int q = 0; q < 6; ++q) o[q] = {__fmul2_rn(a2, acc[q].re), __fmul2_rn(a2, acc[q].im)};
    }
    A.out.offset_rhs(r).store_p(site, o);
    if constexpr (RED == 1) {  // (rt, out) = sum conj(rt) out
      P2 w[6];
      A.rt.offset_rhs(r).load_p(site, w);
      float2 dr = make_float2(0.f, 0.f), di = dr, dj = dr;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        dr = fma2(w[q].re, o[q].re, dr);
        dr = fma2(w[q].im, o[q].im, dr);
        di = fma2(w[q].re, o[q].im, di);
        dj = fma2(w[q].im, o[q].re, dj);
      }
      red[0] = dr.x + dr.y;
      red[1] = (di.x + di.y) - (dj.x + dj.y);
    } else if constexpr (RED == 2) {  // (out, x) = sum conj(out) x, |out|^2
      P2 xs[6];
      A.x.offset_rhs(r).load_p(site, xs);
      float2 dr = make_float2(0.f, 0.f), di = dr, dj = dr, oo = dr;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        dr = fma2(o[q].re, xs[q].re, dr);
        dr = fma2(o[q].im, xs[q].im, dr);
        di = fma2(o[q].re, xs[q].im, di);
        dj = fma2(o[q].im, xs[q].re, dj);
        oo = fma2(o[q].re, o[q].re, oo);
        oo = fma2(o[q].im, o[q].im, oo);
      }
      red[0] = dr.x + dr.y;
      red[1] = (di.x + di.y) - (dj.x + dj.y);
      red[2] = oo.x + oo.y;
    }
  }
  if constexpr (RED != 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k)
      for (int o = 16; o > 0; o >>= 1) red[k] += __shfl_down_sync(0xffffffffu, red[k], o);
    if (tx == 0) {
      const long nsb = (A.g.Vh + 31) / 32;
#pragma unroll
      for (int k = 0; k < 3; ++k) A.partial[((long)q0 * nsb + sblock) * 4 + k] = (double)red[k];
    }
  }
}

// A measured prototype, slower than hop_smp (about 1.5 million copies of 16-byte
// chunk runs of at most 512 bytes per launch at 16^3 x 32 x 16; the data still
// crosses the shared-memory pipe once): kept as a tuner candidate.
// The shared-memory-link kernel with packed arithmetic and two-row links (hop_smp,
// L12) whose neighbour spinors are staged in shared memory by bulk copies: NBUF
// buffers per warp (a warp is 32 consecutive sites of one slice), the copies of
// direction L + NBUF - 1 issued (one chunk per lane) while direction L is computed
// from shared memory.  The neighbours of a warp's sites in one direction lie in a run
// of at most 32 consecutive sites unless the direction wraps around the lattice
// between the warp's rows (y, z, t); such a direction is read from global memory as
// in hop_smp.  A copy that never completes (bounded wait) makes the output NaN, which
// the solver reports.
constexpr int kRunSites = 32;
constexpr int kRunFloat4 = 6 * kRunSites;  // one staged direction: 6 chunks x 32 sites

template <int NBUF>
struct SmtState {
  int base[NBUF];
  bool staged[NBUF];
  unsigned phase[NBUF];
  bool failed;
};

template <int L, int NBUF>
__device__ __forceinline__ void smt_issue(const SmLinks12& sm, float4* stage, unsigned long long* bar,
                                          const SpinorView<P32>& in, long soff, int tx, bool valid,
                                          SmtState<NBUF>& S) {
  constexpr int b = L % NBUF;
  const int lo = __reduce_min_sync(0xffffffffu, valid ? sm.nb[L][tx] : INT_MAX);
  const int hi = __reduce_max_sync(0xffffffffu, valid ? sm.nb[L][tx] : INT_MIN);
  const int span = hi - lo + 1;
  S.staged[b] = span <= kRunSites;
  S.base[b] = lo;
  if (!S.staged[b]) return;
  if (tx == 0) mbar_expect_tx(&bar[b], 6u * (unsigned)span * 16u);
  __syncwarp();
  if (tx < 6) {  // lane q copies chunk q
    fence_proxy_async();  // this buffer's earlier reads (ordered by the last __syncwarp) before the copy
    bulk_g2s(stage + b * kRunFloat4 + tx * kRunSites, in.p + tx * in.stride + soff + lo, (unsigned)span * 16u,
             &bar[b]);
  }
}

template <int L, int NBUF>
__device__ __forceinline__ void smt_step(const HopArgs<P32, 12>& A, const SmLinks12& sm, float4* stage,
                                         unsigned long long* bar, const SpinorView<P32>& in, long soff, int tx,
                                         bool valid, float sg, SmtState<NBUF>& S, P2 acc[6]) {
  if constexpr (L + NBUF - 1 < 8) smt_issue<L + NBUF - 1, NBUF>(sm, stage, bar, in, soff, tx, valid, S);
  constexpr int b = L % NBUF;
  if (S.staged[b]) {
    if (!mbar_wait(&bar[b], S.phase[b])) S.failed = true;
    S.phase[b] ^= 1u;
    if (valid) hop_link_run<P32, 12, L, kRunSites>(sm, tx, sg, stage + b * kRunFloat4, S.base[b], acc);
  } else if (valid) {
    hop_link_smp<P32, 12, L>(A, sm, tx, sg, in, soff, acc);
  }
  __syncwarp();  // every lane has read buffer b before later copies overwrite it
}

// dynamic shared memory: [BY][NBUF][kRunFloat4] float4, then [BY][NBUF] barriers
template <int BY, int NBUF>
constexpr size_t smt_smem() {
  return (size_t)BY * NBUF * kRunFloat4 * sizeof(float4) + (size_t)BY * NBUF * sizeof(unsigned long long);
}

template <int BY, int NBUF>
__global__ void __launch_bounds__(32 * BY) k_hop_smt(HopArgs<P32, 12> A) {
  pdl_enter();
  if (A.stop && *A.stop) return;
  __shared__ SmLinks12 sm;
  extern __shared__ __align__(16) unsigned char smt_raw[];
  const int tx = threadIdx.x, ty = threadIdx.y;
  float4* stage = reinterpret_cast<float4*>(smt_raw) + (size_t)ty * NBUF * kRunFloat4;
  unsigned long long* bar =
      reinterpret_cast<unsigned long long*>(smt_raw + (size_t)BY * NBUF * kRunFloat4 * sizeof(float4)) + ty * NBUF;
  const int sblock = fdiv(blockIdx.x, A.d_ntiles);
  const int stile = blockIdx.x - sblock * A.ntiles;
  const int cb = sblock * 32 + tx;
  const bool valid = cb < A.g.Vh;
  stage_links_sm12<P32, 12, BY>(A, sm, tx, ty, cb, valid);
  if (tx < NBUF) mbar_init(&bar[tx], 1);
  if (tx == 0) mbar_init_fence();
  __syncthreads();
  const int q0 = stile * BY + ty;
  if (q0 >= A.nslices) return;  // a whole warp (one row of slices)
  const int r = fdiv(q0, A.d_ls), s = q0 - r * A.ls;
  const SpinorView<P32> in = A.in.offset_rhs(r);
  const long soff = (long)s * A.g.Vh;
  const float sg = A.dagger ? 1.f : -1.f;
  P2 acc[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) acc[q] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  SmtState<NBUF> S;
#pragma unroll
  for (int k = 0; k < NBUF; ++k) S.phase[k] = 0u;
  S.failed = false;
  smt_issue<0, NBUF>(sm, stage, bar, in, soff, tx, valid, S);
  if constexpr (NBUF > 2) smt_issue<1, NBUF>(sm, stage, bar, in, soff, tx, valid, S);
  if constexpr (NBUF > 3) smt_issue<2, NBUF>(sm, stage, bar, in, soff, tx, valid, S);
  smt_step<0, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  smt_step<1, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  smt_step<2, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  smt_step<3, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  smt_step<4, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  smt_step<5, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  smt_step<6, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  smt_step<7, NBUF>(A, sm, stage, bar, in, soff, tx, valid, sg, S, acc);
  if (!valid) return;
  const long site = soff + cb;
  float2 a2 = bc2((float)A.a);
  if (S.failed) a2 = bc2(__int_as_float(0x7fc00000));  // a copy that never arrived: NaN output
  P2 o[6];
  if (A.xpay) {
    A.x.offset_rhs(r).load_p(site, o);
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = {fma2(a2, acc[q].re, o[q].re), fma2(a2, acc[q].im, o[q].im)};
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = {__fmul2_rn(a2, acc[q].re), __fmul2_rn(a2, acc[q].im)};
  }
  A.out.offset_rhs(r).store_p(site, o);
}

// Tensor-core variant of the 12-rhs FP16 stencil (a measured prototype): one
// direction's link multiply (t forward) for the 12 right-hand sides x 2 spins
// of a site runs as warp-level MMAs, m16n8k16 with FP16 operands and FP32
// accumulation.  Per site it is the real 6 x 6 form of U_t(x) (rows: Re, Im of
// the three output colours) times a 6 x 24 matrix of projected half spinors
// (columns: right-hand side x spin), in three n-tiles of 8 columns; the operand
// rows and columns beyond 6 are zero padding.  The half spinors reach the MMA
// lanes through shared memory (rounded to FP16: the FP16 spinors are stored
// scaled to |psi| <= 1 per site, so |h| <= 2), the products return through
// shared memory to the thread that owns the (site, right-hand side) and are
// reconstructed there; the other seven hops use the packed FP32x2 path.  Block:
// 32 sites x 12 right-hand sides (one warp per right-hand side).
__device__ __forceinline__ unsigned pack_h2(float lo, float hi) {
  const __half2 v = __floats2half2_rn(lo, hi);
  return *reinterpret_cast<const unsigned*>(&v);
}

// element (i, j) of the real form of U: rows Re / Im of the output colour, columns Re / Im of
// the input colour
__device__ __forceinline__ float real_form(const Cx<float> u[9], int i, int j) {
  const Cx<float> e = u[(i % 3) * 3 + (j % 3)];
  if (i < 3) return j < 3 ? e.re : -e.im;
  return j < 3 ? e.im : e.re;
}

template <int P, int RECON>
__global__ void __launch_bounds__(384) k_hop_tc(HopArgs<P, RECON> A) {
  pdl_enter();
  static_assert(P == P16 && RECON == 12, "the tensor-core prototype is the FP16, 12-real stencil");
  if (A.stop && *A.stop) return;
  __shared__ SmLinks12 sm;
  __shared__ __align__(16) unsigned Hs[32][24][4];  // [site][column][k pair]: FP16 pairs, k = 6, 7 zero
  __shared__ __align__(16) float Ds[32][6][24];     // [site][row][column]
  const int tx = threadIdx.x, ty = threadIdx.y;     // site of the block, right-hand side (= warp)
  const int cb = blockIdx.x * 32 + tx;
  const bool valid = cb < A.g.Vh;
  stage_links_sm12<P, RECON, 12>(A, sm, tx, ty, cb, valid);
  __syncthreads();
  const int r = fdiv(ty, A.d_ls), s = ty - r * A.ls;
  const SpinorView<P> in = A.in.offset_rhs(r);
  const long soff = (long)s * A.g.Vh;
  P2 acc[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) acc[q] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  const float sg = A.dagger ? 1.f : -1.f;
  if (valid) {
    hop_link_smp<P, RECON, 0>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 1>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 2>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 3>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 4>(A, sm, tx, sg, in, soff, acc);
    hop_link_smp<P, RECON, 5>(A, sm, tx, sg, in, soff, acc);
  }
  // direction L = 6 (t forward) by MMA
  constexpr int L = 6, MU = 3;
  float f = 0.f;
  {
    unsigned v[2][4] = {{0u, 0u, 0u, 0u}, {0u, 0u, 0u, 0u}};
    if (valid) {
      P2 w[6], h[3];
      float scale;
      in.load_p_raw(soff + sm.nb[L][tx], w, &scale);
      f = sm.neg[L][tx] ? -scale : scale;
      project_p<MU>(w, sg, h);
      // column 2 ty + spin; k = Re of colours 0..2, then Im of colours 0..2
      v[0][0] = pack_h2(h[0].re.x, h[1].re.x);
      v[0][1] = pack_h2(h[2].re.x, h[0].im.x);
      v[0][2] = pack_h2(h[1].im.x, h[2].im.x);
      v[1][0] = pack_h2(h[0].re.y, h[1].re.y);
      v[1][1] = pack_h2(h[2].re.y, h[0].im.y);
      v[1][2] = pack_h2(h[1].im.y, h[2].im.y);
    }
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
      *reinterpret_cast<uint4*>(&Hs[tx][2 * ty + sp][0]) = make_uint4(v[sp][0], v[sp][1], v[sp][2], v[sp][3]);
  }
  __syncthreads();
  {
    const int lane = tx, gq = lane >> 2, tq = lane & 3;
    for (int j = ty; j < 96; j += 12) {  // (site, n-tile) jobs spread over the 12 warps
      const int site = j / 3, tile = j - 3 * site;
      unsigned a0 = 0u;
      if (gq < 6 && tq < 3) {
        Cx<float> u[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const float4 e = sm.U[L][k][site];
          u[2 * k] = {e.x, e.y};
          u[2 * k + 1] = {e.z, e.w};
        }
        reconstruct_row2(u);
        a0 = pack_h2(real_form(u, gq, 2 * tq), real_form(u, gq, 2 * tq + 1));
      }
      const unsigned b0 = Hs[site][8 * tile + gq][tq];
      float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
          "{%0,%1,%2,%3};"
          : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
          : "r"(a0), "r"(0u), "r"(0u), "r"(0u), "r"(b0), "r"(0u));
      if (gq < 6) *reinterpret_cast<float2*>(&Ds[site][gq][8 * tile + 2 * tq]) = make_float2(d0, d1);
    }
  }
  __syncthreads();
  if (!valid) return;
  {
    P2 g[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      g[a].re = *reinterpret_cast<const float2*>(&Ds[tx][a][2 * ty]);
      g[a].im = *reinterpret_cast<const float2*>(&Ds[tx][3 + a][2 * ty]);
    }
    reconstruct_p<MU>(g, sg, f, acc);
  }
  hop_link_smp<P, RECON, 7>(A, sm, tx, sg, in, soff, acc);
  const long site = soff + cb;
  const float2 a2 = bc2((float)A.a);
  P2 o[6];
  if (A.xpay) {
    A.x.offset_rhs(r).load_p(site, o);
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = {fma2(a2, acc[q].re, o[q].re), fma2(a2, acc[q].im, o[q].im)};
  } else {
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = {__fmul2_rn(a2, acc[q].re), __fmul2_rn(a2, acc[q].im)};
  }
  A.out.offset_rhs(r).store_p(site, o);
}

template <int P, int RECON, int BY, int RED, int L12>
__global__ void __launch_bounds__(32 * BY) k_hop_smp(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_smp<P, RECON, BY, RED, L12>(A);
}

// the same with the registers bounded so that 24 warps fit on an SM
template <int P, int RECON, int BY, int RED, int L12>
__global__ void __launch_bounds__(32 * BY, 24 / BY) k_hop_smp_occ(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_smp<P, RECON, BY, RED, L12>(A);
}

template <int P, int RECON, int BY, int TS, int RED>
__global__ void __launch_bounds__(32 * BY) k_hop_sm(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_sm<P, RECON, BY, TS, RED>(A);
}

// the same with the registers bounded so that 1024 threads (32 warps) fit on an SM
template <int P, int RECON, int BY, int TS, int RED>
__global__ void __launch_bounds__(32 * BY, 32 / BY) k_hop_sm_occ(HopArgs<P, RECON> A) {
  pdl_enter();
  hop_sm<P, RECON, BY, TS, RED>(A);
}

// per slice q: out[q * 4 + k] = sum over the nsb site blocks of partial[(q * nsb + b) * 4 + k]
// in a fixed order (one block per slice); the consumer adds the ls slices of a right-hand side
__global__ void k_red_rows(const double* __restrict__ partial, long nsb, double* __restrict__ out) {
  pdl_enter();
  const int q = blockIdx.x;
  double v[3] = {0.0, 0.0, 0.0};
  for (long b = threadIdx.x; b < nsb; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < 3; ++k) v[k] += partial[((long)q * nsb + b) * 4 + k];
  block_sum<3>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) out[(long)q * 4 + k] = v[k];
}

Geom dev_geom(const Lattice& lat) { return make_geom(lat.L, lat.bc, lat.V, lat.Vh); }

template <int P>
SpinorView<P> sview(const Field& f) {
  SpinorView<P> v;
  using T = decltype(v.p);
  v.p = (T)f.data;
  v.norm = f.norm;
  v.stride = f.nsites();
  return v;
}

template <int P, int RECON>
struct HopLaunch {
  HopArgs<P, RECON> args;
  cudaStream_t st;
};

// OCC = 1 (one slice per thread): the register-bounded kernels, blocks of 64
template <int P, int RECON, int TILE, int PF = 0, int OCC = 0>
void launch_tile(HopLaunch<P, RECON>* L, int block) {
  static_assert(OCC == 0 || TILE == 1, "the register-bounded stencil has one slice per thread");
  HopArgs<P, RECON> A = L->args;
  A.ntiles = (A.nslices + TILE - 1) / TILE;
  A.d_ntiles = make_fastdiv((unsigned)A.ntiles);
  if (OCC) block = 64;
  long sblocks = (A.g.Vh + block - 1) / block;
  if constexpr (TILE == 1 && P != P16) {
    if (A.red == 1) {
      if constexpr (OCC)
        launch_k(k_hop_red_occ<P, RECON, 1, PF>, (unsigned)sblocks, block, 0, L->st, A);
      else
        launch_k(k_hop_red<P, RECON, 1, PF>, (unsigned)sblocks, block, 0, L->st, A);
      return;
    }
    if (A.red == 2) {
      if constexpr (OCC)
        launch_k(k_hop_red_occ<P, RECON, 2, PF>, (unsigned)sblocks, block, 0, L->st, A);
      else
        launch_k(k_hop_red<P, RECON, 2, PF>, (unsigned)sblocks, block, 0, L->st, A);
      return;
    }
  }
  if constexpr (OCC)
    launch_k(k_hop_occ<P, RECON, PF>, (unsigned)(sblocks * A.ntiles), block, 0, L->st, A);
  else
    launch_k(k_hop<P, RECON, TILE, PF>, (unsigned)(sblocks * A.ntiles), block, 0, L->st, A);
}

template <int P, int RECON, int PF, int OCC = 0>
void launch_pk(HopLaunch<P, RECON>* L, int block) {
  if constexpr (P == P64) {
    raise(QCD_ERR_UNSUPPORTED, "no packed FP64 stencil");
  } else {
    HopArgs<P, RECON> A = L->args;
    A.ntiles = A.nslices;
    A.d_ntiles = make_fastdiv((unsigned)A.ntiles);
    if (OCC) block = 64;
    const long sblocks = (A.g.Vh + block - 1) / block;
    if constexpr (OCC)
      launch_k(k_hop_pk_occ<P, RECON, PF>, (unsigned)(sblocks * A.ntiles), block, 0, L->st, A);
    else
      launch_k(k_hop_pk<P, RECON, PF>, (unsigned)(sblocks * A.ntiles), block, 0, L->st, A);
  }
}

template <int P, int RECON>
void launch_tc(HopLaunch<P, RECON>* L) {
  if constexpr (P == P16 && RECON == 12) {
    HopArgs<P, RECON> A = L->args;
    if (A.nslices != 12) raise(QCD_ERR_UNSUPPORTED, "the tensor-core prototype takes 12 slices");
    A.ntiles = 1;
    A.d_ntiles = make_fastdiv(1u);
    launch_k(k_hop_tc<P, RECON>, (unsigned)((A.g.Vh + 31) / 32), dim3(32, 12), 0, L->st, A);
  } else {
    raise(QCD_ERR_UNSUPPORTED, "the tensor-core prototype is the FP16, 12-real stencil");
  }
}

template <int P, int RECON, int BY, int TS, int RED = 0, int OCC = 0>
void launch_sm(HopLaunch<P, RECON>* L) {
  HopArgs<P, RECON> A = L->args;
  A.ntiles = (A.nslices + BY * TS - 1) / (BY * TS);
  A.d_ntiles = make_fastdiv((unsigned)A.ntiles);
  long sblocks = (A.g.Vh + 31) / 32;
  if constexpr (OCC)
    launch_k(k_hop_sm_occ<P, RECON, BY, TS, RED>, (unsigned)(sblocks * A.ntiles), dim3(32, BY), 0, L->st, A);
  else
    launch_k(k_hop_sm<P, RECON, BY, TS, RED>, (unsigned)(sblocks * A.ntiles), dim3(32, BY), 0, L->st, A);
}

// OCC = 1: the register-bounded kernel (24 warps per SM); L12 = 1: two-row links
template <int P, int RECON, int BY, int RED = 0, int OCC = 0, int L12 = 0>
void launch_smp(HopLaunch<P, RECON>* L) {
  HopArgs<P, RECON> A = L->args;
  A.ntiles = (A.nslices + BY - 1) / BY;
  A.d_ntiles = make_fastdiv((unsigned)A.ntiles);
  long sblocks = (A.g.Vh + 31) / 32;
  const dim3 grid((unsigned)(sblocks * A.ntiles)), blk(32, BY);
  if constexpr (OCC)
    launch_k(k_hop_smp_occ<P, RECON, BY, RED, L12>, grid, blk, 0, L->st, A);
  else
    launch_k(k_hop_smp<P, RECON, BY, RED, L12>, grid, blk, 0, L->st, A);
}

// the shared-memory-link kernel with bulk-copy staged neighbours (FP32, 12-real links,
// 4 thread rows, NBUF buffers per warp)
template <int P, int RECON, int NBUF>
void launch_smt(HopLaunch<P, RECON>* L) {
  if constexpr (P == P32 && RECON == 12) {
    constexpr size_t smem = smt_smem<4, NBUF>();
    static std::atomic<unsigned long long> attr_mask{0};
    if (first_use_on_device(attr_mask))
      QCD_CK(cudaFuncSetAttribute(k_hop_smt<4, NBUF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    HopArgs<P, RECON> A = L->args;
    A.ntiles = (A.nslices + 3) / 4;
    A.d_ntiles = make_fastdiv((unsigned)A.ntiles);
    const long sblocks = (A.g.Vh + 31) / 32;
    launch_k(k_hop_smt<4, NBUF>, (unsigned)(sblocks * A.ntiles), dim3(32, 4), smem, L->st, A);
  } else {
    raise(QCD_ERR_UNSUPPORTED, "the bulk-copy staged stencil is the FP32, 12-real one");
  }
}

// the packed FP16 stencil with fused inner products (one slice, A.red 1 or 2), SPT sites per
// thread; OCC: the register-bounded kernel (blocks of 64)
template <int P, int RECON, int SPT = 1, int OCC = 0>
void launch_pk_red(HopLaunch<P, RECON>* L, int block) {
  if constexpr (P == P16) {
    const HopArgs<P, RECON>& A = L->args;
    if (OCC) block = 64;
    const unsigned blocks = (unsigned)((A.g.Vh + block * SPT - 1) / (block * SPT));
    if constexpr (OCC) {
      if (A.red == 1)
        launch_k(k_hop_pk_red_occ<P, RECON, 1, SPT>, blocks, block, 0, L->st, A);
      else
        launch_k(k_hop_pk_red_occ<P, RECON, 2, SPT>, blocks, block, 0, L->st, A);
    } else {
      if (A.red == 1)
        launch_k(k_hop_pk_red<P, RECON, 1, SPT>, blocks, block, 0, L->st, A);
      else
        launch_k(k_hop_pk_red<P, RECON, 2, SPT>, blocks, block, 0, L->st, A);
    }
  } else {
    raise(QCD_ERR_UNSUPPORTED, "the packed stencil with fused inner products is the FP16 one");
  }
}

// cfg.tile > 0: register tile of that many slices per thread (k_hop), 101 /
// 201: one slice per thread with prefetch mode 1 / 2; 501 / 511: one slice per thread,
// prefetch mode 0 / 1, blocks of 64 with the registers bounded for 28 warps per SM
// (k_hop_occ, k_hop_red_occ); 301 / 311 / 321: one slice
// per thread with packed arithmetic (k_hop_pk), prefetch mode 0 / 1 / 2; 306 / 316: that
// (prefetch mode 0 / 1) with blocks of 64 and registers bounded for 28 warps per SM; 341 /
// 342 / 344: the FP16 stencil with the fused inner products, 1 / 2 / 4 sites per thread;
// 346: that with one site per thread, register-bounded as 306;
// cfg.tile < 0: shared-memory links (k_hop_sm), -tile = 10 * BY + TS for
// BY thread rows of TS slices each; -tile = 200 + 10 * BY + TS: the same with at most
// 64 registers per thread (32 resident warps per SM); -tile = 500 + 10 * BY + 1:
// packed FP32x2 arithmetic, one slice per thread (k_hop_smp); 600 + ...: the
// same with the registers bounded for 24 resident warps; 700 + ...: that with
// the links staged as two rows; -942: that with the neighbour spinors staged in shared
// memory by bulk copies, 2 buffers per warp (k_hop_smt; FP32, 12-real; a measured
// prototype, slower); -3121: 12 slices, one direction by
// tensor-core MMA (k_hop_tc; FP16, 12-real)
template <int P, int RECON>
void run_cfg(void* ctx, const LaunchCfg& cfg) {
  auto* L = (HopLaunch<P, RECON>*)ctx;
  if constexpr (P == P64) {
    launch_tile<P, RECON, 1>(L, cfg.block);
  } else if (P == P16 && L->args.red && L->args.nslices == 1) {  // the FP16 kernel with fused sums
    if (cfg.tile == 344)
      launch_pk_red<P, RECON, 4>(L, cfg.block);
    else if (cfg.tile == 342)
      launch_pk_red<P, RECON, 2>(L, cfg.block);
    else if (cfg.tile == 346)
      launch_pk_red<P, RECON, 1, 1>(L, 64);
    else
      launch_pk_red<P, RECON, 1>(L, cfg.block);
  } else if (L->args.red && L->args.nslices > 1) {  // fused reductions over several slices
    switch (cfg.tile) {
      case -81: L->args.red == 1 ? launch_sm<P, RECON, 8, 1, 1>(L) : launch_sm<P, RECON, 8, 1, 2>(L); break;
      case -241: L->args.red == 1 ? launch_sm<P, RECON, 4, 1, 1, 1>(L) : launch_sm<P, RECON, 4, 1, 2, 1>(L); break;
      case -281: L->args.red == 1 ? launch_sm<P, RECON, 8, 1, 1, 1>(L) : launch_sm<P, RECON, 8, 1, 2, 1>(L); break;
      case -541: L->args.red == 1 ? launch_smp<P, RECON, 4, 1>(L) : launch_smp<P, RECON, 4, 2>(L); break;
      case -581: L->args.red == 1 ? launch_smp<P, RECON, 8, 1>(L) : launch_smp<P, RECON, 8, 2>(L); break;
      case -641: L->args.red == 1 ? launch_smp<P, RECON, 4, 1, 1>(L) : launch_smp<P, RECON, 4, 2, 1>(L); break;
      case -681: L->args.red == 1 ? launch_smp<P, RECON, 8, 1, 1>(L) : launch_smp<P, RECON, 8, 2, 1>(L); break;
      case -741: L->args.red == 1 ? launch_smp<P, RECON, 4, 1, 1, RECON == 12>(L)
                                  : launch_smp<P, RECON, 4, 2, 1, RECON == 12>(L); break;
      case -781: L->args.red == 1 ? launch_smp<P, RECON, 8, 1, 1, RECON == 12>(L)
                                  : launch_smp<P, RECON, 8, 2, 1, RECON == 12>(L); break;
      default: L->args.red == 1 ? launch_sm<P, RECON, 4, 1, 1>(L) : launch_sm<P, RECON, 4, 1, 2>(L);
    }
  } else {
    switch (cfg.tile) {
      case 1: launch_tile<P, RECON, 1>(L, cfg.block); break;
      case 101: launch_tile<P, RECON, 1, 1>(L, cfg.block); break;
      case 501: launch_tile<P, RECON, 1, 0, 1>(L, 64); break;
      case 511: launch_tile<P, RECON, 1, 1, 1>(L, 64); break;
      case 201: launch_tile<P, RECON, 1, 2>(L, cfg.block); break;
      case 301: launch_pk<P, RECON, 0>(L, cfg.block); break;
      case 311: launch_pk<P, RECON, 1>(L, cfg.block); break;
      case 321: launch_pk<P, RECON, 2>(L, cfg.block); break;
      case 306: launch_pk<P, RECON, 0, 1>(L, 64); break;
      case 316: launch_pk<P, RECON, 1, 1>(L, 64); break;
      case 2: launch_tile<P, RECON, 2>(L, cfg.block); break;
      case 4: launch_tile<P, RECON, 4>(L, cfg.block); break;
      case -41: launch_sm<P, RECON, 4, 1>(L); break;
      case -42: launch_sm<P, RECON, 4, 2>(L); break;
      case -81: launch_sm<P, RECON, 8, 1>(L); break;
      case -241: launch_sm<P, RECON, 4, 1, 0, 1>(L); break;
      case -281: launch_sm<P, RECON, 8, 1, 0, 1>(L); break;
      case -541: launch_smp<P, RECON, 4>(L); break;
      case -581: launch_smp<P, RECON, 8>(L); break;
      case -641: launch_smp<P, RECON, 4, 0, 1>(L); break;
      case -681: launch_smp<P, RECON, 8, 0, 1>(L); break;
      case -741: launch_smp<P, RECON, 4, 0, 1, RECON == 12>(L); break;  // 18-real: the -641 kernel
      case -781: launch_smp<P, RECON, 8, 0, 1, RECON == 12>(L); break;
      case -3121: launch_tc<P, RECON>(L); break;
      case -942: launch_smt<P, RECON, 2>(L); break;
      default: launch_sm<P, RECON, 8, 2>(L); break;
    }
  }
}

template <int P, int RECON>
void hop_impl(const qcd_gauge* gh, const void* links, const Field& in, Field& out, int out_parity,
              int dagger, double a, const Field* x, cudaStream_t st, const int* stop,
              bool allow_tuning, const RedSpec* red) {
  HopLaunch<P, RECON> L;
  HopArgs<P, RECON>& A = L.args;
  A.red = 0;
  A.partial = nullptr;
  A.gpartial = nullptr;
  A.counters = nullptr;
  A.npartial = nullptr;
  const bool multi_red = red && red->mode && in.nrhs * in.ls > 1;
  if (red && red->mode) {
    // several slices: FP32 or FP16 (the sums use the computed output, which the FP16 store
    // then rounds: a relative difference of order 1e-3 / sqrt(sites) in the sum); one: FP32 / FP64
    if (!x || (red->mode == 1 && !red->rt) || (multi_red && P == P64))
      raise(QCD_ERR_ARG, "fused reductions need FP32 / FP16 fields (several slices) or FP64 / FP32 / FP16 "
                         "fields (one), and an x term");
    A.red = red->mode;
    A.partial = red->partial;
    A.gpartial = red->gpartial;
    A.counters = red->counters;
    A.npartial = red->npartial;
    if (red->rt) A.rt = sview<P>(*red->rt);
  }
  A.g = dev_geom(gh->lat);
  A.out_parity = out_parity;
  A.ls = in.ls;
  A.d_ls = make_fastdiv((unsigned)in.ls);
  A.nslices = in.ls * in.nrhs;
  A.dagger = dagger;
  A.xpay = x != nullptr;
  A.a = a;
  A.U.p = (decltype(A.U.p))links;
  A.U.Vh = gh->lat.Vh;
  A.in = sview<P>(in);
  A.out = sview<P>(out);
  A.x = x ? sview<P>(*x) : sview<P>(out);
  A.stop = stop;
  L.st = st;
  std::vector<LaunchCfg> cands;
  const int blocks[] = {64, 128, 256};
  const int tiles[] = {1, 2, 4};
  for (int t : tiles) {
    if (P == P64 && t > 1) continue;  // register budget: one slice per thread in FP64
    if (t > 1 && A.nslices < t) continue;
    for (int b : blocks) cands.push_back({b, t});
  }
  if (P != P64 && A.nslices >= 4) cands.push_back({128, -41});
  if (P != P64 && A.nslices >= 8) cands.push_back({128, -42});
  if (P != P64 && A.nslices >= 8) cands.push_back({256, -81});
  if (P != P64 && A.nslices >= 16) cands.push_back({256, -82});
  if (P == P32 && A.nslices >= 4) cands.push_back({128, -241});
  if (P == P32 && A.nslices >= 8) cands.push_back({256, -281});
  // (two-row staging, -7x1, only where the links are stored as 12 reals: row 2 is then rebuilt anyway)
  if (P != P64 && A.nslices >= 4)
    for (int t : {-541, -641, -741})
      if (t != -741 || RECON == 12) cands.push_back({128, t});
  if (P != P64 && A.nslices >= 8)
    for (int t : {-581, -681, -781})
      if (t != -781 || RECON == 12) cands.push_back({256, t});
  if (P == P16 && RECON == 12 && A.nslices == 12) cands.push_back({384, -3121});  // tensor-core direction
  if (P == P32 && RECON == 12 && A.nslices >= 4) cands.push_back({128, -942});  // bulk-copy staged neighbours
  if (A.red) {  // the fused reduction exists for one slice per thread only
    cands.clear();
    if (P != P16)
      for (int b : blocks) cands.push_back({b, 1});
  }
  if (P != P64 && !(A.red && P == P16))  // one slice per thread with prefetches (memory-bound precisions)
    for (int pf : {101, 201})
      for (int b : blocks) cands.push_back({b, pf});
  if (P == P32 && A.nslices == 1)  // the same register-bounded (blocks of 64, 28 warps per SM)
    for (int t : {501, 511}) cands.push_back({64, t});
  if (A.red && P == P16)  // FP16: the packed stencil, its sums over the values as stored, 1 / 2 / 4 sites a thread
    for (int t : {341, 342, 344})
      for (int b : blocks) cands.push_back({b, t});
  if (A.red && P == P16) cands.push_back({64, 346});  // the same register-bounded (28 warps per SM)
  if (P != P64 && !A.red)  // one slice per thread, packed arithmetic, with 0, 1 or 2 directions of prefetch
    for (int pk : {301, 311, 321})
      for (int b : blocks) cands.push_back({b, pk});
  if (P == P16 && !A.red)  // the packed FP16 stencil with the registers bounded for 28 warps per SM
    for (int pk : {306, 316}) cands.push_back({64, pk});
  if (multi_red) {  // shared-memory links, one slice per thread
    cands = {{128, -41}, {256, -81}, {128, -241}, {256, -281}, {128, -541}, {256, -581}, {128, -641}, {256, -681}};
    if (RECON == 12) {
      cands.push_back({128, -741});
      cands.push_back({256, -781});
    }
  }
  char key[160];
  snprintf(key, sizeof key, "hop p%d r%d L%dx%dx%dx%d ns%d xp%d red%d", P, RECON, gh->lat.L[0],
           gh->lat.L[1], gh->lat.L[2], gh->lat.L[3], A.nslices, A.xpay, A.red);
  LaunchCfg cfg = tune(key, cands, &run_cfg<P, RECON>, &L, st, allow_tuning, stop);
  run_cfg<P, RECON>(&L, cfg);
  QCD_LAUNCH_CK();
  if (multi_red) {  // per right-hand side sums of the per-warp partials
    launch_k(k_red_rows, (unsigned)A.nslices, 256, 0, st, A.partial, (A.g.Vh + 31) / 32, A.gpartial);
    QCD_LAUNCH_CK();
  }
}

}  // namespace

void hop(const qcd_gauge* g, const Field& in, Field& out, int out_parity, int dagger, double a,
         const Field* x, cudaStream_t st, const int* stop, bool allow_tuning, const RedSpec* red) {
  if (in.prec != out.prec || (x && x->prec != out.prec))
    raise(QCD_ERR_ARG, "hop: mixed precisions are not supported");
  if (in.data == out.data || (x && x->data == out.data))
    raise(QCD_ERR_ARG, "hop: output aliases an input");
  if (in.Vh == 0 || in.nrhs * in.ls == 0) return;
  switch (in.prec) {
    case QCD_DF64:
      if (red) raise(QCD_ERR_UNSUPPORTED, "fused reductions are not available in double-float");
      hop_df(g, in, out, out_parity, dagger, a, x, nullptr, 0.0, st, stop, allow_tuning);
      break;
    case QCD_F64:
      hop_impl<P64, 18>(g, g->U64, in, out, out_parity, dagger, a, x, st, stop, allow_tuning, red);
      break;
    case QCD_F32:
      if (g->lat.recon == 12)
        hop_impl<P32, 12>(g, g->U32, in, out, out_parity, dagger, a, x, st, stop, allow_tuning, red);
      else
        hop_impl<P32, 18>(g, g->U32, in, out, out_parity, dagger, a, x, st, stop, allow_tuning, red);
      break;
    default:
      if (g->lat.recon == 12)
        hop_impl<P16, 12>(g, g->U16, in, out, out_parity, dagger, a, x, st, stop, allow_tuning, red);
      else
        hop_impl<P16, 18>(g, g->U16, in, out, out_parity, dagger, a, x, st, stop, allow_tuning, red);
  }
}

}  // namespace qcd
