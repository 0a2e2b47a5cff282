// Building blocks of the Wilson hopping stencil (Eq. (1)) shared by the
// stencil kernels (wilson.cu) and the fused domain-wall stencil (dwf_hop.cu).
//
// Spin structure: in the chiral basis gamma_mu = [[0, B],[B^dag, 0]] with
// B_x = -i sigma_1, B_y = -i sigma_2, B_z = -i sigma_3, B_t = 1.  For a spinor
// (u, l) (upper / lower spin pairs) and sg = -1 for (1 - gamma), +1 for
// (1 + gamma):  (1 + sg gamma)(u, l) = (h, sg B^dag h) with h = u + sg B l.
// Only the half spinor h is multiplied by the link: 2 x 66 flops instead of
// 4 x 66.
#pragma once
#include "common.cuh"
#include "internal.h"

namespace qcd {
namespace stencil {

template <typename R>
__device__ __forceinline__ Cx<R> fmac(R s, Cx<R> a, Cx<R> b) {  // b + s*a
  return {fma(s, a.re, b.re), fma(s, a.im, b.im)};
}

// h = u + sg * B l  (2 spins x 3 colours)
template <int MU, typename R>
__device__ __forceinline__ void project(const Cx<R> psi[12], R sg, Cx<R> h[6]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> b0, b1;
    apply_B<MU>(psi[6 + c], psi[9 + c], b0, b1);
    h[c] = fmac(sg, b0, psi[c]);
    h[3 + c] = fmac(sg, b1, psi[3 + c]);
  }
}

// acc += f (g, sg B^dag g), f = +-1 the boundary factor of the hop (folded into
// the accumulating FMAs instead of negating the half spinor)
template <int MU, typename R>
__device__ __forceinline__ void reconstruct_add(const Cx<R> g[6], R sg, R f, Cx<R> acc[12]) {
  const R fs = f * sg;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<R> b0, b1;
    apply_Bdag<MU>(g[c], g[3 + c], b0, b1);
    acc[c] = fmac(f, g[c], acc[c]);
    acc[3 + c] = fmac(f, g[3 + c], acc[3 + c]);
    acc[6 + c] = fmac(fs, b0, acc[6 + c]);
    acc[9 + c] = fmac(fs, b1, acc[9 + c]);
  }
}

// g = U h (dag = false) or U^dag h (dag = true), for both spins of h
template <bool DAG, typename R>
__device__ __forceinline__ void link_mul(const Cx<R> U[9], const Cx<R> h[6], Cx<R> g[6]) {
#pragma unroll
  for (int sp = 0; sp < 2; ++sp)
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cx<R> acc = {R(0), R(0)};
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (DAG)
          acc = cjmadd(U[b * 3 + a], h[sp * 3 + b], acc);
        else
          acc = cmadd(U[a * 3 + b], h[sp * 3 + b], acc);
      }
      g[sp * 3 + a] = acc;
    }
}

template <int P, int RECON>
struct HopArgs {
  Geom g;
  int out_parity;
  int ls;        // slices per right-hand side
  int nslices;   // ls * nrhs
  int ntiles;    // ceil(nslices / TILE)
  FastDiv d_ls, d_ntiles;  // division by ls and by ntiles
  int dagger;
  int xpay;
  double a;
  LinkView<P, RECON> U;
  SpinorView<P> in, out, x;
  const int* stop;
  int red;             // 0: none; 1: (rt, out); 2: (out, x) and |out|^2
  SpinorView<P> rt;
  double* partial;     // [block][4]
  double* gpartial;    // [group of 64 blocks][4]
  int* counters;       // [group]
  int* npartial;
};

// ----------------------------------------------------------------------------- shared-memory links
// Many slices per site (domain-wall fifth dimension, several right-hand sides):
// a block of 32 sites x BY thread rows loads the 8 links of each of its sites
// once, rebuilds them (12-real) and keeps them in shared memory together with
// the 8 neighbour indices and boundary signs of each site; every thread then
// owns one site and TS slices, reads each link once from shared memory and
// applies it to its TS slices.  Link traffic per block is 8 x 32 links
// whatever the number of slices, and the per-site index arithmetic is done once.
// The links are stored as pairs of complex numbers so that a thread reads a
// link with five 16-byte shared-memory loads: element k is half (k & 1) of pair
// k >> 1; pair 4 holds element 8 and padding.
template <typename R>
struct SmLinks {
  static_assert(sizeof(R) == 4, "shared-memory links are FP32");
  float4 U[8][5][32];        // [2 mu + backward][element pair][site]
  int nb[8][32];             // neighbour checkerboard index
  unsigned char neg[8][32];  // 1 if the hop carries the antiperiodic sign
};

template <int P, int RECON, int TS, int L>
__device__ __forceinline__ void hop_link_sm(const HopArgs<P, RECON>& A, const SmLinks<typename MathType<P>::type>& sm,
                                            int tx, typename MathType<P>::type sg, const SpinorView<P> (&in)[TS],
                                            const long (&soff)[TS], int nt,
                                            Cx<typename MathType<P>::type> (&acc)[TS][12]) {
  using R = typename MathType<P>::type;
  constexpr int MU = L >> 1;
  constexpr bool BACK = (L & 1) != 0;
  const long ncb = sm.nb[L][tx];
  const bool neg = sm.neg[L][tx];
  Cx<R> U[9];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 v = sm.U[L][k][tx];
    U[2 * k] = {v.x, v.y};
    if (k < 4) U[2 * k + 1] = {v.z, v.w};
  }
  const R sgn = BACK ? -sg : sg;
#pragma unroll
  for (int t = 0; t < TS; ++t) {
    if (TS > 1 && t >= nt) break;
    Cx<R> psi[12], h[6], gg[6];
    in[t].load(soff[t] + ncb, psi);
    project<MU>(psi, sgn, h);
    if (neg)
#pragma unroll
      for (int k = 0; k < 6; ++k) h[k] = -h[k];
    link_mul<BACK>(U, h, gg);
    reconstruct_add<MU>(gg, sgn, R(1), acc[t]);
  }
}

// Stage the 8 links of the block's 32 sites (rebuilt from 12 reals if needed),
// their neighbour indices and boundary signs into shared memory: thread row ty
// handles the directions l with l % BY == ty.  The caller synchronises.
template <int P, int RECON, int BY>
__device__ __forceinline__ void stage_links_sm(const HopArgs<P, RECON>& A, SmLinks<typename MathType<P>::type>& sm,
                                               int tx, int ty, int cb, bool valid) {
  using R = typename MathType<P>::type;
  if (valid) {
    SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
#pragma unroll
    for (int l = 0; l < 8; ++l) {
      if (l % BY != ty) continue;
      const int mu = l >> 1;
      int wrap;
      int j = neighbour_index(A.g, c, mu, (l & 1) ? -1 : +1, &wrap);
      sm.nb[l][tx] = j >> 1;
      sm.neg[l][tx] = (unsigned char)(wrap && A.g.apbc[mu]);
      Cx<R> U[9];
      if ((l & 1) == 0)
        A.U.load(A.out_parity, mu, cb, U);  // U_mu(x)
      else
        A.U.load(1 - A.out_parity, mu, j >> 1, U);  // U_mu(x - mu)
#pragma unroll
      for (int k = 0; k < 5; ++k)
        sm.U[l][k][tx] = make_float4(U[2 * k].re, U[2 * k].im, k < 4 ? U[2 * k + 1].re : 0.f,
                                     k < 4 ? U[2 * k + 1].im : 0.f);
    }
  }
}


// ----------------------------------------------------------------------------- packed FP32x2
// The same stencil with the two spins of a chiral half as the two lanes of
// Blackwell's packed FP32 instructions (__ffma2_rn / __fadd2_rn / __fmul2_rn,
// each lane rounded as its scalar counterpart): the link multiplies both spins
// of the half spinor by the same matrix, so one FFMA2 does the work of two
// FFMAs with the link element duplicated in both lanes.  Pairs come from
// SpinorView::load_p (spins 0/1 of colour c at [c], spins 2/3 at [3 + c]).
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 swp(float2 a) { return make_float2(a.y, a.x); }
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

// h = u + sg B l per colour, lanes = the two spins (B from the chiral basis above)
template <int MU>
__device__ __forceinline__ void project_p(const P2 w[6], float sg, P2 h[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const P2& u = w[c];
    const P2& l = w[3 + c];
    if (MU == 0) {  // B l = -i (l_1, l_0)
      h[c].re = fma2(bc2(sg), swp(l.im), u.re);
      h[c].im = fma2(bc2(-sg), swp(l.re), u.im);
    } else if (MU == 1) {  // B l = (-l_1, l_0)
      h[c].re = fma2(make_float2(-sg, sg), swp(l.re), u.re);
      h[c].im = fma2(make_float2(-sg, sg), swp(l.im), u.im);
    } else if (MU == 2) {  // B l = (-i l_0, i l_1)
      h[c].re = fma2(make_float2(sg, -sg), l.im, u.re);
      h[c].im = fma2(make_float2(-sg, sg), l.re, u.im);
    } else {  // B l = l
      h[c].re = fma2(bc2(sg), l.re, u.re);
      h[c].im = fma2(bc2(sg), l.im, u.im);
    }
  }
}

// acc += f (g, sg B^dag g), f = +-1 the boundary factor of the hop
template <int MU>
__device__ __forceinline__ void reconstruct_p(const P2 g[3], float sg, float f, P2 acc[6]) {
  const float fs = f * sg;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    acc[c].re = fma2(bc2(f), g[c].re, acc[c].re);
    acc[c].im = fma2(bc2(f), g[c].im, acc[c].im);
    if (MU == 0) {  // B^dag g = i (g_1, g_0)
      acc[3 + c].re = fma2(bc2(-fs), swp(g[c].im), acc[3 + c].re);
      acc[3 + c].im = fma2(bc2(fs), swp(g[c].re), acc[3 + c].im);
    } else if (MU == 1) {  // B^dag g = (g_1, -g_0)
      acc[3 + c].re = fma2(make_float2(fs, -fs), swp(g[c].re), acc[3 + c].re);
      acc[3 + c].im = fma2(make_float2(fs, -fs), swp(g[c].im), acc[3 + c].im);
    } else if (MU == 2) {  // B^dag g = (i g_0, -i g_1)
      acc[3 + c].re = fma2(make_float2(-fs, fs), g[c].im, acc[3 + c].re);
      acc[3 + c].im = fma2(make_float2(fs, -fs), g[c].re, acc[3 + c].im);
    } else {
      acc[3 + c].re = fma2(bc2(fs), g[c].re, acc[3 + c].re);
      acc[3 + c].im = fma2(bc2(fs), g[c].im, acc[3 + c].im);
    }
  }
}

// Link element k of direction L as (re, re, im, im), from the compact staging
// (two elements per float4) with the lanes duplicated in registers (FFMA2 takes
// the duplicated operand without extra instructions).
__device__ __forceinline__ void link_elems(const SmLinks<float>& sm, int L, int tx, float4 e[9]) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const float4 v = sm.U[L][k][tx];
    e[2 * k] = make_float4(v.x, v.x, v.y, v.y);
    if (k < 4) e[2 * k + 1] = make_float4(v.z, v.z, v.w, v.w);
  }
}

// Links in shared memory as their first two rows (12 reals, three 16-byte
// loads per link); row 2 = conj(row0 x row1) is rebuilt in registers by every
// thread that uses the link: fewer L1/shared-memory wavefronts for ~24 more
// FP32 instructions per link use.
struct SmLinks12 {
  float4 U[8][3][32];        // [2 mu + backward][element pair of rows 0-1][site]
  int nb[8][32];             // neighbour checkerboard index
  unsigned char neg[8][32];  // 1 if the hop carries the antiperiodic sign
};

template <int P, int RECON, int BY>
__device__ __forceinline__ void stage_links_sm12(const HopArgs<P, RECON>& A, SmLinks12& sm, int tx, int ty, int cb,
                                                 bool valid) {
  using R = typename MathType<P>::type;
  if (!valid) return;
  SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
#pragma unroll
  for (int l = 0; l < 8; ++l) {
    if (l % BY != ty) continue;
    const int mu = l >> 1;
    int wrap;
    int j = neighbour_index(A.g, c, mu, (l & 1) ? -1 : +1, &wrap);
    sm.nb[l][tx] = j >> 1;
    sm.neg[l][tx] = (unsigned char)(wrap && A.g.apbc[mu]);
    Cx<R> U[9];
    if ((l & 1) == 0)
      A.U.load(A.out_parity, mu, cb, U);  // U_mu(x)
    else
      A.U.load(1 - A.out_parity, mu, j >> 1, U);  // U_mu(x - mu)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      sm.U[l][k][tx] = make_float4(U[2 * k].re, U[2 * k].im, U[2 * k + 1].re, U[2 * k + 1].im);
  }
}

__device__ __forceinline__ void link_elems(const SmLinks12& sm, int L, int tx, float4 e[9]) {
  Cx<float> u[9];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4 v = sm.U[L][k][tx];
    u[2 * k] = {v.x, v.y};
    u[2 * k + 1] = {v.z, v.w};
  }
  reconstruct_row2(u);
#pragma unroll
  for (int k = 0; k < 9; ++k) e[k] = make_float4(u[k].re, u[k].re, u[k].im, u[k].im);
}

// g = U h (U^dag h for BACK) for both spins of h in the lanes; e[k] = link element k as
// (re, re, im, im)
template <bool BACK>
__device__ __forceinline__ void link_mul_p(const float4 e[9], const P2 h[3], P2 g[3]) {
  // -Im h (forward) or -Re h (backward) for the terms with a minus sign
  float2 nh[3];
#pragma unroll
  for (int b = 0; b < 3; ++b) nh[b] = BACK ? __fmul2_rn(bc2(-1.f), h[b].re) : __fmul2_rn(bc2(-1.f), h[b].im);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 gr = make_float2(0.f, 0.f), gi = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      // forward: U_ab; backward: conj(U_ba)
      const float4 u = e[BACK ? b * 3 + a : a * 3 + b];
      const float2 ur = make_float2(u.x, u.y), ui = make_float2(u.z, u.w);
      if (!BACK) {  // (ur + i ui) h: re = ur h.re - ui h.im, im = ur h.im + ui h.re
        gr = fma2(ur, h[b].re, gr);
        gr = fma2(ui, nh[b], gr);
        gi = fma2(ur, h[b].im, gi);
        gi = fma2(ui, h[b].re, gi);
      } else {  // (ur - i ui) h: re = ur h.re + ui h.im, im = ur h.im - ui h.re
        gr = fma2(ur, h[b].re, gr);
        gr = fma2(ui, h[b].im, gr);
        gi = fma2(ur, h[b].im, gi);
        gi = fma2(ui, nh[b], gi);
      }
    }
    g[a] = {gr, gi};
  }
}

// acc += the hop from direction L (mu = L / 2, backward if L odd) for one slice,
// packed: g = U h (U^dag h backward) with both spins of h in the lanes.  The FP16
// site scale multiplies the hop's boundary factor instead of the 24 loaded values.
template <int P, int RECON, int L, typename SM>
__device__ __forceinline__ void hop_link_smp(const HopArgs<P, RECON>& A, const SM& sm, int tx, float sg,
                                             const SpinorView<P>& in, long soff, P2 acc[6]) {
  constexpr int MU = L >> 1;
  constexpr bool BACK = (L & 1) != 0;
  const long ncb = sm.nb[L][tx];
  const float sgn = BACK ? -sg : sg;
  P2 w[6], h[3], g[3];
  float scale;
  in.load_p_raw(soff + ncb, w, &scale);
  const float f = sm.neg[L][tx] ? -scale : scale;
  project_p<MU>(w, sgn, h);
  float4 e[9];
  link_elems(sm, L, tx, e);
  link_mul_p<BACK>(e, h, g);
  reconstruct_p<MU>(g, sgn, f, acc);
}

// ----------------------------------------------------------------------------- bulk staging
// Neighbour spinors staged in shared memory by the bulk-copy engine (cp.async.bulk
// with an mbarrier that counts the bytes), so that a warp's next direction arrives
// while it computes the current one, with no registers and no load instructions
// of its own.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// generic-proxy accesses of shared memory ordered before later bulk copies into it
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// wait for the completion of the barrier's phase `parity`, at most about 2^20 polls;
// false if it did not complete
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  for (int i = 0; i < (1 << 20); ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// acc += the hop from direction L for one slice (as hop_link_smp), the neighbour's six
// 16-byte chunks read from a staged run: chunk q of site n at run[q * RUN + n - base]
template <int P, int RECON, int L, int RUN, typename SM>
__device__ __forceinline__ void hop_link_run(const SM& sm, int tx, float sg, const float4* run, int base,
                                             P2 acc[6]) {
  static_assert(P == P32, "the staged runs hold FP32 spinors");
  constexpr int MU = L >> 1;
  constexpr bool BACK = (L & 1) != 0;
  const int n = sm.nb[L][tx] - base;
  const float sgn = BACK ? -sg : sg;
  P2 w[6], h[3], g[3];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const float4 d = run[q * RUN + n];
    w[q] = {make_float2(d.x, d.y), make_float2(d.z, d.w)};
  }
  const float f = sm.neg[L][tx] ? -1.f : 1.f;
  project_p<MU>(w, sgn, h);
  float4 e[9];
  link_elems(sm, L, tx, e);
  link_mul_p<BACK>(e, h, g);
  reconstruct_p<MU>(g, sgn, f, acc);
}

// The same for one site whose links come from global memory (single-slice
// stencil): direction MU, forward or backward.
template <int P, int RECON, int MU, bool BACK>
__device__ __forceinline__ void hop_link_gp(const HopArgs<P, RECON>& A, const SiteCoords& c, long cb, float sg,
                                            const SpinorView<P>& in, long soff, P2 acc[6]) {
  int wrap;
  const int j = neighbour_index(A.g, c, MU, BACK ? -1 : +1, &wrap);
  const long ncb = j >> 1;
  const float sgn = BACK ? -sg : sg;
  P2 w[6], h[3], g[3];
  float scale;
  in.load_p_raw(soff + ncb, w, &scale);
  const float f = (wrap && A.g.apbc[MU]) ? -scale : scale;
  Cx<float> u[9];
  A.U.load(BACK ? 1 - A.out_parity : A.out_parity, MU, BACK ? ncb : cb, u);
  float4 e[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) e[k] = make_float4(u[k].re, u[k].re, u[k].im, u[k].im);
  project_p<MU>(w, sgn, h);
  link_mul_p<BACK>(e, h, g);
  reconstruct_p<MU>(g, sgn, f, acc);
}

}  // namespace stencil
}  // namespace qcd
