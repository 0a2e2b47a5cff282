// Column passes of the site-local domain-wall blocks (see dwf.cu for the
// operators): on one (site, colour, spin) column of Ls values, d + e T and
// (alpha - beta T)^-1 with T the twisted lower (P_+ spins) or upper (P_- spins)
// shift of the fifth dimension (factor -m across the wall); the adjoint
// exchanges the shifts.  Shared by the standalone column kernel (dwf.cu) and
// the epilogue of the fused stencil (dwf_hop.cu).
#pragma once
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace qcd {
namespace dwcol {

constexpr int kMaxLs = 64;

// A column operator out = post . inv . pre (in) on the (s, spin) columns, every
// factor optional: pre and post are d + e S, inv is (alpha - beta S)^-1.  The
// adjoint applies post^T, inv^T, pre^T in that order.  Coefficients in the
// kernel's arithmetic type (no FP64 in the FP32 kernels).
enum { kPre = 1, kInv = 2, kPost = 4 };

template <typename R>
struct ColCoef {
  int Ls, flags;
  R mf;
  R pre_d, pre_e, post_d, post_e;
  R ainv, ratio;   // 1 / alpha, beta / alpha
  R apow[kMaxLs];  // beta^k alpha^(-1-k) / den
};

// (d + e T) in place on one column of Ls complex values (stride cs), T = T_lo or T_up
template <typename R>
__device__ __forceinline__ void col_mul(R* re, R* im, int cs, int Ls, bool lower, R d, R e, R mf) {
  const R ew = -mf * e;
  if (lower) {
    const R lr = re[(Ls - 1) * cs], li = im[(Ls - 1) * cs];
    for (int s = Ls - 1; s >= 1; --s) {
      re[s * cs] = fma(e, re[(s - 1) * cs], d * re[s * cs]);
      im[s * cs] = fma(e, im[(s - 1) * cs], d * im[s * cs]);
    }
    re[0] = fma(ew, lr, d * re[0]);
    im[0] = fma(ew, li, d * im[0]);
  } else {
    const R fr = re[0], fi = im[0];
    for (int s = 0; s < Ls - 1; ++s) {
      re[s * cs] = fma(e, re[(s + 1) * cs], d * re[s * cs]);
      im[s * cs] = fma(e, im[(s + 1) * cs], d * im[s * cs]);
    }
    re[(Ls - 1) * cs] = fma(ew, fr, d * re[(Ls - 1) * cs]);
    im[(Ls - 1) * cs] = fma(ew, fi, d * im[(Ls - 1) * cs]);
  }
}

// (alpha - beta T)^-1 in place on one column: the end slice from the closed form,
// the others by substitution psi_s = chi_s / alpha + (beta / alpha) psi_{s-+1}
template <typename R>
__device__ __forceinline__ void col_inv(R* re, R* im, int cs, const ColCoef<R>& c, bool lower) {
  const int Ls = c.Ls;
  if (lower) {
    R pr = c.apow[0] * re[0], pi = c.apow[0] * im[0];
    for (int sp = 1; sp < Ls; ++sp) {
      const R w = -c.mf * c.apow[Ls - sp];
      pr = fma(w, re[sp * cs], pr);
      pi = fma(w, im[sp * cs], pi);
    }
    re[0] = pr;
    im[0] = pi;
    for (int s = 1; s < Ls; ++s) {
      pr = fma(c.ratio, pr, c.ainv * re[s * cs]);
      pi = fma(c.ratio, pi, c.ainv * im[s * cs]);
      re[s * cs] = pr;
      im[s * cs] = pi;
    }
  } else {
    const int l = Ls - 1;
    R pr = c.apow[0] * re[l * cs], pi = c.apow[0] * im[l * cs];
    for (int sp = 0; sp < l; ++sp) {
      const R w = -c.mf * c.apow[sp + 1];
      pr = fma(w, re[sp * cs], pr);
      pi = fma(w, im[sp * cs], pi);
    }
    re[l * cs] = pr;
    im[l * cs] = pi;
    for (int s = l - 1; s >= 0; --s) {
      pr = fma(c.ratio, pr, c.ainv * re[s * cs]);
      pi = fma(c.ratio, pi, c.ainv * im[s * cs]);
      re[s * cs] = pr;
      im[s * cs] = pi;
    }
  }
}

// The same with the column held in registers (Ls <= NR): one read and one write of
// the column instead of two reads and a write (the fused stencil's shared-memory tile)
template <int NR, typename R>
__device__ __forceinline__ void col_inv_reg(R* re, R* im, int cs, const ColCoef<R>& c, bool lower) {
  const int Ls = c.Ls;
  R vr[NR], vi[NR];
#pragma unroll
  for (int s = 0; s < NR; ++s)
    if (s < Ls) {
      vr[s] = re[s * cs];
      vi[s] = im[s * cs];
    }
  if (lower) {
    R pr = c.apow[0] * vr[0], pi = c.apow[0] * vi[0];
#pragma unroll
    for (int sp = 1; sp < NR; ++sp)
      if (sp < Ls) {
        const R w = -c.mf * c.apow[Ls - sp];
        pr = fma(w, vr[sp], pr);
        pi = fma(w, vi[sp], pi);
      }
    re[0] = pr;
    im[0] = pi;
#pragma unroll
    for (int s = 1; s < NR; ++s)
      if (s < Ls) {
        pr = fma(c.ratio, pr, c.ainv * vr[s]);
        pi = fma(c.ratio, pi, c.ainv * vi[s]);
        re[s * cs] = pr;
        im[s * cs] = pi;
      }
  } else {
    const int l = Ls - 1;
    R pr = 0, pi = 0;
#pragma unroll
    for (int sp = 0; sp < NR; ++sp)
      if (sp == l) {
        pr = c.apow[0] * vr[sp];
        pi = c.apow[0] * vi[sp];
      }
#pragma unroll
    for (int sp = 0; sp < NR; ++sp)
      if (sp < l) {
        const R w = -c.mf * c.apow[sp + 1];
        pr = fma(w, vr[sp], pr);
        pi = fma(w, vi[sp], pi);
      }
    // psi_l, then psi_s = chi_s / alpha + (beta / alpha) psi_{s+1} downwards
#pragma unroll
    for (int s = NR - 1; s >= 0; --s) {
      if (s > l) continue;
      if (s < l) {
        pr = fma(c.ratio, pr, c.ainv * vr[s]);
        pi = fma(c.ratio, pi, c.ainv * vi[s]);
      }
      re[s * cs] = pr;
      im[s * cs] = pi;
    }
  }
}

// host description of a column operator
struct ColSpec {
  int flags = 0;
  double pre_d = 1, pre_e = 0, post_d = 1, post_e = 0;
  double alpha = 1, beta = 0;  // inverse of alpha - beta S
};

template <typename R>
inline ColCoef<R> make_coef(const DwParams& p, const ColSpec& cs) {
  ColCoef<R> c;
  c.Ls = p.Ls;
  c.flags = cs.flags;
  c.mf = (R)p.mf;
  c.pre_d = (R)cs.pre_d;
  c.pre_e = (R)cs.pre_e;
  c.post_d = (R)cs.post_d;
  c.post_e = (R)cs.post_e;
  const double ratio = cs.beta / cs.alpha;
  const double den = 1.0 + p.mf * std::pow(ratio, p.Ls);
  c.ainv = (R)(1.0 / cs.alpha);
  c.ratio = (R)ratio;
  double w = 1.0 / (cs.alpha * den);
  for (int k = 0; k < p.Ls; ++k) {
    c.apow[k] = (R)w;
    w *= ratio;
  }
  return c;
}

// W = B A^-1 (A^-1 for Shamir); the adjoint order is handled by the kernels
inline ColSpec w_spec(const DwParams& p) {
  ColSpec cs;
  cs.flags = kInv | (p.mobius() ? kPost : 0);
  cs.alpha = p.alpha();
  cs.beta = p.beta();
  cs.post_d = p.b5;
  cs.post_e = p.c5;
  return cs;
}

// the passes of a column operator (dagger: post^T, inv^T, pre^T) on one complex column;
// NR > 0: the inverse with the column in registers (needs Ls <= NR)
template <typename R, int NR = 0>
__device__ __forceinline__ void col_apply(R* re, R* im, int cs, const ColCoef<R>& c, bool lower, int dagger) {
  const bool first = dagger ? (c.flags & kPost) : (c.flags & kPre);
  const bool last = dagger ? (c.flags & kPre) : (c.flags & kPost);
  if (first) col_mul(re, im, cs, c.Ls, lower, dagger ? c.post_d : c.pre_d, dagger ? c.post_e : c.pre_e, c.mf);
  if (c.flags & kInv) {
    if constexpr (NR > 0)
      col_inv_reg<NR>(re, im, cs, c, lower);
    else
      col_inv(re, im, cs, c, lower);
  }
  if (last) col_mul(re, im, cs, c.Ls, lower, dagger ? c.pre_d : c.post_d, dagger ? c.pre_e : c.post_e, c.mf);
}

}  // namespace dwcol
}  // namespace qcd
