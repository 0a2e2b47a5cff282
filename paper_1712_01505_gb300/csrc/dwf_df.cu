// Double-float site-local inverse of the domain-wall matrix for the outer steps
// of the mixed-precision CG (see wilson_df.cu for the stencil and dfloat.cuh for
// the arithmetic): W = B A^-1 (Shamir, Eq. (2): A^-1), and W^T for the adjoint.
//
// Same column passes as the FP32 / FP64 kernel in dwf.cu, with A = alpha - beta S,
// B = b5 + c5 S: on the columns where S is the lower shift (P_+ spins; P_- for
// the adjoint) the first slice of (A^-1 chi) comes from the closed form
//   psi_0 = sum_s' w_s' chi_s',  w_0 = 1 / (alpha den),
//   w_s' = -m beta^(Ls-s') alpha^(-1-(Ls-s')) / den,
// and psi_s = chi_s / alpha + (beta / alpha) psi_{s-1} for s > 0; on the others
// the last slice comes from w_{Ls-1} = 1 / (alpha den),
// w_s' = -m beta^(s'+1) alpha^(-2-s') / den, and the substitution runs
// downwards; den = 1 + m (beta / alpha)^Ls.  B (before A^-T for the adjoint,
// after A^-1 otherwise) is d psi_s + e psi_{s-+1}.  The closed-form sums are
// Dot2 sums of Ls products; every other step is a Dot2 sum of two products.
#include <cmath>

#include "dfloat.cuh"
#include "internal.h"

namespace qcd {

namespace {

constexpr int kMaxLsDf = 64;

struct AinvDf {
  int Ls, post;      // post: apply B after A^-1 (Mobius)
  F2 wlo[kMaxLsDf];  // closed-form weights of the first slice (lower-shift chirality)
  F2 wup[kMaxLsDf];  // closed-form weights of the last slice (upper-shift chirality)
  F2 ainv, ratio;    // 1 / alpha, beta / alpha
  F2 bd, be, bew;    // B = bd + be S; bew = -m be (the term across the wall)
};

F2 split_host(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}

// (bd + be T) in place on one column of Ls pairs (stride cs)
__device__ __forceinline__ void col_mul_df(F2* col, int cs, int Ls, bool lower, const AinvDf& c) {
  if (lower) {
    const F2 last = col[(Ls - 1) * cs];
    for (int s = Ls - 1; s >= 1; --s) {
      Dot d = dot_first(c.bd, col[s * cs]);
      dot_add(d, c.be, col[(s - 1) * cs]);
      col[s * cs] = dot_value(d);
    }
    Dot d = dot_first(c.bd, col[0]);
    dot_add(d, c.bew, last);
    col[0] = dot_value(d);
  } else {
    const F2 first = col[0];
    for (int s = 0; s < Ls - 1; ++s) {
      Dot d = dot_first(c.bd, col[s * cs]);
      dot_add(d, c.be, col[(s + 1) * cs]);
      col[s * cs] = dot_value(d);
    }
    Dot d = dot_first(c.bd, col[(Ls - 1) * cs]);
    dot_add(d, c.bew, first);
    col[(Ls - 1) * cs] = dot_value(d);
  }
}

// block: (SB sites) x (256 / SB); grid (ceil(Vh / SB), nrhs); dynamic shared memory
// Ls * 24 * SB pairs laid out [s][real][site]
__global__ void __launch_bounds__(256) k_ainv_df(AinvDf c, SpinorView<PDF> in, SpinorView<PDF> out, long Vh,
                                                 int dagger, F2 scale, SpinorView<PDF> x, int has_x,
                                                 const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  F2* sm = reinterpret_cast<F2*>(smraw);
  const int SB = blockDim.x;
  const int r = blockIdx.y;
  const int tx = threadIdx.x;
  const long cb = blockIdx.x * (long)SB + tx;
  const int Ls = c.Ls;
  const int cs = 24 * SB;
  const SpinorView<PDF> inr = in.offset_rhs(r);
  for (int s = threadIdx.y; s < Ls; s += blockDim.y) {
    DCx v[12];
    if (cb < Vh) {
      inr.load_df((long)s * Vh + cb, v);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = {{0.f, 0.f}, {0.f, 0.f}};
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      sm[s * cs + (2 * k) * SB + tx] = v[k].re;
      sm[s * cs + (2 * k + 1) * SB + tx] = v[k].im;
    }
  }
  __syncthreads();
  // one thread per (site, real component): 24 columns of Ls values
  for (int k = threadIdx.y; k < 24; k += blockDim.y) {
    F2* col = sm + k * SB + tx;
    const bool lower = (k < 12) != (dagger != 0);  // spins 0, 1 are reals 0 .. 11
    if (c.post && dagger) col_mul_df(col, cs, Ls, lower, c);
    if (lower) {
      Dot d = dot_first(c.wlo[0], col[0]);
      for (int sp = 1; sp < Ls; ++sp) dot_add(d, c.wlo[sp], col[sp * cs]);
      F2 p = dot_value(d);
      col[0] = p;
      for (int s = 1; s < Ls; ++s) {
        Dot e = dot_first(c.ainv, col[s * cs]);
        dot_add(e, c.ratio, p);
        p = dot_value(e);
        col[s * cs] = p;
      }
    } else {
      const int l = Ls - 1;
      Dot d = dot_first(c.wup[l], col[l * cs]);
      for (int sp = 0; sp < l; ++sp) dot_add(d, c.wup[sp], col[sp * cs]);
      F2 p = dot_value(d);
      col[l * cs] = p;
      for (int s = l - 1; s >= 0; --s) {
        Dot e = dot_first(c.ainv, col[s * cs]);
        dot_add(e, c.ratio, p);
        p = dot_value(e);
        col[s * cs] = p;
      }
    }
    if (c.post && !dagger) col_mul_df(col, cs, Ls, lower, c);
  }
  __syncthreads();
  if (cb >= Vh) return;
  const SpinorView<PDF> outr = out.offset_rhs(r);
  for (int s = threadIdx.y; s < Ls; s += blockDim.y) {
    DCx o[12];
    DCx w[12];
    if (has_x) x.offset_rhs(r).load_df((long)s * Vh + cb, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const F2 re = sm[s * cs + (2 * k) * SB + tx], im = sm[s * cs + (2 * k + 1) * SB + tx];
      Dot dr, di;
      if (has_x) {
        dr = {w[k].re.h, w[k].re.l};
        di = {w[k].im.h, w[k].im.l};
        dot_add(dr, scale, re);
        dot_add(di, scale, im);
      } else {
        dr = dot_first(scale, re);
        di = dot_first(scale, im);
      }
      o[k] = {df_norm(dot_value(dr)), df_norm(dot_value(di))};
    }
    outr.store_df((long)s * Vh + cb, o);
  }
}

SpinorView<PDF> dview(const Field& f) {
  SpinorView<PDF> v;
  v.p = (float4*)f.data;
  v.norm = nullptr;
  v.stride = f.nsites();
  return v;
}

}  // namespace

void dw_ainv_df(const DwParams& p, const Field& in, Field& out, int dagger, double scale, const Field* x,
                cudaStream_t st, const int* stop) {
  if (p.Ls < 1 || p.Ls > kMaxLsDf) raise(QCD_ERR_ARG, "Ls must be in [1, %d]", kMaxLsDf);
  if (in.prec != QCD_DF64 || out.prec != QCD_DF64 || (x && x->prec != QCD_DF64))
    raise(QCD_ERR_ARG, "dw_ainv_df: every operand must be double-float");
  if (in.data == out.data || (x && x->data == out.data)) raise(QCD_ERR_ARG, "dw_ainv: output aliases an input");
  if (in.nsites() == 0 || in.nrhs == 0) return;
  AinvDf c;
  c.Ls = p.Ls;
  c.post = p.mobius();
  const double alpha = p.alpha(), ratio = p.beta() / alpha;
  const double den = 1.0 + p.mf * std::pow(ratio, p.Ls);
  const int Ls = p.Ls;
  // apow[k] = beta^k alpha^(-1-k) / den
  auto apow = [&](int k) { return std::pow(ratio, k) / (alpha * den); };
  for (int s = 0; s < Ls; ++s) {
    // lower shift: w_0 = apow(0), w_s' = -m apow(Ls - s')
    c.wlo[s] = split_host(s == 0 ? apow(0) : -p.mf * apow(Ls - s));
    // upper shift: w_{Ls-1} = apow(0), w_s' = -m apow(s' + 1)
    c.wup[s] = split_host(s == Ls - 1 ? apow(0) : -p.mf * apow(s + 1));
  }
  c.ainv = split_host(1.0 / alpha);
  c.ratio = split_host(ratio);
  c.bd = split_host(p.b5);
  c.be = split_host(p.c5);
  c.bew = split_host(-p.mf * p.c5);
  int SB = 32;
  while (SB > 8 && (size_t)Ls * 24 * SB * sizeof(F2) > 96 * 1024) SB /= 2;
  const size_t smem = (size_t)Ls * 24 * SB * sizeof(F2);
  dim3 blk(SB, 256 / SB);
  dim3 grid((unsigned)((in.Vh + SB - 1) / SB), in.nrhs);
  static std::atomic<unsigned long long> attr_mask{0};
  if (first_use_on_device(attr_mask)) {
    QCD_CK(cudaFuncSetAttribute(k_ainv_df, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  }
  k_ainv_df<<<grid, blk, smem, st>>>(c, dview(in), dview(out), in.Vh, dagger, split_host(scale),
                                     x ? dview(*x) : dview(out), x != nullptr, stop);
  QCD_LAUNCH_CK();
}

}  // namespace qcd
