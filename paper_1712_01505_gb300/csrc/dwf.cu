// Site-local part of the domain-wall matrix (Eq. (2)) and its inverse.
//
// Writing D_DW = A - H/2 with H the 4D Wilson hop acting identically on every
// slice s, the block A couples (s, spin) at one 4D site:
//   (A psi)_s = (5 - M5) psi_s - P_- psi_{s+1} - P_+ psi_{s-1}
//             + m P_+ psi_{Ls-1} [s = 0] + m P_- psi_0 [s = Ls-1]
// With gamma_5 = diag(1,1,-1,-1) the projectors P_+- select spins {0,1} and
// {2,3}.  On the P_+ spins A = a - (lower shift with wrap factor -m), on the
// P_- spins A = a - (upper shift with the same wrap), a = 5 - M5.  The
// inverse of a I - (twisted lower shift) has the closed form
//   (A_+^-1)_{s,s'} = a^(-1-k) * (s >= s' ? 1 : -m) / (1 + m a^-Ls),
//   k = (s - s') mod Ls,
// and A_-^-1 is its transpose (as is A_+^-dag; A is real).  Both are applied
// at every site, colour and spin with Ls real coefficients per output.
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace qcd {

namespace {

constexpr int kMaxLs = 64;

// coefficients in the kernel's arithmetic type (no FP64 in the FP32 kernels)
template <typename R>
struct AinvCoef {
  int Ls;
  R apow[kMaxLs];  // a^(-1-k) / (1 + m a^-Ls)
  R mf;
  R ainv;  // 1 / a
};

// A^-1 per column (site, colour, spin) in O(Ls): on the P_+ spins A is
// a - (lower shift, wrap -m), so with the first slice from the closed form,
//   psi_0 = a^-1 chi_0 / den - m sum_{s'>0} a^(-1-(Ls-s')) chi_s' / den,
// the rest follows by forward substitution psi_s = (chi_s + psi_{s-1}) / a;
// on the P_- spins (upper shift) the last slice comes from the closed form,
//   psi_{Ls-1} = a^-1 chi_{Ls-1} / den - m sum_{s'<Ls-1} a^(-2-s') chi_s' / den,
// and backward substitution psi_s = (chi_s + psi_{s+1}) / a gives the rest.
// A^dag = A^T exchanges the two recurrences between the chiralities.
// The block stages its SB sites for all Ls slices in shared memory (one HBM
// read per 5D site), runs the recurrences in place (thread (site, k) owns the
// complex components k, k + blockDim.y, ...), then writes (site, slice) units.
// block: (SB sites) x (256 / SB); grid: (ceil(Vh/SB), nrhs); dynamic shared
// memory Ls * 24 * SB reals laid out [s][real][site].
template <typename R>
__global__ void __launch_bounds__(256) k_ainv(AinvCoef<R> c, AnyView in, AnyView out, long Vh, int dagger, R scale,
                       AnyView x, int has_x, const int* stop) {
  if (stop && *stop) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* sm = reinterpret_cast<R*>(smraw);
  const int SB = blockDim.x;
  const int r = blockIdx.y;
  const int tx = threadIdx.x;
  const long cb = blockIdx.x * (long)SB + tx;
  const int Ls = c.Ls;
  const int cs = 24 * SB;  // stride between slices
  for (int s = threadIdx.y; s < Ls; s += blockDim.y) {
    Cx<R> v[12];
    if (cb < Vh) {
      any_load<R>(in, r, (long)s * Vh + cb, v);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) v[k] = {R(0), R(0)};
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      sm[s * cs + (2 * k) * SB + tx] = v[k].re;
      sm[s * cs + (2 * k + 1) * SB + tx] = v[k].im;
    }
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 12; k += blockDim.y) {
    R* re = sm + (2 * k) * SB + tx;
    R* im = sm + (2 * k + 1) * SB + tx;
    const bool lower = (k < 6) != (dagger != 0);
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
        pr = (re[s * cs] + pr) * c.ainv;
        pi = (im[s * cs] + pi) * c.ainv;
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
        pr = (re[s * cs] + pr) * c.ainv;
        pi = (im[s * cs] + pi) * c.ainv;
        re[s * cs] = pr;
        im[s * cs] = pi;
      }
    }
  }
  __syncthreads();
  if (cb >= Vh) return;
  for (int s = threadIdx.y; s < Ls; s += blockDim.y) {
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {sm[s * cs + (2 * k) * SB + tx], sm[s * cs + (2 * k + 1) * SB + tx]};
    if (has_x) {
      Cx<R> w[12];
      any_load<R>(x, r, (long)s * Vh + cb, w);
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = {fma(scale, acc[k].re, w[k].re), fma(scale, acc[k].im, w[k].im)};
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = {scale * acc[k].re, scale * acc[k].im};
    }
    any_store<R>(out, r, (long)s * Vh + cb, acc);
  }
}

// out = A in + c * y  (A^dag for dagger)
template <typename R>
__global__ void __launch_bounds__(256) k_ablock(int Ls, R a, R mf, AnyView in, AnyView out, R cy, AnyView y, int has_y,
                         long Vh, int dagger) {
  int r = blockIdx.y;
  long cb = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int s = blockIdx.z * blockDim.y + threadIdx.y;
  if (cb >= Vh || s >= Ls) return;
  Cx<R> v[12], lo[12], up[12];
  any_load<R>(in, r, (long)s * Vh + cb, v);
  int sm = s == 0 ? Ls - 1 : s - 1;
  int spl = s == Ls - 1 ? 0 : s + 1;
  any_load<R>(in, r, (long)sm * Vh + cb, lo);   // psi_{s-1}
  any_load<R>(in, r, (long)spl * Vh + cb, up);  // psi_{s+1}
  // coefficient of psi_{s-1} (lower shift) and psi_{s+1} (upper shift)
  R flo = (s == 0) ? mf : R(-1);
  R fup = (s == Ls - 1) ? mf : R(-1);
  // A: P_+ spins use the lower shift, P_- spins the upper; A^dag swaps them
  R cp_lo = dagger ? R(0) : flo, cp_up = dagger ? fup : R(0);
  R cm_lo = dagger ? flo : R(0), cm_up = dagger ? R(0) : fup;
  Cx<R> o[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    R clo = k < 6 ? cp_lo : cm_lo;
    R cup = k < 6 ? cp_up : cm_up;
    o[k].re = a * v[k].re + clo * lo[k].re + cup * up[k].re;
    o[k].im = a * v[k].im + clo * lo[k].im + cup * up[k].im;
  }
  if (has_y) {
    Cx<R> w[12];
    any_load<R>(y, r, (long)s * Vh + cb, w);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = {fma(cy, w[k].re, o[k].re), fma(cy, w[k].im, o[k].im)};
  }
  any_store<R>(out, r, (long)s * Vh + cb, o);
}

// block: 32 consecutive sites (one warp, coalesced) x 8 slices; grid z covers the slices
dim3 block_for(int) { return dim3(32, 8); }
dim3 grid_for(const Field& f, dim3 blk, int Ls) {
  return dim3((unsigned)((f.Vh + blk.x - 1) / blk.x), f.nrhs, (unsigned)((Ls + blk.y - 1) / blk.y));
}

}  // namespace

void dw_ainv(const DwParams& p, const Field& in, Field& out, int dagger, double scale,
             const Field* x, cudaStream_t st, const int* stop) {
  if (in.prec == QCD_DF64) {
    dw_ainv_df(p, in, out, dagger, scale, x, st, stop);
    return;
  }
  if (p.Ls < 1 || p.Ls > kMaxLs) raise(QCD_ERR_ARG, "Ls must be in [1, %d]", kMaxLs);
  if (in.data == out.data || (x && x->data == out.data))
    raise(QCD_ERR_ARG, "dw_ainv: output aliases an input");
  AnyView xv = x ? any_view(*x) : any_view(out);
  AinvCoef<double> c;
  AinvCoef<float> cf;
  c.Ls = cf.Ls = p.Ls;
  c.mf = p.mf;
  cf.mf = (float)p.mf;
  double a = 5.0 - p.M5;
  double den = 1.0 + p.mf * std::pow(a, -p.Ls);
  for (int k = 0; k < p.Ls; ++k) {
    c.apow[k] = std::pow(a, -1.0 - k) / den;
    cf.apow[k] = (float)c.apow[k];
  }
  c.ainv = 1.0 / a;
  cf.ainv = (float)c.ainv;
  const bool dbl = in.prec == QCD_F64 || out.prec == QCD_F64;
  const size_t rb = dbl ? sizeof(double) : sizeof(float);
  // sites per block: as many as fit 96 KB of staging (at least 8)
  int SB = 32;
  while (SB > 8 && (size_t)p.Ls * 24 * SB * rb > 96 * 1024) SB /= 2;
  const size_t smem = (size_t)p.Ls * 24 * SB * rb;
  dim3 blk(SB, 256 / SB);
  dim3 grid((unsigned)((in.Vh + SB - 1) / SB), in.nrhs);
  static bool attr_set = false;
  if (!attr_set) {
    QCD_CK(cudaFuncSetAttribute(k_ainv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
    QCD_CK(cudaFuncSetAttribute(k_ainv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
    attr_set = true;
  }
  if (dbl)
    k_ainv<double><<<grid, blk, smem, st>>>(c, any_view(in), any_view(out), in.Vh, dagger, scale, xv,
                                            x != nullptr, stop);
  else
    k_ainv<float><<<grid, blk, smem, st>>>(cf, any_view(in), any_view(out), in.Vh, dagger, (float)scale,
                                           xv, x != nullptr, stop);
  QCD_LAUNCH_CK();
}

void dw_block(const DwParams& p, const Field& in, Field& out, int dagger, double c, const Field* y,
              cudaStream_t st) {
  if (in.data == out.data) raise(QCD_ERR_ARG, "dw_block: in and out alias");
  if (in.prec == QCD_DF64 || out.prec == QCD_DF64 || (y && y->prec == QCD_DF64))
    raise(QCD_ERR_UNSUPPORTED, "the domain-wall block A is not available in double-float");
  dim3 blk = block_for(p.Ls);
  dim3 grid = grid_for(in, blk, p.Ls);
  AnyView yv = y ? any_view(*y) : any_view(out);
  double a = 5.0 - p.M5;
  if (in.prec == QCD_F64 || out.prec == QCD_F64)
    k_ablock<double><<<grid, blk, 0, st>>>(p.Ls, a, p.mf, any_view(in), any_view(out), c, yv,
                                           y != nullptr, in.Vh, dagger);
  else
    k_ablock<float><<<grid, blk, 0, st>>>(p.Ls, (float)a, (float)p.mf, any_view(in), any_view(out),
                                          (float)c, yv, y != nullptr, in.Vh, dagger);
  QCD_LAUNCH_CK();
}

}  // namespace qcd
