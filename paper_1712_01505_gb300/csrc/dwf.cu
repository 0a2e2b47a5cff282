// Site-local parts of the domain-wall matrix: Eq. (2) (Shamir) and its Mobius
// generalisation D = A - 1/2 H B.
//
// S is the fifth-dimension chiral shift, (S psi)_s = P_- psi_{s+1} + P_+ psi_{s-1},
// with factor -m on the terms that cross the wall (s = Ls-1 -> 0 and 0 -> Ls-1);
// B = b5 + c5 S and A = (4 - M5) B + 1 - S = alpha - beta S with
// alpha = (4 - M5) b5 + 1, beta = 1 - (4 - M5) c5 (Shamir: B = 1, A = 5 - M5 - S).
// With gamma_5 = diag(1,1,-1,-1) the projectors P_+- select spins {0,1} and
// {2,3}, so every one of these blocks acts on a column (site, colour, spin) of
// Ls values: on the P_+ spins S is the lower shift T_lo (psi_{s-1}, wrap -m),
// on the P_- spins the upper shift T_up (psi_{s+1}, wrap -m); S^T = S^dag
// exchanges the two.  The inverse of alpha - beta T_lo has the closed form
//   (alpha - beta T_lo)^-1_{s,s'} = beta^k alpha^(-1-k) (s >= s' ? 1 : -m) / den,
//   k = (s - s') mod Ls,   den = 1 + m (beta / alpha)^Ls,
// (T_lo^Ls = -m), and that of alpha - beta T_up is its transpose.
#include <cmath>

#include "common.cuh"
#include "dwf_col.cuh"
#include "internal.h"

namespace qcd {

DwParams dw_params(const qcd_fermion& f) {
  DwParams p{f.Ls, f.M5, f.mf};
  if (f.type == QCD_MOBIUS) {
    p.b5 = f.b5;
    p.c5 = f.c5;
  }
  return p;
}

bool is_dw(const qcd_fermion& f) { return f.type == QCD_DWF || f.type == QCD_MOBIUS; }

namespace {

using namespace dwcol;

// out = [x +] scale * (column operator) in.
// The block stages its SB sites for all Ls slices in shared memory (one HBM
// read per 5D site), runs the column passes in place (thread (site, k) owns the
// complex components k, k + blockDim.y, ...), then writes (site, slice) units.
// block: (SB sites) x (256 / SB); grid: (ceil(Vh/SB), nrhs); dynamic shared
// memory Ls * 24 * SB reals laid out [s][real][site].
// PV >= 0: in, out and x all stored in that precision (the common case, compiled for
// that format alone); PV < 0: the precisions read from the views
template <typename R, int PV>
__device__ __forceinline__ void cld(const AnyView& v, int r, long i, Cx<R> out[12]) {
  if constexpr (PV < 0)
    any_load<R>(v, r, i, out);
  else
    any_load_p<R, PV>(v, r, i, out);
}
template <typename R, int PV>
__device__ __forceinline__ void cst(const AnyView& v, int r, long i, const Cx<R> in[12]) {
  if constexpr (PV < 0)
    any_store<R>(v, r, i, in);
  else
    any_store_p<R, PV>(v, r, i, in);
}

template <typename R, int PV>
__global__ void __launch_bounds__(256) k_col(ColCoef<R> c, AnyView in, AnyView out, long Vh, int dagger, R scale,
                                             AnyView x, int has_x, const int* stop) {
  pdl_enter();
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
      cld<R, PV>(in, r, (long)s * Vh + cb, v);
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
    col_apply(re, im, cs, c, (k < 6) != (dagger != 0), dagger);
  }
  __syncthreads();
  if (cb >= Vh) return;
  for (int s = threadIdx.y; s < Ls; s += blockDim.y) {
    Cx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {sm[s * cs + (2 * k) * SB + tx], sm[s * cs + (2 * k + 1) * SB + tx]};
    if (has_x) {
      Cx<R> w[12];
      cld<R, PV>(x, r, (long)s * Vh + cb, w);
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = {fma(scale, acc[k].re, w[k].re), fma(scale, acc[k].im, w[k].im)};
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = {scale * acc[k].re, scale * acc[k].im};
    }
    cst<R, PV>(out, r, (long)s * Vh + cb, acc);
  }
}

// out = (xd + xe S) in + cy (yd + ye S) y, S^T for dagger; one thread per 5D site
template <typename R>
__global__ void __launch_bounds__(256) k_ablock(int Ls, R mf, R xd, R xe, AnyView in, AnyView out, R yd, R ye,
                                                AnyView y, int has_y, long Vh, int dagger) {
  int r = blockIdx.y;
  long cb = blockIdx.x * (long)blockDim.x + threadIdx.x;
  int s = blockIdx.z * blockDim.y + threadIdx.y;
  if (cb >= Vh || s >= Ls) return;
  const int sm = s == 0 ? Ls - 1 : s - 1;
  const int spl = s == Ls - 1 ? 0 : s + 1;
  // S: P_+ spins take psi_{s-1} (factor -m at s = 0), P_- spins psi_{s+1}
  // (factor -m at s = Ls-1); S^T exchanges the shifts between the chiralities
  const R flo = (s == 0) ? -mf : R(1);
  const R fup = (s == Ls - 1) ? -mf : R(1);
  const R p_lo = dagger ? R(0) : flo, p_up = dagger ? fup : R(0);
  const R m_lo = dagger ? flo : R(0), m_up = dagger ? R(0) : fup;
  Cx<R> o[12];
  {
    Cx<R> v[12], lo[12], up[12];
    any_load<R>(in, r, (long)s * Vh + cb, v);
    any_load<R>(in, r, (long)sm * Vh + cb, lo);
    any_load<R>(in, r, (long)spl * Vh + cb, up);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R clo = xe * (k < 6 ? p_lo : m_lo);
      const R cup = xe * (k < 6 ? p_up : m_up);
      o[k].re = xd * v[k].re + clo * lo[k].re + cup * up[k].re;
      o[k].im = xd * v[k].im + clo * lo[k].im + cup * up[k].im;
    }
  }
  if (has_y) {
    Cx<R> v[12], lo[12], up[12];
    any_load<R>(y, r, (long)s * Vh + cb, v);
    if (ye != R(0)) {
      any_load<R>(y, r, (long)sm * Vh + cb, lo);
      any_load<R>(y, r, (long)spl * Vh + cb, up);
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) lo[k] = up[k] = {R(0), R(0)};
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const R clo = ye * (k < 6 ? p_lo : m_lo);
      const R cup = ye * (k < 6 ? p_up : m_up);
      o[k].re += yd * v[k].re + clo * lo[k].re + cup * up[k].re;
      o[k].im += yd * v[k].im + clo * lo[k].im + cup * up[k].im;
    }
  }
  any_store<R>(out, r, (long)s * Vh + cb, o);
}

// block: 32 consecutive sites (one warp, coalesced) x 8 slices; grid z covers the slices
dim3 block_for(int) { return dim3(32, 8); }
dim3 grid_for(const Field& f, dim3 blk, int Ls) {
  return dim3((unsigned)((f.Vh + blk.x - 1) / blk.x), f.nrhs, (unsigned)((Ls + blk.y - 1) / blk.y));
}

void run_col(const DwParams& p, const ColSpec& spec, const Field& in, Field& out, int dagger, double scale,
             const Field* x, cudaStream_t st, const int* stop) {
  if (p.Ls < 1 || p.Ls > kMaxLs) raise(QCD_ERR_ARG, "Ls must be in [1, %d]", kMaxLs);
  if (in.data == out.data || (x && x->data == out.data))
    raise(QCD_ERR_ARG, "domain-wall block: output aliases an input");
  if (in.prec == QCD_DF64 || out.prec == QCD_DF64 || (x && x->prec == QCD_DF64))
    raise(QCD_ERR_UNSUPPORTED, "this domain-wall block is not available in double-float");
  if (in.nsites() == 0 || in.nrhs == 0) return;
  AnyView xv = x ? any_view(*x) : any_view(out);
  const bool dbl = in.prec == QCD_F64 || out.prec == QCD_F64;
  const size_t rb = dbl ? sizeof(double) : sizeof(float);
  // sites per block: as many as fit 96 KB of staging (at least 8)
  int SB = 32;
  while (SB > 8 && (size_t)p.Ls * 24 * SB * rb > 96 * 1024) SB /= 2;
  const size_t smem = (size_t)p.Ls * 24 * SB * rb;
  dim3 blk(SB, 256 / SB);
  dim3 grid((unsigned)((in.Vh + SB - 1) / SB), in.nrhs);
  static std::atomic<unsigned long long> attr_mask{0};
  if (first_use_on_device(attr_mask)) {
    for (const void* k : {(const void*)k_col<double, -1>, (const void*)k_col<double, P64>, (const void*)k_col<float, -1>,
                          (const void*)k_col<float, P32>, (const void*)k_col<float, P16>})
      QCD_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024));
  }
  const int pv = (in.prec == out.prec && (!x || x->prec == out.prec)) ? in.prec : -1;  // one storage format
  const AnyView iv = any_view(in), ov = any_view(out);
  const bool hx = x != nullptr;
  if (dbl) {
    const ColCoef<double> cc = make_coef<double>(p, spec);
    if (pv == QCD_F64)
      launch_k(k_col<double, P64>, grid, blk, smem, st, cc, iv, ov, in.Vh, dagger, scale, xv, hx, stop);
    else
      launch_k(k_col<double, -1>, grid, blk, smem, st, cc, iv, ov, in.Vh, dagger, scale, xv, hx, stop);
  } else {
    const ColCoef<float> cc = make_coef<float>(p, spec);
    const float sc = (float)scale;
    if (pv == QCD_F32)
      launch_k(k_col<float, P32>, grid, blk, smem, st, cc, iv, ov, in.Vh, dagger, sc, xv, hx, stop);
    else if (pv == QCD_F16)
      launch_k(k_col<float, P16>, grid, blk, smem, st, cc, iv, ov, in.Vh, dagger, sc, xv, hx, stop);
    else
      launch_k(k_col<float, -1>, grid, blk, smem, st, cc, iv, ov, in.Vh, dagger, sc, xv, hx, stop);
  }
  QCD_LAUNCH_CK();
}

void blk_coef(const DwParams& p, Blk5 b, double& d, double& e) {
  switch (b) {
    case BLK_A: d = p.alpha(); e = -p.beta(); return;
    case BLK_B: d = p.b5; e = p.c5; return;
    default: d = 1.0; e = 0.0; return;
  }
}

}  // namespace

void dw_ainv(const DwParams& p, const Field& in, Field& out, int dagger, double scale,
             const Field* x, cudaStream_t st, const int* stop) {
  if (in.prec == QCD_DF64) {
    dw_ainv_df(p, in, out, dagger, scale, x, st, stop);
    return;
  }
  run_col(p, w_spec(p), in, out, dagger, scale, x, st, stop);
}

void dw_binv(const DwParams& p, const Field& in, Field& out, cudaStream_t st) {
  ColSpec cs;
  cs.flags = kInv;
  cs.alpha = p.b5;
  cs.beta = -p.c5;
  run_col(p, cs, in, out, 0, 1.0, nullptr, st, nullptr);
}

void dw_a_binv(const DwParams& p, const Field& in, Field& out, cudaStream_t st) {
  ColSpec cs;
  cs.flags = kPost | (p.mobius() ? kInv : 0);
  cs.alpha = p.b5;
  cs.beta = -p.c5;
  cs.post_d = p.alpha();
  cs.post_e = -p.beta();
  run_col(p, cs, in, out, 0, 1.0, nullptr, st, nullptr);
}

void dw_block(const DwParams& p, const Field& in, Field& out, int dagger, double c, const Field* y,
              cudaStream_t st, Blk5 X, Blk5 Y) {
  if (in.data == out.data || (y && y->data == out.data)) raise(QCD_ERR_ARG, "dw_block: output aliases an input");
  if (in.prec == QCD_DF64 || out.prec == QCD_DF64 || (y && y->prec == QCD_DF64))
    raise(QCD_ERR_UNSUPPORTED, "the domain-wall blocks A and B are not available in double-float");
  if (in.nsites() == 0 || in.nrhs == 0) return;
  double xd, xe, yd, ye;
  blk_coef(p, X, xd, xe);
  blk_coef(p, Y, yd, ye);
  yd *= c;
  ye *= c;
  dim3 blk = block_for(p.Ls);
  dim3 grid = grid_for(in, blk, p.Ls);
  AnyView yv = y ? any_view(*y) : any_view(out);
  if (in.prec == QCD_F64 || out.prec == QCD_F64)
    k_ablock<double><<<grid, blk, 0, st>>>(p.Ls, p.mf, xd, xe, any_view(in), any_view(out), yd, ye, yv,
                                           y != nullptr, in.Vh, dagger);
  else
    k_ablock<float><<<grid, blk, 0, st>>>(p.Ls, (float)p.mf, (float)xd, (float)xe, any_view(in), any_view(out),
                                          (float)yd, (float)ye, yv, y != nullptr, in.Vh, dagger);
  QCD_LAUNCH_CK();
}

}  // namespace qcd
