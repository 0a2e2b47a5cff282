// Krylov solvers of Sec. II C on the even-odd preconditioned system:
// BiCGStab (van der Vorst 1992) for the Wilson Schur operator Mhat, CG
// (Hestenes-Stiefel) on Mhat^dag Mhat for the domain-wall one, each for
// `nrhs` right-hand sides with their own scalars.
//
// Mixed precision (the single-precision inner solver of Sec. II C): the
// iteration runs on FP32 or FP16 vectors; every time the iterated residual
// has dropped by `delta` since the previous outer step, or reaches the target,
// an outer step in FP64 adds the inner iterate into the FP64 solution,
// recomputes the true residual b - A x with the FP64 operator and restarts the
// recursion from it while keeping the search direction (reliable update,
// Sleijpen & van der Vorst 1996).  FP64 therefore appears on the device only in
// the true-residual recomputation, the solution accumulation and the global
// sums of the dot products.  With outer = QCD_DF64 (Wilson) the outer steps
// run in double-float instead (FP32 pairs, about 48 bits; see wilson_df.cu),
// and only the final true residual uses the IEEE-FP64 stencil.
//
// The scalars (alpha, beta, omega, rho, |r|^2) never leave the device during
// the inner iteration: per-block partial sums become scalars in the prologue of
// the next vector kernel (alpha, omega) or in the one-block kernel that ends an
// iteration (rho_new, |r|^2, beta and the stop decision).
// Every kernel of the iteration first reads a stop word; when an iteration
// raises it (convergence check due, reliable update due, breakdown, NaN) the
// remaining launches of the chunk do nothing, so a chunk of K iterations can
// be captured once into a CUDA graph and replayed, with one host
// synchronisation per chunk.
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace qcd {

namespace {

enum Flag { FLAG_NONE = 0, FLAG_CHECK = 1, FLAG_UPDATE = 2, FLAG_BREAKDOWN = 3, FLAG_NAN = 4 };

// per right-hand side, device resident
struct Scal {
  double rho[2], rho_new[2], alpha[2], omega[2], beta[2];
  double rr, rr_new;  // CG: |r|^2 before / after the step
  double r2;          // iterated |r|^2 after the last step
  double r2_ref;      // |r|^2 at the last outer step
  double stop2;       // |r|^2 that ends the inner phase for a true-residual check
  double delta2;      // reliable-update trigger (0: none)
  int active;
  int flag;
  int iters;
  int pad;
};

constexpr int kThreads = 256;
constexpr int kMaxPartial = 4;

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ bool bad(double v) { return !isfinite(v); }

// ----------------------------------------------------------------------------- partial sums
// Sum the per-block partials of one right-hand side (one block per rhs).
template <int NR>
__device__ void sum_partials(const double* partial, int nblk, int r, double out[NR]) {
  double v[NR];
#pragma unroll
  for (int k = 0; k < NR; ++k) v[k] = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int k = 0; k < NR; ++k) v[k] += partial[((long)r * nblk + b) * kMaxPartial + k];
  block_sum<NR>(v);
#pragma unroll
  for (int k = 0; k < NR; ++k) out[k] = v[k];
}

template <int NR>
__device__ __forceinline__ void write_partial(double v[NR], double* partial, int r) {
  block_sum<NR>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NR; ++k) partial[((long)r * gridDim.x + blockIdx.x) * kMaxPartial + k] = v[k];
}

#define STOPPED(ctl) (*(ctl) != 0)

// Loads and stores of the solver's vectors: PV >= 0 fixes the storage precision
// at compile time (the iteration kernels, which the host instantiates for the
// inner precision: only that path is compiled, so the register count is that of
// the one format), PV < 0 reads it from the view (the generic kernels).
template <typename R, int PV>
__device__ __forceinline__ void vld(const AnyView& v, int r, long i, Cx<R> out[12]) {
  if constexpr (PV < 0)
    any_load<R>(v, r, i, out);
  else
    any_load_p<R, PV>(v, r, i, out);
}
template <typename R, int PV>
__device__ __forceinline__ void vst(const AnyView& v, int r, long i, const Cx<R> in[12]) {
  if constexpr (PV < 0)
    any_store<R>(v, r, i, in);
  else
    any_store_p<R, PV>(v, r, i, in);
}
// the precision of the inner solution accumulator for inner vectors of precision PV
template <int PV>
__host__ __device__ constexpr int x_prec() {
  return PV < 0 ? -1 : (PV == P64 ? P64 : P32);
}

// ----------------------------------------------------------------------------- BiCGStab kernels
// beta = (rho_new / rho)(alpha / omega) is formed at the end of an iteration by
// k_bicg_check (and by the host when the recursion restarts); the first vector
// kernel of the next iteration moves rho_new into rho.

// p = r + beta (p - omega v); rho = rho_new
template <typename R, int PV = -1>
__global__ void k_bicg_p(AnyView r_, AnyView p_, AnyView v_, long n, Scal* sc, const int* ctl) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.y;
  Scal& s = sc[r];
  if (!s.active) return;
  const Cx<R> be = {(R)s.beta[0], (R)s.beta[1]}, om = {(R)s.omega[0], (R)s.omega[1]};
  if (blockIdx.x == 0 && threadIdx.x == 0) {  // no block of this kernel reads rho
    s.rho[0] = s.rho_new[0];
    s.rho[1] = s.rho_new[1];
  }
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vr[12], vp[12], vv[12];
    vld<R, PV>(r_, r, i, vr);
    vld<R, PV>(p_, r, i, vp);
    vld<R, PV>(v_, r, i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      Cx<R> w = vp[k] - cmul(om, vv[k]);
      vp[k] = vr[k] + cmul(be, w);
    }
    vst<R, PV>(p_, r, i, vp);
  }
}

// partial sums of (a, b) = sum conj(a) b  -> [re, im]
template <typename R, int PV = -1>
__global__ void k_cdot(AnyView a_, AnyView b_, long n, double* partial, const Scal* sc, const int* ctl) {
  pdl_enter();
  if (ctl && STOPPED(ctl)) return;
  int r = blockIdx.y;
  if (sc && !sc[r].active) return;
  double v[2] = {0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> va[12], vb[12];
    vld<R, PV>(a_, r, i, va);
    vld<R, PV>(b_, r, i, vb);
    Cx<R> acc = {R(0), R(0)};
#pragma unroll
    for (int k = 0; k < 12; ++k) acc = cjmadd(va[k], vb[k], acc);
    v[0] += (double)acc.re;
    v[1] += (double)acc.im;
  }
  write_partial<2>(v, partial, r);
}

// The scalars alpha and omega are formed by every block of the vector kernel
// that first needs them, from the partial sums the previous kernel left (the
// same sums in the same order in every block, so every block gets the same
// value); block 0 stores the value for later kernels and raises the flags.
// This saves a one-block kernel and its launch gap per scalar.
// nb_dev (may be null): number of partials written by a stencil with a fused reduction.

// alpha = rho / (rt, v); false (for every block) on NaN or breakdown
__device__ __forceinline__ bool block_alpha(Scal& s, const double* partial, int nb, int r, int* ctl,
                                            double2* al) {
  __shared__ double2 sh;
  __shared__ int ok;
  double d[2];
  sum_partials<2>(partial, nb, r, d);
  if (threadIdx.x == 0) {
    const double2 rv = make_double2(d[0], d[1]);
    const double2 rho = make_double2(s.rho[0], s.rho[1]);
    const double mag = sqrt(rv.x * rv.x + rv.y * rv.y);
    int flag = FLAG_NONE;
    if (bad(rv.x) || bad(rv.y))
      flag = FLAG_NAN;
    else if (mag <= 1e-300 || mag < 1e-24 * sqrt(rho.x * rho.x + rho.y * rho.y))
      flag = FLAG_BREAKDOWN;
    ok = flag == FLAG_NONE;
    if (ok) sh = cdiv(rho, rv);
    if (blockIdx.x == 0) {
      if (ok) {
        s.alpha[0] = sh.x;
        s.alpha[1] = sh.y;
      } else {
        s.flag = flag;
        *ctl = 1;
      }
    }
  }
  __syncthreads();
  *al = sh;
  return ok;
}

// omega = (t, s) / (t, t); false (for every block) on NaN or t = 0
__device__ __forceinline__ bool block_omega(Scal& s, const double* partial, int nb, int r, int* ctl,
                                            double2* om) {
  __shared__ double2 sh;
  __shared__ int ok;
  double d[3];
  sum_partials<3>(partial, nb, r, d);
  if (threadIdx.x == 0) {
    int flag = FLAG_NONE;
    if (bad(d[0]) || bad(d[1]) || bad(d[2]))
      flag = FLAG_NAN;
    else if (d[2] <= 0.0)  // t = 0: s is (numerically) zero or the operator annihilated it
      flag = FLAG_BREAKDOWN;
    ok = flag == FLAG_NONE;
    sh = ok ? make_double2(d[0] / d[2], d[1] / d[2]) : make_double2(0.0, 0.0);
    if (blockIdx.x == 0) {
      s.omega[0] = sh.x;
      s.omega[1] = sh.y;
      if (!ok) {
        s.flag = flag;
        *ctl = 1;
      }
    }
  }
  __syncthreads();
  *om = sh;
  return ok;
}

// alpha from the (rt, v) partials, then s = r - alpha v
template <typename R, int PV = -1>
__global__ void k_bicg_s(AnyView r_, AnyView v_, AnyView s_, long n, Scal* sc, int* ctl, const double* partial,
                         int nblk, const int* nb_dev) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.y;
  Scal& s = sc[r];
  if (!s.active) return;
  double2 a;
  if (!block_alpha(s, partial, nb_dev ? *nb_dev : nblk, r, ctl, &a)) return;
  const Cx<R> al = {(R)a.x, (R)a.y};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vr[12], vv[12];
    vld<R, PV>(r_, r, i, vr);
    vld<R, PV>(v_, r, i, vv);
#pragma unroll
    for (int k = 0; k < 12; ++k) vr[k] = vr[k] - cmul(al, vv[k]);
    vst<R, PV>(s_, r, i, vr);
  }
}

// partial sums of (t, s) [re, im] and |t|^2
template <typename R, int PV = -1>
__global__ void k_ts_tt(AnyView t_, AnyView s_, long n, double* partial, const Scal* sc, const int* ctl) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.y;
  if (!sc[r].active) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vt[12], vs[12];
    vld<R, PV>(t_, r, i, vt);
    vld<R, PV>(s_, r, i, vs);
    Cx<R> acc = {R(0), R(0)};
    R tt = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc = cjmadd(vt[k], vs[k], acc);
      tt = fma(vt[k].re, vt[k].re, fma(vt[k].im, vt[k].im, tt));
    }
    v[0] += (double)acc.re;
    v[1] += (double)acc.im;
    v[2] += (double)tt;
  }
  write_partial<3>(v, partial, r);
}

// omega from the (t, s), |t|^2 partials, then x += alpha p + omega s;  r = s - omega t;
// partials (rt, r) and |r|^2 into partial_out (not the array omega is read from)
template <typename R, typename RX, int PV = -1>
__global__ void k_bicg_xr(AnyView x_, AnyView p_, AnyView s_, AnyView t_, AnyView r_, AnyView rt_,
                          long n, const double* partial_in, int nblk, const int* nb_dev, double* partial_out,
                          Scal* sc, int* ctl) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.y;
  Scal& s = sc[r];
  if (!s.active) return;
  double2 o;
  if (!block_omega(s, partial_in, nb_dev ? *nb_dev : nblk, r, ctl, &o)) return;
  const Cx<R> al = {(R)s.alpha[0], (R)s.alpha[1]}, om = {(R)o.x, (R)o.y};
  const Cx<RX> alx = {(RX)s.alpha[0], (RX)s.alpha[1]}, omx = {(RX)o.x, (RX)o.y};
  double v[3] = {0.0, 0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    // every input first: the stores below may alias nothing the compiler can prove
    Cx<R> vp[12], vs[12], vt[12], vrt[12];
    Cx<RX> vx[12];
    vld<RX, x_prec<PV>()>(x_, r, i, vx);
    vld<R, PV>(p_, r, i, vp);
    vld<R, PV>(s_, r, i, vs);
    vld<R, PV>(t_, r, i, vt);
    vld<R, PV>(rt_, r, i, vrt);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      Cx<RX> pp = {(RX)vp[k].re, (RX)vp[k].im}, ss = {(RX)vs[k].re, (RX)vs[k].im};
      vx[k] = vx[k] + cmul(alx, pp) + cmul(omx, ss);
    }
    vst<RX, x_prec<PV>()>(x_, r, i, vx);
#pragma unroll
    for (int k = 0; k < 12; ++k) vs[k] = vs[k] - cmul(om, vt[k]);
    vst<R, PV>(r_, r, i, vs);
    Cx<R> acc = {R(0), R(0)};
    R rr = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc = cjmadd(vrt[k], vs[k], acc);
      rr = fma(vs[k].re, vs[k].re, fma(vs[k].im, vs[k].im, rr));
    }
    v[0] += (double)acc.re;
    v[1] += (double)acc.im;
    v[2] += (double)rr;
  }
  write_partial<3>(v, partial_out, r);
}

// end of an iteration: rho_new, |r|^2, iteration count, stop decisions
// and the next beta; with decide != 0 any flag stops the chunk at once (the outer
// step is then made for the right-hand sides that have flagged; waiting for others
// to flag too was measured to cost iterations: 12 point sources at 24^3 x 48 ran
// 49-53 iterations with a two-iteration wait, 46-49 without)
__global__ void k_bicg_check(Scal* sc, const double* partial, int nblk, int* ctl, int decide) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.x;
  Scal& s = sc[r];
  if (!s.active) return;
  double d[3];
  sum_partials<3>(partial, nblk, r, d);
  if (threadIdx.x) return;
  s.iters += 1;
  s.rho_new[0] = d[0];
  s.rho_new[1] = d[1];
  s.r2 = d[2];
  if (bad(d[0]) || bad(d[1]) || bad(d[2])) {
    s.flag = FLAG_NAN;
  } else if (d[2] <= s.stop2) {
    s.flag = FLAG_CHECK;
  } else if (s.delta2 > 0.0 && d[2] <= s.delta2 * s.r2_ref) {
    s.flag = FLAG_UPDATE;
  }
  const double2 b = cmul2(cdiv(make_double2(d[0], d[1]), make_double2(s.rho[0], s.rho[1])),
                          cdiv(make_double2(s.alpha[0], s.alpha[1]), make_double2(s.omega[0], s.omega[1])));
  s.beta[0] = b.x;
  s.beta[1] = b.y;
  if (decide && s.flag != FLAG_NONE) *ctl = 1;
}

// ----------------------------------------------------------------------------- CG kernels
// beta = rr_new / rr is formed at the end of an iteration by k_cg_check (and by
// the host when the recursion restarts); the first vector kernel of the next
// iteration moves rr_new into rr.

// p = r + beta p; rr = rr_new
template <typename R, int PV = -1>
__global__ void k_cg_p(AnyView r_, AnyView p_, long n, Scal* sc, const int* ctl) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.y;
  Scal& s = sc[r];
  if (!s.active) return;
  const R be = (R)s.beta[0];
  if (blockIdx.x == 0 && threadIdx.x == 0) s.rr = s.rr_new;  // no block of this kernel reads rr
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vr[12], vp[12];
    vld<R, PV>(r_, r, i, vr);
    vld<R, PV>(p_, r, i, vp);
#pragma unroll
    for (int k = 0; k < 12; ++k) vp[k] = {fma(be, vp[k].re, vr[k].re), fma(be, vp[k].im, vr[k].im)};
    vst<R, PV>(p_, r, i, vp);
  }
}

// alpha = rr / Re(p, q) from the k_rdot partials, formed by every block (see
// block_alpha); false (for every block) on NaN or breakdown
__device__ __forceinline__ bool block_cg_alpha(Scal& s, const double* partial, int nb, int r, int* ctl,
                                               double* al) {
  __shared__ double sh;
  __shared__ int ok;
  double d[2];
  sum_partials<2>(partial, nb, r, d);
  if (threadIdx.x == 0) {
    const int flag = bad(d[0]) ? FLAG_NAN : (d[0] <= 0.0 ? FLAG_BREAKDOWN : FLAG_NONE);
    ok = flag == FLAG_NONE;
    sh = ok ? s.rr / d[0] : 0.0;
    if (blockIdx.x == 0) {
      if (ok) {
        s.alpha[0] = sh;
        s.alpha[1] = 0.0;
      } else {
        s.flag = flag;
        *ctl = 1;
      }
    }
  }
  __syncthreads();
  *al = sh;
  return ok;
}

// alpha from the Re(p, q) partials, then x += alpha p; r -= alpha q; partial |r|^2
// into partial_out (not the array alpha is read from)
template <typename R, typename RX, int PV = -1>
__global__ void k_cg_xr(AnyView x_, AnyView p_, AnyView q_, AnyView r_, long n, const double* partial_in,
                        int nblk, const int* nb_dev, double* partial_out, Scal* sc, int* ctl) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.y;
  Scal& s = sc[r];
  if (!s.active) return;
  double a;
  if (!block_cg_alpha(s, partial_in, nb_dev ? *nb_dev : nblk, r, ctl, &a)) return;
  const R al = (R)a;
  const RX alx = (RX)a;
  double v[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vp[12], vq[12], vr[12];
    Cx<RX> vx[12];
    vld<RX, x_prec<PV>()>(x_, r, i, vx);
    vld<R, PV>(p_, r, i, vp);
    vld<R, PV>(q_, r, i, vq);
    vld<R, PV>(r_, r, i, vr);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      vx[k] = {fma(alx, (RX)vp[k].re, vx[k].re), fma(alx, (RX)vp[k].im, vx[k].im)};
    vst<RX, x_prec<PV>()>(x_, r, i, vx);
    R rr = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      vr[k] = {fma(-al, vq[k].re, vr[k].re), fma(-al, vq[k].im, vr[k].im)};
      rr = fma(vr[k].re, vr[k].re, fma(vr[k].im, vr[k].im, rr));
    }
    vst<R, PV>(r_, r, i, vr);
    v[0] += (double)rr;
  }
  write_partial<1>(v, partial_out, r);
}

// end of an iteration: rr_new, flags and the next beta; decide as in k_bicg_check
__global__ void k_cg_check(Scal* sc, const double* partial, int nblk, int* ctl, int decide) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.x;
  Scal& s = sc[r];
  if (!s.active) return;
  double d[1];
  sum_partials<1>(partial, nblk, r, d);
  if (threadIdx.x) return;
  s.iters += 1;
  s.rr_new = d[0];
  s.r2 = d[0];
  if (bad(d[0]))
    s.flag = FLAG_NAN;
  else if (d[0] <= s.stop2)
    s.flag = FLAG_CHECK;
  else if (s.delta2 > 0.0 && d[0] <= s.delta2 * s.r2_ref)
    s.flag = FLAG_UPDATE;
  s.beta[0] = d[0] / s.rr;
  s.beta[1] = 0.0;
  if (decide && s.flag != FLAG_NONE) *ctl = 1;
}

// partial sums of Re(a, b)
template <typename R, int PV = -1>
__global__ void k_rdot(AnyView a_, AnyView b_, long n, double* partial, const Scal* sc, const int* ctl) {
  pdl_enter();
  if (STOPPED(ctl)) return;
  int r = blockIdx.y;
  if (!sc[r].active) return;
  double v[2] = {0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> va[12], vb[12];
    vld<R, PV>(a_, r, i, va);
    vld<R, PV>(b_, r, i, vb);
    R acc = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc = fma(va[k].re, vb[k].re, fma(va[k].im, vb[k].im, acc));
    v[0] += (double)acc;
  }
  write_partial<2>(v, partial, r);
}

__global__ void k_reset(int* ctl) { *ctl = 0; }

// Blocks of a grid-stride iteration kernel: one full wave (its resident blocks per SM
// times the SMs; fewer for short vectors), so that no partly filled last wave leaves
// SMs idle (the FP32 x / r update holds 3 blocks per SM; launched as 4 per SM, its
// second wave ran on a third of the slots).
unsigned wave_blocks(const void* kernel, long n) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> occ;  // resident blocks per SM, per device
  int dev = 0;
  QCD_CK(cudaGetDevice(&dev));
  int o = 1;
  {
    std::lock_guard<std::mutex> lk(mu);
    auto it = occ.find({dev, kernel});
    if (it == occ.end()) {
      int v = 0;
      QCD_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kernel, kThreads, 0));
      it = occ.emplace(std::make_pair(dev, kernel), std::max(v, 1)).first;
    }
    o = it->second;
  }
  const long need = (n + kThreads - 1) / kThreads;
  return (unsigned)std::max(1L, std::min(need, (long)o * sm_count()));
}
// the most blocks per SM any of them can have (2048 threads of 256): the partial-sum arrays' size
constexpr int kMaxBlocksPerSM = 8;

// blocks of the host-side inner products (cdot_host): 4 per SM
unsigned red_blocks(long n) {
  long b = (n + kThreads - 1) / kThreads;
  long cap = 4L * sm_count();
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

// ----------------------------------------------------------------------------- the solver
struct Solver {
  qcd_gauge* g;
  qcd_fermion f;
  qcd_solver_params prm;
  int nrhs, ls;
  int inner;     // precision of the inner vectors
  int xprec;     // precision of the inner solution accumulator
  cudaStream_t st;
  OpCtx op64, opin;
  // device state
  Scal* sc = nullptr;
  int* ctl = nullptr;
  double* partial = nullptr;
  double* partial2 = nullptr;  // the end-of-iteration partials (k_bicg_xr reads omega's from `partial`)
  double* bpartial = nullptr;  // per-block partials of the fused stencil reductions
  int* counters = nullptr;     // their group counters (zero between launches)
  unsigned nblk = 1;  // blocks of cdot_host (red_blocks); the iteration kernels size their own grids
  // fields
  Field b_e, b_o, bh, x64, r64, t64, u64, xo64, re64;  // FP64
  Field r, rt, p, v, s, t, q, w, xin;        // inner
  std::vector<Scal> hsc;

  bool bicg() const { return prm.method == QCD_BICGSTAB; }
  // BiCGStab inner products fused into the stencil epilogue: one Wilson
  // right-hand side (group sums by the stencil's last blocks), or several stored
  // in FP32 (per-warp partials summed per rhs)
  bool fused() const { return bicg() && f.type == QCD_WILSON && nrhs == 1; }
  bool fused_multi() const { return bicg() && f.type == QCD_WILSON && nrhs > 1 && inner == QCD_F32; }
  // CG: Re(p, q) formed in the epilogue of the last stencil of Mhat^dag (FP32 or FP16;
  // per-warp partials summed per slice when there are several slices, else group sums)
  bool fused_cg() const { return !bicg() && (inner == QCD_F32 || inner == QCD_F16); }
  bool cg_single() const { return fused_cg() && nrhs * ls == 1; }
  long n() const { return r.nsites(); }

  void body() {
    const long nn = n();
    const int dag = prm.dagger;
    if (inner == QCD_F64)
      body_t<double, double, P64>(nn, dag);
    else if (inner == QCD_F32)
      body_t<float, float, P32>(nn, dag);
    else
      body_t<float, float, P16>(nn, dag);
  }

  // grid of a grid-stride kernel over all right-hand sides (one wave per rhs row)
  template <typename K>
  dim3 wave(K kernel, long nn) const {
    return dim3(wave_blocks((const void*)kernel, nn), nrhs);
  }

  // PV: the storage precision of the inner vectors (the solution accumulator is FP64
  // with FP64 vectors, else FP32).  A kernel that writes per-block partial sums hands
  // its block count to the one that reads them.
  template <typename R, typename RX, int PV>
  void body_t(long nn, int dag) {
    if (bicg()) {
      int nb_ts = 0;  // partials of (t, s), |t|^2 from k_ts_tt (the unfused path)
      launch_k(k_bicg_p<R, PV>, wave(k_bicg_p<R, PV>, nn), kThreads, 0, st, any_view(r), any_view(p), any_view(v),
               nn, sc, ctl);
      QCD_LAUNCH_CK();
      if (fused()) {
        // (rt, v) and (t, s), |t|^2 formed in the epilogue of the stencil that writes v / t
        int* npart = ctl + 2;
        RedSpec red1{1, &rt, bpartial, partial, counters, npart};
        RedSpec red2{2, nullptr, bpartial, partial, counters, npart};
        apply_mhat(opin, p, v, dag, st, "in", ctl, &red1);
        launch_k(k_bicg_s<R, PV>, wave(k_bicg_s<R, PV>, nn), kThreads, 0, st, any_view(r), any_view(v), any_view(s),
                 nn, sc, ctl, partial, 0, npart);
        QCD_LAUNCH_CK();
        apply_mhat(opin, s, t, dag, st, "in", ctl, &red2);
      } else if (fused_multi()) {
        // per-rhs sums land in partial[rhs * 4 + k]: one partial per right-hand side
        RedSpec red1{1, &rt, bpartial, partial, nullptr, nullptr};
        RedSpec red2{2, nullptr, bpartial, partial, nullptr, nullptr};
        apply_mhat(opin, p, v, dag, st, "in", ctl, &red1);
        launch_k(k_bicg_s<R, PV>, wave(k_bicg_s<R, PV>, nn), kThreads, 0, st, any_view(r), any_view(v), any_view(s),
                 nn, sc, ctl, partial, 1, nullptr);
        QCD_LAUNCH_CK();
        apply_mhat(opin, s, t, dag, st, "in", ctl, &red2);
      } else {
        apply_mhat(opin, p, v, dag, st, "in", ctl);
        const dim3 gc = wave(k_cdot<R, PV>, nn);
        launch_k(k_cdot<R, PV>, gc, kThreads, 0, st, any_view(rt), any_view(v), nn, partial, sc, ctl);
        QCD_LAUNCH_CK();
        launch_k(k_bicg_s<R, PV>, wave(k_bicg_s<R, PV>, nn), kThreads, 0, st, any_view(r), any_view(v), any_view(s),
                 nn, sc, ctl, partial, (int)gc.x, nullptr);
        QCD_LAUNCH_CK();
        apply_mhat(opin, s, t, dag, st, "in", ctl);
        const dim3 gt = wave(k_ts_tt<R, PV>, nn);
        launch_k(k_ts_tt<R, PV>, gt, kThreads, 0, st, any_view(t), any_view(s), nn, partial, sc, ctl);
        QCD_LAUNCH_CK();
        nb_ts = (int)gt.x;
      }
      const dim3 gx = wave(k_bicg_xr<R, RX, PV>, nn);
      launch_k(k_bicg_xr<R, RX, PV>, gx, kThreads, 0, st, any_view(xin), any_view(p), any_view(s), any_view(t),
               any_view(r), any_view(rt), nn, partial, fused_multi() ? 1 : nb_ts, fused() ? ctl + 2 : nullptr,
               partial2, sc, ctl);
      QCD_LAUNCH_CK();
      launch_k(k_bicg_check, nrhs, kThreads, 0, st, sc, partial2, (int)gx.x, ctl, 1);
      QCD_LAUNCH_CK();
    } else {
      launch_k(k_cg_p<R, PV>, wave(k_cg_p<R, PV>, nn), kThreads, 0, st, any_view(r), any_view(p), nn, sc, ctl);
      QCD_LAUNCH_CK();
      apply_mhat(opin, p, w, dag, st, "in", ctl);  // A p, A = Mhat (Mhat^dag for the adjoint system)
      int nb = 0;
      const int* nb_dev = nullptr;
      if (fused_cg()) {  // (p, q) in the epilogue of q = Mhat^dag w
        int* npart = ctl + 2;
        RedSpec red{1, &p, bpartial, partial, counters, npart};
        apply_mhat(opin, w, q, 1 - dag, st, "in", ctl, &red);
        if (cg_single())
          nb_dev = npart;
        else
          nb = ls;  // one sum per slice
      } else {
        apply_mhat(opin, w, q, 1 - dag, st, "in", ctl);
        const dim3 gr = wave(k_rdot<R, PV>, nn);
        launch_k(k_rdot<R, PV>, gr, kThreads, 0, st, any_view(p), any_view(q), nn, partial, sc, ctl);
        QCD_LAUNCH_CK();
        nb = (int)gr.x;
      }
      const dim3 gx = wave(k_cg_xr<R, RX, PV>, nn);
      launch_k(k_cg_xr<R, RX, PV>, gx, kThreads, 0, st, any_view(xin), any_view(p), any_view(q), any_view(r), nn,
               partial, nb, nb_dev, partial2, sc, ctl);
      QCD_LAUNCH_CK();
      launch_k(k_cg_check, nrhs, kThreads, 0, st, sc, partial2, (int)gx.x, ctl, 1);
      QCD_LAUNCH_CK();
    }
  }

  // Everything a captured chunk bakes into its kernel arguments: the fields'
  // addresses (and the workspace generation, which changes whenever a buffer
  // is reallocated), the operator's parameters and the chunk length.
  std::string graph_key(int k) const {
    char buf[512];
    snprintf(buf, sizeof buf, "m%d i%d n%d l%d d%d t%d k%a M%a m%a L%d ws%ld c%d sc%p %p %p %p %p %p %p %p %p %p %p %p",
             prm.method, inner, nrhs, ls, prm.dagger, f.type, f.kappa, f.M5, f.mf, f.Ls, g->ws.generation, k,
             (void*)sc, (void*)ctl, (void*)partial, (void*)partial2, r.data, p.data, v.data, s.data, t.data, q.data,
             w.data, rt.data);
    const DwParams dp = dw_params(f);  // b5, c5 of a Mobius operator (1, 0 otherwise)
    snprintf(buf + strlen(buf), sizeof buf - strlen(buf), " b%a c%a", dp.b5, dp.c5);
    return std::string(buf) + " x" + std::to_string((uintptr_t)xin.data);
  }

  void run_chunk(int k, bool graph) {
    if (graph) {
      std::string key = graph_key(k);
      auto it = g->graphs.find(key);
      if (it == g->graphs.end()) {
        cudaGraph_t gr;
        long c0 = launches_so_far();
        QCD_CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        k_reset<<<1, 1, 0, st>>>(ctl);
        QCD_LAUNCH_CK();
        for (int i = 0; i < k; ++i) body();
        QCD_CK(cudaStreamEndCapture(st, &gr));
        CachedGraph cg;
        cg.nodes = launches_so_far() - c0;  // captured, not yet executed
        set_launches(c0);
        QCD_CK(cudaGraphInstantiate(&cg.exec, gr, 0));
        cudaGraphDestroy(gr);
        it = g->graphs.emplace(key, cg).first;
      }
      QCD_CK(cudaGraphLaunch(it->second.exec, st));
      note_launches(it->second.nodes);
    } else {
      k_reset<<<1, 1, 0, st>>>(ctl);
      QCD_LAUNCH_CK();
      for (int i = 0; i < k; ++i) body();
    }
  }

  void upload() {
    QCD_CK(cudaMemcpyAsync(sc, hsc.data(), sizeof(Scal) * nrhs, cudaMemcpyHostToDevice, st));
  }
  void download() {
    QCD_CK(cudaMemcpyAsync(hsc.data(), sc, sizeof(Scal) * nrhs, cudaMemcpyDeviceToHost, st));
    QCD_CK(cudaStreamSynchronize(st));
  }

  // host-side complex dot products (rt, r) per rhs (synchronises)
  void cdot_host(const Field& a, const Field& b, std::vector<double>& re, std::vector<double>& im) {
    const int nrhs = a.nrhs;
    dim3 grid(nblk, nrhs);
    if (a.prec == QCD_F64)
      launch_k(k_cdot<double>, grid, kThreads, 0, st, any_view(a), any_view(b), a.nsites(), partial, nullptr,
                                                nullptr);
    else
      launch_k(k_cdot<float>, grid, kThreads, 0, st, any_view(a), any_view(b), a.nsites(), partial, nullptr,
                                               nullptr);
    QCD_LAUNCH_CK();
    std::vector<double> h((size_t)nblk * nrhs * kMaxPartial);
    QCD_CK(cudaMemcpyAsync(h.data(), partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    QCD_CK(cudaStreamSynchronize(st));
    re.assign(nrhs, 0.0);
    im.assign(nrhs, 0.0);
    for (int r2 = 0; r2 < nrhs; ++r2)
      for (unsigned b = 0; b < nblk; ++b) {
        re[r2] += h[((size_t)r2 * nblk + b) * kMaxPartial];
        im[r2] += h[((size_t)r2 * nblk + b) * kMaxPartial + 1];
      }
  }
};

}  // namespace

// Solve on device canonical buffers (b, x: (nrhs, ls, V, 4, 3) complex128).
void solve_device(qcd_gauge* g, const qcd_fermion& f, const qcd_solver_params& prm, const double* b,
                  double* x, int nrhs, qcd_solve_info* info, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  const Lattice& lat = g->lat;
  Solver S;
  S.g = g;
  S.f = f;
  S.prm = prm;
  S.nrhs = nrhs;
  S.ls = is_dw(f) ? f.Ls : 1;
  S.inner = prm.inner;
  S.xprec = prm.inner == QCD_F64 ? QCD_F64 : QCD_F32;
  S.st = st;
  S.op64 = {g, f, QCD_F64};
  S.opin = {g, f, prm.inner};
  const int ls = S.ls;
  const bool dwf = is_dw(f);
  const int dag = prm.dagger;
  // default reliable-update factor: two decades between outer steps for FP32 and for FP16
  // inner vectors (the FP16 spinors are scaled per site; measured at 32^3 x 64 Wilson and
  // 16^3 x 32 x 16 domain-wall, 0.01 takes as many iterations as 0.1 with half the outer steps)
  const double delta = (prm.delta > 0 && prm.delta < 1) ? prm.delta : 0.01;

  S.b_e = ws_field(g, "s.b_e", QCD_F64, ls, nrhs);
  S.b_o = ws_field(g, "s.b_o", QCD_F64, ls, nrhs);
  S.bh = ws_field(g, "s.bh", QCD_F64, ls, nrhs);
  S.x64 = ws_field(g, "s.x64", QCD_F64, ls, nrhs);
  S.r64 = ws_field(g, "s.r64", QCD_F64, ls, nrhs);
  S.t64 = ws_field(g, "s.t64", QCD_F64, ls, nrhs);
  S.u64 = ws_field(g, "s.u64", QCD_F64, ls, nrhs);
  // IEEE-FP64 outer steps of the Wilson solve keep the reconstructed odd half of x
  const bool wil64 = !dwf && !(prm.outer == QCD_DF64 && S.inner != QCD_F64);
  if (wil64) S.xo64 = ws_field(g, "s.xo64", QCD_F64, ls, nrhs);
  // ... and the even half r_e of the full-system residual: the inner residual itself for
  // BiCGStab, the source of Mhat^dag r_e for CG on the normal equations
  if (wil64 && !S.bicg()) S.re64 = ws_field(g, "s.re64", QCD_F64, ls, nrhs);
  Field& r_e64 = S.bicg() ? S.r64 : S.re64;
  S.r = ws_field(g, "s.r", S.inner, ls, nrhs);
  S.p = ws_field(g, "s.p", S.inner, ls, nrhs);
  if (S.bicg()) {
    S.rt = ws_field(g, "s.rt", S.inner, ls, nrhs);
    S.v = ws_field(g, "s.v", S.inner, ls, nrhs);
    S.s = ws_field(g, "s.s", S.inner, ls, nrhs);
    S.t = ws_field(g, "s.t", S.inner, ls, nrhs);
  } else {
    S.q = ws_field(g, "s.q", S.inner, ls, nrhs);
    S.w = ws_field(g, "s.w", S.inner, ls, nrhs);
  }
  S.xin = (S.inner == QCD_F64) ? S.x64 : ws_field(g, "s.xin", S.xprec, ls, nrhs);
  S.nblk = red_blocks(S.r.nsites());
  S.sc = (Scal*)g->ws.get("s.scal", sizeof(Scal) * nrhs);
  S.ctl = (int*)g->ws.get("s.ctl", sizeof(int) * 4);
  // partials of the reduction kernels (and the group sums of the fused stencil
  // reductions); per-block partials of the fused reductions (blocks of >= 64
  // sites) and one counter per group of 64 blocks, zeroed once here
  const size_t nstencil_blocks = (size_t)(lat.Vh / 64 + 1);
  const size_t nwave = (size_t)std::max<long>(S.nblk, (long)kMaxBlocksPerSM * sm_count());  // grid of any wave
  const size_t npart = std::max<size_t>(nwave * nrhs, nstencil_blocks / 64 + 1);
  S.partial = (double*)g->ws.get("s.partial", sizeof(double) * npart * kMaxPartial);
  S.partial2 = (double*)g->ws.get("s.partial2", sizeof(double) * nwave * nrhs * kMaxPartial);
  if (S.fused_multi() || (S.fused_cg() && !S.cg_single()))  // per-warp partials of every slice
    S.bpartial = (double*)g->ws.get("s.bpartialN",
                                    sizeof(double) * (size_t)nrhs * ls * ((lat.Vh + 31) / 32) * kMaxPartial);
  if (S.fused() || S.cg_single()) {
    S.bpartial = (double*)g->ws.get("s.bpartial", sizeof(double) * nstencil_blocks * kMaxPartial);
    const size_t ngroups = nstencil_blocks / 64 + 2;
    const long gen = g->ws.generation;
    S.counters = (int*)g->ws.get("s.counters", sizeof(int) * ngroups);
    if (g->ws.generation != gen) QCD_CK(cudaMemsetAsync(S.counters, 0, sizeof(int) * ngroups, st));
  }
  S.hsc.assign(nrhs, Scal{});
  // Double-float outer steps (mixed solves): the prepared source, the solution
  // and the outer residual live in FP32 pairs and the outer operator
  // applications use the double-float stencil (and A^-1 for domain-wall); the
  // true residual reported at the end is recomputed with the IEEE-FP64
  // operator all the same.
  const bool dfo = prm.outer == QCD_DF64 && S.inner != QCD_F64;
  const OpCtx opdf{g, f, QCD_DF64};
  Field be_d, bo_d, bh_d, x_d, t_d, u_d, r_d;
  if (dfo) {
    be_d = ws_field(g, "s.be_d", QCD_DF64, ls, nrhs);
    bo_d = ws_field(g, "s.bo_d", QCD_DF64, ls, nrhs);
    bh_d = ws_field(g, "s.bh_d", QCD_DF64, ls, nrhs);
    x_d = ws_field(g, "s.x_d", QCD_DF64, ls, nrhs);
    t_d = ws_field(g, "s.t_d", QCD_DF64, ls, nrhs);
    u_d = ws_field(g, "s.u_d", QCD_DF64, ls, nrhs);
    if (!S.bicg()) r_d = ws_field(g, "s.r_d", QCD_DF64, ls, nrhs);
  }
  const Field& r_outer = dfo ? (S.bicg() ? t_d : r_d) : S.r64;
  // CG on the normal equations: the outer step computes the true residual rhat = bhat -
  // Mhat x in the outer precision, where its cancellation happens, and the inner solver's
  // residual Mhat^dag rhat with the inner operator (it is needed only to the inner
  // precision), straight into the inner vector r
  const bool cg_inner_normal = !S.bicg() && S.inner != QCD_F64;

  // ---- even-odd source: b_hat on the even sites
  pack_field(lat, 0, b, S.b_e, st);
  pack_field(lat, 1, b, S.b_o, st);
  std::vector<double> bn_e(nrhs), bn_o(nrhs), bnorm(nrhs);
  blas_norm2(S.b_e, bn_e.data(), st, g);
  blas_norm2(S.b_o, bn_o.data(), st, g);
  for (int r = 0; r < nrhs; ++r) bnorm[r] = std::sqrt(bn_e[r] + bn_o[r]);
  const DwParams dp = dw_params(f);
  if (dfo) {
    blas_copy(S.b_e, be_d, st);
    blas_copy(S.b_o, bo_d, st);
    if (!dwf) {
      hop_df(g, bo_d, bh_d, 0, dag, f.kappa, &be_d, nullptr, 0.0, st);
    } else {
      dw_ainv(dp, bo_d, t_d, 0, 1.0, nullptr, st);
      hop(g, t_d, u_d, 0, 0, 0.5, &be_d, st);
      dw_ainv(dp, u_d, bh_d, 0, 1.0, nullptr, st);
    }
  } else if (!dwf) {
    // bhat = b_e + kappa H_eo b_o
    hop(g, S.b_o, S.bh, 0, dag, f.kappa, &S.b_e, st);
  } else {
    // bhat = W (b_e + 1/2 H_eo W b_o), W = B A^-1 (A^-1 for Shamir)
    dw_ainv(dp, S.b_o, S.t64, 0, 1.0, nullptr, st);
    hop(g, S.t64, S.u64, 0, 0, 0.5, &S.b_e, st);
    dw_ainv(dp, S.u64, S.bh, 0, 1.0, nullptr, st);
  }
  if (prm.x0_given && dwf && dp.mobius()) {
    pack_field(lat, 0, x, S.t64, st);
    dw_block(dp, S.t64, S.x64, 0, 0.0, nullptr, st, BLK_B);  // x' = B x
  } else if (prm.x0_given) {
    pack_field(lat, 0, x, S.x64, st);
  } else {
    blas_zero(S.x64, st);
  }
  if (dfo) {
    if (prm.x0_given)
      blas_copy(S.x64, x_d, st);
    else
      blas_zero(x_d, st);
  }

  // |b - A x| on the full system from the even-odd residual rhat = bhat - Mhat x_e:
  // Wilson: (rhat, 0);  DWF: (A B^-1 rhat, 0)  (exact reconstruction of x_o)
  std::vector<double> rn(nrhs), rfull(nrhs);
  // Outer-step pieces act on the right-hand sides [r0, r0 + n): views of the fields
  // restricted to them (the whole field when n = nrhs)
  auto sub = [&](const Field& f, int r0, int n) { return n == nrhs ? f : f.rhs_range(r0, n); };
  auto normal_residual = [&](const Field& rhat, int r0, int n) {
    Field w = sub(S.w, r0, n), r = sub(S.r, r0, n);
    blas_copy(rhat, w, st);
    apply_mhat(S.opin, w, r, 1 - dag, st, "in");  // A^dag rhat
    blas_norm2(r, rn.data() + r0, st, g);
  };
  auto true_residual = [&](bool x_is_zero, int r0, int n) {
    double* rf = rfull.data() + r0;
    Field t64 = sub(S.t64, r0, n), u64 = sub(S.u64, r0, n), x64 = sub(S.x64, r0, n), bh = sub(S.bh, r0, n);
    Field r64 = sub(S.r64, r0, n);
    if (dfo) {
      Field td = sub(t_d, r0, n), xd = sub(x_d, r0, n), ud = sub(u_d, r0, n), bhd = sub(bh_d, r0, n);
      if (x_is_zero) {
        blas_copy(bhd, td, st);
      } else if (!dwf) {
        // rhat = bhat - x + kappa^2 H_eo H_oe x  (H -> H^dag for the adjoint system)
        hop_df(g, xd, ud, 1, dag, 1.0, nullptr, nullptr, 0.0, st);
        hop_df(g, ud, td, 0, dag, f.kappa * f.kappa, &bhd, &xd, -1.0, st);
      } else {
        apply_mhat(opdf, xd, td, dag, st, "odf");
        blas_axpby(1.0, bhd, -1.0, td, st);  // rhat = bhat - Mhat x
      }
      if (dwf) {  // |A rhat| (to FP64 for the block A; it decides no more than the stop)
        blas_copy(td, t64, st);
        dw_a_binv(dp, t64, u64, st);
        blas_norm2(u64, rf, st, g);
      } else {
        blas_norm2(td, rf, st, g);
      }
      for (int r = r0; r < r0 + n; ++r) rfull[r] = std::sqrt(rfull[r]);
      if (cg_inner_normal) {
        normal_residual(td, r0, n);
        return;
      }
      blas_norm2(sub(r_outer, r0, n), rn.data() + r0, st, g);
      return;
    }
    if (wil64) {
      // Wilson with IEEE-FP64 outer steps: reconstruct x_o = b_o + kappa h, h = H_oe x_e,
      // and form the even half of the full-system residual,
      //   r_e = b_e - x_e + kappa H_eo x_o  (= bhat - Mhat x_e; the odd half is zero up to
      // the rounding of x_o), so that the outer step that reaches the target has already
      // computed the final solution and its true residual.
      Field re = sub(r_e64, r0, n), xo = sub(S.xo64, r0, n), bo = sub(S.b_o, r0, n), be = sub(S.b_e, r0, n);
      if (x_is_zero) {
        blas_copy(bh, re, st);  // x = (0, b_o): r_e = bhat, h = 0
        blas_copy(bo, xo, st);
        blas_zero(u64, st);
      } else {
        hop(g, x64, u64, 1, dag, 1.0, nullptr, st);  // h
        blas_copy(bo, xo, st);
        blas_axpby(f.kappa, u64, 1.0, xo, st);  // x_o
        blas_copy(be, t64, st);
        blas_axpby(-1.0, x64, 1.0, t64, st);  // b_e - x_e
        hop(g, xo, re, 0, dag, f.kappa, &t64, st);  // r_e
      }
      blas_norm2(re, rf, st, g);
      for (int r = r0; r < r0 + n; ++r) rfull[r] = std::sqrt(rfull[r]);
      // the inner residual: r_e (BiCGStab) or A^dag r_e (CG; A = Mhat, Mhat^dag for the adjoint)
      if (cg_inner_normal) {
        normal_residual(re, r0, n);
        return;
      }
      if (!S.bicg()) apply_mhat(S.op64, re, r64, 1 - dag, st, "o64");
      blas_norm2(r64, rn.data() + r0, st, g);
      return;
    }
    if (x_is_zero) {
      blas_copy(bh, t64, st);  // rhat = bhat
    } else {
      apply_mhat(S.op64, x64, t64, dag, st, "o64");
      blas_axpby(1.0, bh, -1.0, t64, st);  // t64 = bhat - Mhat x
    }
    if (dwf) {
      dw_a_binv(dp, t64, u64, st);
      blas_norm2(u64, rf, st, g);
    } else {
      blas_norm2(t64, rf, st, g);
    }
    for (int r = r0; r < r0 + n; ++r) rfull[r] = std::sqrt(rfull[r]);
    // the inner residual: rhat (BiCGStab) or A^dag rhat (CG; A = Mhat, Mhat^dag for the adjoint)
    if (cg_inner_normal) {
      normal_residual(t64, r0, n);
      return;
    }
    if (S.bicg()) {
      blas_copy(t64, r64, st);
    } else {
      apply_mhat(S.op64, t64, r64, 1 - dag, st, "o64");
    }
    blas_norm2(r64, rn.data() + r0, st, g);
  };

  true_residual(!prm.x0_given, 0, nrhs);
  std::vector<double> target(nrhs);
  std::vector<int> conv(nrhs, 0), status(nrhs, QCD_OK), updates(nrhs, 0), restarts(nrhs, 0);
  int nactive = 0;
  for (int r = 0; r < nrhs; ++r) {
    target[r] = prm.tol * bnorm[r];
    if (!std::isfinite(bnorm[r])) {  // NaN or Inf in the source: nothing to iterate on
      status[r] = QCD_ERR_NAN;
      conv[r] = 2;
    } else if (bnorm[r] == 0.0 || rfull[r] <= target[r]) {
      conv[r] = 1;
    } else {
      ++nactive;
    }
  }

  auto restart_from_residual = [&](bool full, int r0, int n) {
    // r (inner) = outer residual; the recursion continues from the true residual
    Field r = sub(S.r, r0, n), rt = sub(S.rt, r0, n), p = sub(S.p, r0, n), v = sub(S.v, r0, n);
    if (!cg_inner_normal) blas_copy(sub(r_outer, r0, n), r, st);
    if (S.inner != QCD_F64) {
      Field xin = sub(S.xin, r0, n);
      blas_zero(xin, st);
    }
    std::vector<double> re, im;
    if (S.bicg()) {
      if (full) {
        blas_copy(r, rt, st);
        blas_zero(p, st);
        blas_zero(v, st);
      }
      S.cdot_host(rt, r, re, im);
    }
    for (int k = 0; k < n; ++k) {
      const int rr = r0 + k;
      Scal& s = S.hsc[rr];
      s.active = !conv[rr];
      s.flag = FLAG_NONE;
      s.r2_ref = rn[rr];
      s.r2 = rn[rr];
      // inner phase ends for a true-residual check at the scaled target
      double ratio = rfull[rr] > 0 ? std::sqrt(rn[rr]) / rfull[rr] : 1.0;
      double tgt = 0.5 * target[rr] * ratio;
      s.stop2 = tgt * tgt;
      s.delta2 = (S.inner == QCD_F64) ? 0.0 : delta * delta;
      if (S.bicg()) {
        if (full) {
          s.rho[0] = 1.0, s.rho[1] = 0.0;
          s.alpha[0] = 1.0, s.alpha[1] = 0.0;
          s.omega[0] = 1.0, s.omega[1] = 0.0;
        }
        s.rho_new[0] = re[k];
        s.rho_new[1] = im[k];
        // the first iteration's beta (later ones are formed by k_bicg_check)
        const std::complex<double> b = (std::complex<double>(s.rho_new[0], s.rho_new[1]) /
                                        std::complex<double>(s.rho[0], s.rho[1])) *
                                       (std::complex<double>(s.alpha[0], s.alpha[1]) /
                                        std::complex<double>(s.omega[0], s.omega[1]));
        s.beta[0] = b.real();
        s.beta[1] = b.imag();
      } else {
        if (full) s.rr = 1.0;
        s.rr_new = rn[rr];
        s.beta[0] = s.rr_new / s.rr;  // the first iteration's beta (p = 0 after a full restart)
        s.beta[1] = 0.0;
      }
    }
    if (full && !S.bicg()) blas_zero(p, st);
  };

  for (int r = 0; r < nrhs; ++r) S.hsc[r].iters = 0;
  if (nactive > 0) restart_from_residual(true, 0, nrhs);
  S.upload();

  // host-side fault injection for tests (no device fault is ever provoked):
  // QCD_FAULT=nan poisons the inner residual with a NaN bit pattern after the
  // first restart, so the device reductions must report it; QCD_FAULT=noconv
  // caps the iteration count at one.
  const char* fault = getenv("QCD_FAULT");
  if (fault && strcmp(fault, "nan") == 0 && nactive > 0) {
    QCD_CK(cudaMemsetAsync(S.r.data, 0xFF, S.r.data_bytes(), st));
    if (S.r.norm) QCD_CK(cudaMemsetAsync(S.r.norm, 0xFF, S.r.norm_bytes(), st));
  }
  const int maxiter = (fault && strcmp(fault, "noconv") == 0) ? 1 : (prm.maxiter > 0 ? prm.maxiter : 100000);
  const bool graph = prm.use_graph != 0;
  const int chunk = graph ? (prm.graph_chunk > 0 ? prm.graph_chunk : 32) : 16;
  bool first = true;
  int done_reason = QCD_OK;
  // Chunk length: the iterations between two outer steps are nearly constant
  // (each removes the same factor delta), so after the first gap has been seen
  // a chunk stops short of the expected next outer step and the last few
  // iterations run in chunks of 8 / 2: few launches are wasted after a stop.
  int last_stop = 0, gap = 0;
  // x64 of a right-hand side changed since its last true_residual (plain FP64 solves)
  std::vector<char> stale(nrhs, 0);
  // run `fn(r0, n)` over the maximal runs of consecutive right-hand sides with sel[r]
  auto for_runs = [&](const std::vector<char>& sel, auto fn) {
    for (int r0 = 0; r0 < nrhs;) {
      if (!sel[r0]) {
        ++r0;
        continue;
      }
      int n = 1;
      while (r0 + n < nrhs && sel[r0 + n]) ++n;
      fn(r0, n);
      r0 += n;
    }
  };
  while (nactive > 0) {
    int maxit = 0;
    for (int r = 0; r < nrhs; ++r)
      if (!conv[r]) maxit = std::max(maxit, S.hsc[r].iters);
    if (maxit >= maxiter) {
      done_reason = QCD_ERR_NOCONV;
      break;
    }
    int k = chunk;
    if (gap > 0) {
      int remaining = last_stop + gap - maxit;
      k = remaining >= chunk ? chunk : (remaining >= 8 && chunk >= 8 ? 8 : std::min(2, chunk));
    }
    const bool capped = k > maxiter - maxit;
    if (capped) k = maxiter - maxit;
    // the first iteration runs un-captured so that the stencil tuner can time
    if (first) {
      S.run_chunk(1, false);
      first = false;
    } else {
      S.run_chunk(k, graph && !capped);
    }
    // a plain FP64 solve iterates on x64 itself: the outer step's x_o and residual are stale
    if (S.inner == QCD_F64)
      for (int r = 0; r < nrhs; ++r) stale[r] = stale[r] || !conv[r];
    S.download();
    // ---- outer step for the right-hand sides whose step is due; the others go on
    // iterating from where they are
    std::vector<char> due(nrhs, 0);
    bool any = false;
    for (int r = 0; r < nrhs; ++r) {
      due[r] = !conv[r] && S.hsc[r].active && S.hsc[r].flag != FLAG_NONE;
      any = any || due[r];
    }
    if (!any) continue;
    {
      int now = 0;
      for (int r = 0; r < nrhs; ++r)
        if (!conv[r]) now = std::max(now, S.hsc[r].iters);
      if (now > last_stop) gap = now - last_stop;
      last_stop = now;
    }
    std::vector<char> full(nrhs, 0);
    for (int r = 0; r < nrhs; ++r) {
      if (!due[r]) continue;
      Scal& s = S.hsc[r];
      if (s.flag == FLAG_NAN) {
        status[r] = QCD_ERR_NAN;
      }
      if (s.flag == FLAG_BREAKDOWN) {
        if (++restarts[r] > 2) status[r] = QCD_ERR_BREAKDOWN;
        full[r] = 1;
      }
    }
    for_runs(due, [&](int r0, int n) {
      if (S.inner != QCD_F64) {
        Field xin = sub(S.xin, r0, n), xo = sub(dfo ? x_d : S.x64, r0, n);
        blas_axpby(1.0, xin, 1.0, xo, st);
      }
      true_residual(false, r0, n);
      for (int r = r0; r < r0 + n; ++r) stale[r] = 0;
    });
    nactive = 0;
    std::vector<char> again(nrhs, 0), again_full(nrhs, 0);
    for (int r = 0; r < nrhs; ++r) {
      if (conv[r]) continue;
      if (!due[r]) {
        ++nactive;
        continue;
      }
      ++updates[r];
      if (rfull[r] <= target[r]) {
        conv[r] = 1;
        S.hsc[r].active = 0;
      } else if (status[r] == QCD_ERR_NAN || status[r] == QCD_ERR_BREAKDOWN) {
        conv[r] = 2;  // give up
        S.hsc[r].active = 0;
      } else {
        ++nactive;
        (full[r] ? again_full : again)[r] = 1;
      }
    }
    if (nactive == 0) break;
    for_runs(again, [&](int r0, int n) { restart_from_residual(false, r0, n); });
    for_runs(again_full, [&](int r0, int n) { restart_from_residual(true, r0, n); });
    S.upload();
  }

  // ---- reconstruct the odd sites and write the solution
  std::vector<double> re_(nrhs), ro_(nrhs);
  Field xe = S.x64, xo = S.t64;
  if (wil64) {
    // x_e = x64 and x_o, h and r_e of the last outer step (recomputed where a plain FP64
    // solve stopped at maxiter after iterating past it)
    for_runs(stale, [&](int r0, int n) { true_residual(false, r0, n); });
    unpack_field(lat, 0, S.x64, x, st);
    unpack_field(lat, 1, S.xo64, x, st);
    blas_norm2(r_e64, re_.data(), st, g);
    // odd half of the full residual: b_o - x_o + kappa h (rounding of the reconstruction)
    blas_copy(S.b_o, S.bh, st);
    blas_axpby(-1.0, S.xo64, 1.0, S.bh, st);
    blas_axpby(f.kappa, S.u64, 1.0, S.bh, st);
    blas_norm2(S.bh, ro_.data(), st, g);
  } else if (!dwf) {
    // h = H_oe x_e (kept), x_o = b_o + kappa h
    if (dfo) {
      hop_df(g, x_d, u_d, 1, dag, 1.0, nullptr, nullptr, 0.0, st);
      blas_copy(bo_d, t_d, st);
      blas_axpby(f.kappa, u_d, 1.0, t_d, st);
      blas_copy(x_d, S.x64, st);
      blas_copy(t_d, S.t64, st);
      blas_copy(u_d, S.u64, st);
    } else {
      hop(g, S.x64, S.u64, 1, dag, 1.0, nullptr, st);
      blas_copy(S.b_o, S.t64, st);
      blas_axpby(f.kappa, S.u64, 1.0, S.t64, st);
    }
    unpack_field(lat, 0, S.x64, x, st);
    unpack_field(lat, 1, S.t64, x, st);
    // true residual on the full system: even part with a fresh FP64 stencil on
    // the reconstructed x_o, odd part b_o - (x_o - kappa h) with the same h
    apply_full_parity(S.op64, xe, xo, S.r64, 0, dag, st, "res");
    blas_axpby(1.0, S.b_e, -1.0, S.r64, st);
    blas_norm2(S.r64, re_.data(), st, g);
    blas_copy(S.b_o, S.bh, st);
    blas_axpby(-1.0, S.t64, 1.0, S.bh, st);
    blas_axpby(f.kappa, S.u64, 1.0, S.bh, st);
    blas_norm2(S.bh, ro_.data(), st, g);
  } else {
    if (dfo) {
      hop(g, x_d, u_d, 1, 0, 0.5, &bo_d, st);  // x'_o = W (b_o + 1/2 H_oe x'_e)
      dw_ainv(dp, u_d, t_d, 0, 1.0, nullptr, st);
      blas_copy(x_d, S.x64, st);
      blas_copy(t_d, S.t64, st);
    } else {
      hop(g, S.x64, S.u64, 1, 0, 0.5, &S.b_o, st);  // x'_o = W (b_o + 1/2 H_oe x'_e)
      dw_ainv(dp, S.u64, S.t64, 0, 1.0, nullptr, st);
    }
    if (dp.mobius()) {  // x = B^-1 x'
      dw_binv(dp, S.x64, S.r64, st);
      dw_binv(dp, S.t64, S.bh, st);
      xe = S.r64;
      xo = S.bh;
    }
    unpack_field(lat, 0, xe, x, st);
    unpack_field(lat, 1, xo, x, st);
    // true residual on the full system, both parities
    apply_full_parity(S.op64, xe, xo, S.u64, 0, dag, st, "res");
    blas_axpby(1.0, S.b_e, -1.0, S.u64, st);
    blas_norm2(S.u64, re_.data(), st, g);
    apply_full_parity(S.op64, xo, xe, S.u64, 1, dag, st, "res");
    blas_axpby(1.0, S.b_o, -1.0, S.u64, st);
    blas_norm2(S.u64, ro_.data(), st, g);
  }
  QCD_CK(cudaStreamSynchronize(st));
  double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  for (int r = 0; r < nrhs; ++r) {
    qcd_solve_info& in = info[r];
    in.iters = S.hsc[r].iters;
    in.outer_updates = updates[r];
    // |b| = 0 gives x = 0 exactly; a non-finite |b| or residual is reported as such
    double res = bnorm[r] > 0 ? std::sqrt(re_[r] + ro_[r]) / bnorm[r]
                              : (bnorm[r] == 0.0 ? 0.0 : std::numeric_limits<double>::quiet_NaN());
    in.true_resid = res;
    in.converged = res <= prm.tol;
    in.status = in.converged ? QCD_OK : (status[r] != QCD_OK ? status[r] : (int)QCD_ERR_NOCONV);
    if (!in.converged && done_reason != QCD_OK && status[r] == QCD_OK) in.status = done_reason;
    in.seconds = secs;
  }
}

}  // namespace qcd
