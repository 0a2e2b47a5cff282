// Fermion force for S = phi^dag (M^dag M)^-1 phi with the Wilson matrix
// M = 1 - kappa H of Eq. (1): with eta = M^-dag phi and X = M^-1 eta,
//   dS = -2 Re(eta^dag dM X) = 2 kappa Re(eta^dag dH X).
// The link U_mu(x) enters H twice: (1 - gamma_mu) U_mu(x) from x to x+mu and
// (1 + gamma_mu) U_mu(x)^dag from x+mu to x (both with the boundary factor s
// of that hop).  With the 18 reals of the link independent,
//   F_ba = s sum_sp X(x+mu)_{sp,b} conj([(1-gamma_mu) eta(x)]_{sp,a})
//   G_ab = s sum_sp X(x)_{sp,a}    conj([(1+gamma_mu) eta(x+mu)]_{sp,b})
//   dS/dRe U_ab = 2 kappa Re(F_ba + G_ab),  dS/dIm U_ab = 2 kappa (Im G_ab - Im F_ba).
// Because (1 -+ gamma)/2 are projectors of rank 2, each sum over four spins
// equals a sum over two of the projected half spinors h = u -+ B l:
//   F_ba = s sum_j h[X(x+mu)]_{j,b} conj(h[eta(x)]_{j,a})   with (1 - gamma)
//   G_ab = s sum_j k[X(x)]_{j,a} conj(k[eta(x+mu)]_{j,b})    with (1 + gamma)
// One thread per link, FP64 throughout, canonical layouts in and out.
#include "common.cuh"
#include "internal.h"

namespace qcd {

namespace {

template <int MU>
__device__ __forceinline__ void proj(const double2* site, double sg, Cx<double> h[6]) {
  Cx<double> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = {site[k].x, site[k].y};
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    Cx<double> b0, b1;
    apply_B<MU>(v[6 + c], v[9 + c], b0, b1);
    h[c] = {fma(sg, b0.re, v[c].re), fma(sg, b0.im, v[c].im)};
    h[3 + c] = {fma(sg, b1.re, v[3 + c].re), fma(sg, b1.im, v[3 + c].im)};
  }
}

template <int MU>
__device__ void force_link(const Geom g, const double2* __restrict__ X, const double2* __restrict__ eta,
                           double* __restrict__ out, long i, double two_kappa) {
  int x[4];
  long r = i;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    x[m] = (int)(r % g.L[m]);
    r /= g.L[m];
  }
  long stride = 1;
#pragma unroll
  for (int m = 0; m < MU; ++m) stride *= g.L[m];
  bool wrap = x[MU] == g.L[MU] - 1;
  long j = wrap ? i - (long)(g.L[MU] - 1) * stride : i + stride;
  double s = (wrap && g.apbc[MU]) ? -two_kappa : two_kappa;
  Cx<double> hX[6], hE[6], kX[6], kE[6];
  proj<MU>(X + j * 12, -1.0, hX);    // (1 - gamma) X(x+mu)
  proj<MU>(eta + i * 12, -1.0, hE);  // (1 - gamma) eta(x)
  proj<MU>(X + i * 12, 1.0, kX);     // (1 + gamma) X(x)
  proj<MU>(eta + j * 12, 1.0, kE);   // (1 + gamma) eta(x+mu)
  double* o = out + ((long)MU * g.V + i) * 18;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Cx<double> F = {0.0, 0.0}, G = {0.0, 0.0};
#pragma unroll
      for (int sp = 0; sp < 2; ++sp) {
        F = cjmadd(hE[sp * 3 + a], hX[sp * 3 + b], F);  // F_ba
        G = cjmadd(kE[sp * 3 + b], kX[sp * 3 + a], G);  // G_ab
      }
      o[(a * 3 + b) * 2] = s * (F.re + G.re);
      o[(a * 3 + b) * 2 + 1] = s * (G.im - F.im);
    }
}

__global__ void k_force(Geom g, const double2* __restrict__ X, const double2* __restrict__ eta,
                        double* __restrict__ out, double two_kappa) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= 4L * g.V) return;
  int mu = (int)(idx / g.V);
  long i = idx - (long)mu * g.V;
  switch (mu) {
    case 0: force_link<0>(g, X, eta, out, i, two_kappa); break;
    case 1: force_link<1>(g, X, eta, out, i, two_kappa); break;
    case 2: force_link<2>(g, X, eta, out, i, two_kappa); break;
    default: force_link<3>(g, X, eta, out, i, two_kappa); break;
  }
}

// F_mu(x) = P_TA(U_mu(x) G_mu(x)^dag), G = dS/dRe U + i dS/dIm U, P_TA(M) = (M - M^dag)/2
// minus its trace / 3: the su(3) element whose pairing tr(i T F) with a generator T is the
// derivative of S along U -> exp(i eps T) U.  One thread per link; the links are read from
// the handle's even-odd FP64 copy.
__global__ void k_force_project(Geom g, const double2* __restrict__ U64, const double* __restrict__ dSdU,
                                double2* __restrict__ F) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= 4L * g.V) return;
  const int mu = (int)(idx / g.V);
  const long i = idx - (long)mu * g.V;
  long r = i;
  int par = 0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    par += (int)(r % g.L[m]);
    r /= g.L[m];
  }
  par &= 1;
  const long cb = i >> 1;
  Cx<double> u[9], gg[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 v = U64[((long)(par * 4 + mu) * 9 + k) * g.Vh + cb];
    u[k] = {v.x, v.y};
    const double* d = dSdU + (idx * 9 + k) * 2;
    gg[k] = {d[0], d[1]};
  }
  Cx<double> m[9];  // M = U G^dag: M_ac = sum_b U_ab conj(G_cb)
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      Cx<double> acc = {0.0, 0.0};
#pragma unroll
      for (int b = 0; b < 3; ++b) acc = cmadd(u[a * 3 + b], conjg(gg[c * 3 + b]), acc);
      m[a * 3 + c] = acc;
    }
  const double tr = (m[0].im + m[4].im + m[8].im) / 3.0;  // Im tr(M) / 3; (M - M^dag)/2 has trace i Im tr M
  double2* o = F + idx * 9;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const Cx<double> x = m[a * 3 + c], y = m[c * 3 + a];
      // ((M - M^dag)/2)_ac = (M_ac - conj(M_ca)) / 2
      double re = 0.5 * (x.re - y.re), im = 0.5 * (x.im + y.im);
      if (a == c) im -= tr;
      o[a * 3 + c] = make_double2(re, im);
    }
}

Geom force_geom(const qcd_gauge* gh) { return make_geom(gh->lat.L, gh->lat.bc, gh->lat.V, gh->lat.Vh); }

void launch_force(const qcd_gauge* gh, const double* X, const double* eta, double* dSdU, double scale,
                  cudaStream_t st) {
  const Geom g = force_geom(gh);
  const long n = 4L * g.V;
  k_force<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, (const double2*)X, (const double2*)eta, dSdU, scale);
  QCD_LAUNCH_CK();
}

}  // namespace

void force_device(const qcd_gauge* gh, const qcd_fermion& f, const double* X, const double* eta,
                  double* dSdU, cudaStream_t st) {
  launch_force(gh, X, eta, dSdU, 2.0 * f.kappa, st);
}

// Even-odd pseudofermion action S = phi_e^dag (Mhat^dag Mhat)^-1 phi_e with Mhat = 1 - kappa^2
// H_eo H_oe: for X = (Mhat^dag Mhat)^-1 phi_e and Y = Mhat X,
//   dS = -2 Re(Y^dag dMhat X) = 2 kappa^2 Re(Y^dag dH_eo H_oe X + ((H^dag)_oe Y)^dag dH_oe X),
// i.e. 2 kappa^2 Re(eta^dag dH xi) with the full fields xi = (X, H_oe X) and
// eta = (Y, (H^dag)_oe Y): the kernel of the full action with 2 kappa^2 for 2 kappa.
void force_eo_device(qcd_gauge* g, const qcd_fermion& f, const double* X, const double* Y, double* dSdU,
                     cudaStream_t st) {
  const Lattice& lat = g->lat;
  Field xe = ws_field(g, "f.xe", QCD_F64, 1, 1), xo = ws_field(g, "f.xo", QCD_F64, 1, 1);
  Field ye = ws_field(g, "f.ye", QCD_F64, 1, 1), yo = ws_field(g, "f.yo", QCD_F64, 1, 1);
  pack_field(lat, 0, X, xe, st);
  pack_field(lat, 0, Y, ye, st);
  hop(g, xe, xo, 1, 0, 1.0, nullptr, st);
  hop(g, ye, yo, 1, 1, 1.0, nullptr, st);
  const size_t bytes = (size_t)lat.V * 12 * 2 * sizeof(double);
  double* xi = (double*)g->ws.get("f.xi", bytes);
  double* eta = (double*)g->ws.get("f.eta", bytes);
  unpack_field(lat, 0, xe, xi, st);
  unpack_field(lat, 1, xo, xi, st);
  unpack_field(lat, 0, ye, eta, st);
  unpack_field(lat, 1, yo, eta, st);
  launch_force(g, xi, eta, dSdU, 2.0 * f.kappa * f.kappa, st);
}

void force_project_device(const qcd_gauge* gh, const double* dSdU, double* F, cudaStream_t st) {
  const Geom g = force_geom(gh);
  const long n = 4L * g.V;
  k_force_project<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(g, (const double2*)gh->U64, dSdU, (double2*)F);
  QCD_LAUNCH_CK();
}

}  // namespace qcd
