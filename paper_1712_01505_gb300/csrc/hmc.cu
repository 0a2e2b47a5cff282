// Molecular-dynamics updates of the gauge field and its momenta (the ensemble
// generation that consumes the solver, Sec. II A): momenta P_mu(x) in su(3)
// (traceless anti-Hermitian 3x3), links advanced as U <- exp(eps P) U, momenta as
// P <- P + c F with F the projected force, and the kinetic term sum |P_ab|^2.
// All on canonical complex128 arrays of 3x3 matrices, one thread per matrix.
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace qcd {

namespace {

constexpr int kThreads = 128;

__device__ __forceinline__ void mat_mul(const Cx<double> a[9], const Cx<double> b[9], Cx<double> c[9]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Cx<double> acc = {0.0, 0.0};
#pragma unroll
      for (int k = 0; k < 3; ++k) acc = cmadd(a[i * 3 + k], b[k * 3 + j], acc);
      c[i * 3 + j] = acc;
    }
}

// exp(A) for a 3x3 complex matrix by scaling and squaring: A / 2^s has Frobenius
// norm <= 1/4, where the Taylor series to order 13 (Horner form) is accurate to
// (1/4)^14 / 14! < 1e-19 relative; then s squarings.
__device__ void mat_exp(const Cx<double> a_in[9], Cx<double> e[9]) {
  double n2 = 0.0;
#pragma unroll
  for (int k = 0; k < 9; ++k) n2 += a_in[k].re * a_in[k].re + a_in[k].im * a_in[k].im;
  int s = 0;
  double nrm = sqrt(n2);
  while (nrm > 0.25 && s < 60) {
    nrm *= 0.5;
    ++s;
  }
  const double sc = ldexp(1.0, -s);
  Cx<double> a[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) a[k] = {a_in[k].re * sc, a_in[k].im * sc};
  // Horner: e = 1 + a/1 (1 + a/2 (1 + ... (1 + a/13)))
#pragma unroll
  for (int k = 0; k < 9; ++k) e[k] = {(k % 4 == 0) ? 1.0 : 0.0, 0.0};
  for (int n = 13; n >= 1; --n) {
    Cx<double> t[9];
    mat_mul(a, e, t);
    const double inv = 1.0 / n;
#pragma unroll
    for (int k = 0; k < 9; ++k) e[k] = {((k % 4 == 0) ? 1.0 : 0.0) + inv * t[k].re, inv * t[k].im};
  }
  for (int i = 0; i < s; ++i) {
    Cx<double> t[9];
    mat_mul(e, e, t);
#pragma unroll
    for (int k = 0; k < 9; ++k) e[k] = t[k];
  }
}

__global__ void k_link_update(double2* __restrict__ U, const double2* __restrict__ P, double eps, long n) {
  const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  Cx<double> a[9], e[9], u[9], o[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const double2 p = P[i * 9 + k], v = U[i * 9 + k];
    a[k] = {eps * p.x, eps * p.y};
    u[k] = {v.x, v.y};
  }
  mat_exp(a, e);
  mat_mul(e, u, o);
#pragma unroll
  for (int k = 0; k < 9; ++k) U[i * 9 + k] = make_double2(o[k].re, o[k].im);
}

// P += c F over n complex entries
__global__ void k_mom_update(double2* __restrict__ P, const double2* __restrict__ F, double c, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 p = P[i], f = F[i];
    P[i] = make_double2(fma(c, f.x, p.x), fma(c, f.y, p.y));
  }
}

constexpr int kEnergyBlocks = 512;
__device__ double g_energy_partial[kEnergyBlocks];

// partial sums of |P_ab|^2 (fixed grid and order: the result does not depend on scheduling)
__global__ void k_mom_energy(const double2* __restrict__ P, long n) {
  double acc[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const double2 p = P[i];
    acc[0] = fma(p.x, p.x, fma(p.y, p.y, acc[0]));
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) g_energy_partial[blockIdx.x] = acc[0];
}

unsigned grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  long cap = 8L * sm_count();
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

void link_update_device(double* U, const double* P, double eps, long nlinks, cudaStream_t st) {
  if (nlinks == 0) return;
  k_link_update<<<(unsigned)((nlinks + kThreads - 1) / kThreads), kThreads, 0, st>>>((double2*)U,
                                                                                   (const double2*)P, eps, nlinks);
  QCD_LAUNCH_CK();
}

void mom_update_device(double* P, const double* F, double c, long nlinks, cudaStream_t st) {
  const long n = nlinks * 9;
  if (n == 0) return;
  k_mom_update<<<grid_for(n), kThreads, 0, st>>>((double2*)P, (const double2*)F, c, n);
  QCD_LAUNCH_CK();
}

double mom_energy_device(const double* P, long nlinks, cudaStream_t st) {
  const long n = nlinks * 9;
  k_mom_energy<<<kEnergyBlocks, kThreads, 0, st>>>((const double2*)P, n);
  QCD_LAUNCH_CK();
  std::vector<double> h(kEnergyBlocks);
  QCD_CK(cudaMemcpyFromSymbolAsync(h.data(), g_energy_partial, sizeof(double) * kEnergyBlocks, 0,
                                   cudaMemcpyDeviceToHost, st));
  QCD_CK(cudaStreamSynchronize(st));
  double s = 0.0;
  for (double v : h) s += v;
  return s;
}

}  // namespace qcd
