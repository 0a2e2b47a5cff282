// Conversions between the canonical complex128 layouts of the C ABI and the
// internal even-odd structure-of-arrays storage (gauge reorder and spinor
// pack / unpack).  These run once per solve (gauge load, source preparation,
// solution write-back).
#include "common.cuh"
#include "dfloat.cuh"
#include "internal.h"

namespace qcd {

namespace {

__device__ __forceinline__ void site_of(const Geom& g, long i, int* parity, long* cb) {
  int x = (int)(i % g.L[0]);
  long r = i / g.L[0];
  int y = (int)(r % g.L[1]);
  r /= g.L[1];
  int z = (int)(r % g.L[2]);
  int t = (int)(r / g.L[2]);
  *parity = (x + y + z + t) & 1;
  *cb = i >> 1;
}

Geom dev_geom(const Lattice& lat) { return make_geom(lat.L, lat.bc, lat.V, lat.Vh); }

// one thread per (mu, site)
__global__ void k_gauge_reorder(Geom g, const double2* __restrict__ U, double2* U64, void* U32,
                                void* U16, int recon) {
  long idx = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (idx >= 4L * g.V) return;
  int mu = (int)(idx / g.V);
  long i = idx % g.V;
  int par;
  long cb;
  site_of(g, i, &par, &cb);
  double2 u[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) u[k] = U[idx * 9 + k];
  long Vh = g.Vh;
  long base9 = (long)(par * 4 + mu) * 9 * Vh + cb;
  long base3 = (long)(par * 4 + mu) * 3 * Vh + cb;
#pragma unroll
  for (int k = 0; k < 9; ++k) U64[base9 + k * Vh] = u[k];
  if (recon == 18) {
    float2* u32 = (float2*)U32;
    __half2* u16 = (__half2*)U16;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      u32[base9 + k * Vh] = make_float2((float)u[k].x, (float)u[k].y);
      u16[base9 + k * Vh] = __floats2half2_rn((float)u[k].x, (float)u[k].y);
    }
  } else {
    float4* u32 = (float4*)U32;
    uint2* u16 = (uint2*)U16;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double2 a = u[2 * k], b = u[2 * k + 1];
      u32[base3 + k * Vh] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
      uint2 d;
      __half2* h = reinterpret_cast<__half2*>(&d);
      h[0] = __floats2half2_rn((float)a.x, (float)a.y);
      h[1] = __floats2half2_rn((float)b.x, (float)b.y);
      u16[base3 + k * Vh] = d;
    }
  }
}

// one thread per (rhs, slice, cb) of the requested parity
template <int P>
__global__ void k_pack(Geom g, int parity, const double2* __restrict__ canon, SpinorView<P> out,
                       int ls, int nrhs) {
  long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long nsites = (long)ls * g.Vh;
  if (n >= nsites * nrhs) return;
  int r = (int)(n / nsites);
  long q = n % nsites;
  int s = (int)(q / g.Vh);
  long cb = q % g.Vh;
  // canonical index of this cb on `parity`
  long i2 = 2 * cb;
  int x0 = (int)(i2 % g.L[0]);
  long rr = i2 / g.L[0];
  int y = (int)(rr % g.L[1]);
  rr /= g.L[1];
  int z = (int)(rr % g.L[2]);
  int t = (int)(rr / g.L[2]);
  long i = i2 + ((parity + y + z + t) & 1);
  (void)x0;
  const double2* src = canon + (((long)r * ls + s) * g.V + i) * 12;
  using R = typename SpinorView<P>::R;
  Cx<R> v[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) v[k] = {(R)src[k].x, (R)src[k].y};
  out.offset_rhs(r).store(q, v);
}

template <int P>
__global__ void k_unpack(Geom g, int parity, SpinorView<P> in, double2* canon, int ls, int nrhs) {
  long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
  long nsites = (long)ls * g.Vh;
  if (n >= nsites * nrhs) return;
  int r = (int)(n / nsites);
  long q = n % nsites;
  int s = (int)(q / g.Vh);
  long cb = q % g.Vh;
  long i2 = 2 * cb;
  long rr = i2 / g.L[0];
  int y = (int)(rr % g.L[1]);
  rr /= g.L[1];
  int z = (int)(rr % g.L[2]);
  int t = (int)(rr / g.L[2]);
  long i = i2 + ((parity + y + z + t) & 1);
  using R = typename SpinorView<P>::R;
  Cx<R> v[12];
  in.offset_rhs(r).load(q, v);
  double2* dst = canon + (((long)r * ls + s) * g.V + i) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = make_double2((double)v[k].re, (double)v[k].im);
}

__global__ void k_zero_parity(Geom g, int parity, double2* canon, long nvec) {
  long n = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (n >= nvec * g.Vh) return;
  long vec = n / g.Vh;
  long cb = n % g.Vh;
  long i2 = 2 * cb;
  long rr = i2 / g.L[0];
  int y = (int)(rr % g.L[1]);
  rr /= g.L[1];
  int z = (int)(rr % g.L[2]);
  int t = (int)(rr / g.L[2]);
  long i = i2 + ((parity + y + z + t) & 1);
  double2* dst = canon + (vec * g.V + i) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) dst[k] = make_double2(0.0, 0.0);
}

template <int P>
SpinorView<P> view_of(const Field& f) {
  SpinorView<P> v;
  using T = decltype(v.p);
  v.p = (T)f.data;
  v.norm = f.norm;
  v.stride = f.nsites();
  return v;
}

unsigned blocks_for(long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

void gauge_reorder(qcd_gauge* g, const double* U_canon_dev, cudaStream_t st) {
  Geom dg = dev_geom(g->lat);
  long n = 4L * g->lat.V;
  k_gauge_reorder<<<blocks_for(n, 256), 256, 0, st>>>(dg, (const double2*)U_canon_dev,
                                                       (double2*)g->U64, g->U32, g->U16,
                                                       g->lat.recon);
  QCD_LAUNCH_CK();
}

void pack_field(const Lattice& lat, int parity, const double* canon, Field& f, cudaStream_t st) {
  Geom dg = dev_geom(lat);
  long n = f.nsites() * f.nrhs;
  if (n == 0) return;
  const double2* c = (const double2*)canon;
  switch (f.prec) {
    case QCD_F64:
      k_pack<P64><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, c, view_of<P64>(f), f.ls, f.nrhs);
      break;
    case QCD_F32:
      k_pack<P32><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, c, view_of<P32>(f), f.ls, f.nrhs);
      break;
    case QCD_DF64:
      k_pack<PDF><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, c, view_of<PDF>(f), f.ls, f.nrhs);
      break;
    default:
      k_pack<P16><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, c, view_of<P16>(f), f.ls, f.nrhs);
  }
  QCD_LAUNCH_CK();
}

void unpack_field(const Lattice& lat, int parity, const Field& f, double* canon, cudaStream_t st) {
  Geom dg = dev_geom(lat);
  long n = f.nsites() * f.nrhs;
  if (n == 0) return;
  double2* c = (double2*)canon;
  switch (f.prec) {
    case QCD_F64:
      k_unpack<P64><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, view_of<P64>(f), c, f.ls, f.nrhs);
      break;
    case QCD_F32:
      k_unpack<P32><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, view_of<P32>(f), c, f.ls, f.nrhs);
      break;
    case QCD_DF64:
      k_unpack<PDF><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, view_of<PDF>(f), c, f.ls, f.nrhs);
      break;
    default:
      k_unpack<P16><<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, view_of<P16>(f), c, f.ls, f.nrhs);
  }
  QCD_LAUNCH_CK();
}

void zero_parity_canon(const Lattice& lat, int parity, double* canon, int nvec, cudaStream_t st) {
  Geom dg = dev_geom(lat);
  long n = (long)nvec * lat.Vh;
  if (n == 0) return;
  k_zero_parity<<<blocks_for(n, 256), 256, 0, st>>>(dg, parity, (double2*)canon, nvec);
  QCD_LAUNCH_CK();
}

}  // namespace qcd
