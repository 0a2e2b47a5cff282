// Domain decomposition of the even-odd Wilson operator and its BiCGStab solve
// (Sec. IV D: pack the boundary, communicate while the bulk is computed,
// unpack; the multi-node measurements of Sec. V B-C).
//
// A qcd_dd handle holds the subdomains of the global lattice that this process
// owns (the geometry and message plan are in dd.cuh).  A half-dslash H_{p,1-p}
// runs as
//   1. k_dd_pack: the two faces of every cut direction of every local
//      subdomain, as spin-projected half spinors (12 reals per face site; the
//      high face already multiplied by U^dag, whose link lives on the sender);
//   2. the exchange, on the handle's communication stream: device-to-device
//      copies between subdomains of this process, NCCL send / receive (loaded
//      at run time) with subdomains of other processes;
//   3. k_dd_interior, concurrently with 2: every hop whose neighbour is inside
//      the subdomain (wrapping locally in uncut directions);
//   4. k_dd_exterior, after 2 and 3: the hops across the cut faces, from the
//      halo, added into the boundary sites.
// Global sums of the solver (dot products, norms) are summed per subdomain in
// FP64 in a fixed order, over this process's subdomains in id order, and over
// processes by an NCCL all-reduce in FP64.
#include <dlfcn.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "dd.cuh"
#include "internal.h"
#include "stencil.cuh"

using namespace qcd;
using namespace qcd::ddgeom;

namespace qcd {
namespace {

using namespace stencil;

constexpr int kThreads = 256;

// ----------------------------------------------------------------------------- NCCL (run-time)
// The few NCCL entry points the transport needs, resolved from libnccl.so.2 when
// a handle is attached to a communicator (no build-time dependency).
typedef int (*nccl_uid_fn)(void*);
typedef int (*nccl_sendrecv_fn)(const void*, size_t, int, int, void*, cudaStream_t);
typedef int (*nccl_recv_fn)(void*, size_t, int, int, void*, cudaStream_t);
typedef int (*nccl_group_fn)();
typedef int (*nccl_allreduce_fn)(const void*, void*, size_t, int, int, void*, cudaStream_t);
typedef int (*nccl_destroy_fn)(void*);

struct NcclApi {
  void* lib = nullptr;
  nccl_uid_fn get_unique_id = nullptr;
  void* comm_init_rank = nullptr;
  nccl_sendrecv_fn send = nullptr;
  nccl_recv_fn recv = nullptr;
  nccl_group_fn group_start = nullptr, group_end = nullptr;
  nccl_allreduce_fn all_reduce = nullptr;
  nccl_destroy_fn comm_destroy = nullptr;
};

constexpr int kNcclUint8 = 1, kNcclFloat64 = 8, kNcclSum = 0;
struct NcclUid {
  char internal[128];
};
typedef int (*nccl_init_uid_fn)(void**, int, NcclUid, int);

NcclApi& nccl() {
  static NcclApi api;
  if (api.lib) return api;
  void* h = dlopen("libnccl.so.2", RTLD_NOW | RTLD_GLOBAL);
  if (!h) h = dlopen("libnccl.so", RTLD_NOW | RTLD_GLOBAL);
  if (!h) raise(QCD_ERR_UNSUPPORTED, "NCCL transport: libnccl.so.2 not found (%s)", dlerror());
  api.get_unique_id = (nccl_uid_fn)dlsym(h, "ncclGetUniqueId");
  api.comm_init_rank = dlsym(h, "ncclCommInitRank");
  api.send = (nccl_sendrecv_fn)dlsym(h, "ncclSend");
  api.recv = (nccl_recv_fn)dlsym(h, "ncclRecv");
  api.group_start = (nccl_group_fn)dlsym(h, "ncclGroupStart");
  api.group_end = (nccl_group_fn)dlsym(h, "ncclGroupEnd");
  api.all_reduce = (nccl_allreduce_fn)dlsym(h, "ncclAllReduce");
  api.comm_destroy = (nccl_destroy_fn)dlsym(h, "ncclCommDestroy");
  if (!api.get_unique_id || !api.comm_init_rank || !api.send || !api.recv || !api.group_start ||
      !api.group_end || !api.all_reduce || !api.comm_destroy)
    raise(QCD_ERR_UNSUPPORTED, "NCCL transport: libnccl lacks a needed entry point");
  api.lib = h;
  return api;
}

void nccl_ck(int r, const char* what) {
  if (r != 0) raise(QCD_ERR_CUDA, "%s failed (NCCL error %d)", what, r);
}

// ----------------------------------------------------------------------------- kernels
template <int P>
struct HaloT;
template <>
struct HaloT<P64> {
  using type = double2;
};
template <>
struct HaloT<P32> {
  using type = float2;
};

template <int P, int RECON>
struct DDArgs {
  Geom g;       // local lattice; apbc only in uncut directions
  int l[4];     // local extents
  int cut;      // bit mu: direction mu is cut
  int lowwall;  // bit mu: the low face of this subdomain is the global boundary and bc[mu] = -1
  int highwall; // bit mu: the same for the high face
  int out_parity;
  int dagger;
  int xpay;
  double a;
  LinkView<P, RECON> U;
  SpinorView<P> in, out, x;
  using H = typename HaloT<P>::type;
  H* send[4][2];
  const H* recv[4][2];
  int F[4];             // half-sites per face
  const int* bsites;    // boundary sites (checkerboard index) of the output parity
  int nb;
};

template <typename H, typename R>
__device__ __forceinline__ void halo_store(H* p, int F, int fh, const Cx<R> h[6]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    H v;
    v.x = h[k].re;
    v.y = h[k].im;
    p[(long)k * F + fh] = v;
  }
}

template <typename H, typename R>
__device__ __forceinline__ void halo_load(const H* p, int F, int fh, Cx<R> h[6]) {
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const H v = p[(long)k * F + fh];
    h[k] = {(R)v.x, (R)v.y};
  }
}

template <int P, int RECON, int MU>
__device__ __forceinline__ void pack_one(const DDArgs<P, RECON>& A, int side, int fh) {
  using R = typename MathType<P>::type;
  const int pin = 1 - A.out_parity;
  int x[4];
  face_site(A.l, MU, side ? A.l[MU] - 1 : 0, pin, fh, x);
  const long cb = local_index(A.l, x) >> 1;
  Cx<R> psi[12], h[6];
  A.in.load(cb, psi);
  const R sg = A.dagger ? R(1) : R(-1);
  if (side == 0) {  // for the forward hop of the -mu neighbour
    project<MU>(psi, sg, h);
    halo_store(A.send[MU][0], A.F[MU], fh, h);
  } else {  // for the backward hop of the +mu neighbour: U_mu(y)^dag (1 - sg gamma) psi(y)
    project<MU>(psi, -sg, h);
    Cx<R> U[9], gg[6];
    A.U.load(pin, MU, cb, U);
    link_mul<true>(U, h, gg);
    halo_store(A.send[MU][1], A.F[MU], fh, gg);
  }
}

// grid (blocks, message slot): slot = 2 * k + side for the k-th cut direction
template <int P, int RECON>
__global__ void __launch_bounds__(kThreads) k_dd_pack(DDArgs<P, RECON> A, int4 mus) {
  const int slot = blockIdx.y;
  const int mu = (&mus.x)[slot >> 1], side = slot & 1;
  const int F = A.F[mu];
  for (int fh = blockIdx.x * blockDim.x + threadIdx.x; fh < F; fh += gridDim.x * blockDim.x) {
    switch (mu) {
      case 0: pack_one<P, RECON, 0>(A, side, fh); break;
      case 1: pack_one<P, RECON, 1>(A, side, fh); break;
      case 2: pack_one<P, RECON, 2>(A, side, fh); break;
      default: pack_one<P, RECON, 3>(A, side, fh); break;
    }
  }
}

// the hops of direction MU whose neighbour lies in the subdomain
template <int P, int RECON, int MU>
__device__ __forceinline__ void interior_dir(const DDArgs<P, RECON>& A, const SiteCoords& c, long cb,
                                             typename MathType<P>::type sg,
                                             Cx<typename MathType<P>::type> acc[12]) {
  using R = typename MathType<P>::type;
  const bool cut = (A.cut >> MU) & 1;
#pragma unroll
  for (int dir = +1; dir >= -1; dir -= 2) {
    int wrap;
    const int j = neighbour_index(A.g, c, MU, dir, &wrap);
    if (wrap && cut) continue;  // served by the halo
    const bool neg = wrap && A.g.apbc[MU];
    Cx<R> U[9], psi[12], h[6], gg[6];
    const R s = dir > 0 ? sg : -sg;
    if (dir > 0)
      A.U.load(A.out_parity, MU, cb, U);
    else
      A.U.load(1 - A.out_parity, MU, j >> 1, U);
    A.in.load(j >> 1, psi);
    project<MU>(psi, s, h);
    if (dir > 0)
      link_mul<false>(U, h, gg);
    else
      link_mul<true>(U, h, gg);
    reconstruct_add<MU>(gg, s, neg ? R(-1) : R(1), acc);
  }
}

template <int P, int RECON>
__global__ void __launch_bounds__(kThreads) k_dd_interior(DDArgs<P, RECON> A) {
  using R = typename MathType<P>::type;
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= A.g.Vh) return;
  const SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
  Cx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
  const R sg = A.dagger ? R(1) : R(-1);
  interior_dir<P, RECON, 0>(A, c, cb, sg, acc);
  interior_dir<P, RECON, 1>(A, c, cb, sg, acc);
  interior_dir<P, RECON, 2>(A, c, cb, sg, acc);
  interior_dir<P, RECON, 3>(A, c, cb, sg, acc);
  const R a = (R)A.a;
  Cx<R> o[12];
  if (A.xpay) {
    A.x.load(cb, o);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = fmac(a, acc[k], o[k]);
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = a * acc[k];
  }
  A.out.store(cb, o);
}

template <int P, int RECON, int MU>
__device__ __forceinline__ void exterior_dir(const DDArgs<P, RECON>& A, const SiteCoords& c, long cb,
                                             typename MathType<P>::type sg,
                                             Cx<typename MathType<P>::type> acc[12]) {
  using R = typename MathType<P>::type;
  if (!((A.cut >> MU) & 1)) return;
  const int fh = face_half_index(A.l, c.x, MU);
  if (c.x[MU] == A.l[MU] - 1) {  // forward hop: U_mu(x) times the +mu neighbour's projected spinor
    Cx<R> U[9], h[6], gg[6];
    halo_load(A.recv[MU][0], A.F[MU], fh, h);
    A.U.load(A.out_parity, MU, cb, U);
    link_mul<false>(U, h, gg);
    reconstruct_add<MU>(gg, sg, ((A.highwall >> MU) & 1) ? R(-1) : R(1), acc);
  }
  if (c.x[MU] == 0) {  // backward hop: the -mu neighbour's U^dag-multiplied half spinor
    Cx<R> gg[6];
    halo_load(A.recv[MU][1], A.F[MU], fh, gg);
    reconstruct_add<MU>(gg, -sg, ((A.lowwall >> MU) & 1) ? R(-1) : R(1), acc);
  }
}

// one thread per boundary site: out(x) += a * (hops across the cut faces)
template <int P, int RECON>
__global__ void __launch_bounds__(kThreads) k_dd_exterior(DDArgs<P, RECON> A) {
  using R = typename MathType<P>::type;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= A.nb) return;
  const int cb = A.bsites[t];
  const SiteCoords c = cb_to_site(A.g, cb, A.out_parity);
  Cx<R> acc[12];
#pragma unroll
  for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
  const R sg = A.dagger ? R(1) : R(-1);
  exterior_dir<P, RECON, 0>(A, c, cb, sg, acc);
  exterior_dir<P, RECON, 1>(A, c, cb, sg, acc);
  exterior_dir<P, RECON, 2>(A, c, cb, sg, acc);
  exterior_dir<P, RECON, 3>(A, c, cb, sg, acc);
  const R a = (R)A.a;
  Cx<R> o[12];
  A.out.load(cb, o);
#pragma unroll
  for (int k = 0; k < 12; ++k) o[k] = fmac(a, acc[k], o[k]);
  A.out.store(cb, o);
}

// ----------------------------------------------------------------------------- BLAS of the solver
// Loads and stores with the storage precision PV fixed at compile time (the solver's
// vectors share one precision), or read from the view (PV < 0)
template <typename R, int PV>
__device__ __forceinline__ void dld(const AnyView& v, long i, Cx<R> out[12]) {
  if constexpr (PV < 0)
    any_load<R>(v, 0, i, out);
  else
    any_load_p<R, PV>(v, 0, i, out);
}
template <typename R, int PV>
__device__ __forceinline__ void dst(const AnyView& v, long i, const Cx<R> in[12]) {
  if constexpr (PV < 0)
    any_store<R>(v, 0, i, in);
  else
    any_store_p<R, PV>(v, 0, i, in);
}

// out = a x + b y + c out (complex host scalars; a term with a zero coefficient is not read)
template <typename R, int PV>
__global__ void k_dd_lin3(double2 a, AnyView x, double2 b, AnyView y, double2 c, AnyView out, long n) {
  const Cx<R> ca = {(R)a.x, (R)a.y}, cb_ = {(R)b.x, (R)b.y}, cc = {(R)c.x, (R)c.y};
  const bool ua = a.x != 0.0 || a.y != 0.0, ub = b.x != 0.0 || b.y != 0.0, uc = c.x != 0.0 || c.y != 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vx[12], vy[12], vo[12];
    if (ua) dld<R, PV>(x, i, vx);
    if (ub) dld<R, PV>(y, i, vy);
    if (uc) dld<R, PV>(out, i, vo);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      Cx<R> o = {R(0), R(0)};
      if (ua) o = cmadd(ca, vx[k], o);
      if (ub) o = cmadd(cb_, vy[k], o);
      if (uc) o = cmadd(cc, vo[k], o);
      vo[k] = o;
    }
    dst<R, PV>(out, i, vo);
  }
}

// per-block partial sums of (x, y) = sum conj(x) y (re, im) and |x|^2: per site in R (FP32
// vectors: FP32, as the single-domain solver's sums), across sites and threads in FP64
template <typename R, int PV>
__global__ void k_dd_dot(AnyView x, AnyView y, long n, double* partial) {
  double v[3] = {0.0, 0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vx[12], vy[12];
    dld<R, PV>(x, i, vx);
    dld<R, PV>(y, i, vy);
    R re = 0, im = 0, xx = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re = fma(vx[k].re, vy[k].re, fma(vx[k].im, vy[k].im, re));
      im = fma(vx[k].re, vy[k].im, fma(-vx[k].im, vy[k].re, im));
      xx = fma(vx[k].re, vx[k].re, fma(vx[k].im, vx[k].im, xx));
    }
    v[0] += (double)re;
    v[1] += (double)im;
    v[2] += (double)xx;
  }
  block_sum<3>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) partial[blockIdx.x * 4 + k] = v[k];
}

// x += alpha p + omega s; r = s - omega t (in lin3's order of operations) and the per-block
// partial sums of (r, rt) and |r|^2 as k_dd_dot forms them
template <typename R, int PV>
__global__ void k_dd_xr(double2 al, double2 om, AnyView p, AnyView s, AnyView t, AnyView x, AnyView r,
                        AnyView rt, long n, double* partial) {
  const Cx<R> a = {(R)al.x, (R)al.y}, w = {(R)om.x, (R)om.y}, mw = {(R)-om.x, (R)-om.y}, one = {R(1), R(0)};
  double v[3] = {0.0, 0.0, 0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vp[12], vs[12], vt[12], vx[12], vr[12];
    dld<R, PV>(p, i, vp);
    dld<R, PV>(s, i, vs);
    dld<R, PV>(t, i, vt);
    dld<R, PV>(x, i, vx);
    dld<R, PV>(rt, i, vr);  // rt here; r is written below
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const Cx<R> zero = {R(0), R(0)};
      vx[k] = cmadd(one, vx[k], cmadd(w, vs[k], cmadd(a, vp[k], zero)));
      vs[k] = cmadd(mw, vt[k], cmadd(one, vs[k], zero));
    }
    dst<R, PV>(x, i, vx);
    dst<R, PV>(r, i, vs);
    R re = 0, im = 0, xx = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re = fma(vs[k].re, vr[k].re, fma(vs[k].im, vr[k].im, re));
      im = fma(vs[k].re, vr[k].im, fma(-vs[k].im, vr[k].re, im));
      xx = fma(vs[k].re, vs[k].re, fma(vs[k].im, vs[k].im, xx));
    }
    v[0] += (double)re;
    v[1] += (double)im;
    v[2] += (double)xx;
  }
  block_sum<3>(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < 3; ++k) partial[blockIdx.x * 4 + k] = v[k];
}

unsigned blocks_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  long cap = 4L * sm_count();
  return (unsigned)std::max(1L, std::min(b, cap));
}

}  // namespace
}  // namespace qcd

// ----------------------------------------------------------------------------- the handle
namespace qcd {
namespace {
struct Sub {
  int id = 0;
  int c[4] = {0, 0, 0, 0};
  qcd_gauge* g = nullptr;
  void* halo = nullptr;       // send and receive faces (sized for FP64)
  int* bsites[2] = {nullptr, nullptr};
  int nb[2] = {0, 0};
  double* partial = nullptr;  // reduction partials
};
}  // namespace
}  // namespace qcd

struct qcd_dd {
  int L[4], P[4], bc[4], l[4], F[4];
  int recon = 18;
  int cut = 0;
  int nsub = 1;
  std::vector<qcd::Sub> subs;  // this process's subdomains, in increasing id
  cudaStream_t comm = nullptr;
  cudaEvent_t ev_pack = nullptr, ev_comm = nullptr;
  void* nccl_comm = nullptr;   // set when the subdomains of other processes are reached by NCCL
  int rank = 0, nranks = 1;
  double* red_dev = nullptr;   // all-reduce staging (NCCL)
  double* red_host = nullptr;  // pinned host copy of the subdomains' reduction partials
  int device = 0;
};

namespace qcd {

void dd_geom_check(const qcd_dd_geom* g) {
  if (!g) raise(QCD_ERR_ARG, "geom is NULL");
  long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (g->P[m] < 1) raise(QCD_ERR_ARG, "P[%d] = %d must be >= 1", m, g->P[m]);
    if (g->L[m] < 2 || g->L[m] % g->P[m]) raise(QCD_ERR_ARG, "L[%d] = %d is not divisible by P = %d", m, g->L[m], g->P[m]);
    const int l = g->L[m] / g->P[m];
    if (l < 2 || (l & 1)) raise(QCD_ERR_ARG, "local extent L[%d] / P[%d] = %d must be even and >= 2", m, m, l);
    if (g->bc[m] != 1 && g->bc[m] != -1) raise(QCD_ERR_ARG, "bc[%d] = %d must be +1 or -1", m, g->bc[m]);
    V *= g->L[m];
    if (V >= (1L << 31)) raise(QCD_ERR_ARG, "lattice volume must be < 2^31 sites");
  }
  if (g->recon != 18 && g->recon != 12) raise(QCD_ERR_ARG, "recon = %d must be 12 or 18", g->recon);
}

int dd_plan(const qcd_dd_geom* g, int id, qcd_dd_msg* sends, qcd_dd_msg* recvs) {
  dd_geom_check(g);
  const int nsub = g->P[0] * g->P[1] * g->P[2] * g->P[3];
  if (id < 0 || id >= nsub) raise(QCD_ERR_ARG, "subdomain id %d out of [0, %d)", id, nsub);
  int l[4], c[4];
  for (int m = 0; m < 4; ++m) l[m] = g->L[m] / g->P[m];
  sub_coords(g->P, id, c);
  int n = 0;
  for (int mu = 0; mu < 4; ++mu) {
    if (g->P[mu] == 1) continue;
    const int F = face_half_sites(l, mu);
    for (int side = 0; side < 2; ++side) {
      // sends: the low face goes to -mu, the high face to +mu; receives: the forward halo
      // comes from +mu (its low face), the backward halo from -mu (its high face)
      if (sends) sends[n + side] = {mu, side, sub_neighbour(g->P, c, mu, side ? +1 : -1), F};
      if (recvs) recvs[n + side] = {mu, side, sub_neighbour(g->P, c, mu, side ? -1 : +1), F};
    }
    n += 2;
  }
  return n;
}

void dd_face_sites(const qcd_dd_geom* g, int mu, int side, int parity, int64_t* out) {
  dd_geom_check(g);
  if (mu < 0 || mu > 3 || (side != 0 && side != 1) || (parity != 0 && parity != 1) || !out)
    raise(QCD_ERR_ARG, "bad face (mu %d, side %d, parity %d)", mu, side, parity);
  int l[4];
  for (int m = 0; m < 4; ++m) l[m] = g->L[m] / g->P[m];
  const int F = face_half_sites(l, mu);
  for (int fh = 0; fh < F; ++fh) {
    int x[4];
    face_site(l, mu, side ? l[mu] - 1 : 0, parity, fh, x);
    out[fh] = local_index(l, x);
  }
}

namespace {

size_t halo_slot_bytes(const qcd_dd* d, int mu, int prec) {
  return (size_t)6 * d->F[mu] * (prec == QCD_F64 ? sizeof(double2) : sizeof(float2));
}

// byte offset of slot (kind 0 send / 1 receive, mu, side) in a subdomain's halo buffer
size_t halo_offset(const qcd_dd* d, int kind, int mu, int side, int prec) {
  size_t off = 0;
  for (int m = 0; m < 4; ++m) {
    if (!((d->cut >> m) & 1)) continue;
    const size_t s = halo_slot_bytes(d, m, prec);
    if (m == mu) return off + (size_t)(2 * kind + side) * s;
    off += 4 * s;
  }
  return off;
}

size_t halo_bytes(const qcd_dd* d, int prec) { return halo_offset(d, 0, 4, 0, prec) + 16; }

int local_of(const qcd_dd* d, int id) {
  for (size_t k = 0; k < d->subs.size(); ++k)
    if (d->subs[k].id == id) return (int)k;
  return -1;
}

template <int P, int RECON>
DDArgs<P, RECON> dd_args(const qcd_dd* d, const Sub& s, const void* links, const Field& in, Field& out,
                         int out_parity, int dagger, double a, const Field* x) {
  DDArgs<P, RECON> A;
  int lbc[4];
  for (int m = 0; m < 4; ++m) lbc[m] = ((d->cut >> m) & 1) ? 1 : d->bc[m];
  A.g = make_geom(d->l, lbc, s.g->lat.V, s.g->lat.Vh);
  for (int m = 0; m < 4; ++m) {
    A.l[m] = d->l[m];
    A.F[m] = d->F[m];
  }
  A.cut = d->cut;
  A.lowwall = A.highwall = 0;
  for (int m = 0; m < 4; ++m) {
    if (!((d->cut >> m) & 1) || d->bc[m] > 0) continue;
    if (s.c[m] == 0) A.lowwall |= 1 << m;
    if (s.c[m] == d->P[m] - 1) A.highwall |= 1 << m;
  }
  A.out_parity = out_parity;
  A.dagger = dagger;
  A.xpay = x != nullptr;
  A.a = a;
  A.U.p = (decltype(A.U.p))links;
  A.U.Vh = s.g->lat.Vh;
  using T = decltype(A.in.p);
  A.in.p = (T)in.data;
  A.in.norm = nullptr;
  A.in.stride = in.nsites();
  A.out.p = (T)out.data;
  A.out.norm = nullptr;
  A.out.stride = out.nsites();
  A.x = A.out;
  if (x) {
    A.x.p = (T)x->data;
    A.x.stride = x->nsites();
  }
  using H = typename HaloT<P>::type;
  for (int m = 0; m < 4; ++m)
    for (int side = 0; side < 2; ++side) {
      A.send[m][side] = ((d->cut >> m) & 1) ? (H*)((char*)s.halo + halo_offset(d, 0, m, side, P == P64 ? QCD_F64 : QCD_F32))
                                            : nullptr;
      A.recv[m][side] = ((d->cut >> m) & 1) ? (const H*)((char*)s.halo + halo_offset(d, 1, m, side, P == P64 ? QCD_F64 : QCD_F32))
                                            : nullptr;
    }
  A.bsites = s.bsites[out_parity];
  A.nb = s.nb[out_parity];
  return A;
}

// out_s = [x_s +] a H_{p,1-p} in_s for every local subdomain s
template <int P, int RECON>
void dd_hop_t(qcd_dd* d, const std::vector<Field>& in, std::vector<Field>& out, int p, int dagger, double a,
              const std::vector<Field>* x, cudaStream_t st) {
  const int prec = P == P64 ? QCD_F64 : QCD_F32;
  std::vector<DDArgs<P, RECON>> args;
  for (size_t k = 0; k < d->subs.size(); ++k) {
    const Sub& s = d->subs[k];
    const void* links = P == P64 ? s.g->U64 : s.g->U32;
    args.push_back(dd_args<P, RECON>(d, s, links, in[k], out[k], p, dagger, a, x ? &(*x)[k] : nullptr));
  }
  int4 mus = make_int4(0, 0, 0, 0);
  int ncut = 0, Fmax = 0;
  for (int m = 0; m < 4; ++m)
    if ((d->cut >> m) & 1) {
      (&mus.x)[ncut++] = m;
      Fmax = std::max(Fmax, d->F[m]);
    }
  // 1. pack
  if (ncut > 0) {
    for (auto& A : args) {
      k_dd_pack<P, RECON><<<dim3(blocks_for(Fmax), 2 * ncut), kThreads, 0, st>>>(A, mus);
      QCD_LAUNCH_CK();
    }
    // 2. exchange on the communication stream
    QCD_CK(cudaEventRecord(d->ev_pack, st));
    QCD_CK(cudaStreamWaitEvent(d->comm, d->ev_pack, 0));
    bool remote = false;
    for (size_t k = 0; k < d->subs.size(); ++k) {
      const Sub& s = d->subs[k];
      for (int m = 0; m < 4; ++m) {
        if (!((d->cut >> m) & 1)) continue;
        const size_t nbytes = halo_slot_bytes(d, m, prec);
        for (int side = 0; side < 2; ++side) {
          // the low face (side 0) feeds the -mu neighbour's forward halo (receive side 0),
          // the high face its +mu neighbour's backward halo (receive side 1)
          const int peer = sub_neighbour(d->P, s.c, m, side ? +1 : -1);
          const int j = local_of(d, peer);
          if (j < 0) {
            remote = true;
            continue;
          }
          QCD_CK(cudaMemcpyAsync((char*)d->subs[j].halo + halo_offset(d, 1, m, side, prec),
                                 (const char*)s.halo + halo_offset(d, 0, m, side, prec), nbytes,
                                 cudaMemcpyDeviceToDevice, d->comm));
        }
      }
    }
    if (remote) {
      if (!d->nccl_comm) raise(QCD_ERR_ARG, "a neighbouring subdomain is held by another process: attach NCCL");
      NcclApi& nc = nccl();
      const Sub& s = d->subs[0];  // one subdomain per process with NCCL
      nccl_ck(nc.group_start(), "ncclGroupStart");
      for (int m = 0; m < 4; ++m) {
        if (!((d->cut >> m) & 1)) continue;
        const size_t nbytes = halo_slot_bytes(d, m, prec);
        for (int side = 0; side < 2; ++side) {
          const int to = sub_neighbour(d->P, s.c, m, side ? +1 : -1);
          nccl_ck(nc.send((const char*)s.halo + halo_offset(d, 0, m, side, prec), nbytes, kNcclUint8, to,
                          d->nccl_comm, d->comm), "ncclSend");
        }
        for (int side = 0; side < 2; ++side) {
          const int from = sub_neighbour(d->P, s.c, m, side ? -1 : +1);
          nccl_ck(nc.recv((char*)s.halo + halo_offset(d, 1, m, side, prec), nbytes, kNcclUint8, from,
                          d->nccl_comm, d->comm), "ncclRecv");
        }
      }
      nccl_ck(nc.group_end(), "ncclGroupEnd");
    }
    QCD_CK(cudaEventRecord(d->ev_comm, d->comm));
  }
  // 3. interior, while the faces travel
  for (size_t k = 0; k < args.size(); ++k) {
    k_dd_interior<P, RECON><<<(unsigned)((d->subs[k].g->lat.Vh + kThreads - 1) / kThreads), kThreads, 0, st>>>(args[k]);
    QCD_LAUNCH_CK();
  }
  // 4. exterior
  if (ncut > 0) {
    QCD_CK(cudaStreamWaitEvent(st, d->ev_comm, 0));
    for (auto& A : args) {
      if (A.nb == 0) continue;
      k_dd_exterior<P, RECON><<<(unsigned)((A.nb + kThreads - 1) / kThreads), kThreads, 0, st>>>(A);
      QCD_LAUNCH_CK();
    }
  }
}

void dd_hop(qcd_dd* d, const std::vector<Field>& in, std::vector<Field>& out, int p, int dagger, double a,
            const std::vector<Field>* x, cudaStream_t st) {
  const int prec = in[0].prec;
  if (prec == QCD_F64)
    dd_hop_t<P64, 18>(d, in, out, p, dagger, a, x, st);
  else if (prec == QCD_F32 && d->recon == 12)
    dd_hop_t<P32, 12>(d, in, out, p, dagger, a, x, st);
  else if (prec == QCD_F32)
    dd_hop_t<P32, 18>(d, in, out, p, dagger, a, x, st);
  else
    raise(QCD_ERR_UNSUPPORTED, "domain decomposition runs in FP64 or FP32");
}

// ---- vectors: one field per local subdomain
using Vec = std::vector<Field>;

Vec dd_vec(qcd_dd* d, const char* name, int prec) {
  Vec v;
  for (auto& s : d->subs) v.push_back(ws_field(s.g, std::string("dd.") + name, prec, 1, 1));
  return v;
}

void lin3(std::complex<double> a, const Vec& x, std::complex<double> b, const Vec& y, std::complex<double> c,
          Vec& out, cudaStream_t st) {
  for (size_t k = 0; k < out.size(); ++k) {
    const long n = out[k].nsites();
    const double2 ca = make_double2(a.real(), a.imag()), cb = make_double2(b.real(), b.imag()),
                  cc = make_double2(c.real(), c.imag());
    const AnyView vx = any_view(x[k]), vy = any_view(y[k]), vo = any_view(out[k]);
    const int pv = (x[k].prec == out[k].prec && y[k].prec == out[k].prec) ? out[k].prec : -1;
    if (pv == QCD_F64)
      k_dd_lin3<double, P64><<<blocks_for(n), kThreads, 0, st>>>(ca, vx, cb, vy, cc, vo, n);
    else if (pv == QCD_F32)
      k_dd_lin3<float, P32><<<blocks_for(n), kThreads, 0, st>>>(ca, vx, cb, vy, cc, vo, n);
    else if (out[k].prec == QCD_F64)
      k_dd_lin3<double, -1><<<blocks_for(n), kThreads, 0, st>>>(ca, vx, cb, vy, cc, vo, n);
    else
      k_dd_lin3<float, -1><<<blocks_for(n), kThreads, 0, st>>>(ca, vx, cb, vy, cc, vo, n);
    QCD_LAUNCH_CK();
  }
}

// sum over this process's subdomains (in id order) and over the processes (NCCL, FP64)
void allreduce(qcd_dd* d, double* v, int n, cudaStream_t st) {
  if (!d->nccl_comm || d->nranks == 1) return;
  NcclApi& nc = nccl();
  QCD_CK(cudaMemcpyAsync(d->red_dev, v, sizeof(double) * n, cudaMemcpyHostToDevice, st));
  nccl_ck(nc.all_reduce(d->red_dev, d->red_dev, (size_t)n, kNcclFloat64, kNcclSum, d->nccl_comm, st),
          "ncclAllReduce");
  QCD_CK(cudaMemcpyAsync(v, d->red_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  QCD_CK(cudaStreamSynchronize(st));
}

// The global sums (over this process's subdomains in id order, then over the processes) of
// the per-block partials that launch(k, nb) leaves in subdomain k's partial buffer: every
// subdomain's partials go to the pinned host buffer together, one synchronisation.
template <typename F>
void global_sums(qcd_dd* d, size_t nsub, F&& launch, double v[3], cudaStream_t st) {
  std::vector<unsigned> nbs;
  size_t off = 0;
  for (size_t k = 0; k < nsub; ++k) {
    const unsigned nb = launch(k);
    QCD_LAUNCH_CK();
    nbs.push_back(nb);
    QCD_CK(cudaMemcpyAsync(d->red_host + off, d->subs[k].partial, sizeof(double) * nb * 4, cudaMemcpyDeviceToHost,
                           st));
    off += (size_t)nb * 4;
  }
  QCD_CK(cudaStreamSynchronize(st));
  v[0] = v[1] = v[2] = 0.0;
  off = 0;
  for (size_t k = 0; k < nsub; ++k) {
    for (unsigned b = 0; b < nbs[k]; ++b)
      for (int j = 0; j < 3; ++j) v[j] += d->red_host[off + (size_t)b * 4 + j];
    off += (size_t)nbs[k] * 4;
  }
  allreduce(d, v, 3, st);
}

// global (x, y) and |x|^2
void dot(qcd_dd* d, const Vec& x, const Vec& y, std::complex<double>* xy, double* xx, cudaStream_t st) {
  double v[3];
  global_sums(d, x.size(), [&](size_t k) {
    const long n = x[k].nsites();
    const unsigned nb = blocks_for(n);
    const int pv = x[k].prec == y[k].prec ? x[k].prec : -1;
    if (pv == QCD_F64)
      k_dd_dot<double, P64><<<nb, kThreads, 0, st>>>(any_view(x[k]), any_view(y[k]), n, d->subs[k].partial);
    else if (pv == QCD_F32)
      k_dd_dot<float, P32><<<nb, kThreads, 0, st>>>(any_view(x[k]), any_view(y[k]), n, d->subs[k].partial);
    else if (x[k].prec == QCD_F64 || y[k].prec == QCD_F64)
      k_dd_dot<double, -1><<<nb, kThreads, 0, st>>>(any_view(x[k]), any_view(y[k]), n, d->subs[k].partial);
    else
      k_dd_dot<float, -1><<<nb, kThreads, 0, st>>>(any_view(x[k]), any_view(y[k]), n, d->subs[k].partial);
    return nb;
  }, v, st);
  if (xy) *xy = std::complex<double>(v[0], v[1]);
  if (xx) *xx = v[2];
}

// x += alpha p + omega s; r = s - omega t; the global (r, rt) and |r|^2 (one pass over the
// vectors, all of the solver's inner precision)
void xr_dot(qcd_dd* d, std::complex<double> alpha, std::complex<double> omega, const Vec& p, const Vec& s,
            const Vec& t, Vec& x, Vec& r, const Vec& rt, std::complex<double>* rrt, double* rr, cudaStream_t st) {
  double v[3];
  const double2 al = make_double2(alpha.real(), alpha.imag()), om = make_double2(omega.real(), omega.imag());
  global_sums(d, p.size(), [&](size_t k) {
    const long n = p[k].nsites();
    const unsigned nb = blocks_for(n);
    const AnyView vp = any_view(p[k]), vs = any_view(s[k]), vt = any_view(t[k]), vx = any_view(x[k]),
                  vr = any_view(r[k]), vrt = any_view(rt[k]);
    if (p[k].prec == QCD_F64)
      k_dd_xr<double, P64><<<nb, kThreads, 0, st>>>(al, om, vp, vs, vt, vx, vr, vrt, n, d->subs[k].partial);
    else
      k_dd_xr<float, P32><<<nb, kThreads, 0, st>>>(al, om, vp, vs, vt, vx, vr, vrt, n, d->subs[k].partial);
    return nb;
  }, v, st);
  *rrt = std::complex<double>(v[0], v[1]);
  *rr = v[2];
}

double norm2(qcd_dd* d, const Vec& y, cudaStream_t st) {
  double n;
  dot(d, y, y, nullptr, &n, st);
  return n;
}

void vcopy(const Vec& a, Vec& b, cudaStream_t st) {
  for (size_t k = 0; k < a.size(); ++k) blas_copy(a[k], b[k], st);
}
void vzero(Vec& a, cudaStream_t st) {
  for (auto& f : a) blas_zero(f, st);
}

// out = Mhat in = in - kappa^2 H_eo H_oe in (H^dag for dagger)
void dd_mhat(qcd_dd* d, double kappa, const Vec& in, Vec& tmp, Vec& out, int dagger, cudaStream_t st) {
  dd_hop(d, in, tmp, 1, dagger, 1.0, nullptr, st);
  dd_hop(d, tmp, out, 0, dagger, -kappa * kappa, &in, st);
}

}  // namespace

// ----------------------------------------------------------------------------- public pieces
void dd_create(const qcd_dd_geom* geom, int nlocal, const int32_t* ids, const void* const* U, cudaStream_t st,
               qcd_dd** out) {
  dd_geom_check(geom);
  if (!out || !ids || !U || nlocal < 1) raise(QCD_ERR_ARG, "dd_create: NULL argument or nlocal < 1");
  qcd_dd* d = new qcd_dd();
  try {
    QCD_CK(cudaGetDevice(&d->device));
    for (int m = 0; m < 4; ++m) {
      d->L[m] = geom->L[m];
      d->P[m] = geom->P[m];
      d->bc[m] = geom->bc[m];
      d->l[m] = geom->L[m] / geom->P[m];
      if (geom->P[m] > 1) d->cut |= 1 << m;
    }
    for (int m = 0; m < 4; ++m) d->F[m] = face_half_sites(d->l, m);
    d->recon = geom->recon;
    d->nsub = geom->P[0] * geom->P[1] * geom->P[2] * geom->P[3];
    std::vector<int> order(nlocal);
    for (int k = 0; k < nlocal; ++k) {
      if (ids[k] < 0 || ids[k] >= d->nsub) raise(QCD_ERR_ARG, "subdomain id %d out of [0, %d)", ids[k], d->nsub);
      if (!U[k]) raise(QCD_ERR_ARG, "gauge field of subdomain %d is NULL", ids[k]);
      order[k] = k;
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) { return ids[a] < ids[b]; });
    for (int k = 1; k < nlocal; ++k)
      if (ids[order[k]] == ids[order[k - 1]]) raise(QCD_ERR_ARG, "subdomain %d given twice", ids[order[k]]);
    QCD_CK(cudaStreamCreateWithFlags(&d->comm, cudaStreamNonBlocking));
    QCD_CK(cudaEventCreateWithFlags(&d->ev_pack, cudaEventDisableTiming));
    QCD_CK(cudaEventCreateWithFlags(&d->ev_comm, cudaEventDisableTiming));
    const long Vloc = (long)d->l[0] * d->l[1] * d->l[2] * d->l[3];
    for (int k : order) {
      Sub s;
      s.id = ids[k];
      sub_coords(d->P, s.id, s.c);
      qcd_geom lg;
      for (int m = 0; m < 4; ++m) {
        lg.L[m] = d->l[m];
        lg.bc[m] = ((d->cut >> m) & 1) ? 1 : d->bc[m];  // cut directions never wrap locally
      }
      lg.recon = d->recon;
      const qcd_status stt = qcd_gauge_load(&lg, U[k], st, &s.g);
      if (stt != QCD_OK) raise(stt, "subdomain %d: %s", s.id, qcd_last_error());
      d->subs.push_back(s);  // owned from here on (freed with the handle)
      Sub& sb = d->subs.back();
      sb.halo = sb.g->ws.get("dd.halo", halo_bytes(d, QCD_F64));
      sb.partial = (double*)sb.g->ws.get("dd.partial", sizeof(double) * 4 * blocks_for(Vloc));
      // boundary sites of each parity: a coordinate on a cut face
      for (int par = 0; par < 2; ++par) {
        std::vector<int> list;
        for (long i = 0; i < Vloc; ++i) {
          int x[4];
          long r = i;
          for (int m = 0; m < 4; ++m) {
            x[m] = (int)(r % d->l[m]);
            r /= d->l[m];
          }
          if (((x[0] + x[1] + x[2] + x[3]) & 1) != par) continue;
          bool edge = false;
          for (int m = 0; m < 4; ++m)
            if (((d->cut >> m) & 1) && (x[m] == 0 || x[m] == d->l[m] - 1)) edge = true;
          if (edge) list.push_back((int)(i >> 1));
        }
        sb.nb[par] = (int)list.size();
        char name[32];
        snprintf(name, sizeof name, "dd.bsites%d", par);
        sb.bsites[par] = (int*)sb.g->ws.get(name, sizeof(int) * std::max<size_t>(1, list.size()));
        if (!list.empty())
          QCD_CK(cudaMemcpyAsync(sb.bsites[par], list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, st));
      }
    }
    size_t npart = 0;
    for (auto& sb : d->subs) npart += (size_t)4 * blocks_for(sb.g->lat.Vh);
    QCD_CK(cudaMallocHost((void**)&d->red_host, sizeof(double) * npart));
    QCD_CK(cudaStreamSynchronize(st));
  } catch (...) {
    dd_free(d);
    throw;
  }
  *out = d;
}

void dd_free(qcd_dd* d) {
  if (!d) return;
  cudaDeviceSynchronize();
  for (auto& s : d->subs)
    if (s.g) qcd_gauge_free(s.g);
  if (d->nccl_comm) nccl().comm_destroy(d->nccl_comm);
  if (d->red_dev) cudaFree(d->red_dev);
  if (d->red_host) cudaFreeHost(d->red_host);
  if (d->comm) cudaStreamDestroy(d->comm);
  if (d->ev_pack) cudaEventDestroy(d->ev_pack);
  if (d->ev_comm) cudaEventDestroy(d->ev_comm);
  delete d;
}

void dd_nccl_unique_id(void* id) {
  if (!id) raise(QCD_ERR_ARG, "id is NULL");
  nccl_ck(nccl().get_unique_id(id), "ncclGetUniqueId");
}

void dd_attach_nccl(qcd_dd* d, const void* uid, int nranks, int rank) {
  if (!d || !uid) raise(QCD_ERR_ARG, "NULL argument");
  if (d->subs.size() != 1 || nranks != d->nsub || rank != d->subs[0].id)
    raise(QCD_ERR_ARG, "the NCCL transport needs one subdomain per process, held by the rank of the same id "
                       "(nranks = %d subdomains)", d->nsub);
  if (d->nccl_comm) raise(QCD_ERR_ARG, "a communicator is already attached");
  NcclApi& nc = nccl();
  NcclUid u;
  memcpy(u.internal, uid, sizeof u.internal);
  nccl_ck(((nccl_init_uid_fn)nc.comm_init_rank)(&d->nccl_comm, nranks, u, rank), "ncclCommInitRank");
  d->rank = rank;
  d->nranks = nranks;
  QCD_CK(cudaMalloc(&d->red_dev, sizeof(double) * 8));
}

namespace {
void check_local_fields(const qcd_dd* d, const void* const* f, const char* what) {
  for (size_t k = 0; k < d->subs.size(); ++k) {
    cudaPointerAttributes a;
    if (!f[k] || cudaPointerGetAttributes(&a, f[k]) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      raise(QCD_ERR_ARG, "%s[%zu] must be a device buffer", what, k);
    }
  }
}
}  // namespace

// ops on canonical local fields (V_loc, 4, 3) complex128, device
void dd_dslash(qcd_dd* d, const qcd_fermion& f, int prec, int op, const void* const* in, void* const* out,
               cudaStream_t st) {
  if (f.type != QCD_WILSON) raise(QCD_ERR_UNSUPPORTED, "domain decomposition is built for the Wilson operator");
  if (prec != QCD_F64 && prec != QCD_F32) raise(QCD_ERR_UNSUPPORTED, "domain decomposition runs in FP64 or FP32");
  if (op < QCD_OP_D_EO || op > QCD_OP_MHAT_DAG) raise(QCD_ERR_UNSUPPORTED, "op %d is not available", op);
  check_local_fields(d, in, "in");
  check_local_fields(d, (const void* const*)out, "out");
  for (size_t k = 0; k < d->subs.size(); ++k)
    if (in[k] == out[k]) raise(QCD_ERR_ARG, "in[%zu] and out[%zu] must not overlap", k, k);
  Vec a = dd_vec(d, "op.a", prec), b = dd_vec(d, "op.b", prec), t = dd_vec(d, "op.t", prec);
  const size_t nloc = d->subs.size();
  if (op == QCD_OP_D_EO || op == QCD_OP_D_OE) {
    const int po = op == QCD_OP_D_EO ? 0 : 1;
    for (size_t k = 0; k < nloc; ++k) pack_field(d->subs[k].g->lat, 1 - po, (const double*)in[k], a[k], st);
    dd_hop(d, a, b, po, 0, 1.0, nullptr, st);
    for (size_t k = 0; k < nloc; ++k) {
      unpack_field(d->subs[k].g->lat, po, b[k], (double*)out[k], st);
      zero_parity_canon(d->subs[k].g->lat, 1 - po, (double*)out[k], 1, st);
    }
    return;
  }
  for (size_t k = 0; k < nloc; ++k) pack_field(d->subs[k].g->lat, 0, (const double*)in[k], a[k], st);
  dd_mhat(d, f.kappa, a, t, b, op == QCD_OP_MHAT_DAG, st);
  for (size_t k = 0; k < nloc; ++k) {
    unpack_field(d->subs[k].g->lat, 0, b[k], (double*)out[k], st);
    zero_parity_canon(d->subs[k].g->lat, 1, (double*)out[k], 1, st);
  }
}

// Even-odd BiCGStab (van der Vorst 1992) on the subdomains with host scalars: FP64, or FP32
// inner iterations with FP64 reliable updates (true residual, solution accumulation and
// global sums in FP64).  The outer step reconstructs x_o = b_o + kappa H_oe x_e and forms
// the even half of the full-system residual r_e = b_e - x_e + kappa H_eo x_o (= bhat -
// Mhat x_e), so the step that reaches tol has the solution and its true residual.
void dd_solve(qcd_dd* d, const qcd_fermion& f, const qcd_solver_params& prm, const void* const* b, void* const* x,
              qcd_solve_info* info, cudaStream_t st) {
  auto t0 = std::chrono::steady_clock::now();
  if (f.type != QCD_WILSON) raise(QCD_ERR_UNSUPPORTED, "domain decomposition is built for the Wilson operator");
  if (prm.method != QCD_BICGSTAB) raise(QCD_ERR_UNSUPPORTED, "the domain-decomposed solve is BiCGStab");
  if (prm.dagger) raise(QCD_ERR_UNSUPPORTED, "the domain-decomposed solve has no adjoint system");
  if (prm.inner != QCD_F64 && prm.inner != QCD_F32) raise(QCD_ERR_UNSUPPORTED, "inner precision FP64 or FP32");
  if (!(prm.tol > 0)) raise(QCD_ERR_ARG, "tol must be > 0");
  if (prm.x0_given) raise(QCD_ERR_UNSUPPORTED, "the domain-decomposed solve starts from x = 0");
  check_local_fields(d, b, "b");
  check_local_fields(d, (const void* const*)x, "x");
  const int inner = prm.inner;
  const double kappa = f.kappa;
  const double delta = (prm.delta > 0 && prm.delta < 1) ? prm.delta : 0.01;
  const size_t nloc = d->subs.size();
  Vec b_e = dd_vec(d, "s.b_e", QCD_F64), b_o = dd_vec(d, "s.b_o", QCD_F64), x64 = dd_vec(d, "s.x64", QCD_F64),
      xo = dd_vec(d, "s.xo", QCD_F64), h64 = dd_vec(d, "s.h", QCD_F64), r64 = dd_vec(d, "s.r64", QCD_F64),
      t64 = dd_vec(d, "s.t64", QCD_F64);
  Vec r = dd_vec(d, "s.r", inner), rt = dd_vec(d, "s.rt", inner), p = dd_vec(d, "s.p", inner),
      v = dd_vec(d, "s.v", inner), s = dd_vec(d, "s.s", inner), t = dd_vec(d, "s.t", inner),
      tmp = dd_vec(d, "s.tmp", inner), xin = dd_vec(d, "s.xin", inner);
  for (size_t k = 0; k < nloc; ++k) {
    pack_field(d->subs[k].g->lat, 0, (const double*)b[k], b_e[k], st);
    pack_field(d->subs[k].g->lat, 1, (const double*)b[k], b_o[k], st);
  }
  const double bnorm = std::sqrt(norm2(d, b_e, st) + norm2(d, b_o, st));
  const double target = prm.tol * bnorm;
  // x = 0: x_o = b_o, h = 0, r_e = bhat = b_e + kappa H_eo b_o
  vzero(x64, st);
  vcopy(b_o, xo, st);
  vzero(h64, st);
  dd_hop(d, b_o, r64, 0, 0, kappa, &b_e, st);
  double rfull = std::sqrt(norm2(d, r64, st));
  auto outer_step = [&]() {  // x64 is current: h, x_o, r_e and |r_e|
    dd_hop(d, x64, h64, 1, 0, 1.0, nullptr, st);
    vcopy(b_o, xo, st);
    for (size_t k = 0; k < nloc; ++k) blas_axpby(kappa, h64[k], 1.0, xo[k], st);
    vcopy(b_e, t64, st);
    for (size_t k = 0; k < nloc; ++k) blas_axpby(-1.0, x64[k], 1.0, t64[k], st);
    dd_hop(d, xo, r64, 0, 0, kappa, &t64, st);
    rfull = std::sqrt(norm2(d, r64, st));
  };
  int iters = 0, updates = 0, status = QCD_OK, restarts = 0;
  const int maxiter = prm.maxiter > 0 ? prm.maxiter : 100000;
  bool conv = bnorm == 0.0 || rfull <= target;
  if (!std::isfinite(bnorm)) {
    status = QCD_ERR_NAN;
    conv = true;
  }
  std::complex<double> rho(1.0), alpha(1.0), omega(1.0), rho_next(0.0);  // rho_next = (rt, r) of the current r
  double r2 = 0.0, r2_ref = 0.0, stop2 = 0.0;
  auto restart = [&](bool full) {
    vcopy(r64, r, st);
    vzero(xin, st);
    if (full) {
      vcopy(r, rt, st);
      vzero(p, st);
      vzero(v, st);
      rho = alpha = omega = 1.0;
    }
    std::complex<double> c;
    dot(d, r, rt, &c, &r2, st);  // (r, rt) = conj((rt, r)) and |r|^2 together
    rho_next = std::conj(c);
    r2_ref = r2;
    const double ratio = rfull > 0 ? std::sqrt(r2) / rfull : 1.0;
    const double tg = 0.5 * target * ratio;
    stop2 = tg * tg;
  };
  if (!conv) restart(true);
  while (!conv && status == QCD_OK) {
    if (iters >= maxiter) {
      status = QCD_ERR_NOCONV;
      break;
    }
    std::complex<double> rho_new = rho_next, rtv, ts;
    double tt;
    bool breakdown = std::abs(rho_new) < 1e-300;
    if (!breakdown) {
      const std::complex<double> beta = (rho_new / rho) * (alpha / omega);
      lin3(1.0, r, -beta * omega, v, beta, p, st);  // p = r + beta (p - omega v)
      dd_mhat(d, kappa, p, tmp, v, 0, st);
      dot(d, rt, v, &rtv, nullptr, st);
      breakdown = std::abs(rtv) <= 1e-300 || std::abs(rtv) < 1e-24 * std::abs(rho_new);
      if (!breakdown) {
        alpha = rho_new / rtv;
        lin3(1.0, r, -alpha, v, 0.0, s, st);  // s = r - alpha v
        dd_mhat(d, kappa, s, tmp, t, 0, st);
        dot(d, t, s, &ts, &tt, st);
        breakdown = !(tt > 0.0);
        if (!breakdown) {
          omega = ts / tt;
          rho = rho_new;
          std::complex<double> c;
          // x += alpha p + omega s, r = s - omega t, |r|^2 and the next iteration's (rt, r)
          xr_dot(d, alpha, omega, p, s, t, xin, r, rt, &c, &r2, st);
          rho_next = std::conj(c);
          ++iters;
        }
      }
    }
    if (!std::isfinite(r2) || !std::isfinite(std::abs(rho_new))) {
      status = QCD_ERR_NAN;
      break;
    }
    const bool update = breakdown || r2 <= stop2 || (inner != QCD_F64 && r2 <= delta * delta * r2_ref);
    if (!update) continue;
    for (size_t k = 0; k < nloc; ++k) blas_axpby(1.0, xin[k], 1.0, x64[k], st);
    outer_step();
    ++updates;
    if (rfull <= target) {
      conv = true;
      break;
    }
    if (breakdown && ++restarts > 2) {
      status = QCD_ERR_BREAKDOWN;
      break;
    }
    restart(breakdown);
  }
  // odd half of the full residual (the rounding of x_o) and the solution
  double ro2 = 0.0;
  for (size_t k = 0; k < nloc; ++k) {
    blas_copy(b_o[k], t64[k], st);
    blas_axpby(-1.0, xo[k], 1.0, t64[k], st);
    blas_axpby(kappa, h64[k], 1.0, t64[k], st);
  }
  ro2 = norm2(d, t64, st);
  for (size_t k = 0; k < nloc; ++k) {
    unpack_field(d->subs[k].g->lat, 0, x64[k], (double*)x[k], st);
    unpack_field(d->subs[k].g->lat, 1, xo[k], (double*)x[k], st);
  }
  QCD_CK(cudaStreamSynchronize(st));
  const double res = bnorm > 0 ? std::sqrt(rfull * rfull + ro2) / bnorm : (bnorm == 0.0 ? 0.0 : NAN);
  info->iters = iters;
  info->outer_updates = updates;
  info->true_resid = res;
  info->converged = res <= prm.tol;
  info->status = info->converged ? QCD_OK : (status != QCD_OK ? status : (int)QCD_ERR_NOCONV);
  info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace qcd
