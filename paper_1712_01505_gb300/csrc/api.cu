// The C ABI of libqcd (declared in include/qcd.h): argument validation,
// handle and workspace management, host/device staging of canonical fields,
// and dispatch to the kernels.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "internal.h"

namespace qcd {

// An NVTX range around an ABI call (visible in Nsight Systems / Compute timelines; costs
// nothing when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

void solve_device(qcd_gauge* g, const qcd_fermion& f, const qcd_solver_params& prm, const double* b,
                  double* x, int nrhs, qcd_solve_info* info, cudaStream_t st);
void force_eo_device(qcd_gauge* g, const qcd_fermion& f, const double* X, const double* Y, double* dSdU,
                     cudaStream_t st);
void force_project_device(const qcd_gauge* g, const double* dSdU, double* F, cudaStream_t st);
void link_update_device(double* U, const double* P, double eps, long nlinks, cudaStream_t st);
void mom_update_device(double* P, const double* F, double c, long nlinks, cudaStream_t st);
double mom_energy_device(const double* P, long nlinks, cudaStream_t st);
void force_device(const qcd_gauge* g, const qcd_fermion& f, const double* X, const double* eta,
                  double* dSdU, cudaStream_t st);
void mhat_noalloc(const qcd_gauge* g, const qcd_fermion& f, int prec, int dagger, const void* in,
                  void* out, int nrhs, cudaStream_t st);

namespace {
thread_local std::string t_err;
std::atomic<long> g_launches{0};
}

void note_launches(long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
void set_launches(long n) { g_launches.store(n, std::memory_order_relaxed); }

void raise(qcd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  throw Error{s, buf};
}

void cuda_check(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  qcd_status s = (e == cudaErrorMemoryAllocation) ? QCD_ERR_OOM : QCD_ERR_CUDA;
  raise(s, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

size_t spinor_site_bytes(int prec) {
  switch (prec) {
    case QCD_F64: return 24 * sizeof(double);
    case QCD_F32: return 24 * sizeof(float);
    case QCD_DF64: return 24 * 2 * sizeof(float);
    default: return 24 * 2;
  }
}

size_t Field::data_bytes() const { return spinor_site_bytes(prec) * (size_t)nsites() * nrhs; }

Field Field::rhs_range(int r0, int n) const {
  Field f = *this;
  size_t per = spinor_site_bytes(prec) * (size_t)nsites();
  f.data = (char*)data + per * r0;
  if (norm) f.norm = norm + (size_t)nsites() * r0;
  f.nrhs = n;
  return f;
}

void* Workspace::get(const std::string& name, size_t bytes) {
  if (bytes == 0) bytes = 16;
  auto it = bufs.find(name);
  if (it != bufs.end() && it->second.bytes >= bytes) return it->second.p;
  if (it != bufs.end()) {
    QCD_CK(cudaFree(it->second.p));
    bufs.erase(it);
  }
  if (getenv("QCD_FAULT") && strcmp(getenv("QCD_FAULT"), "alloc") == 0)
    raise(QCD_ERR_OOM, "workspace allocation of %zu bytes refused (QCD_FAULT=alloc)", bytes);
  void* p = nullptr;
  QCD_CK(cudaMalloc(&p, bytes));
  bufs[name] = {p, bytes};
  ++generation;
  return p;
}

void Workspace::release() {
  for (auto& kv : bufs) cudaFree(kv.second.p);
  bufs.clear();
  ++generation;
}

Field ws_field(qcd_gauge* g, const std::string& name, int prec, int ls, int nrhs) {
  Field f;
  f.prec = prec;
  f.Vh = g->lat.Vh;
  f.ls = ls;
  f.nrhs = nrhs;
  size_t db = f.data_bytes(), nb = f.norm_bytes();
  char* p = (char*)g->ws.get(name, db + nb);
  f.data = p;
  f.norm = nb ? (float*)(p + db) : nullptr;
  return f;
}

namespace {

template <typename F>
qcd_status guarded(F&& fn) {
  try {
    fn();
    t_err.clear();
    return QCD_OK;
  } catch (const Error& e) {
    t_err = e.msg;
    return e.status;
  } catch (const std::exception& e) {
    t_err = e.what();
    return QCD_ERR_CUDA;
  }
}

void check_geom(const qcd_geom* geom) {
  if (!geom) raise(QCD_ERR_ARG, "geom is NULL");
  long V = 1;
  for (int m = 0; m < 4; ++m) {
    if (geom->L[m] < 2 || (geom->L[m] & 1)) raise(QCD_ERR_ARG, "L[%d] = %d must be even and >= 2", m, geom->L[m]);
    if (geom->bc[m] != 1 && geom->bc[m] != -1) raise(QCD_ERR_ARG, "bc[%d] = %d must be +1 or -1", m, geom->bc[m]);
    V *= geom->L[m];
    if (V >= (1L << 31)) raise(QCD_ERR_ARG, "lattice volume must be < 2^31 sites");
  }
  if (geom->recon != 18 && geom->recon != 12) raise(QCD_ERR_ARG, "recon = %d must be 12 or 18", geom->recon);
}

int check_fermion(const qcd_fermion* f) {
  if (!f) raise(QCD_ERR_ARG, "fermion is NULL");
  if (f->type == QCD_WILSON) {
    if (!std::isfinite(f->kappa) || f->kappa <= 0) raise(QCD_ERR_ARG, "kappa must be finite and > 0");
    return 1;
  }
  if (f->type == QCD_DWF || f->type == QCD_MOBIUS) {
    if (f->Ls < 2 || f->Ls > 64) raise(QCD_ERR_ARG, "Ls = %d must be in [2, 64]", f->Ls);
    if (!std::isfinite(f->M5) || !std::isfinite(f->mf)) raise(QCD_ERR_ARG, "M5 and mf must be finite");
    if (f->type == QCD_MOBIUS && (!std::isfinite(f->b5) || !std::isfinite(f->c5)))
      raise(QCD_ERR_ARG, "b5 and c5 must be finite");
    const DwParams p = dw_params(*f);
    // A = alpha - beta S and B = b5 + c5 S are inverted in closed form:
    // (d - e S)^-1 needs d != 0 and 1 + mf (e / d)^Ls != 0
    auto check_block = [&](double d, double e, const char* what) {
      if (std::fabs(d) < 1e-12) raise(QCD_ERR_ARG, "singular fifth-dimension block %s (diagonal %g)", what, d);
      if (std::fabs(1.0 + f->mf * std::pow(e / d, f->Ls)) < 1e-12)
        raise(QCD_ERR_ARG, "singular fifth-dimension block %s", what);
    };
    check_block(p.alpha(), p.beta(), "A");
    check_block(p.b5, -p.c5, "B");
    return f->Ls;
  }
  raise(QCD_ERR_ARG, "unknown fermion type %d", f->type);
}

void check_prec(int prec) {
  if (prec != QCD_F64 && prec != QCD_F32 && prec != QCD_F16 && prec != QCD_DF64)
    raise(QCD_ERR_ARG, "unknown precision %d", prec);
}

// [a, a + n) and [b, b + n) must not share a byte
void check_disjoint(const void* a, const void* b, size_t n) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  if (x < y + n && y < x + n) raise(QCD_ERR_ARG, "in and out must not overlap (%zu-byte fields)", n);
}

void check_gauge(const qcd_gauge* g) {
  if (!g) raise(QCD_ERR_ARG, "gauge handle is NULL");
  int dev = 0;
  QCD_CK(cudaGetDevice(&dev));
  if (dev != g->device) raise(QCD_ERR_ARG, "gauge handle belongs to device %d, current device is %d", g->device, dev);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// A canonical buffer usable on the device: the caller's pointer or a staged copy.
struct Staged {
  double* dev = nullptr;
  bool host = false;
};

Staged stage_in(qcd_gauge* g, const char* name, const void* p, size_t bytes, cudaStream_t st, bool copy) {
  Staged s;
  if (is_device_ptr(p)) {
    s.dev = (double*)p;
    return s;
  }
  s.host = true;
  s.dev = (double*)g->ws.get(name, bytes);
  if (copy) QCD_CK(cudaMemcpyAsync(s.dev, p, bytes, cudaMemcpyHostToDevice, st));
  return s;
}

void stage_out(const Staged& s, void* p, size_t bytes, cudaStream_t st) {
  if (!s.host) return;
  QCD_CK(cudaMemcpyAsync(p, s.dev, bytes, cudaMemcpyDeviceToHost, st));
  QCD_CK(cudaStreamSynchronize(st));
}

Field internal_field(const qcd_gauge* g, int prec, int ls, int nrhs, const void* p) {
  Field f;
  f.prec = prec;
  f.Vh = g->lat.Vh;
  f.ls = ls;
  f.nrhs = nrhs;
  f.data = (void*)p;
  f.norm = prec == QCD_F16 ? (float*)((char*)p + f.data_bytes()) : nullptr;
  return f;
}

}  // namespace
}  // namespace qcd

using namespace qcd;

extern "C" {

const char* qcd_last_error(void) { return t_err.c_str(); }

qcd_status qcd_kernel_launches(uint64_t* count) {
  return guarded([&] {
    if (!count) raise(QCD_ERR_ARG, "count is NULL");
    *count = (uint64_t)launches_so_far();
  });
}

qcd_status qcd_set_tuning(int32_t mode) {
  return guarded([&] {
    if (mode != 0 && mode != 1) raise(QCD_ERR_ARG, "tuning mode must be 0 or 1");
    set_tuning(mode);
  });
}

qcd_status qcd_gauge_load(const qcd_geom* geom, const void* U, void* stream, qcd_gauge** out) {
  NvtxRange nvtx_range("qcd_gauge_load");
  qcd_gauge* g = nullptr;
  qcd_status s = guarded([&] {
    check_geom(geom);
    if (!U || !out) raise(QCD_ERR_ARG, "U and out must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    g = new qcd_gauge();
    QCD_CK(cudaGetDevice(&g->device));
    Lattice& lat = g->lat;
    for (int m = 0; m < 4; ++m) {
      lat.L[m] = geom->L[m];
      lat.bc[m] = geom->bc[m];
    }
    lat.recon = geom->recon;
    lat.V = (long)lat.L[0] * lat.L[1] * lat.L[2] * lat.L[3];
    lat.Vh = lat.V / 2;
    QCD_CK(cudaStreamCreateWithFlags(&g->work, cudaStreamNonBlocking));
    QCD_CK(cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming));
    QCD_CK(cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming));
    size_t links = 4 * (size_t)lat.V;
    g->U64 = g->ws.get("gauge.U64", links * 18 * sizeof(double));
    g->U32 = g->ws.get("gauge.U32", links * lat.recon * sizeof(float));
    g->U16 = g->ws.get("gauge.U16", links * lat.recon * 2);
    g->Udf = g->ws.get("gauge.Udf", links * 18 * 2 * sizeof(float));
    size_t bytes = links * 18 * sizeof(double);
    Staged su = stage_in(g, "io.gauge", U, bytes, st, true);
    gauge_reorder(g, su.dev, st);
    links_to_df(g, st);
    QCD_CK(cudaStreamSynchronize(st));
  });
  if (s != QCD_OK) {
    if (g) {
      cudaDeviceSynchronize();
      for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second.exec);
      g->graphs.clear();
      g->ws.release();
      if (g->work) cudaStreamDestroy(g->work);
      if (g->ev_in) cudaEventDestroy(g->ev_in);
      if (g->ev_out) cudaEventDestroy(g->ev_out);
      delete g;
    }
    if (out) *out = nullptr;
    return s;
  }
  *out = g;
  return QCD_OK;
}

qcd_status qcd_gauge_free(qcd_gauge* g) {
  return guarded([&] {
    if (!g) return;
    cudaDeviceSynchronize();
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second.exec);
    g->graphs.clear();
    g->ws.release();
    cudaStreamDestroy(g->work);
    cudaEventDestroy(g->ev_in);
    cudaEventDestroy(g->ev_out);
    delete g;
  });
}

size_t qcd_field_bytes(const qcd_geom* geom, const qcd_fermion* fermion, qcd_prec prec, int32_t nrhs) {
  size_t out = 0;
  guarded([&] {
    check_geom(geom);
    int ls = check_fermion(fermion);
    check_prec(prec);
    if (nrhs < 1) raise(QCD_ERR_ARG, "nrhs must be >= 1");
    Field f;
    f.prec = prec;
    f.Vh = (long)geom->L[0] * geom->L[1] * geom->L[2] * geom->L[3] / 2;
    f.ls = ls;
    f.nrhs = nrhs;
    out = f.data_bytes() + f.norm_bytes();
  });
  return out;
}

qcd_status qcd_field_pack(const qcd_gauge* gc, const qcd_fermion* fermion, qcd_prec prec, int32_t parity,
                          const void* canon, void* internal, int32_t nrhs, void* stream) {
  NvtxRange nvtx_range("qcd_field_pack");
  return guarded([&] {
    check_gauge(gc);
    qcd_gauge* g = const_cast<qcd_gauge*>(gc);
    int ls = check_fermion(fermion);
    check_prec(prec);
    if (parity != 0 && parity != 1) raise(QCD_ERR_ARG, "parity must be 0 or 1");
    if (!canon || !internal || nrhs < 1) raise(QCD_ERR_ARG, "NULL buffer or nrhs < 1");
    if (!is_device_ptr(internal)) raise(QCD_ERR_ARG, "internal buffers must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    size_t cb = (size_t)nrhs * ls * g->lat.V * 12 * 16;
    Staged si = stage_in(g, "io.in", canon, cb, st, true);
    Field f = internal_field(g, prec, ls, nrhs, internal);
    pack_field(g->lat, parity, si.dev, f, st);
    if (si.host) QCD_CK(cudaStreamSynchronize(st));
  });
}

qcd_status qcd_field_unpack(const qcd_gauge* gc, const qcd_fermion* fermion, qcd_prec prec, int32_t parity,
                            const void* internal, void* canon, int32_t nrhs, void* stream) {
  NvtxRange nvtx_range("qcd_field_unpack");
  return guarded([&] {
    check_gauge(gc);
    qcd_gauge* g = const_cast<qcd_gauge*>(gc);
    int ls = check_fermion(fermion);
    check_prec(prec);
    if (parity != 0 && parity != 1) raise(QCD_ERR_ARG, "parity must be 0 or 1");
    if (!canon || !internal || nrhs < 1) raise(QCD_ERR_ARG, "NULL buffer or nrhs < 1");
    if (!is_device_ptr(internal)) raise(QCD_ERR_ARG, "internal buffers must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    size_t cb = (size_t)nrhs * ls * g->lat.V * 12 * 16;
    // host canon: the other parity must survive, so copy it in first
    Staged so = stage_in(g, "io.out", canon, cb, st, true);
    Field f = internal_field(g, prec, ls, nrhs, internal);
    unpack_field(g->lat, parity, f, so.dev, st);
    stage_out(so, canon, cb, st);
  });
}

qcd_status qcd_dslash(const qcd_gauge* gc, const qcd_fermion* fermion, qcd_prec prec, int32_t op,
                      const void* in, void* out, int32_t nrhs, int32_t layout, void* stream) {
  NvtxRange nvtx_range("qcd_dslash");
  return guarded([&] {
    check_gauge(gc);
    qcd_gauge* g = const_cast<qcd_gauge*>(gc);
    int ls = check_fermion(fermion);
    check_prec(prec);
    if (op < QCD_OP_D_EO || op > QCD_OP_FULL_DAG) raise(QCD_ERR_ARG, "unknown op %d", op);
    if (layout != QCD_LAYOUT_CANON && layout != QCD_LAYOUT_INTERNAL) raise(QCD_ERR_ARG, "unknown layout %d", layout);
    if (!in || !out) raise(QCD_ERR_ARG, "in and out must not be NULL");
    if (in == out) raise(QCD_ERR_ARG, "in and out must not overlap");
    if (nrhs < 1 || nrhs > 64) raise(QCD_ERR_ARG, "nrhs = %d must be in [1, 64]", nrhs);
    cudaStream_t st = (cudaStream_t)stream;
    OpCtx c{g, *fermion, prec};
    const bool dwf = is_dw(*fermion);
    if (dwf && prec == QCD_DF64 && (op == QCD_OP_FULL || op == QCD_OP_FULL_DAG))
      raise(QCD_ERR_UNSUPPORTED, "the unpreconditioned domain-wall matrix is not available in double-float");
    if (layout == QCD_LAYOUT_INTERNAL) {
      if (op == QCD_OP_FULL || op == QCD_OP_FULL_DAG) raise(QCD_ERR_UNSUPPORTED, "FULL ops need the canonical layout");
      if (!is_device_ptr(in) || !is_device_ptr(out)) raise(QCD_ERR_ARG, "internal buffers must be device memory");
      Field fi = internal_field(g, prec, ls, nrhs, in);
      Field fo = internal_field(g, prec, ls, nrhs, out);
      check_disjoint(in, out, fi.data_bytes() + fi.norm_bytes());
      if (op == QCD_OP_D_EO) hop(g, fi, fo, 0, 0, 1.0, nullptr, st);
      else if (op == QCD_OP_D_OE) hop(g, fi, fo, 1, 0, 1.0, nullptr, st);
      else apply_mhat(c, fi, fo, op == QCD_OP_MHAT_DAG, st, "dslash");
      return;
    }
    size_t cb = (size_t)nrhs * ls * g->lat.V * 12 * 16;
    check_disjoint(in, out, cb);
    Staged si = stage_in(g, "io.in", in, cb, st, true);
    Staged so = stage_in(g, "io.out", out, cb, st, false);
    Field a = ws_field(g, "d.a", prec, ls, nrhs);
    Field b = ws_field(g, "d.b", prec, ls, nrhs);
    const int nvec = nrhs * ls;
    switch (op) {
      case QCD_OP_D_EO:
      case QCD_OP_D_OE: {
        int po = op == QCD_OP_D_EO ? 0 : 1;
        pack_field(g->lat, 1 - po, si.dev, a, st);
        hop(g, a, b, po, 0, 1.0, nullptr, st);
        unpack_field(g->lat, po, b, so.dev, st);
        zero_parity_canon(g->lat, 1 - po, so.dev, nvec, st);
        break;
      }
      case QCD_OP_MHAT:
      case QCD_OP_MHAT_DAG:
        pack_field(g->lat, 0, si.dev, a, st);
        apply_mhat(c, a, b, op == QCD_OP_MHAT_DAG, st, "dslash");
        unpack_field(g->lat, 0, b, so.dev, st);
        zero_parity_canon(g->lat, 1, so.dev, nvec, st);
        break;
      default: {
        int dag = op == QCD_OP_FULL_DAG;
        Field e = ws_field(g, "d.e", prec, ls, nrhs);
        pack_field(g->lat, 0, si.dev, a, st);
        pack_field(g->lat, 1, si.dev, b, st);
        apply_full_parity(c, a, b, e, 0, dag, st, "dslash");
        unpack_field(g->lat, 0, e, so.dev, st);
        apply_full_parity(c, b, a, e, 1, dag, st, "dslash");
        unpack_field(g->lat, 1, e, so.dev, st);
      }
    }
    (void)dwf;
    stage_out(so, out, cb, st);
  });
}

qcd_status qcd_solve(const qcd_gauge* gc, const qcd_fermion* fermion, const qcd_solver_params* params,
                     const void* b, void* x, int32_t nrhs, qcd_solve_info* info, void* stream) {
  NvtxRange nvtx_range("qcd_solve");
  return guarded([&] {
    check_gauge(gc);
    qcd_gauge* g = const_cast<qcd_gauge*>(gc);
    int ls = check_fermion(fermion);
    if (!params || !b || !x || !info) raise(QCD_ERR_ARG, "NULL argument");
    if (nrhs < 1 || nrhs > 64) raise(QCD_ERR_ARG, "nrhs = %d must be in [1, 64]", nrhs);
    const qcd_solver_params& p = *params;
    if (p.method != QCD_BICGSTAB && p.method != QCD_CG_NORMAL) raise(QCD_ERR_ARG, "unknown method %d", p.method);
    if (is_dw(*fermion) && p.dagger) raise(QCD_ERR_UNSUPPORTED, "dagger solves are Wilson only");
    if (!(p.tol > 0) || !std::isfinite(p.tol)) raise(QCD_ERR_ARG, "tol must be finite and > 0");
    if (p.inner != QCD_F64 && p.inner != QCD_F32 && p.inner != QCD_F16)
      raise(QCD_ERR_ARG, "inner precision must be QCD_F64, QCD_F32 or QCD_F16 (got %d)", p.inner);
    if (p.outer != QCD_F64 && p.outer != QCD_DF64)
      raise(QCD_ERR_ARG, "outer precision must be QCD_F64 or QCD_DF64 (got %d)", p.outer);
    if (p.maxiter < 0) raise(QCD_ERR_ARG, "maxiter must be >= 0");
    if (p.delta < 0 || p.delta >= 1) raise(QCD_ERR_ARG, "delta must be in [0, 1)");
    cudaStream_t user = (cudaStream_t)stream;
    size_t cb = (size_t)nrhs * ls * g->lat.V * 12 * 16;
    // the solver runs on the handle's own (capturable) stream, ordered after
    // the caller's stream and before the return
    QCD_CK(cudaEventRecord(g->ev_in, user));
    QCD_CK(cudaStreamWaitEvent(g->work, g->ev_in, 0));
    cudaStream_t st = g->work;
    Staged sb = stage_in(g, "io.in", b, cb, st, true);
    Staged sx = stage_in(g, "io.out", x, cb, st, p.x0_given != 0);
    for (int r = 0; r < nrhs; ++r) memset(&info[r], 0, sizeof(qcd_solve_info));
    solve_device(g, *fermion, p, sb.dev, sx.dev, nrhs, info, st);
    stage_out(sx, x, cb, st);
    QCD_CK(cudaEventRecord(g->ev_out, st));
    QCD_CK(cudaStreamWaitEvent(user, g->ev_out, 0));
    QCD_CK(cudaStreamSynchronize(st));
    qcd_status worst = QCD_OK;
    for (int r = 0; r < nrhs; ++r)
      if (info[r].status != QCD_OK) worst = (qcd_status)info[r].status;
    if (worst != QCD_OK) raise(worst, "solve did not reach tol for every right-hand side (see info)");
  });
}

qcd_status qcd_norm2(const qcd_gauge* gc, const qcd_fermion* fermion, const void* psi, int32_t nrhs,
                     double* out, void* stream) {
  NvtxRange nvtx_range("qcd_norm2");
  return guarded([&] {
    check_gauge(gc);
    qcd_gauge* g = const_cast<qcd_gauge*>(gc);
    int ls = check_fermion(fermion);
    if (!psi || !out) raise(QCD_ERR_ARG, "NULL argument");
    if (nrhs < 1 || nrhs > 64) raise(QCD_ERR_ARG, "nrhs = %d must be in [1, 64]", nrhs);
    cudaStream_t st = (cudaStream_t)stream;
    long per = (long)ls * g->lat.V * 12;
    size_t cb = (size_t)nrhs * per * 16;
    Staged s = stage_in(g, "io.in", psi, cb, st, true);
    canon_norm2(s.dev, per, nrhs, out, st, g);
  });
}

qcd_status qcd_mhat_noalloc(const qcd_gauge* gc, const qcd_fermion* fermion, qcd_prec prec,
                            int32_t dagger, const void* in, void* out, int32_t nrhs, void* stream) {
  return guarded([&] {
    check_gauge(gc);
    check_fermion(fermion);
    if (fermion->type != QCD_WILSON) raise(QCD_ERR_UNSUPPORTED, "qcd_mhat_noalloc is for Wilson fermions");
    check_prec(prec);
    if (dagger != 0 && dagger != 1) raise(QCD_ERR_ARG, "dagger must be 0 or 1");
    if (!in || !out) raise(QCD_ERR_ARG, "in and out must not be NULL");
    if (in == out) raise(QCD_ERR_ARG, "in and out must not overlap");
    if (nrhs < 1 || nrhs > 64) raise(QCD_ERR_ARG, "nrhs = %d must be in [1, 64]", nrhs);
    if (!is_device_ptr(in) || !is_device_ptr(out)) raise(QCD_ERR_ARG, "in and out must be device memory");
    const Field fi = internal_field(gc, prec, 1, nrhs, in);
    check_disjoint(in, out, fi.data_bytes() + fi.norm_bytes());
    mhat_noalloc(gc, *fermion, prec, dagger, in, out, nrhs, (cudaStream_t)stream);
  });
}

qcd_status qcd_force(const qcd_gauge* gc, const qcd_fermion* fermion, const void* X, const void* eta,
                     void* dSdU, void* stream) {
  NvtxRange nvtx_range("qcd_force");
  return guarded([&] {
    check_gauge(gc);
    check_fermion(fermion);
    if (fermion->type != QCD_WILSON) raise(QCD_ERR_UNSUPPORTED, "the force is implemented for Wilson fermions");
    if (!X || !eta || !dSdU) raise(QCD_ERR_ARG, "NULL argument");
    if (!is_device_ptr(X) || !is_device_ptr(eta) || !is_device_ptr(dSdU))
      raise(QCD_ERR_ARG, "qcd_force takes device buffers");
    force_device(gc, *fermion, (const double*)X, (const double*)eta, (double*)dSdU, (cudaStream_t)stream);
  });
}

qcd_status qcd_force_eo(const qcd_gauge* gc, const qcd_fermion* fermion, const void* X, const void* Y,
                        void* dSdU, void* stream) {
  NvtxRange nvtx_range("qcd_force_eo");
  return guarded([&] {
    check_gauge(gc);
    check_fermion(fermion);
    if (fermion->type != QCD_WILSON) raise(QCD_ERR_UNSUPPORTED, "the force is implemented for Wilson fermions");
    if (!X || !Y || !dSdU) raise(QCD_ERR_ARG, "NULL argument");
    if (!is_device_ptr(X) || !is_device_ptr(Y) || !is_device_ptr(dSdU))
      raise(QCD_ERR_ARG, "qcd_force_eo takes device buffers");
    force_eo_device(const_cast<qcd_gauge*>(gc), *fermion, (const double*)X, (const double*)Y, (double*)dSdU,
                    (cudaStream_t)stream);
  });
}

qcd_status qcd_force_project(const qcd_gauge* gc, const void* dSdU, void* F, void* stream) {
  NvtxRange nvtx_range("qcd_force_project");
  return guarded([&] {
    check_gauge(gc);
    if (!dSdU || !F) raise(QCD_ERR_ARG, "NULL argument");
    if (dSdU == F) raise(QCD_ERR_ARG, "dSdU and F must not overlap");
    if (!is_device_ptr(dSdU) || !is_device_ptr(F)) raise(QCD_ERR_ARG, "qcd_force_project takes device buffers");
    force_project_device(gc, (const double*)dSdU, (double*)F, (cudaStream_t)stream);
  });
}

qcd_status qcd_link_update(void* U, const void* P, double eps, int64_t nlinks, void* stream) {
  NvtxRange nvtx_range("qcd_link_update");
  return guarded([&] {
    if (!U || !P) raise(QCD_ERR_ARG, "NULL argument");
    if (nlinks < 0) raise(QCD_ERR_ARG, "nlinks must be >= 0");
    if (U == P) raise(QCD_ERR_ARG, "U and P must not overlap");
    if (!std::isfinite(eps)) raise(QCD_ERR_ARG, "eps must be finite");
    if (!is_device_ptr(U) || !is_device_ptr(P)) raise(QCD_ERR_ARG, "qcd_link_update takes device buffers");
    link_update_device((double*)U, (const double*)P, eps, (long)nlinks, (cudaStream_t)stream);
  });
}

qcd_status qcd_mom_update(void* P, const void* F, double c, int64_t nlinks, void* stream) {
  return guarded([&] {
    if (!P || !F) raise(QCD_ERR_ARG, "NULL argument");
    if (nlinks < 0) raise(QCD_ERR_ARG, "nlinks must be >= 0");
    if (!is_device_ptr(P) || !is_device_ptr(F)) raise(QCD_ERR_ARG, "qcd_mom_update takes device buffers");
    mom_update_device((double*)P, (const double*)F, c, (long)nlinks, (cudaStream_t)stream);
  });
}

qcd_status qcd_mom_energy(const void* P, int64_t nlinks, double* out, void* stream) {
  return guarded([&] {
    if (!P || !out) raise(QCD_ERR_ARG, "NULL argument");
    if (nlinks < 0) raise(QCD_ERR_ARG, "nlinks must be >= 0");
    if (!is_device_ptr(P)) raise(QCD_ERR_ARG, "qcd_mom_energy takes a device buffer");
    *out = mom_energy_device((const double*)P, (long)nlinks, (cudaStream_t)stream);
  });
}

}  // extern "C"

// ----------------------------------------------------------------------------- domain decomposition
extern "C" {

int32_t qcd_dd_plan(const qcd_dd_geom* geom, int32_t id, qcd_dd_msg* sends, qcd_dd_msg* recvs) {
  int32_t n = -1;
  if (guarded([&] { n = dd_plan(geom, id, sends, recvs); }) != QCD_OK) return -1;
  return n;
}

qcd_status qcd_dd_face_sites(const qcd_dd_geom* geom, int32_t mu, int32_t side, int32_t parity,
                             int64_t* sites) {
  return guarded([&] { dd_face_sites(geom, mu, side, parity, sites); });
}

qcd_status qcd_dd_create(const qcd_dd_geom* geom, int32_t nlocal, const int32_t* ids, const void* const* U,
                         void* stream, qcd_dd** out) {
  NvtxRange nvtx_range("qcd_dd_create");
  if (out) *out = nullptr;
  return guarded([&] {
    if (!out) raise(QCD_ERR_ARG, "out is NULL");
    dd_create(geom, nlocal, ids, U, (cudaStream_t)stream, out);
  });
}

qcd_status qcd_dd_free(qcd_dd* dd) {
  return guarded([&] { dd_free(dd); });
}

qcd_status qcd_dd_nccl_unique_id(void* id) {
  return guarded([&] { dd_nccl_unique_id(id); });
}

qcd_status qcd_dd_attach_nccl(qcd_dd* dd, const void* unique_id, int32_t nranks, int32_t rank) {
  return guarded([&] { dd_attach_nccl(dd, unique_id, nranks, rank); });
}

qcd_status qcd_dd_dslash(qcd_dd* dd, const qcd_fermion* fermion, qcd_prec prec, int32_t op,
                         const void* const* in, void* const* out, void* stream) {
  NvtxRange nvtx_range("qcd_dd_dslash");
  return guarded([&] {
    if (!dd || !in || !out) raise(QCD_ERR_ARG, "NULL argument");
    check_fermion(fermion);
    check_prec(prec);
    dd_dslash(dd, *fermion, prec, op, in, out, (cudaStream_t)stream);
  });
}

qcd_status qcd_dd_solve(qcd_dd* dd, const qcd_fermion* fermion, const qcd_solver_params* params,
                        const void* const* b, void* const* x, qcd_solve_info* info, void* stream) {
  NvtxRange nvtx_range("qcd_dd_solve");
  qcd_status s = guarded([&] {
    if (!dd || !params || !b || !x || !info) raise(QCD_ERR_ARG, "NULL argument");
    check_fermion(fermion);
    dd_solve(dd, *fermion, *params, b, x, info, (cudaStream_t)stream);
  });
  if (s == QCD_OK && info && !info->converged) {
    t_err = "solve did not reach tol (see info)";
    return (qcd_status)info->status;
  }
  return s;
}

}  // extern "C"
