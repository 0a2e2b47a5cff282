// qcd_mhat_noalloc: the even-odd Wilson operator Mhat (or Mhat^dag) on
// INTERNAL-layout buffers without any device allocation.
//
// qcd_dslash(QCD_OP_MHAT, ...) keeps its odd-parity intermediate H_oe in in a
// vector of the gauge handle's workspace, which it allocates with cudaMalloc
// on first use.  Some callers cannot have the library allocate: a framework
// whose own allocator has already reserved the device memory it manages, a
// program that must not pay for the device-wide synchronisation that
// cudaMalloc / cudaFree imply in the middle of its pipeline, or software held
// to a fixed memory footprint after initialisation.  For them this variant
// keeps the intermediate in a file-scope device array of fixed size instead.
//
// The array is QCD_NOALLOC_SCRATCH_BYTES bytes and exists once per GPU that
// loads the library, for the life of the process.  Its device address is
// looked up once per device, on that device's first call (which is why that
// first call should come before any stream capture).  All calls share the
// array: calls whose work overlaps on the GPU (other streams, other host
// threads) race on it and must be serialised by the caller.  The intermediate
// is overwritten in full before it is read, so nothing needs clearing; the
// array keeps the last call's contents.
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace qcd {

namespace {

constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[QCD_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

// device address of the scratch array on the current device (looked up once)
void* scratch_address() {
  int dev = 0;
  QCD_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) raise(QCD_ERR_UNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      raise(QCD_ERR_CUDA, "cudaGetSymbolAddress(no-alloc scratch) failed on device %d: %s", dev,
            cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

void mhat_noalloc(const qcd_gauge* g, const qcd_fermion& f, int prec, int dagger, const void* in,
                  void* out, int nrhs, cudaStream_t st) {
  Field fi, fo, tmp;
  for (Field* x : {&fi, &fo, &tmp}) {
    x->prec = prec;
    x->Vh = g->lat.Vh;
    x->ls = 1;
    x->nrhs = nrhs;
  }
  const size_t need = tmp.data_bytes() + tmp.norm_bytes();
  if (need > (size_t)QCD_NOALLOC_SCRATCH_BYTES)
    raise(QCD_ERR_ARG,
          "qcd_mhat_noalloc: the intermediate needs %zu bytes (Vh = %ld sites x %d right-hand sides), more "
          "than the %u-byte scratch; use qcd_dslash instead",
          need, g->lat.Vh, nrhs, (unsigned)QCD_NOALLOC_SCRATCH_BYTES);
  char* s = (char*)scratch_address();
  tmp.data = s;
  tmp.norm = tmp.norm_bytes() ? (float*)(s + tmp.data_bytes()) : nullptr;
  fi.data = const_cast<void*>(in);
  fi.norm = prec == QCD_F16 ? (float*)((char*)in + fi.data_bytes()) : nullptr;
  fo.data = out;
  fo.norm = prec == QCD_F16 ? (float*)((char*)out + fo.data_bytes()) : nullptr;
  const double k2 = f.kappa * f.kappa;
  // Mhat = 1 - kappa^2 H_eo H_oe (H -> H^dag for the adjoint); no tuner timing here
  hop(g, fi, tmp, 1, dagger, 1.0, nullptr, st, nullptr, false);
  hop(g, tmp, fo, 0, dagger, -k2, &fi, st, nullptr, false);
}

}  // namespace qcd
