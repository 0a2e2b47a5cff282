// Host-side internals of libqcd shared between translation units.
#pragma once
#include <atomic>
#include <cuda_runtime.h>

#include <cstdarg>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "qcd.h"

namespace qcd {
struct AnyView;
}

namespace qcd {

// ----------------------------------------------------------------------------- errors
struct Error {
  qcd_status status;
  std::string msg;
};

[[noreturn]] void raise(qcd_status s, const char* fmt, ...);
void cuda_check(cudaError_t e, const char* what, const char* file, int line);
#define QCD_CK(call) ::qcd::cuda_check((call), #call, __FILE__, __LINE__)
// count one kernel launch and check it (a launch error leaves no sticky state)
void note_launches(long n);
long launches_so_far();
void set_launches(long n);
#define QCD_LAUNCH_CK()           \
  do {                            \
    ::qcd::note_launches(1);      \
    ::qcd::cuda_check(cudaGetLastError(), "kernel launch", __FILE__, __LINE__); \
  } while (0)

// True the first time a call site asks on the current device (mask: that call
// site's static bitmask of devices): per-device one-time setup such as raising
// a kernel's dynamic shared-memory limit.
inline bool first_use_on_device(std::atomic<unsigned long long>& mask) {
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  return (mask.fetch_or(bit) & bit) == 0;
}

// Launch a kernel with the programmatic-serialization attribute (unless QCD_PDL=0):
// every kernel launched this way starts with pdl_enter() (common.cuh).
bool pdl_enabled();
template <typename... KArgs, typename... Args>
void launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  ::qcd::cuda_check(cudaLaunchKernelEx(&cfg, kernel, args...), "kernel launch", __FILE__, __LINE__);
}

// ----------------------------------------------------------------------------- lattice
struct Lattice {
  int L[4];
  int bc[4];
  int recon;
  long V, Vh;
};

// ----------------------------------------------------------------------------- fields
// A single-parity internal vector: nrhs right-hand sides, each `ls` slices of
// Vh sites, stored component-major (see common.cuh).
struct Field {
  int prec = QCD_F64;
  void* data = nullptr;
  float* norm = nullptr;  // FP16 only: one scale per site
  long Vh = 0;
  int ls = 1;
  int nrhs = 1;
  long nsites() const { return Vh * ls; }
  size_t data_bytes() const;
  size_t norm_bytes() const { return prec == QCD_F16 ? sizeof(float) * (size_t)nsites() * nrhs : 0; }
  // view of right-hand sides [r0, r0 + n)
  Field rhs_range(int r0, int n) const;
};

size_t spinor_site_bytes(int prec);  // bytes per site of the component arrays

// ----------------------------------------------------------------------------- workspace
struct Workspace {
  struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
  };
  std::map<std::string, Buf> bufs;
  long generation = 0;  // bumped whenever a buffer is (re)allocated or freed
  void* get(const std::string& name, size_t bytes);
  void release();
};

}  // namespace qcd

// ----------------------------------------------------------------------------- the handle
namespace qcd {
// an instantiated CUDA graph of solver iterations and the kernels it holds
struct CachedGraph {
  cudaGraphExec_t exec = nullptr;
  long nodes = 0;
};
}  // namespace qcd

struct qcd_gauge {
  std::map<std::string, qcd::CachedGraph> graphs;  // captured solver chunks, by graph key
  qcd::Lattice lat;
  void* U64 = nullptr;  // FP64, 18 reals
  void* U32 = nullptr;  // FP32, lat.recon reals
  void* U16 = nullptr;  // FP16, lat.recon reals
  void* Udf = nullptr;  // double-float, 18 reals as hi/lo FP32 pairs
  qcd::Workspace ws;
  cudaStream_t work = nullptr;  // private stream (capturable) for the solver
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int device = 0;
};

namespace qcd {

// A field in the handle's workspace.
Field ws_field(qcd_gauge* g, const std::string& name, int prec, int ls, int nrhs);

// ----------------------------------------------------------------------------- layout (layout.cu)
void gauge_reorder(qcd_gauge* g, const double* U_canon_dev, cudaStream_t st);
// canonical complex128 (nrhs, ls, V, 4, 3) <-> internal parity field
void pack_field(const Lattice& lat, int parity, const double* canon, Field& f, cudaStream_t st);
void unpack_field(const Lattice& lat, int parity, const Field& f, double* canon, cudaStream_t st);
void zero_parity_canon(const Lattice& lat, int parity, double* canon, int nvec, cudaStream_t st);

// ----------------------------------------------------------------------------- stencils (wilson.cu)
// out = a * H_{p,1-p} in           (x == nullptr)
// out = x + a * H_{p,1-p} in       (x != nullptr)
// with H -> H^dag for dagger; all slices (ls) and right-hand sides of `in`.
// `stop` (device int, may be null): the kernel does nothing when *stop != 0
// (used by the solver's captured iteration chunks).
// `red` (may be null; x given): an inner product fused into the epilogue.
//   mode 1: (rt, out)          -> k = 0, 1 (re, im)
//   mode 2: (out, x), |out|^2  -> k = 0, 1, 2
// One right-hand side (FP32/FP64): every block writes an FP64 partial sum to
// partial[block * 4 + k]; the last block of each group of 64 blocks to finish
// (counted in counters[group], which start at 0 and are reset) sums its group
// in order into gpartial[group * 4 + k]; *npartial receives the number of groups.
// Several slices (FP32: right-hand sides, domain-wall slices): every warp (32
// sites of one slice q) writes partial[(q * ceil(Vh/32) + site block) * 4 + k]
// and a second kernel sums each slice in order into gpartial[q * 4 + k]: the ls
// slice sums of right-hand side r are gpartial[(r * ls + s) * 4 + k] (counters
// and npartial unused).
struct RedSpec {
  int mode;
  const Field* rt;
  double* partial;
  double* gpartial;
  int* counters;
  int* npartial;
};
void hop(const qcd_gauge* g, const Field& in, Field& out, int out_parity, int dagger, double a,
         const Field* x, cudaStream_t st, const int* stop = nullptr, bool allow_tuning = true,
         const RedSpec* red = nullptr);

// ----------------------------------------------------------------------------- double float (wilson_df.cu)
// out = [x1 + c2 x2 +] a * H_{p,1-p} in on double-float fields (x2 only with x1)
void hop_df(const qcd_gauge* g, const Field& in, Field& out, int out_parity, int dagger, double a,
            const Field* x1, const Field* x2, double c2, cudaStream_t st, const int* stop = nullptr,
            bool allow_tuning = true);
void links_to_df(qcd_gauge* g, cudaStream_t st);  // Udf from U64
// conversions and y = a x + b y with a double-float operand (called by blas.cu)
void df_copy(const Field& src, Field& dst, cudaStream_t st);
void df_axpby(double a, const Field& x, double b, Field& y, cudaStream_t st);
unsigned df_norm2_blocks(long n);
void df_norm2_partials(const Field& x, double* partial, unsigned nb, cudaStream_t st);

// ----------------------------------------------------------------------------- domain wall (dwf.cu)
// Shamir (Eq. (2)) and Mobius domain-wall: D = A - 1/2 H B with the site-local
// blocks B = b5 + c5 S and A = (4 - M5) B + 1 - S = alpha - beta S, S the
// fifth-dimension chiral shift (P_- from s+1, P_+ from s-1, -mf across the wall).
// Shamir is b5 = 1, c5 = 0 (B = 1, A = 5 - M5 - S).  The solver works with
// x' = B x, for which D B^-1 = A B^-1 - 1/2 H has the Shamir structure with the
// site-local inverse W = B A^-1.
struct DwParams {
  int Ls;
  double M5, mf;
  double b5 = 1.0, c5 = 0.0;
  bool mobius() const { return !(b5 == 1.0 && c5 == 0.0); }
  double alpha() const { return (4.0 - M5) * b5 + 1.0; }
  double beta() const { return 1.0 - (4.0 - M5) * c5; }
};
DwParams dw_params(const qcd_fermion& f);
bool is_dw(const qcd_fermion& f);  // QCD_DWF or QCD_MOBIUS
// out = [x +] c * W in, W = B A^-1 (dagger: W^T = A^-T B^T); A^-1 for Shamir
void dw_ainv(const DwParams& p, const Field& in, Field& out, int dagger, double c, const Field* x,
             cudaStream_t st, const int* stop = nullptr);
// the same on double-float fields (dwf_df.cu; dw_ainv dispatches to it)
void dw_ainv_df(const DwParams& p, const Field& in, Field& out, int dagger, double c, const Field* x,
                cudaStream_t st, const int* stop = nullptr);
// out = B^-1 in (the physical solution from x'); FP32 / FP64
void dw_binv(const DwParams& p, const Field& in, Field& out, cudaStream_t st);
// out = A B^-1 in (the full residual from the even-odd one); A for Shamir
void dw_a_binv(const DwParams& p, const Field& in, Field& out, cudaStream_t st);
// fused stencil (dwf_hop.cu): out = [x +] a * W H_{p,1-p} in (dagger: W^T (H^dag)_{p,1-p} in),
// one launch; FP32 / FP16 fields with Ls <= 32 (dw_hop_w_fusable)
bool dw_hop_w_fusable(const DwParams& p, int prec);
void dw_hop_w(const qcd_gauge* g, const DwParams& p, const Field& in, Field& out, int out_parity, int dagger,
              double a, const Field* x, cudaStream_t st, const int* stop = nullptr);
// site-local blocks of dw_block
enum Blk5 { BLK_ONE = 0, BLK_A = 1, BLK_B = 2 };
// out = X in + c * Y y (y may be null), X, Y in {1, A, B}; X^T, Y^T for dagger
void dw_block(const DwParams& p, const Field& in, Field& out, int dagger, double c, const Field* y,
              cudaStream_t st, Blk5 X = BLK_A, Blk5 Y = BLK_ONE);

// ----------------------------------------------------------------------------- BLAS (blas.cu)
void blas_zero(Field& f, cudaStream_t st);
void blas_copy(const Field& src, Field& dst, cudaStream_t st);  // any precision -> any
// y = a*x + b*y (real host scalars), any precisions
void blas_axpby(double a, const Field& x, double b, Field& y, cudaStream_t st);
// per right-hand side |x|^2 into host array (synchronises st)
void blas_norm2(const Field& x, double* out_host, cudaStream_t st, qcd_gauge* g);
// per right-hand side sum |z|^2 of a canonical complex128 device array (synchronises st)
void canon_norm2(const double* z, long n_per_rhs, int nrhs, double* out_host, cudaStream_t st,
                 qcd_gauge* g);

// ----------------------------------------------------------------------------- operators (ops.cu)
struct OpCtx {
  qcd_gauge* g;
  qcd_fermion f;
  int prec;
};
// Schur operator on even sites: out = Mhat in (dagger: Mhat^dag); uses workspace temporaries
// `red` is forwarded to the final stencil, whose epilogue forms out (Wilson; for
// domain-wall only with dagger, where the final step is the stencil).
void apply_mhat(const OpCtx& c, const Field& in, Field& out, int dagger, cudaStream_t st,
                const char* tag, const int* stop = nullptr, const RedSpec* red = nullptr);
// out_p = in_p - kappa H in_other (Wilson) or A in_p - 1/2 H in_other (DWF), parity p
void apply_full_parity(const OpCtx& c, const Field& in_same, const Field& in_other, Field& out,
                       int parity, int dagger, cudaStream_t st, const char* tag);
AnyView any_view(const Field& f);

// ----------------------------------------------------------------------------- domain decomposition (dd.cu)
void dd_geom_check(const qcd_dd_geom* g);
int dd_plan(const qcd_dd_geom* g, int id, qcd_dd_msg* sends, qcd_dd_msg* recvs);
void dd_face_sites(const qcd_dd_geom* g, int mu, int side, int parity, int64_t* out);
void dd_create(const qcd_dd_geom* geom, int nlocal, const int32_t* ids, const void* const* U, cudaStream_t st,
               qcd_dd** out);
void dd_free(qcd_dd* d);
void dd_nccl_unique_id(void* id);
void dd_attach_nccl(qcd_dd* d, const void* uid, int nranks, int rank);
void dd_dslash(qcd_dd* d, const qcd_fermion& f, int prec, int op, const void* const* in, void* const* out,
               cudaStream_t st);
void dd_solve(qcd_dd* d, const qcd_fermion& f, const qcd_solver_params& prm, const void* const* b, void* const* x,
              qcd_solve_info* info, cudaStream_t st);

// ----------------------------------------------------------------------------- tuner (tune.cu)
struct LaunchCfg {
  int block;  // threads per block
  int tile;   // right-hand sides / slices per thread
};
bool tuning_enabled();
void set_tuning(int mode);
// candidates are tried with `run` (which must be idempotent) when the key is
// new and the stream is not capturing; returns the cached or chosen config.
// `stop` (may be null): the kernels' stop word; no timing while it is raised.
LaunchCfg tune(const std::string& key, const std::vector<LaunchCfg>& cands,
               void (*run)(void* ctx, const LaunchCfg& cfg), void* ctx, cudaStream_t st,
               bool allow_timing = true, const int* stop = nullptr);

// device properties
int sm_count();

}  // namespace qcd
