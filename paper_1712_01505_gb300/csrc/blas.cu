// Level-1 vector operations on internal single-parity fields ("BLAS-like
// functions", Sec. V C): zero, precision-converting copy, axpby, and norms
// with the global sum in FP64.  The solver's fused, device-scalar variants
// live in solver.cu.
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace qcd {

AnyView any_view(const Field& f) {
  AnyView v;
  v.prec = f.prec;
  v.p = f.data;
  v.norm = f.norm;
  v.stride = f.nsites();
  return v;
}

namespace {

constexpr int kThreads = 256;

unsigned grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  long cap = 8L * sm_count();
  return (unsigned)(b < cap ? (b > 0 ? b : 1) : cap);
}

// The storage precisions PX, PY of the operands are template arguments (the host
// dispatches on the fields' precisions), so a kernel holds only its own formats'
// code and registers.
// grid: (blocks, nrhs); grid-stride over the sites of one right-hand side
template <typename R, int PX, int PY>
__global__ void k_axpby(R a, AnyView x, R b, AnyView y, long n) {
  int r = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> vx[12], vy[12];
    if (a != R(0)) any_load_p<R, PX>(x, r, i, vx);
    if (b != R(0)) any_load_p<R, PY>(y, r, i, vy);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      Cx<R> o = {R(0), R(0)};
      if (a != R(0)) o = {a * vx[k].re, a * vx[k].im};
      if (b != R(0)) o = {fma(b, vy[k].re, o.re), fma(b, vy[k].im, o.im)};
      vy[k] = o;
    }
    any_store_p<R, PY>(y, r, i, vy);
  }
}

template <typename R, int PX, int PY>
__global__ void k_copy(AnyView x, AnyView y, long n) {
  int r = blockIdx.y;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> v[12];
    any_load_p<R, PX>(x, r, i, v);
    any_store_p<R, PY>(y, r, i, v);
  }
}

// f(PX, PY) with PX, PY the runtime precisions px, py (F64 / F32 / F16) as
// std::integral_constant arguments
template <typename F>
void dispatch2(int px, int py, F&& f) {
  auto with_y = [&](auto cx) {
    if (py == P64)
      f(cx, std::integral_constant<int, P64>{});
    else if (py == P32)
      f(cx, std::integral_constant<int, P32>{});
    else
      f(cx, std::integral_constant<int, P16>{});
  };
  if (px == P64)
    with_y(std::integral_constant<int, P64>{});
  else if (px == P32)
    with_y(std::integral_constant<int, P32>{});
  else
    with_y(std::integral_constant<int, P16>{});
}

// per-block partial sums of |x|^2: per-site sums in R, per-thread and
// cross-thread sums in double
template <typename R, int PX>
__global__ void k_norm2(AnyView x, long n, double* partial) {
  int r = blockIdx.y;
  double acc[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    Cx<R> v[12];
    any_load_p<R, PX>(x, r, i, v);
    R s = 0;
#pragma unroll
    for (int k = 0; k < 12; ++k) s = fma(v[k].re, v[k].re, fma(v[k].im, v[k].im, s));
    acc[0] += (double)s;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partial[(long)r * gridDim.x + blockIdx.x] = acc[0];
}

// per-block partial sums of |z|^2 over a canonical complex128 array (one rhs per grid row)
__global__ void k_canon_norm2(const double2* __restrict__ z, long n_per_rhs, double* partial) {
  int r = blockIdx.y;
  const double2* zr = z + (long)r * n_per_rhs;
  double acc[1] = {0.0};
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n_per_rhs; i += (long)gridDim.x * blockDim.x) {
    double2 v = zr[i];
    acc[0] = fma(v.x, v.x, fma(v.y, v.y, acc[0]));
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partial[(long)r * gridDim.x + blockIdx.x] = acc[0];
}

}  // namespace

void canon_norm2(const double* z, long n_per_rhs, int nrhs, double* out_host, cudaStream_t st,
                 qcd_gauge* g) {
  unsigned nb = grid_for(n_per_rhs);
  double* partial = (double*)g->ws.get("blas.cnorm2.partial", sizeof(double) * nb * nrhs);
  k_canon_norm2<<<dim3(nb, nrhs), kThreads, 0, st>>>((const double2*)z, n_per_rhs, partial);
  QCD_LAUNCH_CK();
  std::vector<double> h((size_t)nb * nrhs);
  QCD_CK(cudaMemcpyAsync(h.data(), partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  QCD_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < nrhs; ++r) {
    double s = 0;
    for (unsigned b = 0; b < nb; ++b) s += h[(size_t)r * nb + b];
    out_host[r] = s;
  }
}

void blas_zero(Field& f, cudaStream_t st) {
  if (f.data) QCD_CK(cudaMemsetAsync(f.data, 0, f.data_bytes(), st));
  if (f.norm) QCD_CK(cudaMemsetAsync(f.norm, 0, f.norm_bytes(), st));
}

void blas_copy(const Field& src, Field& dst, cudaStream_t st) {
  if (src.nsites() != dst.nsites() || src.nrhs != dst.nrhs) raise(QCD_ERR_ARG, "copy: shape mismatch");
  long n = src.nsites();
  if (n == 0) return;
  if (src.prec == dst.prec) {
    QCD_CK(cudaMemcpyAsync(dst.data, src.data, src.data_bytes(), cudaMemcpyDeviceToDevice, st));
    if (src.norm) QCD_CK(cudaMemcpyAsync(dst.norm, src.norm, src.norm_bytes(), cudaMemcpyDeviceToDevice, st));
    return;
  }
  if (src.prec == QCD_DF64 || dst.prec == QCD_DF64) {
    df_copy(src, dst, st);
    return;
  }
  dim3 grid(grid_for(n), src.nrhs);
  const AnyView vs = any_view(src), vd = any_view(dst);
  dispatch2(src.prec, dst.prec, [&](auto cx, auto cy) {
    constexpr int PX = decltype(cx)::value, PY = decltype(cy)::value;
    if constexpr (PX == P64 || PY == P64)
      k_copy<double, PX, PY><<<grid, kThreads, 0, st>>>(vs, vd, n);
    else
      k_copy<float, PX, PY><<<grid, kThreads, 0, st>>>(vs, vd, n);
  });
  QCD_LAUNCH_CK();
}

void blas_axpby(double a, const Field& x, double b, Field& y, cudaStream_t st) {
  if (x.nsites() != y.nsites() || x.nrhs != y.nrhs) raise(QCD_ERR_ARG, "axpby: shape mismatch");
  long n = x.nsites();
  if (n == 0) return;
  if (x.prec == QCD_DF64 || y.prec == QCD_DF64) {
    df_axpby(a, x, b, y, st);
    return;
  }
  dim3 grid(grid_for(n), x.nrhs);
  const AnyView vx = any_view(x), vy = any_view(y);
  dispatch2(x.prec, y.prec, [&](auto cx, auto cy) {
    constexpr int PX = decltype(cx)::value, PY = decltype(cy)::value;
    if constexpr (PX == P64 || PY == P64)
      k_axpby<double, PX, PY><<<grid, kThreads, 0, st>>>(a, vx, b, vy, n);
    else
      k_axpby<float, PX, PY><<<grid, kThreads, 0, st>>>((float)a, vx, (float)b, vy, n);
  });
  QCD_LAUNCH_CK();
}

void blas_norm2(const Field& x, double* out_host, cudaStream_t st, qcd_gauge* g) {
  long n = x.nsites();
  if (n == 0) {
    for (int r = 0; r < x.nrhs; ++r) out_host[r] = 0;
    return;
  }
  unsigned nb = x.prec == QCD_DF64 ? df_norm2_blocks(n) : grid_for(n);
  double* partial = (double*)g->ws.get("blas.norm2.partial", sizeof(double) * nb * x.nrhs);
  dim3 grid(nb, x.nrhs);
  if (x.prec == QCD_DF64) {
    df_norm2_partials(x, partial, nb, st);
  } else {
    if (x.prec == QCD_F64)
      k_norm2<double, P64><<<grid, kThreads, 0, st>>>(any_view(x), n, partial);
    else if (x.prec == QCD_F32)
      k_norm2<float, P32><<<grid, kThreads, 0, st>>>(any_view(x), n, partial);
    else
      k_norm2<float, P16><<<grid, kThreads, 0, st>>>(any_view(x), n, partial);
    QCD_LAUNCH_CK();
  }
  std::vector<double> h((size_t)nb * x.nrhs);
  QCD_CK(cudaMemcpyAsync(h.data(), partial, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  QCD_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < x.nrhs; ++r) {
    double s = 0;
    for (unsigned b = 0; b < nb; ++b) s += h[(size_t)r * nb + b];
    out_host[r] = s;
  }
}

}  // namespace qcd
