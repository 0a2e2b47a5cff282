// Composite operators built from the stencil and the site-local kernels:
// the even-odd Schur operators of the Wilson and domain-wall matrices and the
// unpreconditioned matrices on a pair of parity fields.
//
// Wilson (M = 1 - kappa H, Eq. (1) in hopping form):
//   Mhat     = 1 - kappa^2 H_eo H_oe
//   Mhat^dag = 1 - kappa^2 (H^dag)_eo (H^dag)_oe
// Domain-wall (D = A - 1/2 H B with site-local A, B, see dwf.cu; Shamir, Eq. (2):
// B = 1), the Schur operator of D B^-1 = A B^-1 - 1/2 H with W = B A^-1:
//   Mhat     = 1 - 1/4 W H_eo W H_oe
//   Mhat^dag = 1 - 1/4 (H^dag)_eo W^dag (H^dag)_oe W^dag
#include <string>

#include "common.cuh"
#include "internal.h"

namespace qcd {

void apply_mhat(const OpCtx& c, const Field& in, Field& out, int dagger, cudaStream_t st,
                const char* tag, const int* stop, const RedSpec* red) {
  std::string t = tag;
  if (c.f.type == QCD_WILSON) {
    Field tmp = ws_field(c.g, t + ".mhat.t", c.prec, in.ls, in.nrhs);
    const double k2 = c.f.kappa * c.f.kappa;
    hop(c.g, in, tmp, 1, dagger, 1.0, nullptr, st, stop);
    hop(c.g, tmp, out, 0, dagger, -k2, &in, st, stop, true, red);
    return;
  }
  if (red && !dagger) raise(QCD_ERR_UNSUPPORTED, "domain-wall Mhat fuses reductions into Mhat^dag only");
  const DwParams p = dw_params(c.f);
  Field t1 = ws_field(c.g, t + ".mhat.t1", c.prec, in.ls, in.nrhs);
  Field t2 = ws_field(c.g, t + ".mhat.t2", c.prec, in.ls, in.nrhs);
  if (dw_hop_w_fusable(p, c.prec) && in.ls == p.Ls) {  // W fused into the stencil's epilogue
    if (!dagger) {
      dw_hop_w(c.g, p, in, t2, 1, 0, 1.0, nullptr, st, stop);    // W H_oe in
      dw_hop_w(c.g, p, t2, out, 0, 0, -0.25, &in, st, stop);     // in - 1/4 W H_eo (...)
    } else {
      dw_ainv(p, in, t1, 1, 1.0, nullptr, st, stop);             // W^dag in
      dw_hop_w(c.g, p, t1, t2, 1, 1, 1.0, nullptr, st, stop);    // W^dag (H^dag)_oe (...)
      hop(c.g, t2, out, 0, 1, -0.25, &in, st, stop, true, red);  // in - 1/4 (H^dag)_eo (...)
    }
    return;
  }
  if (!dagger) {
    hop(c.g, in, t1, 1, 0, 1.0, nullptr, st, stop);       // H_oe in
    dw_ainv(p, t1, t2, 0, 1.0, nullptr, st, stop);        // W H_oe in
    hop(c.g, t2, t1, 0, 0, 1.0, nullptr, st, stop);       // H_eo W H_oe in
    dw_ainv(p, t1, out, 0, -0.25, &in, st, stop);         // in - 1/4 W (...)
  } else {
    dw_ainv(p, in, t1, 1, 1.0, nullptr, st, stop);        // W^dag in
    hop(c.g, t1, t2, 1, 1, 1.0, nullptr, st, stop);       // (H^dag)_oe
    dw_ainv(p, t2, t1, 1, 1.0, nullptr, st, stop);        // W^dag
    hop(c.g, t1, out, 0, 1, -0.25, &in, st, stop, true, red);  // in - 1/4 (H^dag)_eo (...)
  }
}

// out_p = the full matrix restricted to output parity p, applied to (in_e, in_o):
//   Wilson:  out_p = in_p - kappa H_{p,1-p} in_{1-p}
//   DWF:     out_p = A in_p - 1/2 H_{p,1-p} B in_{1-p}
//            (adjoint: A^T in_p - 1/2 B^T (H^dag)_{p,1-p} in_{1-p}; B = 1 for Shamir)
void apply_full_parity(const OpCtx& c, const Field& in_same, const Field& in_other, Field& out,
                       int parity, int dagger, cudaStream_t st, const char* tag) {
  if (c.f.type == QCD_WILSON) {
    hop(c.g, in_other, out, parity, dagger, -c.f.kappa, &in_same, st);
    return;
  }
  if (c.prec == QCD_DF64)
    raise(QCD_ERR_UNSUPPORTED, "the unpreconditioned domain-wall matrix is not available in double-float");
  const DwParams p = dw_params(c.f);
  Field t = ws_field(c.g, std::string(tag) + ".full.t", c.prec, in_same.ls, in_same.nrhs);
  if (!p.mobius()) {
    hop(c.g, in_other, t, parity, dagger, 1.0, nullptr, st);
    dw_block(p, in_same, out, dagger, -0.5, &t, st);
  } else if (!dagger) {
    Field u = ws_field(c.g, std::string(tag) + ".full.u", c.prec, in_same.ls, in_same.nrhs);
    dw_block(p, in_other, u, 0, 0.0, nullptr, st, BLK_B);              // B in_other
    hop(c.g, u, t, parity, 0, 1.0, nullptr, st);                        // H B in_other
    dw_block(p, in_same, out, 0, -0.5, &t, st, BLK_A, BLK_ONE);         // A in_same - 1/2 (...)
  } else {
    hop(c.g, in_other, t, parity, 1, 1.0, nullptr, st);                 // H^dag in_other
    dw_block(p, in_same, out, 1, -0.5, &t, st, BLK_A, BLK_B);           // A^T in_same - 1/2 B^T (...)
  }
}

}  // namespace qcd
