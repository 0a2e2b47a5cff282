/*
 * libqcd — GB300 (sm_103a) lattice-QCD fermion solver.
 *
 * The operations are those of Kanamori & Matsufuru, "Practical Implementation
 * of Lattice QCD Simulation on Intel Xeon Phi Knights Landing"
 * (arXiv:1712.01505):
 *   - the Wilson fermion matrix, Eq. (1), used in hopping-parameter form
 *       M = 1 - kappa H,  kappa = 1/(2(m0+4))   (so M = 2 kappa D_W),
 *       H psi(x) = sum_mu (1-gamma_mu) U_mu(x) psi(x+mu)
 *                       + (1+gamma_mu) U_mu(x-mu)^dag psi(x-mu);
 *   - the domain-wall fermion matrix, Eq. (2), with the fifth dimension kept
 *     as an internal degree of freedom (Sec. II B 2), m0 = -M5 in its 4D
 *     Wilson blocks, P_+- = (1 +- gamma_5)/2 and quark mass m = mf;
 *   - BiCGStab for Wilson and CG on the normal equations for domain-wall
 *     (Sec. II C), with a reduced-precision inner solver (Sec. II C, last
 *     paragraph) corrected by double-precision outer steps.
 * Both operators are even-odd (Schur) preconditioned on the even sites.
 *
 * Conventions
 *   - Dirac matrices in the chiral basis: gamma_k = [[0,-i sigma_k],[i sigma_k,0]],
 *     gamma_4 = [[0,1],[1,0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4 = diag(1,1,-1,-1).
 *   - Canonical site index i = x + Lx*(y + Ly*(z + Lz*t)); parity (x+y+z+t) mod 2.
 *   - Canonical fields are interleaved complex128 (re, im doubles):
 *       gauge  U[mu][i][a][b]          shape (4, V, 3, 3),  U_ab of U_mu(x)
 *       spinor psi[r][i][spin][colour] shape (nrhs, V, 4, 3)
 *       domain-wall spinor             shape (nrhs, Ls, V, 4, 3), s slowest
 *       force  dSdU[mu][i][a][b][2]    shape (4, V, 3, 3, 2) float64
 *   - Boundary factors bc[mu] = +1 (periodic) or -1 (antiperiodic) multiply a
 *     hop that wraps around direction mu; they are applied in the stencil and
 *     never folded into the stored links.
 *
 * Memory, streams and errors
 *   - Pointers to canonical fields may be device or host memory; the library
 *     inspects them with cudaPointerGetAttributes.  Host buffers are staged
 *     through device memory owned by the gauge handle and the call returns
 *     only after the result has reached the host.
 *   - The caller owns every buffer it passes and the library never frees one.
 *     A qcd_gauge handle owns its reordered link copies and a workspace of
 *     device vectors (Krylov vectors, staging, reduction scratch), all
 *     released by qcd_gauge_free.
 *   - Work is ordered on the caller's stream (`stream` = cudaStream_t, NULL
 *     for the legacy default stream).  qcd_dslash, qcd_field_pack/unpack and
 *     qcd_force on device buffers are asynchronous; qcd_solve returns once the
 *     solve has finished because it fills `info`.
 *   - Every call returns a qcd_status; arguments are validated on the host
 *     before anything is launched.  qcd_last_error() gives a message for the
 *     last failing call of the calling thread.
 *   - Calls that share one gauge handle must not run concurrently from
 *     several host threads (they share the handle's workspace).
 */
#ifndef QCD_H
#define QCD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QCD_OK = 0,
  QCD_ERR_ARG = 1,         /* invalid argument (detected before any launch)        */
  QCD_ERR_CUDA = 2,        /* a CUDA runtime call failed                           */
  QCD_ERR_OOM = 3,         /* device allocation failed                             */
  QCD_ERR_NOCONV = 4,      /* maxiter reached; x holds the best iterate            */
  QCD_ERR_BREAKDOWN = 5,   /* BiCGStab breakdown persisted after restarts          */
  QCD_ERR_NAN = 6,         /* a reduction produced NaN or Inf                       */
  QCD_ERR_TIMEOUT = 7,     /* reserved: a bounded device wait gave up               */
  QCD_ERR_UNSUPPORTED = 8  /* valid but unsupported combination of arguments        */
} qcd_status;

/* Storage / arithmetic precision of internal fields and operator applications.
 * QCD_DF64 ("double-float") keeps every real as an unevaluated sum hi + lo of
 * two FP32 numbers (|lo| <= ulp(hi)/2 on store) and multiplies and sums with
 * error-free transformations (TwoSum, TwoProd by FMA; the compensated dot
 * product "Dot2" of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26 (2005)):
 * about 48 significant bits from FP32 instructions, for GPUs whose FP64 rate
 * is a small fraction of FP32.  Converting a double gives hi = x rounded to
 * 24 significant bits and lo = fl32(x - hi): hi + lo is within 2^-48 |x| of x
 * for 2^-100 <= |x| < 2^100 (below that the low part may underflow).
 * QCD_DF64 is available in qcd_field_pack / unpack, in qcd_dslash (every op
 * for Wilson; D_EO, D_OE, MHAT, MHAT_DAG for domain-wall) and as the outer
 * precision of qcd_solve. */
typedef enum { QCD_F64 = 0, QCD_F32 = 1, QCD_F16 = 2, QCD_DF64 = 3 } qcd_prec;

typedef enum { QCD_WILSON = 0, QCD_DWF = 1, QCD_MOBIUS = 2 } qcd_fermion_type;

typedef enum {
  QCD_OP_D_EO = 0,     /* out_even = H_eo in_odd  (hopping term only, no kappa)    */
  QCD_OP_D_OE = 1,     /* out_odd  = H_oe in_even                                  */
  QCD_OP_MHAT = 2,     /* even-odd Schur operator on even sites (see qcd_dslash)   */
  QCD_OP_MHAT_DAG = 3, /* its adjoint                                              */
  QCD_OP_FULL = 4,     /* the unpreconditioned matrix M (Wilson) or D_DW (Eq. (2)) */
  QCD_OP_FULL_DAG = 5  /* its adjoint                                              */
} qcd_op;

typedef enum {
  QCD_LAYOUT_CANON = 0,   /* canonical complex128 full-lattice fields            */
  QCD_LAYOUT_INTERNAL = 1 /* library-private single-parity buffers of `prec`     */
} qcd_layout;

typedef enum { QCD_BICGSTAB = 0, QCD_CG_NORMAL = 1 } qcd_method;

/* Lattice extents L[mu] (mu = x,y,z,t; Sec. II A: x_mu = 1..L_mu), all even
 * and >= 2; boundary factors bc[mu] = +1 or -1 (Sec. II B 1: periodic or
 * antiperiodic); recon = 18 (full links) or 12 (two rows stored, the third
 * rebuilt as conj(row0 x row1); applies to the FP32 and FP16 copies). */
typedef struct {
  int32_t L[4];
  int32_t bc[4];
  int32_t recon;
} qcd_geom;

/* type = QCD_WILSON: kappa = 1/(2(m0+4)) of Eq. (1).
 * type = QCD_DWF: Ls = N_s >= 2 (fifth-dimension size), M5 (m0 = -M5 in the
 * D_W blocks of Eq. (2)), mf = m of Eq. (2); kappa, b5 and c5 are ignored.
 * type = QCD_MOBIUS: the Mobius generalisation of Eq. (2) (Brower, Neff and
 * Orginos), D = (b5 D_W + 1) - (1 - c5 D_W) S, with D_W = 4 - M5 - H/2 the 4D
 * Wilson matrix of mass -M5 and (S psi)_s = P_- psi_{s+1} + P_+ psi_{s-1}
 * (factor -mf across the wall); b5 = 1, c5 = 0 is Eq. (2).  Needs b5 != 0,
 * alpha = (4 - M5) b5 + 1 != 0 and nonsingular fifth-dimension blocks
 * A = alpha - beta S, B = b5 + c5 S (beta = 1 - (4 - M5) c5).
 * b5 and c5 are appended after the Shamir fields. */
typedef struct {
  int32_t type;
  double kappa;
  int32_t Ls;
  double M5;
  double mf;
  double b5;
  double c5;
} qcd_fermion;

/* method: QCD_BICGSTAB (the paper's choice for Wilson) or QCD_CG_NORMAL (CG on
 *   Mhat^dag Mhat; its choice for domain-wall, whose spectrum reaches into the
 *   left half plane, Sec. II C).  BiCGStab on domain-wall runs, and reports
 *   QCD_ERR_NOCONV / QCD_ERR_BREAKDOWN when it does not reach tol.
 * tol: target |b - A x| / |b| on the full, unpreconditioned system.
 * maxiter: cap on inner Krylov iterations (summed over restarts).
 * inner: precision of the inner iterations (QCD_F64: plain double solve;
 *   QCD_F32 / QCD_F16: mixed precision with reliable updates -- true residual
 *   recomputed and solution accumulated in the outer precision, below).
 * delta: a reliable update is made when the iterated residual has dropped by
 *   this factor since the last one (0 < delta < 1; 0 selects 0.01).
 * use_graph: capture `graph_chunk` inner iterations in one CUDA graph and
 *   check convergence once per graph launch (0 = plain launches).
 * x0_given: x holds an initial guess on entry (warm start).
 * dagger: solve with the adjoint operator (A^dag x = b); Wilson only.
 * outer: precision of the operator applications of the outer steps of a
 *   mixed solve (source preparation, reliable-update residuals b - Mhat x,
 *   reconstruction of the odd sites): QCD_F64 (IEEE double, the default when
 *   zero-initialised) or QCD_DF64 (double-float; the solution is then also
 *   accumulated in double-float).  The final true_resid is computed with IEEE
 *   FP64 operators either way; ignored when inner = QCD_F64. */
typedef struct {
  int32_t method;
  double tol;
  int32_t maxiter;
  int32_t inner;
  double delta;
  int32_t use_graph;
  int32_t graph_chunk;
  int32_t x0_given;
  int32_t dagger;
  int32_t outer;
} qcd_solver_params;

/* Per right-hand side result of qcd_solve. */
typedef struct {
  int32_t iters;         /* inner Krylov iterations                               */
  int32_t outer_updates; /* double-precision reliable updates performed           */
  int32_t converged;     /* 1 if true_resid <= tol                                */
  int32_t status;        /* qcd_status for this right-hand side                   */
  double true_resid;     /* |b - A x| / |b| recomputed in FP64 on the full system  */
  double seconds;        /* wall time of the whole qcd_solve call                  */
} qcd_solve_info;

typedef struct qcd_gauge qcd_gauge;

/* Load a gauge field (Sec. II A: links U_mu(x) in SU(3)).
 * U: canonical complex128 (4, V, 3, 3), device or host.  The library keeps
 * even-odd reordered copies in FP64 (18 reals), in FP32 and FP16 (geom->recon
 * reals) and in double-float (18 hi/lo FP32 pairs); the caller's buffer is not
 * referenced after the call returns.
 * Errors: QCD_ERR_ARG for a NULL pointer, odd or non-positive extents, bc not
 * +-1, recon not 12/18, or V >= 2^31; QCD_ERR_OOM if the copies do not fit. */
qcd_status qcd_gauge_load(const qcd_geom* geom, const void* U, void* stream, qcd_gauge** out);

/* Release a handle and everything it owns (NULL is accepted).  Synchronises
 * the device before freeing. */
qcd_status qcd_gauge_free(qcd_gauge* g);

/* Bytes of one INTERNAL single-parity buffer holding `nrhs` right-hand sides
 * of `fermion` (Ls slices for domain-wall) in precision `prec`; 0 on invalid
 * arguments. */
size_t qcd_field_bytes(const qcd_geom* geom, const qcd_fermion* fermion, qcd_prec prec,
                       int32_t nrhs);

/* Convert between canonical complex128 fields and INTERNAL buffers.
 * pack: the sites of `parity` (0 even, 1 odd) of `canon` (nrhs, [Ls,] V, 4, 3)
 * are written to `internal` (qcd_field_bytes bytes, device memory) in `prec`
 * (FP16: binary16 of psi/s with s the largest |component| of the site, round
 * to nearest even).  unpack: the reverse; sites of the other parity in
 * `canon` are left untouched.  `canon` may be host or device memory. */
qcd_status qcd_field_pack(const qcd_gauge* g, const qcd_fermion* fermion, qcd_prec prec,
                          int32_t parity, const void* canon, void* internal, int32_t nrhs,
                          void* stream);
qcd_status qcd_field_unpack(const qcd_gauge* g, const qcd_fermion* fermion, qcd_prec prec,
                            int32_t parity, const void* internal, void* canon, int32_t nrhs,
                            void* stream);

/* Apply an operator (Eq. (1) / Eq. (2)) to `nrhs` right-hand sides at once;
 * the links of a site are loaded once for all of them.
 *   Wilson:      D_EO = H_eo,  D_OE = H_oe,  MHAT = 1 - kappa^2 H_eo H_oe,
 *                MHAT_DAG = 1 - kappa^2 (H^dag)_eo (H^dag)_oe, FULL = 1 - kappa H.
 *   Domain-wall: D_EO / D_OE = the 4D hop H on every s slice;
 *                MHAT = 1 - 1/4 W H_eo W H_oe with W = B A^-1 the inverse of
 *                the site-local part A B^-1 of D B^-1 (Shamir: B = 1, W = A^-1
 *                with A = 5 - M5 plus the s couplings of Eq. (2); Mobius:
 *                D = A - 1/2 H B, see qcd_fermion);
 *                MHAT_DAG = 1 - 1/4 (H^dag)_eo W^dag (H^dag)_oe W^dag;
 *                FULL = D (Eq. (2) for Shamir).
 *                MHAT is the Schur complement of D B^-1 on the even sites,
 *                left-multiplied by the inverse of its even-even block; the
 *                solver works with x' = B x.
 * layout CANON: in/out are full-lattice canonical complex128 fields (device or
 *   host); for D_EO the odd sites of `in` are read and out is written on the
 *   even sites and zeroed on the odd ones (D_OE: the reverse; MHAT: even to
 *   even).  The arithmetic runs in `prec`.
 * layout INTERNAL: in/out are single-parity device buffers in `prec` (see
 *   qcd_field_bytes / qcd_field_pack); FULL is not available there.
 * in and out must not overlap.  Asynchronous on device buffers. */
qcd_status qcd_dslash(const qcd_gauge* g, const qcd_fermion* fermion, qcd_prec prec, int32_t op,
                      const void* in, void* out, int32_t nrhs, int32_t layout, void* stream);

/* Solve A x = b for nrhs right-hand sides (A = M for Wilson, D_DW for
 * domain-wall; A^dag with params->dagger), by even-odd preconditioned
 * BiCGStab (Wilson) or CG on Mhat^dag Mhat, then reconstruction of the odd
 * sites (domain-wall: of x' = B x, then x = B^-1 x').  b, x: canonical
 * complex128, device or host.  info: host array of
 * nrhs entries.  Returns QCD_OK when every right-hand side reached tol,
 * QCD_ERR_NOCONV / QCD_ERR_BREAKDOWN / QCD_ERR_NAN otherwise (x then holds the
 * last double-precision iterate). */
qcd_status qcd_solve(const qcd_gauge* g, const qcd_fermion* fermion,
                     const qcd_solver_params* params, const void* b, void* x, int32_t nrhs,
                     qcd_solve_info* info, void* stream);

/* Fermion force for S = phi^dag (M^dag M)^-1 phi (Wilson, full M = 1 - kappa H):
 * given eta = M^-dag phi and X = M^-1 eta (canonical (V,4,3) complex128,
 * device), write dS/dRe U_ab and dS/dIm U_ab for every link into dSdU
 * ((4, V, 3, 3, 2) float64, device), treating the 18 reals of a link as
 * independent:  dS = 2 kappa Re(eta^dag dH X).  Asynchronous. */
qcd_status qcd_force(const qcd_gauge* g, const qcd_fermion* fermion, const void* X,
                     const void* eta, void* dSdU, void* stream);

/* Fermion force of the even-odd pseudofermion action S = phi_e^dag (Mhat^dag
 * Mhat)^-1 phi_e (Wilson, Mhat = 1 - kappa^2 H_eo H_oe on the even sites; the
 * consumer of repeated solves in ensemble generation, Sec. II A): given
 * X = (Mhat^dag Mhat)^-1 phi_e and Y = Mhat X as canonical (V,4,3) complex128
 * fields (device; their odd sites are ignored), write dS/dRe U_ab and
 * dS/dIm U_ab into dSdU ((4, V, 3, 3, 2) float64, device):
 *   dS = 2 kappa^2 Re(eta^dag dH xi),  xi = (X, H_oe X),  eta = (Y, (H^dag)_oe Y).
 * X and Y can be had from two solves: z = the even part of the solution of
 * M^dag z = (phi_e, 0) is (Mhat^dag)^-1 phi_e, so Y = z and X = the even part
 * of the solution of M x = (z, 0); S = |z|^2.  Asynchronous. */
qcd_status qcd_force_eo(const qcd_gauge* g, const qcd_fermion* fermion, const void* X,
                        const void* Y, void* dSdU, void* stream);

/* Project a link derivative onto su(3): F_mu(x) = P_TA(U_mu(x) G_mu(x)^dag) with
 * G = dS/dRe U + i dS/dIm U (dSdU as written by qcd_force / qcd_force_eo) and
 * P_TA(M) = (M - M^dag)/2 - tr(M - M^dag)/6, using the handle's links.  For a
 * traceless Hermitian T, the derivative of S along U_mu(x) -> exp(i eps T) U_mu(x)
 * is tr(i T F_mu(x)).  F: canonical (4, V, 3, 3) complex128, device.
 * Asynchronous. */
qcd_status qcd_force_project(const qcd_gauge* g, const void* dSdU, void* F, void* stream);

/* Molecular-dynamics updates on canonical arrays of nlinks 3x3 complex128
 * matrices (device; e.g. (4, V, 3, 3) gauge links and su(3) momenta):
 *   qcd_link_update: U <- exp(eps P) U for every link (P traceless
 *     anti-Hermitian; exp by scaling and squaring of a degree-13 Taylor
 *     polynomial, accurate to rounding);
 *   qcd_mom_update:  P <- P + c F;
 *   qcd_mom_energy:  *out = sum over all entries of |P_ab|^2 (= sum tr(P^dag P)),
 *     summed in FP64 in a fixed order; synchronises the stream.  Its partial
 *     sums live in one fixed device array per GPU: calls whose GPU work
 *     overlaps must be ordered by the caller.
 * A gauge handle holds copies of the links: load a new one after updating U.
 * QCD_ERR_ARG for NULL pointers, host pointers or nlinks < 0. */
qcd_status qcd_link_update(void* U, const void* P, double eps, int64_t nlinks, void* stream);
qcd_status qcd_mom_update(void* P, const void* F, double c, int64_t nlinks, void* stream);
qcd_status qcd_mom_energy(const void* P, int64_t nlinks, double* out, void* stream);

/* Squared norm |psi|^2 (sum over sites, spins, colours of |component|^2) of
 * each of the nrhs right-hand sides of a canonical complex128 field
 * (nrhs, [Ls,] V, 4, 3), summed in FP64; e.g. the action S = |eta|^2 with
 * eta = M^-dag phi (Sec. II A: S_F = psi^dag D^-1 psi).  psi: device or host;
 * out: host array of nrhs doubles.  Synchronises the stream. */
qcd_status qcd_norm2(const qcd_gauge* g, const qcd_fermion* fermion, const void* psi, int32_t nrhs,
                     double* out, void* stream);

/* Diagnostics and test hooks (environment variables, read by the library):
 *   QCD_TUNECACHE=<file>   the autotuner's persistent cache (see qcd_set_tuning);
 *   QCD_TUNE_VERBOSE=1     print every timed launch shape to stderr;
 *   QCD_PDL=0              launch the kernels without programmatic dependent
 *                          launch (by default each stencil / solver kernel may be
 *                          scheduled while its predecessor drains; results are
 *                          the same either way);
 *   QCD_FAULT=alloc        every device workspace allocation fails (QCD_ERR_OOM);
 *   QCD_FAULT=nan          qcd_solve poisons its inner residual with NaN after the
 *                          first restart, which the device reductions must report
 *                          (QCD_ERR_NAN);
 *   QCD_FAULT=noconv       qcd_solve stops after one inner iteration (QCD_ERR_NOCONV).
 * The main entry points open an NVTX range named after themselves. */

/* Message describing the last failing call on this thread ("" if none). */
const char* qcd_last_error(void);

/* Autotuner control: mode 0 = off (default launch shapes), 1 = on (default).
 * The tuner times candidate block / tile shapes of the stencil kernels on
 * first use of each (kernel, lattice, precision, nrhs) key and caches the
 * fastest; the cache is also read from and written to the file named by the
 * environment variable QCD_TUNECACHE when set. */
qcd_status qcd_set_tuning(int32_t mode);

/* Allocation-free Wilson Schur operator (the paper has no counterpart; this
 * entry point exists for callers that cannot let the library allocate device
 * memory -- e.g. a framework whose allocator already owns the GPU's memory,
 * a pipeline that cannot afford the device-wide synchronisation of
 * cudaMalloc/cudaFree, or code held to a fixed footprint after start-up).
 * Computes the same as qcd_dslash(g, fermion, prec, dagger ? QCD_OP_MHAT_DAG
 * : QCD_OP_MHAT, in, out, nrhs, QCD_LAYOUT_INTERNAL, stream): out = in -
 * kappa^2 H_eo H_oe in (H -> H^dag for dagger != 0) on INTERNAL single-parity
 * device buffers, without calling cudaMalloc, cudaFree or any allocating
 * routine.  The odd-parity intermediate lives in a fixed device array of
 * QCD_NOALLOC_SCRATCH_BYTES bytes inside the library (present on every GPU
 * that loads the library until the process exits).
 *   - Wilson fermions only (QCD_ERR_UNSUPPORTED otherwise).
 *   - QCD_ERR_ARG if the intermediate (Vh * nrhs sites in `prec`) exceeds
 *     QCD_NOALLOC_SCRATCH_BYTES, before anything is launched.
 *   - The first call on a device looks up the array's device address on that
 *     device; make that first call before any stream capture.
 *   - Every call uses the same array and leaves its contents behind: calls
 *     whose GPU work overlaps (different streams or host threads) race on it
 *     and must be ordered by the caller.
 *   - The stencil runs with the tuner's cached launch shape if there is one,
 *     else the default shape (no timing runs). */
#define QCD_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
qcd_status qcd_mhat_noalloc(const qcd_gauge* g, const qcd_fermion* fermion, qcd_prec prec,
                            int32_t dagger, const void* in, void* out, int32_t nrhs, void* stream);

/* ---------------------------------------------------------------------------
 * Domain decomposition (Sec. IV D; the multi-node runs of Sec. V B-C).
 *
 * The global lattice L[mu] is divided into P[mu] subdomains per direction, of
 * local extent l[mu] = L[mu] / P[mu], which must be even and >= 2 (a site's
 * parity is then the same in local and global coordinates).  Subdomain id =
 * c_x + P_x (c_y + P_y (c_z + P_z c_t)) for grid coordinates c; it holds the
 * global sites c[mu] l[mu] + x[mu], 0 <= x[mu] < l[mu], in the canonical order
 * of the local lattice (x + l_x (y + l_y (z + l_z t))).
 *
 * A half-dslash of output parity p: every subdomain packs, for each cut
 * direction mu (P[mu] > 1), its two faces of input-parity sites as spin-projected
 * half spinors (6 complex numbers, 12 reals per face site; Sec. IV D) -- the low
 * face x_mu = 0 as (1 + sg gamma_mu) psi for the forward hops of its -mu
 * neighbour, the high face as U_mu^dag (1 - sg gamma_mu) psi for the backward
 * hops of its +mu neighbour (sg = -1, or +1 for the adjoint); the faces travel
 * while the interior hops are computed; the hops across the faces are then
 * added to the boundary sites.  Boundary factors bc[mu] = -1 apply to the hops
 * that cross the global boundary.  Subdomains held by this process exchange by
 * device-to-device copies; subdomains of other processes by NCCL send / receive
 * (qcd_dd_attach_nccl), with the solver's FP64 sums all-reduced by NCCL.
 * -------------------------------------------------------------------------- */
typedef struct {
  int32_t L[4];   /* global extents                                              */
  int32_t P[4];   /* subdomains per direction (>= 1)                             */
  int32_t bc[4];  /* global boundary factors, +1 or -1                           */
  int32_t recon;  /* 12 or 18 reals per stored FP32 link                         */
} qcd_dd_geom;

typedef struct qcd_dd qcd_dd;

/* One face message of a subdomain, for the half-dslash of either parity.
 * Sends: side 0 = the low face (x_mu = 0), to the -mu neighbour; side 1 = the
 * high face, to the +mu neighbour.  Receives: side 0 = the halo of the forward
 * hops, from the +mu neighbour's low face; side 1 = the halo of the backward
 * hops, from the -mu neighbour's high face.  nsites = face sites of one parity
 * (l_x l_y l_z l_t / l_mu / 2), each 6 complex numbers in the field's
 * precision, stored component-major. */
typedef struct {
  int32_t mu;
  int32_t side;
  int32_t peer;   /* the other subdomain's id */
  int32_t nsites;
} qcd_dd_msg;

/* The messages of subdomain `id` in the order the NCCL transport posts them
 * (per cut direction in increasing mu: side 0, side 1).  Host only, no GPU
 * needed.  sends / recvs (may be NULL) receive up to 8 entries each.  Returns
 * the number of messages of each kind, or -1 on invalid arguments. */
int32_t qcd_dd_plan(const qcd_dd_geom* geom, int32_t id, qcd_dd_msg* sends, qcd_dd_msg* recvs);

/* Local canonical indices of the sites of one face message, in message order:
 * the sites of `parity` on the face x_mu = 0 (side 0) or x_mu = l_mu - 1
 * (side 1); `sites` holds nsites entries.  Host only. */
qcd_status qcd_dd_face_sites(const qcd_dd_geom* geom, int32_t mu, int32_t side, int32_t parity,
                             int64_t* sites);

/* Create the subdomains ids[0 .. nlocal) held by this process.  U[k]: the
 * canonical local gauge field (4, V_loc, 3, 3) complex128 of subdomain ids[k]
 * (links U_mu(x) of its own sites), device or host.  Each subdomain keeps its
 * own link copies (FP64, FP32) and workspace on the current device.
 * QCD_ERR_ARG for extents that do not divide into even local extents >= 2,
 * ids out of range or repeated. */
qcd_status qcd_dd_create(const qcd_dd_geom* geom, int32_t nlocal, const int32_t* ids, const void* const* U,
                         void* stream, qcd_dd** out);
qcd_status qcd_dd_free(qcd_dd* dd);

/* NCCL transport between processes (one subdomain per process, rank = its id,
 * nranks = the number of subdomains).  qcd_dd_nccl_unique_id writes the 128-byte
 * ncclUniqueId that rank 0 creates and the caller distributes; libnccl.so.2 is
 * loaded at run time.  QCD_ERR_UNSUPPORTED if NCCL cannot be loaded. */
qcd_status qcd_dd_nccl_unique_id(void* id);
qcd_status qcd_dd_attach_nccl(qcd_dd* dd, const void* unique_id, int32_t nranks, int32_t rank);

/* Operators on the local subdomains: in[k], out[k] are canonical local fields
 * (V_loc, 4, 3) complex128 on the device for subdomain ids[k] (the order given
 * to qcd_dd_create).  op: QCD_OP_D_EO, QCD_OP_D_OE, QCD_OP_MHAT, QCD_OP_MHAT_DAG
 * (Wilson, as qcd_dslash); prec: QCD_F64 or QCD_F32.  Asynchronous on `stream`
 * (the exchange runs on the handle's own stream, ordered by events). */
qcd_status qcd_dd_dslash(qcd_dd* dd, const qcd_fermion* fermion, qcd_prec prec, int32_t op,
                         const void* const* in, void* const* out, void* stream);

/* Even-odd BiCGStab on the subdomains (Wilson, one right-hand side): inner
 * QCD_F64, or QCD_F32 with FP64 reliable updates (params->delta; 0 selects
 * 0.01); tol is the target |b - M x| / |b| on the full global system; dagger,
 * x0_given, graphs and CG are not available.  b[k], x[k]: canonical local
 * fields on the device.  info: one entry for the whole system.  Every process
 * must call it together (the dot products are global). */
qcd_status qcd_dd_solve(qcd_dd* dd, const qcd_fermion* fermion, const qcd_solver_params* params,
                        const void* const* b, void* const* x, qcd_solve_info* info, void* stream);

/* Instrumentation: the number of kernels this library has launched in this
 * process so far (a replayed CUDA graph counts each of its kernel nodes). */
qcd_status qcd_kernel_launches(uint64_t* count);

#ifdef __cplusplus
}
#endif

#endif /* QCD_H */
