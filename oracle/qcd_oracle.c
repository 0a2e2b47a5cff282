/*
 * FP64 CPU oracle for the lattice-QCD fermion solve of Kanamori & Matsufuru,
 * "Practical Implementation of Lattice QCD Simulation on Intel Xeon Phi Knights
 * Landing" (arXiv:1712.01505).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * restatement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg load it.  It shares no code, header
 * or table with the CUDA library and includes nothing from it.
 *
 * Everything is double precision complex (C99 `double complex`), one lattice
 * site at a time, with the spin structure applied as explicit 4x4 matrices
 * (no spin-projection trick, no even-odd storage, no fusion).
 *
 * Canonical layouts (shared convention with the inputs, not code):
 *   site index   i = x + Lx*(y + Ly*(z + Lz*t)),  mu = 0,1,2,3 <-> x,y,z,t
 *   gauge field  U[mu][i][a][b]        (4, V, 3, 3) complex, U_ab of U_mu(x)
 *   4D spinor    psi[i][spin][colour]  (V, 4, 3) complex
 *   5D spinor    psi[s][i][spin][col]  (Ls, V, 4, 3) complex, s slowest
 *   bc[mu]       +1 periodic / -1 antiperiodic: the factor a hop picks up
 *                when it wraps around the lattice in direction mu.
 *
 * Readings of the paper used here (the paper leaves them open):
 *   - Dirac matrices in the chiral basis, gamma_k = [[0,-i s_k],[i s_k,0]],
 *     gamma_4 = [[0,1],[1,0]], gamma_5 = gamma_1 gamma_2 gamma_3 gamma_4.
 *   - Wilson operator in hopping-parameter form M = 1 - kappa*H with
 *     kappa = 1/(2(m0+4)), i.e. M = 2 kappa D_W of Eq. (1).
 *   - P_+- = (1 +- gamma_5)/2 in the domain-wall matrix of Eq. (2); the m0 of
 *     the 4D Wilson block is -M5, so the diagonal block is (5 - M5) - H/2.
 *   - Even-odd (Schur) preconditioning on the even sites; for domain-wall the
 *     parity is the 4D parity and the 5D-diagonal block A is inverted per site.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------------ */
/* Dirac matrices (Sec. II B, Eq. (1); basis: chiral, see header)            */
/* ------------------------------------------------------------------------ */

static cplx GAMMA[5][4][4]; /* [0..3] = gamma_1..gamma_4, [4] = gamma_5 */

static void matmul4(cplx c[4][4], cplx a[4][4], cplx b[4][4]) {
  cplx t[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cplx s = 0;
      for (int k = 0; k < 4; ++k) s += a[i][k] * b[k][j];
      t[i][j] = s;
    }
  memcpy(c, t, sizeof t);
}

__attribute__((constructor)) static void init_gamma(void) {
  const cplx sigma[3][2][2] = {{{0, 1}, {1, 0}}, {{0, -I}, {I, 0}}, {{1, 0}, {0, -1}}};
  memset(GAMMA, 0, sizeof GAMMA);
  for (int k = 0; k < 3; ++k)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        GAMMA[k][a][2 + b] = -I * sigma[k][a][b];
        GAMMA[k][2 + a][b] = I * sigma[k][a][b];
      }
  GAMMA[3][0][2] = GAMMA[3][1][3] = GAMMA[3][2][0] = GAMMA[3][3][1] = 1;
  cplx t[4][4];
  matmul4(t, GAMMA[0], GAMMA[1]);
  matmul4(t, t, GAMMA[2]);
  matmul4(GAMMA[4], t, GAMMA[3]);
}

/* Export the matrices so tests can check the Clifford algebra they satisfy. */
void ora_gamma(int k, double* out_re_im /* 4*4*2 */) {
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      out_re_im[(i * 4 + j) * 2] = creal(GAMMA[k][i][j]);
      out_re_im[(i * 4 + j) * 2 + 1] = cimag(GAMMA[k][i][j]);
    }
}

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Threads of the following oracle calls (n >= 1); a no-op without OpenMP. */
void ora_set_num_threads(int n) {
#ifdef _OPENMP
  if (n >= 1) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct {
  int L[4];
  int bc[4];
  long V;
} geom_t;

static geom_t make_geom(const int* L, const int* bc) {
  geom_t g;
  g.V = 1;
  for (int m = 0; m < 4; ++m) {
    g.L[m] = L[m];
    g.bc[m] = bc[m];
    g.V *= L[m];
  }
  return g;
}

static void site_coords(const geom_t* g, long i, int x[4]) {
  for (int m = 0; m < 4; ++m) {
    x[m] = (int)(i % g->L[m]);
    i /= g->L[m];
  }
}

static long site_index(const geom_t* g, const int x[4]) {
  return x[0] + (long)g->L[0] * (x[1] + (long)g->L[1] * (x[2] + (long)g->L[2] * x[3]));
}

static int site_parity(const geom_t* g, long i) {
  int x[4];
  site_coords(g, i, x);
  return (x[0] + x[1] + x[2] + x[3]) & 1;
}

/* Neighbour of x one step along +mu (dir=+1) or -mu (dir=-1); *phase receives
 * the boundary factor bc[mu] if the step wraps, else 1. */
static long neighbour(const geom_t* g, const int x[4], int mu, int dir, double* phase) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  *phase = 1.0;
  y[mu] += dir;
  if (y[mu] == g->L[mu]) {
    y[mu] = 0;
    *phase = g->bc[mu];
  } else if (y[mu] < 0) {
    y[mu] = g->L[mu] - 1;
    *phase = g->bc[mu];
  }
  return site_index(g, y);
}

/* ------------------------------------------------------------------------ */
/* Wilson hopping term H (Eq. (1)):                                          */
/*   H psi(x) = sum_mu (1 - gamma_mu) U_mu(x) psi(x+mu)                      */
/*            + (1 + gamma_mu) U_mu(x-mu)^dag psi(x-mu)                      */
/* and its adjoint H^dag (projectors exchanged), at one site.                */
/* ------------------------------------------------------------------------ */

/* out[s][a] += phase * sum_{s'} P[s][s'] * (W psi)[s'][a], where W = U or U^dag. */
static void add_term(cplx out[4][3], cplx P[4][4], const cplx* U, int use_dagger, const cplx* psi,
                     double phase) {
  cplx Wpsi[4][3];
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < 3; ++a) {
      cplx acc = 0;
      for (int b = 0; b < 3; ++b) {
        cplx w = use_dagger ? conj(U[b * 3 + a]) : U[a * 3 + b];
        acc += w * psi[s * 3 + b];
      }
      Wpsi[s][a] = acc;
    }
  for (int s = 0; s < 4; ++s)
    for (int a = 0; a < 3; ++a) {
      cplx acc = 0;
      for (int t = 0; t < 4; ++t) acc += P[s][t] * Wpsi[t][a];
      out[s][a] += phase * acc;
    }
}

static void hop_site(const geom_t* g, const cplx* U, const cplx* in, long i, int dagger,
                     cplx out[4][3]) {
  int x[4];
  site_coords(g, i, x);
  memset(out, 0, sizeof(cplx) * 12);
  for (int mu = 0; mu < 4; ++mu) {
    cplx Pminus[4][4], Pplus[4][4];
    for (int s = 0; s < 4; ++s)
      for (int t = 0; t < 4; ++t) {
        cplx one = (s == t) ? 1.0 : 0.0;
        Pminus[s][t] = one - GAMMA[mu][s][t];
        Pplus[s][t] = one + GAMMA[mu][s][t];
      }
    double pf, pb;
    long yf = neighbour(g, x, mu, +1, &pf);
    long yb = neighbour(g, x, mu, -1, &pb);
    const cplx* Uf = U + ((long)mu * g->V + i) * 9;  /* U_mu(x)    */
    const cplx* Ub = U + ((long)mu * g->V + yb) * 9; /* U_mu(x-mu) */
    /* H:     forward (1-gamma) U_mu(x) psi(x+mu),  backward (1+gamma) U^dag psi(x-mu)
     * H^dag: forward (1+gamma) U_mu(x) psi(x+mu),  backward (1-gamma) U^dag psi(x-mu) */
    add_term(out, dagger ? Pplus : Pminus, Uf, 0, in + yf * 12, pf);
    add_term(out, dagger ? Pminus : Pplus, Ub, 1, in + yb * 12, pb);
  }
}

/* out = H in (dagger=0) or H^dag in (dagger=1) on the full 4D lattice.
 * out_parity = -1: all sites; 0/1: only sites of that parity are computed,
 * the others are set to zero (the parity restriction H_{p,1-p} when the input
 * vanishes on parity p). */
void ora_hop(const int* L, const int* bc, const cplx* U, const cplx* in, cplx* out, int dagger,
             int out_parity) {
  geom_t g = make_geom(L, bc);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < g.V; ++i) {
    cplx o[4][3];
    if (out_parity >= 0 && site_parity(&g, i) != out_parity) {
      memset(out + i * 12, 0, sizeof(cplx) * 12);
      continue;
    }
    hop_site(&g, U, in, i, dagger, o);
    memcpy(out + i * 12, o, sizeof o);
  }
}

/* (H in)(x) at a list of sites only: out[k] = (H in)(sites[k]), 12 complex each. */
void ora_hop_sites(const int* L, const int* bc, const cplx* U, const cplx* in, const long* sites,
                   long nsites, cplx* out, int dagger) {
  geom_t g = make_geom(L, bc);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < nsites; ++k) {
    cplx o[4][3];
    hop_site(&g, U, in, sites[k], dagger, o);
    memcpy(out + k * 12, o, sizeof o);
  }
}

/* Wilson matrix in hopping-parameter form, M = 1 - kappa H (M^dag: H -> H^dag). */
void ora_wilson(const int* L, const int* bc, double kappa, const cplx* U, const cplx* in, cplx* out,
                int dagger) {
  geom_t g = make_geom(L, bc);
  ora_hop(L, bc, U, in, out, dagger, -1);
#pragma omp parallel for schedule(static)
  for (long k = 0; k < g.V * 12; ++k) out[k] = in[k] - kappa * out[k];
}

/* ------------------------------------------------------------------------ */
/* Vector helpers                                                            */
/* ------------------------------------------------------------------------ */

static cplx vdot(long n, const cplx* a, const cplx* b) { /* sum conj(a_i) b_i */
  double re = 0, im = 0;
#pragma omp parallel for reduction(+ : re, im) schedule(static)
  for (long k = 0; k < n; ++k) {
    cplx p = conj(a[k]) * b[k];
    re += creal(p);
    im += cimag(p);
  }
  return re + I * im;
}

static double vnorm2(long n, const cplx* a) { return creal(vdot(n, a, a)); }

/* ------------------------------------------------------------------------ */
/* Krylov solvers on an abstract operator                                    */
/* ------------------------------------------------------------------------ */

typedef void (*op_fn)(void* ctx, const cplx* in, cplx* out);

/* BiCGStab (van der Vorst 1992) for A x = b, x holds the initial guess.
 * Stops when the recomputed residual satisfies |b - A x| <= tol_abs; when the
 * recursive residual reaches the bound but the true one does not, the
 * iteration restarts from the true residual.  Returns the iteration count
 * (negative if maxiter was reached). */
static long bicgstab(op_fn A, void* ctx, long n, const cplx* b, cplx* x, double tol_abs,
                     long maxiter) {
  cplx* r = malloc(sizeof(cplx) * n);
  cplx* rt = malloc(sizeof(cplx) * n);
  cplx* p = malloc(sizeof(cplx) * n);
  cplx* v = malloc(sizeof(cplx) * n);
  cplx* s = malloc(sizeof(cplx) * n);
  cplx* t = malloc(sizeof(cplx) * n);
  long it = 0;
  int done = 0;
  while (!done) {
    A(ctx, x, r); /* r = b - A x */
    for (long k = 0; k < n; ++k) r[k] = b[k] - r[k];
    if (sqrt(vnorm2(n, r)) <= tol_abs) break;
    if (it >= maxiter) {
      it = -it;
      break;
    }
    memcpy(rt, r, sizeof(cplx) * n);
    memset(p, 0, sizeof(cplx) * n);
    memset(v, 0, sizeof(cplx) * n);
    cplx rho = 1, alpha = 1, omega = 1;
    while (it < maxiter) {
      cplx rho_new = vdot(n, rt, r);
      cplx beta = (rho_new / rho) * (alpha / omega);
      rho = rho_new;
      for (long k = 0; k < n; ++k) p[k] = r[k] + beta * (p[k] - omega * v[k]);
      A(ctx, p, v);
      alpha = rho / vdot(n, rt, v);
      for (long k = 0; k < n; ++k) s[k] = r[k] - alpha * v[k];
      A(ctx, s, t);
      double tt = vnorm2(n, t);
      omega = (tt > 0) ? vdot(n, t, s) / tt : 0.0;
      for (long k = 0; k < n; ++k) {
        x[k] += alpha * p[k] + omega * s[k];
        r[k] = s[k] - omega * t[k];
      }
      ++it;
      if (sqrt(vnorm2(n, r)) <= tol_abs || omega == 0.0) break;
    }
    if (it >= maxiter) {
      A(ctx, x, r);
      for (long k = 0; k < n; ++k) r[k] = b[k] - r[k];
      if (sqrt(vnorm2(n, r)) > tol_abs) it = -it;
      done = 1;
    }
  }
  free(r), free(rt), free(p), free(v), free(s), free(t);
  return it;
}

/* Conjugate gradient (Hestenes-Stiefel) for a Hermitian positive definite A.
 * `check(ctx2, x)` returns nonzero when x is accepted; it is consulted when the
 * recursive residual drops below rtol_abs, and on rejection the recursion is
 * restarted from the true residual with the bound lowered tenfold. */
typedef int (*accept_fn)(void* ctx, const cplx* x);

static long cg(op_fn A, void* ctx, long n, const cplx* b, cplx* x, double rtol_abs,
               accept_fn check, void* cctx, long maxiter) {
  cplx* r = malloc(sizeof(cplx) * n);
  cplx* p = malloc(sizeof(cplx) * n);
  cplx* q = malloc(sizeof(cplx) * n);
  long it = 0;
  for (;;) {
    A(ctx, x, r);
    for (long k = 0; k < n; ++k) r[k] = b[k] - r[k];
    memcpy(p, r, sizeof(cplx) * n);
    double rr = vnorm2(n, r);
    while (sqrt(rr) > rtol_abs && it < maxiter) {
      A(ctx, p, q);
      double alpha = rr / creal(vdot(n, p, q));
      for (long k = 0; k < n; ++k) {
        x[k] += alpha * p[k];
        r[k] -= alpha * q[k];
      }
      double rr_new = vnorm2(n, r);
      double beta = rr_new / rr;
      rr = rr_new;
      for (long k = 0; k < n; ++k) p[k] = r[k] + beta * p[k];
      ++it;
    }
    if (check(cctx, x)) break;
    if (it >= maxiter) {
      it = -it;
      break;
    }
    rtol_abs *= 0.1;
  }
  free(r), free(p), free(q);
  return it;
}

/* ------------------------------------------------------------------------ */
/* Wilson even-odd system (Schur complement on even sites)                   */
/*   M = [[1, -k H_eo], [-k H_oe, 1]],  Mhat = 1 - k^2 H_eo H_oe             */
/*   bhat_e = b_e + k H_eo b_o,  x_o = b_o + k H_oe x_e                      */
/* Vectors are full-lattice arrays that vanish on the parity not in use.    */
/* ------------------------------------------------------------------------ */

typedef struct {
  const int* L;
  const int* bc;
  double kappa;
  const cplx* U;
  int dagger;
  cplx* tmp;
  long V;
} wil_ctx;

static void wilson_mhat(void* c, const cplx* in, cplx* out) {
  wil_ctx* w = c;
  ora_hop(w->L, w->bc, w->U, in, w->tmp, w->dagger, 1);  /* odd  <- even */
  ora_hop(w->L, w->bc, w->U, w->tmp, out, w->dagger, 0); /* even <- odd  */
  for (long k = 0; k < w->V * 12; ++k) out[k] = in[k] - w->kappa * w->kappa * out[k];
}

/* out = Mhat in (or Mhat^dag), in and out live on even sites. */
void ora_wilson_mhat(const int* L, const int* bc, double kappa, const cplx* U, const cplx* in,
                     cplx* out, int dagger) {
  geom_t g = make_geom(L, bc);
  wil_ctx w = {L, bc, kappa, U, dagger, malloc(sizeof(cplx) * g.V * 12), g.V};
  wilson_mhat(&w, in, out);
  free(w.tmp);
}

/* Solve M x = b (dagger=0) or M^dag x = b (dagger=1) on the full lattice with
 * even-odd preconditioned BiCGStab.  x is overwritten.  Returns the BiCGStab
 * iteration count; *resid receives |b - M x| / |b| on the full system. */
long ora_wilson_solve(const int* L, const int* bc, double kappa, const cplx* U, const cplx* b,
                      cplx* x, double tol, long maxiter, int dagger, double* resid) {
  geom_t g = make_geom(L, bc);
  long n = g.V * 12;
  cplx* be = calloc(n, sizeof(cplx));
  cplx* bo = calloc(n, sizeof(cplx));
  cplx* bh = malloc(sizeof(cplx) * n);
  cplx* xe = calloc(n, sizeof(cplx));
  cplx* t = malloc(sizeof(cplx) * n);
  for (long i = 0; i < g.V; ++i) {
    cplx* dst = site_parity(&g, i) ? bo : be;
    memcpy(dst + i * 12, b + i * 12, sizeof(cplx) * 12);
  }
  ora_hop(L, bc, U, bo, t, dagger, 0); /* bhat_e = b_e + k H_eo b_o */
  for (long k = 0; k < n; ++k) bh[k] = be[k] + kappa * t[k];
  wil_ctx w = {L, bc, kappa, U, dagger, malloc(sizeof(cplx) * n), g.V};
  /* the full residual equals (rhat_e, 0) after exact reconstruction */
  double bnorm = sqrt(vnorm2(n, b));
  long it = bicgstab(wilson_mhat, &w, n, bh, xe, tol * bnorm, maxiter);
  ora_hop(L, bc, U, xe, t, dagger, 1); /* x_o = b_o + k H_oe x_e */
  for (long k = 0; k < n; ++k) x[k] = xe[k] + bo[k] + kappa * t[k];
  ora_wilson(L, bc, kappa, U, x, t, dagger);
  for (long k = 0; k < n; ++k) t[k] = b[k] - t[k];
  *resid = sqrt(vnorm2(n, t)) / bnorm;
  free(be), free(bo), free(bh), free(xe), free(t), free(w.tmp);
  return it;
}

/* ------------------------------------------------------------------------ */
/* Domain-wall matrix (Eq. (2))                                              */
/*   (D psi)_s = (D_W + 1) psi_s - P_- psi_{s+1} - P_+ psi_{s-1}              */
/*             + m P_+ psi_{Ls-1} [s = 0] + m P_- psi_0 [s = Ls-1]             */
/* with D_W + 1 = (5 - M5) - H/2 and P_+- = (1 +- gamma_5)/2.                 */
/* The s-couplings (everything but -H/2) form the per-site block A.          */
/* ------------------------------------------------------------------------ */

/* The 4Ls x 4Ls matrix A over (s, spin), index s*4 + spin; A^dag if dagger. */
static void dw_block(int Ls, double M5, double mf, int dagger, cplx* A) {
  int n = 4 * Ls;
  cplx Pp[4][4], Pm[4][4];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cplx one = (i == j) ? 1.0 : 0.0;
      Pp[i][j] = 0.5 * (one + GAMMA[4][i][j]);
      Pm[i][j] = 0.5 * (one - GAMMA[4][i][j]);
    }
  memset(A, 0, sizeof(cplx) * n * n);
  for (int s = 0; s < Ls; ++s)
    for (int i = 0; i < 4; ++i) {
      A[(s * 4 + i) * n + s * 4 + i] += 5.0 - M5;
      for (int j = 0; j < 4; ++j) {
        if (s + 1 < Ls) A[(s * 4 + i) * n + (s + 1) * 4 + j] += -Pm[i][j];
        if (s > 0) A[(s * 4 + i) * n + (s - 1) * 4 + j] += -Pp[i][j];
      }
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      A[(0 * 4 + i) * n + (Ls - 1) * 4 + j] += mf * Pp[i][j];
      A[((Ls - 1) * 4 + i) * n + 0 * 4 + j] += mf * Pm[i][j];
    }
  if (dagger) {
    for (int r = 0; r < n; ++r)
      for (int c = r; c < n; ++c) {
        cplx a = A[r * n + c], bq = A[c * n + r];
        A[r * n + c] = conj(bq);
        A[c * n + r] = conj(a);
      }
  }
}

/* Gauss-Jordan inverse with partial pivoting of an n x n complex matrix. */
static int invert(int n, const cplx* A, cplx* Ainv) {
  cplx* a = malloc(sizeof(cplx) * n * n);
  memcpy(a, A, sizeof(cplx) * n * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Ainv[r * n + c] = (r == c) ? 1.0 : 0.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    for (int r = col + 1; r < n; ++r)
      if (cabs(a[r * n + col]) > cabs(a[piv * n + col])) piv = r;
    if (cabs(a[piv * n + col]) == 0.0) {
      free(a);
      return -1;
    }
    if (piv != col)
      for (int c = 0; c < n; ++c) {
        cplx t = a[col * n + c];
        a[col * n + c] = a[piv * n + c];
        a[piv * n + c] = t;
        t = Ainv[col * n + c];
        Ainv[col * n + c] = Ainv[piv * n + c];
        Ainv[piv * n + c] = t;
      }
    cplx d = a[col * n + col];
    for (int c = 0; c < n; ++c) {
      a[col * n + c] /= d;
      Ainv[col * n + c] /= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      cplx f = a[r * n + col];
      if (f == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        a[r * n + c] -= f * a[col * n + c];
        Ainv[r * n + c] -= f * Ainv[col * n + c];
      }
    }
  }
  free(a);
  return 0;
}

/* out = B in, for a 4Ls x 4Ls (s,spin) matrix B applied at every site and colour. */
static void apply_block(int Ls, long V, const cplx* B, const cplx* in, cplx* out) {
  int n = 4 * Ls;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < V; ++i)
    for (int c = 0; c < 3; ++c)
      for (int r = 0; r < n; ++r) {
        cplx acc = 0;
        for (int q = 0; q < n; ++q) {
          int s = q / 4, sp = q % 4;
          acc += B[r * n + q] * in[((long)s * V + i) * 12 + sp * 3 + c];
        }
        int s = r / 4, sp = r % 4;
        out[((long)s * V + i) * 12 + sp * 3 + c] = acc;
      }
}

/* 5D hop: the 4D H (or H^dag) on every s slice, optionally parity restricted. */
static void hop5(const int* L, const int* bc, int Ls, const cplx* U, const cplx* in, cplx* out,
                 int dagger, int out_parity) {
  geom_t g = make_geom(L, bc);
  for (int s = 0; s < Ls; ++s)
    ora_hop(L, bc, U, in + (long)s * g.V * 12, out + (long)s * g.V * 12, dagger, out_parity);
}

/* out = D_DW in (dagger=0) or D_DW^dag in (dagger=1), Eq. (2). */
void ora_dw(const int* L, const int* bc, int Ls, double M5, double mf, const cplx* U,
            const cplx* in, cplx* out, int dagger) {
  geom_t g = make_geom(L, bc);
  long n = (long)Ls * g.V * 12;
  cplx* A = malloc(sizeof(cplx) * 16 * Ls * Ls);
  cplx* t = malloc(sizeof(cplx) * n);
  dw_block(Ls, M5, mf, dagger, A);
  apply_block(Ls, g.V, A, in, out);
  hop5(L, bc, Ls, U, in, t, dagger, -1);
  for (long k = 0; k < n; ++k) out[k] -= 0.5 * t[k];
  free(A), free(t);
}

/* out = A^{-1} in (or A^{-dag} in) at every 4D site: the inverse of the
 * site-local part of Eq. (2), computed by Gauss-Jordan elimination. */
void ora_dw_ainv(int Ls, long V, double M5, double mf, const cplx* in, cplx* out, int dagger) {
  int n = 4 * Ls;
  cplx* A = malloc(sizeof(cplx) * n * n);
  cplx* Ai = malloc(sizeof(cplx) * n * n);
  dw_block(Ls, M5, mf, dagger, A);
  invert(n, A, Ai);
  apply_block(Ls, V, Ai, in, out);
  free(A), free(Ai);
}

/* out = A in (or A^dag in), the site-local block itself. */
void ora_dw_block_apply(int Ls, long V, double M5, double mf, const cplx* in, cplx* out,
                        int dagger) {
  cplx* A = malloc(sizeof(cplx) * 16 * Ls * Ls);
  dw_block(Ls, M5, mf, dagger, A);
  apply_block(Ls, V, A, in, out);
  free(A);
}

/* Domain-wall even-odd system.  D = [[A, -H_eo/2], [-H_oe/2, A]];
 *   Mhat     = 1 - 1/4 A^-1 H_eo A^-1 H_oe                  (even sites)
 *   Mhat^dag = 1 - 1/4 (H^dag)_eo A^-dag (H^dag)_oe A^-dag
 *   bhat_e   = A^-1 (b_e + 1/2 H_eo A^-1 b_o),  x_o = A^-1 (b_o + 1/2 H_oe x_e) */
typedef struct {
  const int* L;
  const int* bc;
  int Ls;
  const cplx* U;
  long V;
  cplx* Ai;  /* A^-1   (4Ls)^2 */
  cplx* Aid; /* A^-dag (4Ls)^2 */
  cplx *t1, *t2, *t3;
} dw_ctx;

static void dw_mhat_apply(dw_ctx* d, const cplx* in, cplx* out, int dagger) {
  long n = (long)d->Ls * d->V * 12;
  if (!dagger) {
    hop5(d->L, d->bc, d->Ls, d->U, in, d->t1, 0, 1); /* H_oe in       */
    apply_block(d->Ls, d->V, d->Ai, d->t1, d->t2);   /* A^-1 H_oe in  */
    hop5(d->L, d->bc, d->Ls, d->U, d->t2, d->t1, 0, 0);
    apply_block(d->Ls, d->V, d->Ai, d->t1, d->t2);
  } else {
    apply_block(d->Ls, d->V, d->Aid, in, d->t1);
    hop5(d->L, d->bc, d->Ls, d->U, d->t1, d->t2, 1, 1);
    apply_block(d->Ls, d->V, d->Aid, d->t2, d->t1);
    hop5(d->L, d->bc, d->Ls, d->U, d->t1, d->t2, 1, 0);
  }
  for (long k = 0; k < n; ++k) out[k] = in[k] - 0.25 * d->t2[k];
}

static void dw_normal(void* c, const cplx* in, cplx* out) { /* Mhat^dag Mhat */
  dw_ctx* d = c;
  dw_mhat_apply(d, in, d->t3, 0);
  dw_mhat_apply(d, d->t3, out, 1);
}

static int dw_alloc(dw_ctx* d, const int* L, const int* bc, int Ls, double M5, double mf,
                    const cplx* U) {
  geom_t g = make_geom(L, bc);
  int n = 4 * Ls;
  long nv = (long)Ls * g.V * 12;
  d->L = L, d->bc = bc, d->Ls = Ls, d->U = U, d->V = g.V;
  cplx* A = malloc(sizeof(cplx) * n * n);
  d->Ai = malloc(sizeof(cplx) * n * n);
  d->Aid = malloc(sizeof(cplx) * n * n);
  dw_block(Ls, M5, mf, 0, A);
  int rc = invert(n, A, d->Ai);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) d->Aid[r * n + c] = conj(d->Ai[c * n + r]);
  free(A);
  d->t1 = malloc(sizeof(cplx) * nv);
  d->t2 = malloc(sizeof(cplx) * nv);
  d->t3 = malloc(sizeof(cplx) * nv);
  return rc;
}

static void dw_free(dw_ctx* d) { free(d->Ai), free(d->Aid), free(d->t1), free(d->t2), free(d->t3); }

void ora_dw_mhat(const int* L, const int* bc, int Ls, double M5, double mf, const cplx* U,
                 const cplx* in, cplx* out, int dagger) {
  dw_ctx d;
  dw_alloc(&d, L, bc, Ls, M5, mf, U);
  dw_mhat_apply(&d, in, out, dagger);
  dw_free(&d);
}

typedef struct {
  const int* L;
  const int* bc;
  int Ls;
  double M5, mf;
  const cplx* U;
  const cplx* b;
  const cplx* bo;
  cplx* x;
  cplx* t;
  cplx* u;
  double tol_abs;
  dw_ctx* d;
  double resid;
} dw_check_ctx;

/* reconstruct x_o from x_e and accept when |b - D x| <= tol |b| on the full system */
static int dw_accept(void* c, const cplx* xe) {
  dw_check_ctx* k = c;
  dw_ctx* d = k->d;
  long n = (long)d->Ls * d->V * 12;
  hop5(k->L, k->bc, k->Ls, k->U, xe, k->t, 0, 1);
  for (long q = 0; q < n; ++q) k->t[q] = k->bo[q] + 0.5 * k->t[q];
  apply_block(d->Ls, d->V, d->Ai, k->t, k->u);
  for (long q = 0; q < n; ++q) k->x[q] = xe[q] + k->u[q];
  ora_dw(k->L, k->bc, k->Ls, k->M5, k->mf, k->U, k->x, k->t, 0);
  for (long q = 0; q < n; ++q) k->t[q] = k->b[q] - k->t[q];
  k->resid = sqrt(vnorm2(n, k->t));
  return k->resid <= k->tol_abs;
}

/* Solve D_DW x = b by CG on Mhat^dag Mhat (even sites) plus reconstruction.
 * Returns the CG iteration count; *resid receives |b - D x| / |b|. */
long ora_dw_solve(const int* L, const int* bc, int Ls, double M5, double mf, const cplx* U,
                  const cplx* b, cplx* x, double tol, long maxiter, double* resid) {
  geom_t g = make_geom(L, bc);
  long n = (long)Ls * g.V * 12;
  dw_ctx d;
  dw_alloc(&d, L, bc, Ls, M5, mf, U);
  cplx* be = calloc(n, sizeof(cplx));
  cplx* bo = calloc(n, sizeof(cplx));
  cplx* bh = malloc(sizeof(cplx) * n);
  cplx* rhs = malloc(sizeof(cplx) * n);
  cplx* xe = calloc(n, sizeof(cplx));
  cplx* t = malloc(sizeof(cplx) * n);
  cplx* u = malloc(sizeof(cplx) * n);
  for (int s = 0; s < Ls; ++s)
    for (long i = 0; i < g.V; ++i) {
      long off = ((long)s * g.V + i) * 12;
      memcpy((site_parity(&g, i) ? bo : be) + off, b + off, sizeof(cplx) * 12);
    }
  apply_block(Ls, g.V, d.Ai, bo, t); /* bhat_e = A^-1 (b_e + 1/2 H_eo A^-1 b_o) */
  hop5(L, bc, Ls, U, t, u, 0, 0);
  for (long q = 0; q < n; ++q) t[q] = be[q] + 0.5 * u[q];
  apply_block(Ls, g.V, d.Ai, t, bh);
  dw_mhat_apply(&d, bh, rhs, 1); /* normal equations: Mhat^dag bhat */
  double bnorm = sqrt(vnorm2(n, b));
  dw_check_ctx k = {L, bc, Ls, M5, mf, U, b, bo, x, t, u, tol * bnorm, &d, 0.0};
  /* |b - Dx| = |A (Mhat x_e - bhat)| and |Mhat^dag r| <= |Mhat| |r|: start
   * from the normal-residual bound tol*|b|/4 and tighten on rejection */
  long it = cg(dw_normal, &d, n, rhs, xe, 0.25 * tol * bnorm, dw_accept, &k, maxiter);
  dw_accept(&k, xe);
  *resid = k.resid / bnorm;
  dw_free(&d);
  free(be), free(bo), free(bh), free(rhs), free(xe), free(t), free(u);
  return it;
}

/* ------------------------------------------------------------------------ */
/* Fermion force for S = phi^dag (M^dag M)^-1 phi with M = 1 - kappa H:      */
/*   eta = M^-dag phi, X = M^-1 eta, dS = 2 kappa Re(eta^dag dH X).           */
/* For the link U_mu(x) joining x and x+mu (boundary factor s):              */
/*   F_ba = s sum_sp X(x+mu)_{sp,b} conj([(1-gamma_mu) eta(x)]_{sp,a})         */
/*   G_ab = s sum_sp X(x)_{sp,a}    conj([(1+gamma_mu) eta(x+mu)]_{sp,b})      */
/*   dS/dRe U_ab = 2 kappa Re(F_ba + G_ab),                                   */
/*   dS/dIm U_ab = 2 kappa (-Im F_ba + Im G_ab).                              */
/* dSdU has layout (4, V, 3, 3, 2) reals.                                    */
/* ------------------------------------------------------------------------ */
void ora_wilson_force(const int* L, const int* bc, double kappa, const cplx* X, const cplx* eta,
                      double* dSdU) {
  geom_t g = make_geom(L, bc);
#pragma omp parallel for collapse(2) schedule(static)
  for (int mu = 0; mu < 4; ++mu)
    for (long i = 0; i < g.V; ++i) {
      int x[4];
      site_coords(&g, i, x);
      double ph;
      long y = neighbour(&g, x, mu, +1, &ph);
      cplx pe[4][3], qe[4][3]; /* (1-gamma) eta(x),  (1+gamma) eta(x+mu) */
      for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
          cplx accm = 0, accp = 0;
          for (int t = 0; t < 4; ++t) {
            cplx one = (s == t) ? 1.0 : 0.0;
            accm += (one - GAMMA[mu][s][t]) * eta[i * 12 + t * 3 + a];
            accp += (one + GAMMA[mu][s][t]) * eta[y * 12 + t * 3 + a];
          }
          pe[s][a] = accm;
          qe[s][a] = accp;
        }
      double* out = dSdU + ((long)mu * g.V + i) * 18;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          cplx F = 0, G = 0; /* F_ba and G_ab */
          for (int s = 0; s < 4; ++s) {
            F += X[y * 12 + s * 3 + b] * conj(pe[s][a]);
            G += X[i * 12 + s * 3 + a] * conj(qe[s][b]);
          }
          F *= ph;
          G *= ph;
          out[(a * 3 + b) * 2] = 2.0 * kappa * (creal(F) + creal(G));
          out[(a * 3 + b) * 2 + 1] = 2.0 * kappa * (-cimag(F) + cimag(G));
        }
    }
}
