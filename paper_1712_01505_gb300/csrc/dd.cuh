// Domain decomposition bookkeeping shared by the host plan and the kernels
// (Sec. IV D: the lattice is divided among processes; each hop that leaves a
// subdomain is served from a halo of spin-projected half spinors exchanged
// with the neighbouring subdomain, Sec. V B-C).
//
// The global lattice L[mu] is cut into P[mu] subdomains per direction, each of
// local extent l[mu] = L[mu] / P[mu] (even, so that a site's local parity is
// its global parity).  Subdomain id = c_x + P_x (c_y + P_y (c_z + P_z c_t)).
// Local sites use the canonical order of the local lattice.
//
// For a cut direction mu (P[mu] > 1) a subdomain exchanges, per half-dslash
// with output parity p, two faces of input-parity (1 - p) sites:
//   side 0 (low face, x_mu = 0): the projected half spinor (1 + sg gamma_mu) psi(y),
//     sent to the -mu neighbour, which multiplies it by its U_mu(x) for the
//     forward hop of its high-face sites x (y = x + mu);
//   side 1 (high face, x_mu = l_mu - 1): U_mu(y)^dag (1 - sg gamma_mu) psi(y),
//     sent to the +mu neighbour for the backward hop of its low-face sites.
// A face message holds the 6 complex components of each half spinor for the
// l_V / l_mu / 2 face sites of one parity, ordered by the face index below.
#pragma once

namespace qcd {
namespace ddgeom {

// half face index of local site x on the face orthogonal to mu: the other three
// coordinates in increasing direction order, lexicographic, halved (the first of
// them has an even extent, so each parity of the face is numbered 0 .. F - 1)
__host__ __device__ inline int face_half_index(const int l[4], const int x[4], int mu) {
  int f = 0, stride = 1;
  for (int nu = 0; nu < 4; ++nu) {
    if (nu == mu) continue;
    f += x[nu] * stride;
    stride *= l[nu];
  }
  return f >> 1;
}

// the site of parity `par` with half face index fh on the face x_mu = X
__host__ __device__ inline void face_site(const int l[4], int mu, int X, int par, int fh, int x[4]) {
  int d[3], k = 0;
  for (int nu = 0; nu < 4; ++nu)
    if (nu != mu) d[k++] = nu;
  const int f = 2 * fh;
  const int a0 = f % l[d[0]];  // even: l[d[0]] is even
  const int rest = f / l[d[0]];
  const int b = rest % l[d[1]], c = rest / l[d[1]];
  x[mu] = X;
  x[d[0]] = a0 + ((par + X + b + c) & 1);
  x[d[1]] = b;
  x[d[2]] = c;
}

__host__ __device__ inline int local_index(const int l[4], const int x[4]) {
  return x[0] + l[0] * (x[1] + l[1] * (x[2] + l[2] * x[3]));
}

// half-sites per face of direction mu
__host__ __device__ inline int face_half_sites(const int l[4], int mu) {
  return (l[0] * l[1] * l[2] * l[3] / l[mu]) / 2;
}

inline int sub_id(const int P[4], const int c[4]) { return c[0] + P[0] * (c[1] + P[1] * (c[2] + P[2] * c[3])); }

inline void sub_coords(const int P[4], int id, int c[4]) {
  for (int m = 0; m < 4; ++m) {
    c[m] = id % P[m];
    id /= P[m];
  }
}

// the subdomain one step along +-mu (periodic in the grid)
inline int sub_neighbour(const int P[4], const int c[4], int mu, int dir) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  d[mu] = (d[mu] + dir + P[mu]) % P[mu];
  return sub_id(P, d);
}

}  // namespace ddgeom
}  // namespace qcd
