"""Domain decomposition of the lattice (Sec. IV D): partition helpers and the binding of the
``qcd_dd_*`` calls of ``include/qcd.h`` (argument marshalling only; packing, the exchange,
the stencils and the solver run in ``libqcd.so``).

The global lattice ``L`` is cut into ``P[mu]`` subdomains per direction, of local extent
``l = L // P`` (even, >= 2).  Subdomain ``id = c_x + P_x (c_y + P_y (c_z + P_z c_t))`` holds the
global sites ``c * l + x`` in the canonical order of the local lattice.  One process may hold
several subdomains (they exchange faces by device copies: the one-GPU configuration), or one
subdomain per process with NCCL between processes (``attach_nccl``).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import qcd


def local_extents(L, P):
    l = tuple(int(a) // int(b) for a, b in zip(L, P))
    for a, b, c in zip(L, P, l):
        if a % b or c < 2 or c % 2:
            raise ValueError(f"L = {tuple(L)} does not divide into even local extents >= 2 with P = {tuple(P)}")
    return l


def sub_coords(P, sid):
    c = []
    for m in range(4):
        c.append(sid % P[m])
        sid //= P[m]
    return tuple(c)


def sub_id(P, c):
    return int(c[0] + P[0] * (c[1] + P[1] * (c[2] + P[2] * c[3])))


def global_sites(L, P, sid):
    """Global canonical index of every local site of subdomain ``sid``, in local canonical order."""
    l = local_extents(L, P)
    c = sub_coords(P, sid)
    t, z, y, x = np.meshgrid(*[np.arange(n) for n in l[::-1]], indexing="ij")
    g = [x.reshape(-1) + c[0] * l[0], y.reshape(-1) + c[1] * l[1], z.reshape(-1) + c[2] * l[2],
         t.reshape(-1) + c[3] * l[3]]
    return g[0] + L[0] * (g[1] + L[1] * (g[2] + L[2] * g[3]))


def scatter_gauge(U, L, P, sid):
    """The links U_mu(x) of the subdomain's sites, canonical local (4, V_loc, 3, 3)."""
    return np.ascontiguousarray(U[:, global_sites(L, P, sid)])


def scatter_spinor(psi, L, P, sid):
    """A global (V, 4, 3) field restricted to the subdomain, canonical local (V_loc, 4, 3)."""
    return np.ascontiguousarray(psi[global_sites(L, P, sid)])


def gather_spinor(parts, L, P, ids):
    """Assemble local (V_loc, 4, 3) fields of the subdomains ``ids`` into a global (V, 4, 3) field."""
    V = int(np.prod(L))
    out = np.zeros((V, 4, 3), dtype=np.complex128)
    for sid, part in zip(ids, parts):
        out[global_sites(L, P, sid)] = part
    return out


def geom(L, P, bc, recon=18):
    g = qcd.DDGeom()
    g.L[:] = list(L)
    g.P[:] = list(P)
    g.bc[:] = list(bc)
    g.recon = recon
    return g


def plan(L, P, bc, sid):
    """(sends, recvs) of subdomain ``sid``: lists of dicts mu, side, peer, nsites (host only)."""
    lib = qcd.load_library()
    sends, recvs = (qcd.DDMsg * 8)(), (qcd.DDMsg * 8)()
    n = lib.qcd_dd_plan(ctypes.byref(geom(L, P, bc)), sid, sends, recvs)
    if n < 0:
        raise qcd.QCDError(qcd.ERR_ARG, lib.qcd_last_error().decode())
    as_d = lambda m: {"mu": m.mu, "side": m.side, "peer": m.peer, "nsites": m.nsites}  # noqa: E731
    return [as_d(sends[k]) for k in range(n)], [as_d(recvs[k]) for k in range(n)]


def face_sites(L, P, bc, mu, side, parity):
    """Local canonical indices of the sites of one face message, in message order (host only)."""
    l = local_extents(L, P)
    n = int(np.prod(l)) // l[mu] // 2
    out = np.empty(n, dtype=np.int64)
    lib = qcd.load_library()
    qcd._check(lib.qcd_dd_face_sites(ctypes.byref(geom(L, P, bc)), mu, side, parity,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return out


def _ptrs(tensors):
    arr = (ctypes.c_void_p * len(tensors))()
    for k, t in enumerate(tensors):
        if not t.is_contiguous():
            raise ValueError("fields must be contiguous")
        arr[k] = t.data_ptr()
    return arr


class Decomposition:
    """The subdomains ``ids`` of this process (``qcd_dd_create``); ``U_local[k]`` holds the links of
    subdomain ``ids[k]`` (device tensor or host array, canonical local layout)."""

    def __init__(self, L, P, bc, ids, U_local, recon=18, stream=None):
        self.L, self.P, self.bc = tuple(L), tuple(P), tuple(bc)
        self.ids = [int(i) for i in ids]
        self.l = local_extents(L, P)
        self.geom = geom(L, P, bc, recon)
        lib = qcd.load_library()
        idarr = (ctypes.c_int32 * len(self.ids))(*self.ids)
        uarr = (ctypes.c_void_p * len(self.ids))()
        for k, u in enumerate(U_local):
            uarr[k] = qcd._ptr(u).value
        h = ctypes.c_void_p()
        qcd._check(lib.qcd_dd_create(ctypes.byref(self.geom), len(self.ids), idarr, uarr, qcd._stream(stream),
                                     ctypes.byref(h)))
        self.handle = h

    def attach_nccl(self, unique_id: bytes, nranks: int, rank: int):
        buf = ctypes.create_string_buffer(bytes(unique_id), 128)
        qcd._check(qcd.load_library().qcd_dd_attach_nccl(self.handle, buf, nranks, rank))

    def dslash(self, fermion, op, inp, out, prec="f64", stream=None):
        op = qcd.OPS[op] if isinstance(op, str) else op
        qcd._check(qcd.load_library().qcd_dd_dslash(self.handle, ctypes.byref(fermion), qcd.PREC[prec], op,
                                                    _ptrs(inp), _ptrs(out), qcd._stream(stream)))
        return out

    def solve(self, fermion, b, x, stream=None, check=True, **kw):
        prm = qcd.solver_params(**kw)
        info = qcd.SolveInfo()
        st = qcd.load_library().qcd_dd_solve(self.handle, ctypes.byref(fermion), ctypes.byref(prm), _ptrs(b),
                                             _ptrs(x), ctypes.byref(info), qcd._stream(stream))
        if check:
            qcd._check(st)
        return info.as_dict(), st

    def free(self):
        if self.handle:
            qcd._check(qcd.load_library().qcd_dd_free(self.handle))
            self.handle = None


def nccl_unique_id() -> bytes:
    buf = ctypes.create_string_buffer(128)
    qcd._check(qcd.load_library().qcd_dd_nccl_unique_id(buf))
    return buf.raw
