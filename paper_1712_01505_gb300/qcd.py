"""Thin Python binding of the C ABI in ``include/qcd.h`` (argument marshalling only).

Every operation runs in ``libqcd.so`` (hand-written sm_103a CUDA).  Fields are
passed as torch tensors (device memory, used in place) or numpy arrays (host
memory, staged by the library), in the canonical complex128 layouts:

* gauge field ``(4, V, 3, 3)``
* spinor ``(nrhs, V, 4, 3)`` (Wilson) or ``(nrhs, Ls, V, 4, 3)`` (domain-wall);
  a single right-hand side may drop the leading ``nrhs`` axis
* force ``(4, V, 3, 3, 2)`` float64

There is no fallback: if the library is missing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqcd.so")

# qcd_status
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOCONV, ERR_BREAKDOWN, ERR_NAN, ERR_TIMEOUT, ERR_UNSUPPORTED = range(9)
STATUS_NAMES = ["OK", "ERR_ARG", "ERR_CUDA", "ERR_OOM", "ERR_NOCONV", "ERR_BREAKDOWN", "ERR_NAN",
                "ERR_TIMEOUT", "ERR_UNSUPPORTED"]
# qcd_prec
F64, F32, F16, DF64 = 0, 1, 2, 3
PREC = {"f64": F64, "f32": F32, "f16": F16, "df64": DF64, F64: F64, F32: F32, F16: F16, DF64: DF64}
# qcd_fermion_type
WILSON, DWF, MOBIUS = 0, 1, 2
# qcd_op
D_EO, D_OE, MHAT, MHAT_DAG, FULL, FULL_DAG = range(6)
OPS = {"D_EO": D_EO, "D_OE": D_OE, "MHAT": MHAT, "MHAT_DAG": MHAT_DAG, "FULL": FULL, "FULL_DAG": FULL_DAG}
# qcd_layout
CANON, INTERNAL = 0, 1
# qcd_method
BICGSTAB, CG_NORMAL = 0, 1

# every symbol the header declares
SYMBOLS = ["qcd_gauge_load", "qcd_gauge_free", "qcd_field_bytes", "qcd_field_pack", "qcd_field_unpack",
           "qcd_dslash", "qcd_solve", "qcd_force", "qcd_last_error", "qcd_set_tuning", "qcd_kernel_launches",
           "qcd_mhat_noalloc", "qcd_norm2", "qcd_force_eo", "qcd_force_project", "qcd_link_update",
           "qcd_mom_update", "qcd_mom_energy", "qcd_dd_plan", "qcd_dd_face_sites", "qcd_dd_create", "qcd_dd_free",
           "qcd_dd_nccl_unique_id", "qcd_dd_attach_nccl", "qcd_dd_dslash", "qcd_dd_solve"]


class QCDError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{name}: {msg}")


class Geom(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32 * 4), ("bc", ctypes.c_int32 * 4), ("recon", ctypes.c_int32)]


class Fermion(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("kappa", ctypes.c_double), ("Ls", ctypes.c_int32),
                ("M5", ctypes.c_double), ("mf", ctypes.c_double), ("b5", ctypes.c_double),
                ("c5", ctypes.c_double)]


class SolverParams(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int32), ("tol", ctypes.c_double), ("maxiter", ctypes.c_int32),
                ("inner", ctypes.c_int32), ("delta", ctypes.c_double), ("use_graph", ctypes.c_int32),
                ("graph_chunk", ctypes.c_int32), ("x0_given", ctypes.c_int32), ("dagger", ctypes.c_int32),
                ("outer", ctypes.c_int32)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("outer_updates", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("status", ctypes.c_int32), ("true_resid", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class DDGeom(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32 * 4), ("P", ctypes.c_int32 * 4), ("bc", ctypes.c_int32 * 4),
                ("recon", ctypes.c_int32)]


class DDMsg(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_int32), ("side", ctypes.c_int32), ("peer", ctypes.c_int32),
                ("nsites", ctypes.c_int32)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libqcd.so (after torch, so that both share one CUDA runtime)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    try:
        import torch  # noqa: F401  (loads the CUDA runtime first)
    except ImportError:
        pass
    lib = ctypes.CDLL(path)
    vp, i32 = ctypes.c_void_p, ctypes.c_int32
    lib.qcd_gauge_load.argtypes = [ctypes.POINTER(Geom), vp, vp, ctypes.POINTER(vp)]
    lib.qcd_gauge_free.argtypes = [vp]
    lib.qcd_field_bytes.argtypes = [ctypes.POINTER(Geom), ctypes.POINTER(Fermion), i32, i32]
    lib.qcd_field_bytes.restype = ctypes.c_size_t
    lib.qcd_field_pack.argtypes = [vp, ctypes.POINTER(Fermion), i32, i32, vp, vp, i32, vp]
    lib.qcd_field_unpack.argtypes = [vp, ctypes.POINTER(Fermion), i32, i32, vp, vp, i32, vp]
    lib.qcd_dslash.argtypes = [vp, ctypes.POINTER(Fermion), i32, i32, vp, vp, i32, i32, vp]
    lib.qcd_solve.argtypes = [vp, ctypes.POINTER(Fermion), ctypes.POINTER(SolverParams), vp, vp, i32,
                              ctypes.POINTER(SolveInfo), vp]
    lib.qcd_force.argtypes = [vp, ctypes.POINTER(Fermion), vp, vp, vp, vp]
    lib.qcd_last_error.restype = ctypes.c_char_p
    lib.qcd_set_tuning.argtypes = [i32]
    lib.qcd_kernel_launches.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
    lib.qcd_mhat_noalloc.argtypes = [vp, ctypes.POINTER(Fermion), i32, i32, vp, vp, i32, vp]
    lib.qcd_norm2.argtypes = [vp, ctypes.POINTER(Fermion), vp, i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.qcd_force_eo.argtypes = [vp, ctypes.POINTER(Fermion), vp, vp, vp, vp]
    lib.qcd_force_project.argtypes = [vp, vp, vp, vp]
    lib.qcd_link_update.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int64, vp]
    lib.qcd_mom_update.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int64, vp]
    lib.qcd_mom_energy.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), vp]
    pp = ctypes.POINTER(vp)
    lib.qcd_dd_plan.argtypes = [ctypes.POINTER(DDGeom), i32, ctypes.POINTER(DDMsg), ctypes.POINTER(DDMsg)]
    lib.qcd_dd_plan.restype = i32
    lib.qcd_dd_face_sites.argtypes = [ctypes.POINTER(DDGeom), i32, i32, i32, ctypes.POINTER(ctypes.c_int64)]
    lib.qcd_dd_create.argtypes = [ctypes.POINTER(DDGeom), i32, ctypes.POINTER(i32), pp, vp, ctypes.POINTER(vp)]
    lib.qcd_dd_free.argtypes = [vp]
    lib.qcd_dd_nccl_unique_id.argtypes = [vp]
    lib.qcd_dd_attach_nccl.argtypes = [vp, vp, i32, i32]
    lib.qcd_dd_dslash.argtypes = [vp, ctypes.POINTER(Fermion), i32, i32, pp, pp, vp]
    lib.qcd_dd_solve.argtypes = [vp, ctypes.POINTER(Fermion), ctypes.POINTER(SolverParams), pp, pp,
                                 ctypes.POINTER(SolveInfo), vp]
    for name in ("qcd_gauge_load", "qcd_gauge_free", "qcd_field_pack", "qcd_field_unpack", "qcd_dslash",
                 "qcd_solve", "qcd_force", "qcd_set_tuning", "qcd_kernel_launches", "qcd_mhat_noalloc",
                 "qcd_norm2", "qcd_force_eo", "qcd_force_project", "qcd_link_update", "qcd_mom_update",
                 "qcd_mom_energy", "qcd_dd_face_sites", "qcd_dd_create", "qcd_dd_free", "qcd_dd_nccl_unique_id",
                 "qcd_dd_attach_nccl", "qcd_dd_dslash", "qcd_dd_solve"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status: int):
    if status != OK:
        raise QCDError(status, load_library().qcd_last_error().decode())


def _ptr(a):
    """Device pointer of a torch tensor or host pointer of a numpy array (must be contiguous)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(a.data_ptr())


def _stream(stream):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return ctypes.c_void_p(0)


def wilson(kappa: float) -> Fermion:
    """Wilson fermion, Eq. (1), hopping parameter kappa = 1/(2(m0+4))."""
    return Fermion(WILSON, float(kappa), 0, 0.0, 0.0, 0.0, 0.0)


def dwf(Ls: int, M5: float, mf: float) -> Fermion:
    """Domain-wall fermion, Eq. (2): N_s = Ls, m0 = -M5, quark mass mf."""
    return Fermion(DWF, 0.0, int(Ls), float(M5), float(mf), 1.0, 0.0)


def mobius(Ls: int, M5: float, mf: float, b5: float, c5: float) -> Fermion:
    """Mobius domain-wall fermion: D = (b5 D_W + 1) - (1 - c5 D_W) S, Eq. (2) at b5 = 1, c5 = 0."""
    return Fermion(MOBIUS, 0.0, int(Ls), float(M5), float(mf), float(b5), float(c5))


def kernel_launches() -> int:
    """Kernels launched by the library so far in this process."""
    n = ctypes.c_uint64()
    _check(load_library().qcd_kernel_launches(ctypes.byref(n)))
    return int(n.value)


def set_tuning(on: bool):
    _check(load_library().qcd_set_tuning(1 if on else 0))


@dataclass
class Gauge:
    """A loaded gauge field (qcd_gauge handle)."""
    L: tuple
    bc: tuple
    recon: int
    handle: ctypes.c_void_p

    @classmethod
    def load(cls, U, L, bc=(1, 1, 1, -1), recon=18, stream=None) -> "Gauge":
        lib = load_library()
        g = Geom((ctypes.c_int32 * 4)(*L), (ctypes.c_int32 * 4)(*bc), recon)
        h = ctypes.c_void_p()
        _check(lib.qcd_gauge_load(ctypes.byref(g), _ptr(U), _stream(stream), ctypes.byref(h)))
        return cls(tuple(L), tuple(bc), int(recon), h)

    @property
    def geom(self) -> Geom:
        return Geom((ctypes.c_int32 * 4)(*self.L), (ctypes.c_int32 * 4)(*self.bc), self.recon)

    @property
    def V(self) -> int:
        return int(np.prod(self.L))

    def free(self):
        if self.handle:
            _check(load_library().qcd_gauge_free(self.handle))
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def field_bytes(gauge: Gauge, fermion: Fermion, prec="f32", nrhs=1) -> int:
    g = gauge.geom
    return int(load_library().qcd_field_bytes(ctypes.byref(g), ctypes.byref(fermion), PREC[prec], nrhs))


def field_pack(gauge, fermion, prec, parity, canon, internal, nrhs=1, stream=None):
    _check(load_library().qcd_field_pack(gauge.handle, ctypes.byref(fermion), PREC[prec], parity,
                                         _ptr(canon), _ptr(internal), nrhs, _stream(stream)))


def field_unpack(gauge, fermion, prec, parity, internal, canon, nrhs=1, stream=None):
    _check(load_library().qcd_field_unpack(gauge.handle, ctypes.byref(fermion), PREC[prec], parity,
                                           _ptr(internal), _ptr(canon), nrhs, _stream(stream)))


def dslash(gauge, fermion, op, inp, out, prec="f64", nrhs=1, layout=CANON, stream=None):
    """qcd_dslash: out = op(in) for nrhs right-hand sides (see include/qcd.h)."""
    op = OPS[op] if isinstance(op, str) else int(op)
    _check(load_library().qcd_dslash(gauge.handle, ctypes.byref(fermion), PREC[prec], op, _ptr(inp),
                                     _ptr(out), nrhs, layout, _stream(stream)))
    return out


NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024


def mhat_noalloc(gauge, fermion, inp, out, prec="f32", dagger=False, nrhs=1, stream=None):
    """qcd_mhat_noalloc: Wilson Mhat (Mhat^dag) on INTERNAL buffers without device allocation."""
    _check(load_library().qcd_mhat_noalloc(gauge.handle, ctypes.byref(fermion), PREC[prec], int(dagger),
                                           _ptr(inp), _ptr(out), nrhs, _stream(stream)))
    return out


def solver_params(method=BICGSTAB, tol=1e-10, maxiter=100000, inner="f64", delta=0.0, use_graph=False,
                  graph_chunk=32, x0_given=False, dagger=False, outer="f64") -> SolverParams:
    return SolverParams(method, tol, maxiter, PREC[inner], delta, int(use_graph), graph_chunk, int(x0_given),
                        int(dagger), PREC[outer])


def solve(gauge, fermion, b, x, nrhs=1, stream=None, check=True, **kw):
    """qcd_solve: x = A^-1 b; returns the list of per-rhs info dicts."""
    prm = solver_params(**kw)
    info = (SolveInfo * nrhs)()
    st = load_library().qcd_solve(gauge.handle, ctypes.byref(fermion), ctypes.byref(prm), _ptr(b), _ptr(x),
                                  nrhs, info, _stream(stream))
    if check:
        _check(st)
    return [i.as_dict() for i in info], st


def norm2(gauge, fermion, psi, nrhs=1, stream=None):
    """qcd_norm2: |psi|^2 per right-hand side (FP64 sums), as a list of floats."""
    out = (ctypes.c_double * nrhs)()
    _check(load_library().qcd_norm2(gauge.handle, ctypes.byref(fermion), _ptr(psi), nrhs, out,
                                    _stream(stream)))
    return list(out)


def force(gauge, fermion, X, eta, out, stream=None):
    """qcd_force: dS/dU for S = phi^dag (M^dag M)^-1 phi given X = M^-1 eta, eta = M^-dag phi."""
    _check(load_library().qcd_force(gauge.handle, ctypes.byref(fermion), _ptr(X), _ptr(eta), _ptr(out),
                                    _stream(stream)))
    return out


def force_eo(gauge, fermion, X, Y, out, stream=None):
    """qcd_force_eo: dS/dU for S = phi_e^dag (Mhat^dag Mhat)^-1 phi_e given X = (Mhat^dag Mhat)^-1 phi_e and
    Y = Mhat X (canonical full-lattice fields, odd sites ignored)."""
    _check(load_library().qcd_force_eo(gauge.handle, ctypes.byref(fermion), _ptr(X), _ptr(Y), _ptr(out),
                                       _stream(stream)))
    return out


def force_project(gauge, dSdU, out, stream=None):
    """qcd_force_project: F = P_TA(U G^dag), G = dS/dRe U + i dS/dIm U, as (4, V, 3, 3) complex128."""
    _check(load_library().qcd_force_project(gauge.handle, _ptr(dSdU), _ptr(out), _stream(stream)))
    return out


def link_update(U, P, eps, stream=None):
    """qcd_link_update: U <- exp(eps P) U for every 3x3 matrix of U (device complex128 arrays)."""
    _check(load_library().qcd_link_update(_ptr(U), _ptr(P), float(eps), U.numel() // 9, _stream(stream)))
    return U


def mom_update(P, F, c, stream=None):
    """qcd_mom_update: P <- P + c F."""
    _check(load_library().qcd_mom_update(_ptr(P), _ptr(F), float(c), P.numel() // 9, _stream(stream)))
    return P


def mom_energy(P, stream=None) -> float:
    """qcd_mom_energy: sum over all entries of |P_ab|^2."""
    out = ctypes.c_double()
    _check(load_library().qcd_mom_energy(_ptr(P), P.numel() // 9, ctypes.byref(out), _stream(stream)))
    return out.value
