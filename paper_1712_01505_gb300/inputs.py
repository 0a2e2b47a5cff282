"""Seeded synthetic inputs shared by the GPU library's tests and benchmark and the oracle.

This module holds no operator, solver or force arithmetic: it only draws the
random gauge fields and sources the workloads are defined on, in the canonical
layouts (gauge ``(4, V, 3, 3)``, spinor ``(V, 4, 3)`` or ``(Ls, V, 4, 3)``,
site index ``x + Lx*(y + Ly*(z + Lz*t))``, complex128).

Gauge fields are the "smoothed random" SU(3) links U = exp(i eps H) with H a
random Hermitian traceless 3x3 matrix of Gaussian entries, reunitarised so that
det U = 1; they stand in for the Monte Carlo ensembles of the paper (Sec. II A),
whose links are SU(3) matrices.
"""
from __future__ import annotations

import os
import tempfile

import numpy as np


def volume(L) -> int:
    return int(np.prod(L))


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def reunitarize(U: np.ndarray) -> np.ndarray:
    """Project (..., 3, 3) matrices close to SU(3) onto SU(3).

    Row 0 is normalised, row 1 is Gram-Schmidt orthogonalised against it and
    normalised, row 2 = conj(row0 x row1), which gives det = 1.
    """
    U = np.array(U, dtype=np.complex128, copy=True)
    r0 = U[..., 0, :]
    r0 = r0 / np.linalg.norm(r0, axis=-1, keepdims=True)
    r1 = U[..., 1, :]
    r1 = r1 - np.sum(np.conj(r0) * r1, axis=-1, keepdims=True) * r0
    r1 = r1 / np.linalg.norm(r1, axis=-1, keepdims=True)
    r2 = np.conj(np.cross(r0, r1))
    return np.stack([r0, r1, r2], axis=-2)


def random_su3_near_identity(n: int, eps: float, rng: np.random.Generator) -> np.ndarray:
    """n matrices exp(i eps H), H Hermitian traceless with Gaussian entries (row-major draws)."""
    g = rng.standard_normal((n, 3, 3, 2))
    A = g[..., 0] + 1j * g[..., 1]
    H = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real / 3.0
    H = H - tr[:, None, None] * np.eye(3)
    lam, vec = np.linalg.eigh(H)
    U = (vec * np.exp(1j * eps * lam)[:, None, :]) @ np.conj(np.swapaxes(vec, -1, -2))
    return reunitarize(U)


def gauge_field(L, eps: float, seed: int) -> np.ndarray:
    """Smoothed random SU(3) gauge field, shape (4, V, 3, 3); links drawn mu-major then by site.

    Fields of 2^20 sites or more are cached as .npy files in $QCD_INPUT_CACHE
    (default: the system temporary directory), since drawing one takes tens of
    seconds; the cache key is (L, eps, seed) and the content is the same array.
    """
    V = volume(L)
    path = None
    if V >= (1 << 20):
        d = os.environ.get("QCD_INPUT_CACHE", os.path.join(tempfile.gettempdir(), "qcd_inputs"))
        path = os.path.join(d, f"gauge_{'x'.join(map(str, L))}_eps{eps:g}_seed{int(seed)}.npy")
        if os.path.exists(path):
            return np.load(path)
    U = random_su3_near_identity(4 * V, eps, _rng(seed)).reshape(4, V, 3, 3)
    if path:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = f"{path}.{os.getpid()}.tmp.npy"
        np.save(tmp, U)
        os.replace(tmp, path)
    return U


def unit_gauge(L) -> np.ndarray:
    """Free field U = 1."""
    V = volume(L)
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3)).copy()


def random_gauge_transform(V: int, seed: int) -> np.ndarray:
    """Random SU(3) matrices Omega(x), shape (V, 3, 3) (QR of a Gaussian matrix, det fixed to 1)."""
    g = _rng(seed).standard_normal((V, 3, 3, 2))
    Q, R = np.linalg.qr(g[..., 0] + 1j * g[..., 1])
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[:, None, None]


def gaussian_source(shape, seed: int) -> np.ndarray:
    """Complex Gaussian field: real and imaginary parts ~ N(0, 1); shape e.g. (V, 4, 3)."""
    g = _rng(seed).standard_normal(tuple(shape) + (2,))
    return g[..., 0] + 1j * g[..., 1]


def z2_source(shape, seed: int) -> np.ndarray:
    """Complex Z2 noise: real and imaginary parts independently +-1/sqrt(2)."""
    s = _rng(seed).integers(0, 2, size=tuple(shape) + (2,)) * 2 - 1
    return (s[..., 0] + 1j * s[..., 1]) / np.sqrt(2.0)


def point_sources(L, seed: int):
    """The 12 spin-colour point sources at one random site x0.

    Returns (x0, b) with b of shape (12, V, 4, 3); right-hand side k = 3*spin + colour
    is 1 at (x0, spin, colour) and 0 elsewhere.
    """
    V = volume(L)
    x0 = int(_rng(seed).integers(0, V))
    b = np.zeros((12, V, 4, 3), dtype=np.complex128)
    for k in range(12):
        b[k, x0, k // 3, k % 3] = 1.0
    return x0, b


def su3_momenta(shape, seed: int) -> np.ndarray:
    """Random su(3) elements (traceless anti-Hermitian 3x3), shape + (3, 3): i times the traceless
    part of the Hermitian part of a complex Gaussian matrix."""
    g = _rng(seed).standard_normal(tuple(shape) + (3, 3, 2))
    a = g[..., 0] + 1j * g[..., 1]
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return 1j * (h - tr[..., None, None] * np.eye(3))
