"""Flop and byte model of the fermion matrices and of the even-odd stencils.

Two conventions are kept apart:

* the paper's Table I (Sec. II B 3): per site of the full matrix, single
  precision, every operand counted once per use (no cache reuse):
  Wilson 1368 flop and 1536 B, domain-wall (N_s = 8) 11520 flop and 8256 B;
* the roofline of the GPU stencils: the hopping term alone (1320 flop per
  output site) and the compulsory HBM traffic of one half-dslash (each link
  and each input / output spinor moved once).
"""
from __future__ import annotations

COMPLEX = 2
SPINOR_REALS = 4 * 3 * COMPLEX          # 24
HALF_SPINOR_REALS = 2 * 3 * COMPLEX     # 12
LINK_REALS = {18: 18, 12: 12}

# one direction of the hopping term: spin projection (6 complex additions),
# SU(3) x half spinor (2 x (9 complex multiplications + 6 complex additions)),
# and, for all but the first direction, the accumulation of a full spinor
PROJECT_FLOP = 6 * 2
LINK_MUL_FLOP = 2 * (9 * 6 + 6 * 2)     # 132
ACCUMULATE_FLOP = 12 * 2                # 24
HOP_FLOP_SITE = 8 * (PROJECT_FLOP + LINK_MUL_FLOP) + 7 * ACCUMULATE_FLOP   # 1320
DIAG_FLOP_SITE = 2 * SPINOR_REALS       # (m0 + 4) psi - H psi / 2: a multiply and an add per real
FIFTH_DIM_FLOP_SITE = 72                # domain-wall s-couplings: P_+ psi_{s-1} + P_- psi_{s+1} terms


def real_bytes(prec: str) -> int:
    return {"f64": 8, "f32": 4, "f16": 2}[prec]


def spinor_bytes(prec: str) -> int:
    """Stored bytes of one site spinor (FP16 adds its FP32 scale)."""
    return SPINOR_REALS * real_bytes(prec) + (4 if prec == "f16" else 0)


def link_bytes(prec: str, recon: int = 18) -> int:
    return LINK_REALS[recon] * real_bytes(prec)


def table1_wilson(prec: str = "f32"):
    """(flop, bytes) per site of the full Wilson matrix, Table I convention."""
    flop = HOP_FLOP_SITE + DIAG_FLOP_SITE
    nbytes = 8 * (spinor_bytes(prec) + link_bytes(prec)) + 2 * spinor_bytes(prec)
    return flop, nbytes


def table1_domain_wall(ns: int, prec: str = "f32"):
    """(flop, bytes) per 4D site of the domain-wall matrix, Table I convention: the links
    once per 4D site, each of the ns slices with 8 neighbour spinors, its own and its output."""
    flop = ns * (HOP_FLOP_SITE + DIAG_FLOP_SITE + FIFTH_DIM_FLOP_SITE)
    nbytes = 8 * link_bytes(prec) + ns * (8 * spinor_bytes(prec) + 2 * spinor_bytes(prec))
    return flop, nbytes


def hop_compulsory_bytes(prec: str, recon: int = 18, slices: int = 1) -> float:
    """HBM bytes per output (site, slice) of one half-dslash: links shared by `slices`."""
    return 8 * link_bytes(prec, recon) / slices + 2 * spinor_bytes(prec)
