"""GPU parity of the domain-wall operator (Eq. (2)) and its CG solve against the FP64 oracle.

The 4D hop acts on every fifth-dimension slice with shared links; the site-local block A and
its closed-form inverse act along s.  Tolerances as for Wilson (FP64 1e-13 element-wise,
FP32 1e-6 and FP16 2e-3 norm-wise); solves to |b - D x| / |b| <= 1e-10 by the oracle's D.
"""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, max_err, rel_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
M5, MF = 1.8, 0.02
TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3}


def _check(out, ref, prec):
    if prec == "f64":
        assert max_err(out, ref) < TOL["f64"]
    else:
        assert rel_err(out, ref) < TOL[prec]


def _case(L, Ls, seed, nrhs=1):
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, seed)
    shape = (nrhs, Ls, V, 4, 3) if nrhs > 1 else (Ls, V, 4, 3)
    return V, U, inputs.gaussian_source(shape, seed + 1)


@pytest.mark.parametrize("L,Ls", [((4, 4, 4, 8), 8), ((6, 4, 2, 10), 5)])
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("f16", 18)])
def test_dw_hop_on_every_slice(L, Ls, prec, recon):
    device()
    V, U, psi = _case(L, Ls, 31)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=recon)
    f = qcd.dwf(Ls, M5, MF)
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "D_EO", to_dev(psi), out, prec=prec)
    torch.cuda.synchronize()
    par = ora.parity(L)
    ref = np.empty_like(psi)
    for s in range(Ls):
        inp = psi[s].copy()
        inp[par == 0] = 0
        ref[s] = ora.hop(L, BC, U, inp, out_parity=0)
    _check(out, ref, prec)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("dag", [False, True])
def test_dw_mhat_and_full(prec, dag):
    device()
    L, Ls = (4, 4, 4, 8), 8
    V, U, psi = _case(L, Ls, 41)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=18)
    f = qcd.dwf(Ls, M5, MF)
    par = ora.parity(L)
    pe = psi.copy()
    pe[:, par == 1] = 0
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", to_dev(psi), out, prec=prec)
    torch.cuda.synchronize()
    _check(out, ora.dw_mhat(L, BC, Ls, M5, MF, U, pe, dagger=dag), prec)
    qcd.dslash(g, f, "FULL_DAG" if dag else "FULL", to_dev(psi), out, prec=prec)
    torch.cuda.synchronize()
    _check(out, ora.dw(L, BC, Ls, M5, MF, U, psi, dagger=dag), prec)


def test_dw_multi_rhs():
    device()
    L, Ls, nrhs = (4, 4, 2, 6), 6, 3
    V, U, psi = _case(L, Ls, 51, nrhs=nrhs)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.dwf(Ls, M5, MF)
    out = torch.empty(psi.shape, dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "FULL", to_dev(psi), out, prec="f32", nrhs=nrhs)
    torch.cuda.synchronize()
    for r in range(nrhs):
        assert rel_err(out[r], ora.dw(L, BC, Ls, M5, MF, U, psi[r])) < 1e-6


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
def test_dw_cg_solve(inner):
    device()
    L, Ls = (4, 4, 4, 8), 8
    V, U, b = _case(L, Ls, 61)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.dwf(Ls, M5, MF)
    x = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, method=qcd.CG_NORMAL, tol=1e-10, inner=inner,
                        use_graph=True, graph_chunk=16)
    assert info[0]["converged"], info
    xr = x.cpu().numpy()
    res = np.linalg.norm(b - ora.dw(L, BC, Ls, M5, MF, U, xr)) / np.linalg.norm(b)
    assert res <= 1e-10
    xo, _, _ = ora.dw_solve(L, BC, Ls, M5, MF, U, b, tol=1e-12)
    assert np.linalg.norm(xr - xo) / np.linalg.norm(xo) < 1e-7


def test_dw_bicgstab_reports_its_outcome():
    """Sec. II C takes CG on the normal equations for domain-wall because BiCGStab fails on its
    spectrum.  BiCGStab on the domain-wall Mhat runs (no refusal); whatever it reaches, the status
    and the true residual it reports describe the x it returns (checked with the oracle's D)."""
    device()
    L, Ls = (4, 4, 4, 8), 8
    V, U, b = _case(L, Ls, 71)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.dwf(Ls, M5, MF)
    x = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    info, st = qcd.solve(g, f, to_dev(b), x, method=qcd.BICGSTAB, tol=1e-10, maxiter=3000, inner="f64",
                         check=False)
    res = np.linalg.norm(b - ora.dw(L, BC, Ls, M5, MF, U, x.cpu().numpy())) / np.linalg.norm(b)
    if info[0]["converged"]:
        assert st == qcd.OK and res <= 1e-10
    else:
        assert st in (qcd.ERR_NOCONV, qcd.ERR_BREAKDOWN, qcd.ERR_NAN)
    if np.isfinite(res):
        assert abs(res - info[0]["true_resid"]) <= 1e-6 * res + 1e-14


# ----------------------------------------------------------------------------- double-float
# hi + lo pairs of FP32 (see test_gpu_dfloat.py for the bound): element-wise 1e-12 of the
# largest output for the hop; M_hat adds two A^-1 applications whose closed-form sums run over
# Ls terms with weights below 1 / (5 - M5), the same bound holds.
DF_TOL = 1e-12


@pytest.mark.parametrize("L,Ls", [((4, 4, 4, 8), 8), ((6, 4, 2, 10), 5)])
def test_dw_double_float_hop_on_every_slice(L, Ls):
    device()
    V, U, psi = _case(L, Ls, 31)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.dwf(Ls, M5, MF)
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "D_OE", to_dev(psi), out, prec="df64")
    torch.cuda.synchronize()
    par = ora.parity(L)
    ref = np.empty_like(psi)
    for s in range(Ls):
        inp = psi[s].copy()
        inp[par == 1] = 0
        ref[s] = ora.hop(L, BC, U, inp, out_parity=1)
    assert max_err(out, ref) < DF_TOL


@pytest.mark.parametrize("dag", [False, True])
@pytest.mark.parametrize("Ls", [8, 16])
def test_dw_double_float_mhat(dag, Ls):
    device()
    L = (4, 4, 4, 8)
    V, U, psi = _case(L, Ls, 41)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.dwf(Ls, M5, MF)
    par = ora.parity(L)
    pe = psi.copy()
    pe[:, par == 1] = 0
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", to_dev(psi), out, prec="df64")
    torch.cuda.synchronize()
    assert max_err(out, ora.dw_mhat(L, BC, Ls, M5, MF, U, pe, dagger=dag)) < DF_TOL
    with pytest.raises(qcd.QCDError, match="ERR_UNSUPPORTED"):
        qcd.dslash(g, f, "FULL", to_dev(psi), out, prec="df64")


@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_dw_cg_solve_with_double_float_outer_steps(inner):
    device()
    L, Ls = (4, 4, 4, 8), 8
    V, U, b = _case(L, Ls, 61)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.dwf(Ls, M5, MF)
    x = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, method=qcd.CG_NORMAL, tol=1e-10, inner=inner,
                        use_graph=True, graph_chunk=16, outer="df64")
    assert info[0]["converged"], info
    xr = x.cpu().numpy()
    res = np.linalg.norm(b - ora.dw(L, BC, Ls, M5, MF, U, xr)) / np.linalg.norm(b)
    assert res <= 1e-10
    assert abs(res - info[0]["true_resid"]) <= 1e-6 * res
    assert info[0]["outer_updates"] >= 2


def test_full_size_dw_hop_on_sampled_sites():
    """Domain-wall benchmark lattice (16^3 x 32, Ls = 16, eps = 0.2 links seed 3, Gaussian source
    seed 0): the FP32 12-real hop on all slices in the benchmark's INTERNAL-layout launch, checked
    on sampled (site, slice) outputs the oracle computes one by one."""
    device()
    L, Ls = (16, 16, 16, 32), 16
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 3)
    psi = inputs.gaussian_source((Ls, V, 4, 3), 0)
    par = ora.parity(L)
    even = np.flatnonzero(par == 0)
    rng = np.random.default_rng(9)
    sites = np.concatenate([even[:32], even[-32:], rng.choice(even, 128, replace=False)])
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.dwf(Ls, M5, MF)
    nb = qcd.field_bytes(g, f, "f32")
    bi = torch.empty(nb, dtype=torch.uint8, device=device())
    bo = torch.empty(nb, dtype=torch.uint8, device=device())
    qcd.field_pack(g, f, "f32", 1, to_dev(psi), bi)
    qcd.dslash(g, f, "D_EO", bi, bo, prec="f32", layout=qcd.INTERNAL)
    out = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.field_unpack(g, f, "f32", 0, bo, out)
    torch.cuda.synchronize()
    idx = torch.from_numpy(sites).to(device())
    for s in (0, 7, Ls - 1):
        inp = psi[s].copy()
        inp[par == 0] = 0
        ref = ora.hop_sites(L, BC, U, inp, sites)
        assert rel_err(out[s][idx].cpu().numpy(), ref) < 1e-6
    g.free()
