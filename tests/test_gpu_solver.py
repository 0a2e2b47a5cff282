"""GPU solves (Sec. II C) against the FP64 oracle: every solution must satisfy
|b - A x| / |b| <= 1e-10 with A applied by the ORACLE's full operator, and agree with
the oracle's own solution to within the conditioning of the system."""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


def oracle_resid_wilson(L, kappa, U, b, x, dagger=False):
    return np.linalg.norm(b - ora.wilson(L, BC, kappa, U, x, dagger=dagger)) / np.linalg.norm(b)


def test_config1_wilson_4x4x4x4_fp64_bicgstab():
    """4^4, eps = 0.3 links (seed 1), kappa = 0.12, Gaussian source (seed 0), FP64 EO BiCGStab to 1e-10."""
    device()
    L, kappa = (4, 4, 4, 4), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 1)
    b = inputs.gaussian_source((V, 4, 3), 0)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(kappa)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, method=qcd.BICGSTAB, tol=1e-10, inner="f64")
    xr = x.cpu().numpy()
    assert info[0]["converged"] and info[0]["true_resid"] <= 1e-10
    assert oracle_resid_wilson(L, kappa, U, b, xr) <= 1e-10
    xo, _, res_o = ora.wilson_solve(L, BC, kappa, U, b, tol=1e-12)
    assert np.linalg.norm(xr - xo) / np.linalg.norm(xo) < 1e-8


@pytest.mark.parametrize("inner", ["f64", "f32", "f16"])
@pytest.mark.parametrize("graph", [False, True])
def test_wilson_mixed_precision_reaches_1e10(inner, graph):
    device()
    L, kappa = (8, 8, 8, 8), 0.124
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 4)
    b = inputs.z2_source((V, 4, 3), 0)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(kappa)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, method=qcd.BICGSTAB, tol=1e-10, inner=inner,
                        use_graph=graph, graph_chunk=16)
    assert info[0]["converged"], info
    assert oracle_resid_wilson(L, kappa, U, b, x.cpu().numpy()) <= 1e-10
    if inner != "f64":
        assert info[0]["outer_updates"] >= 2


@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_wilson_cg_normal_adjoint_system(inner):
    # CG on the normal equations of the adjoint system: A = Mhat^dag, iterated on A^dag A = Mhat Mhat^dag
    device()
    L, kappa = (4, 4, 6, 8), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 9)
    b = inputs.gaussian_source((V, 4, 3), 10)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(kappa)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, method=qcd.CG_NORMAL, tol=1e-10, inner=inner, dagger=True)
    assert info[0]["converged"], info
    assert oracle_resid_wilson(L, kappa, U, b, x.cpu().numpy(), dagger=True) <= 1e-10


@pytest.mark.parametrize("method", ["bicgstab", "cg"])
@pytest.mark.parametrize("dagger", [False, True])
def test_wilson_fp16_inner_with_fused_sums(method, dagger):
    # one right-hand side with FP16 inner vectors: the inner products come from the epilogue of
    # the packed FP16 stencil (BiCGStab: (rt, v), (t, s), |t|^2; CG on the normal equations:
    # Re(p, q)); a lattice whose last site block is ragged
    device()
    L, kappa = (6, 6, 4, 8), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 7)
    b = inputs.gaussian_source((V, 4, 3), 8)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(kappa)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    m = qcd.BICGSTAB if method == "bicgstab" else qcd.CG_NORMAL
    info, _ = qcd.solve(g, f, to_dev(b), x, method=m, tol=1e-10, inner="f16", dagger=dagger, use_graph=True,
                        graph_chunk=8)
    assert info[0]["converged"], info
    assert oracle_resid_wilson(L, kappa, U, b, x.cpu().numpy(), dagger=dagger) <= 1e-10
    assert info[0]["outer_updates"] >= 2


def test_wilson_dagger_solve_and_warm_start():
    device()
    L, kappa = (4, 4, 6, 8), 0.12
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 5)
    b = inputs.gaussian_source((V, 4, 3), 6)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(kappa)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, tol=1e-11, inner="f32", dagger=True)
    assert oracle_resid_wilson(L, kappa, U, b, x.cpu().numpy(), dagger=True) <= 1e-11
    # warm start from the converged solution: no inner iterations are needed
    info2, _ = qcd.solve(g, f, to_dev(b), x, tol=1e-10, inner="f32", dagger=True, x0_given=True)
    assert info2[0]["iters"] == 0 and info2[0]["converged"]


def test_wilson_multi_rhs_point_sources():
    """The 12 spin-colour point sources at one site, solved together (per-rhs scalars)."""
    device()
    L, kappa = (4, 4, 4, 8), 0.124
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 4)
    x0, b = inputs.point_sources(L, 0)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(kappa)
    x = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, nrhs=12, tol=1e-10, inner="f32", use_graph=True, graph_chunk=8)
    xr = x.cpu().numpy()
    for k in range(12):
        assert info[k]["converged"]
        assert oracle_resid_wilson(L, kappa, U, b[k], xr[k]) <= 1e-10


def test_solver_reports_noconv_with_best_iterate():
    device()
    L, kappa = (4, 4, 4, 8), 0.124
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 8)
    b = inputs.gaussian_source((V, 4, 3), 9)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(kappa)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info, st = qcd.solve(g, f, to_dev(b), x, tol=1e-12, maxiter=3, inner="f32", check=False)
    assert st == qcd.ERR_NOCONV
    assert not info[0]["converged"] and info[0]["iters"] <= 3
    r = oracle_resid_wilson(L, kappa, U, b, x.cpu().numpy())
    assert r < 1.0 and abs(r - info[0]["true_resid"]) < 1e-6 * max(r, 1e-30)


def test_full_size_12rhs_hop_on_sampled_sites():
    """Batched benchmark lattice (24^3 x 48, eps = 0.2 links seed 4, the 12 point sources plus
    Gaussian noise so that every output is nonzero): the FP32 12-rhs D_eo in the benchmark's
    INTERNAL-layout launch, checked on sampled outputs of every right-hand side."""
    device()
    L = (24, 24, 24, 48)
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 4)
    psi = inputs.gaussian_source((12, V, 4, 3), 5)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(0.124)
    nb = qcd.field_bytes(g, f, "f32", 12)
    bi = torch.empty(nb, dtype=torch.uint8, device=device())
    bo = torch.empty(nb, dtype=torch.uint8, device=device())
    qcd.field_pack(g, f, "f32", 1, to_dev(psi), bi, nrhs=12)
    qcd.dslash(g, f, "D_EO", bi, bo, prec="f32", nrhs=12, layout=qcd.INTERNAL)
    out = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.field_unpack(g, f, "f32", 0, bo, out, nrhs=12)
    torch.cuda.synchronize()
    par = ora.parity(L)
    even = np.flatnonzero(par == 0)
    sites = np.random.default_rng(6).choice(even, 96, replace=False)
    idx = torch.from_numpy(sites).to(device())
    from tests.gpu_util import rel_err
    for r in range(12):
        inp = psi[r].copy()
        inp[par == 0] = 0
        ref = ora.hop_sites(L, BC, U, inp, sites)
        assert rel_err(out[r][idx].cpu().numpy(), ref) < 1e-6
    g.free()
