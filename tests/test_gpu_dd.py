"""Domain decomposition on one GPU (Sec. IV D): several subdomains in one process, faces
exchanged by device copies while the interior is computed.  The decomposed operators are
checked against the oracle's operators on the whole lattice, and the decomposed BiCGStab against
the oracle's full-system residual."""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import dd, inputs, qcd
from tests.gpu_util import device, max_err, rel_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
GRIDS = [((4, 4, 4, 8), (1, 1, 1, 2)), ((8, 4, 4, 8), (2, 1, 1, 2)), ((4, 4, 4, 4), (2, 2, 2, 2)),
         ((8, 8, 4, 4), (4, 2, 1, 1)), ((4, 4, 4, 8), (1, 1, 1, 1))]  # the last: no cut at all


def _setup(L, P, seed, recon=18):
    U = inputs.gauge_field(L, 0.3, seed)
    ids = list(range(int(np.prod(P))))
    D = dd.Decomposition(L, P, BC, ids, [to_dev(dd.scatter_gauge(U, L, P, s)) for s in ids], recon=recon)
    return U, ids, D


@pytest.mark.parametrize("L,P", GRIDS)
@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 18), ("f32", 12)])
def test_decomposed_operators_match_the_oracle(L, P, prec, recon):
    device()
    U, ids, D = _setup(L, P, 31, recon)
    V = int(np.prod(L))
    psi = inputs.gaussian_source((V, 4, 3), 32)
    par = ora.parity(L)
    f = qcd.wilson(0.124)
    inp = [to_dev(dd.scatter_spinor(psi, L, P, s)) for s in ids]
    out = [torch.empty_like(t) for t in inp]
    for op in ("D_EO", "D_OE", "MHAT", "MHAT_DAG"):
        D.dslash(f, op, inp, out, prec=prec)
        torch.cuda.synchronize()
        got = dd.gather_spinor([t.cpu().numpy() for t in out], L, P, ids)
        if op in ("D_EO", "D_OE"):
            po = 0 if op == "D_EO" else 1
            src = psi.copy()
            src[par == po] = 0
            ref = ora.hop(L, BC, U, src, out_parity=po)
        else:
            src = psi.copy()
            src[par == 1] = 0
            ref = ora.wilson_mhat(L, BC, 0.124, U, src, dagger=op == "MHAT_DAG")
        if prec == "f64":
            assert max_err(got, ref) < 1e-13, op
        else:
            assert rel_err(got, ref) < 1e-6, op
    D.free()


def test_decomposed_mhat_equals_the_single_domain_operator():
    device()
    L, P = (8, 4, 4, 8), (2, 1, 1, 2)
    U, ids, D = _setup(L, P, 33)
    V = int(np.prod(L))
    psi = inputs.gaussian_source((V, 4, 3), 34)
    psi[ora.parity(L) == 1] = 0
    f = qcd.wilson(0.13)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    whole = torch.empty((V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "MHAT", to_dev(psi), whole, prec="f64")
    inp = [to_dev(dd.scatter_spinor(psi, L, P, s)) for s in ids]
    out = [torch.empty_like(t) for t in inp]
    D.dslash(f, "MHAT", inp, out, prec="f64")
    torch.cuda.synchronize()
    got = dd.gather_spinor([t.cpu().numpy() for t in out], L, P, ids)
    assert max_err(got, whole.cpu().numpy()) < 1e-14  # the same sums in another order
    g.free()
    D.free()


@pytest.mark.parametrize("L,P", [((8, 4, 4, 8), (2, 1, 1, 2)), ((4, 4, 4, 8), (1, 1, 1, 2))])
@pytest.mark.parametrize("inner", ["f64", "f32"])
def test_decomposed_bicgstab_reaches_1e10_on_the_full_system(L, P, inner):
    device()
    U, ids, D = _setup(L, P, 35)
    kappa = 0.124
    V = int(np.prod(L))
    b = inputs.gaussian_source((V, 4, 3), 36)
    bl = [to_dev(dd.scatter_spinor(b, L, P, s)) for s in ids]
    xl = [torch.zeros_like(t) for t in bl]
    info, _ = D.solve(qcd.wilson(kappa), bl, xl, tol=1e-10, inner=inner, delta=1e-3)
    x = dd.gather_spinor([t.cpu().numpy() for t in xl], L, P, ids)
    res = np.linalg.norm(b - ora.wilson(L, BC, kappa, U, x)) / np.linalg.norm(b)
    assert res <= 1e-10 and info["converged"], info
    assert abs(res - info["true_resid"]) <= 1e-3 * res
    if inner == "f32":
        assert info["outer_updates"] >= 2
    # the single-domain solve of the same system takes about as many iterations
    g = qcd.Gauge.load(to_dev(U), L, BC)
    x1 = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info1, _ = qcd.solve(g, qcd.wilson(kappa), to_dev(b), x1, tol=1e-10, inner=inner, delta=1e-3)
    assert abs(info["iters"] - info1[0]["iters"]) <= max(3, info1[0]["iters"] // 10)
    g.free()
    D.free()


def test_argument_checks():
    device()
    L, P = (4, 4, 4, 8), (1, 1, 1, 2)
    U = inputs.gauge_field(L, 0.3, 37)
    Ul = [to_dev(dd.scatter_gauge(U, L, P, s)) for s in (0, 1)]
    with pytest.raises(qcd.QCDError):
        dd.Decomposition(L, P, BC, [0, 0], Ul)  # repeated id
    with pytest.raises(qcd.QCDError):
        dd.Decomposition(L, P, BC, [0, 2], Ul)  # out of range
    # one of two subdomains without a transport to the other: the operator refuses to run
    D = dd.Decomposition(L, P, BC, [0], Ul[:1])
    psi = to_dev(inputs.gaussian_source((int(np.prod(L)) // 2, 4, 3), 38))
    out = torch.empty_like(psi)
    with pytest.raises(qcd.QCDError, match="NCCL"):
        D.dslash(qcd.wilson(0.12), "D_EO", [psi], [out])
    torch.cuda.synchronize()
    D.free()


def test_zero_source_gives_zero_solution():
    device()
    L, P = (4, 4, 4, 8), (1, 1, 1, 2)
    _, ids, D = _setup(L, P, 39)
    bl = [torch.zeros((int(np.prod(L)) // 2, 4, 3), dtype=torch.complex128, device=device()) for _ in ids]
    xl = [torch.full_like(t, 1.0) for t in bl]
    info, st = D.solve(qcd.wilson(0.12), bl, xl, tol=1e-10, inner="f32")
    assert st == qcd.OK and info["converged"] and info["true_resid"] == 0.0
    assert all(float(t.abs().max()) == 0.0 for t in xl)
    D.free()
