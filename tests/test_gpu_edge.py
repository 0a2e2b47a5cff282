"""Edge cases and failure paths of the C ABI on the GPU: empty (zero) sources, limits on sizes,
degenerate parameters, NaN input, host buffers, and host-side allocation-fault injection."""
import os

import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, max_err, rel_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)


@pytest.fixture(scope="module")
def small():
    L = (4, 4, 4, 8)
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 91)
    return L, V, U


def test_zero_source_gives_zero_solution(small):
    device()
    L, V, U = small
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    b = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    x = torch.full_like(b, 7.0)
    info, st = qcd.solve(g, f, b, x, tol=1e-10, inner="f32")
    assert st == qcd.OK and info[0]["iters"] == 0 and info[0]["converged"]
    assert torch.count_nonzero(x).item() == 0


def test_tiny_kappa_is_almost_identity(small):
    device()
    L, V, U = small
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(1e-6)
    b = inputs.gaussian_source((V, 4, 3), 92)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, tol=1e-10, inner="f64")
    assert info[0]["iters"] <= 2
    r = np.linalg.norm(b - ora.wilson(L, BC, 1e-6, U, x.cpu().numpy())) / np.linalg.norm(b)
    assert r <= 1e-10


def test_host_buffers_match_device_buffers(small):
    device()
    L, V, U = small
    g = qcd.Gauge.load(U, L, BC)  # host gauge
    f = qcd.wilson(0.12)
    b = inputs.gaussian_source((V, 4, 3), 93)
    xh = np.zeros_like(b)
    qcd.solve(g, f, b, xh, tol=1e-11, inner="f32")
    xd = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    qcd.solve(g, f, to_dev(b), xd, tol=1e-11, inner="f32")
    assert np.array_equal(xh, xd.cpu().numpy())  # same arithmetic, bit for bit


def test_nan_source_is_reported_not_hung(small):
    device()
    L, V, U = small
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    b = inputs.gaussian_source((V, 4, 3), 94)
    b[5, 1, 2] = np.nan
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    info, st = qcd.solve(g, f, to_dev(b), x, tol=1e-10, inner="f32", check=False)
    assert st != qcd.OK and not info[0]["converged"]


def test_argument_limits(small):
    device()
    L, V, U = small
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    a = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    b = torch.zeros_like(a)
    with pytest.raises(qcd.QCDError) as e:
        qcd.dslash(g, f, "D_EO", a, b, nrhs=65)
    assert e.value.status == qcd.ERR_ARG
    with pytest.raises(qcd.QCDError) as e:
        qcd.dslash(g, f, 9, a, b)
    assert e.value.status == qcd.ERR_ARG
    with pytest.raises(qcd.QCDError) as e:
        qcd.dslash(g, qcd.dwf(1, 1.8, 0.02), "D_EO", a, b)
    assert e.value.status == qcd.ERR_ARG
    with pytest.raises(qcd.QCDError) as e:
        qcd.dslash(g, f, "D_EO", a, a)
    assert e.value.status == qcd.ERR_ARG
    with pytest.raises(qcd.QCDError) as e:
        qcd.solve(g, f, a, b, tol=-1.0)
    assert e.value.status == qcd.ERR_ARG
    with pytest.raises(qcd.QCDError) as e:
        qcd.dslash(g, f, "FULL", a, b, layout=qcd.INTERNAL)
    assert e.value.status == qcd.ERR_UNSUPPORTED


def test_many_rhs_in_one_launch(small):
    """nrhs = 64 (the maximum) through one stencil launch; spot-check the first and last."""
    device()
    L, V, U = small
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(0.12)
    psi = inputs.gaussian_source((64, V, 4, 3), 95)
    out = torch.empty_like(to_dev(psi))
    qcd.dslash(g, f, "D_EO", to_dev(psi), out, prec="f32", nrhs=64)
    torch.cuda.synchronize()
    par = ora.parity(L)
    for r in (0, 63):
        inp = psi[r].copy()
        inp[par == 0] = 0
        assert rel_err(out[r], ora.hop(L, BC, U, inp, out_parity=0)) < 1e-6


def test_domain_wall_ls2(small):
    device()
    L, V, U = small
    Ls = 2
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.dwf(Ls, 1.8, 0.02)
    psi = inputs.gaussian_source((Ls, V, 4, 3), 96)
    out = torch.empty_like(to_dev(psi))
    qcd.dslash(g, f, "FULL", to_dev(psi), out, prec="f64")
    torch.cuda.synchronize()
    assert max_err(out, ora.dw(L, BC, Ls, 1.8, 0.02, U, psi)) < 1e-13


def test_allocation_fault_injection_on_the_host(small):
    """QCD_FAULT=alloc makes every workspace allocation fail: the call returns ERR_OOM cleanly."""
    device()
    L, V, U = small
    os.environ["QCD_FAULT"] = "alloc"
    try:
        with pytest.raises(qcd.QCDError) as e:
            qcd.Gauge.load(to_dev(U), L, BC)
        assert e.value.status == qcd.ERR_OOM
    finally:
        del os.environ["QCD_FAULT"]
    g = qcd.Gauge.load(to_dev(U), L, BC)  # and the library still works afterwards
    g.free()


@pytest.mark.parametrize("fault,status", [("nan", "ERR_NAN"), ("noconv", "ERR_NOCONV")])
@pytest.mark.parametrize("inner", ["f32", "f16"])
def test_solver_fault_injection_on_the_host(small, fault, status, inner):
    """QCD_FAULT=nan poisons the inner residual (the device reductions must flag it); QCD_FAULT=noconv
    caps the iterations: the solve returns the matching status, and the next solve is clean."""
    device()
    L, V, U = small
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    b = to_dev(inputs.gaussian_source((V, 4, 3), 3))
    x = torch.zeros_like(b)
    os.environ["QCD_FAULT"] = fault
    try:
        info, st = qcd.solve(g, f, b, x, tol=1e-10, inner=inner, use_graph=True, check=False)
    finally:
        del os.environ["QCD_FAULT"]
    assert qcd.STATUS_NAMES[st] == status, (st, info)
    assert not info[0]["converged"]
    x.zero_()
    info, st = qcd.solve(g, f, b, x, tol=1e-10, inner=inner, use_graph=True)
    assert st == qcd.OK and info[0]["converged"]


_PDL_CHILD = r"""
import sys
import numpy as np, torch
from paper_1712_01505_gb300 import inputs, qcd
L, BC = (8, 4, 4, 8), (1, 1, 1, -1)
V = int(np.prod(L))
U = torch.from_numpy(inputs.gauge_field(L, 0.3, 41)).cuda()
b = torch.from_numpy(inputs.gaussian_source((V, 4, 3), 42)).cuda()
g = qcd.Gauge.load(U, L, BC, recon=12)
f = qcd.wilson(0.12)
o = torch.empty_like(b)
qcd.dslash(g, f, "MHAT", b, o, prec="f32")
x = torch.zeros_like(b)
qcd.solve(g, f, b, x, method=qcd.BICGSTAB, tol=1e-10, inner="f32", outer="df64", use_graph=True, graph_chunk=8)
Ls = 8
bd = torch.from_numpy(inputs.gaussian_source((Ls, V, 4, 3), 43)).cuda()
fd = qcd.mobius(Ls, 1.8, 0.02, 1.5, 0.5)
xd = torch.zeros_like(bd)
qcd.solve(g, fd, bd, xd, method=qcd.CG_NORMAL, tol=1e-10, inner="f32", use_graph=True, graph_chunk=8)
torch.cuda.synchronize()
np.save(sys.argv[1], np.concatenate([o.cpu().numpy().ravel(), x.cpu().numpy().ravel(), xd.cpu().numpy().ravel()]))
"""


def test_programmatic_launch_does_not_change_results(tmp_path):
    """QCD_PDL=0 (plain stream order) and the default (programmatic dependent launch) give the
    same bits for an operator, a Wilson BiCGStab and a Mobius CG solve (both runs share one
    tuning cache, so they run the same launch shapes)."""
    device()
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, QCD_TUNECACHE=str(tmp_path / "tune.txt"),
               PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    outs = []
    for pdl in ("0", "1"):
        out = tmp_path / f"pdl{pdl}.npy"
        r = subprocess.run([sys.executable, "-c", _PDL_CHILD, str(out)], cwd=root, env=dict(env, QCD_PDL=pdl),
                           capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1])
