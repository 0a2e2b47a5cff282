"""Double-float (FP32 pair) operators and outer solver steps against the FP64 oracle.

Tolerances.  Storage: hi = fl32(x), lo = fl32(x - hi) represents x to within
2^-48 |x| (hi carries 24 bits, lo rounds the exact remainder to 24 more) for
2^-100 < |x| < 2^100.  Operator: every output real is a sum of at most
8 x (2 + 6) terms; TwoSum / TwoProd are exact and only the FP32 low-part
additions round, so the error is below n u^2 sum|terms| with u = 2^-24 and
n <~ 100 operations on the low part, i.e. < 1e-12 of the largest output
for unitary links (|U_ab| <= 1); the element-wise tests use that bound.
Solves: full-system residual <= 1e-10 with the oracle's operator."""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, max_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
DF_TOL = 1e-12


def _case(L, seed=3, eps=0.4):
    V = int(np.prod(L))
    return V, inputs.gauge_field(L, eps, seed), inputs.gaussian_source((V, 4, 3), seed + 100)


def test_pack_unpack_roundtrip_within_2_pow_48():
    device()
    L = (6, 4, 6, 10)
    V, U, psi = _case(L, seed=9)
    # magnitudes spread over 2^-80 .. 2^80
    scale = np.exp2(np.random.default_rng(1).integers(-80, 81, size=psi.shape))
    psi = psi * scale
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.1)
    buf = torch.empty(qcd.field_bytes(g, f, "df64"), dtype=torch.uint8, device=device())
    back = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    for parity in (0, 1):
        qcd.field_pack(g, f, "df64", parity, to_dev(psi), buf)
        qcd.field_unpack(g, f, "df64", parity, buf, back)
    torch.cuda.synchronize()
    b = back.cpu().numpy()
    # split error <= 2^-48 |x|, plus the rounding of the FP64 sum hi + lo on unpack
    for part in (np.real, np.imag):
        assert np.all(np.abs(part(b) - part(psi)) <= 2.0 ** -47 * np.abs(part(psi)))
    # exactly representable values survive unchanged
    exact = np.round(psi.real / scale) * scale + 0j
    qcd.field_pack(g, f, "df64", 0, to_dev(exact), buf)
    back.zero_()
    qcd.field_unpack(g, f, "df64", 0, buf, back)
    par = ora.parity(L)
    assert np.array_equal(back.cpu().numpy()[par == 0], exact[par == 0])


def test_split_edge_values():
    """Values at the edges of the split: a mantissa of all ones (the rounding carries into the
    exponent), powers of two, FP32-exact values, zeros, and magnitudes outside 2^-100 .. 2^100
    (the FP64 conversion path), each within 2^-47 of its value after a pack / unpack."""
    device()
    L = (2, 2, 2, 2)
    V = 16
    vals = [np.nextafter(2.0, 0.0), -np.nextafter(1.0, 0.0), 1.0, -0.5, 2.0 ** 99, 2.0 ** -99,
            np.nextafter(2.0 ** 100, 0.0), 1.0 + 2.0 ** -24, 1.0 + 2.0 ** -25, 1.0 - 2.0 ** -53, 0.0, -0.0,
            3.0e-35, -7.0e-40, 1.0e35, -2.0e31, 0.1, -1.0 / 3.0, np.pi, 2.0 ** -60 * np.e]
    vals = np.array(vals * ((V * 12 + len(vals) - 1) // len(vals)))[: V * 12]
    psi = (vals + 1j * vals[::-1]).reshape(V, 4, 3)
    U = inputs.gauge_field(L, 0.3, 1)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.1)
    buf = torch.empty(qcd.field_bytes(g, f, "df64"), dtype=torch.uint8, device=device())
    back = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    for parity in (0, 1):
        qcd.field_pack(g, f, "df64", parity, to_dev(psi), buf)
        qcd.field_unpack(g, f, "df64", parity, buf, back)
    torch.cuda.synchronize()
    b = back.cpu().numpy()
    for part in (np.real, np.imag):
        err = np.abs(part(b) - part(psi))
        big = np.abs(part(psi)) >= 1e-30  # below FP32's normal range the low part underflows
        assert np.all(err[big] <= 2.0 ** -47 * np.abs(part(psi))[big])
        assert np.all(err[~big] <= 1e-44)


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 6, 10), (2, 2, 2, 2)])
@pytest.mark.parametrize("op", ["D_EO", "D_OE"])
def test_hop_parity(L, op):
    device()
    V, U, psi = _case(L)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    out = torch.empty((V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, op, to_dev(psi), out, prec="df64")
    torch.cuda.synchronize()
    po = 0 if op == "D_EO" else 1
    par = ora.parity(L)
    inp = psi.copy()
    inp[par == po] = 0
    ref = ora.hop(L, BC, U, inp, out_parity=po)
    assert max_err(out, ref) < DF_TOL
    assert np.all(out.cpu().numpy()[par != po] == 0)


@pytest.mark.parametrize("dag", [False, True])
def test_mhat_and_full_parity(dag):
    device()
    L, kappa = (6, 4, 6, 10), 0.124
    V, U, psi = _case(L, seed=5)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(kappa)
    par = ora.parity(L)
    pe = psi.copy()
    pe[par == 1] = 0
    out = torch.empty((V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", to_dev(psi), out, prec="df64")
    torch.cuda.synchronize()
    assert max_err(out, ora.wilson_mhat(L, BC, kappa, U, pe, dagger=dag)) < DF_TOL
    qcd.dslash(g, f, "FULL_DAG" if dag else "FULL", to_dev(psi), out, prec="df64")
    torch.cuda.synchronize()
    assert max_err(out, ora.wilson(L, BC, kappa, U, psi, dagger=dag)) < DF_TOL


def test_multi_rhs():
    device()
    L, nrhs = (4, 4, 6, 6), 3
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.4, 7)
    psi = inputs.gaussian_source((nrhs, V, 4, 3), 17)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    out = torch.empty((nrhs, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "D_OE", to_dev(psi), out, prec="df64", nrhs=nrhs)
    torch.cuda.synchronize()
    par = ora.parity(L)
    for r in range(nrhs):
        inp = psi[r].copy()
        inp[par == 1] = 0
        assert max_err(out[r], ora.hop(L, BC, U, inp, out_parity=1)) < DF_TOL


def test_sampled_sites_at_32x32x32x64():
    """Benchmark lattice (32^3 x 64, eps = 0.2, Z2 source): INTERNAL-layout double-float D_EO on
    sampled output sites the oracle computes one by one."""
    device()
    L = (32, 32, 32, 64)
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 2)
    psi = inputs.z2_source((V, 4, 3), 0)
    par = ora.parity(L)
    rng = np.random.default_rng(5)
    even = np.flatnonzero(par == 0)
    sites = np.concatenate([even[:64], even[-64:], rng.choice(even, 512, replace=False)])
    inp = psi.copy()
    inp[par == 0] = 0
    ref = ora.hop_sites(L, BC, U, inp, sites)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(0.125)
    nb = qcd.field_bytes(g, f, "df64")
    bi = torch.empty(nb, dtype=torch.uint8, device=device())
    bo = torch.empty(nb, dtype=torch.uint8, device=device())
    qcd.field_pack(g, f, "df64", 1, to_dev(psi), bi)
    qcd.dslash(g, f, "D_EO", bi, bo, prec="df64", layout=qcd.INTERNAL)
    out = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    qcd.field_unpack(g, f, "df64", 0, bo, out)
    torch.cuda.synchronize()
    got = out[torch.from_numpy(sites).to(device())].cpu().numpy()
    assert max_err(got, ref) < DF_TOL
    g.free()


def _resid(L, kappa, U, b, x, dagger=False):
    return np.linalg.norm(b - ora.wilson(L, BC, kappa, U, x, dagger=dagger)) / np.linalg.norm(b)


@pytest.mark.parametrize("inner", ["f32", "f16"])
@pytest.mark.parametrize("method", [qcd.BICGSTAB, qcd.CG_NORMAL])
def test_solve_with_double_float_outer_steps(inner, method):
    device()
    L, kappa = (8, 8, 8, 8), 0.124
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 4)
    b = inputs.z2_source((V, 4, 3), 0)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(kappa)
    runs = {}
    for outer in ("f64", "df64"):
        x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
        info, _ = qcd.solve(g, f, to_dev(b), x, method=method, tol=1e-10, inner=inner, use_graph=True,
                            graph_chunk=16, outer=outer)
        r = _resid(L, kappa, U, b, x.cpu().numpy())
        assert info[0]["converged"] and r <= 1e-10, (outer, info)
        # the reported residual is the library's own IEEE-FP64 recomputation
        assert abs(r - info[0]["true_resid"]) <= 1e-6 * r
        runs[outer] = info[0]
    assert runs["df64"]["outer_updates"] >= 2
    assert abs(runs["df64"]["iters"] - runs["f64"]["iters"]) <= max(3, runs["f64"]["iters"] // 10)


def test_dagger_warm_start_and_point_sources():
    device()
    L, kappa = (4, 4, 4, 8), 0.124
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 4)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(kappa)
    b = inputs.gaussian_source((V, 4, 3), 6)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    qcd.solve(g, f, to_dev(b), x, tol=1e-11, inner="f32", dagger=True, outer="df64")
    assert _resid(L, kappa, U, b, x.cpu().numpy(), dagger=True) <= 1e-11
    info, _ = qcd.solve(g, f, to_dev(b), x, tol=1e-10, inner="f32", dagger=True, x0_given=True, outer="df64")
    assert info[0]["iters"] == 0 and info[0]["converged"]
    _, bs = inputs.point_sources(L, 0)
    xs = torch.zeros((12, V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(bs), xs, nrhs=12, tol=1e-10, inner="f32", use_graph=True, graph_chunk=8,
                        outer="df64")
    xr = xs.cpu().numpy()
    for k in range(12):
        assert info[k]["converged"] and _resid(L, kappa, U, bs[k], xr[k]) <= 1e-10


def test_argument_checks():
    device()
    L = (4, 4, 4, 4)
    V, U, psi = _case(L)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    x = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    with pytest.raises(qcd.QCDError, match="ERR_ARG"):
        qcd.solve(g, qcd.wilson(0.12), to_dev(psi), x, inner="df64")
    with pytest.raises(qcd.QCDError, match="ERR_ARG"):
        qcd.solve(g, qcd.wilson(0.12), to_dev(psi), x, inner="f32", outer="f32")
    d = qcd.dwf(4, 1.8, 0.1)
    xd = torch.zeros((4, V, 4, 3), dtype=torch.complex128, device=device())
    bd = to_dev(inputs.gaussian_source((4, V, 4, 3), 1))
    with pytest.raises(qcd.QCDError, match="ERR_UNSUPPORTED"):
        qcd.dslash(g, d, "FULL_DAG", bd, xd, prec="df64")
