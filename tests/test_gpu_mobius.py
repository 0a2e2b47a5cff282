"""GPU parity of the Mobius domain-wall operator D = A - 1/2 H B and its CG solve against the
FP64 oracle.

The library's even-odd operator is that of D B^-1 (x' = B x): Mhat = 1 - 1/4 W H_eo W H_oe with
W = B A^-1 applied by one site-local kernel.  Tolerances as for Shamir (FP64 1e-13 element-wise,
FP32 1e-6 and FP16 2e-3 norm-wise, double-float 1e-12 element-wise); solves to
|b - D x| / |b| <= 1e-10 by the oracle's D.
"""
import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, max_err, rel_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
M5, MF = 1.8, 0.02
B5, C5 = 1.5, 0.5  # b5 - c5 = 1: the Shamir kernel scaled by b5 + c5 = 2
TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3}
DF_TOL = 1e-12


def _check(out, ref, prec):
    if prec in ("f64", "df64"):
        assert max_err(out, ref) < (TOL["f64"] if prec == "f64" else DF_TOL)
    else:
        assert rel_err(out, ref) < TOL[prec]


def _case(L, Ls, seed, nrhs=1):
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, seed)
    shape = (nrhs, Ls, V, 4, 3) if nrhs > 1 else (Ls, V, 4, 3)
    return V, U, inputs.gaussian_source(shape, seed + 1)


@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dag", [False, True])
@pytest.mark.parametrize("b5,c5", [(B5, C5), (2.0, 0.0), (1.2, 0.9)])
def test_mobius_mhat_and_full(prec, dag, b5, c5):
    device()
    L, Ls = (4, 4, 4, 8), 8
    V, U, psi = _case(L, Ls, 81)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=18)
    f = qcd.mobius(Ls, M5, MF, b5, c5)
    par = ora.parity(L)
    pe = psi.copy()
    pe[:, par == 1] = 0
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", to_dev(psi), out, prec=prec)
    torch.cuda.synchronize()
    _check(out, ora.mobius_mhat(L, BC, Ls, M5, MF, b5, c5, U, pe, dagger=dag), prec)
    if prec == "df64":
        return
    qcd.dslash(g, f, "FULL_DAG" if dag else "FULL", to_dev(psi), out, prec=prec)
    torch.cuda.synchronize()
    _check(out, ora.mobius(L, BC, Ls, M5, MF, b5, c5, U, psi, dagger=dag), prec)


@pytest.mark.parametrize("op", ["MHAT", "MHAT_DAG", "FULL", "FULL_DAG"])
def test_b5_1_c5_0_runs_the_shamir_kernels(op):
    """qcd.mobius(b5 = 1, c5 = 0) is Eq. (2): the same launches, bit for bit."""
    device()
    L, Ls = (4, 4, 2, 6), 6
    V, U, psi = _case(L, Ls, 83)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    a = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    b = torch.empty_like(a)
    qcd.dslash(g, qcd.mobius(Ls, M5, MF, 1.0, 0.0), op, to_dev(psi), a, prec="f32")
    qcd.dslash(g, qcd.dwf(Ls, M5, MF), op, to_dev(psi), b, prec="f32")
    torch.cuda.synchronize()
    assert torch.equal(a, b)


@pytest.mark.parametrize("Ls", [5, 16])
def test_mobius_double_float_mhat_ragged(Ls):
    """Odd Ls and a lattice whose half volume is not a multiple of the kernel's site tile."""
    device()
    L = (6, 4, 2, 10)
    V, U, psi = _case(L, Ls, 85)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.mobius(Ls, M5, MF, B5, C5)
    par = ora.parity(L)
    pe = psi.copy()
    pe[:, par == 1] = 0
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    for dag in (False, True):
        qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", to_dev(psi), out, prec="df64")
        torch.cuda.synchronize()
        assert max_err(out, ora.mobius_mhat(L, BC, Ls, M5, MF, B5, C5, U, pe, dagger=dag)) < DF_TOL


def test_mobius_multi_rhs_full():
    device()
    L, Ls, nrhs = (4, 4, 2, 6), 6, 3
    V, U, psi = _case(L, Ls, 87, nrhs=nrhs)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.mobius(Ls, M5, MF, B5, C5)
    out = torch.empty(psi.shape, dtype=torch.complex128, device=device())
    qcd.dslash(g, f, "FULL", to_dev(psi), out, prec="f32", nrhs=nrhs)
    torch.cuda.synchronize()
    for r in range(nrhs):
        assert rel_err(out[r], ora.mobius(L, BC, Ls, M5, MF, B5, C5, U, psi[r])) < 1e-6


@pytest.mark.parametrize("inner,outer", [("f64", "f64"), ("f32", "f64"), ("f32", "df64"), ("f16", "df64")])
def test_mobius_cg_solve(inner, outer):
    device()
    L, Ls = (4, 4, 4, 8), 8
    V, U, b = _case(L, Ls, 89)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.mobius(Ls, M5, MF, B5, C5)
    x = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, method=qcd.CG_NORMAL, tol=1e-10, inner=inner, outer=outer,
                        use_graph=True, graph_chunk=16)
    assert info[0]["converged"], info
    xr = x.cpu().numpy()
    res = np.linalg.norm(b - ora.mobius(L, BC, Ls, M5, MF, B5, C5, U, xr)) / np.linalg.norm(b)
    assert res <= 1e-10
    assert abs(res - info[0]["true_resid"]) <= 1e-6 * res + 1e-14


def test_mobius_solve_from_an_initial_guess_and_two_rhs():
    device()
    L, Ls, nrhs = (4, 4, 2, 8), 6, 2
    V, U, b = _case(L, Ls, 91, nrhs=nrhs)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.mobius(Ls, M5, MF, B5, C5)
    x = torch.zeros(b.shape, dtype=torch.complex128, device=device())
    info, _ = qcd.solve(g, f, to_dev(b), x, nrhs=nrhs, method=qcd.CG_NORMAL, tol=1e-10, inner="f32")
    xr = x.cpu().numpy()
    for r in range(nrhs):
        assert info[r]["converged"], info
        res = np.linalg.norm(b[r] - ora.mobius(L, BC, Ls, M5, MF, B5, C5, U, xr[r])) / np.linalg.norm(b[r])
        assert res <= 1e-10
    # restart from the solution with a perturbation: few iterations, same answer
    x0 = xr + 1e-6 * inputs.gaussian_source(b.shape, 92)
    x = to_dev(x0)
    info2, _ = qcd.solve(g, f, to_dev(b), x, nrhs=nrhs, method=qcd.CG_NORMAL, tol=1e-10, inner="f32",
                         x0_given=True)
    for r in range(nrhs):
        assert info2[r]["converged"] and info2[r]["iters"] < info[r]["iters"], (info, info2)
    assert rel_err(x, xr) < 1e-6  # both solutions have residual 1e-10; D has condition number < 1e4


@pytest.mark.parametrize("b5,c5,M5_", [(0.0, 0.5, M5), (1.5, 0.5, 4.0 + 1.0 / 1.5 + 1e-16)])
def test_mobius_rejects_singular_blocks(b5, c5, M5_):
    """The fifth-dimension blocks are inverted in closed form, which needs nonzero diagonals:
    b5 = 0 (B = c5 S) and alpha = (4 - M5) b5 + 1 = 0 are refused before any launch."""
    device()
    L, Ls = (4, 4, 4, 4), 4
    V, U, psi = _case(L, Ls, 93)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    with pytest.raises(qcd.QCDError, match="ERR_ARG"):
        qcd.dslash(g, qcd.mobius(Ls, M5_, MF, b5, c5), "MHAT", to_dev(psi), out, prec="f32")


@pytest.mark.parametrize("Ls", [32, 36])
@pytest.mark.parametrize("mobius", [False, True])
def test_mhat_at_the_fused_limit_and_beyond(Ls, mobius):
    """Ls <= 32 runs the stencil with W in its epilogue (one launch per hop), larger Ls the hop and
    the column kernel as two launches: both against the oracle, FP32 and FP16, both adjoints."""
    device()
    L = (2, 2, 2, 4)
    V, U, psi = _case(L, Ls, 95)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    b5, c5 = (B5, C5) if mobius else (1.0, 0.0)
    f = qcd.mobius(Ls, M5, MF, b5, c5)
    par = ora.parity(L)
    pe = psi.copy()
    pe[:, par == 1] = 0
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    for prec in ("f32", "f16"):
        for dag in (False, True):
            qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", to_dev(psi), out, prec=prec)
            torch.cuda.synchronize()
            _check(out, ora.mobius_mhat(L, BC, Ls, M5, MF, b5, c5, U, pe, dagger=dag), prec)


def _neighbours(L, sites):
    """Canonical indices of the 8 neighbours (x +- mu) of each canonical site; shape (n, 8)."""
    Lx, Ly, Lz, Lt = L
    x = sites % Lx
    y = (sites // Lx) % Ly
    z = (sites // (Lx * Ly)) % Lz
    t = sites // (Lx * Ly * Lz)
    c = [x, y, z, t]
    out = []
    for mu in range(4):
        for d in (1, -1):
            cc = list(c)
            cc[mu] = (cc[mu] + d) % L[mu]
            out.append(cc[0] + Lx * (cc[1] + Ly * (cc[2] + Lz * cc[3])))
    return np.stack(out, axis=1)


def _mhat_sampled(L, Ls, b5, c5, U, psi, xs, dagger):
    """(Mhat psi_e)(x) at even sites xs for all slices, from the oracle's site-restricted hop and
    the dense fifth-dimension blocks: Mhat = 1 - 1/4 W H_eo W H_oe (adjoint: with W^T and H^dag,
    W^T applied first)."""
    V = int(np.prod(L))
    par = ora.parity(L)
    pe = psi.copy()
    pe[:, par == 1] = 0
    if dagger:
        pe = ora.mobius_block(Ls, M5, MF, b5, c5, "W", pe, dagger=True)
        pe[:, par == 1] = 0
    ys = np.unique(_neighbours(L, xs).reshape(-1))  # odd neighbours of the sampled even sites
    t1 = np.stack([ora.hop_sites(L, BC, U, pe[s], ys, dagger=dagger) for s in range(Ls)])
    if not dagger:
        t1 = ora.mobius_block(Ls, M5, MF, b5, c5, "W", t1)
    else:
        t1 = ora.mobius_block(Ls, M5, MF, b5, c5, "W", t1, dagger=True)
    u = np.empty((Ls, len(xs), 4, 3), dtype=complex)
    for s in range(Ls):
        full = np.zeros((V, 4, 3), dtype=complex)
        full[ys] = t1[s]
        u[s] = ora.hop_sites(L, BC, U, full, xs, dagger=dagger)
    if not dagger:
        u = ora.mobius_block(Ls, M5, MF, b5, c5, "W", u)
    return psi[:, xs] - 0.25 * u


@pytest.mark.parametrize("mobius", [False, True])
@pytest.mark.parametrize("prec", ["f32", "f16"])
def test_full_size_fused_mhat_on_sampled_sites(mobius, prec):
    """Domain-wall benchmark lattice (16^3 x 32, Ls = 16, eps = 0.2 links seed 3, Gaussian source
    seed 0): Mhat and Mhat^dag in the benchmark's INTERNAL-layout launches (the hop with W in its
    epilogue, tuner-chosen shape), checked on sampled even sites the oracle computes one by one."""
    device()
    L, Ls = (16, 16, 16, 32), 16
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 3)
    psi = inputs.gaussian_source((Ls, V, 4, 3), 0)
    even = np.flatnonzero(ora.parity(L) == 0)
    rng = np.random.default_rng(17)
    xs = np.concatenate([even[:8], even[-8:], rng.choice(even, 32, replace=False)])
    b5, c5 = (B5, C5) if mobius else (1.0, 0.0)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.mobius(Ls, M5, MF, b5, c5)
    nb = qcd.field_bytes(g, f, prec)
    bi = torch.empty(nb, dtype=torch.uint8, device=device())
    bo = torch.empty(nb, dtype=torch.uint8, device=device())
    qcd.field_pack(g, f, prec, 0, to_dev(psi), bi)
    out = torch.zeros((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    idx = torch.from_numpy(xs).to(device())
    for dag in (False, True):
        qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", bi, bo, prec=prec, layout=qcd.INTERNAL)
        qcd.field_unpack(g, f, prec, 0, bo, out)
        torch.cuda.synchronize()
        ref = _mhat_sampled(L, Ls, b5, c5, U, psi, xs, dag)
        assert rel_err(out[:, idx].cpu().numpy(), ref) < TOL[prec], (dag, prec)
    g.free()


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_mhat_at_the_largest_ls(prec):
    """Ls = 64, the library's limit: the column kernels stage 8 sites per block (the staging
    tile of 64 slices x 24 reals fills the shared memory), in every precision of the operator."""
    device()
    L, Ls = (2, 2, 2, 4), 64
    V, U, psi = _case(L, Ls, 97)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    par = ora.parity(L)
    pe = psi.copy()
    pe[:, par == 1] = 0
    out = torch.empty((Ls, V, 4, 3), dtype=torch.complex128, device=device())
    for b5, c5 in ((1.0, 0.0), (B5, C5)):
        f = qcd.mobius(Ls, M5, MF, b5, c5)
        for dag in (False, True):
            qcd.dslash(g, f, "MHAT_DAG" if dag else "MHAT", to_dev(psi), out, prec=prec)
            torch.cuda.synchronize()
            _check(out, ora.mobius_mhat(L, BC, Ls, M5, MF, b5, c5, U, pe, dagger=dag), prec)
    with pytest.raises(qcd.QCDError, match="ERR_ARG"):
        qcd.dslash(g, qcd.mobius(65, M5, MF, B5, C5), "MHAT", to_dev(inputs.gaussian_source((65, V, 4, 3), 98)),
                   torch.empty((65, V, 4, 3), dtype=torch.complex128, device=device()), prec="f32")
