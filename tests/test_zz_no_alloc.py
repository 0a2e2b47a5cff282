"""qcd_mhat_noalloc: the allocation-free Wilson Schur operator, for callers that cannot let the
library call cudaMalloc (their own allocator already owns the device memory, or the device-wide
synchronisation that cudaMalloc/cudaFree implies is unacceptable where they call us).

It must give what qcd_dslash(QCD_OP_MHAT[_DAG], QCD_LAYOUT_INTERNAL) gives, on two calls in a
row (the shared scratch array keeps the previous call's contents), agree with the FP64 oracle's
Mhat, leave the device's free memory unchanged, and refuse sizes beyond its fixed scratch and
overlapping buffers.  Kept in a file collected last so that a failure here stops a `-x` run
only after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as ora
from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, max_err, rel_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
# against qcd_dslash (same kernels, same order: equal up to the launch shape) and against the
# oracle (FP64 element-wise, FP32 1e-6 and FP16 2e-3 norm-wise, double-float 1e-12)
TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3, "df64": 1e-12}


def _unpack(g, f, prec, buf, V, nrhs):
    out = torch.zeros((nrhs, V, 4, 3), dtype=torch.complex128, device=device())
    qcd.field_unpack(g, f, prec, 0, buf, out, nrhs=nrhs)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _close(got, want, prec):
    return (max_err(got, want) if prec in ("f64", "df64") else rel_err(got, want)) < TOL[prec]


def _call(lib, g, f, prec, dagger, src, out, nrhs, stream):
    return lib.qcd_mhat_noalloc(g.handle, ctypes.byref(f), qcd.PREC[prec], dagger, ctypes.c_void_p(src),
                                ctypes.c_void_p(out), nrhs, stream)


@pytest.mark.parametrize("nrhs", [1, 4])
@pytest.mark.parametrize("prec", ["f64", "f32", "f16", "df64"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_noalloc_matches_dslash_and_oracle_on_two_calls(prec, dagger, nrhs):
    device()
    L, kappa = (8, 4, 6, 10), 0.124
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 21)
    psi = inputs.gaussian_source((nrhs, V, 4, 3), 22)
    par = ora.parity(L)
    psi[:, par == 1] = 0  # Mhat acts on the even sites
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(kappa)
    lib = qcd.load_library()
    nb = qcd.field_bytes(g, f, prec, nrhs)
    src = torch.empty(nb, dtype=torch.uint8, device=device())
    ref = torch.empty(nb, dtype=torch.uint8, device=device())
    outs = [torch.empty(nb, dtype=torch.uint8, device=device()) for _ in range(2)]
    qcd.field_pack(g, f, prec, 0, to_dev(psi), src, nrhs=nrhs)
    qcd.dslash(g, f, "MHAT_DAG" if dagger else "MHAT", src, ref, prec=prec, nrhs=nrhs, layout=qcd.INTERNAL)
    want = _unpack(g, f, prec, ref, V, nrhs)
    oracle = np.stack([ora.wilson_mhat(L, BC, kappa, U, psi[r], dagger=bool(dagger))[par == 0] for r in range(nrhs)])
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k, out in enumerate(outs):
        out.fill_(0xFF)  # poison the output
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = _call(lib, g, f, prec, dagger, src.data_ptr(), out.data_ptr(), nrhs, stream)
        assert st == qcd.OK, lib.qcd_last_error().decode()
        torch.cuda.synchronize()
        if k > 0:  # the first call on a device may load the module; later ones allocate nothing
            assert torch.cuda.mem_get_info()[0] == free0
        got = _unpack(g, f, prec, out, V, nrhs)
        assert _close(got, want, prec)
        assert _close(got[:, par == 0], oracle, prec)
    g.free()


def test_noalloc_refuses_sizes_beyond_its_scratch():
    device()
    L = (16, 16, 16, 16)
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.2, 23)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    nrhs = 8  # 32768 sites x 8 rhs x 192 B = 50 MB of intermediate > 32 MiB
    nb = qcd.field_bytes(g, f, "f64", nrhs)
    assert (V // 2) * nrhs * 192 > qcd.NOALLOC_SCRATCH_BYTES
    a = torch.zeros(nb, dtype=torch.uint8, device=device())
    b = torch.zeros(nb, dtype=torch.uint8, device=device())
    lib = qcd.load_library()
    assert _call(lib, g, f, "f64", 0, a.data_ptr(), b.data_ptr(), nrhs, None) == qcd.ERR_ARG
    assert "scratch" in lib.qcd_last_error().decode()
    g.free()


def test_noalloc_refuses_overlapping_buffers():
    device()
    L = (4, 4, 4, 4)
    U = inputs.gauge_field(L, 0.2, 24)
    g = qcd.Gauge.load(to_dev(U), L, BC)
    f = qcd.wilson(0.12)
    nb = qcd.field_bytes(g, f, "f32")
    a = torch.zeros(2 * nb, dtype=torch.uint8, device=device())
    lib = qcd.load_library()
    for shift in (16, nb - 16):  # out starts inside in
        assert _call(lib, g, f, "f32", 0, a.data_ptr(), a.data_ptr() + shift, 1, None) == qcd.ERR_ARG
        assert "overlap" in lib.qcd_last_error().decode()
    assert _call(lib, g, f, "f32", 0, a.data_ptr(), a.data_ptr() + nb, 1, None) == qcd.OK  # adjacent is fine
    torch.cuda.synchronize()
    g.free()
