"""qcd_mhat_noalloc: the allocation-free Wilson Schur operator for callers that cannot let
the library call cudaMalloc (their allocator owns the device memory, or a device-wide
synchronisation from cudaMalloc/cudaFree is unacceptable where they call us).

It must give what qcd_dslash(QCD_OP_MHAT[_DAG], QCD_LAYOUT_INTERNAL) gives, on two calls in a
row (the shared scratch array keeps the previous call's contents), and refuse sizes beyond its
fixed scratch.  Kept in a file collected last so that a failure here stops a `-x` run only
after every other test has run.
"""
import ctypes

import numpy as np
import pytest

from paper_1712_01505_gb300 import inputs, qcd
from tests.gpu_util import device, max_err, rel_err, to_dev, torch

pytestmark = pytest.mark.gpu

BC = (1, 1, 1, -1)
TOL = {"f64": 1e-13, "f32": 1e-6, "f16": 2e-3}


def _unpack(g, f, prec, buf, V):
    out = torch.zeros((V, 4, 3), dtype=torch.complex128, device=device())
    qcd.field_unpack(g, f, prec, 0, buf, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("prec", ["f64", "f32", "f16"])
@pytest.mark.parametrize("dagger", [0, 1])
def test_noalloc_matches_dslash_on_two_calls(prec, dagger):
    device()
    L = (8, 4, 6, 10)
    V = int(np.prod(L))
    U = inputs.gauge_field(L, 0.3, 21)
    psi = inputs.gaussian_source((V, 4, 3), 22)
    g = qcd.Gauge.load(to_dev(U), L, BC, recon=12)
    f = qcd.wilson(0.124)
    lib = qcd.load_library()
    nb = qcd.field_bytes(g, f, prec)
    src = torch.empty(nb, dtype=torch.uint8, device=device())
    ref = torch.empty(nb, dtype=torch.uint8, device=device())
    qcd.field_pack(g, f, prec, 0, to_dev(psi), src)
    qcd.dslash(g, f, "MHAT_DAG" if dagger else "MHAT", src, ref, prec=prec, layout=qcd.INTERNAL)
    want = _unpack(g, f, prec, ref, V)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out = torch.full((nb,), 0xFF, dtype=torch.uint8, device=device())  # poison the output
        st = lib.qcd_mhat_noalloc(g.handle, ctypes.byref(f), qcd.PREC[prec], dagger,
                                  ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(out.data_ptr()), 1, stream)
        assert st == qcd.OK, lib.qcd_last_error().decode()
        got = _unpack(g, f, prec, out, V)
        if prec == "f64":
            assert max_err(got, want) < TOL[prec]
        else:
            assert rel_err(got, want) < TOL[prec]
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
    st = lib.qcd_mhat_noalloc(g.handle, ctypes.byref(f), qcd.F64, 0, ctypes.c_void_p(a.data_ptr()),
                              ctypes.c_void_p(b.data_ptr()), nrhs, None)
    assert st == qcd.ERR_ARG
    assert "scratch" in lib.qcd_last_error().decode()
    g.free()
