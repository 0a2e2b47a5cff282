"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every
symbol include/qcd.h declares, the binding mirrors the header's structs, and the
host-side argument validation works without touching a device."""
import ctypes
import os
import re

import pytest

from paper_1712_01505_gb300 import qcd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qcd.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1712_01505_gb300 import build

    build.build()
    return qcd.load_library()


def header_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:qcd_status|size_t|int32_t|const char\*)\s+(qcd_\w+)\s*\(", src, re.M)))


def test_header_declares_the_binding_symbols():
    assert header_functions() == sorted(qcd.SYMBOLS)


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_struct_layouts_match_header():
    # field order and C types of the ABI structs (offsets as a C compiler lays them out)
    assert ctypes.sizeof(qcd.Geom) == 36
    assert qcd.Fermion.kappa.offset == 8 and qcd.Fermion.Ls.offset == 16 and qcd.Fermion.mf.offset == 32
    assert qcd.Fermion.c5.offset == 48 and ctypes.sizeof(qcd.Fermion) == 56
    assert qcd.SolverParams.tol.offset == 8 and qcd.SolverParams.delta.offset == 24
    assert qcd.SolverParams.outer.offset == 48 and ctypes.sizeof(qcd.SolverParams) == 56
    assert ctypes.sizeof(qcd.SolveInfo) == 32


def test_struct_layouts_match_a_c_compiler(tmp_path):
    """Every field offset and struct size of the binding equals what gcc makes of include/qcd.h."""
    import shutil
    import subprocess

    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    structs = {"qcd_geom": qcd.Geom, "qcd_fermion": qcd.Fermion, "qcd_solver_params": qcd.SolverParams,
               "qcd_solve_info": qcd.SolveInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "qcd.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append(f'  printf("enum QCD_DF64 %d\\n", (int)QCD_DF64);')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, c = line.split()
        got[(a, b)] = int(c)
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
    assert got[("enum", "QCD_DF64")] == qcd.DF64


def test_field_bytes_host_validation(lib):
    g = qcd.Geom((ctypes.c_int32 * 4)(4, 4, 4, 8), (ctypes.c_int32 * 4)(1, 1, 1, -1), 18)
    f = qcd.wilson(0.12)
    Vh = 4 * 4 * 4 * 8 // 2
    assert lib.qcd_field_bytes(ctypes.byref(g), ctypes.byref(f), qcd.F32, 1) == Vh * 96
    assert lib.qcd_field_bytes(ctypes.byref(g), ctypes.byref(f), qcd.F64, 2) == 2 * Vh * 192
    assert lib.qcd_field_bytes(ctypes.byref(g), ctypes.byref(f), qcd.F16, 1) == Vh * (48 + 4)
    assert lib.qcd_field_bytes(ctypes.byref(g), ctypes.byref(f), qcd.DF64, 1) == Vh * 192
    d = qcd.dwf(8, 1.8, 0.02)
    assert lib.qcd_field_bytes(ctypes.byref(g), ctypes.byref(d), qcd.F32, 1) == 8 * Vh * 96
    bad = qcd.Geom((ctypes.c_int32 * 4)(4, 3, 4, 8), (ctypes.c_int32 * 4)(1, 1, 1, -1), 18)
    assert lib.qcd_field_bytes(ctypes.byref(bad), ctypes.byref(f), qcd.F32, 1) == 0
    assert "even" in lib.qcd_last_error().decode()
    badf = qcd.wilson(-1.0)
    assert lib.qcd_field_bytes(ctypes.byref(g), ctypes.byref(badf), qcd.F32, 1) == 0


def test_gauge_load_rejects_bad_geometry_before_any_launch(lib):
    h = ctypes.c_void_p()
    g = qcd.Geom((ctypes.c_int32 * 4)(4, 4, 4, 8), (ctypes.c_int32 * 4)(1, 1, 1, 2), 18)
    st = lib.qcd_gauge_load(ctypes.byref(g), ctypes.c_void_p(1), None, ctypes.byref(h))
    assert st == qcd.ERR_ARG and "bc" in lib.qcd_last_error().decode()
    g = qcd.Geom((ctypes.c_int32 * 4)(4, 4, 4, 8), (ctypes.c_int32 * 4)(1, 1, 1, -1), 10)
    assert lib.qcd_gauge_load(ctypes.byref(g), ctypes.c_void_p(1), None, ctypes.byref(h)) == qcd.ERR_ARG
    assert lib.qcd_gauge_load(None, ctypes.c_void_p(1), None, ctypes.byref(h)) == qcd.ERR_ARG
    assert lib.qcd_gauge_free(None) == qcd.OK
    assert lib.qcd_set_tuning(3) == qcd.ERR_ARG
