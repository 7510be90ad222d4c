"""The C-ABI library builds, loads and exports every function include/*.h declares.

No compute call is made: these run without a GPU.
"""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(dyson_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_1309_5994_gb300 import build
    return build.build()


def test_header_declares_the_five_calls():
    names = declared_functions()
    for call in ("dyson_init", "dyson_build_sigma", "dyson_solve_columns", "dyson_observables",
                 "dyson_destroy", "dyson_last_error"):
        assert call in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = declared_functions() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_loads_and_reports_version(libpath):
    from paper_1309_5994_gb300 import binding
    lib = binding.load()
    assert lib.dyson_version().decode().startswith("gb300-dyson")
    for name in binding.EXPORTS:
        assert hasattr(lib, name)
    assert set(binding.EXPORTS) <= declared_functions()


def test_init_rejects_bad_arguments_without_touching_a_gpu(libpath):
    import ctypes as C
    from paper_1309_5994_gb300 import binding
    lib = binding.load()
    h = C.c_void_p()
    # NULL out pointer and NULL structs are rejected before any CUDA call
    assert lib.dyson_init(None, None, None, None, None, 0, None) == -1
    assert lib.dyson_init(C.byref(h), None, None, None, None, 0, None) == -1
    lat = binding.Lattice(0, 4)
    con = binding.Contour(4, 4, 0.1, 1.0)
    trap = binding.Trap(0.1, 0.0)
    U = (C.c_double * 16)()
    drv = binding.Drive(C.cast(U, C.POINTER(C.c_double)), C.cast(U, C.POINTER(C.c_double)))
    assert lib.dyson_init(C.byref(h), C.byref(lat), C.byref(con), C.byref(trap), C.byref(drv), 0, None) == -1
    assert b"sites" in lib.dyson_last_error(None)
    lat = binding.Lattice(2, 2)
    con = binding.Contour(4, 4, -0.1, 1.0)
    assert lib.dyson_init(C.byref(h), C.byref(lat), C.byref(con), C.byref(trap), C.byref(drv), 0, None) == -1
    # the largest sizes: 65535 sites, a contour of 2048 points
    big = binding.Lattice(256, 256)
    con = binding.Contour(4, 4, 0.1, 1.0)
    assert lib.dyson_init(C.byref(h), C.byref(big), C.byref(con), C.byref(trap), C.byref(drv), 0, None) == -1
    long = binding.Contour(1000, 49, 0.1, 1.0)
    assert lib.dyson_init(C.byref(h), C.byref(lat), C.byref(long), C.byref(trap), C.byref(drv), 0, None) == -1
    assert b"2048" in lib.dyson_last_error(None)
    nan_trap = binding.Trap(float("nan"), 0.0)
    assert lib.dyson_init(C.byref(h), C.byref(lat), C.byref(con), C.byref(nan_trap), C.byref(drv), 0, None) == -1
    assert lib.dyson_build_sigma(None) == -1
