"""The allocation-free block-column solve against the regular FP64 solve.

dyson_solve_block_column_noalloc serves callers that may not allocate device
memory while they run (a device heap reserved by another framework's pool,
latency-bound loops, tools that must not change the library's footprint): its
scratch is a fixed file-scope device array.  This file is collected last so a
failure here leaves every other test already run.  Two calls in a row, on
different sources, must each match dyson_solve_columns (FP64) within the FP64
path's 1e-12 relative tolerance; the second call sees the first call's leftover
scratch contents and leaves the device's free memory unchanged.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu


def _noalloc(lib, torch, p, lam_dev, J_dev, source, out):
    sweeps = C.c_int32(0)
    rc = lib.dyson_solve_block_column_noalloc(
        C.c_void_p(lam_dev.data_ptr()), C.c_void_p(J_dev.data_ptr()), p.Lx, p.Ly, p.Nt, p.Nm, p.dt, p.beta,
        source, 1e-13, 400, C.c_void_p(out.data_ptr()), C.byref(sweeps),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.dyson_noalloc_last_error().decode()
    return sweeps.value


def test_noalloc_matches_regular_solve_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_5994_gb300 import binding
    lib = binding.load()
    p = wl.random_tables(wl.small(L=4, Ly=3, Nt=20, Nm=12, trap_c=0.3, U0=16.0, aU=0.1, aJ=0.2, omega=8.0),
                         seed=21, rel=0.2)
    s = binding.Solver(p, device=0, stream=torch.cuda.current_stream())
    s.build_sigma()
    lam_dev = torch.empty((p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
    assert lib.dyson_copy_sigma(s.h, C.c_void_p(lam_dev.data_ptr()), 1) == 0
    J_dev = torch.from_numpy(np.ascontiguousarray(p.J)).to("cuda:0")
    for k, source in enumerate((5, 0)):
        ref = torch.empty((1, p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
        s.solve([source], precision=binding.PREC_F64, tol=1e-13, max_sweeps=400, g_out=ref)
        out = torch.full((p.Nr, p.Nc, p.Nc), float("nan"), dtype=torch.complex128, device="cuda:0")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        sweeps = _noalloc(lib, torch, p, lam_dev, J_dev, source, out)
        torch.cuda.synchronize()
        if k == 1:
            # the promise itself: once its kernels are loaded, a call changes no device footprint
            assert torch.cuda.mem_get_info()[0] == free0
        assert sweeps > 1
        err = (torch.abs(out - ref[0]).max() / torch.abs(ref[0]).max()).item()
        assert err < 1e-12, f"source {source}: relative difference {err:.3e}"
    s.close()


def test_noalloc_rejects_oversized_block_columns():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1309_5994_gb300 import binding
    lib = binding.load()
    dummy = torch.zeros(2, dtype=torch.complex128, device="cuda:0")
    # 16 x 16 sites at Nc = 256 need 256 * 256^2 * 16 bytes = 256 MiB > 16 MiB of scratch
    rc = lib.dyson_solve_block_column_noalloc(C.c_void_p(dummy.data_ptr()), C.c_void_p(dummy.data_ptr()),
                                              16, 16, 112, 32, 0.05, 2.0, 0, 1e-12, 10,
                                              C.c_void_p(dummy.data_ptr()), None, None)
    assert rc == -1 and b"exceeds" in lib.dyson_noalloc_last_error()
