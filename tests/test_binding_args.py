"""The Python binding refuses host, mis-typed or mis-sized tensors and arrays for the C ABI's
pointer arguments before the library sees a pointer: a host address handed to a kernel would
fault the GPU.  No GPU is needed (the solver below has no context and no library)."""
import numpy as np
import pytest
import torch

import workloads as wl
from paper_1309_5994_gb300 import binding


class _NoLib:
    def __getattr__(self, name):
        raise AssertionError(f"the library was called ({name}) with unchecked arguments")


def _fake_solver(p):
    s = binding.Solver.__new__(binding.Solver)
    s.lib, s.p, s._torch, s.h, s.device = _NoLib(), p, torch, None, 0
    return s


def test_device_buffer_refuses_host_and_mis_typed_tensors():
    for t in (torch.zeros(4, dtype=torch.complex128), torch.zeros(4, dtype=torch.float64)):
        with pytest.raises(ValueError):
            binding.device_buffer(t, torch.complex128, 4, None, "t")


def test_solver_checks_arguments_before_calling_the_library():
    p = wl.small(L=2, Ly=2, Nt=3, Nm=2)
    s = _fake_solver(p)
    n_el = p.Nr * p.Nc * p.Nc
    host = torch.zeros(n_el, dtype=torch.complex128)
    with pytest.raises(ValueError):
        s.selfenergy_step(host)
    with pytest.raises(ValueError):
        s.local_greens(out=host)
    with pytest.raises(ValueError):
        s.solve([0], g_out=host)
    with pytest.raises(ValueError):
        s.solve_vectors([0], [0], g_out=host)
    with pytest.raises(ValueError):
        s.solve_vectors([0], [0, 1])
    with pytest.raises(ValueError):
        s.adjoint(np.zeros(p.Nr + 1))
    with pytest.raises(ValueError):
        s.adjoint_obs(np.zeros(p.Nr - 1))
    f = torch.zeros(p.Nr * p.Nt, dtype=torch.float64)
    with pytest.raises(ValueError):
        s.observables_device(f, f, f)
