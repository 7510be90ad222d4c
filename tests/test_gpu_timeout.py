"""The bounded waits of the tensor-core pipelines run out on a healthy pipeline.

dyson_set_wait_limit shortens the time limit of the pipeline waits (the sweep GEMM
and the split-product residual) to a nanosecond: the first wait that is not met at
once expires, the CTA raises its error flag, lets its in-flight copies and MMAs land
(those drain waits keep their 2 s), frees its tensor memory and exits, and the solve
returns DYSON_ERR_TIMEOUT.  With the default limit restored the same context solves
correctly.  No fault and no hang is involved: every wait is bounded and the
expiry path is the kernels' ordinary exit.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import dyson

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_expired_pipeline_wait_returns_timeout_and_the_context_recovers(torch_cuda, lib):
    from paper_1309_5994_gb300 import binding
    torch = torch_cuda
    p = wl.random_tables(wl.small(L=2, Ly=2, Nt=24, Nm=16, trap_c=0.3, U0=20.0), seed=41, rel=0.2)
    S = dyson.setup(p)
    sources = [0, 3]
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    s = binding.Solver(p, device=0)
    s.set_sweep_variant(binding.SWEEP_SINGLE_CTA)          # one CTA per tile, no cluster
    s.build_sigma()
    g = torch.empty((len(sources), p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
    try:
        s.set_wait_limit(1e-9)
        with pytest.raises(binding.DysonError) as e:
            s.solve(sources, precision=binding.PREC_TF32X3_F64REF, tol=1e-12, g_out=g)
        assert e.value.code == -5                            # DYSON_ERR_TIMEOUT
        assert "time limit" in str(e.value)
    finally:
        s.set_wait_limit(0.0)                                # back to 2 s for this device
    res = s.solve(sources, precision=binding.PREC_TF32X3_F64REF, tol=1e-12, g_out=g)
    assert res.status == 0
    got = g.cpu().numpy()
    for q in range(len(sources)):
        want = ref[:, :, q * p.Nc:(q + 1) * p.Nc]
        assert np.abs(got[q] - want).max() / np.abs(want).max() < 1e-12
    with pytest.raises(binding.DysonError) as e:
        s.set_wait_limit(-1.0)
    assert e.value.code == -1
    s.close()
