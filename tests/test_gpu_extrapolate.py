"""Delta t -> 0 extrapolation (Sec. IV.D) on the GPU against the oracle."""
import numpy as np
import pytest

import workloads as wl
from oracle import extrapolate as ex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("ms", [(1,), (1, 2), (1, 2, 4), (1, 3, 5, 6)])
def test_combination_matches_the_oracle(torch_cuda, lib, ms):
    from paper_1309_5994_gb300 import binding
    torch = torch_cuda
    rng = np.random.default_rng(11)
    rows, nt0 = 37, 29                               # ragged against the 256-thread blocks
    tabs = [rng.normal(size=(rows, m * nt0 + (b % 2))) for b, m in enumerate(ms)]
    tabs[0][3, 0] = np.nan                           # NaN (D at t = 0) stays NaN
    got = binding.extrapolate_dt([torch.from_numpy(t).cuda() for t in tabs], ms).cpu().numpy()
    ref = ex.extrapolate(tabs, 0.05, ms, nt0)
    assert np.isnan(got[3, 0]) and np.isnan(ref[3, 0])
    ok = ~np.isnan(ref)
    assert np.abs(got[ok] - ref[ok]).max() <= 1e-14 * np.abs(ref[ok]).max()


@pytest.mark.parametrize("bad", ["m0", "order", "short", "many"])
def test_invalid_arguments_are_rejected_on_the_host(torch_cuda, lib, bad):
    from paper_1309_5994_gb300 import binding
    torch = torch_cuda
    t = lambda n: torch.zeros((4, n), dtype=torch.float64, device="cuda")
    cases = {"m0": ([t(5), t(10)], (2, 4)), "order": ([t(5), t(20), t(10)], (1, 4, 2)),
             "short": ([t(5), t(8)], (1, 2)), "many": ([t(5)] * 5, (1, 2, 3, 4, 5))}
    tabs, ms = cases[bad]
    with pytest.raises(binding.DysonError, match="INVALID_ARG"):
        binding.extrapolate_dt(tabs, ms)


@pytest.mark.parametrize("prec,tol,bound", [(0, 1e-13, 1e-11), (1, 1e-11, 1e-8)])
def test_extrapolated_observables_match_the_oracle(torch_cuda, lib, prec, tol, bound):
    """Three refined contours of a driven 3x2 lattice, all block columns, quadratic extrapolation."""
    from paper_1309_5994_gb300.extrapolate import extrapolated_observables
    p0 = wl.small(L=3, Ly=2, Nt=8, Nm=4, dt=0.1, beta=1.0, trap_c=0.3, U0=8.0, J0=1.0, aU=0.1, aJ=0.2,
                  omega=5.0)
    ms = (1, 2, 4)
    probs = [wl.refine(p0, m) for m in ms]
    got = extrapolated_observables(probs, ms, precision=prec, tol=tol, keep_raw=True)
    raw = [ex.observables_dense(q) for q in probs]
    for k, name in enumerate(("n", "ekin", "docc")):
        ref = ex.extrapolate([r[k] for r in raw], p0.dt, ms, p0.Nt)
        g = got[name].cpu().numpy()
        assert g.shape == (p0.Nr, p0.Nt)
        ok = ~np.isnan(ref)
        assert np.array_equal(ok, ~np.isnan(g))
        assert np.abs(g[ok] - ref[ok]).max() <= bound * np.abs(ref[ok]).max(), name
        for b in range(len(ms)):                     # and the per-grid tables it combined
            rb = raw[b][k]
            gb = got["raw"][name][b].cpu().numpy()
            okb = ~np.isnan(rb)
            assert np.abs(gb[okb] - rb[okb]).max() <= bound * np.abs(rb[okb]).max(), (name, b)
