"""Batched solves of uneven instances (dyson_batch_*) against the oracle.

Tolerances: the batched solve is the mixed-precision path refined to an FP64
Dyson residual, so small cases are held to the same 1e-12 as
dyson_solve_columns; full-size samples of the uneven batch are held to 1e-8
on G columns (refined to a residual of 1e-10; the conditioning of I - K is
O(10-100) on these contours) and 1e-6 on densities, the reduced-precision bound.
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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SMALL = [
    dict(L=2, Ly=2, Nt=24, Nm=16, trap_c=0.3, U0=20.0),                                  # Nc = 64
    dict(L=3, Ly=2, Nt=40, Nm=48, trap_c=0.2, U0=16.0, aU=0.1, aJ=0.2, omega=20.0),      # Nc = 128
    dict(L=1, Ly=3, Nt=72, Nm=48, trap_c=0.1, U0=20.0),                                  # Nc = 192
]


def _solvers(torch, problems):
    from paper_1309_5994_gb300 import binding
    stream = torch.cuda.Stream(device=0)
    out = []
    for p in problems:
        s = binding.Solver(p, device=0, stream=stream)
        s.build_sigma()
        out.append(s)
    return out, stream


def test_batch_of_uneven_contours_matches_dense(torch_cuda, lib):
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    problems = [wl.random_tables(wl.small(**kw), seed=21 + k, rel=0.2) for k, kw in enumerate(SMALL)]
    solvers, stream = _solvers(torch, problems)
    sources = [[0, 3], [1, 2, 5], [2]]
    g = [torch.empty((len(src), p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
         for src, p in zip(sources, problems)]
    b = binding.Batch(solvers)
    res = b.solve(sources, tol=1e-13, max_sweeps=400, graph_sweeps=6, g_outs=g)
    torch.cuda.synchronize()
    assert all(r.status == 0 for r in res)
    assert b.launch_count() > 0 and b.launch_count() % 3 == 0          # gather, GEMM, check per sweep
    for k, p in enumerate(problems):
        S = dyson.setup(p)
        ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources[k]))
        got = g[k].cpu().numpy()
        for q in range(len(sources[k])):
            assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12
        assert res[k].report["refinements"] > 0 and res[k].report["sweeps"] > 0
    b.close()


def test_batch_matches_single_context_solves(torch_cuda, lib):
    """The same instances solved one context at a time give the same G to FP64 rounding."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    problems = [wl.random_tables(wl.small(**kw), seed=31 + k, rel=0.2) for k, kw in enumerate(SMALL[:2])]
    solvers, stream = _solvers(torch, problems)
    sources = [[1], [0, 4]]
    gb = [torch.empty((len(s), p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
          for s, p in zip(sources, problems)]
    b = binding.Batch(solvers)
    b.solve(sources, tol=1e-12, g_outs=gb)
    nb = [sv.observables()[0] for sv in solvers]
    for k, (sv, p) in enumerate(zip(solvers, problems)):
        gs = torch.empty_like(gb[k])
        sv.solve(sources[k], precision=1, tol=1e-12, g_out=gs)
        torch.cuda.synchronize()
        assert _rel(gb[k].cpu().numpy(), gs.cpu().numpy()) < 1e-11
        ns = sv.observables()[0]
        for i in sources[k]:
            assert np.abs(nb[k][i] - ns[i]).max() < 1e-11
    b.close()


def test_batch_rejects_bad_members(torch_cuda, lib):
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    good = wl.small(**SMALL[0])
    bad = wl.small(L=2, Ly=2, Nt=7, Nm=5)                                   # Nc = 19: no tensor-core path
    solvers, _ = _solvers(torch, [good, bad])
    with pytest.raises(binding.DysonError) as e:
        binding.Batch([solvers[0], solvers[0]])
    assert e.value.code == -1
    b = binding.Batch(solvers)
    with pytest.raises(binding.DysonError) as e:
        b.solve([[0], [0]])
    assert e.value.code == -1
    b.close()


def test_uneven_batch_of_64_sampled(torch_cuda, lib):
    """Six instances of the seeded uneven batch (L in 8..24, Nc in {128, 192, 256}),
    one block column each, solved in one batch: sampled vector columns and the
    source-site densities against the oracle's complex128 series."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    allp = wl.uneven_batch()
    problems = [p for p in allp if p.Lx <= 12][:6]                         # the oracle's share stays small
    assert {p.Nc for p in problems} == {128, 192, 256}
    solvers, _ = _solvers(torch, problems)
    sources = [[p.Nr // 2 + p.Lx // 2] for p in problems]                  # a site near the trap centre
    g = [torch.empty((1, p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0") for p in problems]
    b = binding.Batch(solvers)
    res = b.solve(sources, tol=1e-10, g_outs=g)
    assert all(r.status == 0 for r in res)
    rng = np.random.default_rng(4)
    for k, p in enumerate(problems):
        S = dyson.setup(p)
        i = sources[k][0]
        zs = [int(z) for z in rng.choice(p.Nc, 2, replace=False)]
        B = dyson.rhs_vector_columns(S, [(i, z) for z in zs])
        ref, _, _ = dyson.neumann_solve(S, B, tol=1e-15, max_sweeps=400)
        assert dyson.residual(S, B, ref) < 1e-11
        got = g[k][0].cpu().numpy()
        for c, z in enumerate(zs):
            assert _rel(got[:, :, z], ref[:, :, c]) < 1e-8
        n, _, _ = solvers[k].observables()
        Bn = dyson.rhs_vector_columns(S, [(i, t) for t in range(p.Nt)])
        Gn, _, _ = dyson.neumann_solve(S, Bn, tol=1e-15, max_sweeps=400)
        n_ref = np.array([np.real(-1j * Gn[i, t, t]) for t in range(p.Nt)])
        assert np.abs(n[i] - n_ref).max() / np.abs(n_ref).max() < 1e-6
    b.close()


@pytest.mark.parametrize("inner", ["series", "auto"])
def test_batch_with_a_divergent_member(torch_cuda, lib, inner):
    """One instance with rho(K) = 1.41 (J/U = 1/2) among convergent ones.  With the
    series only, the batch returns DIVERGED for it and still solves the others to
    1e-12; by default the divergent member is then solved by GMRES, to 1e-12 too."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    divergent = wl.small(L=3, Ly=3, Nt=24, Nm=16, dt=0.05, beta=2.0, trap_c=0.0, U0=4.0, J0=2.0)
    problems = [wl.random_tables(wl.small(**SMALL[0]), seed=41, rel=0.2), divergent,
                wl.random_tables(wl.small(**SMALL[1]), seed=42, rel=0.2)]
    solvers, _ = _solvers(torch, problems)
    if inner == "series":
        solvers[1].set_inner_solver(binding.INNER_SERIES)
    sources = [[1], [4], [2]]
    g = [torch.empty((1, p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0") for p in problems]
    b = binding.Batch(solvers)
    res = b.solve(sources, tol=1e-12, g_outs=g, allow=(0, -4))
    if inner == "series":
        assert [r.status for r in res] == [0, -4, 0]
    else:
        assert [r.status for r in res] == [0, 0, 0] and res[1].report["inner_gmres"] == 1
    for k in ((0, 2) if inner == "series" else (0, 1, 2)):
        p = problems[k]
        S = dyson.setup(p)
        ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources[k]))
        assert _rel(g[k][0].cpu().numpy(), ref) < 1e-12
    b.close()
