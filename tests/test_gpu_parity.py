"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Floating-point tolerances:
* FP64 path: 1e-12 relative (max-norm over the compared block, relative to its
  max-norm) on problems whose series partial sums stay O(1);
* mixed-precision path with FP64 residual refinement to tol: the same 1e-12
  bound, since the refined result is fixed by the FP64 residual;
* full-size sampled checks: 1e-6 relative on G and on densities, the bound for
  reduced-precision paths.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import dyson, observables

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _solver(p):
    from paper_1309_5994_gb300 import binding
    s = binding.Solver(p, device=0)
    s.build_sigma()
    return s


def _solve(torch, s, p, sources, prec, tol=1e-13, max_sweeps=400, allow=(0,)):
    g = torch.empty((len(sources), p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
    res = s.solve(sources, precision=prec, tol=tol, max_sweeps=max_sweeps, g_out=g, allow=allow)
    return g.cpu().numpy(), res


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SMALL = [
    dict(L=3, Ly=2, Nt=7, Nm=5, trap_c=0.3, aU=0.1, aJ=0.2, omega=6.0),     # Nc = 19: ragged tiles
    dict(L=2, Ly=2, Nt=3, Nm=1, beta=0.5),                                    # Nm = 1
    dict(L=5, Ly=1, Nt=40, Nm=20, trap_c=0.1),                                # chain, Nc = 100 (2 tiles)
    dict(L=1, Ly=1, Nt=10, Nm=6),                                             # one site: no bonds, G = Lambda
]


@pytest.mark.parametrize("kw", SMALL)
def test_sigma_matches_oracle(torch_cuda, lib, kw):
    p = wl.small(**kw)
    S = dyson.setup(p)
    s = _solver(p)
    got = s.sigma()
    assert _rel(got, S.Lam) < 1e-13


def test_sigma_trapped_4x4(torch_cuda, lib):
    p = wl.trapped_4x4_nc64()
    S = dyson.setup(p)
    s = _solver(p)
    assert _rel(s.sigma(), S.Lam) < 1e-13


@pytest.mark.parametrize("kw", SMALL)
@pytest.mark.parametrize("prec", [0, 1])
def test_solve_small_matches_dense(torch_cuda, lib, kw, prec):
    p = wl.random_tables(wl.small(**kw), seed=7, rel=0.2)
    S = dyson.setup(p)
    sources = list(range(p.Nr)) + [0]        # every site, plus a repeat
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    s = _solver(p)
    got, res = _solve(torch_cuda, s, p, sources, prec, tol=1e-13)
    for q in range(len(sources)):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12
    if p.Nr == 1:                            # no bonds: G = Lambda, up to the Lambda build's rounding
        assert _rel(got[0][0], S.Lam[0]) < 1e-13


TC_CASES = [
    dict(L=2, Ly=2, Nt=24, Nm=16, trap_c=0.3, U0=20.0),                     # Nc = 64: one M tile per half
    dict(L=3, Ly=2, Nt=40, Nm=48, trap_c=0.2, U0=16.0, aU=0.1, aJ=0.2, omega=20.0),   # Nc = 128
    dict(L=1, Ly=3, Nt=72, Nm=48, trap_c=0.1, U0=20.0),                     # Nc = 192: 3 M tiles
]


@pytest.mark.parametrize("kw", TC_CASES)
def test_tensor_core_path_matches_dense(torch_cuda, lib, kw):
    """Contour lengths that are multiples of 64 run the 3xTF32 tcgen05 sweep."""
    p = wl.random_tables(wl.small(**kw), seed=11, rel=0.2)
    S = dyson.setup(p)
    sources = list(range(p.Nr))
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    s = _solver(p)
    s.profile(True)
    got, res = _solve(torch_cuda, s, p, sources, 1, tol=1e-13)
    launches = s.profile_query(2)[0] + s.profile_query(5)[0]
    assert launches > 0                                     # a tensor-core sweep ran
    assert s.profile_query(5)[0] == 0                        # the single-CTA form is the default
    assert s.profile_query(4)[0] == res.report["refinements"] > 0   # every residual used BF16 slice products
    for q in range(len(sources)):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12


@pytest.mark.parametrize("kw", TC_CASES[:2])
def test_uniform_hopping_residual_matches_dense(torch_cuda, lib, kw):
    """Hopping equal on every bond (the trapped and driven lattices): the residual folds J(t)
    into the Lambda slices and sums the neighbours' columns as exact fixed-point integers,
    with no FP64 gather. The refined result must meet the dense solve at 1e-12 all the same
    (seven slices at this tolerance)."""
    p = wl.small(**kw)
    assert np.all(p.J == p.J[:1])                            # one J(t) row for every bond
    S = dyson.setup(p)
    sources = list(range(p.Nr))
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    s = _solver(p)
    s.profile(True)
    got, res = _solve(torch_cuda, s, p, sources, 1, tol=1e-13)
    assert s.profile_query(4)[0] == res.report["refinements"] > 0
    for q in range(len(sources)):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12


@pytest.mark.parametrize("tables", ["per_bond", "uniform"])
@pytest.mark.parametrize("tol", [1e-8, 1e-6])
def test_short_slice_residual_at_loose_tolerances(torch_cuda, lib, tol, tables):
    """Tolerances of 1e-8 and looser compute the FP64-accurate residual from the first five
    operand slices (15 products): the residual the solve reports must still be the true
    residual of the returned G, re-evaluated in complex128 by the oracle, to 2 % of the tolerance.
    Per-bond hopping gathers X in FP64; uniform hopping sums it in fixed point."""
    p = wl.small(**TC_CASES[0])
    if tables == "per_bond":
        p = wl.random_tables(p, seed=31, rel=0.2)
    S = dyson.setup(p)
    sources = list(range(p.Nr))
    s = _solver(p)
    s.profile(True)
    got, res = _solve(torch_cuda, s, p, sources, 1, tol=tol)
    assert s.profile_query(4)[0] == res.report["refinements"] > 0
    B = dyson.rhs_block_columns(S, sources)
    G = np.concatenate([got[q] for q in range(len(sources))], axis=2)
    D = G - B - dyson.apply_K(S, G)
    R = np.maximum(np.abs(D.real), np.abs(D.imag))       # the tensor-core path's norm: the larger component
    true = max(R[:, :, q * p.Nc:(q + 1) * p.Nc].max() / np.abs(B[:, :, q * p.Nc:(q + 1) * p.Nc]).max()
               for q in range(len(sources)))
    assert true <= tol and abs(res.report["residual"] - true) <= 0.02 * tol


def test_pair_kernel_ragged_column_tiles(torch_cuda, lib):
    """Nc = 128 with the CTA-pair sweep selected.  Three block columns make 384
    vector columns: the last 256-column tile has its odd CTA's half wholly past the end."""
    p = wl.random_tables(wl.small(**TC_CASES[1]), seed=12, rel=0.2)
    S = dyson.setup(p)
    sources = [0, 3, 5]
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    s = _solver(p)
    s.set_sweep_variant(1)
    s.set_support_truncation(False)          # truncated sweeps would run on the single-CTA kernel
    s.profile(True)
    got, res = _solve(torch_cuda, s, p, sources, 1, tol=1e-13)
    assert s.profile_query(5)[0] > 0 and s.profile_query(2)[0] == 0
    for q, i in enumerate(sources):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12


FUSED_CASES = [
    # (problem, sources, variant): Nc = 128, three block columns (the last 256-column
    # tile's odd half wholly past the end); Nc = 256 in both fused forms; Nc = 384
    # (three row groups of 256) on a chain
    (dict(L=3, Ly=2, Nt=40, Nm=48, trap_c=0.2, U0=16.0, aU=0.1, aJ=0.2, omega=20.0), [0, 3, 5], 2),
    (dict(L=4, Ly=3, Nt=96, Nm=64, trap_c=0.1, U0=20.0, aU=0.1, aJ=0.2, omega=20.0), [0, 5, 11, 6], 2),
    (dict(L=4, Ly=3, Nt=96, Nm=64, trap_c=0.1, U0=20.0, aU=0.1, aJ=0.2, omega=20.0), [0, 5, 11, 6], 3),
    (dict(L=3, Ly=1, Nt=160, Nm=64, trap_c=0.1, U0=20.0), [0, 1, 2], 2),
]


@pytest.mark.parametrize("kw,sources,variant", FUSED_CASES)
def test_fused_sweep_matches_dense(torch_cuda, lib, kw, sources, variant):
    """The fused gather + GEMM sweep (one launch per sweep, X gathered into shared
    memory) equals the dense solve, and no gather or unfused GEMM launch runs."""
    p = wl.random_tables(wl.small(**kw), seed=17, rel=0.2)
    S = dyson.setup(p)
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    s = _solver(p)
    s.set_sweep_variant(variant)
    s.profile(True)
    got, res = _solve(torch_cuda, s, p, sources, 1, tol=1e-13)
    assert s.profile_query(8)[0] > 0
    assert s.profile_query(2)[0] == s.profile_query(5)[0] == s.profile_query(6)[0] == 0
    for q in range(len(sources)):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12
    n, e, _ = s.observables()
    for q, src in enumerate(sources):
        n_ref, e_ref, _ = observables.observables_block_column(S, src, ref[:, :, q * p.Nc:(q + 1) * p.Nc])
        assert np.abs(n[src] - n_ref).max() < 1e-11 and np.abs(e[src] - e_ref).max() < 1e-11


@pytest.mark.parametrize("kw,sources,variant", FUSED_CASES[:2] + [(FUSED_CASES[1][0], list(range(12)), 2)])
def test_graph_replayed_series_is_bit_identical(torch_cuda, lib, kw, sources, variant):
    """The inner series replayed from captured graphs (its stopping rule applied on the
    device, one host synchronisation per graph of sweeps) returns the same G bit for bit,
    the same sweep and refinement counts and the same residual as the loop with one
    synchronisation per sweep: after truncated first sweeps (a few sources) and without
    them (every site a source), and with a graph of 2 sweeps, where the series stops
    inside a replay."""
    p = wl.random_tables(wl.small(**kw), seed=23, rel=0.2)
    out, syncs = {}, {}
    for gsw in (0, 16, 2):
        s = _solver(p)
        s.set_sweep_variant(variant)
        s.set_graph_sweeps(gsw)
        got, res = _solve(torch_cuda, s, p, sources, 1, tol=1e-10)
        out[gsw] = (got, res.report["sweeps"], res.report["refinements"], res.report["residual"])
        syncs[gsw] = res.report["host_syncs"]
        if gsw == 16:
            from paper_1309_5994_gb300 import binding
            for bad in (3, -2, 66):
                with pytest.raises(binding.DysonError):
                    s.set_graph_sweeps(bad)
        s.close()
    for gsw in (16, 2):
        assert np.array_equal(out[gsw][0], out[0][0])
        assert out[gsw][1:] == out[0][1:]
    # fewer waits for the device with graphs: one per replay instead of one per sweep
    # (GMRES steps, where a case switches to them, wait once each in both)
    assert syncs[16] < syncs[0]


@pytest.mark.parametrize("case", ["nc64_ragged", "nc256_pair", "nc256_fused"])
def test_support_truncation_is_bit_identical(torch_cuda, lib, case):
    """Skipping the (site, column-tile) blocks the first series has not reached yet
    changes no bit of the result and no sweep count; both agree with the dense solve.
    Nc = 64: five block columns in two 256-column tiles (the second ragged), four
    sources sharing a tile.  Nc = 256 with the CTA-pair variant: the truncated first
    series runs on the single-CTA kernel, the later refinements on the pair.  Nc = 256
    with the fused variant: the fused kernel skips the tiles itself."""
    if case == "nc64_ragged":
        kw, sources, variant = dict(L=6, Ly=5, Nt=24, Nm=16, trap_c=0.1, U0=20.0), [0, 7, 29, 13, 22], 0
    else:
        kw, sources = dict(L=4, Ly=3, Nt=96, Nm=64, trap_c=0.1, U0=20.0), [0, 11]
        variant = 1 if case == "nc256_pair" else 2
    p = wl.random_tables(wl.small(**kw), seed=13, rel=0.2)
    out = {}
    for trunc in (True, False):
        s = _solver(p)
        s.set_sweep_variant(variant)
        s.set_support_truncation(trunc)
        s.profile(True)
        out[trunc] = _solve(torch_cuda, s, p, sources, 1, tol=1e-13) + (
            s.profile_query(2)[0], s.profile_query(5)[0], s.profile_query(8)[0])
        s.close()
    (g1, r1, single1, pair1, fused1), (g0, r0, single0, pair0, fused0) = out[True], out[False]
    assert np.array_equal(g1, g0)
    assert r1.report["sweeps"] == r0.report["sweeps"] and r1.report["refinements"] == r0.report["refinements"]
    if variant == 1:
        assert single1 > 0 and pair1 > 0 and single0 == 0
    if variant == 2:
        assert single1 == pair1 == single0 == pair0 == 0 and fused1 > 0 and fused0 > 0
    S = dyson.setup(p)
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    for q in range(len(sources)):
        assert _rel(g1[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12


def test_c4v_wedge_solve_equals_the_full_solve(torch_cuda, lib):
    """App. A: a centred trap and a uniform drive keep C4v.  The 4x4 lattice has 3
    orbits (corners, edges, centre); solving their representatives and filling the
    rest by symmetry gives every block column and observable of the full solve."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    p = wl.small(L=4, Ly=4, Nt=24, Nm=16, trap_c=0.3, U0=20.0, aU=0.1, aJ=0.2, omega=20.0)
    S = dyson.setup(p)
    sources = list(range(p.Nr))
    full = _solver(p)
    g_full, r_full = _solve(torch, full, p, sources, 1, tol=1e-13)
    n_full, e_full, d_full = full.observables()
    sym = _solver(p)
    sym.set_symmetry(binding.SYMMETRY_C4V)
    g_sym, r_sym = _solve(torch, sym, p, sources, 1, tol=1e-13)
    n_sym, e_sym, d_sym = sym.observables()
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    for q in range(p.Nr):
        assert _rel(g_sym[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12
        assert _rel(g_sym[q], g_full[q]) < 1e-12
    assert np.abs(n_sym - n_full).max() < 1e-12 and np.abs(e_sym - e_full).max() < 1e-12
    assert np.allclose(d_sym[:, 1:], d_full[:, 1:], rtol=0, atol=1e-10)
    # three representatives solved instead of sixteen block columns
    assert r_sym.report["gemm_flops"] < 0.3 * r_full.report["gemm_flops"]
    bad = _solver(wl.random_tables(p, seed=2, rel=0.1))
    with pytest.raises(binding.DysonError) as e:
        bad.set_symmetry(binding.SYMMETRY_C4V)
    assert e.value.code == -1


def test_autotune_picks_a_measured_candidate_and_solves(torch_cuda, lib):
    """Nc = 128: the tuner times both sweep variants over chunks of 1, 2, 4, 6 block
    columns, keeps the fastest (within its 2 % margin), and the solve under that
    choice still equals the dense solve."""
    p = wl.random_tables(wl.small(**TC_CASES[1]), seed=23, rel=0.2)
    S = dyson.setup(p)
    s = _solver(p)
    t = s.autotune(6)
    cands = t["candidates"]
    assert {c["chunk"] for c in cands} == {1, 2, 4, 6} and {c["variant"] for c in cands} == {0, 1, 2}
    best = cands[0]                  # the documented rule: a later candidate wins only when > 2 % faster
    for c in cands[1:]:
        if c["vector_columns_per_s"] > 1.02 * best["vector_columns_per_s"]:
            best = c
    assert (t["sweep_variant"], t["chunk_block_columns"]) == (best["variant"], best["chunk"])
    assert 1.02 * t["vector_columns_per_s"] >= max(c["vector_columns_per_s"] for c in cands)
    assert all(c["vector_columns_per_s"] > 0 for c in cands)
    sources = list(range(p.Nr))
    got, res = _solve(torch_cuda, s, p, sources, 1, tol=1e-13)
    assert res.report["chunks"] == -(-len(sources) // t["chunk_block_columns"])
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    for q in range(len(sources)):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12


@pytest.mark.parametrize("prec", [0, 1])
def test_trapped_4x4_all_columns_and_observables(torch_cuda, lib, prec):
    p = wl.trapped_4x4_nc64()
    S = dyson.setup(p)
    sources = list(range(p.Nr))
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    s = _solver(p)
    got, res = _solve(torch_cuda, s, p, sources, prec, tol=1e-13)
    for q in range(p.Nr):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12
    n, ekin, D = s.observables()
    for i in range(p.Nr):
        n_r, e_r, D_r = observables.observables_block_column(S, i, ref[:, :, i * p.Nc:(i + 1) * p.Nc])
        assert np.abs(n[i] - n_r).max() < 1e-12
        assert np.abs(ekin[i] - e_r).max() < 1e-12
        assert np.isnan(D[i, 0]) and np.abs(D[i, 1:] - D_r[1:]).max() < 1e-10


def test_unsolved_sites_report_nan(torch_cuda, lib):
    p = wl.small(L=3, Nt=5, Nm=4)
    s = _solver(p)
    s.solve([4], precision=0)
    n, _, _ = s.observables()
    assert np.all(np.isfinite(n[4])) and np.all(np.isnan(np.delete(n, 4, axis=0)))


def test_error_codes(torch_cuda, lib):
    from paper_1309_5994_gb300 import binding
    p = wl.small(L=3, Nt=5, Nm=4)
    s = binding.Solver(p, device=0)
    with pytest.raises(binding.DysonError) as e:
        s.solve([0])
    assert e.value.code == -7                               # solve before build_sigma
    s.build_sigma()
    with pytest.raises(binding.DysonError) as e:
        s.solve([p.Nr])
    assert e.value.code == -1                               # source out of range
    r = s.solve([0], max_sweeps=1, allow=(-3,))
    assert r.status == -3 and r.report["sweeps"] == 1       # not converged, results still written
    for call in (lambda: s.solve([]), lambda: s.local_greens([])):
        with pytest.raises(binding.DysonError) as e:        # no source site
            call()
        assert e.value.code == -1


def test_slow_series_reports_not_converged(torch_cuda, lib):
    """One imaginary point at beta = 1 puts the Matsubara block's spectral radius
    at 0.997: the series needs thousands of sweeps and the solve says so."""
    from paper_1309_5994_gb300 import binding
    p = wl.small(L=2, Ly=2, Nt=3, Nm=1)
    s = _solver(p)
    s.set_inner_solver(binding.INNER_SERIES)
    for prec in (0, 1):
        r = s.solve([0, 1], precision=prec, tol=1e-12, max_sweeps=50, allow=(-3,))
        assert r.status == -3
    n, _, _ = s.observables()
    assert np.all(np.isfinite(n[:2]))
    # AUTO: a series that runs through its sweep budget hands the chunk over to GMRES
    s.set_inner_solver(binding.INNER_AUTO)
    got, r = _solve(torch_cuda, s, p, [0, 1], 1, tol=1e-12, max_sweeps=50)
    assert r.status == 0 and r.report["inner_gmres"] == 1
    S = dyson.setup(p)
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, [0, 1]))
    for q in range(2):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-10


DIVERGENT = dict(L=3, Ly=3, Nt=24, Nm=16, dt=0.05, beta=2.0, trap_c=0.0, U0=4.0, J0=2.0)   # rho(K) = 1.41


def test_divergent_series_reports_diverged(torch_cuda, lib):
    """J/U = 1/2: the spectral radius of K is 1.41, so the series of App. C
    diverges.  The FP64 series and the mixed path forced to the series must
    report DIVERGED, keep the context usable and leave the CUDA context clean
    (no launch on a missing state)."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    p = wl.small(**DIVERGENT)
    S = dyson.setup(p)
    assert np.abs(np.linalg.eigvals(dyson.dense_K(S))).max() > 1.3
    s = _solver(p)
    s.set_inner_solver(binding.INNER_SERIES)
    g = torch.empty((1, p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
    for prec in (0, 1):
        res = s.solve([4], precision=prec, tol=1e-12, max_sweeps=400, g_out=g, allow=(-4,))
        assert res.status == -4
    s.observables()                                          # the context still answers
    torch.cuda.synchronize()
    ok = _solver(wl.small(**SMALL[0]))
    assert ok.solve([0], precision=1, tol=1e-12).status == 0


@pytest.mark.parametrize("inner", ["auto", "gmres"])
def test_gmres_solves_where_the_series_diverges(torch_cuda, lib, inner):
    """The same divergent problem with the GMRES inner solver of App. C (chosen by
    AUTO after the series fails, or forced): the refined result equals the dense
    solve to 1e-12."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    p = wl.random_tables(wl.small(**DIVERGENT), seed=9, rel=0.1)
    S = dyson.setup(p)
    s = _solver(p)
    if inner == "gmres":
        s.set_inner_solver(binding.INNER_GMRES, 24)
    sources = [0, 4, 8]
    got, res = _solve(torch, s, p, sources, 1, tol=1e-13, max_sweeps=400)
    assert res.status == 0 and res.report["inner_gmres"] == 1
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    for q in range(len(sources)):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12


@pytest.mark.parametrize("kw", [SMALL[0], TC_CASES[0], TC_CASES[1]])
def test_forced_gmres_matches_dense(torch_cuda, lib, kw):
    """GMRES as the inner solver on convergent problems: FP32 CUDA-core matvec
    (Nc = 19) and the 3xTF32 tensor-core matvec (Nc = 64, 128), restart 8."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    p = wl.random_tables(wl.small(**kw), seed=19, rel=0.2)
    S = dyson.setup(p)
    s = _solver(p)
    s.set_inner_solver(binding.INNER_GMRES, 8)
    sources = list(range(min(p.Nr, 3)))
    got, res = _solve(torch, s, p, sources, 1, tol=1e-13, max_sweeps=400)
    assert res.status == 0 and res.report["inner_gmres"] == 1
    ref = dyson.dense_solve(S, dyson.rhs_block_columns(S, sources))
    for q in range(len(sources)):
        assert _rel(got[q], ref[:, :, q * p.Nc:(q + 1) * p.Nc]) < 1e-12


def test_driven_32x32_sampled_columns_mixed_gmres(torch_cuda, lib):
    """32x32 lattice, driven, Nc = 384, one block column in mixed precision: the
    FP32 series cannot serve here (its partial sums peak ~2e7 above the result),
    so AUTO refines with GMRES.  Sampled vector columns against the oracle's
    complex128 GMRES (residual 1e-12)."""
    p = wl.driven_32x32_nc384()
    S = dyson.setup(p)
    s = _solver(p)
    src = 527
    got, res = _solve(torch_cuda, s, p, [src], 1, tol=1e-10, max_sweeps=400)
    assert res.status == 0 and res.report["inner_gmres"] == 1
    zs = [0, 159, 200, 330]
    B = dyson.rhs_vector_columns(S, [(src, z) for z in zs])
    ref, _, hist = dyson.gmres_solve(S, B, tol=1e-12, d_max=60, max_restarts=4)
    assert hist[-1] <= 1e-12
    for c, z in enumerate(zs):
        assert _rel(got[0][:, :, z], ref[:, :, c]) < 1e-7


def test_driven_32x32_sampled_columns_fp64(torch_cuda, lib):
    """32x32 lattice, driven, Nc = 384: one block column in FP64, sampled vector
    columns against the oracle's complex128 series run for the same 130 sweeps.

    On this contour the series' partial sums peak ~2e7 above the result, so
    either FP64 series carries amplified rounding (the update bottoms out near
    6e-10 after 130 sweeps and never reaches a 1e-12 tolerance), and
    NOT_CONVERGED is the expected status. Measured on a GB300, the GPU series
    and the oracle's differ by 2.6e-10, 3.7e-10, 5.6e-11 and 6.0e-12 at the four
    source times; they are compared at 2e-9.
    """
    p = wl.driven_32x32_nc384()
    S = dyson.setup(p)
    s = _solver(p)
    src = 527                                            # near the trap centre
    got, res = _solve(torch_cuda, s, p, [src], 0, tol=1e-15, max_sweeps=130, allow=(0, -3))
    assert res.report["sweeps"] == 130
    zs = [0, 159, 200, 330]                              # forward, backward, imaginary source times
    B = dyson.rhs_vector_columns(S, [(src, z) for z in zs])
    ref, _, _ = dyson.neumann_solve(S, B, tol=1e-16, max_sweeps=130)
    for c, z in enumerate(zs):
        assert _rel(got[0][:, :, z], ref[:, :, c]) < 2e-9


def test_trapped_16x16_sampled_columns_mixed(torch_cuda, lib):
    """16x16 lattice, Nc = 256, the benchmark's launch shape: sampled vector
    columns of two block columns against the oracle's complex128 series."""
    p = wl.trapped_16x16_nc256()
    S = dyson.setup(p)
    s = _solver(p)
    sources = [0, 119]                                       # a corner and a near-centre site
    got, res = _solve(torch_cuda, s, p, sources, 1, tol=1e-10, max_sweeps=300)
    rng = np.random.default_rng(3)
    cols = [(q, int(z)) for q in range(2) for z in rng.choice(p.Nc, 3, replace=False)]
    B = dyson.rhs_vector_columns(S, [(sources[q], z) for q, z in cols])
    ref, _, _ = dyson.neumann_solve(S, B, tol=1e-15, max_sweeps=400)
    assert dyson.residual(S, B, ref) < 1e-11
    for c, (q, z) in enumerate(cols):
        assert _rel(got[q][:, :, z], ref[:, :, c]) < 1e-6
    # densities of the source sites at all forward times
    n, _, _ = s.observables()
    i = sources[1]
    Bn = dyson.rhs_vector_columns(S, [(i, k) for k in range(p.Nt)])
    Gn, _, _ = dyson.neumann_solve(S, Bn, tol=1e-15, max_sweeps=400)
    n_ref = np.array([np.real(-1j * Gn[i, k, k]) for k in range(p.Nt)])
    assert np.abs(n[i] - n_ref).max() / np.abs(n_ref).max() < 1e-6


def test_trapped_16x16_bench_launch_shape_sampled_columns(torch_cuda, lib):
    """The benchmark's launch configuration on its workload: 16 block columns of the 16x16,
    Nc = 256 lattice in one chunk (the fused sweep on CTA pairs, as the tuner picks, support
    truncation on, the inner series from replayed graphs of 16 sweeps), mixed precision at
    the benchmark's tolerance 1e-6, sources 112..127 (one of its batches).  Sampled vector columns of four block columns, and the densities of two
    sources at three times, against the oracle's complex128 series; bound 1e-6 relative."""
    torch = torch_cuda
    from paper_1309_5994_gb300 import binding
    p = wl.trapped_16x16_nc256()
    S = dyson.setup(p)
    s = _solver(p)
    s.set_sweep_variant(binding.SWEEP_FUSED_PAIR)
    s.set_chunk(16)
    s.profile(True)
    sources = list(range(112, 128))
    g = torch.empty((len(sources), p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda:0")
    res = s.solve(sources, precision=binding.PREC_TF32X3_F64REF, tol=1e-6, max_sweeps=400, g_out=g)
    assert res.report["chunks"] == 1
    assert s.profile_query(binding.KERNEL_SWEEP_TC_FUSED)[0] > 0          # the fused sweep ran
    assert res.report["host_syncs"] < res.report["sweeps"]                 # from replayed graphs
    rng = np.random.default_rng(11)
    picks = [(q, int(z)) for q in (0, 5, 10, 15) for z in rng.choice(p.Nc, 2, replace=False)]
    dens = [(q, z) for q in (0, 7) for z in (0, p.Nt // 2, p.Nt - 1)]
    allp = picks + dens
    got = torch.stack([g[q, :, :, z] for q, z in allp], dim=-1).cpu().numpy()     # [Nr, Nc, columns]
    del g
    B = dyson.rhs_vector_columns(S, [(sources[q], z) for q, z in allp])
    ref, _, _ = dyson.neumann_solve(S, B, tol=1e-15, max_sweeps=400)
    assert dyson.residual(S, B, ref) < 1e-11
    k = len(picks)
    assert _rel(got[:, :, :k], ref[:, :, :k]) < 1e-6           # max-norm error relative to max |G|
    n, _, _ = s.observables()
    for c, (q, z) in enumerate(dens, start=len(picks)):
        i = sources[q]
        n_ref = np.real(-1j * ref[i, z, c])
        assert abs(n[i, z] - n_ref) < 1e-6 * abs(n_ref)
