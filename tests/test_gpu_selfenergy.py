"""Self-energy step (Sec. III, Eqs. (defnSigmatilde), (defnSigma); Sec. IV.C mixing loop) on the GPU
against the oracle."""
import numpy as np
import pytest

import workloads as wl
from oracle import dyson
from oracle import selfenergy as se

pytestmark = pytest.mark.gpu

DRIVEN = dict(L=3, Ly=2, Nt=7, Nm=5, dt=0.1, beta=1.0, U0=10.0, J0=1.0, trap_c=0.3, aU=0.1, aJ=0.2, omega=6.0)
SMALL = dict(L=2, Ly=2, Nt=4, Nm=3, dt=0.1, U0=8.0, J0=0.5, trap_c=0.2, aU=0.1, aJ=0.2, omega=5.0)


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


def _random_gloc(p, seed):
    rng = np.random.default_rng(seed)
    shape = (p.Nr, p.Nc, p.Nc)
    return 0.3 * (rng.normal(size=shape) + 1j * rng.normal(size=shape))


@pytest.mark.parametrize("kw", [DRIVEN, SMALL, dict(L=2, Ly=1, Nt=3, Nm=2, dt=0.2, beta=2.0, U0=6.0, J0=1.0)])
def test_sigma_tilde_and_local_block_match_the_oracle(torch_cuda, lib, kw):
    torch = torch_cuda
    p = wl.small(**kw)
    S = dyson.setup(p)
    gloc = _random_gloc(p, 5)
    s = _solver(p)
    out = torch.empty((p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda")
    s.selfenergy_step(torch.from_numpy(gloc).cuda(), mix=1.0, sigma_tilde=out)
    got = out.cpu().numpy()
    lam = s.sigma()
    for i in range(p.Nr):
        K = se.cumulant_sum(S.contour, S.eps[i], S.U[i], S.Lam[i])
        ref = se.sigma_tilde(S, K, gloc, i)
        assert np.abs(got[i] - ref).max() <= 1e-12 * np.abs(ref).max(), i
        B = se.local_block(S.Lam[i], ref, p.Nt)
        assert np.abs(lam[i] - B).max() <= 1e-10 * np.abs(B).max(), i


def test_sigma_tilde_vanishes_without_interaction(torch_cuda, lib):
    """U = 0: the connected two-particle part equals its disconnected (Wick) parts, so the
    contraction kernel and the GEMM terms cancel."""
    torch = torch_cuda
    p = wl.small(L=3, Ly=2, Nt=6, Nm=4, dt=0.1, U0=0.0, J0=1.0, trap_c=0.3)
    S = dyson.setup(p)
    gloc = _random_gloc(p, 6)
    s = _solver(p)
    out = torch.empty((p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda")
    s.selfenergy_step(torch.from_numpy(gloc).cuda(), mix=1.0, sigma_tilde=out)
    got = out.cpu().numpy()
    for i in range(p.Nr):
        F = se.hybridisation(S, gloc, i)
        scale = np.abs(S.Lam[i] @ F @ S.Lam[i]).max()
        assert np.abs(got[i]).max() <= 1e-13 * scale


def test_self_consistent_loop_matches_the_oracle(torch_cuda, lib):
    from paper_1309_5994_gb300.selfconsistency import self_consistent
    p = wl.small(**SMALL)
    blocks, St, Gloc, its, hist = se.self_consistent(p, mix=0.7, delta_sc=1e-11, max_iter=60)
    s = _solver(p)
    r = self_consistent(s, mix=0.7, delta_sc=1e-11, max_iter=60, precision=0, tol=1e-14)
    assert r["converged"] and abs(r["iterations"] - its) <= 1
    n = min(len(hist), len(r["history"]))
    h0, h1 = np.array(hist[:n - 2]), np.array(r["history"][:n - 2])
    assert np.all(np.abs(h1 - h0) <= 1e-6 * h0 + 1e-9)
    g = r["gloc"].cpu().numpy()
    assert np.abs(g - Gloc).max() <= 1e-9 * np.abs(Gloc).max()
    assert np.abs(s.sigma() - blocks).max() <= 1e-9 * np.abs(blocks).max()


def test_mixed_precision_loop_agrees_with_fp64(torch_cuda, lib):
    """Nc = 64 (the tensor-core sweeps and the split-product residual run on the installed blocks)."""
    from paper_1309_5994_gb300.selfconsistency import self_consistent
    p = wl.small(L=3, Ly=3, Nt=24, Nm=16, dt=0.05, beta=2.0, U0=20.0, J0=1.0, trap_c=0.05, aU=0.1, aJ=0.2,
                 omega=20.0)
    out = {}
    for prec, tol in ((0, 1e-13), (1, 1e-11)):
        s = _solver(p)
        s.profile(True)
        out[prec] = self_consistent(s, mix=0.7, delta_sc=1e-8, max_iter=40, precision=prec, tol=tol)
        if prec == 1:
            assert s.profile_query(2)[0] > 0 and s.profile_query(4)[0] > 0
        out[prec]["lam"] = s.sigma()
        s.close()
    assert out[0]["converged"] and out[1]["converged"]
    g0, g1 = out[0]["gloc"].cpu().numpy(), out[1]["gloc"].cpu().numpy()
    assert np.abs(g1 - g0).max() <= 1e-8 * np.abs(g0).max()
    assert np.abs(out[1]["lam"] - out[0]["lam"]).max() <= 1e-8 * np.abs(out[0]["lam"]).max()


def test_step_arguments_and_state(torch_cuda, lib):
    from paper_1309_5994_gb300 import binding
    torch = torch_cuda
    p = wl.small(**SMALL)
    s = binding.Solver(p, device=0)
    g = torch.zeros((p.Nr, p.Nc, p.Nc), dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.DysonError, match="STATE"):
        s.selfenergy_step(g)                                  # Lambda not built
    s.build_sigma()
    with pytest.raises(binding.DysonError, match="INVALID_ARG"):
        s.selfenergy_step(g, mix=0.0)
    s.selfenergy_step(torch.from_numpy(_random_gloc(p, 1)).cuda(), mix=0.7)
    with pytest.raises(binding.DysonError, match="STATE"):
        s.adjoint(np.ones(p.Nr))                              # the adjoint differentiates the atomic Lambda
    s.build_sigma()                                           # back to Sigma = 0
    S = dyson.setup(p)
    assert np.abs(s.sigma() - S.Lam).max() < 1e-13


@pytest.mark.parametrize("depth", [2, 5])
def test_anderson_mixing_reaches_the_same_fixed_point_sooner(torch_cuda, lib, depth):
    """Anderson acceleration (an addition to the paper's linear mixing) converges to the oracle's
    fixed point of the linear loop, in fewer iterations."""
    from paper_1309_5994_gb300.selfconsistency import self_consistent
    p = wl.small(**SMALL)
    blocks, St, Gloc, its, hist = se.self_consistent(p, mix=0.7, delta_sc=1e-11, max_iter=60)
    s = _solver(p)
    r = self_consistent(s, mix=0.7, delta_sc=1e-11, max_iter=60, precision=0, tol=1e-14, anderson=depth)
    assert r["converged"] and r["iterations"] < its
    g = r["gloc"].cpu().numpy()
    assert np.abs(g - Gloc).max() <= 1e-8 * np.abs(Gloc).max()
    assert np.abs(s.sigma() - blocks).max() <= 1e-8 * np.abs(blocks).max()


def test_anderson_depth_is_checked(torch_cuda, lib):
    from paper_1309_5994_gb300 import binding
    s = _solver(wl.small(**SMALL))
    with pytest.raises(binding.DysonError, match="INVALID_ARG"):
        s.set_anderson(7)
    s.set_anderson(0)


def test_sharded_loop_in_one_process_is_the_plain_loop(torch_cuda, lib):
    from paper_1309_5994_gb300.selfconsistency import self_consistent, self_consistent_sharded
    p = wl.small(**SMALL)
    a = self_consistent(_solver(p), mix=0.7, delta_sc=1e-10, max_iter=60, precision=0, tol=1e-14)
    b = self_consistent_sharded(_solver(p), mix=0.7, delta_sc=1e-10, max_iter=60, precision=0, tol=1e-14)
    assert a["iterations"] == b["iterations"] and np.allclose(a["history"], b["history"], rtol=1e-9, atol=0)
    assert torch_cuda.equal(a["gloc"], b["gloc"])


def test_c4v_loop_solves_one_site_per_orbit(torch_cuda, lib):
    """App. A inside the loop of Sec. IV.C: with a centred trap and a uniform drive the local
    Green's functions of one site per orbit (the others are copies, G_{g(r),g(r)} = G_{r,r})
    give the fixed point of the loop that solves every site, from 3 block columns per iteration
    instead of 9 on the 3x3 lattice (corners, edges, centre)."""
    from paper_1309_5994_gb300 import binding
    from paper_1309_5994_gb300.selfconsistency import self_consistent
    p = wl.small(L=3, Ly=3, Nt=6, Nm=4, dt=0.1, beta=1.0, U0=10.0, J0=1.0, trap_c=0.3, aU=0.1, aJ=0.2,
                 omega=6.0)
    out = {}
    for mode in (binding.SYMMETRY_NONE, binding.SYMMETRY_C4V):
        s = _solver(p)
        s.set_symmetry(mode)
        out[mode] = self_consistent(s, mix=0.7, delta_sc=1e-11, max_iter=60, precision=0, tol=1e-14)
        out[mode]["lam"] = s.sigma()
        s.close()
    a, b = out[binding.SYMMETRY_NONE], out[binding.SYMMETRY_C4V]
    assert a["converged"] and b["converged"] and abs(a["iterations"] - b["iterations"]) <= 1
    ga, gb = a["gloc"].cpu().numpy(), b["gloc"].cpu().numpy()
    assert np.abs(gb - ga).max() <= 1e-10 * np.abs(ga).max()
    assert np.abs(b["lam"] - a["lam"]).max() <= 1e-10 * np.abs(a["lam"]).max()
    fa = sum(r["gemm_flops"] for r in a["reports"]) / a["iterations"]
    fb = sum(r["gemm_flops"] for r in b["reports"]) / b["iterations"]
    assert fb < 0.45 * fa
    # one step from the same C4v-invariant G_loc: the contraction over the 3 representatives,
    # copied to their orbits, gives every site's Sigma~ of the full contraction
    torch = torch_cuda
    st = {}
    for mode in (binding.SYMMETRY_NONE, binding.SYMMETRY_C4V):
        s = _solver(p)
        s.set_symmetry(mode)
        st[mode] = torch.empty_like(b["gloc"])
        s.selfenergy_step(b["gloc"], mix=1.0, sigma_tilde=st[mode])
        s.close()
    s0, s1 = st[binding.SYMMETRY_NONE].cpu().numpy(), st[binding.SYMMETRY_C4V].cpu().numpy()
    assert np.abs(s0).max() > 1e-3
    assert np.abs(s1 - s0).max() <= 1e-12 * np.abs(s0).max()


def test_fixed_point_does_not_depend_on_where_the_real_branches_end(torch_cuda, lib):
    """Causality of the whole loop on the GPU: the self-consistent local Green's functions of a
    driven lattice with Nt = 4, restricted to their times, are those of the same lattice with
    Nt = 7 (contributions later than every external time cancel between the real branches in
    the lattice solve and in the cumulant contraction)."""
    from paper_1309_5994_gb300.selfconsistency import self_consistent
    kw = dict(SMALL)
    Nm = kw["Nm"]
    g = {}
    for Nt in (4, 7):
        kw["Nt"] = Nt
        s = _solver(wl.small(**kw))
        r = self_consistent(s, mix=0.7, delta_sc=1e-12, max_iter=80, precision=0, tol=1e-14)
        assert r["converged"]
        g[Nt] = r["gloc"].cpu().numpy()
        s.close()
    Ns, Nl = 4, 7
    ix = np.array(list(range(Ns)) + [2 * Nl - Ns + j for j in range(Ns)] + [2 * Nl + m for m in range(Nm)])
    assert np.abs(g[Nl][:, ix][:, :, ix] - g[Ns]).max() <= 1e-11 * np.abs(g[Ns]).max()
