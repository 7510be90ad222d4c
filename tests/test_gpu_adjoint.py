"""Vector-column solves, transposed (row) solves and the adjoint gradients on the GPU."""
import numpy as np
import pytest

import workloads as wl
from oracle import adjoint, dyson

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


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [
    dict(L=3, Ly=2, Nt=7, Nm=5, trap_c=0.3, aU=0.1, aJ=0.2, omega=6.0),       # Nc = 19: CUDA-core paths
    dict(L=2, Ly=3, Nt=24, Nm=16, trap_c=0.3, U0=20.0, aU=0.1, aJ=0.2, omega=20.0),   # Nc = 64: tensor cores
    dict(L=3, Ly=2, Nt=40, Nm=48, trap_c=0.2, U0=16.0, aU=0.1, aJ=0.2, omega=20.0),   # Nc = 128: CTA pairs
]


@pytest.mark.parametrize("kw", CASES)
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("transposed", [False, True])
def test_vector_columns_and_rows_match_dense(torch_cuda, lib, kw, prec, transposed):
    p = wl.random_tables(wl.small(**kw), seed=13, rel=0.2)
    S = dyson.setup(p)
    rng = np.random.default_rng(5)
    n = 37                                                   # two groups of 32, the second padded
    sites = rng.integers(0, p.Nr, n)
    times = rng.integers(0, p.Nc, n)
    if transposed:
        S = adjoint.transposed_setup(S)
    ref = dyson.dense_solve(S, dyson.rhs_vector_columns(S, list(zip(sites, times))))
    s = _solver(p)
    s.set_sweep_variant(1)                                   # the CTA-pair form where Nc allows it
    if transposed:
        s.transpose_sigma()
    g = torch_cuda.empty((n, p.Nr, p.Nc), dtype=torch_cuda.complex128, device="cuda:0")
    s.solve_vectors(sites, times, precision=prec, tol=1e-13, g_out=g)
    got = g.cpu().numpy()
    for q in range(n):
        assert _rel(got[q], ref[:, :, q]) < 1e-12
    if transposed:
        from paper_1309_5994_gb300 import binding
        with pytest.raises(binding.DysonError) as e:
            s.solve([0])
        assert e.value.code == -7                            # block columns need the upright Lambda
        s.transpose_sigma()
        s.solve([0])


@pytest.mark.parametrize("kw", CASES)
def test_adjoint_matches_oracle(torch_cuda, lib, kw):
    p = wl.random_tables(wl.small(**kw), seed=17, rel=0.15)
    w = np.random.default_rng(3).uniform(0, 1, p.Nr)
    L, gU, gJ = adjoint.gradients(p, w)
    s = _solver(p)
    for prec in (0, 1):
        Lg, gUg, gJg, res = s.adjoint(w, precision=prec, tol=1e-13)
        assert abs(Lg - L) < 1e-12 * max(1.0, abs(L))
        assert np.abs(gUg - gU).max() < 1e-10 * max(1.0, np.abs(gU).max())
        assert np.abs(gJg - gJ).max() < 1e-10 * max(1.0, np.abs(gJ).max())


@pytest.mark.parametrize("kw", CASES[:2])
def test_density_and_double_occupancy_adjoint_matches_oracle(torch_cuda, lib, kw):
    """L = sum_i w_i n_i(t) + v_i D_i(t) at an inner forward time: loss and
    gradients against the oracle's adjoint, FP64 and mixed paths."""
    p = wl.random_tables(wl.small(**kw), seed=29, rel=0.15)
    rng = np.random.default_rng(6)
    w, v = rng.uniform(0, 1, p.Nr), rng.uniform(0, 1, p.Nr)
    kf = p.Nt - 2
    L, gU, gJ = adjoint.obs_gradients(p, w=w, v=v, t_index=kf)
    s = _solver(p)
    for prec in (0, 1):
        Lg, gUg, gJg, res = s.adjoint_obs(w, v, t_index=kf, precision=prec, tol=1e-13)
        assert abs(Lg - L) < 1e-11 * max(1.0, abs(L))
        assert np.abs(gUg - gU).max() < 1e-9 * max(1.0, np.abs(gU).max())
        assert np.abs(gJg - gJ).max() < 1e-9 * max(1.0, np.abs(gJ).max())
    # double occupancies alone
    Ld, gUd, gJd = adjoint.obs_gradients(p, v=v, t_index=kf)
    Lg, gUg, gJg, _ = s.adjoint_obs(None, v, t_index=kf, precision=1, tol=1e-13)
    assert abs(Lg - Ld) < 1e-11 * max(1.0, abs(Ld))
    assert np.abs(gUg - gUd).max() < 1e-9 * max(1.0, np.abs(gUd).max())


def test_double_occupancy_amplitude_gradient_matches_finite_differences(torch_cuda, lib):
    """Drive amplitude s (reading 12): d/ds of sum_i v_i D_i(t_final) from the GPU
    adjoint through the chain rule against central differences of the GPU loss."""
    kw = dict(L=2, Ly=3, Nt=24, Nm=16, dt=0.05, trap_c=0.3, U0=20.0, aU=0.1, aJ=0.2, omega=20.0)
    v = np.random.default_rng(12).uniform(0, 1, 6)
    base = wl.small(**kw, amp=1.0)
    s = _solver(base)
    _, gU, gJ, _ = s.adjoint_obs(None, v, precision=1, tol=1e-13)
    dU, dJ = wl.drive_derivative_tables(base)
    chain = float(np.sum(gU * dU) + np.sum(gJ * dJ))
    h = 1e-4
    vals = [_solver(wl.small(**kw, amp=a)).adjoint_obs(None, v, precision=1, tol=1e-13)[0] for a in (1 + h, 1 - h)]
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - chain) < 1e-6 * max(abs(fd), 1e-3), (fd, chain)


def test_autograd_amplitude_gradient(torch_cuda, lib):
    """The drive built from a torch scalar s: s.grad through torch.autograd equals
    the oracle's chain rule of its adjoint gradients."""
    torch = torch_cuda
    from paper_1309_5994_gb300.autograd import weighted_density
    kw = dict(L=2, Ly=3, Nt=24, Nm=16, dt=0.05, trap_c=0.3, U0=20.0, aU=0.1, aJ=0.2, omega=20.0)
    p = wl.small(**kw)
    w = np.random.default_rng(8).uniform(0, 1, p.Nr)
    s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    t = torch.arange(p.Nt, dtype=torch.float64) * p.dt
    U = (20.0 * (1 + 0.1 * s * torch.sin(20 * t))).expand(p.Nr, p.Nt)
    J = (1.0 - 0.2 * s * torch.sin(20 * t)).expand(p.Nb, p.Nt)
    L = weighted_density(U, J, p, w, precision=1, tol=1e-13)
    L.backward()
    Lo, gU, gJ = adjoint.gradients(wl.small(**kw, amp=1.0), w)
    dU, dJ = wl.drive_derivative_tables(wl.small(**kw, amp=1.0))
    assert abs(L.item() - Lo) < 1e-12
    assert abs(s.grad.item() - float(np.sum(gU * dU) + np.sum(gJ * dJ))) < 1e-10 * max(1.0, abs(s.grad.item()))


def test_driven_24x24_amplitude_gradient_matches_finite_differences(torch_cuda, lib):
    """24x24 lattice, Nc = 256, the 32x32 lattice's drive scaled by s: d/ds of
    sum_i w_i n_i(t_final) from the adjoint (chain rule through the U and J
    tables) against central differences with h = 1e-4, to 1e-5 relative."""
    w = wl.loss_weights()
    base = wl.driven_24x24_nc256(1.0)
    s = _solver(base)
    L0, gU, gJ, res = s.adjoint(w, precision=1, tol=1e-11)
    dU, dJ = wl.drive_derivative_tables(base)
    chain = float(np.sum(gU * dU) + np.sum(gJ * dJ))
    h = 1e-4
    vals = []
    for amp in (1.0 + h, 1.0 - h):
        sp = _solver(wl.driven_24x24_nc256(amp))
        vals.append(sp.adjoint(w, precision=1, tol=1e-11)[0])
        sp.close()
    fd = (vals[0] - vals[1]) / (2 * h)
    assert abs(fd - chain) < 1e-5 * max(abs(fd), 1e-3), (fd, chain)
    # one bond-time entry directly
    b, k = 300, 40
    Jp, Jm = base.J.copy(), base.J.copy()
    Jp[b, k] += 1e-3
    Jm[b, k] -= 1e-3
    lp = _solver(base.with_tables(J=Jp)).adjoint(w, precision=1, tol=1e-11)[0]
    lm = _solver(base.with_tables(J=Jm)).adjoint(w, precision=1, tol=1e-11)[0]
    fdJ = (lp - lm) / 2e-3
    assert abs(fdJ - gJ[b, k]) < 1e-5 * max(abs(fdJ), 1e-6) + 1e-9, (fdJ, gJ[b, k])
