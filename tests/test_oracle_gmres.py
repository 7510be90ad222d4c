"""Pins of the oracle's preconditioned GMRES (App. C) against things other than itself."""
import numpy as np
import pytest

import workloads as wl
from oracle import dyson

CONVERGENT = dict(L=3, Ly=2, Nt=7, Nm=5, trap_c=0.3, aU=0.1, aJ=0.2, omega=6.0)
DIVERGENT = dict(L=3, Ly=3, Nt=24, Nm=16, dt=0.05, beta=2.0, trap_c=0.0, U0=4.0, J0=2.0)   # rho(K) = 1.41


def _cols(p):
    return [(0, 0), (1, 3), (p.Lx * p.Ly - 1, p.Nt + 2), (2, p.Nt + p.Nt // 2)]


@pytest.mark.parametrize("kw", [CONVERGENT, DIVERGENT])
def test_gmres_equals_the_dense_solve(kw):
    """Also where the series of App. C diverges (spectral radius 1.41)."""
    p = wl.random_tables(wl.small(**kw), seed=6, rel=0.1)
    S = dyson.setup(p)
    B = dyson.rhs_vector_columns(S, _cols(p))
    G, its, hist = dyson.gmres_solve(S, B, tol=1e-13, d_max=30, max_restarts=10)
    ref = dyson.dense_solve(S, B)
    assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()
    assert hist[-1] <= 1e-13


def test_gmres_at_zero_hopping_returns_the_preconditioned_rhs():
    """J = 0: the residue z0 = K B vanishes, so u0 = P b = Lambda delta is exact with no iteration."""
    p = wl.small(L=2, Ly=2, Nt=5, Nm=4, J0=0.0)
    S = dyson.setup(p)
    B = dyson.rhs_vector_columns(S, [(1, 2), (3, 7)])
    G, its, _ = dyson.gmres_solve(S, B, tol=1e-14)
    assert its == 0 and np.array_equal(G, B)


@pytest.mark.parametrize("d", [1, 3, 6])
def test_gmres_residual_never_exceeds_the_series_at_equal_depth(d):
    """d GMRES steps search B + span(K B, ..., K^d B), the affine space of the
    series' partial sum after d sweeps, and minimise the residual there."""
    p = wl.random_tables(wl.small(**CONVERGENT), seed=8, rel=0.2)
    S = dyson.setup(p)
    B = dyson.rhs_vector_columns(S, _cols(p))
    Gg, its, _ = dyson.gmres_solve(S, B, tol=0.0, d_max=d, max_restarts=0)
    Gs, _, _ = dyson.neumann_solve(S, B, tol=0.0, max_sweeps=d)
    assert its == d

    def res2(G):
        R = B - (G - dyson.apply_K(S, G))
        return np.sqrt((np.abs(R) ** 2).sum(axis=(0, 1)))

    assert np.all(res2(Gg) <= res2(Gs) * (1 + 1e-10))
