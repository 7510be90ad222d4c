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


# ---- the blocked form of Sec. IV.D: one Krylov space for a block of right-hand sides ----

@pytest.mark.parametrize("kw", [CONVERGENT, DIVERGENT])
def test_block_gmres_equals_the_dense_solve(kw):
    """One block column (Nc right-hand sides at one site) and a block of scattered
    vector columns, also where the series diverges."""
    p = wl.random_tables(wl.small(**kw), seed=8, rel=0.1)
    S = dyson.setup(p)
    ref_fn = dyson.dense_solve
    for B in (dyson.rhs_block_columns(S, [1]), dyson.rhs_vector_columns(S, _cols(p))):
        G, its, hist = dyson.block_gmres_solve(S, B, tol=1e-13, d_max=8, max_restarts=10)
        ref = ref_fn(S, B)
        assert np.abs(G - ref).max() <= 1e-12 * np.abs(ref).max()
        assert hist[-1] <= 1e-13


def test_block_gmres_of_one_column_is_gmres():
    """With a block of one column the block Arnoldi process is the Arnoldi process: the
    same iterations and the same solution as the column-by-column GMRES."""
    p = wl.random_tables(wl.small(**CONVERGENT), seed=9, rel=0.1)
    S = dyson.setup(p)
    B = dyson.rhs_vector_columns(S, [(2, 3)])
    G1, its1, _ = dyson.block_gmres_solve(S, B, tol=1e-12, d_max=40)
    G2, its2, _ = dyson.gmres_solve(S, B, tol=1e-12, d_max=40)
    assert its1 == its2
    assert np.abs(G1 - G2).max() <= 1e-12 * np.abs(G2).max()


@pytest.mark.parametrize("d", [1, 2, 4])
def test_block_residual_never_exceeds_each_columns_gmres_at_equal_depth(d):
    """After d block steps the shared space B + span of (I-K)^k R0 (k < d, all columns
    of R0) contains every column's own affine Krylov space of depth d, so each
    column's minimal residual there is no larger than its own GMRES residual."""
    p = wl.random_tables(wl.small(L=4, Ly=3, Nt=10, Nm=6, trap_c=0.2, aU=0.1, aJ=0.2, omega=6.0), seed=10,
                         rel=0.1)
    S = dyson.setup(p)
    B = dyson.rhs_vector_columns(S, [(0, 1), (5, 4), (11, 12), (6, 20)])
    bnorm = np.sqrt((np.abs(B) ** 2).sum(axis=(0, 1)))

    def col_res(G):
        Z = B - (G - dyson.apply_K(S, G))
        return np.sqrt((np.abs(Z) ** 2).sum(axis=(0, 1))) / bnorm

    Gb, _, _ = dyson.block_gmres_solve(S, B, tol=0.0, d_max=d, max_restarts=0)
    Gc, _, _ = dyson.gmres_solve(S, B, tol=0.0, d_max=d, max_restarts=0)
    assert np.all(col_res(Gb) <= col_res(Gc) * (1 + 1e-9) + 1e-14)
