"""Pins of the oracle's adjoint gradients against central finite differences."""
import numpy as np
import pytest

import workloads as wl
from oracle import adjoint, atomic, contour


@pytest.mark.parametrize("k", [0, 1, 3])
def test_atomic_derivative_matches_finite_differences(k):
    c = contour.make_contour(5, 4, 0.07, 1.3)
    U = 9.0 * (1 + 0.2 * np.sin(3.0 * np.arange(5) * 0.07))
    V, mu = 0.4, 0.1

    def lam(Uv):
        return atomic.atomic_gf(c, V - Uv[0] / 2 - mu, Uv, 1.3)

    h = 1e-5
    Up, Um = U.copy(), U.copy()
    Up[k] += h
    Um[k] -= h
    fd = (lam(Up) - lam(Um)) / (2 * h)
    an = adjoint.atomic_gf_dU(c, V - U[0] / 2 - mu, U, 1.3, k)
    assert np.abs(fd - an).max() < 1e-8 * max(1.0, np.abs(an).max())


def _problem():
    p = wl.small(L=3, Ly=2, Nt=5, Nm=4, dt=0.1, trap_c=0.3, U0=8.0, aU=0.1, aJ=0.2, omega=6.0)
    return wl.random_tables(p, seed=4, rel=0.15)


def test_adjoint_gradients_match_finite_differences():
    p = _problem()
    w = np.random.default_rng(2).uniform(0, 1, p.Nr)
    L, gU, gJ = adjoint.gradients(p, w)
    assert abs(L - adjoint.loss(p, w)) < 1e-13
    h = 1e-5
    for (l, k) in [(0, 0), (2, 1), (4, 3), (5, 4)]:
        Up, Um = p.U.copy(), p.U.copy()
        Up[l, k] += h
        Um[l, k] -= h
        fd = (adjoint.loss(p.with_tables(U=Up), w) - adjoint.loss(p.with_tables(U=Um), w)) / (2 * h)
        assert abs(fd - gU[l, k]) < 1e-7 * max(1.0, abs(fd)), (l, k, fd, gU[l, k])
    for (b, k) in [(0, 0), (3, 2), (6, 4)]:
        Jp, Jm = p.J.copy(), p.J.copy()
        Jp[b, k] += h
        Jm[b, k] -= h
        fd = (adjoint.loss(p.with_tables(J=Jp), w) - adjoint.loss(p.with_tables(J=Jm), w)) / (2 * h)
        assert abs(fd - gJ[b, k]) < 1e-7 * max(1.0, abs(fd)), (b, k, fd, gJ[b, k])


def test_amplitude_gradient_is_the_chain_rule():
    """d/ds of the scaled drive (U and J modulations times s) equals sum(gU dU/ds) + sum(gJ dJ/ds)."""
    def make(s):
        return wl.small(L=2, Ly=2, Nt=6, Nm=4, dt=0.05, trap_c=0.2, U0=20.0, aU=0.1, aJ=0.2, omega=20.0, amp=s)

    w = np.array([0.3, 0.9, 0.5, 0.1])
    p = make(1.0)
    _, gU, gJ = adjoint.gradients(p, w)
    dU, dJ = wl.drive_derivative_tables(p)
    chain = float(np.sum(gU * dU) + np.sum(gJ * dJ))
    h = 1e-4
    fd = (adjoint.loss(make(1.0 + h), w) - adjoint.loss(make(1.0 - h), w)) / (2 * h)
    assert abs(fd - chain) < 1e-6 * max(1.0, abs(fd))


def test_density_and_double_occupancy_gradients_match_finite_differences():
    """L = sum_i w_i n_i(t_f) + v_i D_i(t_f): the generalised adjoint (rows of G at
    the entries D reads, plus D's explicit dependence on U(t_f), U(0) and J(t_f))
    against central differences of the forward observables; with v = 0 it is the
    density adjoint exactly."""
    p = _problem()
    rng = np.random.default_rng(2)
    w, v = rng.uniform(0, 1, p.Nr), rng.uniform(0, 1, p.Nr)
    L0, gU0, gJ0 = adjoint.gradients(p, w)
    L1, gU1, gJ1 = adjoint.obs_gradients(p, w=w)
    assert abs(L0 - L1) < 1e-14 and np.abs(gU0 - gU1).max() < 1e-15 and np.abs(gJ0 - gJ1).max() < 1e-15
    kf = 3
    L, gU, gJ = adjoint.obs_gradients(p, w=w, v=v, t_index=kf)
    assert abs(L - adjoint.obs_loss(p, w, v, kf)) < 1e-13
    h = 1e-5
    for (l, k) in [(0, 0), (2, 1), (4, kf), (1, kf), (5, 4)]:
        Up, Um = p.U.copy(), p.U.copy()
        Up[l, k] += h
        Um[l, k] -= h
        fd = (adjoint.obs_loss(p.with_tables(U=Up), w, v, kf) - adjoint.obs_loss(p.with_tables(U=Um), w, v, kf)) / (2 * h)
        assert abs(fd - gU[l, k]) < 1e-7 * max(1.0, abs(fd)), (l, k, fd, gU[l, k])
    for (b, k) in [(0, 0), (3, 2), (6, kf), (2, kf)]:
        Jp, Jm = p.J.copy(), p.J.copy()
        Jp[b, k] += h
        Jm[b, k] -= h
        fd = (adjoint.obs_loss(p.with_tables(J=Jp), w, v, kf) - adjoint.obs_loss(p.with_tables(J=Jm), w, v, kf)) / (2 * h)
        assert abs(fd - gJ[b, k]) < 1e-7 * max(1.0, abs(fd)), (b, k, fd, gJ[b, k])
