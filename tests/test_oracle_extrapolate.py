"""Pins of the oracle's Delta t -> 0 extrapolation (Sec. IV.D) against things other than itself."""
import numpy as np
import pytest

import workloads as wl
from oracle import extrapolate as ex


def test_richardson_weights_are_the_textbook_values():
    """Steps h, h/2, h/4: the quadratic fit at 0 is (f_h - 6 f_{h/2} + 8 f_{h/4}) / 3; the linear
    fit through h, h/2 is 2 f_{h/2} - f_h."""
    assert np.allclose(ex.weights_at_zero([0.1, 0.05, 0.025]), [1 / 3, -2.0, 8 / 3], rtol=0, atol=1e-14)
    assert np.allclose(ex.weights_at_zero([0.1, 0.05]), [-1.0, 2.0], rtol=0, atol=1e-14)
    assert ex.weights_at_zero([0.3]) == pytest.approx([1.0])


@pytest.mark.parametrize("ms", [(1, 2, 4), (1, 3, 5), (1, 2)])
def test_polynomial_data_is_reproduced_exactly(ms):
    """A polynomial of degree len(ms) - 1 in the step is extrapolated to its constant term."""
    rng = np.random.default_rng(3)
    Nt0, h0 = 7, 0.1
    coef = rng.normal(size=(len(ms), 5, Nt0))
    vals = []
    for m in ms:
        h = h0 / m
        on_coarse = sum(coef[d] * h ** d for d in range(len(ms)))
        f = np.full((5, m * (Nt0 - 1) + 1 + 3), np.nan)        # longer grid: extra points are ignored
        f[:, : m * (Nt0 - 1) + 1 : m] = on_coarse
        vals.append(f)
    out = ex.extrapolate(vals, h0, ms, Nt0)
    assert np.abs(out - coef[0]).max() <= 1e-12 * np.abs(coef[0]).max()


def test_refined_grid_keeps_the_final_time_and_the_drive():
    p = wl.small(L=2, Ly=2, Nt=9, Nm=4, dt=0.1, aU=0.1, aJ=0.2, omega=5.0)
    q = wl.refine(p, 4)
    assert (q.Nt, q.Nm, q.dt, q.Nc) == (36, 16, 0.025, 4 * p.Nc)
    assert np.array_equal(q.U[:, ::4], p.U) and np.array_equal(q.J[:, ::4], p.J)


def test_points_past_the_coarse_grid_leave_the_observables_unchanged():
    """The refined grid runs m - 1 points past the coarse grid's last time; by the t_max
    independence of the contour the observables at the coarse times are those of a grid
    that stops there."""
    p = wl.small(L=2, Ly=2, Nt=6, Nm=4, dt=0.1, aU=0.1, aJ=0.2, omega=5.0)
    q = wl.refine(p, 2)
    short = wl.uniform_problem("short", 2, 2 * p.Nt - 1, 2 * p.Nm, p.dt / 2, p.beta, p.mu, p.trap_c, 8.0, 1.0,
                               Ly=2, aU=0.1, aJ=0.2, omega=5.0)
    a = ex.observables_dense(q)
    b = ex.observables_dense(short)
    for x, y in zip(a, b):
        assert np.allclose(x[:, : short.Nt], y, rtol=0, atol=1e-12, equal_nan=True)


def test_extrapolated_observables_converge_at_third_order():
    """The raw observables of a driven 2x2 lattice carry a first-order step error (successive
    differences halve with the step); the quadratic extrapolation from (h, h/2, h/4) removes the
    first two orders, so its successive differences fall by ~8 per halving, the linear one's by ~4."""
    p0 = wl.small(L=2, Ly=2, Nt=9, Nm=4, dt=0.1, beta=1.0, trap_c=0.3, U0=8.0, J0=1.0,
                  aU=0.1, aJ=0.2, omega=5.0)
    ms = (1, 2, 4, 8, 16)
    raw = {m: [ex.on_coarse_times(f, m, p0.Nt)[:, 1:] for f in ex.observables_dense(wl.refine(p0, m))]
           for m in ms}
    for q in range(3):                                     # n, ekin, D (D undefined at t = 0)
        f = {m: raw[m][q] for m in ms}
        d = [np.abs(f[m] - f[2 * m]).max() for m in (1, 2, 4, 8)]
        if q < 2:
            assert 1.8 < d[2] / d[3] < 2.8                 # first order
        quad = [sum(w * f[m] for w, m in zip(ex.weights_at_zero([1 / a, 1 / (2 * a), 1 / (4 * a)]),
                                             (a, 2 * a, 4 * a))) for a in (1, 2, 4)]
        lin = [sum(w * f[m] for w, m in zip(ex.weights_at_zero([1 / a, 1 / (2 * a)]), (a, 2 * a)))
               for a in (2, 4, 8)]
        rq = np.abs(quad[0] - quad[1]).max() / np.abs(quad[1] - quad[2]).max()
        rl = np.abs(lin[0] - lin[1]).max() / np.abs(lin[1] - lin[2]).max()
        assert rq > 6.0 and 3.0 < rl < 5.5
        assert np.abs(quad[1] - quad[2]).max() < 0.25 * d[3]
