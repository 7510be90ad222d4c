"""Delta t -> 0 extrapolation of contour results (Sec. IV.D).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
leg use this module.

The contour step enters every result of the discretised contour at first order
(left-rule phases and quadrature).  Sec. IV.D removes it by computing the same
observable at three step sizes, fitting a quadratic in the step and reading the
fit at step 0 (and cross-checks with the linear fit).  Written out: for steps
h_0 > h_1 > ... > h_{n-1} and values f_b, the polynomial of degree n - 1 through
the points (h_b, f_b), evaluated at 0, is the Lagrange sum

    f(0) = sum_b f_b L_b(0),   L_b(0) = prod_{c != b} h_c / (h_c - h_b).

Reading (the paper does not say how the grids are refined): step b divides the
coarsest step by an integer, h_b = h_0 / m_b, and refines the whole contour,
every branch with m_b times the points (workloads.refine); the real-time grid
then covers the coarse grid's times.  Results are compared at the coarsest
grid's times t_k = k h_0, which are index k m_b of grid b.

Parity: pinned by the textbook Richardson weights, by exactness on polynomial
data, and by the convergence order of extrapolated densities of a driven
lattice (tests/test_oracle_extrapolate.py).
"""
from __future__ import annotations

import numpy as np

from . import dyson
from .observables import observables


def weights_at_zero(h) -> np.ndarray:
    """L_b(0) for the steps h (distinct, positive)."""
    h = np.asarray(h, dtype=np.float64)
    w = np.ones(len(h))
    for b in range(len(h)):
        for c in range(len(h)):
            if c != b:
                w[b] *= h[c] / (h[c] - h[b])
    return w


def on_coarse_times(f: np.ndarray, m: int, Nt0: int) -> np.ndarray:
    """Samples t_k = k h_0, k = 0..Nt0-1, of an array [..., Nt_b] on grid h_0 / m."""
    if f.shape[-1] < m * (Nt0 - 1) + 1:
        raise ValueError("grid too short for the coarse times")
    return f[..., : m * (Nt0 - 1) + 1 : m]


def extrapolate(values, h0: float, ms, Nt0: int) -> np.ndarray:
    """Extrapolate values[b] ([..., Nt_b] on step h0 / ms[b]) to step 0 at the coarse times."""
    h = [h0 / m for m in ms]
    w = weights_at_zero(h)
    out = np.zeros(values[0].shape[:-1] + (Nt0,))
    for f, m, wb in zip(values, ms, w):
        out += wb * on_coarse_times(np.asarray(f, dtype=np.float64), m, Nt0)
    return out


def observables_dense(p, sources=None):
    """(n, ekin, D) [Nr, Nt] of p from dense solves of the block columns `sources` (default: all)."""
    S = dyson.setup(p)
    src = range(p.Nr) if sources is None else sources
    G = {}
    for s in src:
        B = dyson.rhs_block_columns(S, [s])
        G[s] = dyson.dense_solve(S, B)
    return observables(S, G)
