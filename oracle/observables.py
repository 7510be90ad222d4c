"""Observables of Sec. III.A and App. B, read from one block column of G.

For source site i the block column G(:, i) holds G_ji(z, z') for every site j.
On the forward branch (contour index k = time t_k):

  n_i(t_k)     = Re[-i G_ii(z_k, z_k)]                       (density per spin, G(t, t+0))
  ekin_i(t_k)  = Re[-i sum_{j in NN(i)} J_ij(t_k) G_ji(z_k, z_k)]
  D_i(t_k)     = ( Re[(G_ii(z_k, z_k) - G_ii(z_{k-1}, z_k)) / dt]
                   - eps_i n_i(t_k) - ekin_i(t_k) ) / U_i(t_k),   k >= 1,

the last being Eq. (docc) with App. B's one-sided difference for the time
derivative.  D is not defined at k = 0 and is returned as NaN there.

Reading (sign of the hopping): the Dyson equation as printed, G = Lambda +
Lambda W J G, is the Green's function of the model with hopping +J; Eq. (model)
has -J.  On the bipartite square lattice the two are related by
c_i -> (-1)^(x_i+y_i) c_i, which leaves G_ii, n_i and D_i unchanged and flips
the sign of nearest-neighbour elements.  The kinetic-energy formula of
Sec. III.A is written for Eq. (model), so on the solved G it carries the factor
-i instead of +i; with it, Eq. (docc) holds for the solved G (checked in the
tests at U = 0, where the double-occupancy term drops out).

Parity: pinned at J = 0 (n = rho_s + rho_d, D at its exact discrete value) and at
U = 0 (the free-fermion densities and the equation of motion dG/dt = eps n + ekin,
both at first order in dt) in tests/test_oracle_pins.py, and at U, J != 0 by the
O(J^2) double occupancy of the self-consistent Hubbard dimer against exact
diagonalisation (tests/test_oracle_selfenergy.py).
"""
from __future__ import annotations

import numpy as np


def observables_block_column(S, i: int, Gcol: np.ndarray):
    """(n, ekin, D) for source site i from Gcol = G(:, i) of shape [Nr, Nc, Nc]."""
    c = S.contour
    Nt = c.Nt
    k = np.arange(Nt)                 # forward-branch contour indices are the time indices
    Gii = Gcol[i]
    g_eq = Gii[k, k]                  # G_ii(t_k, t_k+0)
    n = np.real(-1j * g_eq)
    acc = np.zeros(Nt, dtype=np.complex128)
    for j, b in S.nbrs[i]:
        acc += S.Jz[b][k] * Gcol[j][k, k]
    ekin = np.real(-1j * acc)
    D = np.full(Nt, np.nan)
    if Nt > 1:
        dG = (g_eq[1:] - Gii[k[1:] - 1, k[1:]]) / c.dt
        with np.errstate(divide="ignore", invalid="ignore"):   # U = 0 leaves D undefined
            D[1:] = (np.real(dG) - S.eps[i] * n[1:] - ekin[1:]) / S.U[i, 1:]
    return n, ekin, D


def observables(S, G_by_source: dict):
    """Stack observables for several sources; G_by_source maps site -> G(:, site)."""
    Nt = S.contour.Nt
    n = np.full((S.Nr, Nt), np.nan)
    ekin = np.full((S.Nr, Nt), np.nan)
    D = np.full((S.Nr, Nt), np.nan)
    for i, Gcol in G_by_source.items():
        n[i], ekin[i], D[i] = observables_block_column(S, i, Gcol)
    return n, ekin, D


def observables_from_pairs(S, i: int, pairs: dict):
    """Same as observables_block_column but from a dict {(j, i): G_ji} (homogeneous solver)."""
    Nr, Nc = S.Nr, S.Nc
    Gcol = np.zeros((Nr, Nc, Nc), dtype=np.complex128)
    for (j, ii), g in pairs.items():
        if ii == i:
            Gcol[j] = g
    return observables_block_column(S, i, Gcol)
