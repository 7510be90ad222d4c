"""Trapped square lattice of Sec. II, Eq. (model) and Eq. (onsitelevels).

Sites i = y*Lx + x with open boundaries; the trap is V_trap(r) = c*|r|^2 about
the geometric centre of the lattice (Sec. V.A gives V_trap proportional to |r|^2);
eps_i = V_trap(r_i) - U_i(0)/2 - mu (Eq. onsitelevels).  Bonds are listed
horizontal first, then vertical.

Parity: the neighbour lists and levels are pinned by the open-boundary sine-mode
solve of homogeneous lattices and the exact C4v symmetry of G_ii in a centred
trap (tests/test_oracle_pins.py).
"""
from __future__ import annotations

import numpy as np


def site_xy(Lx: int, Ly: int):
    i = np.arange(Lx * Ly)
    return i % Lx, i // Lx


def bond_list(Lx: int, Ly: int):
    """[(i, j)] for every nearest-neighbour bond, in the documented bond order."""
    out = []
    for y in range(Ly):
        for x in range(Lx - 1):
            out.append((y * Lx + x, y * Lx + x + 1))
    for y in range(Ly - 1):
        for x in range(Lx):
            out.append((y * Lx + x, (y + 1) * Lx + x))
    return out


def neighbours(Lx: int, Ly: int):
    """For each site, the list of (neighbour site, bond index)."""
    nb = [[] for _ in range(Lx * Ly)]
    for b, (i, j) in enumerate(bond_list(Lx, Ly)):
        nb[i].append((j, b))
        nb[j].append((i, b))
    return nb


def trap_potential(Lx: int, Ly: int, c: float) -> np.ndarray:
    x, y = site_xy(Lx, Ly)
    rx = x - (Lx - 1) / 2.0
    ry = y - (Ly - 1) / 2.0
    return c * (rx * rx + ry * ry)


def onsite_levels(Lx: int, Ly: int, c: float, U0_site: np.ndarray, mu: float) -> np.ndarray:
    """eps_i of Eq. (onsitelevels) for a static trap; U0_site = U_i(t=0)."""
    return trap_potential(Lx, Ly, c) - 0.5 * U0_site - mu


def adjacency(Lx: int, Ly: int) -> np.ndarray:
    """Dense 0/1 nearest-neighbour matrix (for small-lattice checks)."""
    A = np.zeros((Lx * Ly, Lx * Ly))
    for i, j in bond_list(Lx, Ly):
        A[i, j] = A[j, i] = 1.0
    return A
