"""Discretised Kadanoff-Baym-Keldysh contour (Sec. IV.A and Fig. 1).

The paper fixes only N_t = 2*N_real + N_imag and a first-order time step error;
the grid below is this project's reading of it:

* forward branch, contour indices 0..Nt-1, physical time t_k = k*dt (k = index);
* backward branch, indices Nt..2Nt-1, index Nt+q carries time t_{Nt-1-q};
* imaginary branch, indices 2Nt..2Nt+Nm-1, tau_m = m*dtau, dtau = beta/Nm,
  attached at t = 0 (the Fig. 1 caption identifies the attachment point with t = 0).

Contour order is index order.  Quadrature weights are the left rectangle rule
of the contour measure dz: +dt forward, -dt backward, -i*dtau imaginary.

Parity: the grid, the weights and the equal-point order are pinned through what
they produce: the brute-force atomic trace, the exact independence of the
contour end, and the first-order approach of the lattice function to the
continuum sum rules (tests/test_oracle_pins.py).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FWD, BWD, IMAG = 0, 1, 2


@dataclass
class Contour:
    Nt: int
    Nm: int
    dt: float
    beta: float
    branch: np.ndarray   # [Nc] int: FWD / BWD / IMAG
    k: np.ndarray        # [Nc] int: real-time index on FWD/BWD, imaginary index m on IMAG
    W: np.ndarray        # [Nc] complex128 quadrature weights

    @property
    def Nc(self) -> int:
        return 2 * self.Nt + self.Nm

    @property
    def dtau(self) -> float:
        return self.beta / self.Nm


def make_contour(Nt: int, Nm: int, dt: float, beta: float) -> Contour:
    Nc = 2 * Nt + Nm
    branch = np.empty(Nc, dtype=np.int64)
    k = np.empty(Nc, dtype=np.int64)
    W = np.empty(Nc, dtype=np.complex128)
    for z in range(Nc):
        if z < Nt:
            branch[z], k[z], W[z] = FWD, z, dt
        elif z < 2 * Nt:
            branch[z], k[z], W[z] = BWD, 2 * Nt - 1 - z, -dt
        else:
            branch[z], k[z], W[z] = IMAG, z - 2 * Nt, -1j * (beta / Nm)
    return Contour(Nt, Nm, dt, beta, branch, k, W)


def later(c: Contour, z: int, zp: int) -> bool:
    """True when z lies after zp on the contour.

    Equal points follow the equal-time reading of G(t, t+0): a diagonal element
    is 'lesser' (c^dagger later) on the forward and imaginary branches and
    'greater' on the backward branch.  With this choice the contributions of
    contour points later than max(t, t') cancel exactly between the two real
    branches, so results do not depend on where the real branches end.
    """
    if z != zp:
        return z > zp
    return c.branch[z] == BWD
