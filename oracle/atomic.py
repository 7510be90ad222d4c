"""Atomic-limit contour Green's function of one site (Sec. III).

Lambda_i(z, z') = -i <T_C c_{i sigma}(z) c^dagger_{i sigma}(z')> over H_0^(i)(t),
the single-site Hamiltonian eps_i n_up + eps_i n_dn + U_i(t) n_up n_dn, with the
thermal state of H_0^(i)(0) at inverse temperature beta (Sec. II).

In the particle-number basis {|0>, |down>, |up>, |up down>} the energies are
E_0 = 0, E_sigma = eps, E_d = 2 eps + U (Sec. III), and c_sigma(t) only picks up
the phases zeta_nu(t) = exp(i int_0^t E_nu) of Eq. (cumulanttabulation), since
H_0^(i)(t) commutes with itself at all times.  Removing one sigma particle
happens in two channels:

  p = 1:  |sigma>  -> |0>,        energy E_sigma - E_0 = eps
  p = 2:  |up dn>  -> |sigma-bar>, energy E_d - E_sigma = eps + U(t)

so that, with Phi_p(z) the integrated channel energy,

  Lambda(z, z') = -i sum_p exp(-i (Phi_p(z) - Phi_p(z'))) * ( a_p  if z later than z'
                                                             -b_p  otherwise )

with a_1 = rho_0, b_1 = rho_sigma, a_2 = rho_sigma, b_2 = rho_d, the Boltzmann
weights of Eq. (Z).  On the real branches Phi_p(t_k) = dt * sum_{m<k} E_p(t_m)
(left-rule tabulation of the phases); on the imaginary branch
Phi_p(-i tau) = -i tau E_p(0).

Parity: pinned by a brute-force 4-state trace over T_C-ordered products of the
Fock-space operators (tests), the anticommutator and density sum rules, and the
Matsubara weights.
"""
from __future__ import annotations

import numpy as np

from .contour import Contour, BWD, IMAG


def boltzmann_log_weights(eps0: float, U0: float, beta: float):
    """log rho_0, log rho_sigma (each spin), log rho_d of exp(-beta H_0(0)) / Z (Eq. Z)."""
    E = np.array([0.0, eps0, eps0, 2.0 * eps0 + U0])
    x = -beta * E
    xmax = x.max()
    logZ = xmax + np.log(np.exp(x - xmax).sum())
    return x[0] - logZ, x[1] - logZ, x[3] - logZ


def channel_phases(c: Contour, E_real: np.ndarray) -> np.ndarray:
    """Phi(z) for one channel whose energy on the real grid is E_real[k] = E(t_k)."""
    Phi = np.empty(c.Nc, dtype=np.complex128)
    cum = np.concatenate([[0.0], np.cumsum(E_real)[:-1]]) * c.dt  # dt * sum_{m<k} E(t_m)
    for z in range(c.Nc):
        if c.branch[z] == IMAG:
            Phi[z] = -1j * (c.k[z] * c.dtau) * E_real[0]
        else:
            Phi[z] = cum[c.k[z]]
    return Phi


def later_matrix(c: Contour) -> np.ndarray:
    """Boolean [Nc, Nc]: z later than z' (with the equal-point rule of contour.later)."""
    idx = np.arange(c.Nc)
    M = idx[:, None] > idx[None, :]
    M[idx, idx] = (c.branch == BWD)
    return M


def atomic_gf(c: Contour, eps: float, U_t: np.ndarray, beta: float) -> np.ndarray:
    """Lambda_i(z, z') as an [Nc, Nc] complex128 array.

    eps: the site's level eps_i; U_t: U_i(t_k) on the real grid (U_t[0] = U_i(0)).
    """
    U_t = np.asarray(U_t, dtype=np.float64)
    lr0, lrs, lrd = boltzmann_log_weights(eps, U_t[0], beta)
    E1 = np.full(c.Nt, eps)
    E2 = eps + U_t
    later = later_matrix(c)
    out = np.zeros((c.Nc, c.Nc), dtype=np.complex128)
    for E, la, lb in ((E1, lr0, lrs), (E2, lrs, lrd)):
        Phi = channel_phases(c, E)
        dPhi = Phi[:, None] - Phi[None, :]
        # weight * exp(-i dPhi) evaluated as exp(log weight - i dPhi) to keep
        # large imaginary-time exponents finite.
        out += np.where(later, np.exp(la - 1j * dPhi), -np.exp(lb - 1j * dPhi))
    return -1j * out


def atomic_gfs(c: Contour, eps: np.ndarray, U: np.ndarray, beta: float) -> np.ndarray:
    """Lambda for every site: [Nr, Nc, Nc]."""
    return np.stack([atomic_gf(c, eps[i], U[i], beta) for i in range(len(eps))])


def atomic_density(eps0: float, U0: float, beta: float):
    """(n_sigma, D) of the atomic thermal state: rho_sigma + rho_d and rho_d."""
    _, lrs, lrd = boltzmann_log_weights(eps0, U0, beta)
    return np.exp(lrs) + np.exp(lrd), np.exp(lrd)
