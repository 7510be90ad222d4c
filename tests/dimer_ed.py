"""Exact diagonalisation of the Hubbard dimer (two sites, levels eps = -U/2, hopping J), the
independent reference of the oracle's physics pins: explicit 16 x 16 Fock-space matrices
(Jordan-Wigner), the thermal state exp(-beta H) / Z and Heisenberg operators in real and
imaginary time.  Test infrastructure only."""
import numpy as np


def dimer_fock():
    """c_1up, c_1dn, c_2up, c_2dn on the 16 states of two sites (Jordan-Wigner)."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    ops = []
    for k in range(4):
        m = np.array([[1.0]])
        for j in range(4):
            m = np.kron(m, Z if j < k else (a if j == k else I))
        ops.append(m)
    return ops


def dimer_spectrum(U, J, beta):
    """Eigenpairs of the Hubbard dimer (eps = -U/2, hopping J), its thermal state and c_1up."""
    c1u, c1d, c2u, c2d = dimer_fock()
    n = lambda c: c.T @ c
    H = -U / 2 * (n(c1u) + n(c1d) + n(c2u) + n(c2d)) + U * (n(c1u) @ n(c1d) + n(c2u) @ n(c2d))
    H = H + J * (c1u.T @ c2u + c2u.T @ c1u + c1d.T @ c2d + c2d.T @ c1d)
    w, V = np.linalg.eigh(H)
    w = w - w.min()
    rho = V @ np.diag(np.exp(-beta * w)) @ V.T
    return w, V, rho / np.trace(rho), c1u


def dimer_matsubara_exact(U, J, beta, taus):
    """-i <c_1up(tau) c_1up^+(0)> of the Hubbard dimer by exact diagonalisation."""
    w, V, rho, c = dimer_spectrum(U, J, beta)
    out = []
    for t in taus:
        c_t = V @ np.diag(np.exp(t * w)) @ V.T @ c @ V @ np.diag(np.exp(-t * w)) @ V.T
        out.append(-1j * np.trace(rho @ c_t @ c.T))
    return np.array(out)


def dimer_greater_exact(U, J, beta, ts):
    """G^>(t, 0) = -i <c_1up(t) c_1up^+(0)> of the Hubbard dimer by exact diagonalisation."""
    w, V, rho, c = dimer_spectrum(U, J, beta)
    out = []
    for t in ts:
        c_t = V @ np.diag(np.exp(1j * t * w)) @ V.T @ c @ V @ np.diag(np.exp(-1j * t * w)) @ V.T
        out.append(-1j * np.trace(rho @ c_t @ c.T))
    return np.array(out)
