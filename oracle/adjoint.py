"""Gradients of weighted sums of site densities and double occupancies (no
counterpart in the paper; derived here).

Loss:   L = sum_i w_i n_i(t_f),  n_i(t_f) = Re[-i G_ii(z_f, z_f)],  z_f = forward point t_f.

From G = (I - K)^{-1} Lambda with K = Lambda W J, and (I - K)^{-1} = I + G W J:

    dG = (I + G W J) dLambda (I + W J G) + G W dJ G.

With the column c_i = G e_i and the row r_i^T = e_i^T G (e_i the unit vector at
(i, z_f)), gamma_i = e_i + W J c_i and rho_i^T = e_i^T + r_i^T W J,

    dL = sum_i w_i Re[-i (rho_i^T dLambda gamma_i + r_i^T W dJ c_i)].

A row of G solves the same equation with every Lambda_l transposed:
r_i = Lambda^T e_i + Lambda^T W J r_i.  Hence per bond b = (l, m) and time t_k
(contour points Z_k: the forward and backward points of t_k, and the imaginary
points when k = 0, where J takes its t = 0 value)

    dL/dJ_b(t_k) = sum_i w_i Re[-i sum_{z in Z_k} W(z) (r_i(l,z) c_i(m,z) + r_i(m,z) c_i(l,z))],

and per site l, with M_l = sum_i w_i gamma_i[l] rho_i[l]^T,

    dL/dU_l(t_k) = Re[-i sum_{z,z'} (dLambda_l/dU_l(t_k))(z,z') M_l(z',z)],

dLambda_l/dU_l(t_k) being the derivative of the closed form of Sec. III
(atomic_gf_dU).  Parity: pinned against central finite differences of the
loss (tests), which use only the forward oracle.
"""
from __future__ import annotations

import numpy as np

from .atomic import boltzmann_log_weights, channel_phases, later_matrix
from .contour import Contour, IMAG
from .dyson import Setup, dense_solve, neumann_solve, rhs_vector_columns, setup


def atomic_gf_dU(c: Contour, eps: float, U_t: np.ndarray, beta: float, k: int) -> np.ndarray:
    """d Lambda(z, z') / d U(t_k) of atomic.atomic_gf, eps = V - U(0)/2 - mu held as a
    function of U(0) (so k = 0 also moves eps, the Boltzmann weights and all phases)."""
    U_t = np.asarray(U_t, dtype=np.float64)
    lr0, lrs, lrd = boltzmann_log_weights(eps, U_t[0], beta)
    E1 = np.full(c.Nt, eps)
    E2 = eps + U_t
    later = later_matrix(c)
    m = np.where(c.branch == IMAG, 0, c.k)                 # real-time index of each point
    tau = np.where(c.branch == IMAG, c.k * c.dtau, 0.0)
    imag = c.branch == IMAG
    # d eps / d U(t_k) = -1/2 for k = 0
    deps = -0.5 if k == 0 else 0.0
    # d Phi_1(z): real dt*m*eps; imaginary -i tau eps
    dPhi1 = np.where(imag, -1j * tau * deps, c.dt * m * deps)
    # d Phi_2(z): real dt*sum_{j<m}(eps + U_j); imaginary -i tau (eps + U_0)
    dU0 = 1.0 if k == 0 else 0.0
    dPhi2 = np.where(imag, -1j * tau * (deps + dU0), c.dt * (m * deps + (m > k)))
    # Boltzmann weights: E = (0, eps, eps, 2 eps + U0)
    dE = np.array([0.0, deps, deps, 2 * deps + dU0])
    rho = np.exp(np.array([lr0, lrs, lrs, lrd]))
    dlogZ = -beta * np.dot(rho, dE)
    dl0, dls, dld = -beta * dE[0] - dlogZ, -beta * dE[1] - dlogZ, -beta * dE[3] - dlogZ
    out = np.zeros((c.Nc, c.Nc), dtype=np.complex128)
    for E, la, lb, dla, dlb, dPhi in ((E1, lr0, lrs, dl0, dls, dPhi1), (E2, lrs, lrd, dls, dld, dPhi2)):
        Phi = channel_phases(c, E)
        dP = Phi[:, None] - Phi[None, :]
        ddP = dPhi[:, None] - dPhi[None, :]
        term = np.where(later, np.exp(la - 1j * dP), -np.exp(lb - 1j * dP))
        dlog = np.where(later, dla, dlb) - 1j * ddP
        out += term * dlog
    return -1j * out


def loss(p, w, solver="dense") -> float:
    """L = sum_i w_i n_i(t_f), t_f the last forward point."""
    S = setup(p)
    zf = p.Nt - 1
    B = rhs_vector_columns(S, [(i, zf) for i in range(S.Nr)])
    G = dense_solve(S, B) if solver == "dense" else neumann_solve(S, B, tol=1e-15, max_sweeps=1000)[0]
    return float(sum(w[i] * np.real(-1j * G[i, zf, i]) for i in range(S.Nr)))


def transposed_setup(S: Setup) -> Setup:
    """The same problem with every site block Lambda_l transposed (rows of G)."""
    return Setup(S.Lx, S.Ly, S.contour, S.eps, S.U, S.Jz, np.ascontiguousarray(np.transpose(S.Lam, (0, 2, 1))),
                 S.nbrs)


def gradients(p, w, solver="dense"):
    """(L, dL/dU [Nr, Nt], dL/dJ [Nb, Nt]) by the adjoint formulas above."""
    S = setup(p)
    c = S.contour
    Nr, Nc, Nt = S.Nr, S.Nc, c.Nt
    zf = Nt - 1
    cols = [(i, zf) for i in range(Nr)]
    ST = transposed_setup(S)
    if solver == "dense":
        C = dense_solve(S, rhs_vector_columns(S, cols))            # C[:, :, i] = G e_i
        R = dense_solve(ST, rhs_vector_columns(ST, cols))          # R[:, :, i] = G^T e_i
    else:
        C = neumann_solve(S, rhs_vector_columns(S, cols), tol=1e-15, max_sweeps=1000)[0]
        R = neumann_solve(ST, rhs_vector_columns(ST, cols), tol=1e-15, max_sweeps=1000)[0]
    L = float(sum(w[i] * np.real(-1j * C[i, zf, i]) for i in range(Nr)))
    W = c.W
    # points carrying each real time index, imaginary points for k = 0
    Zk = [[z for z in range(Nc) if (c.branch[z] != IMAG and c.k[z] == k) or (k == 0 and c.branch[z] == IMAG)]
          for k in range(Nt)]
    gJ = np.zeros((len(S.Jz), Nt))
    from .lattice import bond_list
    for b, (l, m) in enumerate(bond_list(S.Lx, S.Ly)):
        for k in range(Nt):
            z = np.array(Zk[k])
            val = 0.0 + 0.0j
            for i in range(Nr):
                val += w[i] * np.sum(W[z] * (R[l, z, i] * C[m, z, i] + R[m, z, i] * C[l, z, i]))
            gJ[b, k] = np.real(-1j * val)
    # gamma_i[l](z) = delta_il delta_{z zf} + W(z) sum_m J_lm(z) c_i(m, z);  rho_i[l] likewise with r_i
    gU = np.zeros((Nr, Nt))
    for l in range(Nr):
        gam = np.zeros((Nc, Nr), dtype=np.complex128)
        rho = np.zeros((Nc, Nr), dtype=np.complex128)
        for m_, b in S.nbrs[l]:
            gam += (W * S.Jz[b])[:, None] * C[m_]
            rho += (W * S.Jz[b])[:, None] * R[m_]
        gam[zf, l] += 1.0
        rho[zf, l] += 1.0
        M = (gam * w[None, :]) @ rho.T                               # M_l = sum_i w_i gamma_i rho_i^T
        for k in range(Nt):
            dLam = atomic_gf_dU(c, S.eps[l], S.U[l], c.beta, k)
            gU[l, k] = np.real(-1j * np.sum(dLam * M.T))
    return L, gU, gJ


# ----------------------------------------------------------------------------
# densities and double occupancies: L = sum_i w_i n_i(t_f) + v_i D_i(t_f)
# ----------------------------------------------------------------------------
#
# Both observables of Sec. III.A / Eq. (docc) at the forward time t_f are
# real-linear in the column c_i = G e_(i, z_f) (z_f the forward point of t_f):
#   n_i = Im c_i(i, z_f),
#   D_i = [ (Re c_i(i, z_f) - Re c_i(i, z_f - 1)) / dt - eps_i n_i
#           - Im sum_j J_ij(t_f) c_i(j, z_f) ] / U_i(t_f),
# so L = sum_i Re(beta_i . c_i) with a sparse complex weight vector beta_i, and
#   dL = sum_i Re(beta_i . dG e_i) + (explicit terms of D)
# with beta_i . dG e_i = rho_i^T dLambda gamma_i + psi_i^T W dJ c_i, where
# psi_i = sum_a beta_ia r_a (rows of G at the entries a of beta_i),
# rho_i = beta_i + W J psi_i and gamma_i = e_i + W J c_i.  The explicit terms:
# dD_i/dU_i(t_f) = -D_i / U_i(t_f); through eps_i = V - U_i(0)/2 - mu,
# dD_i/dU_i(0) = n_i / (2 U_i(t_f)); through e_kin,
# dD_i/dJ_ij(t_f) = -Im c_i(j, z_f) / U_i(t_f).

def _obs_weights(S: Setup, w, v, kf):
    """beta_i as {(site, point): coefficient} for every i."""
    dt, zf = S.contour.dt, kf
    out = []
    for i in range(S.Nr):
        b = {}
        def add(key, val):
            b[key] = b.get(key, 0.0) + val
        if w is not None and w[i] != 0.0:
            add((i, zf), -1j * w[i])                            # Im x = Re(-i x)
        if v is not None and v[i] != 0.0:
            Ui = S.U[i, kf]
            add((i, zf), v[i] / (dt * Ui))
            add((i, zf - 1), -v[i] / (dt * Ui))
            add((i, zf), v[i] * 1j * S.eps[i] / Ui)             # -eps Im x = Re(i eps x)
            for j, bnd in S.nbrs[i]:
                add((j, zf), v[i] * 1j * S.Jz[bnd][zf] / Ui)     # -J Im x = Re(i J x)
        out.append(b)
    return out


def obs_loss(p, w=None, v=None, t_index=None) -> float:
    """L = sum_i w_i n_i(t_f) + v_i D_i(t_f) from the dense forward solve (t_f >= 1)."""
    S = setup(p)
    kf = p.Nt - 1 if t_index is None else t_index
    C = dense_solve(S, rhs_vector_columns(S, [(i, kf) for i in range(S.Nr)]))
    dt = S.contour.dt
    L = 0.0
    for i in range(S.Nr):
        c = C[:, :, i]
        n = np.imag(c[i, kf])
        if w is not None:
            L += w[i] * n
        if v is not None:
            ekin = np.imag(sum(S.Jz[b][kf] * c[j, kf] for j, b in S.nbrs[i]))
            D = ((np.real(c[i, kf]) - np.real(c[i, kf - 1])) / dt - S.eps[i] * n - ekin) / S.U[i, kf]
            L += v[i] * D
    return float(L)


def obs_gradients(p, w=None, v=None, t_index=None):
    """(L, dL/dU [Nr, Nt], dL/dJ [Nb, Nt]) of L = sum_i w_i n_i(t_f) + v_i D_i(t_f)."""
    S = setup(p)
    c = S.contour
    Nr, Nc, Nt = S.Nr, S.Nc, c.Nt
    kf = Nt - 1 if t_index is None else t_index
    assert 1 <= kf < Nt
    betas = _obs_weights(S, w, v, kf)
    C = dense_solve(S, rhs_vector_columns(S, [(i, kf) for i in range(Nr)]))
    ST = transposed_setup(S)
    keys = sorted({key for b in betas for key in b})
    Rk = dense_solve(ST, rhs_vector_columns(ST, keys))             # rows of G at the weighted entries
    col = {key: n for n, key in enumerate(keys)}
    Psi = np.zeros((Nr, Nc, Nr), dtype=np.complex128)
    for i, b in enumerate(betas):
        for key, val in b.items():
            Psi[:, :, i] += val * Rk[:, :, col[key]]
    L = float(sum(np.real(sum(val * C[a, z, i] for (a, z), val in b.items())) for i, b in enumerate(betas)))
    W = c.W
    Zk = [[z for z in range(Nc) if (c.branch[z] != IMAG and c.k[z] == k) or (k == 0 and c.branch[z] == IMAG)]
          for k in range(Nt)]
    from .lattice import bond_list
    bonds = bond_list(S.Lx, S.Ly)
    gJ = np.zeros((len(bonds), Nt))
    for bnd, (l, m) in enumerate(bonds):
        for k in range(Nt):
            z = np.array(Zk[k])
            val = np.sum(W[z][:, None] * (Psi[l, z, :] * C[m, z, :] + Psi[m, z, :] * C[l, z, :]))
            gJ[bnd, k] = np.real(val)
    gU = np.zeros((Nr, Nt))
    for l in range(Nr):
        gam = np.zeros((Nc, Nr), dtype=np.complex128)
        rho = np.zeros((Nc, Nr), dtype=np.complex128)
        for m_, bnd in S.nbrs[l]:
            gam += (W * S.Jz[bnd])[:, None] * C[m_]
            rho += (W * S.Jz[bnd])[:, None] * Psi[m_]
        gam[kf, l] += 1.0
        for i, b in enumerate(betas):
            for (a, z), val in b.items():
                if a == l:
                    rho[z, i] += val
        M = gam @ rho.T                                              # M_l = sum_i gamma_i rho_i^T
        for k in range(Nt):
            dLam = atomic_gf_dU(c, S.eps[l], S.U[l], c.beta, k)
            gU[l, k] = np.real(np.sum(dLam * M.T))
    # explicit dependence of D on U(t_f), U(0) (through eps) and J(t_f)
    if v is not None:
        dt = c.dt
        bond_of = {}
        for bnd, (l, m) in enumerate(bonds):
            bond_of[(l, m)] = bond_of[(m, l)] = bnd
        for i in range(Nr):
            if v[i] == 0.0:
                continue
            ci = C[:, :, i]
            n = np.imag(ci[i, kf])
            ekin = np.imag(sum(S.Jz[b][kf] * ci[j, kf] for j, b in S.nbrs[i]))
            Ui = S.U[i, kf]
            D = ((np.real(ci[i, kf]) - np.real(ci[i, kf - 1])) / dt - S.eps[i] * n - ekin) / Ui
            gU[i, kf] += v[i] * (-D / Ui)
            gU[i, 0] += v[i] * n / (2.0 * Ui)
            for j, b in S.nbrs[i]:
                gJ[b, kf] += v[i] * (-np.imag(ci[j, kf]) / Ui)
    return L, gU, gJ
