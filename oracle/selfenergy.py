"""Self-energy step of the strong-coupling expansion (Sec. III, Eqs. (selfcons),
(defnSigma), (defnSigmatilde); Sec. IV.C, Eq. (Sigmamix) and the convergence rule).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
leg use this module.

Everything is the plain definition written out, for small contours (the
two-particle function is an [Nc]^4 tensor):

* two-particle function of the isolated site, by explicit 4 x 4 Fock-space
  matrices (basis {|0>, |dn>, |up>, |up dn>}) and Heisenberg operators on the
  discretised contour,
      G2_{s s1}(1, 2; 1', 2') = (-i)^2 Tr[rho T_C c_s(1) c_s1(2) c+_s1(1') c+_s(2')],
  rho = exp(-beta H_0(0)) / Z;
* its cumulant (the second-order one of Sec. III),
      G2~_{s s1} = G2_{s s1} + G(1,1') G(2,2') delta_{s s1} - G(1,2') G(2,1'),
  summed over the spin s1 of the neighbour:  K(a, b; c, d) = sum_{s1} G2~_{s s1}(a, b; c, d);
* Eq. (defnSigmatilde) on the contour quadrature (weights W, hopping J(z) as in
  the Dyson solve):
      F_i(c, b)       = sum_{j in NN(i)} W_c J_ij(c) Gloc_j(c, b) J_ji(b) W_b,
      Sigma~_i(a, d)  = - sum_{b, c} K_i(a, b; c, d) F_i(c, b);
* Eq. (defnSigma) with contour products and inverses: Sigma = G0^-1 * Sigma~ * G0^-1,
  and the local Dyson equation B = G0 + G0 * Sigma * B gives the block that
  replaces Lambda_i = G0_i in the lattice solve; with matrices,
      B_i = G0_i (G0_i - Sigma~_i)^-1 G0_i,
  which needs no inverse of G0 (see the readings for the turning points);
* the self-consistency loop of Sec. IV.C: Sigma = lambda Sigma_new + (1 - lambda)
  Sigma_old (Sigma is linear in Sigma~, so the mixing acts on Sigma~), converged
  when N_bd^-1 |dSigma~|_F + |dSigma~|_max <= delta_sc (N_bd the number of
  block-diagonal entries).

Readings (the paper does not fix them):
* The turning points of the discretised contour: the last forward and the first
  backward point carry one time (G0 has equal columns there, right null vector
  v = e_{Nt-1} - e_{Nt}), and so do the last backward and the first imaginary
  point (equal rows, left null vector u = e_{2Nt-1} - e_{2Nt}); Sigma~ has the
  same equal columns and rows.  G0 - Sigma~ is therefore singular too, and B is
  formed as G0 (G0 - Sigma~ + u v^T / 2)^-1 G0, which does not depend on the
  filled-in direction (B is the same for any such rank-one completion, and it
  equals (I - G0 T)^-1 G0 with T = G0^+ Sigma~ G0^+, the pseudo-inverse form of
  W Sigma W).  The continuum G0 is invertible; on long real-time branches its
  matrix also has one singular value that falls exponentially with the branch
  length (the zero of the atomic Green's function between its two levels), so
  forming Sigma itself amplifies rounding, and the convergence measure of
  Sec. IV.C is taken on Sigma~ (delta_sc = 1e-8 by default).
* T_C order on the discretised contour is index order; at one contour point,
  creators count as later than annihilators on the forward and imaginary
  branches and as earlier on the backward branch (the equal-time reading of the
  two-point function, contour.later); two operators of one kind at one point keep
  their order in the product (the fermionic sign makes the choice immaterial).
* The spin s of the self-energy is up (paramagnetic: both spins are equal).

Parity: the two-particle machinery is pinned by the atomic two-point function
(its closed form, atomic.atomic_gf), Wick's theorem at U = 0 (the cumulant
vanishes at every point, coincident ones included), the exchange antisymmetry of
G2 and the equal-point value rho_d; B_i by the local Dyson equation; and the
whole step (cumulant, contraction, local block, loop) by physics: on the Hubbard
dimer the O(J^2) term of the self-consistent local Green's function, extrapolated
to dtau, dt -> 0, is that of exact diagonalisation on the imaginary branch and on
the real-time branch (G^>(t, 0)), which the lattice Dyson equation without
self-energy misses; and the self-consistent fixed point restricted to the times
of a shorter contour is that of the shorter contour to rounding, the discrete
causality that a wrong branch order or weight would break; and under a drive the
self-consistent particle number sum_i n_i(t) becomes constant as dt -> 0, which
Lambda alone does not give (tests/test_oracle_selfenergy.py).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.linalg as sla

from . import dyson
from .contour import BWD, IMAG, Contour


# ---------------------------------------------------------------------------
# Fock space of one site
# ---------------------------------------------------------------------------

def fock_ops():
    """c_up, c_dn on {|0>, |dn>, |up>, |up dn>} (index 2 n_up + n_dn, Jordan-Wigner with up first)."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    return np.kron(a, I), np.kron(Z, a)


def _evolutions(c: Contour, eps: float, U_t: np.ndarray):
    """U(z) from 0 to each contour point and its inverse: prod_m exp(-i dt H(t_m)) on the
    real branches (left rule), exp(-tau H(0)) on the imaginary branch."""
    c_up, c_dn = fock_ops()
    n_up, n_dn = c_up.T @ c_up, c_dn.T @ c_dn

    def H(U):
        return eps * (n_up + n_dn) + U * (n_up @ n_dn)

    Uop = []
    for z in range(c.Nc):
        if c.branch[z] == IMAG:
            Uop.append(sla.expm(-(c.k[z] * c.dtau) * H(U_t[0])))
        else:
            M = np.eye(4, dtype=complex)
            for m in range(c.k[z]):
                M = sla.expm(-1j * c.dt * H(U_t[m])) @ M
            Uop.append(M)
    rho = sla.expm(-c.beta * H(U_t[0]))
    rho = rho / np.trace(rho)
    return np.array(Uop), np.array([np.linalg.inv(M) for M in Uop]), rho


def _heisenberg(O, Uop, Uinv):
    """O(z) = U(z)^-1 O U(z) for every contour point: [Nc, 4, 4]."""
    return np.einsum("zij,jk,zkl->zil", Uinv, O, Uop)


def _priority(c: Contour, creator: bool) -> np.ndarray:
    """1 where an operator of this kind counts as later at its own contour point."""
    bwd = c.branch == BWD
    return (~bwd if creator else bwd).astype(np.int64)


def tc_product(c: Contour, rho, ops):
    """(-i)^n... without the prefactor: Tr[rho T_C O_1(z_1) ... O_4(z_4)] for every (z_1..z_4).

    ops: four (O(z) array [Nc,4,4], is_creator) in product order.  Returns [Nc]^4."""
    Nc = c.Nc
    z = np.arange(Nc)
    keys = []
    for k, (_, cre) in enumerate(ops):
        key = (2 * z + _priority(c, cre)) * 4 + (3 - k)      # larger = later; ties keep product order
        shape = [1, 1, 1, 1]
        shape[k] = Nc
        keys.append(key.reshape(shape))
    keys = np.broadcast_arrays(*keys)
    out = np.zeros((Nc,) * 4, dtype=complex)
    for perm in itertools.permutations(range(4)):
        # perm: operator indices from latest (leftmost) to earliest
        mask = np.ones((Nc,) * 4, dtype=bool)
        for u in range(3):
            mask &= keys[perm[u]] > keys[perm[u + 1]]
        if not mask.any():
            continue
        inv = sum(1 for x in range(4) for y in range(x + 1, 4) if perm[x] > perm[y])
        sign = -1.0 if inv % 2 else 1.0
        X = [ops[perm[u]][0] for u in range(4)]
        # Tr[rho X1(z_p1) X2(z_p2) X3(z_p3) X4(z_p4)] over all index tuples
        M1 = np.einsum("ij,pjk->pik", rho, X[0])
        M2 = np.einsum("pik,qkl->pqil", M1, X[1])
        M3 = np.einsum("pqil,rlm->pqrim", M2, X[2])
        val = np.einsum("pqrim,smi->pqrs", M3, X[3])       # indices in the order of perm
        # back to (z_1, z_2, z_3, z_4) of the product order
        val = np.transpose(val, np.argsort(perm))
        out[mask] = sign * val[mask]
    return out


def two_point(c: Contour, eps: float, U_t: np.ndarray):
    """-i Tr[rho T_C c_up(z) c+_up(z')] from the same Fock-space machinery: [Nc, Nc]."""
    Uop, Uinv, rho = _evolutions(c, eps, U_t)
    c_up, _ = fock_ops()
    A = _heisenberg(c_up, Uop, Uinv)
    Ad = _heisenberg(c_up.T, Uop, Uinv)
    z = np.arange(c.Nc)
    ka = (2 * z + _priority(c, False)) * 2 + 1
    kc = (2 * z + _priority(c, True)) * 2
    later = ka[:, None] > kc[None, :]
    aa = np.einsum("ij,ajk,bki->ab", rho, A, Ad)            # Tr[rho c(a) c+(b)]
    cc = np.einsum("ij,bjk,aki->ab", rho, Ad, A)            # Tr[rho c+(b) c(a)]
    return -1j * np.where(later, aa, -cc)


def two_particle(c: Contour, eps: float, U_t: np.ndarray, same_spin: bool):
    """G2_{up s1}(a, b; c, d) = (-i)^2 Tr[rho T_C c_up(a) c_s1(b) c+_s1(c) c+_up(d)], [Nc]^4."""
    Uop, Uinv, rho = _evolutions(c, eps, U_t)
    c_up, c_dn = fock_ops()
    c_s1 = c_up if same_spin else c_dn
    ops = [(_heisenberg(c_up, Uop, Uinv), False), (_heisenberg(c_s1, Uop, Uinv), False),
           (_heisenberg(c_s1.T, Uop, Uinv), True), (_heisenberg(c_up.T, Uop, Uinv), True)]
    return -tc_product(c, rho, ops)                         # (-i)^2 = -1


def cumulant_sum(c: Contour, eps: float, U_t: np.ndarray, G0=None):
    """K(a, b; c, d) = sum_{s1} G2~_{up s1}(a, b; c, d) (the cumulant of Sec. III summed over s1)."""
    if G0 is None:
        G0 = two_point(c, eps, U_t)
    K = two_particle(c, eps, U_t, True) + two_particle(c, eps, U_t, False)
    K = K + np.einsum("ac,bd->abcd", G0, G0)                # delta_{s s1}: only s1 = s
    K = K - 2.0 * np.einsum("ad,bc->abcd", G0, G0)          # both spins s1
    return K


# ---------------------------------------------------------------------------
# Eqs. (defnSigmatilde), (defnSigma) and the local block
# ---------------------------------------------------------------------------

def hybridisation(S, Gloc: np.ndarray, i: int) -> np.ndarray:
    """F_i(c, b) = sum_{j in NN(i)} W_c J_ij(c) Gloc_j(c, b) J_ji(b) W_b."""
    W = S.contour.W
    F = np.zeros((S.Nc, S.Nc), dtype=complex)
    for j, b in S.nbrs[i]:
        wj = W * S.Jz[b]
        F += wj[:, None] * Gloc[j] * wj[None, :]
    return F


def sigma_tilde(S, K: np.ndarray, Gloc: np.ndarray, i: int) -> np.ndarray:
    """Sigma~_i(a, d) = - sum_{b, c} K_i(a, b; c, d) F_i(c, b)."""
    return -np.einsum("abcd,cb->ad", K, hybridisation(S, Gloc, i))


def weighted_sigma(G0: np.ndarray, St: np.ndarray) -> np.ndarray:
    """T = W Sigma W = G0^+ Sigma~ G0^+ (the contour inverse read with the pseudo-inverse)."""
    Gp = np.linalg.pinv(G0, rcond=1e-12)
    return Gp @ St @ Gp


def sigma_contour(S, G0: np.ndarray, St: np.ndarray) -> np.ndarray:
    """Sigma = W^-1 G0^+ Sigma~ G0^+ W^-1 (only where G0 is well conditioned)."""
    Wi = 1.0 / S.contour.W
    return Wi[:, None] * weighted_sigma(G0, St) * Wi[None, :]


def turning_vectors(Nt: int, Nc: int):
    """u = (e_{2Nt-1} - e_{2Nt}) / sqrt 2, v = (e_{Nt-1} - e_{Nt}) / sqrt 2."""
    u = np.zeros(Nc)
    v = np.zeros(Nc)
    u[2 * Nt - 1], u[2 * Nt] = 1.0, -1.0
    v[Nt - 1], v[Nt] = 1.0, -1.0
    return u / np.sqrt(2.0), v / np.sqrt(2.0)


def local_block(G0: np.ndarray, St: np.ndarray, Nt: int) -> np.ndarray:
    """B = G0 (G0 - Sigma~ + u v^T)^-1 G0, the solution of the local Dyson equation B = G0 + G0 * Sigma * B."""
    u, v = turning_vectors(Nt, G0.shape[0])
    return G0 @ np.linalg.solve(G0 - St + np.outer(u, v), G0)


def local_greens(S, blocks: np.ndarray) -> np.ndarray:
    """Gloc_j = G_jj of the lattice solve G = B + B W J G (dense), for every site: [Nr, Nc, Nc]."""
    S2 = dyson.Setup(S.Lx, S.Ly, S.contour, S.eps, S.U, S.Jz, blocks, S.nbrs)
    G = dyson.dense_solve(S2, dyson.rhs_block_columns(S2, range(S.Nr)))
    return np.stack([G[j, :, j * S.Nc:(j + 1) * S.Nc] for j in range(S.Nr)])


def self_consistent(p, mix: float = 0.7, delta_sc: float = 1e-8, max_iter: int = 40):
    """The loop of Sec. IV.C.  Returns (blocks B_i, mixed Sigma~ per site, the last Gloc,
    iterations, history of the measure)."""
    S = dyson.setup(p)
    G0 = S.Lam
    Ks = [cumulant_sum(S.contour, S.eps[i], S.U[i], G0[i]) for i in range(S.Nr)]
    St = np.zeros_like(G0)
    blocks = G0.copy()
    hist = []
    n_bd = S.Nr * S.Nc * S.Nc
    for it in range(1, max_iter + 1):
        Gloc = local_greens(S, blocks)
        St_new = np.stack([sigma_tilde(S, Ks[i], Gloc, i) for i in range(S.Nr)])
        d = St_new - St
        crit = np.sqrt((np.abs(d) ** 2).sum()) / n_bd + np.abs(d).max()
        hist.append(float(crit))
        St = mix * St_new + (1.0 - mix) * St                  # Eq. (Sigmamix); Sigma_old = 0 at the start
        blocks = np.stack([local_block(G0[i], St[i], p.Nt) for i in range(S.Nr)])
        if crit <= delta_sc:
            break
    return blocks, St, Gloc, it, hist
