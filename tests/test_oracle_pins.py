"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: a brute-force
many-body trace, closed forms, an exact diagonalisation, exact invariances of
the discretised contour, or a continuum limit approached at the expected order.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as wl
from oracle import atomic, contour, dyson, lattice, observables


# ---------------------------------------------------------------------------
# atomic-limit function: brute-force trace over the 4-state Fock space
# ---------------------------------------------------------------------------

def fock_ops():
    """c_up, c_dn on the basis {|0>, |dn>, |up>, |up dn>} (Jordan-Wigner, up first)."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])     # annihilator on one mode
    Z = np.diag([1.0, -1.0])
    I = np.eye(2)
    # basis index = 2*n_up + n_dn  ->  mode order (up, dn)
    c_up = np.kron(a, I)
    c_dn = np.kron(Z, a)
    return c_up, c_dn


def brute_force_atomic(c, eps, U_t, beta):
    """-i Tr[rho T_C c(z) c^dag(z')] by explicit matrices; rho = exp(-beta H(0))/Z."""
    c_up, c_dn = fock_ops()
    n_up, n_dn = c_up.T @ c_up, c_dn.T @ c_dn

    def H(U):
        return eps * (n_up + n_dn) + U * (n_up @ n_dn)

    rho = sla.expm(-beta * H(U_t[0]))
    rho /= np.trace(rho)
    # evolution operator from 0 to each contour point
    Uop = []
    for z in range(c.Nc):
        if c.branch[z] == contour.IMAG:
            Uop.append(sla.expm(-(c.k[z] * c.dtau) * H(U_t[0])))   # exp(-tau H(0))
        else:
            M = np.eye(4, dtype=complex)
            for m in range(c.k[z]):                                 # prod_m exp(-i dt H(t_m))
                M = sla.expm(-1j * c.dt * H(U_t[m])) @ M
            Uop.append(M)
    Uinv = [np.linalg.inv(M) for M in Uop]
    cz = [Uinv[z] @ c_up @ Uop[z] for z in range(c.Nc)]
    cdz = [Uinv[z] @ c_up.T @ Uop[z] for z in range(c.Nc)]
    G = np.empty((c.Nc, c.Nc), dtype=complex)
    for z in range(c.Nc):
        for zp in range(c.Nc):
            if contour.later(c, z, zp):
                G[z, zp] = -1j * np.trace(rho @ cz[z] @ cdz[zp])
            else:
                G[z, zp] = +1j * np.trace(rho @ cdz[zp] @ cz[z])
    return G


@pytest.mark.parametrize("eps,U0,beta,drive", [(-4.0, 8.0, 1.0, False), (-2.5, 7.0, 0.7, True),
                                               (1.3, 3.0, 2.0, True)])
def test_atomic_matches_fock_space_trace(eps, U0, beta, drive):
    c = contour.make_contour(5, 4, 0.13, beta)
    t = np.arange(5) * 0.13
    U_t = U0 * (1.0 + (0.3 * np.sin(4.0 * t) if drive else np.zeros_like(t)))
    ref = brute_force_atomic(c, eps, U_t, beta)
    got = atomic.atomic_gf(c, eps, U_t, beta)
    assert np.abs(got - ref).max() < 1e-12


def test_atomic_equal_time_anticommutator_and_density():
    c = contour.make_contour(7, 6, 0.05, 1.5)
    eps, U0 = -3.0, 7.0
    Lam = atomic.atomic_gf(c, eps, np.full(7, U0), 1.5)
    n, D = atomic.atomic_density(eps, U0, 1.5)
    for k in range(c.Nt):
        zf, zb = k, 2 * c.Nt - 1 - k
        # {c, c^dag} = 1:  G^>(t,t) - G^<(t,t) = -i
        assert abs((Lam[zb, zf] - Lam[zf, zb]) - (-1j)) < 1e-14
        # density per spin = -i G(t, t+0) = rho_sigma + rho_d
        assert abs(-1j * Lam[zf, zf] - n) < 1e-14
    # particle-hole symmetric level eps = -U/2 gives half filling
    n_ph, _ = atomic.atomic_density(-U0 / 2, U0, 1.5)
    assert abs(n_ph - 0.5) < 1e-15


def test_atomic_double_occupancy_formula():
    """J = 0: App. B's difference quotient of the lesser function is
    Re[i sum_p b_p (1 - exp(i E_p dt))/dt] = sum_p b_p sin(E_p dt)/dt, so Eq. (docc)
    returns rho_d up to an O(dt^2) error (the O(dt) term is imaginary)."""
    eps, U0, beta = -4.0, 9.0, 1.0
    errs = []
    for dt in (0.02, 0.01, 0.005):
        p = wl.small(L=2, Nt=6, Nm=4, dt=dt, beta=beta, trap_c=0.0, U0=U0, J0=0.0, mu=-(eps + U0 / 2))
        S = dyson.setup(p)
        G = dyson.neumann_solve(S, dyson.rhs_block_columns(S, [0]))[0]
        n, ekin, D = observables.observables_block_column(S, 0, G)
        e = S.eps[0]
        _, lrs, lrd = atomic.boltzmann_log_weights(e, U0, beta)
        rs, rd = np.exp(lrs), np.exp(lrd)
        D_disc = (rs * np.sin(e * dt) / dt + rd * np.sin((e + U0) * dt) / dt - e * (rs + rd)) / U0
        assert np.abs(ekin).max() == 0.0
        assert np.abs(n - (rs + rd)).max() < 1e-14
        assert np.abs(D[1:] - D_disc).max() < 1e-12
        errs.append(np.abs(D[1:] - rd).max())
    assert 3.6 < errs[0] / errs[1] < 4.4 and 3.6 < errs[1] / errs[2] < 4.4


# ---------------------------------------------------------------------------
# the Dyson solve
# ---------------------------------------------------------------------------

def test_J0_gives_atomic_function():
    p = wl.small(L=3, J0=0.0)
    S = dyson.setup(p)
    B = dyson.rhs_block_columns(S, [0, 4])
    G, sweeps, _ = dyson.neumann_solve(S, B)
    assert sweeps == 1 and np.array_equal(G, B)


@pytest.mark.parametrize("L,Ly,seed", [(2, 2, 1), (3, 3, 2), (3, 2, 3)])
def test_series_matches_dense_inverse(L, Ly, seed):
    p = wl.random_tables(wl.small(L=L, Ly=Ly, Nt=6, Nm=4, aU=0.1, aJ=0.2, omega=6.0), seed=seed, rel=0.3)
    S = dyson.setup(p)
    B = dyson.rhs_block_columns(S, range(S.Nr))
    Gd = dyson.dense_solve(S, B)
    Gn, _, _ = dyson.neumann_solve(S, B, tol=1e-15)
    assert np.abs(Gd - Gn).max() < 1e-13
    assert dyson.residual(S, B, Gn) < 1e-13
    assert dyson.residual(S, B, Gd) < 1e-13


@pytest.mark.parametrize("Lx,Ly,drive", [(3, 3, False), (4, 3, True)])
def test_homogeneous_sine_basis_matches_dense(Lx, Ly, drive):
    kw = dict(aU=0.1, aJ=0.2, omega=6.0) if drive else {}
    p = wl.small(L=Lx, Ly=Ly, Nt=5, Nm=4, trap_c=0.0, **kw)
    S = dyson.setup(p)
    srcs = [0, Lx + 1]
    G = dyson.dense_solve(S, dyson.rhs_block_columns(S, srcs))
    pairs = [(j, i) for i in srcs for j in range(S.Nr)]
    H = dyson.homogeneous_solve(S, pairs)
    for q, i in enumerate(srcs):
        for j in range(S.Nr):
            assert np.abs(H[(j, i)] - G[j, :, q * S.Nc:(q + 1) * S.Nc]).max() < 1e-12


def _index_map(cA, cB):
    pos = {(cB.branch[z], cB.k[z]): z for z in range(cB.Nc)}
    return np.array([pos[(cA.branch[z], cA.k[z])] for z in range(cA.Nc)])


def test_result_independent_of_contour_end():
    """Contributions after max(t, t') cancel exactly between the real branches."""
    kw = dict(L=3, Nm=4, trap_c=0.4, aU=0.15, aJ=0.25, omega=5.0)
    SA = dyson.setup(wl.small(Nt=5, **kw))
    SB = dyson.setup(wl.small(Nt=9, **kw))
    GA = dyson.dense_solve(SA, dyson.rhs_block_columns(SA, [4]))
    GB = dyson.dense_solve(SB, dyson.rhs_block_columns(SB, [4]))
    mp = _index_map(SA.contour, SB.contour)
    assert np.abs(GA - GB[:, mp][:, :, mp]).max() < 1e-13


def test_c4v_symmetry_of_local_function():
    """The centred trap keeps the C4v point group (App. A): G_ii is equal on symmetry partners."""
    L = 4
    S = dyson.setup(wl.small(L=L, Nt=4, Nm=4, trap_c=0.4, aU=0.1, aJ=0.2, omega=5.0))
    x, y = lattice.site_xy(L, L)
    G = dyson.dense_solve(S, dyson.rhs_block_columns(S, range(S.Nr)))
    Nc = S.Nc
    Gloc = np.stack([G[i, :, i * Nc:(i + 1) * Nc] for i in range(S.Nr)])
    ops = [lambda a, b: (a, b), lambda a, b: (L - 1 - a, b), lambda a, b: (a, L - 1 - b),
           lambda a, b: (b, a), lambda a, b: (L - 1 - b, L - 1 - a), lambda a, b: (L - 1 - a, L - 1 - b),
           lambda a, b: (b, L - 1 - a), lambda a, b: (L - 1 - b, a)]
    for op in ops:
        for i in range(S.Nr):
            xx, yy = op(x[i], y[i])
            assert np.abs(Gloc[i] - Gloc[yy * L + xx]).max() < 1e-13


def test_free_fermions_fix_hopping_sign_and_kinetic_energy():
    """U = 0: the atomic function is a free level and G is the free-fermion function.

    The printed Dyson equation gives the free fermions of h = eps + J*A, with
    O(dt) error on the discretised contour; the kinetic energy read with the -i
    factor makes Eq. (docc) hold (dG/dt = eps n + ekin when U = 0).
    """
    L, beta, eps0 = 3, 1.0, 0.3
    errs, eom = [], []
    for dt, Nm in ((0.05, 16), (0.025, 32), (0.0125, 64)):
        Nt = int(round(0.5 / dt))
        p = wl.small(L=L, Nt=Nt, Nm=Nm, dt=dt, beta=beta, trap_c=0.0, U0=0.0, mu=-eps0)
        S = dyson.setup(p)
        i = 4
        G = dyson.dense_solve(S, dyson.rhs_block_columns(S, [i]))
        h = S.eps[0] * np.eye(L * L) + lattice.adjacency(L, L)
        w, V = np.linalg.eigh(h)
        f = V @ np.diag(1.0 / (1.0 + np.exp(beta * w))) @ V.T
        k = Nt // 2
        errs.append(np.abs(G[:, k, k] - 1j * f[i, :]).max())   # G^<_ji(t,t) = i <c_i^dag c_j>
        n, ekin, _ = observables.observables_block_column(S, i, G)
        kk = np.arange(1, Nt)
        dG = np.real((G[i][kk, kk] - G[i][kk - 1, kk]) / dt)
        eom.append(np.abs(dG - S.eps[i] * n[1:] - ekin[1:]).max())
        assert np.all(ekin < 0.0)      # thermal kinetic energy is negative
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2
    assert eom[0] / eom[2] > 6.0 and eom[2] < 2e-3


def _hubbard_one_matsubara(tau, beta, E1, E2, w1, w2, lam):
    """Continuum G_M(tau) = -<T c(tau) c^dag> of G(iw) = 1/(1/Lambda(iw) - lam), 0 < tau < beta."""
    # Lambda(x) = w1/(x-E1) + w2/(x-E2);  G = N/D with N = w1(x-E2)+w2(x-E1), D = (x-E1)(x-E2) - lam N
    Ncoef = np.array([w1 + w2, -(w1 * E2 + w2 * E1)])
    Dcoef = np.polysub(np.polymul([1.0, -E1], [1.0, -E2]), lam * Ncoef)
    roots = np.roots(Dcoef)
    dD = np.polyder(Dcoef)
    out = np.zeros_like(tau)
    for x in roots:
        x = np.real_if_close(x)
        r = np.polyval(Ncoef, x) / np.polyval(dD, x)
        out = out - np.real(r * np.exp(-tau * x) / (1.0 + np.exp(-beta * x)))
    return out


def test_matsubara_block_converges_to_continuum_hubbard_one():
    """The imaginary-branch block decouples exactly; its rectangle rule is first order in dtau."""
    L, beta, U0, eps = 3, 1.0, 6.0, -2.0
    errs = []
    for Nm in (32, 64, 128):
        p = wl.small(L=L, Nt=2, Nm=Nm, beta=beta, trap_c=0.0, U0=U0, mu=-(eps + U0 / 2))
        S = dyson.setup(p)
        i = 0
        H = dyson.homogeneous_solve(S, [(i, i)])[(i, i)]
        zi = 2 * S.contour.Nt + np.arange(1, Nm)            # tau_m, m >= 1, column tau' = 0
        got = np.real(H[zi, 2 * S.contour.Nt] / 1j)         # contour G = i G_M on the imaginary branch
        tau = np.arange(1, Nm) * (beta / Nm)
        lr0, lrs, lrd = atomic.boltzmann_log_weights(S.eps[0], U0, beta)
        w1, w2 = np.exp(lr0) + np.exp(lrs), np.exp(lrs) + np.exp(lrd)
        px, lx = dyson.sine_modes(L)
        ref = np.zeros_like(tau)
        for a in range(L):
            for b in range(L):
                ref += (px[0, a] * px[0, b]) ** 2 * _hubbard_one_matsubara(
                    tau, beta, S.eps[0], S.eps[0] + U0, w1, w2, lx[a] + lx[b])
        errs.append(np.abs(got - ref).max())
    assert errs[2] < 0.02
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def _equilibrium_and_anticommutator(dt, Nm, T=0.6):
    """On a 3x3 trapped lattice: (i) the spread over t of G_44(t + 0.2, t) without a drive,
    (ii) the largest deviation of G^>_ij(t, t) - G^<_ij(t, t) from -i delta_ij with a drive."""
    Nt = int(round(T / dt)) + 1
    lag = int(round(0.2 / dt))
    S = dyson.setup(wl.small(L=3, Nt=Nt, Nm=Nm, dt=dt, beta=1.0, trap_c=0.3, U0=8.0, J0=1.0))
    G = dyson.dense_solve(S, dyson.rhs_block_columns(S, [4]))
    vals = np.array([G[4, k + lag, k] for k in range(Nt - lag)])
    spread = np.abs(vals - vals[0]).max()
    S = dyson.setup(wl.small(L=3, Nt=Nt, Nm=Nm, dt=dt, beta=1.0, trap_c=0.3, U0=8.0, J0=1.0,
                             aU=0.2, aJ=0.3, omega=5.0))
    G = dyson.dense_solve(S, dyson.rhs_block_columns(S, range(S.Nr)))
    Nc, err = S.Nc, 0.0
    for k in range(Nt):
        zf, zb = k, 2 * Nt - 1 - k           # forward diagonal: lesser; backward diagonal: greater
        for j in range(S.Nr):
            d = G[:, zb, j * Nc + zb] - G[:, zf, j * Nc + zf]
            d[j] += 1j
            err = max(err, np.abs(d).max())
    return spread, err


def test_equilibrium_translation_invariance_and_equal_time_anticommutator():
    """Without a drive G(t + s, t) does not depend on t, and at equal times
    G^> - G^< = -i delta_ij (the canonical anticommutator), both of the continuum theory.
    On the discretised contour both hold to first order: the deviations fall by about 2
    when dt and dtau are halved (the translation invariance needs dtau refined as well: the
    imaginary branch carries the initial correlations)."""
    r = [_equilibrium_and_anticommutator(dt, Nm) for dt, Nm in ((0.1, 8), (0.05, 16), (0.025, 32))]
    spread = [x[0] for x in r]
    anti = [x[1] for x in r]
    assert spread[2] < 0.5 * spread[0] and spread[1] / spread[2] > 1.5
    assert 1.7 < anti[0] / anti[1] < 2.3 and 1.7 < anti[1] / anti[2] < 2.3


def test_kinetic_energy_second_order_term_is_that_of_exact_diagonalisation():
    """The lattice Dyson equation with Lambda alone is exact to first order in J for the
    off-diagonal G_ji (one hop between two atomic propagators), so the kinetic energy
    e_kin = Re[-i sum_j J_ij G_ji(t, t)] is exact at O(J^2).  On the Hubbard dimer (U = 4,
    beta = 1) its O(J^2) coefficient, extrapolated to dt -> 0 from three grids, equals
    J <c_1^+ c_2> / J^2 of exact diagonalisation to 1e-3 at every time of the equilibrium
    run.  This pins the hopping term of the solve, its contour weights and the sign and
    factor of the kinetic energy at U != 0."""
    from dimer_ed import dimer_fock, dimer_spectrum
    from oracle import extrapolate as ex
    U, beta, h, dt0, Nt0, Nm0 = 4.0, 1.0, 0.02, 0.1, 4, 4
    ms = (1, 2, 3)
    c2 = []
    for m in ms:
        p = wl.uniform_problem("dimer", 2, m * Nt0, m * Nm0, dt0 / m, beta, 0.0, 0.0, U, h, Ly=1)
        S = dyson.setup(p)
        G = dyson.dense_solve(S, dyson.rhs_block_columns(S, [0]))
        c2.append((observables.observables_block_column(S, 0, G)[1] / h ** 2)[::m][:Nt0])
    got = sum(w * c for w, c in zip(ex.weights_at_zero([1.0 / m for m in ms]), c2))
    c1u, _, c2u, _ = dimer_fock()
    _, _, rho, _ = dimer_spectrum(U, h, beta)
    exact = h * np.trace(rho @ c1u.T @ c2u) / h ** 2
    assert exact < 0 and np.abs(got - exact).max() < 1e-3 * abs(exact)
