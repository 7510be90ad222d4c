"""Pins of the oracle's self-energy step (Sec. III, Eqs. (selfcons)-(defnSigmatilde)) against
facts fixed by the many-body definitions and by physics: the closed-form two-point function,
Wick's theorem, exchange antisymmetry, equal-point values, the local Dyson equation, and the
second-order term of the exactly diagonalised Hubbard dimer."""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import atomic, contour, dyson, observables
from oracle import extrapolate as ex
from oracle import selfenergy as se

from dimer_ed import dimer_fock, dimer_greater_exact, dimer_matsubara_exact, dimer_spectrum


@pytest.fixture(scope="module")
def grid():
    c = contour.make_contour(4, 3, 0.11, 1.3)
    U_t = 7.0 * (1.0 + 0.2 * np.sin(5.0 * np.arange(4) * 0.11))
    return c, U_t


def test_two_point_function_equals_the_closed_form(grid):
    """The Fock-space machinery that builds the two-particle function reproduces Lambda of Sec. III
    (itself pinned to a separate trace over T_C-ordered products)."""
    c, U_t = grid
    for eps in (-3.5, 0.7):
        assert np.abs(se.two_point(c, eps, U_t) - atomic.atomic_gf(c, eps, U_t, c.beta)).max() < 1e-13


@pytest.mark.parametrize("eps", [-1.3, 0.4])
def test_cumulant_vanishes_without_interaction(grid, eps):
    """U = 0: the site is non-interacting, Wick's theorem holds for every contour ordering
    (coincident points included), so the cumulant of both spin channels is zero."""
    c, _ = grid
    for same in (True, False):
        G0 = se.two_point(c, eps, np.zeros(c.Nt))
        G2 = se.two_particle(c, eps, np.zeros(c.Nt), same)
        wick = -np.einsum("ac,bd->abcd", G0, G0) * (1.0 if same else 0.0) + np.einsum("ad,bc->abcd", G0, G0)
        assert np.abs(G2 - wick).max() < 1e-14
    assert np.abs(se.cumulant_sum(c, eps, np.zeros(c.Nt))).max() < 1e-14


def test_cumulant_is_nonzero_with_interaction(grid):
    c, U_t = grid
    assert np.abs(se.cumulant_sum(c, -3.5, U_t)).max() > 0.05


def test_exchange_antisymmetry(grid):
    """Same spins: swapping the two annihilators or the two creators flips the sign."""
    c, U_t = grid
    G2 = se.two_particle(c, -3.5, U_t, True)
    assert np.abs(G2 + np.transpose(G2, (1, 0, 2, 3))).max() < 1e-15
    assert np.abs(G2 + np.transpose(G2, (0, 1, 3, 2))).max() < 1e-15
    # opposite spins: swapping both pairs at once exchanges the roles of the two spins,
    # which the paramagnetic site leaves unchanged
    G2o = se.two_particle(c, -3.5, U_t, False)
    assert np.abs(G2o - np.transpose(G2o, (1, 0, 3, 2))).max() < 1e-13


def test_equal_point_values_are_the_atomic_occupations(grid):
    """All four operators at one point: on the forward and imaginary branches the creators are
    later, the product is n_up n_dn and G2_{up dn} = (-i)^2 rho_d; on the backward branch the
    annihilators are later, the product is (1 - n_up)(1 - n_dn) and G2 = (-i)^2 rho_0."""
    c, U_t = grid
    eps = -2.9
    G2o = se.two_particle(c, eps, U_t, False)
    lr0, _, lrd = atomic.boltzmann_log_weights(eps, U_t[0], c.beta)
    for z in range(c.Nc):
        want = -np.exp(lr0) if c.branch[z] == contour.BWD else -np.exp(lrd)
        assert abs(G2o[z, z, z, z] - want) < 1e-14


def test_turning_points_make_the_atomic_matrix_singular():
    """The last forward and the first backward point carry one time, and so do the last backward
    and the first imaginary point: G0 has equal columns at the first pair and equal rows at the
    second, rank Nc - 1; Sigma~ has the same structure."""
    p = wl.small(L=2, Ly=1, Nt=5, Nm=4, dt=0.1, aU=0.1, aJ=0.2, omega=5.0)
    S = dyson.setup(p)
    G0 = S.Lam[0]
    Nt = p.Nt
    assert np.array_equal(G0[:, Nt - 1], G0[:, Nt]) and np.array_equal(G0[2 * Nt - 1], G0[2 * Nt])
    sv = np.linalg.svd(G0, compute_uv=False)
    assert sv[-1] < 1e-14 * sv[0] and sv[-2] > 0.1
    St = se.sigma_tilde(S, se.cumulant_sum(S.contour, S.eps[0], S.U[0], G0), S.Lam, 0)
    assert np.abs(St[:, Nt - 1] - St[:, Nt]).max() < 1e-15 and np.abs(St[2 * Nt - 1] - St[2 * Nt]).max() < 1e-15


def test_local_block_solves_the_local_dyson_equation():
    """B = G0 (G0 - Sigma~ + u v^T)^-1 G0 equals (I - G0 T)^-1 G0 with T = G0^+ Sigma~ G0^+, i.e. it
    satisfies B = G0 + G0 W Sigma W B with Sigma = W^-1 G0^+ Sigma~ G0^+ W^-1 (where G0 is well
    conditioned), and for an invertible G0 it is G0 (G0 - Sigma~)^-1 G0."""
    p = wl.small(L=2, Ly=1, Nt=5, Nm=4, dt=0.1, aU=0.1, aJ=0.2, omega=5.0)
    S = dyson.setup(p)
    G0 = S.Lam[0]
    St = se.sigma_tilde(S, se.cumulant_sum(S.contour, S.eps[0], S.U[0], G0), S.Lam, 0)
    B = se.local_block(G0, St, p.Nt)
    Sig = se.sigma_contour(S, G0, St)
    W = S.contour.W
    assert np.abs(B - G0 - G0 @ (W[:, None] * Sig * W[None, :]) @ B).max() < 1e-12 * np.abs(B).max()
    rng = np.random.default_rng(4)
    A = G0 + 0.3 * np.eye(G0.shape[0])                     # invertible: the plain-inverse form
    R = 0.05 * (rng.normal(size=G0.shape) + 1j * rng.normal(size=G0.shape))
    T = np.linalg.solve(A, np.linalg.solve(A.T, R.T).T)   # A^-1 R A^-1
    Ba = np.linalg.solve(np.eye(A.shape[0]) - A @ T, A)
    assert np.abs(Ba - A @ np.linalg.solve(A - R, A)).max() < 1e-11 * np.abs(Ba).max()


def test_sigma_tilde_vanishes_at_zero_hopping_and_scales_as_J_squared():
    """Sigma~ carries the hopping twice (Eq. (defnSigmatilde)): zero at J = 0, x4 when J doubles
    (for a fixed Gloc)."""
    p = wl.small(L=2, Ly=2, Nt=4, Nm=3, dt=0.1, U0=6.0, J0=0.3)
    S = dyson.setup(p)
    K = se.cumulant_sum(S.contour, S.eps[0], S.U[0], S.Lam[0])
    Gloc = S.Lam
    s1 = se.sigma_tilde(S, K, Gloc, 0)
    S.Jz = 2.0 * S.Jz
    s2 = se.sigma_tilde(S, K, Gloc, 0)
    assert np.abs(s2 - 4.0 * s1).max() < 1e-13 * np.abs(s2).max()
    S.Jz = 0.0 * S.Jz
    assert np.abs(se.sigma_tilde(S, K, Gloc, 0)).max() == 0.0


def test_self_consistency_converges_to_a_fixed_point():
    """The loop of Sec. IV.C reaches the criterion, and its result reproduces itself."""
    p = wl.small(L=2, Ly=2, Nt=4, Nm=3, dt=0.1, U0=8.0, J0=0.5, trap_c=0.2, aU=0.1, aJ=0.2, omega=5.0)
    blocks, St, Gloc, its, hist = se.self_consistent(p, mix=0.7, delta_sc=1e-11, max_iter=60)
    assert hist[-1] <= 1e-11 and its < 60
    S = dyson.setup(p)
    G2 = se.local_greens(S, blocks)
    St2 = np.stack([se.sigma_tilde(S, se.cumulant_sum(S.contour, S.eps[i], S.U[i], S.Lam[i]), G2, i)
                    for i in range(S.Nr)])
    assert np.abs(St2 - St).max() < 1e-8 * np.abs(St).max()
    # and it differs from the first-order (Sigma = 0) lattice function
    assert np.abs(G2 - se.local_greens(S, S.Lam)).max() > 1e-4


def test_second_order_term_is_that_of_exact_diagonalisation():
    """The point of the self-energy step: the strong-coupling expansion to second order in J.
    On the Hubbard dimer the O(J^2) coefficient of the self-consistent local Green's function
    (Matsubara block, extrapolated to dtau -> 0 from three grids) equals the one of the exact
    dimer (exact diagonalisation, continuum imaginary time), while the lattice Dyson equation
    without self-energy (Lambda alone) gets it wrong, here even in sign.  This checks the
    cumulant's signs and factors, the contraction and the local block against physics."""
    U, beta, h, Nm0 = 4.0, 1.0, 0.02, 8
    ms = (1, 2, 4)

    def dimer(Nm, J):
        return wl.uniform_problem("dimer", 2, 2, Nm, 0.05, beta, 0.0, 0.0, U, J, Ly=1)

    def g_tau0(p, G):                      # G_11(tau_m, 0) on the imaginary block
        z0 = 2 * p.Nt
        return G[0][z0:z0 + p.Nm, z0]

    c2_sc, c2_hi = [], []
    for m in ms:
        p0, ph = dimer(Nm0 * m, 0.0), dimer(Nm0 * m, h)
        S0, Sh = dyson.setup(p0), dyson.setup(ph)
        g0 = g_tau0(p0, se.local_greens(S0, S0.Lam))
        blocks, _, _, _, _ = se.self_consistent(ph, mix=0.7, delta_sc=1e-13, max_iter=60)
        gsc = g_tau0(ph, se.local_greens(Sh, blocks))
        ghi = g_tau0(ph, se.local_greens(Sh, Sh.Lam))
        c2_sc.append(((gsc - g0) / h ** 2)[::m][:Nm0])
        c2_hi.append(((ghi - g0) / h ** 2)[::m][:Nm0])
    w = ex.weights_at_zero([1.0 / m for m in ms])
    sc = sum(wb * c for wb, c in zip(w, c2_sc))
    hi = sum(wb * c for wb, c in zip(w, c2_hi))
    taus = np.arange(Nm0) * beta / Nm0
    exact = (dimer_matsubara_exact(U, h, beta, taus) - dimer_matsubara_exact(U, 0.0, beta, taus)) / h ** 2
    k = slice(1, None)                     # tau = 0 is an equal-time point (its ordering differs)
    scale = np.abs(exact[k]).max()
    assert np.abs(sc[k] - exact[k]).max() < 0.02 * scale
    assert np.abs(hi[k] - exact[k]).max() > 1.0 * scale


def test_real_time_second_order_term_is_that_of_exact_diagonalisation():
    """The same check on the real-time branch: the O(J^2) coefficient of the self-consistent
    G_11^>(t, 0) (forward branch, extrapolated to dt -> 0 from three grids that refine the real
    and the imaginary step together) equals the exact dimer's, to about 1 % of its size, while
    Lambda alone misses it by more than its size.  This exercises the real-time branches of the
    cumulant, the contour weights of the contraction and the turning-point handling of the
    local block, which the Matsubara check does not reach."""
    U, beta, h, dt0, Nt0, Nm0 = 4.0, 1.0, 0.02, 0.1, 4, 4
    ms = (1, 2, 3)

    def dimer(m, J):
        return wl.uniform_problem("dimer", 2, m * Nt0, m * Nm0, dt0 / m, beta, 0.0, 0.0, U, J, Ly=1)

    def g_t0(p, G):                        # G_11(t_k, 0) on the forward branch
        return G[0][:p.Nt, 0]

    c2_sc, c2_hi = [], []
    for m in ms:
        p0, ph = dimer(m, 0.0), dimer(m, h)
        S0, Sh = dyson.setup(p0), dyson.setup(ph)
        g0 = g_t0(p0, se.local_greens(S0, S0.Lam))
        blocks, _, _, _, _ = se.self_consistent(ph, mix=0.7, delta_sc=1e-13, max_iter=60)
        gsc = g_t0(ph, se.local_greens(Sh, blocks))
        ghi = g_t0(ph, se.local_greens(Sh, Sh.Lam))
        c2_sc.append(((gsc - g0) / h ** 2)[::m][:Nt0])
        c2_hi.append(((ghi - g0) / h ** 2)[::m][:Nt0])
    w = ex.weights_at_zero([1.0 / m for m in ms])
    sc = sum(wb * c for wb, c in zip(w, c2_sc))
    hi = sum(wb * c for wb, c in zip(w, c2_hi))
    ts = np.arange(Nt0) * dt0
    exact = (dimer_greater_exact(U, h, beta, ts) - dimer_greater_exact(U, 0.0, beta, ts)) / h ** 2
    k = slice(1, None)                     # t = 0 is the equal-time point
    scale = np.abs(exact[k]).max()
    assert np.abs(sc[k] - exact[k]).max() < 0.02 * scale
    assert np.abs(hi[k] - exact[k]).max() > 1.0 * scale


def test_fixed_point_does_not_depend_on_where_the_real_branches_end():
    """Entries of the self-consistent Sigma~ and G_loc whose times are all before the end of a
    shorter contour are the same on a longer one (driven dimer): contributions later than every
    external time cancel between the two real branches in the cumulant contraction as in the
    lattice solve.  A wrong operator order or weight on one branch breaks the cancellation."""
    U, J, beta, dt, Nm = 4.0, 0.3, 1.0, 0.1, 4

    def prob(Nt):
        return wl.uniform_problem("d", 2, Nt, Nm, dt, beta, 0.1, 0.0, U, J, Ly=1, aU=0.2, aJ=0.3, omega=3.0)

    Ns, Nl = 4, 7
    _, St_s, Gl_s, _, _ = se.self_consistent(prob(Ns), mix=0.7, delta_sc=1e-14, max_iter=80)
    _, St_l, Gl_l, _, _ = se.self_consistent(prob(Nl), mix=0.7, delta_sc=1e-14, max_iter=80)
    ix = np.array(list(range(Ns)) + [2 * Nl - Ns + j for j in range(Ns)] + [2 * Nl + m for m in range(Nm)])
    assert np.abs(St_s).max() > 1e-3
    assert np.abs(St_l[:, ix][:, :, ix] - St_s).max() < 1e-14
    assert np.abs(Gl_l[:, ix][:, :, ix] - Gl_s).max() < 1e-13


def _particle_number_drift(dt, with_selfenergy):
    """max_t N(t) - min_t N(t), N(t) = sum_i n_i(t) from the local Green's functions of a driven
    2x2 lattice (U and J modulated) on t <= 0.6."""
    Nt = int(round(0.6 / dt)) + 1
    p = wl.small(L=2, Nt=Nt, Nm=8, dt=dt, beta=1.0, trap_c=0.3, U0=8.0, J0=0.5, aU=0.2, aJ=0.3, omega=5.0)
    S = dyson.setup(p)
    blocks = S.Lam
    if with_selfenergy:
        blocks = se.self_consistent(p, mix=0.7, delta_sc=1e-10, max_iter=80)[0]
    g = se.local_greens(S, blocks)
    N = np.array([sum(np.real(-1j * g[i][k, k]) for i in range(S.Nr)) for k in range(Nt)])
    return N.max() - N.min()


def test_self_consistency_conserves_particle_number_as_dt_vanishes():
    """Under a drive the total particle number N = sum_i n_i(t) is constant (Sec. V): the
    self-consistent solution's drift falls with the time step (about first order), while the
    lattice Dyson equation with Lambda alone (no self-energy) keeps a drift that does not
    vanish, so the conservation comes from the self-energy step."""
    sc = [_particle_number_drift(dt, True) for dt in (0.1, 0.05)]
    lam = [_particle_number_drift(dt, False) for dt in (0.1, 0.05)]
    assert sc[1] < 0.45 * sc[0]
    assert lam[1] > 0.6 * lam[0]
    assert sc[1] < 0.35 * lam[1]


def test_double_occupancy_second_order_term_is_that_of_exact_diagonalisation():
    """The observables of Sec. III.A on the self-consistent solution: the O(J^2) coefficient
    of the dimer's double occupancy, read from G through Eq. (docc) (one-sided time
    difference, kinetic energy from the neighbour's G_ji) and extrapolated to dt -> 0 from
    three grids, equals <n_up n_dn> of the exact dimer in its thermal state to 1 %, at every
    time of the equilibrium run; Lambda alone misses it by half its size or more.  This pins
    the D formula and the kinetic-energy factor at U != 0 and J != 0 together."""
    U, beta, h, dt0, Nt0, Nm0 = 4.0, 1.0, 0.02, 0.1, 4, 4
    ms = (1, 2, 3)

    def dimer(m, J):
        return wl.uniform_problem("dimer", 2, m * Nt0, m * Nm0, dt0 / m, beta, 0.0, 0.0, U, J, Ly=1)

    def docc(p, blocks):
        S = dataclasses.replace(dyson.setup(p), Lam=blocks)
        G = dyson.dense_solve(S, dyson.rhs_block_columns(S, [0]))
        return observables.observables_block_column(S, 0, G)[2]

    c2_sc, c2_hi = [], []
    for m in ms:
        p0, ph = dimer(m, 0.0), dimer(m, h)
        D0 = docc(p0, dyson.setup(p0).Lam)
        Dsc = docc(ph, se.self_consistent(ph, mix=0.7, delta_sc=1e-13, max_iter=60)[0])
        Dhi = docc(ph, dyson.setup(ph).Lam)
        c2_sc.append(((Dsc - D0) / h ** 2)[::m][1:Nt0])
        c2_hi.append(((Dhi - D0) / h ** 2)[::m][1:Nt0])
    w = ex.weights_at_zero([1.0 / m for m in ms])
    sc = sum(wb * c for wb, c in zip(w, c2_sc))
    hi = sum(wb * c for wb, c in zip(w, c2_hi))

    def exact_docc(J):
        _, _, rho, _ = dimer_spectrum(U, J, beta)
        c1u, c1d, _, _ = dimer_fock()
        return np.trace(rho @ (c1u.T @ c1u) @ (c1d.T @ c1d))

    exact = (exact_docc(h) - exact_docc(0.0)) / h ** 2
    assert np.abs(sc - exact).max() < 0.01 * abs(exact)
    assert np.abs(hi - exact).min() > 0.5 * abs(exact)
