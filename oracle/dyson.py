"""Lattice Dyson equation on the discretised contour (Sec. IV.D and App. C).

Eq. (Glatt2) with the block structure of Eq. (Ginvblockstruct): the inverse
lattice Green's function has the diagonal blocks B_i = Lambda_i^{-1} (no
self-energy on this path, so B_i^{-1} = Lambda_i, the atomic-limit function of
Sec. III) and the hopping blocks -J_ij, which are diagonal in contour time.
Written with the contour quadrature weights W(z) of the discretised contour
integral, the equation reads

    G = Lambda + Lambda W J G,                 i.e.   G = (I - K)^{-1} Lambda,
    K[(i,z), (j,zb)] = Lambda_i(z, zb) W(zb) J_ij(zb)   for nearest neighbours i, j.

App. C writes the solution as the series sum_nu (B^{-1} J)^nu B^{-1} b; for one
block column (source site s) that is the iteration

    G^(0) = Lambda delta_s,   G^(n+1) = Lambda delta_s + K G^(n).

Four independent solvers are provided: the dense definition (small lattices),
the series above, the preconditioned GMRES of App. C (which also converges
where the series does not; column by column, and in the blocked form of
Sec. IV.D with one Krylov space per block of right-hand sides), and, for
homogeneous lattices, the exact diagonalisation of the hopping matrix by the
open-boundary sine modes (the momentum-space check the paper uses in Sec. IV.D).

Reading: the hopping on the imaginary branch is J(t=0), the value of the
initial equilibrium Hamiltonian.

Parity: pinned in tests/test_oracle_pins.py and tests/test_oracle_gmres.py: the
series, the dense solve and GMRES (column by column and blocked) agree (1e-12 to
1e-13), the blocked form with one column is the column form, its residual after d
block steps is never above each column's own GMRES residual at depth d, the dense solve equals
the sine-mode diagonalisation of homogeneous lattices, J = 0 returns Lambda, the
result does not depend on where the real branches end, G_ii has the C4v symmetry,
and the free-fermion (U = 0), Hubbard-I Matsubara, time-translation and
anticommutator limits of the continuum are reached at first order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .contour import Contour, make_contour, IMAG
from .lattice import neighbours, onsite_levels, bond_list, site_xy
from .atomic import atomic_gfs


@dataclass
class Setup:
    Lx: int
    Ly: int
    contour: Contour
    eps: np.ndarray       # [Nr]
    U: np.ndarray         # [Nr, Nt]
    Jz: np.ndarray        # [Nb, Nc] hopping of each bond at each contour point
    Lam: np.ndarray       # [Nr, Nc, Nc]
    nbrs: list            # per site: [(j, b)]

    @property
    def Nr(self):
        return self.Lx * self.Ly

    @property
    def Nc(self):
        return self.contour.Nc


def hopping_on_contour(c: Contour, J: np.ndarray) -> np.ndarray:
    """J_b(z): the real-grid table read at each contour point's time; J_b(0) on IMAG."""
    kz = np.where(c.branch == IMAG, 0, c.k)
    return J[:, kz]


def setup(p) -> Setup:
    """Everything the solvers need for a workloads.Problem."""
    c = make_contour(p.Nt, p.Nm, p.dt, p.beta)
    eps = onsite_levels(p.Lx, p.Ly, p.trap_c, p.U[:, 0], p.mu)
    Lam = atomic_gfs(c, eps, p.U, p.beta)
    return Setup(p.Lx, p.Ly, c, eps, np.asarray(p.U, dtype=np.float64),
                 hopping_on_contour(c, np.asarray(p.J, dtype=np.float64)), Lam,
                 neighbours(p.Lx, p.Ly))


# ----------------------------------------------------------------------------
# right-hand sides: block columns (one source site, all Nc source times) or
# vector columns (one source site, one source time)
# ----------------------------------------------------------------------------

def rhs_block_columns(S: Setup, sources) -> np.ndarray:
    """Lambda delta_s for each source s: [Nr, Nc, len(sources)*Nc], column (q, z')."""
    sources = list(sources)
    B = np.zeros((S.Nr, S.Nc, len(sources) * S.Nc), dtype=np.complex128)
    for q, s in enumerate(sources):
        B[s, :, q * S.Nc:(q + 1) * S.Nc] = S.Lam[s]
    return B


def rhs_vector_columns(S: Setup, cols) -> np.ndarray:
    """Lambda delta_s e_{z'} for each (s, z') in cols: [Nr, Nc, len(cols)]."""
    B = np.zeros((S.Nr, S.Nc, len(cols)), dtype=np.complex128)
    for q, (s, zp) in enumerate(cols):
        B[s, :, q] = S.Lam[s][:, zp]
    return B


# ----------------------------------------------------------------------------
# the operator K and its solvers
# ----------------------------------------------------------------------------

def apply_K(S: Setup, X: np.ndarray) -> np.ndarray:
    """(K X)_i = Lambda_i W sum_{j in NN(i)} J_ij X_j for X of shape [Nr, Nc, ncols]."""
    W = S.contour.W
    Y = np.empty_like(X)
    for i in range(S.Nr):
        acc = np.zeros_like(X[i])
        for j, b in S.nbrs[i]:
            acc += S.Jz[b][:, None] * X[j]
        Y[i] = S.Lam[i] @ (W[:, None] * acc)
    return Y


def dense_K(S: Setup) -> np.ndarray:
    """K as a dense [Nr*Nc, Nr*Nc] matrix (small lattices only)."""
    Nc, W = S.Nc, S.contour.W
    K = np.zeros((S.Nr * Nc, S.Nr * Nc), dtype=np.complex128)
    for i in range(S.Nr):
        for j, b in S.nbrs[i]:
            K[i * Nc:(i + 1) * Nc, j * Nc:(j + 1) * Nc] = S.Lam[i] * (W * S.Jz[b])[None, :]
    return K


def dense_solve(S: Setup, B: np.ndarray) -> np.ndarray:
    """The definition: solve (I - K) G = B directly.  B, G: [Nr, Nc, ncols]."""
    n = S.Nr * S.Nc
    K = dense_K(S)
    G = np.linalg.solve(np.eye(n) - K, B.reshape(n, -1))
    return G.reshape(B.shape)


def residual(S: Setup, B: np.ndarray, G: np.ndarray) -> float:
    """max |G - B - K G|, re-evaluated in complex128."""
    return float(np.abs(G - B - apply_K(S, G)).max())


def neumann_solve(S: Setup, B: np.ndarray, tol: float = 1e-14, max_sweeps: int = 500):
    """The series of App. C:  G <- B + K G, starting from G = B.

    Stops when the max-norm of the update falls to tol * max|B|.  Returns
    (G, sweeps, history of update norms).
    """
    scale = np.abs(B).max()
    G = B.copy()
    hist = []
    for n in range(1, max_sweeps + 1):
        Gn = B + apply_K(S, G)
        d = float(np.abs(Gn - G).max()) / scale
        hist.append(d)
        G = Gn
        if d <= tol:
            return G, n, hist
    return G, max_sweeps, hist


def gmres_solve(S: Setup, B: np.ndarray, tol: float = 1e-13, d_max: int = 40, max_restarts: int = 20):
    """Preconditioned GMRES of App. C, column by column.

    With A = B_hat - J and the block-diagonal preconditioner P = B_hat^{-1}
    (here Lambda with the contour weights), the preconditioned operator is
    P A = I - K.  Following the appendix's steps:
      1. initial guess u0 = P b = B (the right-hand side Lambda delta), residue
         z0 = P (b - A u0) = K B, q1 = z0 / |z0|;
      2. for d = 1..d_max: w = (I - K) q_d; for i = 1..d: h_id = <q_i|w>,
         w <- w - h_id q_i (modified Gram-Schmidt); h_{d+1,d} = |w|;
         q_{d+1} = w / h_{d+1,d};
      3. y minimises | |z0| e_1 - H_d y |_2 (a least-squares solve of the small
         (d+1) x d Hessenberg system), u = u0 + Q_d y;
    restarting from u when d reaches d_max.  Every column (the last axis of B)
    has its own Krylov space.  The stopping rule (a reading: the paper gives an
    absolute bound, Eq. (GMRESconvergence)) is relative: the preconditioned
    residual |P(b - A u)|_2 <= tol |B|_2 for every column.

    Returns (G, iterations, history of the largest relative residual).
    """
    ncol = B.shape[2]
    bnorm = np.sqrt((np.abs(B) ** 2).sum(axis=(0, 1)))
    U = B.copy()
    hist, its = [], 0
    for _ in range(max_restarts + 1):
        Z = B - (U - apply_K(S, U))                  # P(b - A u) = B - (I - K) u
        beta = np.sqrt((np.abs(Z) ** 2).sum(axis=(0, 1)))
        rel = beta / bnorm
        hist.append(float(rel.max()))
        if rel.max() <= tol:
            return U, its, hist
        Q = [Z / np.where(beta > 0, beta, 1.0)]
        H = np.zeros((ncol, d_max + 1, d_max), dtype=complex)
        done = np.zeros(ncol, dtype=bool)
        for d in range(d_max):
            its += 1
            W = Q[d] - apply_K(S, Q[d])
            for i in range(d + 1):
                h = (np.conj(Q[i]) * W).sum(axis=(0, 1))
                H[:, i, d] = h
                W = W - h[None, None, :] * Q[i]
            hn = np.sqrt((np.abs(W) ** 2).sum(axis=(0, 1)))
            H[:, d + 1, d] = hn
            Q.append(W / np.where(hn > 0, hn, 1.0))
            # least-squares residual of each column at dimension d + 1
            res = np.empty(ncol)
            for n in range(ncol):
                g = np.zeros(d + 2, dtype=complex)
                g[0] = beta[n]
                y = np.linalg.lstsq(H[n, :d + 2, :d + 1], g, rcond=None)[0]
                res[n] = np.linalg.norm(g - H[n, :d + 2, :d + 1] @ y)
            done = (res <= tol * bnorm) | (hn <= 1e-300)
            if done.all():
                break
        dd = d + 1
        for n in range(ncol):
            g = np.zeros(dd + 1, dtype=complex)
            g[0] = beta[n]
            y = np.linalg.lstsq(H[n, :dd + 1, :dd], g, rcond=None)[0]
            for i in range(dd):
                U[:, :, n] += y[i] * Q[i][:, :, n]
    Z = B - (U - apply_K(S, U))
    hist.append(float((np.sqrt((np.abs(Z) ** 2).sum(axis=(0, 1))) / bnorm).max()))
    return U, its, hist


def block_gmres_solve(S: Setup, B: np.ndarray, tol: float = 1e-13, d_max: int = 20, max_restarts: int = 20):
    """GMRES of App. C applied to a block of right-hand sides at once (Sec. IV.D,
    Eq. (blockedGMRESproblem) with the unit-vector blocks of Eq. (unitblock)).

    Reading: the blocked system is solved with one Krylov space shared by all
    columns of B (block Arnoldi), so that projections and updates act on blocks.
    With the same preconditioner as gmres_solve (the operator is I - K) and the
    same initial guess U0 = B:
      1. R0 = B - (I - K) U0, reduced QR R0 = V_1 C (V_1 orthonormal columns);
      2. for d = 1..d_max: W = (I - K) V_d; for i = 1..d: H_id = V_i^H W,
         W <- W - V_i H_id (block Gram-Schmidt, two passes); W = V_{d+1} H_{d+1,d}
         (reduced QR);
      3. Y minimises |E_1 C - H_d Y|_F over the ((d+1)p) x (dp) block Hessenberg
         matrix H_d, U = U0 + [V_1 .. V_d] Y;
    restarting from U when d reaches d_max.  Stopping rule as in gmres_solve: the
    residual of every column relative to that column of B, in the 2-norm.

    Returns (G, block iterations, history of the largest relative residual).
    """
    Nr, Nc, p = B.shape
    n = Nr * Nc

    def op(X):
        Y = X.reshape(Nr, Nc, -1)
        return (Y - apply_K(S, Y)).reshape(n, -1)

    Bm = B.reshape(n, p)
    bnorm = np.linalg.norm(Bm, axis=0)
    U = Bm.copy()
    hist, its = [], 0
    for _ in range(max_restarts + 1):
        R = Bm - op(U)
        rel = np.linalg.norm(R, axis=0) / bnorm
        hist.append(float(rel.max()))
        if rel.max() <= tol:
            return U.reshape(Nr, Nc, p), its, hist
        V1, C = np.linalg.qr(R)
        V = [V1]
        H = np.zeros(((d_max + 1) * p, d_max * p), dtype=complex)
        Y = None
        for d in range(d_max):
            its += 1
            W = op(V[d])
            for _pass in range(2):
                for i in range(d + 1):
                    h = V[i].conj().T @ W
                    H[i * p:(i + 1) * p, d * p:(d + 1) * p] += h
                    W = W - V[i] @ h
            Vn, Hn = np.linalg.qr(W)
            H[(d + 1) * p:(d + 2) * p, d * p:(d + 1) * p] = Hn
            V.append(Vn)
            E = np.zeros(((d + 2) * p, p), dtype=complex)
            E[:p] = C
            Hd = H[:(d + 2) * p, :(d + 1) * p]
            Y = np.linalg.lstsq(Hd, E, rcond=None)[0]
            res = np.linalg.norm(E - Hd @ Y, axis=0) / bnorm
            if res.max() <= tol:
                break
        U = U + np.concatenate(V[:d + 1], axis=1) @ Y
    R = Bm - op(U)
    hist.append(float((np.linalg.norm(R, axis=0) / bnorm).max()))
    return U.reshape(Nr, Nc, p), its, hist


# ----------------------------------------------------------------------------
# homogeneous lattice: exact solve in the sine basis (momentum-space check)
# ----------------------------------------------------------------------------

def sine_modes(L: int) -> tuple:
    """Open-chain eigenvectors phi_n(x) = sqrt(2/(L+1)) sin(pi n (x+1)/(L+1)) and
    eigenvalues 2 cos(pi n/(L+1)), n = 1..L, of the 1D nearest-neighbour matrix."""
    n = np.arange(1, L + 1)
    x = np.arange(L)
    phi = np.sqrt(2.0 / (L + 1)) * np.sin(np.pi * np.outer(x + 1, n) / (L + 1))  # [x, n]
    lam = 2.0 * np.cos(np.pi * n / (L + 1))
    return phi, lam


def homogeneous_solve(S: Setup, pairs) -> dict:
    """G_ij (all Nc x Nc) for the requested site pairs of a homogeneous lattice.

    Requires one level eps, one U(t) and one J(t) for every site and bond.  The
    hopping matrix J(t) A is diagonalised by the 2D sine modes with eigenvalues
    lambda_nm = 2cos(pi n/(Lx+1)) + 2cos(pi m/(Ly+1)), so
    G_ij = sum_nm phi_nm(i) phi_nm(j) (I - lambda_nm Lambda W J)^{-1} Lambda.
    """
    if not (np.allclose(S.eps, S.eps[0]) and np.allclose(S.U, S.U[0]) and np.allclose(S.Jz, S.Jz[0])):
        raise ValueError("homogeneous_solve needs a homogeneous lattice")
    Lam, WJ = S.Lam[0], S.contour.W * S.Jz[0]
    px, lx = sine_modes(S.Lx)
    py, ly = sine_modes(S.Ly)
    x, y = site_xy(S.Lx, S.Ly)
    out = {pr: np.zeros((S.Nc, S.Nc), dtype=np.complex128) for pr in pairs}
    I = np.eye(S.Nc)
    for a in range(S.Lx):
        for b in range(S.Ly):
            g = np.linalg.solve(I - (lx[a] + ly[b]) * Lam * WJ[None, :], Lam)
            for (i, j) in pairs:
                out[(i, j)] += px[x[i], a] * py[y[i], b] * px[x[j], a] * py[y[j], b] * g
    return out


def bonds(S: Setup):
    return bond_list(S.Lx, S.Ly)
