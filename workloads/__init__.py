"""Seeded synthetic workloads for the lattice Dyson solve.

This module only *describes* problems: lattice size, contour sizes, trap
curvature, chemical potential, inverse temperature and the drive tables
U_i(t_k), J_b(t_k) sampled on the real-time grid t_k = k*dt.  It holds none of
the method's arithmetic (no atomic-limit function, no Dyson algebra), so both
the CPU oracle and the CUDA path can take their inputs from here without
sharing any code with each other.

Conventions shared by every consumer (they are interface definitions, and each
side implements them on its own):

* sites: i = y*Lx + x, 0 <= x < Lx, 0 <= y < Ly, open boundaries;
* bonds: first the horizontal bonds (x,y)-(x+1,y) with index y*(Lx-1)+x, then
  the vertical bonds (x,y)-(x,y+1) with index Ly*(Lx-1) + y*Lx + x;
* drive tables are row-major: U[i, k] = U_i(t_k), J[b, k] = J_b(t_k).

The shapes follow the paper's workload (Sec. V): a 2D square lattice with a
harmonic trap V = c*|r|^2 and a modulated lattice depth that makes U(t) and J(t)
oscillate at hbar*omega ~ U_0, here with J/U ~ 0.05.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import List

import numpy as np


def n_bonds(Lx: int, Ly: int) -> int:
    """Number of nearest-neighbour bonds of an open Lx x Ly lattice."""
    return Ly * (Lx - 1) + Lx * (Ly - 1)


@dataclass
class Problem:
    """One trapped, possibly driven, lattice on a discretised contour."""

    name: str
    Lx: int
    Ly: int
    Nt: int            # real-time points per branch
    Nm: int            # imaginary-time points
    dt: float          # real-time step
    beta: float        # inverse temperature of the initial state
    mu: float          # chemical potential
    trap_c: float      # trap curvature: V_trap(r) = trap_c * |r|^2
    U: np.ndarray      # [Nr, Nt] float64, U_i(t_k)
    J: np.ndarray      # [Nb, Nt] float64, J_b(t_k)
    meta: dict = field(default_factory=dict)

    @property
    def Nr(self) -> int:
        return self.Lx * self.Ly

    @property
    def Nb(self) -> int:
        return n_bonds(self.Lx, self.Ly)

    @property
    def Nc(self) -> int:
        return 2 * self.Nt + self.Nm

    def with_tables(self, U=None, J=None, **kw) -> "Problem":
        return replace(self,
                       U=self.U.copy() if U is None else np.ascontiguousarray(U, dtype=np.float64),
                       J=self.J.copy() if J is None else np.ascontiguousarray(J, dtype=np.float64),
                       **kw)


def real_times(Nt: int, dt: float) -> np.ndarray:
    """The real-time sample points t_k = k*dt, k = 0..Nt-1 (t = 0 is the start of the drive)."""
    return np.arange(Nt, dtype=np.float64) * dt


def uniform_problem(name, L, Nt, Nm, dt, beta, mu, trap_c, U0, J0, *,
                    Ly=None, aU=0.0, aJ=0.0, omega=0.0, phase=0.0, amp=1.0) -> Problem:
    """A lattice whose sites and bonds all share one drive.

    U(t) = U0*(1 + amp*aU*sin(omega*t + phase)),  J(t) = J0 - amp*aJ*sin(omega*t + phase).
    With aU = aJ = 0 the problem is in equilibrium.
    """
    Lx = L
    Ly = L if Ly is None else Ly
    t = real_times(Nt, dt)
    s = np.sin(omega * t + phase)
    Ut = U0 * (1.0 + amp * aU * s)
    Jt = J0 - amp * aJ * s
    U = np.repeat(Ut[None, :], Lx * Ly, axis=0)
    J = np.repeat(Jt[None, :], n_bonds(Lx, Ly), axis=0)
    meta = dict(U0=U0, J0=J0, aU=aU, aJ=aJ, omega=omega, phase=phase, amp=amp)
    return Problem(name, Lx, Ly, Nt, Nm, dt, beta, mu, trap_c, U, J, meta)


def drive_derivative_tables(p: Problem):
    """dU/d(amp) and dJ/d(amp) of a uniform_problem drive, for chain-rule checks."""
    m = p.meta
    t = real_times(p.Nt, p.dt)
    s = np.sin(m["omega"] * t + m["phase"])
    dU = np.repeat((m["U0"] * m["aU"] * s)[None, :], p.Nr, axis=0)
    dJ = np.repeat((-m["aJ"] * s)[None, :], p.Nb, axis=0)
    return dU, dJ


# --------------------------------------------------------------------------
# The workloads (all synthetic, shaped like the paper's Sec. V runs).
# --------------------------------------------------------------------------

def trapped_4x4_nc64() -> Problem:
    """4x4 lattice, U=20, J=1, trap 0.5|r|^2, beta=1, Nt=24, Nm=16, dt=0.05 (Nc=64)."""
    return uniform_problem("trapped_L4_Nc64", 4, 24, 16, 0.05, 1.0, 0.0, 0.5, 20.0, 1.0)


def trapped_16x16_nc256() -> Problem:
    """16x16 lattice, U=20, J=1, trap 0.02|r|^2, beta=2, Nt=112, Nm=32, dt=0.05 (Nc=256)."""
    return uniform_problem("trapped_L16_Nc256", 16, 112, 32, 0.05, 2.0, 0.0, 0.02, 20.0, 1.0)


def driven_32x32_nc384() -> Problem:
    """32x32 lattice, U(t)=20(1+0.1 sin 20t), J(t)=1-0.2 sin 20t, trap 0.005|r|^2, beta=2, Nc=384."""
    return uniform_problem("driven_L32_Nc384", 32, 160, 64, 0.05, 2.0, 0.0, 0.005, 20.0, 1.0,
                           aU=0.1, aJ=0.2, omega=20.0)


def uneven_batch(seed: int = 1309, count: int = 64) -> List[Problem]:
    """Uneven batch: L~U{8..24}, Nc~{128,192,256} (Nm=Nc/4), U~U[12,30], c~U[0.005,0.05], phase~U[0,2pi)."""
    rng = np.random.default_rng(seed)
    out = []
    for n in range(count):
        L = int(rng.integers(8, 25))
        Nc = int(rng.choice([128, 192, 256]))
        U0 = float(rng.uniform(12.0, 30.0))
        c = float(rng.uniform(0.005, 0.05))
        ph = float(rng.uniform(0.0, 2.0 * np.pi))
        Nm = Nc // 4
        Nt = (Nc - Nm) // 2
        out.append(uniform_problem(f"uneven_{n:02d}_L{L}_Nc{Nc}", L, Nt, Nm, 0.05, 2.0, 0.0, c, U0, 1.0,
                                   aU=0.1, aJ=0.2, omega=20.0, phase=ph))
    return out


def driven_24x24_nc256(amp: float = 1.0) -> Problem:
    """24x24 lattice, Nt=96, Nm=64 (Nc=256), drive of the 32x32 lattice scaled by the amplitude `amp`."""
    return uniform_problem("driven_L24_Nc256", 24, 96, 64, 0.05, 2.0, 0.0, 0.005, 20.0, 1.0,
                           aU=0.1, aJ=0.2, omega=20.0, amp=amp)


def loss_weights(seed: int = 5, Nr: int = 576) -> np.ndarray:
    """Site weights w_i ~ U[0,1] of the adjoint loss sum_i w_i n_i(t_final)."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=Nr)


def small(name="small", L=3, Nt=6, Nm=4, dt=0.1, beta=1.0, mu=0.0, trap_c=0.3, U0=8.0, J0=1.0,
          Ly=None, **drive) -> Problem:
    """A small lattice for exhaustive checks (dense solves finish in well under a second)."""
    return uniform_problem(name, L, Nt, Nm, dt, beta, mu, trap_c, U0, J0, Ly=Ly, **drive)


def refine(p: Problem, m: int) -> Problem:
    """The same uniform_problem on a contour whose step is divided by the integer m.

    Every branch gets m times the points (Nt' = m*Nt, Nm' = m*Nm, so Nc' = m*Nc):
    the real-time grid covers the times of p (t_k of p is index m*k) and m - 1
    finer points past its last one, which leave the results at earlier times
    unchanged (the t_max independence of the contour).  The drive tables are
    resampled from the drive parameters.
    """
    if m < 1 or int(m) != m:
        raise ValueError("m must be a positive integer")
    if "U0" not in p.meta:
        raise ValueError("refine needs a uniform_problem (its drive parameters)")
    d = p.meta
    return uniform_problem(f"{p.name}_dt/{m}", p.Lx, m * p.Nt, m * p.Nm, p.dt / m, p.beta, p.mu,
                           p.trap_c, d["U0"], d["J0"], Ly=p.Ly, aU=d["aU"], aJ=d["aJ"], omega=d["omega"],
                           phase=d["phase"], amp=d["amp"])


def random_tables(p: Problem, seed: int, rel: float = 0.1) -> Problem:
    """Perturb every site's U and every bond's J independently (breaks all lattice symmetry)."""
    rng = np.random.default_rng(seed)
    U = p.U * (1.0 + rel * rng.uniform(-1.0, 1.0, size=p.U.shape))
    J = p.J * (1.0 + rel * rng.uniform(-1.0, 1.0, size=p.J.shape))
    return p.with_tables(U=U, J=J, name=p.name + f"_rand{seed}")


def sample_sources(Nr: int, count: int, seed: int) -> np.ndarray:
    """A seeded subset of source sites (block columns), sorted, without repeats."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(Nr, size=min(count, Nr), replace=False)).astype(np.int32)
