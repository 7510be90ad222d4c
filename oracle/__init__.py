"""CPU oracle for the lattice Dyson solve of Dirks, Mikelsons, Krishnamurthy and
Freericks, "Simulation of inhomogeneous distributions of ultracold atoms in an
optical lattice via a massively parallel implementation of nonequilibrium
strong-coupling perturbation theory" (arXiv:1309.5994).

THIS PACKAGE IS TEST INFRASTRUCTURE.  It is a plain, slow, complex128 NumPy
restatement of what the GPU path computes, written from the paper and kept
independent of the CUDA code (no shared kernels, headers, helpers, tables or
constants).  Only the test-suite, the smoke check of ``__graft_entry__`` and the
CPU-baseline leg of ``bench.py`` may import it.  The product path never calls
it and has no CPU fallback.

Modules
-------
contour      Sec. IV.A / Fig. 1: discretised Kadanoff-Baym-Keldysh contour and
             its quadrature weights.
lattice      Sec. II, Eq. (model)/(onsitelevels): sites, bonds, trap.
atomic       Sec. III, Eqs. (cumulanttabulation)-(Z): atomic-limit contour
             Green's function Lambda_i of each site.
dyson        Sec. IV.D, Eqs. (Glatt2)/(Ginvblockstruct), App. C: the lattice
             Dyson equation G = Lambda + Lambda W J G, solved densely, by the
             series in powers of J, and in the sine basis for homogeneous
             lattices.
observables  Sec. III.A and App. B: density, kinetic energy, double occupancy.
adjoint      Gradients of weighted densities and double occupancies (no
             counterpart in the paper; derived from the Dyson equation).
extrapolate  Sec. IV.D: quadratic (or linear) extrapolation of results on
             refined contours to step 0.

Parity status of every function is stated in its docstring; functions whose
results are not fixed by an independent pin say "parity unpinned".
"""
from . import contour, lattice, atomic, dyson, observables, adjoint, extrapolate  # noqa: F401
