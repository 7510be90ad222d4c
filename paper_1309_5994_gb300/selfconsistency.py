"""The self-consistency loop of Sec. IV.C on one context.

Each iteration solves the block columns of every site with the current local
blocks (dyson_local_greens, only the diagonal blocks G_jj are kept), takes a
self-energy step from them (dyson_selfenergy_step: Eqs. (defnSigmatilde) and
(defnSigma), mixing of Eq. (Sigmamix), new local blocks installed) and stops when
the paper's measure, taken on Sigma~, N_bd^-1 |dSigma~|_F + |dSigma~|_max, falls
to delta_sc (default 1e-8).
"""
from __future__ import annotations

from . import binding, dist


def self_consistent(solver, mix=0.7, delta_sc=None, max_iter=40, precision=binding.PREC_F64, tol=1e-13,
                    max_sweeps=400, anderson=0):
    """Run the loop on a Solver whose Lambda has been built.  Returns a dict with the
    iteration count, the history of the measure, whether it converged, the last
    local Green's functions (device tensor [Nr, Nc, Nc]) and the solve reports.
    anderson: 0 mixes linearly (Eq. (Sigmamix)); 1..6 accelerates with Anderson mixing
    of that depth (dyson_selfenergy_set_anderson)."""
    if delta_sc is None:
        delta_sc = 1e-8
    solver.set_anderson(anderson)
    gloc = None
    hist, reports = [], []
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        gloc, res = solver.local_greens(None, precision=precision, tol=tol, max_sweeps=max_sweeps, out=gloc)
        reports.append(res.report)
        crit = solver.selfenergy_step(gloc, mix)
        hist.append(crit)
        if crit <= delta_sc:
            converged = True
            break
    return {"iterations": it, "history": hist, "converged": converged, "gloc": gloc, "reports": reports,
            "delta_sc": delta_sc}


def self_consistent_sharded(solver, mix=0.7, delta_sc=None, max_iter=40, precision=binding.PREC_F64, tol=1e-13,
                            max_sweeps=400, anderson=0):
    """The same loop over the ranks of torch.distributed (one GPU each).  Each rank solves the
    block columns of its share of the sites (dist.shard_sites) and the local Green's functions
    are summed over the ranks (each rank fills only its rows); every rank then takes the same
    self-energy step on the full set, so all ranks install identical local blocks and report the
    same measure.  With one process it is self_consistent."""
    import torch
    if delta_sc is None:
        delta_sc = 1e-8
    rank, world = (torch.distributed.get_rank(), torch.distributed.get_world_size()) \
        if torch.distributed.is_available() and torch.distributed.is_initialized() else (0, 1)
    sites = dist.shard_sites(solver.p.Nr, rank, world)
    solver.set_anderson(anderson)
    gloc = None
    hist, reports = [], []
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        if gloc is None:
            dev = solver.device if isinstance(solver.device, torch.device) else torch.device("cuda", solver.device)
            gloc = torch.zeros((solver.p.Nr, solver.p.Nc, solver.p.Nc), dtype=torch.complex128, device=dev)
        else:
            gloc.zero_()
        if sites:
            _, res = solver.local_greens(sites, precision=precision, tol=tol, max_sweeps=max_sweeps, out=gloc)
            reports.append(res.report)
        dist.sum_rows_(gloc)
        crit = solver.selfenergy_step(gloc, mix)
        hist.append(crit)
        if crit <= delta_sc:
            converged = True
            break
    return {"iterations": it, "history": hist, "converged": converged, "gloc": gloc, "reports": reports,
            "delta_sc": delta_sc, "sites": sites}
