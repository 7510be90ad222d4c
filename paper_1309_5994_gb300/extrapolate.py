"""Observables extrapolated to contour step 0 (Sec. IV.D).

The same problem is solved on contours whose step is the coarsest one divided
by the integers m_b (the caller supplies the refined problems, e.g. with
workloads.refine), the observables of each solve stay on the device, and
dyson_extrapolate_dt combines them at the coarsest grid's times: three grids
give the paper's quadratic extrapolation, two the linear cross-check.
"""
from __future__ import annotations

from . import binding


def extrapolated_observables(problems, m, sources=None, precision=binding.PREC_F64, tol=1e-12,
                             max_sweeps=400, device=0, stream=None, keep_raw=False):
    """problems[b]: the problem on step h_0 / m[b] (m[0] = 1).  Solves the block columns
    `sources` (default: every site) on each contour and returns a dict with the
    extrapolated 'n', 'ekin', 'docc' ([Nr, Nt_0] float64 tensors on `device`) and,
    with keep_raw, the per-grid tables under 'raw'."""
    import torch
    dev = torch.device("cuda", device)
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    raw = []
    reports = []
    for p in problems:
        s = binding.Solver(p, device=device, stream=stream)
        try:
            s.build_sigma()
            r = s.solve(range(p.Nr) if sources is None else sources, precision=precision, tol=tol,
                        max_sweeps=max_sweeps)
            reports.append(r.report)
            tabs = [torch.empty((p.Nr, p.Nt), dtype=torch.float64, device=dev) for _ in range(3)]
            s.observables_device(*tabs)
            raw.append(tabs)
        finally:
            s.close()
    out = {}
    with torch.cuda.stream(stream):
        for q, name in enumerate(("n", "ekin", "docc")):
            out[name] = binding.extrapolate_dt([t[q] for t in raw], m, stream=stream)
    out["reports"] = reports
    if keep_raw:
        out["raw"] = {name: [t[q] for t in raw] for q, name in enumerate(("n", "ekin", "docc"))}
    return out
