#!/usr/bin/env python3
"""Benchmark of the lattice Dyson solve on GB300.

Workload: the 16x16 trapped lattice on the Nc = 256 contour (112 + 112 real-time
points, dt = 0.05, 32 imaginary points, beta = 2, U = 20, J = 1, trap
0.02 |r|^2, mu = 0): every block column G(:, s) solved to a relative FP64 Dyson
residual <= tol with the mixed-precision path (3xTF32 tcgen05 series sweeps,
FP64 residual refinement).  A step builds Lambda, solves one batch of
`--batch` block columns (disjoint per rank and per step, cycling through the
256 sources) and computes the observables of those sources; the metric is
block columns per second over all ranks.

Also measured: the same steps end to end through the C ABI from host buffers
(e2e), the plain FP64 GPU series on two block columns (speed-up and the error
of the mixed result against it), and the CPU oracle on a bounded sample
(cpu_baseline).  `--impl reference` times the CPU oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "contour-GEMM TFLOP/s and G columns/s vs plain FP64 on one GB300 at rel err 1e-6"
UNIT = "block columns/s"
WORKLOAD = ("16x16 trapped lattice (256 sites, open boundaries), Nc=256 (112+112 real-time points dt=0.05, "
            "32 imaginary), U=20, J=1, V=0.02|r|^2, mu=0, beta=2; all 256 block columns cycled in batches")
# Measured peaks of this GPU (MEASURED_PEAKS.json, burst) and the recipe's nominal ratios
NOMINAL_TF32_OVER_BF16 = 1.1 / 2.25
NOMINAL_FP64_TFLOPS = 1.25          # 152 SMs x 4 FP64 flop/clk x 2.07 GHz (recipe's nominal FP64 rate)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--batch", type=int, default=16, help="block columns per step per GPU")
    ap.add_argument("--tol", type=float, default=1e-6,
                    help="relative FP64 Dyson residual: the metric is quoted at relative error 1e-6; the "
                         "errors of the result against the FP64 series run to 1e-12 are measured and reported")
    ap.add_argument("--f64-columns", type=int, default=2, help="block columns timed on the plain FP64 path")
    ap.add_argument("--cpu-columns", type=int, default=32, help="vector columns in the CPU oracle sample")
    ap.add_argument("--no-extras", action="store_true", help="skip e2e, FP64 and CPU legs (profiling runs)")
    ap.add_argument("--uneven-instances", type=int, default=64,
                    help="instances of the seeded uneven batch in the batched-solve leg (0 skips it)")
    ap.add_argument("--no-driven", action="store_true", help="skip the driven 32x32 (Nc = 384) leg")
    ap.add_argument("--no-selfenergy", action="store_true", help="skip the self-consistency loop leg")
    ap.add_argument("--sweep-variant", default="auto",
                    choices=["auto", "single_cta", "cta_pair", "fused_pair", "fused_pair_wide"],
                    help="override the autotuner's sweep variant (profiling runs: kernel timings under a "
                         "profiler can flip the tuner's choice)")
    ap.add_argument("--lattice", type=int, default=16,
                    help="lattice side; 16 is the benchmark workload, smaller sides serve ncu captures only")
    return ap.parse_args()


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_trapped16x16_16cols.json")


def load_traffic():
    """DRAM bytes per launch of each kernel kind at the benchmark size, from an ncu
    capture (profiles/), kept only while the kernel's source is unchanged."""
    import hashlib
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
    except OSError:
        return {}
    out = {}
    for name, e in rec.get("kernels", {}).items():
        try:
            with open(os.path.join(ROOT, e["source"]), "rb") as f:
                same = hashlib.sha256(f.read()).hexdigest() == e["sha256"]
        except OSError:
            same = False
        out[name] = e["bytes_per_launch"] if same else None
    return out


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        self.index = ids[local_rank] if local_rank < len(ids) and ids[local_rank].strip().isdigit() else str(local_rank)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        return summarise_clocks(out)


def summarise_clocks(out: str):
    """Median SM clock, maximum SM clock and the throttle reasons seen, from the CSV lines
    (no header, no units) of ClockSampler.FIELDS; lines that do not parse are skipped."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 8:
            continue
        try:
            sm.append(float(f[0]))
            smax.append(float(f[1]))
        except ValueError:
            continue
        for nm, v in zip(names, f[4:8]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------
def oracle_sample(p, site: int, zps, tol: float, S=None):
    """Time the CPU oracle's complex128 series on vector columns (site, z') of p,
    stopped at the relative update tol."""
    from oracle import dyson
    if S is None:
        S = dyson.setup(p)
    B = dyson.rhs_vector_columns(S, [(site, int(z)) for z in zps])
    t = time.perf_counter()
    G, sweeps, _ = dyson.neumann_solve(S, B, tol=tol, max_sweeps=400)
    dt = time.perf_counter() - t
    return dt, sweeps, S


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline(p, ncols: int, tol: float):
    import numpy as np
    zps = np.linspace(0, p.Nc - 1, ncols).astype(int)
    dt, sweeps, _ = oracle_sample(p, 119, zps, tol)
    per_block = dt * p.Nc / ncols
    return {"value": 1.0 / per_block, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": (f"{ncols} of the 256 vector columns of block column 119, complex128 series to {tol:g} "
                       f"({sweeps} sweeps, {dt:.2f} s), scaled linearly to one block column")}


def selfenergy_leg(args, dev, stream):
    """The self-consistency loop of Sec. IV.C (self-energy steps between lattice solves) on a
    driven 8x8 trapped lattice, Nc = 64 (24 + 24 real-time points dt = 0.05, 16 imaginary),
    U(t) = 20 (1 + 0.1 sin 20t), J(t) = 1 - 0.2 sin 20t, trap 0.02 |r|^2, beta = 2: all 64 block
    columns per iteration in mixed precision (residual 1e-10), mixing 0.7, until the paper's
    measure (taken on Sigma~) falls to 1e-8 (at most 40 iterations)."""
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    from paper_1309_5994_gb300.selfconsistency import self_consistent
    p = wl.uniform_problem("se_L8_Nc64_driven", 8, 24, 16, 0.05, 2.0, 0.0, 0.02, 20.0, 1.0,
                           aU=0.1, aJ=0.2, omega=20.0)
    s = binding.Solver(p, device=dev.index, stream=stream)
    s.build_sigma()
    s.local_greens(None, precision=binding.PREC_TF32X3_F64REF, tol=1e-10)     # warm-up: tables, buffers
    s.build_sigma()
    s.profile(True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r = self_consistent(s, mix=0.7, max_iter=40, precision=binding.PREC_TF32X3_F64REF, tol=1e-10)
    torch.cuda.synchronize(dev)
    secs = time.perf_counter() - t0
    n_conn, ms_conn = s.profile_query(7)
    s.profile(False)
    # the same loop with Anderson acceleration (depth 5) in place of the linear mixing
    s.build_sigma()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    ra = self_consistent(s, mix=0.7, max_iter=40, precision=binding.PREC_TF32X3_F64REF, tol=1e-10, anderson=5)
    torch.cuda.synchronize(dev)
    secs_aa = time.perf_counter() - t0
    # Anderson again, with the lattice solves reduced to one site per C4v orbit (App. A)
    s.set_symmetry(binding.SYMMETRY_C4V)
    s.build_sigma()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rc = self_consistent(s, mix=0.7, max_iter=40, precision=binding.PREC_TF32X3_F64REF, tol=1e-10, anderson=5)
    torch.cuda.synchronize(dev)
    secs_c4v = time.perf_counter() - t0
    s.close()
    its = r["iterations"]
    flops = 8.0 * p.Nc ** 4 * p.Nr                   # the [Nc]^4 contraction per site, complex MACs x 8
    ach = flops / (ms_conn / n_conn * 1e-3) / 1e12 if n_conn else None
    return {"workload": "8x8 driven trapped lattice, Nc=64 (24+24 real-time points dt=0.05, 16 imaginary), "
                        "U=20(1+0.1 sin 20t), J=1-0.2 sin 20t, V=0.02|r|^2, beta=2",
            "iterations": its, "converged": r["converged"], "criterion": r["history"][-1],
            "delta_sc": r["delta_sc"], "history": [float(f"{h:.3e}") for h in r["history"]],
            "seconds": secs, "seconds_per_iteration": secs / its,
            "lattice_solve_sweeps_per_iteration": [q["sweeps"] for q in r["reports"]],
            "anderson5": {"iterations": ra["iterations"], "converged": ra["converged"], "seconds": secs_aa,
                          "history": [float(f"{h:.3e}") for h in ra["history"]]},
            "anderson5_c4v": {"iterations": rc["iterations"], "converged": rc["converged"], "seconds": secs_c4v,
                              "history": [float(f"{h:.3e}") for h in rc["history"]],
                              "note": "local Green's functions of one site per C4v orbit (10 of 64)"},
            "selfenergy_conn": {"launches": n_conn, "avg_ms": ms_conn / n_conn if n_conn else None,
                                "share_of_loop": ms_conn * 1e-3 / secs,
                                "roofline": {"bound": "alu", "achieved": ach, "peak": NOMINAL_FP64_TFLOPS,
                                             "unit": "TFLOP/s", "frac": ach / NOMINAL_FP64_TFLOPS if ach else None,
                                             "peak_source": "nominal FP64 rate (no measured FP64 peak); "
                                                            "achieved counts 8 Nc^4 flops per site (the "
                                                            "[Nc]^4 cumulant contraction)"}}}


def batched_uneven_leg(args, dev, stream):
    """The seeded uneven batch (lattice sides 8..24, Nc in {128, 192, 256}, U, trap and
    drive phase drawn per instance): one block column per instance (the site next to
    the trap centre) solved to the same FP64 residual, once as one dyson_batch
    (shared sweep launches under CUDA graphs) and once instance by instance."""
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    problems = wl.uneven_batch(count=args.uneven_instances)
    solvers = []
    for p in problems:
        s = binding.Solver(p, device=dev.index, stream=stream)
        s.build_sigma()
        solvers.append(s)
    sources = [[p.Nr // 2 + p.Lx // 2] for p in problems]
    batch = binding.Batch(solvers)
    # instances whose series diverges (spectral radius of Lambda W J above 1) end
    # with DIVERGED; the paper hands those to GMRES, which this leg does not run
    batch.solve(sources, tol=args.tol, allow=(0, -4))      # warm-up: tables, graph, buffers
    torch.cuda.synchronize(dev)
    l0 = batch.launch_count()
    t0 = time.perf_counter()
    res = batch.solve(sources, tol=args.tol, allow=(0, -4))
    torch.cuda.synchronize(dev)
    t_batch = time.perf_counter() - t0
    graph_launches = batch.launch_count() - l0
    t0 = time.perf_counter()
    for s, src in zip(solvers, sources):
        s.solve(src, precision=binding.PREC_TF32X3_F64REF, tol=args.tol, max_sweeps=400, allow=(0, -4))
    torch.cuda.synchronize(dev)
    t_seq = time.perf_counter() - t0
    n = len(problems)
    conv = [k for k, r in enumerate(res) if r.status == 0]
    flops = sum(r.report["gemm_flops"] for r in res)
    out = {"value": len(conv) / t_batch, "unit": UNIT, "instances": n, "block_columns_converged": len(conv),
           "diverged_instances": [k for k, r in enumerate(res) if r.status == -4],
           "value_note": "converged block columns per second of the whole batch (diverged instances' time included)",
           "shapes": {"lattice_sides": sorted({p.Lx for p in problems}), "Nc": sorted({p.Nc for p in problems})},
           "seconds": t_batch, "contour_gemm_tflops": flops / t_batch / 1e12,
           "sequential_value": len(conv) / t_seq, "speedup_vs_sequential": t_seq / t_batch,
           "sweeps_max": max(r.report["sweeps"] for r in res),
           "refinements_max": max(r.report["refinements"] for r in res),
           "max_rel_residual_converged": max(res[k].report["residual"] for k in conv) if conv else None,
           "graph_kernel_launches": graph_launches, "tol_rel_residual": args.tol}
    batch.close()
    for s in solvers:
        s.close()
    return out


def driven_leg(args, dev, stream):
    """The driven 32x32 lattice (Nc = 384, U(t) = 20(1 + 0.1 sin 20t), J(t) = 1 - 0.2 sin 20t):
    one block column near the trap centre in mixed precision (the FP32 series
    cannot serve on this contour, so the AUTO inner solver runs GMRES) against the
    plain FP64 series run for 105 sweeps, where its update reaches its floor."""
    import numpy as np
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    p = wl.driven_32x32_nc384()
    s = binding.Solver(p, device=dev.index, stream=stream)
    s.build_sigma()
    src = [527]
    s.solve(src, precision=binding.PREC_TF32X3_F64REF, tol=args.tol, max_sweeps=400)   # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rm = s.solve(src, precision=binding.PREC_TF32X3_F64REF, tol=args.tol, max_sweeps=400)
    torch.cuda.synchronize(dev)
    t_mixed = time.perf_counter() - t0
    n_mixed = s.observables()[0][src[0]].copy()
    t0 = time.perf_counter()
    rf = s.solve(src, precision=binding.PREC_F64, tol=1e-15, max_sweeps=105, allow=(0, -3))
    torch.cuda.synchronize(dev)
    t_f64 = time.perf_counter() - t0
    n_f64 = s.observables()[0][src[0]].copy()
    s.close()
    return {"workload": "32x32 driven lattice, Nc=384 (160+160 real-time points dt=0.05, 64 imaginary), "
                        "block column of site 527",
            "mixed": {"seconds": t_mixed, "value": 1.0 / t_mixed, "unit": UNIT, "sweeps": rm.report["sweeps"],
                      "refinements": rm.report["refinements"], "rel_residual": rm.report["residual"],
                      "inner_solver": "gmres" if rm.report["inner_gmres"] else "series"},
            "plain_f64": {"seconds": t_f64, "value": 1.0 / t_f64, "unit": UNIT, "sweeps": rf.report["sweeps"],
                          "final_update": rf.report["update"],
                          "note": "the FP64 series' update floors near 5e-8 on this contour (partial sums peak ~2e7 "
                                  "above the result), so it cannot reach the mixed path's residual"},
            "speedup_vs_plain_f64": t_f64 / t_mixed,
            "density_rel_diff_mixed_vs_f64": float(np.abs(n_mixed - n_f64).max() / np.abs(n_f64).max())}


def wedge_leg(args, dev, stream, tuning):
    """All 256 sources of the 16x16 workload, whose centred trap and uniform drive
    keep C4v (App. A): the 36 orbit representatives are solved and the other
    sites' observables filled by symmetry."""
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    p = wl.trapped_16x16_nc256()
    s = binding.Solver(p, device=dev.index, stream=stream)
    s.set_sweep_variant(tuning["sweep_variant"])
    s.set_chunk(tuning["chunk_block_columns"])
    s.build_sigma()
    s.set_symmetry(binding.SYMMETRY_C4V)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r = s.solve(list(range(p.Nr)), precision=binding.PREC_TF32X3_F64REF, tol=args.tol, max_sweeps=400)
    n, _, _ = s.observables()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    s.close()
    L = p.Lx
    orbits = {min(y2 * L + x2 for x2, y2 in ((x, y), (L - 1 - x, y), (x, L - 1 - y), (y, x), (L - 1 - y, L - 1 - x),
                                              (L - 1 - x, L - 1 - y), (y, L - 1 - x), (L - 1 - y, x)))
              for y in range(L) for x in range(L)}
    return {"sources": p.Nr, "representatives_solved": len(orbits), "status": r.status,
            "seconds": dt, "site_observables_per_s": p.Nr / dt, "unit": "sources with observables per second",
            "note": "not the benchmark metric: block columns actually solved are the orbit representatives"}


def run_reference(args, rank, world):
    """The CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np
    import workloads as wl
    from oracle import dyson
    p = wl.trapped_16x16_nc256()
    S = dyson.setup(p)
    ncols = 16
    times = []
    for step in range(args.warmup + args.steps):
        site = (step * 37) % p.Nr
        zps = np.linspace(step % 16, p.Nc - 1, ncols).astype(int)
        dt, _, _ = oracle_sample(p, site, zps, args.tol, S)
        if step >= args.warmup:
            times.append(dt * p.Nc / ncols)      # seconds per block column
    per_block = sum(times) / len(times)
    value = 1.0 / per_block
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_block * 1e3 * ncols / p.Nc,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"{ncols} vector columns of one block column"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                             "sample": f"{ncols} vector columns per step, complex128 series to {args.tol:g}, "
                                       "scaled to block columns"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gb300(args, rank, world, local):
    import numpy as np
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding, dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = wl.trapped_16x16_nc256() if args.lattice == 16 else wl.uniform_problem(
        f"trapped_L{args.lattice}_Nc256", args.lattice, 112, 32, 0.05, 2.0, 0.0, 0.02, 20.0, 1.0)
    stream = torch.cuda.Stream(device=dev)
    solver = binding.Solver(p, device=local, stream=stream)
    PREC = binding.PREC_TF32X3_F64REF

    def step(k, s=solver):
        src = dist.step_sources(p.Nr, args.batch, rank, world, k)
        s.build_sigma()
        return s.solve(src, precision=PREC, tol=args.tol, max_sweeps=400)

    # sweep variant and chunk picked by the library's autotuner on this workload
    solver.build_sigma()
    tuning = solver.autotune(args.batch)
    if args.sweep_variant != "auto":
        tuning["sweep_variant"] = binding.SWEEP_NAMES.index(args.sweep_variant)
        solver.set_sweep_variant(tuning["sweep_variant"])
    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize(dev)
    dist.barrier(local)

    # ---- timed region: device events on the library stream ----
    solver.profile(True)
    launches0 = solver.launch_count()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    ev0.record(stream)
    reports = []
    for k in range(args.steps):
        reports.append(step(args.warmup + k).report)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    dist.barrier(local)
    elapsed_ms = ev0.elapsed_time(ev1)
    gpu_launches = solver.launch_count() - launches0
    kstats = {name: solver.profile_query(kk) for kk, name in binding.KERNEL_NAMES.items()}
    solver.profile(False)
    max_ms = dist.max_over_ranks(elapsed_ms, device=dev)

    cols_total = world * args.steps * args.batch
    value = cols_total / (max_ms * 1e-3)
    flops = sum(r["gemm_flops"] for r in reports)
    tflops_local = flops / (elapsed_ms * 1e-3) / 1e12
    sweeps = [r["sweeps"] for r in reports]
    refinements = [r["refinements"] for r in reports]
    residual = max(r["residual"] for r in reports)

    # ---- rooflines per kernel kind; the one with the largest device time is reported ----
    peaks, peak_src = load_peaks()
    traffic = load_traffic() if args.lattice == 16 else {}
    Nc, Nr = p.Nc, p.Nr
    ncol = args.batch * Nc
    alg_flops = 8.0 * Nc * Nc * Nr * ncol                   # contour-GEMM flops of one sweep / residual
    state_bytes = 2.0 * Nc * 4 * Nr * ncol                  # one FP32 planar chunk state
    note = "achieved counts algorithmic complex-GEMM flops (8 Nc^2 per site and vector column)"
    rooflines = {}
    for name, (n, ms) in kstats.items():
        if not n:
            continue
        dur = ms / n * 1e-3
        if name == "gather_tc":
            ach = 2 * state_bytes / dur / 1e9
            peak = peaks["hbm_gbs"]
            r = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                 "algorithmic_bytes_per_launch": 2 * state_bytes,
                 "peak_source": f"{peak_src} copy bandwidth; bytes = read d + write X (FP32 planar state)"}
        elif name in ("sweep_f64", "residual_f64"):
            ach = alg_flops / dur / 1e12
            r = {"bound": "alu", "achieved": ach, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                 "frac": ach / NOMINAL_FP64_TFLOPS,
                 "peak_source": "nominal FP64 rate from SM count x FP64 flop/clk x max clock (no measured FP64 peak)"}
        elif name == "residual_split_bf16":
            ach = alg_flops / dur / 1e12
            peak = peaks["bf16_tflops"]
            r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                 "executed_tflops": 28 * ach,
                 "peak_source": f"{peak_src} bf16 burst; {note}, the 7-slice split executes 28 BF16 products"}
        else:
            ach = alg_flops / dur / 1e12
            peak = peaks["bf16_tflops"] * NOMINAL_TF32_OVER_BF16
            r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                 "executed_tflops": 3 * ach, "executed_frac": 3 * ach / peak,
                 "peak_source": f"{peak_src} bf16 burst x nominal tf32/bf16 ratio; {note}, the 3xTF32 split "
                                f"executes 3x"}
        r["traffic"] = traffic.get(name)
        r["kernel"] = name
        r["avg_ms"] = ms / n
        rooflines[name] = r
    dom_name = max(kstats.items(), key=lambda kv: kv[1][1])[0]
    roof = rooflines[dom_name]
    kernels = {nm: {"launches": n, "avg_ms": (ms / n if n else None), "total_ms": ms,
                    "share": ms / max(sum(v[1] for v in kstats.values()), 1e-9)}
               for nm, (n, ms) in kstats.items() if n}

    extras = {}
    if not args.no_extras:
        # ---- e2e through the C ABI from host buffers: init (tables H2D), build, solve, observables D2H ----
        h2d = p.U.nbytes + p.J.nbytes + 4 * args.batch
        d2h = 3 * p.Nr * p.Nt * 8
        torch.cuda.synchronize(dev)
        dist.barrier(local)
        t0 = time.perf_counter()
        for k in range(args.steps):
            s2 = binding.Solver(p, device=local, stream=stream)
            s2.set_sweep_variant(tuning["sweep_variant"])
            s2.set_chunk(tuning["chunk_block_columns"])
            s2.build_sigma()
            # the same source batches as the timed device steps
            s2.solve(dist.step_sources(p.Nr, args.batch, rank, world, args.warmup + k), precision=PREC,
                     tol=args.tol, max_sweeps=400)
            s2.observables()
            s2.close()
        torch.cuda.synchronize(dev)
        e2e_s = dist.max_over_ranks(time.perf_counter() - t0, device=dev)
        extras["e2e"] = {"value": cols_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h}
        if rank == 0:
            # ---- plain FP64 GPU series on a few block columns, and the mixed result's error ----
            nf = args.f64_columns
            srcs = list(range(nf))
            g64 = torch.empty((nf, Nr, Nc, Nc), dtype=torch.complex128, device=dev)
            gmx = torch.empty_like(g64)
            solver.build_sigma()
            # timed: the FP64 series stopped at the same relative level as the mixed path
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            r64 = solver.solve(srcs, precision=binding.PREC_F64, tol=args.tol, max_sweeps=400, g_out=g64,
                               allow=(0, -3))
            torch.cuda.synchronize(dev)
            t64 = time.perf_counter() - t0
            # the accuracy reference: the FP64 series to 1e-12 (its update bottoms out near
            # 1e-13 on this contour, partial sums peaking ~200x above the result)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            r64t = solver.solve(srcs, precision=binding.PREC_F64, tol=1e-12, max_sweeps=400, g_out=g64,
                                allow=(0, -3))
            torch.cuda.synchronize(dev)
            t64t = time.perf_counter() - t0
            n64, _, _ = solver.observables()
            rmx = solver.solve(srcs, precision=PREC, tol=args.tol, max_sweeps=400, g_out=gmx)
            nmx, _, _ = solver.observables()
            den = torch.abs(g64).max().item()
            gerr = torch.abs(gmx - g64).max().item() / den
            gii = torch.stack([g64[q, s] for q, s in enumerate(srcs)])
            gii_m = torch.stack([gmx[q, s] for q, s in enumerate(srcs)])
            gii_err = (torch.abs(gii_m - gii).max() / torch.abs(gii).max()).item()
            nerr = float(np.abs(nmx[srcs] - n64[srcs]).max() / np.abs(n64[srcs]).max())
            f64_rate = nf / t64
            extras["plain_f64"] = {"value": f64_rate, "unit": UNIT, "block_columns": nf, "tol_rel_update": args.tol,
                                   "sweeps": r64.report["sweeps"], "status": r64.status,
                                   "final_update": r64.report["update"],
                                   "tflops": r64.report["gemm_flops"] / t64 / 1e12,
                                   "tight": {"tol_rel_update": 1e-12, "value": nf / t64t, "unit": UNIT,
                                             "sweeps": r64t.report["sweeps"], "status": r64t.status,
                                             "final_update": r64t.report["update"]}}
            extras["speedup_vs_plain_f64"] = (value / world) / f64_rate
            extras["rel_err_vs_plain_f64"] = {"reference": "FP64 series to 1e-12", "G": gerr, "G_ii": gii_err,
                                              "density": nerr, "within_1e-6": bool(max(gii_err, nerr) <= 1e-6)}
            del g64, gmx
            # the single-GPU legs run at N = 1 only: with more ranks every GPU would wait for them
            if world == 1:
                extras["cpu_baseline"] = cpu_baseline(p, args.cpu_columns, args.tol)
                if args.uneven_instances > 0:
                    extras["batched_uneven"] = batched_uneven_leg(args, dev, stream)
                if not args.no_driven:
                    extras["driven_32x32"] = driven_leg(args, dev, stream)
                extras["c4v_wedge_all_sources"] = wedge_leg(args, dev, stream, tuning)
                if not args.no_selfenergy:
                    extras["selfenergy_loop"] = selfenergy_leg(args, dev, stream)

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "tf32x3+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.lattice == 16 else
                       f"profiling case, not the benchmark: {args.lattice}x{args.lattice} lattice on the same contour",
                       "block_columns_per_step_per_gpu": args.batch,
                       "precision": "3xTF32 tcgen05 series sweeps + FP64 Dyson residual refinement",
                       "tol_rel_residual": args.tol, "lattice": [p.Lx, p.Ly], "Nc": Nc,
                       "l2": f"inputs larger than L2: {48 * Nr * Nc * Nc * args.batch / 1e9:.1f} GB of state per step",
                       "parallelism": f"block columns sharded over {world} GPU(s), no data-path collective"},
            "contour_gemm_tflops": tflops_local * world,
            "vector_columns_per_s": value * Nc,
            "sweeps_per_step": sweeps, "refinements_per_step": refinements, "max_rel_residual": residual,
            "autotune": {"sweep_variant": binding.SWEEP_NAMES[tuning["sweep_variant"]],
                         "variant_pinned": args.sweep_variant != "auto",
                         "chunk_block_columns": tuning["chunk_block_columns"],
                         "candidates": [(binding.SWEEP_NAMES[c["variant"]], c["chunk"],
                                         round(c["vector_columns_per_s"])) for c in tuning["candidates"]]},
            "roofline": roof, "rooflines": rooflines, "kernels": kernels, "clocks": clk,
            "gpu_launches": gpu_launches}
    line.update(extras)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    from paper_1309_5994_gb300 import dist
    rank, world, local = dist.env_ranks()
    if args.impl == "reference":
        run_reference(args, rank, world)      # rank 0 only; other ranks exit without work
        return
    dist.init("nccl")
    run_gb300(args, rank, world, local)


if __name__ == "__main__":
    main()
