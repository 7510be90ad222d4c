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

Also measured (single-GPU legs, N = 1): the same steps end to end through the C
ABI from host buffers (e2e); the plain FP64 GPU series on the sources of a
timed step (speed-up, and the timed step's error against the FP64 series run to
1e-12); the CPU oracle on a bounded sample (cpu_baseline, and the timed step's
error against the oracle's complex128 series on sampled vector columns); the
other workloads of the benchmark description (4x4 FP64, driven 32x32 streamed
in tuned chunks, the uneven batch, the 24x24 adjoint); the C4v wedge and the
self-consistency loop.  The TF32 and FP64 peaks the rooflines divide by are
measured at start-up (torch.matmul, best of several).  `--impl reference`
times the CPU oracle as the reference arm.
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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--batch", type=int, default=16, help="block columns per step per GPU")
    ap.add_argument("--tol", type=float, default=1e-6,
                    help="relative FP64 Dyson residual: the metric is quoted at relative error 1e-6; the "
                         "errors of a timed step's result against the FP64 series run to 1e-12 and against "
                         "the CPU oracle are measured and reported")
    ap.add_argument("--cpu-columns", type=int, default=32, help="vector columns in the CPU oracle timing sample")
    ap.add_argument("--no-extras", action="store_true", help="skip every leg after the timed region (profiling runs)")
    ap.add_argument("--uneven-instances", type=int, default=64,
                    help="instances of the seeded uneven batch in the batched-solve leg (0 skips it)")
    ap.add_argument("--driven-columns", type=int, default=6,
                    help="block columns of the driven 32x32 (Nc = 384) leg, streamed in tuned chunks (0 skips it)")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 24x24 adjoint leg")
    ap.add_argument("--no-selfenergy", action="store_true", help="skip the self-consistency loop leg")
    ap.add_argument("--graph-sweeps", type=int, default=16,
                    help="sweeps per captured graph of the inner series (0: one host synchronisation per sweep)")
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


def measure_matmul_peaks(dev):
    """Dense TF32 and FP64 rates of this GPU, measured here: torch.matmul of square
    matrices (float32 with TF32 allowed, 8192^3, best of 5; float64, 4096^3, best of 3),
    2 n^3 flops over CUDA-event time.  No GPU setting is changed."""
    import torch

    def best(dtype, n, reps):
        a = torch.randn(n, n, device=dev, dtype=dtype)
        b = torch.randn(n, n, device=dev, dtype=dtype)
        for _ in range(2):
            a @ b
        torch.cuda.synchronize(dev)
        ms = float("inf")
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            a @ b
            e1.record()
            torch.cuda.synchronize(dev)
            ms = min(ms, e0.elapsed_time(e1))
        del a, b
        return 2.0 * n ** 3 / (ms * 1e-3) / 1e12

    saved = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        tf32 = best(torch.float32, 8192, 5)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = saved
    fp64 = best(torch.float64, 4096, 3)
    torch.cuda.empty_cache()
    return {"tf32_tflops": tf32, "fp64_tflops": fp64,
            "how": "torch.matmul float32 with TF32 allowed 8192^3 (best of 5) and float64 4096^3 (best of 3), "
                   "2 n^3 flops over CUDA-event time, measured in this run"}


def bench_config(args, p, world):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": WORKLOAD if args.lattice == 16 else
            f"profiling case, not the benchmark: {args.lattice}x{args.lattice} lattice on the same contour",
            "block_columns_per_step_per_gpu": args.batch, "tol_rel_residual": args.tol,
            "lattice": [p.Lx, p.Ly], "Nc": p.Nc,
            # complex128 G, FP32 right-hand side and two FP32 states per vector column and site
            "l2": f"inputs larger than L2: {40 * p.Nr * p.Nc * p.Nc * args.batch / 1e9:.1f} GB of state per step",
            "parallelism": f"block columns sharded over {world} GPU(s), no data-path collective"}


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
# CPU oracle (the cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(p, site: int, zps, tol: float, S=None):
    """The CPU oracle's complex128 series on vector columns (site, z') of p, stopped at
    the relative update tol: (seconds, sweeps, G [Nr][Nc][len(zps)], setup)."""
    from oracle import dyson
    if S is None:
        S = dyson.setup(p)
    B = dyson.rhs_vector_columns(S, [(site, int(z)) for z in zps])
    t = time.perf_counter()
    G, sweeps, _ = dyson.neumann_solve(S, B, tol=tol, max_sweeps=400)
    dt = time.perf_counter() - t
    return dt, sweeps, G, S


def blas_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(n[0])
    except Exception:
        pass
    return os.cpu_count() or 1


def cpu_baseline_leg(p, ncols: int, tol: float, site: int, g_mixed=None):
    """The oracle timed on `ncols` vector columns of block column `site` (the cpu_baseline),
    then, untimed, its series to 1e-12 on 8 of those vector columns as the accuracy
    reference of the GPU's mixed-precision block column g_mixed [Nr][Nc][Nc] (if given)."""
    import numpy as np
    zps = np.linspace(0, p.Nc - 1, ncols).astype(int)
    dt, sweeps, _, S = oracle_sample(p, site, zps, tol)
    per_block = dt * p.Nc / ncols
    out = {"value": 1.0 / per_block, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
           "sample": (f"{ncols} of the 256 vector columns of block column {site}, complex128 series to {tol:g} "
                      f"({sweeps} sweeps, {dt:.2f} s), scaled linearly to one block column")}
    err = None
    if g_mixed is not None:
        zref = np.linspace(3, p.Nc - 4, 8).astype(int)
        _, sw_ref, Gref, _ = oracle_sample(p, site, zref, 1e-12, S)
        got = np.stack([g_mixed[:, :, z] for z in zref], axis=2)
        den = np.abs(Gref).max()
        diag = np.array([Gref[site, :, k] for k in range(len(zref))])
        diag_got = np.array([got[site, :, k] for k in range(len(zref))])
        err = {"reference": f"oracle complex128 series to 1e-12 ({sw_ref} sweeps), 8 vector columns of block "
                            f"column {site}",
               "G": float(np.abs(got - Gref).max() / den),
               "G_ii": float(np.abs(diag_got - diag).max() / np.abs(diag).max())}
    return out, err


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
        dt, _, _, _ = oracle_sample(p, site, zps, args.tol, S)
        if step >= args.warmup:
            times.append(dt * p.Nc / ncols)      # seconds per block column
    per_block = sum(times) / len(times)
    value = 1.0 / per_block
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_block * 1e3 * ncols / p.Nc,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
            "config": bench_config(args, p, world),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
                             "sample": f"each step: {ncols} vector columns of one block column, complex128 series "
                                       f"to {args.tol:g}, scaled to block columns"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# single-GPU legs
# ---------------------------------------------------------------------------
def plain_f64_leg(args, dev, solver, sources, PREC, value_per_gpu):
    """The plain FP64 GPU series on the sources of the first timed step, at the timed
    step's tolerance (speed-up), and the timed step's own result (re-solved on the same
    chunk, so bit for bit the timed computation) against the FP64 series run to 1e-12 on
    two of those sources.  Returns (leg record, errors, speed-up, mixed G of sources[0])."""
    import numpy as np
    import torch
    from paper_1309_5994_gb300 import binding
    p = solver.p
    Nr, Nc = p.Nr, p.Nc
    nq = len(sources)
    solver.build_sigma()
    gmx = torch.empty((nq, Nr, Nc, Nc), dtype=torch.complex128, device=dev)
    rmx = solver.solve(sources, precision=PREC, tol=args.tol, max_sweeps=400, g_out=gmx)
    nmx, _, _ = solver.observables()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r64 = solver.solve(sources, precision=binding.PREC_F64, tol=args.tol, max_sweeps=400, allow=(0, -3))
    torch.cuda.synchronize(dev)
    t64 = time.perf_counter() - t0
    two = sources[:2]
    g64 = torch.empty((2, Nr, Nc, Nc), dtype=torch.complex128, device=dev)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r64t = solver.solve(two, precision=binding.PREC_F64, tol=1e-12, max_sweeps=400, g_out=g64, allow=(0, -3))
    torch.cuda.synchronize(dev)
    t64t = time.perf_counter() - t0
    n64, _, _ = solver.observables()
    den = torch.abs(g64).max().item()
    gerr = torch.abs(gmx[:2] - g64).max().item() / den
    gii = torch.stack([g64[q, s] for q, s in enumerate(two)])
    gii_m = torch.stack([gmx[q, s] for q, s in enumerate(two)])
    gii_err = (torch.abs(gii_m - gii).max() / torch.abs(gii).max()).item()
    nerr = float(np.abs(nmx[two] - n64[two]).max() / np.abs(n64[two]).max())
    f64_rate = nq / t64
    g0 = gmx[0].cpu().numpy()
    del gmx, g64
    torch.cuda.empty_cache()
    leg = {"value": f64_rate, "unit": UNIT, "block_columns": nq, "sources": "those of the first timed step",
           "tol_rel_update": args.tol, "sweeps": r64.report["sweeps"], "status": r64.status,
           "tflops": r64.report["gemm_flops"] / t64 / 1e12,
           "tight": {"tol_rel_update": 1e-12, "block_columns": 2, "value": 2 / t64t, "unit": UNIT,
                     "sweeps": r64t.report["sweeps"], "final_update": r64t.report["update"]},
           "mixed_resolve_residual": rmx.report["residual"]}
    err = {"reference": "FP64 GPU series to 1e-12 on 2 of the step's sources", "G": gerr, "G_ii": gii_err,
           "density": nerr}
    return leg, err, value_per_gpu / f64_rate, g0


def trapped_4x4_leg(args, dev, stream):
    """The 4x4 trapped lattice (Nc = 64) in the plain FP64 path: all 16 block columns
    to an update of 1e-12 (its parity with the oracle's dense solve at 1e-12 is
    tests/test_gpu_parity.py::test_trapped_4x4_all_columns_and_observables)."""
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    p = wl.trapped_4x4_nc64()
    s = binding.Solver(p, device=dev.index, stream=stream)
    s.build_sigma()
    src = list(range(p.Nr))
    s.solve(src, precision=binding.PREC_F64, tol=1e-12)
    reps = 5
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(reps):
        r = s.solve(src, precision=binding.PREC_F64, tol=1e-12)
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t0) / reps
    s.close()
    return {"value": p.Nr / dt, "unit": UNIT, "seconds": dt, "sweeps": r.report["sweeps"],
            "final_update": r.report["update"], "tflops": r.report["gemm_flops"] / dt / 1e12}


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
    # instances whose series diverges (spectral radius of Lambda W J above 1) end with
    # DIVERGED in the batch; the paper hands those to GMRES, which finishes them below
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
           "seconds": t_batch, "contour_gemm_tflops": flops / t_batch / 1e12,
           "sequential_value": len(conv) / t_seq, "speedup_vs_sequential": t_seq / t_batch,
           "sweeps_max": max(r.report["sweeps"] for r in res),
           "max_rel_residual_converged": max(res[k].report["residual"] for k in conv) if conv else None,
           "graph_kernel_launches": graph_launches}
    batch.close()
    for s in solvers:
        s.close()
    return out


def driven_leg(args, dev, stream):
    """The driven 32x32 lattice (Nc = 384, U(t) = 20(1 + 0.1 sin 20t), J(t) = 1 - 0.2 sin 20t):
    `--driven-columns` block columns around the trap centre in mixed precision, streamed in
    the chunks and sweep variant the autotuner picks (the FP32 series cannot serve on this
    contour, so the AUTO inner solver runs GMRES), against the plain FP64 series on one
    of them run for 105 sweeps, where its update reaches its floor."""
    import numpy as np
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    p = wl.driven_32x32_nc384()
    s = binding.Solver(p, device=dev.index, stream=stream)
    s.build_sigma()
    tuning = s.autotune(args.driven_columns)
    c0 = p.Nr // 2 + p.Lx // 2
    src = [(c0 + 37 * q) % p.Nr for q in range(args.driven_columns)]
    s.solve(src[:1], precision=binding.PREC_TF32X3_F64REF, tol=args.tol, max_sweeps=400)   # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rm = s.solve(src, precision=binding.PREC_TF32X3_F64REF, tol=args.tol, max_sweeps=400)
    torch.cuda.synchronize(dev)
    t_mixed = time.perf_counter() - t0
    n_mixed = s.observables()[0][src[0]].copy()
    t0 = time.perf_counter()
    rf = s.solve(src[:1], precision=binding.PREC_F64, tol=1e-15, max_sweeps=105, allow=(0, -3))
    torch.cuda.synchronize(dev)
    t_f64 = time.perf_counter() - t0
    n_f64 = s.observables()[0][src[0]].copy()
    s.close()
    per_col = t_mixed / len(src)
    return {"value": len(src) / t_mixed, "unit": UNIT, "block_columns": len(src),
            "chunk_block_columns": tuning["chunk_block_columns"],
            "sweep_variant": binding.SWEEP_NAMES[tuning["sweep_variant"]], "chunks": rm.report["chunks"],
            "matvecs": rm.report["sweeps"], "refinements": rm.report["refinements"],
            "rel_residual": rm.report["residual"], "inner_solver": "gmres" if rm.report["inner_gmres"] else "series",
            "plain_f64_seconds_per_block_column": t_f64, "plain_f64_final_update": rf.report["update"],
            "speedup_vs_plain_f64": t_f64 / per_col,
            "density_rel_diff_mixed_vs_f64": float(np.abs(n_mixed - n_f64).max() / np.abs(n_f64).max())}


def adjoint_leg(args, dev, stream):
    """The adjoint on the 24x24 lattice (Nc = 256, the driven lattice's drive scaled by
    an amplitude s): L = sum_i w_i n_i(t_final), its gradients with respect to every
    U_i(t_k) and J_b(t_k) (forward vector columns, transposed solves, contractions), and
    dL/ds through the chain rule against central differences of L with h = 1e-4."""
    import numpy as np
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    w = wl.loss_weights()
    base = wl.driven_24x24_nc256(1.0)
    s = binding.Solver(base, device=dev.index, stream=stream)
    s.build_sigma()
    s.adjoint(w, precision=binding.PREC_TF32X3_F64REF, tol=1e-11)                 # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    L0, gU, gJ, res = s.adjoint(w, precision=binding.PREC_TF32X3_F64REF, tol=1e-11)
    torch.cuda.synchronize(dev)
    t_grad = time.perf_counter() - t0
    s.close()
    dU, dJ = wl.drive_derivative_tables(base)
    chain = float(np.sum(gU * dU) + np.sum(gJ * dJ))
    h = 1e-4
    vals = []
    for amp in (1.0 + h, 1.0 - h):
        sp = binding.Solver(wl.driven_24x24_nc256(amp), device=dev.index, stream=stream)
        sp.build_sigma()
        vals.append(sp.adjoint(w, precision=binding.PREC_TF32X3_F64REF, tol=1e-11)[0])
        sp.close()
    fd = (vals[0] - vals[1]) / (2 * h)
    return {"seconds_per_gradient": t_grad, "gradients_per_s": 1.0 / t_grad, "loss": L0,
            "gradient_entries": int(gU.size + gJ.size), "dL_ds_adjoint": chain, "dL_ds_central_difference": fd,
            "rel_diff": abs(fd - chain) / max(abs(fd), 1e-300)}


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
    s.observables()
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    s.close()
    return {"sources": p.Nr, "representatives_solved": 36, "status": r.status, "seconds": dt,
            "site_observables_per_s": p.Nr / dt}


def selfenergy_leg(args, dev, stream, fp64_peak):
    """The self-consistency loop of Sec. IV.C (self-energy steps between lattice solves) on a
    driven 8x8 trapped lattice, Nc = 64 (24 + 24 real-time points dt = 0.05, 16 imaginary),
    U(t) = 20 (1 + 0.1 sin 20t), J(t) = 1 - 0.2 sin 20t, trap 0.02 |r|^2, beta = 2: all 64 block
    columns per iteration in mixed precision (residual 1e-10), mixing 0.7, until the paper's
    measure (taken on Sigma~) falls to 1e-8 (at most 40 iterations); then with Anderson
    acceleration, and with Anderson and the C4v reduction."""
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding
    from paper_1309_5994_gb300.selfconsistency import self_consistent
    p = wl.uniform_problem("se_L8_Nc64_driven", 8, 24, 16, 0.05, 2.0, 0.0, 0.02, 20.0, 1.0,
                           aU=0.1, aJ=0.2, omega=20.0)
    s = binding.Solver(p, device=dev.index, stream=stream)
    s.build_sigma()
    s.local_greens(None, precision=binding.PREC_TF32X3_F64REF, tol=1e-10)     # warm-up: tables, buffers
    out = {}
    for name, kw, sym in (("linear", {}, False), ("anderson5", {"anderson": 5}, False),
                          ("anderson5_c4v", {"anderson": 5}, True)):
        if sym:
            s.set_symmetry(binding.SYMMETRY_C4V)
        s.build_sigma()
        s.profile(True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = self_consistent(s, mix=0.7, max_iter=40, precision=binding.PREC_TF32X3_F64REF, tol=1e-10, **kw)
        torch.cuda.synchronize(dev)
        secs = time.perf_counter() - t0
        n_conn, ms_conn = s.profile_query(binding.KERNEL_SELFENERGY)
        s.profile(False)
        out[name] = {"iterations": r["iterations"], "converged": r["converged"],
                     "criterion": float(f"{r['history'][-1]:.3e}"), "seconds": round(secs, 4)}
        if name == "linear" and n_conn:
            # executed FP64 work of the connected contraction: per site and (a, b, d) one
            # complex FMA pair per imaginary point and per real-branch interval (4), i.e.
            # (16 Nm + 64) Nc^3 flops (the per-(a, b, d) coefficient tables excluded)
            flops = (16.0 * p.Nm + 64.0) * p.Nc ** 3 * p.Nr
            ach = flops / (ms_conn / n_conn * 1e-3) / 1e12
            out["selfenergy_conn"] = {"avg_ms": ms_conn / n_conn, "share_of_loop": ms_conn * 1e-3 / secs,
                                      "roofline": {"bound": "alu", "achieved": ach, "peak": fp64_peak,
                                                   "unit": "TFLOP/s", "frac": ach / fp64_peak,
                                                   "peak_source": "FP64 matmul rate measured in this run"}}
    s.close()
    return out


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gb300(args, rank, world, local):
    import torch
    import workloads as wl
    from paper_1309_5994_gb300 import binding, dist

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = wl.trapped_16x16_nc256() if args.lattice == 16 else wl.uniform_problem(
        f"trapped_L{args.lattice}_Nc256", args.lattice, 112, 32, 0.05, 2.0, 0.0, 0.02, 20.0, 1.0)
    stream = torch.cuda.Stream(device=dev)
    mm = measure_matmul_peaks(dev)
    solver = binding.Solver(p, device=local, stream=stream)
    solver.set_graph_sweeps(args.graph_sweeps)
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
    host_syncs = [r["host_syncs"] for r in reports]
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
    slices = 15 if args.tol >= 1e-8 else 28
    rooflines = {}
    for name, (n, ms) in kstats.items():
        if not n or name == "selfenergy_conn":
            continue
        dur = ms / n * 1e-3
        if name == "gather_tc":
            ach = 2 * state_bytes / dur / 1e9
            peak = peaks["hbm_gbs"]
            r = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                 "peak_source": f"{peak_src} copy bandwidth; bytes = read d + write X (FP32 planar state)"}
        elif name in ("sweep_f64", "residual_f64"):
            ach = alg_flops / dur / 1e12
            r = {"bound": "alu", "achieved": ach, "peak": mm["fp64_tflops"], "unit": "TFLOP/s",
                 "frac": ach / mm["fp64_tflops"], "peak_source": "FP64 matmul rate measured in this run"}
        elif name == "residual_split_bf16":
            ach = alg_flops / dur / 1e12
            peak = peaks["bf16_tflops"]
            r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                 "executed_tflops": slices * ach, "executed_frac": slices * ach / peak,
                 "peak_source": f"{peak_src} bf16 burst; {note}; the slice split executes {slices} BF16 products"}
        else:
            ach = alg_flops / dur / 1e12
            peak = mm["tf32_tflops"]
            r = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                 "executed_tflops": 3 * ach, "executed_frac": 3 * ach / peak,
                 "peak_source": f"TF32 matmul rate measured in this run; {note}; the 3xTF32 split executes 3x"}
        r["traffic"] = traffic.get(name)
        r["kernel"] = name
        r["avg_ms"] = ms / n
        rooflines[name] = r
    dom_name = max(kstats.items(), key=lambda kv: kv[1][1])[0]
    roof = rooflines[dom_name]
    total_ms = max(sum(v[1] for v in kstats.values()), 1e-9)
    kernels = {nm: {"launches": n, "avg_ms": round(ms / n, 4), "share": round(ms / total_ms, 4)}
               for nm, (n, ms) in kstats.items() if n}

    extras, summary = {}, {}
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
            s2.set_graph_sweeps(args.graph_sweeps)
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
        # the single-GPU legs run at N = 1 only: with more ranks every GPU would wait for them
        if world == 1:
            first = dist.step_sources(p.Nr, args.batch, rank, world, args.warmup)
            leg, err_f64, speedup, g0 = plain_f64_leg(args, dev, solver, first, PREC, value)
            extras["plain_f64"] = leg
            extras["cpu_baseline"], err_oracle = cpu_baseline_leg(p, args.cpu_columns, args.tol, first[0], g0)
            del g0
            summary["speedup_vs_plain_f64"] = speedup
            summary["rel_err_timed_step"] = {"vs_f64_series": err_f64, "vs_oracle": err_oracle,
                                             "within_1e-6": bool(max(err_f64["G_ii"], err_f64["density"],
                                                                     err_oracle["G_ii"]) <= 1e-6)}
            cfg = {"trapped_16x16_nc256": {"value": value, "unit": UNIT, "tflops": tflops_local,
                                           "dominant_kernel_frac": roof["frac"]}}
            cfg["trapped_4x4_nc64_f64"] = trapped_4x4_leg(args, dev, stream)
            if args.driven_columns > 0:
                cfg["driven_32x32_nc384"] = driven_leg(args, dev, stream)
            if args.uneven_instances > 0:
                cfg["uneven_batch"] = batched_uneven_leg(args, dev, stream)
            if not args.no_adjoint:
                cfg["adjoint_24x24_nc256"] = adjoint_leg(args, dev, stream)
            extras["c4v_wedge_all_sources"] = wedge_leg(args, dev, stream, tuning)
            if not args.no_selfenergy:
                extras["selfenergy_loop"] = selfenergy_leg(args, dev, stream, mm["fp64_tflops"])
            summary["configs"] = cfg
            extras["configs"] = cfg

    if rank != 0:
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": max_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "tf32x3+f64", "data": "synthetic",
            "config": bench_config(args, p, world),
            "precision": "3xTF32 tcgen05 series sweeps + FP64 Dyson residual refinement",
            "measured_peaks": mm, "rooflines": rooflines, "kernels": kernels,
            "autotune": {"sweep_variant": binding.SWEEP_NAMES[tuning["sweep_variant"]],
                         "variant_pinned": args.sweep_variant != "auto",
                         "chunk_block_columns": tuning["chunk_block_columns"],
                         "candidates": [(binding.SWEEP_NAMES[c["variant"]], c["chunk"],
                                         round(c["vector_columns_per_s"])) for c in tuning["candidates"]]},
            "contour_gemm_tflops": tflops_local * world, "vector_columns_per_s": value * Nc,
            "sweeps_per_step": sweeps, "refinements_per_step": refinements, "max_rel_residual": residual,
            "host_syncs_per_step": host_syncs, "graph_sweeps": args.graph_sweeps,
            "clocks": clk, "gpu_launches": gpu_launches, "roofline": roof}
    line.update(extras)
    # the verification summary closes the line (compact, rounded), so that a kept tail of
    # the output shows it
    if summary:
        line["summary"] = compact_summary(summary, roof)
    print(json.dumps(line), flush=True)


def _r(x, digits=3):
    if isinstance(x, float):
        return float(f"{x:.{digits}g}")
    if isinstance(x, dict):
        return {k: _r(v, digits) for k, v in x.items() if k not in ("reference", "unit")}
    return x


def compact_summary(summary, roof):
    cfg = summary.get("configs", {})
    out = {"speedup_vs_plain_f64": _r(summary.get("speedup_vs_plain_f64")),
           "err_vs_f64_series_1e-12": _r(summary["rel_err_timed_step"]["vs_f64_series"]),
           "err_vs_oracle_1e-12": _r(summary["rel_err_timed_step"]["vs_oracle"]),
           "within_1e-6": summary["rel_err_timed_step"]["within_1e-6"],
           "dominant_kernel": {"name": roof["kernel"], "frac": _r(roof["frac"]),
                               "executed_frac": _r(roof.get("executed_frac"))}}
    c = cfg.get("trapped_16x16_nc256")
    if c:
        out["c2_16x16"] = {"value": _r(c["value"]), "tflops": _r(c["tflops"])}
    c = cfg.get("trapped_4x4_nc64_f64")
    if c:
        out["c1_4x4_f64"] = {"value": _r(c["value"]), "update": _r(c["final_update"])}
    c = cfg.get("driven_32x32_nc384")
    if c:
        out["c3_driven"] = {"value": _r(c["value"]), "cols": c["block_columns"], "chunk": c["chunk_block_columns"],
                            "residual": _r(c["rel_residual"]), "speedup_vs_f64": _r(c["speedup_vs_plain_f64"]),
                            "dn_vs_f64": _r(c["density_rel_diff_mixed_vs_f64"])}
    c = cfg.get("uneven_batch")
    if c:
        out["c4_uneven"] = {"value": _r(c["value"]), "converged": c["block_columns_converged"],
                            "speedup_vs_seq": _r(c["speedup_vs_sequential"])}
    c = cfg.get("adjoint_24x24_nc256")
    if c:
        out["c5_adjoint"] = {"s_per_gradient": _r(c["seconds_per_gradient"]), "fd_rel_diff": _r(c["rel_diff"])}
    return out


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
