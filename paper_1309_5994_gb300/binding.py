"""ctypes binding of libdyson.so (the C ABI of include/dyson.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Loading fails with an exception when the library has not been built;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libdyson.so")
_lib = None

DYSON_OK = 0
ERR_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "NOT_CONVERGED", -4: "DIVERGED", -5: "TIMEOUT",
             -6: "CUDA", -7: "STATE"}
PREC_F64 = 0
PREC_TF32X3_F64REF = 1
KERNEL_SWEEP_F64, KERNEL_SWEEP_F32, KERNEL_SWEEP_TC, KERNEL_RESIDUAL_F64, KERNEL_RESIDUAL_SPLIT = 0, 1, 2, 3, 4
KERNEL_SWEEP_TC_PAIR, KERNEL_GATHER_TC, KERNEL_SELFENERGY, KERNEL_SWEEP_TC_FUSED = 5, 6, 7, 8
KERNEL_NAMES = {0: "sweep_f64", 1: "sweep_f32_simt", 2: "sweep_tc_3xtf32", 3: "residual_f64",
                4: "residual_split_bf16", 5: "sweep_tc_3xtf32_pair", 6: "gather_tc", 7: "selfenergy_conn",
                8: "sweep_tc_fused"}


class Lattice(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32)]


class Contour(C.Structure):
    _fields_ = [("Nt", C.c_int32), ("Nm", C.c_int32), ("dt", C.c_double), ("beta", C.c_double)]


class Trap(C.Structure):
    _fields_ = [("curvature", C.c_double), ("mu", C.c_double)]


class Drive(C.Structure):
    _fields_ = [("U", C.POINTER(C.c_double)), ("J", C.POINTER(C.c_double))]


class Tuning(C.Structure):
    _fields_ = [("sweep_variant", C.c_int32), ("chunk_block_columns", C.c_int32),
                ("vector_columns_per_s", C.c_double), ("n_candidates", C.c_int32),
                ("cand_variant", C.c_int32 * 32), ("cand_chunk", C.c_int32 * 32),
                ("cand_vector_columns_per_s", C.c_double * 32)]

    def as_dict(self):
        n = self.n_candidates
        return {"sweep_variant": self.sweep_variant, "chunk_block_columns": self.chunk_block_columns,
                "vector_columns_per_s": self.vector_columns_per_s,
                "candidates": [{"variant": self.cand_variant[k], "chunk": self.cand_chunk[k],
                                "vector_columns_per_s": self.cand_vector_columns_per_s[k]} for k in range(n)]}


class Report(C.Structure):
    _fields_ = [("sweeps", C.c_int32), ("refinements", C.c_int32), ("chunks", C.c_int32),
                ("status", C.c_int32), ("update", C.c_double), ("residual", C.c_double),
                ("gemm_flops", C.c_double), ("seconds", C.c_double), ("kernel_launches", C.c_int64),
                ("inner_gmres", C.c_int32), ("host_syncs", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["dyson_init", "dyson_build_sigma", "dyson_copy_sigma", "dyson_solve_columns",
           "dyson_observables", "dyson_solve_vector_columns", "dyson_transpose_sigma", "dyson_adjoint",
           "dyson_profile", "dyson_profile_query", "dyson_set_chunk",
           "dyson_launch_count", "dyson_destroy", "dyson_last_error", "dyson_version",
           "dyson_solve_block_column_noalloc", "dyson_noalloc_last_error", "dyson_set_sweep_variant",
           "dyson_set_wait_limit", "dyson_set_graph_sweeps",
           "dyson_batch_create", "dyson_batch_solve", "dyson_batch_launch_count", "dyson_batch_last_error",
           "dyson_batch_destroy", "dyson_set_inner_solver", "dyson_autotune", "dyson_set_symmetry",
           "dyson_adjoint_obs", "dyson_extrapolate_dt", "dyson_set_support_truncation", "dyson_local_greens",
           "dyson_selfenergy_step", "dyson_selfenergy_set_anderson"]
SYMMETRY_NONE, SYMMETRY_C4V = 0, 1
INNER_SERIES, INNER_GMRES, INNER_AUTO = 0, 1, 2
SWEEP_SINGLE_CTA, SWEEP_CTA_PAIR, SWEEP_FUSED_PAIR, SWEEP_FUSED_PAIR_WIDE = 0, 1, 2, 3
SWEEP_NAMES = ["single_cta", "cta_pair", "fused_pair", "fused_pair_wide"]


def load(path: str = _LIB_PATH):
    """Load libdyson.so and declare the signatures of include/dyson.h."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run __graft_entry__.build() (no CPU fallback exists)")
    lib = C.CDLL(path)
    P = C.c_void_p
    lib.dyson_init.argtypes = [C.POINTER(P), C.POINTER(Lattice), C.POINTER(Contour), C.POINTER(Trap),
                               C.POINTER(Drive), C.c_int, P]
    lib.dyson_build_sigma.argtypes = [P]
    lib.dyson_copy_sigma.argtypes = [P, P, C.c_int]
    lib.dyson_solve_columns.argtypes = [P, C.POINTER(C.c_int32), C.c_int64, C.c_int, C.c_double, C.c_int32, P,
                                        C.POINTER(Report)]
    lib.dyson_observables.argtypes = [P, P, P, P, C.c_int]
    lib.dyson_solve_vector_columns.argtypes = [P, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.c_int64, C.c_int,
                                               C.c_double, C.c_int32, P, C.POINTER(Report)]
    lib.dyson_transpose_sigma.argtypes = [P]
    lib.dyson_adjoint.argtypes = [P, P, C.c_int32, C.c_int, C.c_double, C.c_int32, P, P, P, C.POINTER(Report)]
    lib.dyson_adjoint_obs.argtypes = [P, P, P, C.c_int32, C.c_int, C.c_double, C.c_int32, P, P, P,
                                      C.POINTER(Report)]
    lib.dyson_profile.argtypes = [P, C.c_int]
    lib.dyson_profile_query.argtypes = [P, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double)]
    lib.dyson_set_chunk.argtypes = [P, C.c_int32]
    lib.dyson_set_sweep_variant.argtypes = [P, C.c_int]
    lib.dyson_set_wait_limit.argtypes = [P, C.c_double]
    lib.dyson_set_graph_sweeps.argtypes = [P, C.c_int]
    lib.dyson_set_inner_solver.argtypes = [P, C.c_int, C.c_int32]
    lib.dyson_autotune.argtypes = [P, C.c_int32, C.POINTER(Tuning)]
    lib.dyson_set_symmetry.argtypes = [P, C.c_int]
    lib.dyson_set_support_truncation.argtypes = [P, C.c_int]
    lib.dyson_local_greens.argtypes = [P, C.POINTER(C.c_int32), C.c_int64, C.c_int, C.c_double, C.c_int32, P,
                                       C.POINTER(Report)]
    lib.dyson_selfenergy_step.argtypes = [P, P, C.c_double, P, C.POINTER(C.c_double)]
    lib.dyson_selfenergy_set_anderson.argtypes = [P, C.c_int32]
    lib.dyson_launch_count.argtypes = [P]
    lib.dyson_launch_count.restype = C.c_int64
    lib.dyson_solve_block_column_noalloc.argtypes = [P, P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_double,
                                                     C.c_double, C.c_int32, C.c_double, C.c_int32, P,
                                                     C.POINTER(C.c_int32), P]
    lib.dyson_noalloc_last_error.restype = C.c_char_p
    lib.dyson_batch_create.argtypes = [C.POINTER(P), C.POINTER(P), C.c_int32]
    lib.dyson_batch_solve.argtypes = [P, C.POINTER(C.POINTER(C.c_int32)), C.POINTER(C.c_int32), C.c_double,
                                      C.c_int32, C.c_int32, C.POINTER(P), C.POINTER(Report)]
    lib.dyson_batch_launch_count.argtypes = [P]
    lib.dyson_batch_launch_count.restype = C.c_int64
    lib.dyson_batch_last_error.argtypes = [P]
    lib.dyson_batch_last_error.restype = C.c_char_p
    lib.dyson_batch_destroy.argtypes = [P]
    lib.dyson_batch_destroy.restype = None
    lib.dyson_destroy.argtypes = [P]
    lib.dyson_destroy.restype = None
    lib.dyson_last_error.argtypes = [P]
    lib.dyson_last_error.restype = C.c_char_p
    lib.dyson_version.restype = C.c_char_p
    lib.dyson_extrapolate_dt.argtypes = [C.c_int32, C.POINTER(P), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                         C.c_int32, P, C.c_int, P]
    _lib = lib
    return lib


class DysonError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def extrapolate_dt(tables, m, out=None, stream=None):
    """Delta t -> 0 extrapolation (dyson_extrapolate_dt) of float64 device tensors
    tables[b] of shape [rows, nt_b] computed on contours of step h_0 / m[b];
    returns out, [rows, nt_0] on the device of tables[0]."""
    import torch
    lib = load()
    n = len(tables)
    t0 = tables[0]
    for t in tables:
        if t.dtype != torch.float64 or not t.is_cuda or t.dim() != 2 or not t.is_contiguous():
            raise ValueError("tables must be contiguous 2-D float64 CUDA tensors")
        if t.shape[0] != t0.shape[0] or t.device != t0.device:
            raise ValueError("tables must share rows and device")
    if out is None:
        out = torch.empty_like(t0)
    if stream is None:
        stream = torch.cuda.current_stream(t0.device)
    ptrs = (C.c_void_p * n)(*[t.data_ptr() for t in tables])
    nt = (C.c_int32 * n)(*[t.shape[1] for t in tables])
    mm = (C.c_int32 * n)(*[int(x) for x in m])
    rc = lib.dyson_extrapolate_dt(n, ptrs, nt, mm, t0.shape[0], C.c_void_p(out.data_ptr()), t0.device.index,
                                  C.c_void_p(stream.cuda_stream))
    if rc != 0:
        raise DysonError(rc, lib.dyson_last_error(None).decode())
    return out


@dataclass
class SolveResult:
    status: int
    report: dict


def device_buffer(t, dtype, numel: int, device, name: str):
    """Raw pointer of the tensor `t` for a DEVICE argument of the C ABI, after checking
    that it is a contiguous CUDA tensor of `dtype` with `numel` elements on GPU `device`
    (None: any).  The library takes the pointer as it is, so a host or mis-sized tensor
    is refused here, before any kernel could touch it."""
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous {dtype} CUDA tensor")
    if t.numel() != numel:
        raise ValueError(f"{name} must hold {numel} elements, not {t.numel()}")
    if device is not None and t.device.index != device:
        raise ValueError(f"{name} is on cuda:{t.device.index}; the context is on cuda:{device}")
    return C.c_void_p(t.data_ptr())


class Solver:
    """One context of the C ABI for a workloads.Problem-like object.

    `stream` is a torch.cuda.Stream (or None for torch's current stream).
    """

    def __init__(self, problem, device: int = 0, stream=None):
        import torch
        self.lib = load()
        self.p = problem
        self._torch = torch
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        self._U = np.ascontiguousarray(problem.U, dtype=np.float64)
        self._J = np.ascontiguousarray(problem.J, dtype=np.float64)
        lat = Lattice(problem.Lx, problem.Ly)
        con = Contour(problem.Nt, problem.Nm, problem.dt, problem.beta)
        trap = Trap(problem.trap_c, problem.mu)
        drv = Drive(self._U.ctypes.data_as(C.POINTER(C.c_double)), self._J.ctypes.data_as(C.POINTER(C.c_double)))
        h = C.c_void_p()
        rc = self.lib.dyson_init(C.byref(h), C.byref(lat), C.byref(con), C.byref(trap), C.byref(drv), device,
                                 C.c_void_p(stream.cuda_stream))
        if rc != 0:
            raise DysonError(rc, self.lib.dyson_last_error(None).decode())
        self.h = h
        self.device = device

    def _check(self, rc, ok=(0,)):
        if rc not in ok:
            raise DysonError(rc, self.lib.dyson_last_error(self.h).decode())
        return rc

    def build_sigma(self):
        self._check(self.lib.dyson_build_sigma(self.h))

    def sigma(self):
        """Lambda as a host complex128 array [Nr, Nc, Nc]."""
        out = np.empty((self.p.Nr, self.p.Nc, self.p.Nc), dtype=np.complex128)
        self._check(self.lib.dyson_copy_sigma(self.h, out.ctypes.data, 0))
        return out

    def solve(self, sources, precision=PREC_F64, tol=1e-13, max_sweeps=400, g_out=None, allow=(0,)):
        """Solve block columns for `sources`; g_out: optional complex128 device tensor
        of shape [len(sources), Nr, Nc, Nc].  Returns SolveResult."""
        src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32))
        rep = Report()
        gptr = None
        if g_out is not None:
            gptr = device_buffer(g_out, self._torch.complex128, len(src) * self.p.Nr * self.p.Nc * self.p.Nc,
                                 self.device, "g_out")
        rc = self.lib.dyson_solve_columns(self.h, src.ctypes.data_as(C.POINTER(C.c_int32)), len(src), precision,
                                          tol, max_sweeps, gptr, C.byref(rep))
        self._check(rc, ok=allow)
        return SolveResult(rc, rep.as_dict())

    def solve_vectors(self, sites, times, precision=PREC_F64, tol=1e-13, max_sweeps=400, g_out=None, allow=(0,)):
        """Solve vector columns (sites[q], times[q]); g_out: optional complex128 device
        tensor of shape [n, Nr, Nc].  Returns SolveResult."""
        s = np.ascontiguousarray(np.asarray(sites, dtype=np.int32))
        t = np.ascontiguousarray(np.asarray(times, dtype=np.int32))
        if s.shape != t.shape:
            raise ValueError("sites and times must have the same length")
        rep = Report()
        gptr = None
        if g_out is not None:
            gptr = device_buffer(g_out, self._torch.complex128, len(s) * self.p.Nr * self.p.Nc, self.device,
                                 "g_out")
        rc = self.lib.dyson_solve_vector_columns(self.h, s.ctypes.data_as(C.POINTER(C.c_int32)),
                                                 t.ctypes.data_as(C.POINTER(C.c_int32)), len(s), precision, tol,
                                                 max_sweeps, gptr, C.byref(rep))
        self._check(rc, ok=allow)
        return SolveResult(rc, rep.as_dict())

    def adjoint(self, w, t_index=None, precision=PREC_TF32X3_F64REF, tol=1e-11, max_sweeps=400, allow=(0,)):
        """(loss, dL/dU [Nr, Nt], dL/dJ [Nb, Nt], SolveResult) of L = sum_i w_i n_i(t_index)."""
        t_index = self.p.Nt - 1 if t_index is None else t_index
        w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
        if w.shape != (self.p.Nr,):
            raise ValueError(f"w must have shape ({self.p.Nr},)")
        loss = C.c_double()
        gU = np.zeros((self.p.Nr, self.p.Nt))
        gJ = np.zeros((max(self.p.Nb, 1), self.p.Nt))
        rep = Report()
        rc = self.lib.dyson_adjoint(self.h, w.ctypes.data, t_index, precision, tol, max_sweeps, C.byref(loss),
                                    gU.ctypes.data, gJ.ctypes.data, C.byref(rep))
        self._check(rc, ok=allow)
        return loss.value, gU, gJ[:self.p.Nb], SolveResult(rc, rep.as_dict())

    def adjoint_obs(self, w_density=None, w_docc=None, t_index=None, precision=PREC_TF32X3_F64REF, tol=1e-11,
                    max_sweeps=400, allow=(0,)):
        """(loss, dL/dU, dL/dJ, SolveResult) of L = sum_i w_density_i n_i(t) + w_docc_i D_i(t)."""
        t_index = self.p.Nt - 1 if t_index is None else t_index
        wn = None if w_density is None else np.ascontiguousarray(np.asarray(w_density, dtype=np.float64))
        wd = None if w_docc is None else np.ascontiguousarray(np.asarray(w_docc, dtype=np.float64))
        for nm, a in (("w_density", wn), ("w_docc", wd)):
            if a is not None and a.shape != (self.p.Nr,):
                raise ValueError(f"{nm} must have shape ({self.p.Nr},)")
        loss = C.c_double()
        gU = np.zeros((self.p.Nr, self.p.Nt))
        gJ = np.zeros((max(self.p.Nb, 1), self.p.Nt))
        rep = Report()
        rc = self.lib.dyson_adjoint_obs(self.h, None if wn is None else wn.ctypes.data,
                                        None if wd is None else wd.ctypes.data, t_index, precision, tol, max_sweeps,
                                        C.byref(loss), gU.ctypes.data, gJ.ctypes.data, C.byref(rep))
        self._check(rc, ok=allow)
        return loss.value, gU, gJ[:self.p.Nb], SolveResult(rc, rep.as_dict())

    def transpose_sigma(self):
        self._check(self.lib.dyson_transpose_sigma(self.h))

    def observables(self):
        """(n, ekin, D) as host numpy arrays [Nr, Nt]."""
        shape = (self.p.Nr, self.p.Nt)
        n, e, d = (np.empty(shape) for _ in range(3))
        self._check(self.lib.dyson_observables(self.h, n.ctypes.data, e.ctypes.data, d.ctypes.data, 0))
        return n, e, d

    def observables_device(self, n, ekin, docc):
        """(n, ekin, D) into float64 device tensors of Nr * Nt elements each."""
        size, f64 = self.p.Nr * self.p.Nt, self._torch.float64
        ptrs = [device_buffer(t, f64, size, self.device, nm) for t, nm in ((n, "n"), (ekin, "ekin"), (docc, "docc"))]
        self._check(self.lib.dyson_observables(self.h, *ptrs, 1))

    def launch_count(self) -> int:
        return int(self.lib.dyson_launch_count(self.h))

    def set_chunk(self, cols: int):
        self._check(self.lib.dyson_set_chunk(self.h, cols))

    def set_symmetry(self, mode: int):
        self._check(self.lib.dyson_set_symmetry(self.h, mode))

    def autotune(self, max_block_columns: int) -> dict:
        """Time the sweep candidates on this context, keep the fastest; returns the report."""
        t = Tuning()
        self._check(self.lib.dyson_autotune(self.h, max_block_columns, C.byref(t)))
        return t.as_dict()

    def set_inner_solver(self, solver: int, restart: int = 0):
        self._check(self.lib.dyson_set_inner_solver(self.h, solver, restart))

    def local_greens(self, sources=None, precision=PREC_F64, tol=1e-13, max_sweeps=400, out=None, allow=(0,)):
        """Diagonal blocks G_ss of the block columns `sources` (default: every site) into
        `out`, a complex128 device tensor [Nr, Nc, Nc] (allocated when None).  Returns (out, SolveResult)."""
        torch = self._torch
        src = np.ascontiguousarray(np.asarray(range(self.p.Nr) if sources is None else sources, dtype=np.int32))
        if out is None:
            out = torch.zeros((self.p.Nr, self.p.Nc, self.p.Nc), dtype=torch.complex128,
                              device=torch.device("cuda", self.device))
        optr = device_buffer(out, torch.complex128, self.p.Nr * self.p.Nc * self.p.Nc, self.device, "out")
        rep = Report()
        rc = self.lib.dyson_local_greens(self.h, src.ctypes.data_as(C.POINTER(C.c_int32)), len(src), precision, tol,
                                         max_sweeps, optr, C.byref(rep))
        self._check(rc, ok=allow)
        return out, SolveResult(rc, rep.as_dict())

    def selfenergy_step(self, gloc, mix=0.7, sigma_tilde=None):
        """One self-energy step from the local Green's functions `gloc` (device [Nr, Nc, Nc]);
        installs the new local blocks and returns the convergence measure."""
        n_el, c128 = self.p.Nr * self.p.Nc * self.p.Nc, self._torch.complex128
        gptr = device_buffer(gloc, c128, n_el, self.device, "gloc")
        st = device_buffer(sigma_tilde, c128, n_el, self.device, "sigma_tilde") if sigma_tilde is not None else None
        crit = C.c_double()
        self._check(self.lib.dyson_selfenergy_step(self.h, gptr, mix, st, C.byref(crit)))
        return crit.value

    def set_anderson(self, depth: int):
        """0: linear mixing of the self-energy steps; 1..6: Anderson acceleration of that depth."""
        self._check(self.lib.dyson_selfenergy_set_anderson(self.h, depth))

    def set_support_truncation(self, enable: bool):
        self._check(self.lib.dyson_set_support_truncation(self.h, 1 if enable else 0))

    def set_wait_limit(self, seconds: float):
        """Time limit of the tensor-core pipelines' bounded waits on this device (0: the default 2 s)."""
        self._check(self.lib.dyson_set_wait_limit(self.h, float(seconds)))

    def set_graph_sweeps(self, sweeps: int):
        """Sweeps per captured graph of the inner series (0: one synchronisation per sweep)."""
        self._check(self.lib.dyson_set_graph_sweeps(self.h, int(sweeps)))

    def set_sweep_variant(self, variant: int):
        self._check(self.lib.dyson_set_sweep_variant(self.h, variant))

    def profile(self, enable: bool):
        self._check(self.lib.dyson_profile(self.h, 1 if enable else 0))

    def profile_query(self, kind: int):
        n = C.c_int64()
        ms = C.c_double()
        self._check(self.lib.dyson_profile_query(self.h, kind, C.byref(n), C.byref(ms)))
        return n.value, ms.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.dyson_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """dyson_batch over Solver objects that share one device and one stream.

    solve() runs the mixed-precision solve of every instance's block columns
    with shared sweep launches (see include/dyson.h); results per instance."""

    def __init__(self, solvers):
        self.lib = load()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[sv.h for sv in self.solvers])
        h = C.c_void_p()
        rc = self.lib.dyson_batch_create(C.byref(h), arr, len(self.solvers))
        if rc != 0:
            raise DysonError(rc, self.lib.dyson_last_error(None).decode())
        self.h = h

    def solve(self, sources, tol=1e-10, max_sweeps=400, graph_sweeps=8, g_outs=None, allow=(0,)):
        """sources[k]: block-column source sites of instance k; g_outs: None or per
        instance None / a complex128 device tensor [len(sources[k]), Nr, Nc, Nc]."""
        n = len(self.solvers)
        if len(sources) != n:
            raise ValueError(f"sources must list {n} instances")
        keep = [np.ascontiguousarray(np.asarray(s, dtype=np.int32)) for s in sources]
        ptrs = (C.POINTER(C.c_int32) * n)(*[k.ctypes.data_as(C.POINTER(C.c_int32)) for k in keep])
        counts = (C.c_int32 * n)(*[len(k) for k in keep])
        gp = None
        if g_outs is not None:
            vals = []
            for sv, k, g in zip(self.solvers, keep, g_outs):
                if g is None:
                    vals.append(None)
                    continue
                vals.append(device_buffer(g, sv._torch.complex128, len(k) * sv.p.Nr * sv.p.Nc * sv.p.Nc, sv.device,
                                          "g_outs[i]").value)
            gp = (C.c_void_p * n)(*vals)
        reps = (Report * n)()
        rc = self.lib.dyson_batch_solve(self.h, ptrs, counts, tol, max_sweeps, graph_sweeps, gp, reps)
        if rc not in allow:
            raise DysonError(rc, self.lib.dyson_batch_last_error(self.h).decode())
        return [SolveResult(r.status, r.as_dict()) for r in reps]

    def launch_count(self) -> int:
        return int(self.lib.dyson_batch_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dyson_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
