"""Python binding of the GB300 line-preconditioned CG solver library.

Argument marshalling only: every step of the solver runs in the CUDA
kernels of ``libpcg.so`` (built from ``csrc/`` by ``build.py``); this module
converts Python objects and torch tensors into the plain pointers and sizes
of the C-ABI declared in ``include/pcg.h`` and calls it.  The functions keep
the C names (``pcg_create``, ``pcg_solve``, ``pcg_apply_A``, ``pcg_precond``,
...); ``Solver`` bundles them for convenience.  There is no fallback: if the
library is missing or cannot be loaded, importing a solver raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
from typing import Optional

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpcg.so")

PCG_OK, PCG_ERR_INVALID_ARG, PCG_ERR_OOM, PCG_ERR_CUDA, PCG_NOT_CONVERGED, PCG_BREAKDOWN, PCG_TIMEOUT, PCG_PENDING = range(8)
PCG_GEOM_BOX, PCG_GEOM_LATLON, PCG_GEOM_CUBED_PANEL = 0, 1, 2
PCG_FP64, PCG_MIXED = 0, 1
PCG_PREC_LINE, PCG_PREC_MULTIGRID, PCG_PREC_MULTIGRID_F32 = 0, 1, 2
PCG_ALG_INTERLEAVED, PCG_ALG_SINGLE_REDUCTION = 0, 1
STATUS_NAMES = {0: "ok", 1: "invalid_arg", 2: "oom", 3: "cuda", 4: "not_converged", 5: "breakdown", 6: "timeout",
                7: "pending"}

EXPORTED = (
    "pcg_create", "pcg_solve", "pcg_solve_host", "pcg_rhs_stats", "pcg_apply_A", "pcg_precond",
    "pcg_apply_A_f32", "pcg_precond_f32", "pcg_time_sweeps", "pcg_time_passes", "pcg_sync", "pcg_device_bytes", "pcg_kernel_launches",
    "pcg_last_error", "pcg_destroy", "pcg_precond_noalloc",
    "pcg_server_create", "pcg_serve_submit", "pcg_serve_step", "pcg_serve_poll", "pcg_serve_info",
    "pcg_server_last_error", "pcg_server_destroy",
)


class pcg_grid_t(ctypes.Structure):
    _fields_ = [("geometry", ctypes.c_int), ("n_x", ctypes.c_int), ("n_y", ctypes.c_int), ("n_z", ctypes.c_int),
                ("nrhs", ctypes.c_int), ("z_iface", ctypes.POINTER(ctypes.c_double)),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lat0", ctypes.c_double), ("lat1", ctypes.c_double)]


class pcg_coeffs_t(ctypes.Structure):
    _fields_ = [("alpha_e", ctypes.POINTER(ctypes.c_double)), ("alpha_n", ctypes.POINTER(ctypes.c_double)),
                ("beta_iface", ctypes.POINTER(ctypes.c_double)), ("lambda2", ctypes.c_double)]


class pcg_opts_t(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("inner_tol", ctypes.c_double), ("inner_maxit", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("passes_per_launch", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("preconditioner", ctypes.c_int),
                ("algorithm", ctypes.c_int)]


class pcg_stats_t(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int), ("outer_sweeps", ctypes.c_int),
                ("stagnated", ctypes.c_int), ("relres_recursive", ctypes.c_double),
                ("relres_true", ctypes.c_double), ("elapsed_ms", ctypes.c_double),
                ("relres_floor", ctypes.c_double)]


_lib: Optional[ctypes.CDLL] = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpcg.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1302_7193_gb300.build`")
    lib = ctypes.CDLL(path)
    P, D, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int
    lib.pcg_create.argtypes = [ctypes.POINTER(pcg_grid_t), ctypes.POINTER(pcg_coeffs_t), ctypes.POINTER(pcg_opts_t),
                               ctypes.POINTER(ctypes.c_void_p)]
    lib.pcg_create.restype = I
    for name in ("pcg_solve", "pcg_solve_host"):
        getattr(lib, name).argtypes = [P, P, P, D, I, ctypes.POINTER(pcg_stats_t)]
        getattr(lib, name).restype = I
    lib.pcg_rhs_stats.argtypes = [P, I, ctypes.POINTER(pcg_stats_t)]
    lib.pcg_rhs_stats.restype = I
    for name in ("pcg_apply_A", "pcg_precond", "pcg_apply_A_f32", "pcg_precond_f32"):
        getattr(lib, name).argtypes = [P, P, P]
        getattr(lib, name).restype = I
    lib.pcg_time_sweeps.argtypes = [P, P, I, I, ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.pcg_time_sweeps.restype = I
    lib.pcg_time_passes.argtypes = [P, P, I, I, ctypes.POINTER(D)]
    lib.pcg_time_passes.restype = I
    lib.pcg_sync.argtypes = [P]
    lib.pcg_sync.restype = I
    lib.pcg_device_bytes.argtypes = [P]
    lib.pcg_device_bytes.restype = ctypes.c_size_t
    lib.pcg_kernel_launches.argtypes = [P]
    lib.pcg_kernel_launches.restype = ctypes.c_longlong
    lib.pcg_last_error.argtypes = [P]
    lib.pcg_last_error.restype = ctypes.c_char_p
    lib.pcg_destroy.argtypes = [P]
    lib.pcg_destroy.restype = None
    lib.pcg_precond_noalloc.argtypes = [ctypes.POINTER(pcg_grid_t), ctypes.POINTER(pcg_coeffs_t), P, P, P]
    lib.pcg_precond_noalloc.restype = I
    lib.pcg_server_create.argtypes = [ctypes.c_size_t, I, ctypes.POINTER(pcg_opts_t), ctypes.POINTER(ctypes.c_void_p)]
    lib.pcg_server_create.restype = I
    lib.pcg_serve_submit.argtypes = [P, ctypes.POINTER(pcg_grid_t), ctypes.POINTER(pcg_coeffs_t), P, D,
                                     ctypes.POINTER(ctypes.c_uint64)]
    lib.pcg_serve_submit.restype = I
    lib.pcg_serve_step.argtypes = [P, I, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.pcg_serve_step.restype = I
    lib.pcg_serve_poll.argtypes = [P, ctypes.c_uint64, P, ctypes.POINTER(pcg_stats_t)]
    lib.pcg_serve_poll.restype = I
    lib.pcg_serve_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(ctypes.c_size_t),
                                   ctypes.POINTER(ctypes.c_longlong)]
    lib.pcg_serve_info.restype = I
    lib.pcg_server_last_error.argtypes = [P]
    lib.pcg_server_last_error.restype = ctypes.c_char_p
    lib.pcg_server_destroy.argtypes = [P]
    lib.pcg_server_destroy.restype = None
    _lib = lib
    return lib


class PCGError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


@dataclasses.dataclass
class Stats:
    status: int
    iterations: int
    outer_sweeps: int
    stagnated: int
    relres_recursive: float
    relres_true: float
    elapsed_ms: float
    relres_floor: float = 0.0

    @property
    def status_name(self) -> str:
        return STATUS_NAMES.get(self.status, str(self.status))


def _stats(s: pcg_stats_t) -> Stats:
    return Stats(s.status, s.iterations, s.outer_sweeps, s.stagnated, s.relres_recursive, s.relres_true, s.elapsed_ms,
                 s.relres_floor)


def _dptr(arr, dtype_name: str, n: int) -> int:
    """Device pointer of a contiguous CUDA torch tensor with n elements."""
    import torch
    want = {"f64": torch.float64, "f32": torch.float32}[dtype_name]
    if not isinstance(arr, torch.Tensor) or not arr.is_cuda:
        raise TypeError("expected a CUDA torch tensor")
    if arr.dtype != want or not arr.is_contiguous() or arr.numel() != n:
        raise ValueError(f"expected a contiguous {want} tensor with {n} elements, got {arr.dtype} {tuple(arr.shape)}")
    return arr.data_ptr()


def _hptr(a, n: int):
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or a.size != n:
        raise ValueError(f"expected a C-contiguous float64 numpy array with {n} elements")
    return a.ctypes.data_as(ctypes.c_void_p)


def _dbl(a):
    import numpy as np
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def pcg_create(problem, nrhs: int = 1, precision: int = PCG_FP64, inner_tol: float = 0.0, inner_maxit: int = 0,
               max_outer: int = 0, passes_per_launch: int = 0, stream: Optional[int] = None,
               preconditioner: int = PCG_PREC_LINE, algorithm: int = PCG_ALG_INTERLEAVED):
    """Marshal a problem description (any object with the fields of
    ``workloads.Problem``) into pcg_create; returns (handle, keepalive)."""
    lib = load_library()
    z, zp = _dbl(problem.z_iface)
    be, bp = _dbl(problem.beta_iface)
    ae, aep = _dbl(getattr(problem, "alpha_e", None))
    an, anp = _dbl(getattr(problem, "alpha_n", None))
    g = pcg_grid_t(int(problem.kind), int(problem.n_x), int(problem.n_y), int(problem.n_z), int(nrhs), zp,
                   float(getattr(problem, "lx", 1.0)), float(getattr(problem, "ly", 1.0)),
                   float(getattr(problem, "lat0", 0.0)), float(getattr(problem, "lat1", 0.0)))
    c = pcg_coeffs_t(aep, anp, bp, float(problem.lambda2))
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        except Exception:
            stream = 0
    o = pcg_opts_t(int(precision), float(inner_tol), int(inner_maxit), int(max_outer), int(passes_per_launch),
                   ctypes.c_void_p(stream or 0), int(preconditioner), int(algorithm))
    h = ctypes.c_void_p()
    rc = lib.pcg_create(ctypes.byref(g), ctypes.byref(c), ctypes.byref(o), ctypes.byref(h))
    if rc != PCG_OK:
        raise PCGError(rc, lib.pcg_last_error(None).decode())
    return h, (z, be, ae, an)


class Solver:
    """One pcg_t handle.  Vectors are torch tensors of nrhs * n_z * n_y * n_x
    elements in the layout [nrhs][n_z][n_y][n_x].

    precision:      "fp64" (PCG_FP64) or "mixed" (PCG_MIXED: FP32 inner PCG
                    inside FP64 iterative refinement).
    preconditioner: "line" (the paper's vertical-line preconditioner),
                    "multigrid" (one V-cycle with line smoothing, FP64) or
                    "multigrid-f32" (the same V-cycle in FP32 inside the FP64
                    CG); the multigrid options need precision "fp64".
    algorithm:      "interleaved" (Algorithm 1, two sweeps per iteration) or
                    "single-reduction" (one sweep and one reduction per
                    iteration; line preconditioner, n_z <= 256).
    Further keyword arguments go to pcg_create (inner_tol, inner_maxit,
    max_outer, passes_per_launch, stream)."""

    def __init__(self, problem, nrhs: int = 1, precision: str = "fp64", preconditioner: str = "line",
                 algorithm: str = "interleaved", **kw):
        self.lib = load_library()
        self.problem = problem
        self.nrhs = nrhs
        self.n = int(problem.n_x) * int(problem.n_y) * int(problem.n_z) * nrhs
        prec = {"fp64": PCG_FP64, "mixed": PCG_MIXED}[precision]
        self.precision = precision
        self.preconditioner = preconditioner
        pc = {"line": PCG_PREC_LINE, "multigrid": PCG_PREC_MULTIGRID,
              "multigrid-f32": PCG_PREC_MULTIGRID_F32}[preconditioner]
        self.algorithm = algorithm
        alg = {"interleaved": PCG_ALG_INTERLEAVED, "single-reduction": PCG_ALG_SINGLE_REDUCTION}[algorithm]
        self.h, self._keep = pcg_create(problem, nrhs=nrhs, precision=prec, preconditioner=pc, algorithm=alg, **kw)

    def _check(self, rc: int, allow=(PCG_OK,)):
        if rc not in allow:
            raise PCGError(rc, self.lib.pcg_last_error(self.h).decode())
        return rc

    def pcg_solve(self, b, x, tol: float = 1e-8, maxit: int = 100000) -> Stats:
        st = pcg_stats_t()
        rc = self.lib.pcg_solve(self.h, _dptr(b, "f64", self.n), _dptr(x, "f64", self.n), float(tol), int(maxit),
                                ctypes.byref(st))
        self._check(rc, allow=(PCG_OK, PCG_NOT_CONVERGED, PCG_BREAKDOWN))
        return _stats(st)

    solve = pcg_solve

    def pcg_solve_host(self, b, x, tol: float = 1e-8, maxit: int = 100000) -> Stats:
        st = pcg_stats_t()
        rc = self.lib.pcg_solve_host(self.h, _hptr(b, self.n), _hptr(x, self.n), float(tol), int(maxit),
                                     ctypes.byref(st))
        self._check(rc, allow=(PCG_OK, PCG_NOT_CONVERGED, PCG_BREAKDOWN))
        return _stats(st)

    solve_host = pcg_solve_host

    def pcg_rhs_stats(self, rhs: int) -> Stats:
        st = pcg_stats_t()
        self._check(self.lib.pcg_rhs_stats(self.h, int(rhs), ctypes.byref(st)))
        return _stats(st)

    def pcg_apply_A(self, x, y):
        self._check(self.lib.pcg_apply_A(self.h, _dptr(x, "f64", self.n), _dptr(y, "f64", self.n)))

    def pcg_precond(self, r, z):
        self._check(self.lib.pcg_precond(self.h, _dptr(r, "f64", self.n), _dptr(z, "f64", self.n)))

    def pcg_apply_A_f32(self, x, y):
        self._check(self.lib.pcg_apply_A_f32(self.h, _dptr(x, "f32", self.n), _dptr(y, "f32", self.n)))

    def pcg_precond_f32(self, r, z):
        self._check(self.lib.pcg_precond_f32(self.h, _dptr(r, "f32", self.n), _dptr(z, "f32", self.n)))

    apply_A, precond, apply_A_f32, precond_f32 = pcg_apply_A, pcg_precond, pcg_apply_A_f32, pcg_precond_f32

    def pcg_time_sweeps(self, b, precision: str = "fp64", passes: int = 10):
        """Mean device ms per launch of (preconditioner sweep, SpMV sweep)."""
        a, c = ctypes.c_double(), ctypes.c_double()
        prec = {"fp64": PCG_FP64, "mixed": PCG_MIXED}[precision]
        self._check(self.lib.pcg_time_sweeps(self.h, _dptr(b, "f64", self.n), prec, int(passes),
                                             ctypes.byref(a), ctypes.byref(c)))
        return a.value, c.value

    def pcg_time_passes(self, b, precision: str = "fp64", passes: int = 20) -> float:
        """Mean device ms of one pass (both sweeps) with the passes back to back."""
        a = ctypes.c_double()
        prec = {"fp64": PCG_FP64, "mixed": PCG_MIXED}[precision]
        self._check(self.lib.pcg_time_passes(self.h, _dptr(b, "f64", self.n), prec, int(passes), ctypes.byref(a)))
        return a.value

    def pcg_sync(self):
        self._check(self.lib.pcg_sync(self.h))

    @property
    def device_bytes(self) -> int:
        return int(self.lib.pcg_device_bytes(self.h))

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.pcg_kernel_launches(self.h))

    def close(self):
        if self.h:
            self.lib.pcg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def problem_structs(problem, nrhs: int = 1):
    """pcg_grid_t / pcg_coeffs_t of a problem description, with the arrays
    they point to (keep the third value alive while the structs are used)."""
    z, zp = _dbl(problem.z_iface)
    be, bp = _dbl(problem.beta_iface)
    ae, aep = _dbl(getattr(problem, "alpha_e", None))
    an, anp = _dbl(getattr(problem, "alpha_n", None))
    g = pcg_grid_t(int(problem.kind), int(problem.n_x), int(problem.n_y), int(problem.n_z), int(nrhs), zp,
                   float(getattr(problem, "lx", 1.0)), float(getattr(problem, "ly", 1.0)),
                   float(getattr(problem, "lat0", 0.0)), float(getattr(problem, "lat1", 0.0)))
    c = pcg_coeffs_t(aep, anp, bp, float(problem.lambda2))
    return g, c, (z, be, ae, an)


class Server:
    """One pcg_server_t: served solves, either batched line-preconditioned
    mixed-precision solves (preconditioner="line") or multigrid-preconditioned
    FP64 CG solves by a pool of worker threads (preconditioner="multigrid-f32")."""

    def __init__(self, budget_bytes: int, max_slots: int = 64, inner_tol: float = 0.0, inner_maxit: int = 0,
                 max_outer: int = 0, epochs_per_launch: int = 0, stream: Optional[int] = None,
                 preconditioner: str = "line"):
        self.lib = load_library()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except Exception:
                stream = 0
        pc = {"line": PCG_PREC_LINE, "multigrid-f32": PCG_PREC_MULTIGRID_F32}[preconditioner]
        o = pcg_opts_t(PCG_MIXED, float(inner_tol), int(inner_maxit), int(max_outer), int(epochs_per_launch),
                       ctypes.c_void_p(stream or 0), pc)
        h = ctypes.c_void_p()
        rc = self.lib.pcg_server_create(ctypes.c_size_t(int(budget_bytes)), int(max_slots), ctypes.byref(o),
                                        ctypes.byref(h))
        if rc != PCG_OK:
            raise PCGError(rc, self.lib.pcg_server_last_error(None).decode())
        self.h = h
        self.sizes = {}

    def pcg_serve_submit(self, problem, b, tol: float = 1e-8) -> int:
        import numpy as np
        g, c, keep = problem_structs(problem)
        n = int(problem.n_x) * int(problem.n_y) * int(problem.n_z)
        bb = np.ascontiguousarray(b, dtype=np.float64).ravel()
        rid = ctypes.c_uint64()
        rc = self.lib.pcg_serve_submit(self.h, ctypes.byref(g), ctypes.byref(c), _hptr(bb, n), float(tol),
                                       ctypes.byref(rid))
        if rc != PCG_OK:
            raise PCGError(rc, self.lib.pcg_server_last_error(self.h).decode())
        self.sizes[rid.value] = n
        return rid.value

    submit = pcg_serve_submit

    def pcg_serve_step(self, max_epochs: int = 8):
        a, q = ctypes.c_int(), ctypes.c_int()
        rc = self.lib.pcg_serve_step(self.h, int(max_epochs), ctypes.byref(a), ctypes.byref(q))
        if rc != PCG_OK:
            raise PCGError(rc, self.lib.pcg_server_last_error(self.h).decode())
        return a.value, q.value

    step = pcg_serve_step

    def pcg_serve_poll(self, rid: int, want_x: bool = True):
        """(x, Stats) once the request has finished, else None."""
        import numpy as np
        x = np.empty(self.sizes[rid]) if want_x else None
        st = pcg_stats_t()
        rc = self.lib.pcg_serve_poll(self.h, ctypes.c_uint64(rid), x.ctypes.data_as(ctypes.c_void_p) if want_x else None,
                                     ctypes.byref(st))
        if rc == PCG_PENDING:
            return None
        if rc != PCG_OK:
            raise PCGError(rc, self.lib.pcg_server_last_error(self.h).decode())
        del self.sizes[rid]
        return x, _stats(st)

    poll = pcg_serve_poll

    def pcg_serve_info(self):
        a, q, u, e = ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t(), ctypes.c_longlong()
        self.lib.pcg_serve_info(self.h, ctypes.byref(a), ctypes.byref(q), ctypes.byref(u), ctypes.byref(e))
        return {"active": a.value, "pending": q.value, "used_bytes": u.value, "epochs": e.value}

    info = pcg_serve_info

    def close(self):
        if self.h:
            self.lib.pcg_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
