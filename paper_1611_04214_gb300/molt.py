"""Python binding of the C ABI in ``include/molt.h`` (argument marshalling only).

Every computation runs in ``libmolt.so``; this module converts torch tensors and streams to
raw pointers and return codes to exceptions.  There is no fallback: if the library is
missing, importing the binding's loader raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmolt.so")

MOLT_OK, MOLT_ERR_ARG, MOLT_ERR_NOT_CONVERGED, MOLT_ERR_CUDA, MOLT_ERR_OOM, MOLT_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
BC = {"periodic": 0, "neumann": 1, "dirichlet": 2}
PRECISION = {"fp32": 0, "fp64": 1}
SCHEME = {"be": 0, "bdf2": 1, "sdirk2": 2, "sdirk3": 3, "sdc2": 4, "bdf3": 5}
LTE_ESTIMATOR = {"richardson": 0, "sdc2": 1, "bdf2": 2}          # molt_adaptive.estimator

# Every symbol declared in include/molt.h.
EXPORTS = [
    "molt_grid_create", "molt_grid_destroy", "molt_solver_create", "molt_solver_destroy",
    "molt_set_params", "molt_set_bc", "molt_reset_history", "molt_step", "molt_run_host",
    "molt_energy", "molt_mass", "molt_helmholtz_apply", "molt_quadrature_weights",
    "molt_last_error", "molt_kernel_launches", "molt_profile_enable", "molt_profile_collect",
    "molt_helmholtz_columns_noalloc", "molt_helmholtz_columns_noalloc_status", "molt_set_execution", "molt_graph_fallbacks",
    "molt_column_tma_launches", "molt_batch_create", "molt_batch_destroy", "molt_batch_points",
    "molt_batch_offsets", "molt_batch_set_execution", "molt_batch_step", "molt_selftest_bounded_wait",
    "molt_step_adaptive",
    "molt_vch_step", "molt_fma_throughput_probe", "molt_helmholtz_rows_tc", "molt_vch_step_adaptive",
    "molt_batch_autotune", "molt_batch_set_schedule", "molt_autotune", "molt_batch_helmholtz_apply",
    "molt_solver3d_create", "molt_solver3d_destroy", "molt_solver3d_step", "molt_solver3d_apply",
    "molt_solver3d_launches", "molt_fch1d_create", "molt_fch1d_destroy", "molt_fch1d_step", "molt_fch1d_launches",
    "molt_fch2d_create", "molt_fch2d_destroy", "molt_fch2d_step", "molt_fch2d_launches",
]
EXECUTION = {"host_loop": 0, "graph": 1}
PROFILE_SLOTS = 32
PASS_NAMES = ["H", "pass1", "pass2", "pass3", "pass4", "pass1d_a", "pass1d_b", ""]


class _Adaptive(ctypes.Structure):
    _fields_ = [("lte_tol", ctypes.c_double), ("dt_min", ctypes.c_double), ("dt_max", ctypes.c_double),
                ("theta", ctypes.c_double), ("gamma", ctypes.c_double), ("estimator", ctypes.c_int)]


class _AdaptiveInfo(ctypes.Structure):
    _fields_ = [("dt_used", ctypes.c_double), ("dt_next", ctypes.c_double), ("eta", ctypes.c_double),
                ("rejections", ctypes.c_int), ("max_iters", ctypes.c_int)]


class _Tuning(ctypes.Structure):
    _fields_ = [("pass_", ctypes.c_int), ("axis", ctypes.c_int), ("chosen", ctypes.c_int),
                ("candidates", ctypes.c_int), ("launch", ctypes.c_int * 4), ("ms", ctypes.c_double * 4),
                ("tc_rel_diff", ctypes.c_double)]


LAUNCH_NAMES = {0: "default", 1: "rows_one_block", 2: "rows_cluster2", 3: "rows_general", 4: "cols_tma",
                5: "cols_cp_async", 6: "cols_general", 7: "rows_tensor_core"}


class MoltError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"molt status {status}: {message}")
        self.status = status


class NotConverged(MoltError):
    pass


class _Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("quad_order", ctypes.c_int), ("precision", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iter", ctypes.c_int)]


class _StepInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("stages", ctypes.c_int), ("iters", ctypes.c_int * 4),
                ("total_iters", ctypes.c_int), ("residual", ctypes.c_double), ("tol_used", ctypes.c_double)]


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libmolt.so (built by ``paper_1611_04214_gb300.build``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1611_04214_gb300.build` "
                          "(the library has no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (args, res) in signatures().items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def signatures() -> dict:
    """ctypes argument and result types of every entry point of include/molt.h."""
    P, I, D, VP = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    return {
        "molt_grid_create": ([ctypes.POINTER(P), I, I, I, D, D, I], I),
        "molt_grid_destroy": ([P], None),
        "molt_solver_create": ([ctypes.POINTER(P), P, ctypes.POINTER(_Params)], I),
        "molt_solver_destroy": ([P], None),
        "molt_set_params": ([P, ctypes.POINTER(_Params)], I),
        "molt_set_bc": ([P, I], I),
        "molt_reset_history": ([P], I),
        "molt_step": ([P, VP, D, I, VP, ctypes.POINTER(_StepInfo)], I),
        "molt_run_host": ([P, VP, D, I, I, VP, ctypes.POINTER(_StepInfo)], I),
        "molt_energy": ([P, VP, ctypes.POINTER(D), VP], I),
        "molt_mass": ([P, VP, ctypes.POINTER(D), VP], I),
        "molt_helmholtz_apply": ([P, I, D, VP, VP, VP], I),
        "molt_helmholtz_rows_tc": ([P, D, VP, VP, VP], I),
        "molt_quadrature_weights": ([D, I, ctypes.POINTER(I), I, ctypes.POINTER(D)], I),
        "molt_last_error": ([P], ctypes.c_char_p),
        "molt_kernel_launches": ([P], ctypes.c_longlong),
        "molt_profile_enable": ([P, I], I),
        "molt_profile_collect": ([P, ctypes.POINTER(D), ctypes.POINTER(ctypes.c_longlong)], I),
        "molt_helmholtz_columns_noalloc": ([I, I, D, I, I, D, VP, VP, VP], I),
        "molt_helmholtz_columns_noalloc_status": ([VP, ctypes.POINTER(ctypes.c_uint)], I),
        "molt_set_execution": ([P, I], I),
        "molt_graph_fallbacks": ([P], ctypes.c_longlong),
        "molt_column_tma_launches": ([], ctypes.c_longlong),
        "molt_selftest_bounded_wait": ([ctypes.POINTER(I), ctypes.POINTER(D)], I),
        "molt_fma_throughput_probe": ([I, ctypes.POINTER(D)], I),
        "molt_step_adaptive": ([P, VP, D, ctypes.POINTER(_Adaptive), VP, ctypes.POINTER(_AdaptiveInfo)], I),
        "molt_vch_step": ([P, VP, VP, D, I, VP, ctypes.POINTER(_StepInfo)], I),
        "molt_vch_step_adaptive": ([P, VP, VP, D, ctypes.POINTER(_Adaptive), VP, ctypes.POINTER(_AdaptiveInfo)], I),
        "molt_batch_create": ([ctypes.POINTER(VP), I, VP, I, I, D, I], I),
        "molt_batch_destroy": ([VP], I),
        "molt_batch_points": ([VP], ctypes.c_longlong),
        "molt_batch_offsets": ([VP, ctypes.POINTER(ctypes.c_longlong)], I),
        "molt_batch_set_execution": ([VP, I], I),
        "molt_batch_autotune": ([VP, ctypes.POINTER(D), VP, ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "molt_batch_set_schedule": ([VP, I, I], I),
        "molt_batch_helmholtz_apply": ([VP, I, ctypes.POINTER(D), VP, VP, VP], I),
        "molt_solver3d_create": ([ctypes.POINTER(VP), I, I, I, D, D, D, I, ctypes.POINTER(_Params)], I),
        "molt_solver3d_destroy": ([VP], I),
        "molt_solver3d_step": ([VP, VP, D, I, VP, ctypes.POINTER(_StepInfo)], I),
        "molt_solver3d_apply": ([VP, I, D, VP, VP, VP], I),
        "molt_solver3d_launches": ([VP], ctypes.c_longlong),
        "molt_fch1d_create": ([ctypes.POINTER(VP), I, I, D, I, D, ctypes.POINTER(_Params)], I),
        "molt_fch1d_destroy": ([VP], I),
        "molt_fch1d_step": ([VP, VP, D, VP, ctypes.POINTER(_StepInfo)], I),
        "molt_fch1d_launches": ([VP], ctypes.c_longlong),
        "molt_fch2d_create": ([ctypes.POINTER(VP), I, I, D, D, I, D, ctypes.POINTER(_Params)], I),
        "molt_fch2d_destroy": ([VP], I),
        "molt_fch2d_step": ([VP, VP, D, VP, ctypes.POINTER(_StepInfo)], I),
        "molt_fch2d_launches": ([VP], ctypes.c_longlong),
        "molt_autotune": ([P, VP, ctypes.POINTER(_Tuning), I, ctypes.POINTER(I)], I),
        "molt_batch_step": ([VP, VP, ctypes.POINTER(D), I, VP, ctypes.POINTER(I), ctypes.POINTER(D),
                             ctypes.POINTER(I)], I),
    }


def _check(status: int, handle=None):
    if status == MOLT_OK:
        return
    msg = load_library().molt_last_error(handle).decode()
    if status == MOLT_ERR_NOT_CONVERGED:
        raise NotConverged(status, msg)
    raise MoltError(status, msg)


def molt_quadrature_weights(nu: float, M: int, offsets, side: str):
    """Weights of J^L (side 'L') or J^R ('R') for integer node offsets (host-only call)."""
    lib = load_library()
    offs = (ctypes.c_int * (M + 1))(*[int(o) for o in offsets])
    out = (ctypes.c_double * (M + 1))()
    _check(lib.molt_quadrature_weights(float(nu), int(M), offs, 0 if side == "L" else 1, out))
    return list(out)


def molt_helmholtz_columns_noalloc(nx: int, ny: int, Ly: float, bc: str, quad_order: int, c: float, inp, out,
                                   stream=None):
    """The allocation-free FP32 column sweep (see include/molt.h) on contiguous CUDA float32 tensors."""
    lib = load_library()
    for t in (inp, out):
        if not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous() or t.numel() != nx * ny:
            raise ValueError("expected contiguous CUDA float32 tensors of ny x nx elements")
    _check(lib.molt_helmholtz_columns_noalloc(int(nx), int(ny), float(Ly), BC[bc], int(quad_order), float(c),
                                              ctypes.c_void_p(inp.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                              _stream_handle(stream)))


def molt_helmholtz_columns_noalloc_status(stream=None) -> int:
    """Status word of the last allocation-free column sweep (0 = complete; see include/molt.h)."""
    word = ctypes.c_uint(0)
    _check(load_library().molt_helmholtz_columns_noalloc_status(_stream_handle(stream), ctypes.byref(word)))
    return int(word.value)


def molt_column_tma_launches() -> int:
    """Column-sweep kernels launched with TMA tile loads since the library was loaded (diagnostics)."""
    return int(load_library().molt_column_tma_launches())


def molt_fma_throughput_probe(precision: str) -> float:
    """Sustained FMA throughput of the current GPU in TFLOP/s ("fp32" or "fp64"; diagnostics)."""
    out = ctypes.c_double(0.0)
    _check(load_library().molt_fma_throughput_probe(PRECISION[precision], ctypes.byref(out)))
    return float(out.value)


def molt_selftest_bounded_wait():
    """Run one kernel whose bounded wait cannot complete; returns (timed_out, seconds waited)."""
    t = ctypes.c_int(0)
    sec = ctypes.c_double(0.0)
    _check(load_library().molt_selftest_bounded_wait(ctypes.byref(t), ctypes.byref(sec)))
    return bool(t.value), float(sec.value)


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


@dataclass
class StepInfo:
    status: int
    stages: int
    iters: list = field(default_factory=list)
    total_iters: int = 0
    residual: float = 0.0
    tol_used: float = 0.0


class Solver:
    """A grid + solver pair of the C ABI (molt_grid_create + molt_solver_create)."""

    def __init__(self, nx: int, ny: int = 1, Lx: float = 6.283185307179586, Ly: float = 6.283185307179586,
                 bc: str = "periodic", eps: float = 0.1, quad_order: int = 4, precision: str = "fp32",
                 tol: float = 1e-10, max_iter: int = 500):
        lib = load_library()
        self._lib = lib
        self.nx, self.ny, self.bc, self.precision = nx, ny, bc, precision
        self.dim = 1 if ny == 1 else 2
        g = ctypes.c_void_p()
        _check(lib.molt_grid_create(ctypes.byref(g), self.dim, nx, ny, Lx, Ly, BC[bc]))
        self._grid = g
        self._params = _Params(eps, quad_order, PRECISION[precision], tol, max_iter)
        s = ctypes.c_void_p()
        st = lib.molt_solver_create(ctypes.byref(s), g, ctypes.byref(self._params))
        if st != MOLT_OK:
            msg = lib.molt_last_error(None).decode()
            lib.molt_grid_destroy(g)
            self._grid = None
            raise MoltError(st, msg)
        self._h = s

    @property
    def dtype(self):
        import torch
        return torch.float32 if self.precision == "fp32" else torch.float64

    def close(self):
        if getattr(self, "_h", None):
            self._lib.molt_solver_destroy(self._h)
            self._h = None
        if getattr(self, "_grid", None):
            self._lib.molt_grid_destroy(self._grid)
            self._grid = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _field(self, t):
        if not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != self.nx * self.ny:
            raise ValueError(f"expected a contiguous CUDA {self.dtype} tensor of {self.ny}x{self.nx} elements")
        return ctypes.c_void_p(t.data_ptr())

    def set_params(self, eps=None, quad_order=None, tol=None, max_iter=None):
        p = self._params
        if eps is not None:
            p.eps = eps
        if quad_order is not None:
            p.quad_order = quad_order
        if tol is not None:
            p.tol = tol
        if max_iter is not None:
            p.max_iter = max_iter
        _check(self._lib.molt_set_params(self._h, ctypes.byref(p)), self._h)

    def set_bc(self, bc: str):
        _check(self._lib.molt_set_bc(self._h, BC[bc]), self._h)
        self.bc = bc

    def set_execution(self, mode: str):
        """'graph' (device-driven stage loops, the default) or 'host_loop'."""
        _check(self._lib.molt_set_execution(self._h, EXECUTION[mode]), self._h)

    def graph_fallbacks(self) -> int:
        return int(self._lib.molt_graph_fallbacks(self._h))

    def reset_history(self):
        _check(self._lib.molt_reset_history(self._h), self._h)

    def step(self, u, dt: float, scheme: str, stream=None, raise_on_nonconvergence: bool = True) -> StepInfo:
        info = _StepInfo()
        st = self._lib.molt_step(self._h, self._field(u), float(dt), SCHEME[scheme], _stream_handle(stream),
                                 ctypes.byref(info))
        out = StepInfo(info.status, info.stages, list(info.iters)[: max(info.stages, 0)], info.total_iters,
                       info.residual, info.tol_used)
        if st == MOLT_ERR_NOT_CONVERGED and not raise_on_nonconvergence:
            return out
        _check(st, self._h)
        return out

    def vch_step(self, u1, u2, dt: float, scheme: str = "be", stream=None,
                 raise_on_nonconvergence: bool = True) -> StepInfo:
        """One vector Cahn-Hilliard step (Sec. 5.2) in place on the two component fields."""
        info = _StepInfo()
        st = self._lib.molt_vch_step(self._h, self._field(u1), self._field(u2), float(dt), SCHEME[scheme],
                                     _stream_handle(stream), ctypes.byref(info))
        out = StepInfo(info.status, info.stages, list(info.iters)[: max(info.stages, 0)], info.total_iters,
                       info.residual, info.tol_used)
        if st == MOLT_ERR_NOT_CONVERGED and not raise_on_nonconvergence:
            return out
        _check(st, self._h)
        return out

    def run_host(self, u_host, dt: float, scheme: str, nsteps: int, stream=None,
                 raise_on_nonconvergence: bool = True) -> StepInfo:
        """End-to-end call on a host (CPU) tensor: copy in, nsteps steps, copy back."""
        if u_host.is_cuda or u_host.dtype != self.dtype or not u_host.is_contiguous():
            raise ValueError("expected a contiguous host tensor of the solver's dtype")
        info = _StepInfo()
        st = self._lib.molt_run_host(self._h, ctypes.c_void_p(u_host.data_ptr()), float(dt), SCHEME[scheme],
                                     int(nsteps), _stream_handle(stream), ctypes.byref(info))
        if not (st == MOLT_ERR_NOT_CONVERGED and not raise_on_nonconvergence):
            _check(st, self._h)
        return StepInfo(info.status, info.stages, list(info.iters)[: max(info.stages, 0)], info.total_iters,
                        info.residual, info.tol_used)

    def energy(self, u, stream=None) -> float:
        out = ctypes.c_double()
        _check(self._lib.molt_energy(self._h, self._field(u), ctypes.byref(out), _stream_handle(stream)), self._h)
        return out.value

    def mass(self, u, stream=None) -> float:
        out = ctypes.c_double()
        _check(self._lib.molt_mass(self._h, self._field(u), ctypes.byref(out), _stream_handle(stream)), self._h)
        return out.value

    def helmholtz_apply(self, axis: int, c: float, inp, out, stream=None):
        _check(self._lib.molt_helmholtz_apply(self._h, int(axis), float(c), self._field(inp), self._field(out),
                                              _stream_handle(stream)), self._h)

    def helmholtz_rows_tc(self, c: float, inp, out, stream=None):
        """H_c along x on the tensor cores (FP16 split products; see include/molt.h)."""
        _check(self._lib.molt_helmholtz_rows_tc(self._h, float(c), self._field(inp), self._field(out),
                                                _stream_handle(stream)), self._h)

    def step_adaptive(self, u, dt: float, lte_tol: float, dt_min: float, dt_max: float, theta: float = 0.8,
                      gamma: float = 1.3, estimator: str = "richardson", stream=None) -> dict:
        """One accepted step of adaptive size (Algorithm 1) with the "richardson" (BE), "sdc2"
        (BE-SDC2) or "bdf2" (BE-BDF2) LTE estimate; returns dt_used, dt_next, eta, rejections,
        max_iters.  BE-BDF2 keeps the previous accepted state in the solver between calls."""
        a = _Adaptive(lte_tol, dt_min, dt_max, theta, gamma, LTE_ESTIMATOR[estimator])
        info = _AdaptiveInfo()
        _check(self._lib.molt_step_adaptive(self._h, self._field(u), float(dt), ctypes.byref(a),
                                            _stream_handle(stream), ctypes.byref(info)), self._h)
        return {"dt_used": info.dt_used, "dt_next": info.dt_next, "eta": info.eta,
                "rejections": info.rejections, "max_iters": info.max_iters}

    def vch_step_adaptive(self, u1, u2, dt: float, lte_tol: float, dt_min: float, dt_max: float,
                          theta: float = 0.8, gamma: float = 1.3, estimator: str = "bdf2", stream=None) -> dict:
        """One accepted adaptive step of the vector model (Algorithm 1) with the "richardson" or
        "bdf2" (BE-BDF2) estimate; returns dt_used, dt_next, eta, rejections, max_iters."""
        a = _Adaptive(lte_tol, dt_min, dt_max, theta, gamma, LTE_ESTIMATOR[estimator])
        info = _AdaptiveInfo()
        _check(self._lib.molt_vch_step_adaptive(self._h, self._field(u1), self._field(u2), float(dt), ctypes.byref(a),
                                                _stream_handle(stream), ctypes.byref(info)), self._h)
        return {"dt_used": info.dt_used, "dt_next": info.dt_next, "eta": info.eta,
                "rejections": info.rejections, "max_iters": info.max_iters}

    def autotune(self, stream=None) -> list:
        """Time the kernel families of every sweep of a step and keep the fastest (molt_autotune);
        returns one dict per sweep: pass, axis, chosen, and the ms of each candidate (-1: unavailable)."""
        arr = (_Tuning * 16)()
        n = ctypes.c_int(0)
        _check(self._lib.molt_autotune(self._h, _stream_handle(stream), arr, 16, ctypes.byref(n)), self._h)
        out = []
        for t in arr[:min(n.value, 16)]:
            out.append({"pass": t.pass_, "axis": "x" if t.axis == 0 else "y", "chosen": LAUNCH_NAMES[t.chosen],
                        "ms": {LAUNCH_NAMES[t.launch[i]]: t.ms[i] for i in range(t.candidates)},
                        "tc_rel_diff": t.tc_rel_diff if 7 in list(t.launch[:t.candidates]) else None})
        return out

    def kernel_launches(self) -> int:
        return int(self._lib.molt_kernel_launches(self._h))

    def profile_enable(self, on: bool = True):
        _check(self._lib.molt_profile_enable(self._h, 1 if on else 0), self._h)

    def profile_collect(self) -> dict:
        """{kernel name: (total ms, launches)} since the last collect (slots of molt_profile_collect)."""
        ms = (ctypes.c_double * PROFILE_SLOTS)()
        cnt = (ctypes.c_longlong * PROFILE_SLOTS)()
        _check(self._lib.molt_profile_collect(self._h, ms, cnt), self._h)
        out = {}
        for slot in range(PROFILE_SLOTS):
            if cnt[slot] == 0:
                continue
            if slot < 8:
                name = f"rows_{PASS_NAMES[slot]}"
            elif slot < 16:
                name = f"cols_agg_{PASS_NAMES[slot - 8]}"
            elif slot == 16:
                name = "cols_carry"
            else:
                name = f"cols_final_{PASS_NAMES[slot - 17]}"
            out[name] = (ms[slot], int(cnt[slot]))
        return out


class _Instance(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("Lx", ctypes.c_double), ("Ly", ctypes.c_double),
                ("eps", ctypes.c_double)]


@dataclass
class BatchStepInfo:
    status: int
    iters: list
    residual: list
    instance_status: list


class Batch:
    """Independent 2D FP32 instances stepped together (molt_batch_*): one packed device field holds
    every instance back to back; `offsets[i]` is where instance i (ny_i x nx_i, x fastest) starts."""

    def __init__(self, instances, bc: str = "neumann", quad_order: int = 4, tol: float = 1e-6,
                 max_iter: int = 200):
        """instances: sequence of (nx, ny, Lx, Ly, eps)."""
        lib = load_library()
        self._lib = lib
        self.count = len(instances)
        arr = (_Instance * self.count)(*[_Instance(int(a), int(b), float(c), float(d), float(e))
                                         for (a, b, c, d, e) in instances])
        self.shapes = [(int(b), int(a)) for (a, b, _, _, _) in instances]
        h = ctypes.c_void_p()
        _check(lib.molt_batch_create(ctypes.byref(h), self.count, ctypes.cast(arr, ctypes.c_void_p), BC[bc],
                                     int(quad_order), float(tol), int(max_iter)))
        self._h = h
        self.points = int(lib.molt_batch_points(h))
        offs = (ctypes.c_longlong * self.count)()
        _check(lib.molt_batch_offsets(h, offs))
        self.offsets = [int(o) for o in offs]

    def set_execution(self, mode: str):
        _check(self._lib.molt_batch_set_execution(self._h, EXECUTION[mode]))

    def autotune(self, dt, stream=None) -> dict:
        """Pick the launch schedule of the batched passes by timing (molt_batch_autotune); returns the
        chosen grids (0 = one block per work item) and the 4 x 4 table of ms per iteration."""
        dts = (ctypes.c_double * self.count)(*[float(x) for x in dt])
        table = (ctypes.c_double * 16)()
        gr, gc = ctypes.c_int(0), ctypes.c_int(0)
        _check(self._lib.molt_batch_autotune(self._h, dts, _stream_handle(stream), table, ctypes.byref(gr),
                                             ctypes.byref(gc)))
        return {"grid_rows": gr.value, "grid_cols": gc.value, "ms_per_iteration": [list(table[4 * i:4 * i + 4])
                                                                                   for i in range(4)]}

    def set_schedule(self, grid_rows: int, grid_cols: int):
        """Blocks per row / column launch of the batched passes (0 = one block per work item)."""
        _check(self._lib.molt_batch_set_schedule(self._h, int(grid_rows), int(grid_cols)))

    def helmholtz_apply(self, axis: int, c, fin, fout, stream=None):
        """out = H_{c_i} in for every instance along axis 0 (x) or 1 (y) (molt_batch_helmholtz_apply);
        fin, fout: packed contiguous CUDA float32 tensors; c: one value per instance."""
        for t in (fin, fout):
            if not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous() or t.numel() != self.points:
                raise ValueError("expected packed contiguous CUDA float32 fields of the batch")
        cs = (ctypes.c_double * self.count)(*[float(x) for x in c])
        _check(self._lib.molt_batch_helmholtz_apply(self._h, int(axis), cs, ctypes.c_void_p(fin.data_ptr()),
                                                    ctypes.c_void_p(fout.data_ptr()), _stream_handle(stream)))

    def pack(self, fields):
        """Host arrays (one per instance, shape (ny, nx)) -> one packed float32 numpy array."""
        import numpy as np
        out = np.empty(self.points, dtype=np.float32)
        for (ny, nx), o, f in zip(self.shapes, self.offsets, fields):
            out[o:o + ny * nx] = np.asarray(f, dtype=np.float32).reshape(-1)
        return out

    def unpack(self, packed):
        """Packed array (numpy or CPU tensor) -> list of (ny, nx) arrays."""
        return [packed[o:o + ny * nx].reshape(ny, nx) for (ny, nx), o in zip(self.shapes, self.offsets)]

    def step(self, u, dt, scheme: str = "be", stream=None, raise_on_nonconvergence: bool = True) -> BatchStepInfo:
        """One step of every instance in place on the packed CUDA float32 tensor u; dt: per instance."""
        if not u.is_cuda or u.dtype.itemsize != 4 or not u.is_contiguous() or u.numel() != self.points:
            raise ValueError("expected the packed contiguous CUDA float32 field of the batch")
        dts = (ctypes.c_double * self.count)(*[float(x) for x in dt])
        it = (ctypes.c_int * self.count)()
        res = (ctypes.c_double * self.count)()
        sts = (ctypes.c_int * self.count)()
        status = self._lib.molt_batch_step(self._h, ctypes.c_void_p(u.data_ptr()), dts, SCHEME[scheme],
                                           _stream_handle(stream), it, res, sts)
        info = BatchStepInfo(status, list(it), list(res), list(sts))
        if status != MOLT_OK and (status != MOLT_ERR_NOT_CONVERGED or raise_on_nonconvergence):
            _check(status, None)
        return info

    def close(self):
        if getattr(self, "_h", None):
            self._lib.molt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Solver3D:
    """The 3D split stage solver of the C ABI (molt_solver3d_*): FP32 fields [nz][ny][nx]."""

    def __init__(self, nx: int, ny: int, nz: int, Lx: float = 6.283185307179586, Ly: float = 6.283185307179586,
                 Lz: float = 6.283185307179586, bc: str = "periodic", eps: float = 0.1, quad_order: int = 4,
                 tol: float = 1e-10, max_iter: int = 500):
        lib = load_library()
        self._lib = lib
        self.shape = (nz, ny, nx)
        self._params = _Params(eps, quad_order, PRECISION["fp32"], tol, max_iter)
        h = ctypes.c_void_p()
        _check(lib.molt_solver3d_create(ctypes.byref(h), nx, ny, nz, Lx, Ly, Lz, BC[bc], ctypes.byref(self._params)))
        self._h = h

    def _field(self, t):
        if not t.is_cuda or t.dtype.itemsize != 4 or not t.is_contiguous() or tuple(t.shape) != self.shape:
            raise ValueError(f"expected a contiguous CUDA float32 tensor of shape {self.shape}")
        return ctypes.c_void_p(t.data_ptr())

    def step(self, u, dt: float, scheme: str = "be", stream=None, raise_on_nonconvergence: bool = True) -> StepInfo:
        info = _StepInfo()
        st = self._lib.molt_solver3d_step(self._h, self._field(u), float(dt), SCHEME[scheme], _stream_handle(stream),
                                          ctypes.byref(info))
        out = StepInfo(info.status, info.stages, list(info.iters)[: max(info.stages, 0)], info.total_iters,
                       info.residual, info.tol_used)
        if st == MOLT_ERR_NOT_CONVERGED and not raise_on_nonconvergence:
            return out
        _check(st, None)
        return out

    def helmholtz_apply(self, axis: int, c: float, inp, out, stream=None):
        """out = H_c inp along axis 0 (x), 1 (y) or 2 (z)."""
        _check(self._lib.molt_solver3d_apply(self._h, int(axis), float(c), self._field(inp), self._field(out),
                                             _stream_handle(stream)))

    def kernel_launches(self) -> int:
        return int(self._lib.molt_solver3d_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            self._lib.molt_solver3d_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _FchSteps:
    """Argument marshalling shared by the sixth-order solvers (``<prefix>_create / _step /
    _launches / _destroy`` of molt_fch1d_* and molt_fch2d_*)."""

    _prefix = ""

    def _open(self, shape, precision: str, eps: float, quad_order: int, tol: float, max_iter: int, create_args):
        lib = load_library()
        self._lib = lib
        self.shape = tuple(shape)
        self._itemsize = 4 if precision == "fp32" else 8
        self._params = _Params(eps, quad_order, PRECISION[precision], tol, max_iter)
        h = ctypes.c_void_p()
        _check(getattr(lib, self._prefix + "_create")(ctypes.byref(h), *create_args, ctypes.byref(self._params)))
        self._h = h

    def _field(self, t):
        if (not t.is_cuda or t.dtype.itemsize != self._itemsize or not t.is_floating_point() or not t.is_contiguous()
                or tuple(t.shape) != self.shape):
            raise ValueError(f"expected a contiguous CUDA tensor of shape {self.shape} with {self._itemsize}-byte floats")
        return ctypes.c_void_p(t.data_ptr())

    def step(self, u, dt: float, stream=None, raise_on_nonconvergence: bool = True) -> StepInfo:
        """One BE step in place on u; StepInfo with the iterations, residual and tolerance used."""
        info = _StepInfo()
        st = getattr(self._lib, self._prefix + "_step")(self._h, self._field(u), float(dt), _stream_handle(stream),
                                                        ctypes.byref(info))
        out = StepInfo(info.status, info.stages, list(info.iters)[: max(info.stages, 0)], info.total_iters,
                       info.residual, info.tol_used)
        if st == MOLT_ERR_NOT_CONVERGED and not raise_on_nonconvergence:
            return out
        _check(st, None)
        return out

    def kernel_launches(self) -> int:
        return int(getattr(self._lib, self._prefix + "_launches")(self._h))

    def close(self):
        if getattr(self, "_h", None):
            getattr(self._lib, self._prefix + "_destroy")(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Fch1D(_FchSteps):
    """BE steps of the sixth-order model on independent 1D lines (molt_fch1d_*): fields [lines][nx]
    of u (the paper's variable) in FP32 or FP64."""

    _prefix = "molt_fch1d"

    def __init__(self, nx: int, lines: int = 1, L: float = 6.283185307179586, bc: str = "periodic",
                 eps: float = 0.18, eta: float = 1.0, quad_order: int = 6, tol: float = 1e-10, max_iter: int = 500,
                 precision: str = "fp64"):
        self._open((lines, nx), precision, eps, quad_order, tol, max_iter, (nx, lines, L, BC[bc], float(eta)))


class Fch2D(_FchSteps):
    """BE steps of the sixth-order model on a 2D grid (molt_fch2d_*): fields [ny][nx] of u in FP32
    or FP64."""

    _prefix = "molt_fch2d"

    def __init__(self, nx: int, ny: int, Lx: float = 6.283185307179586, Ly: float = 6.283185307179586,
                 bc: str = "periodic", eps: float = 0.18, eta: float = 1.0, quad_order: int = 6, tol: float = 1e-10,
                 max_iter: int = 500, precision: str = "fp64"):
        self._open((ny, nx), precision, eps, quad_order, tol, max_iter, (nx, ny, Lx, Ly, BC[bc], float(eta)))
