"""Thin Python binding of the C ABI in include/opf_admm.h (ctypes).

Argument marshalling only: every step of the solve runs in libopf_admm.so
(host precompute in C++, iterations in sm_103a kernels).  There is no CPU
fallback: importing this module raises if the library is missing, and
device calls raise if CUDA is unavailable.  PyTorch supplies the device
memory arena (caching allocator) and the stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import feeders as _F

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libopf_admm.so")
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libopf_admm.so not built ({_LIB_PATH}); run python -m paper_2501_08293_b300.build")
lib = C.CDLL(_LIB_PATH)

OK, NOT_CONVERGED = 0, 1
CRIT_ABS, CRIT_REL, CRIT_BOTH, CRIT_NEVER = 0, 1, 2, 3
FP64, FP32 = 0, 1
RES_PAPER, RES_TEXTBOOK = 0, 1
DECOMP_FINE, DECOMP_PAPER = 0, 1
SC_XUPDATE_CUDA_CORES, SC_XUPDATE_TENSOR = 0, 1
ENGINE_AUTO, ENGINE_GRAPH, ENGINE_HOSTLOOP, ENGINE_PERSISTENT = 0, 1, 2, 3


class Params(C.Structure):
    _fields_ = [("rho", C.c_double), ("eps_abs_prim", C.c_double), ("eps_abs_dual", C.c_double),
                ("eps_rel", C.c_double), ("criterion", C.c_int32), ("max_iter", C.c_int32),
                ("check_every", C.c_int32), ("precision", C.c_int32), ("residual_form", C.c_int32),
                ("warm_start", C.c_int32), ("engine", C.c_int32), ("adaptive_rho", C.c_int32),
                ("rb_mu", C.c_double), ("rb_tau", C.c_double)]


class CreateOptions(C.Structure):
    _fields_ = [("chunks", C.c_int32), ("decomposition", C.c_int32), ("_reserved", C.c_int32 * 6)]


class Info(C.Structure):
    _fields_ = [("status", C.c_int32), ("iters", C.c_int32), ("first_rel_iter", C.c_int32),
                ("rho_changes", C.c_int32), ("pres", C.c_double), ("dres", C.c_double),
                ("eps_prim", C.c_double), ("eps_dual", C.c_double), ("objective", C.c_double),
                ("seconds", C.c_double), ("rho", C.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("_")}


class Dims(C.Structure):
    _fields_ = [("n_global", C.c_int32), ("n_local", C.c_int32), ("n_comp", C.c_int32),
                ("n_rows", C.c_int32), ("n_rows_reduced", C.c_int32), ("max_n", C.c_int32),
                ("n_tiles", C.c_int32), ("n_blocks", C.c_int32), ("sum_n2", C.c_int64),
                ("device_bytes", C.c_int64), ("max_chunk_locals", C.c_int32),
                ("max_chunk_halo", C.c_int32), ("max_chunk_operator", C.c_int32),
                ("max_chunk_copies", C.c_int32)]


class ServerConfig(C.Structure):
    _fields_ = [("device_budget_bytes", C.c_int64), ("max_active", C.c_int32), ("round_iters", C.c_int32),
                ("max_chunks", C.c_int32), ("iters_per_bus", C.c_int32), ("_reserved", C.c_int32 * 2),
                ("params", Params)]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("submitted", "admitted", "completed", "converged", "warm_started",
                                         "evicted", "rounds", "iterations", "resident_bytes")] + \
               [("active", C.c_int32), ("pending", C.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int32)
EXPORTS = {
    "opf_abi_version": (C.c_int32, []),
    "opf_record_size": (C.c_size_t, [C.c_int32]),
    "opf_status_string": (C.c_char_p, [C.c_int32]),
    "opf_last_error": (C.c_char_p, []),
    "opf_params_default": (None, [C.POINTER(Params)]),
    "opf_problem_create": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P, C.c_int32,
                                       C.POINTER(C.c_void_p)]),
    "opf_problem_create_ex": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P, C.c_int32,
                                          C.POINTER(CreateOptions), C.POINTER(C.c_void_p)]),
    "opf_get_dims": (C.c_int32, [_P, C.POINTER(Dims)]),
    "opf_update_lines": (C.c_int32, [_P, _I, _P, C.c_int32, _P]),
    "opf_set_line_status": (C.c_int32, [_P, C.c_int32, C.c_int32, _P, _I]),
    "opf_problem_upload": (C.c_int32, [_P, _P, C.c_size_t, _P]),
    "opf_admm_solve": (C.c_int32, [_P, C.POINTER(Params), _P, C.POINTER(Info)]),
    "opf_get_state": (C.c_int32, [_P, _D, _D, _D, _P]),
    "opf_set_state": (C.c_int32, [_P, _D, _D, _P]),
    "opf_get_structure": (C.c_int32, [_P, _I, _I, _I, _I, _I]),
    "opf_get_solution": (C.c_int32, [_P] + [_D] * 11 + [_P]),
    "opf_get_operator": (C.c_int32, [_P, C.c_int32, _D, _D, _I]),
    "opf_profile_kernels": (C.c_int32, [_P, C.POINTER(Params), C.c_int32, _P, _D]),
    "opf_debug_config": (C.c_int32, [_P, C.c_int64, C.c_int32, C.c_int32]),
    "opf_engine_for": (C.c_int32, [_P, C.c_int32, _I]),
    "opf_profile_persistent": (C.c_int32, [_P, C.POINTER(Params), C.c_int32, _P, _D]),
    "opf_profile_persistent_ctas": (C.c_int32, [_P, C.POINTER(Params), C.c_int32, _P, _D]),
    "opf_chunk_stats": (C.c_int32, [_P, _I]),
    "opf_residuals_noalloc": (C.c_int32, [_P, _P, _P, _P, C.c_int64, C.c_double, C.c_double, _P, _P]),
    "opf_component_operator": (C.c_int32, [_D, _D, C.c_int32, C.c_int32, _D, _D, _I]),
    "opf_tuning_set": (C.c_int32, [C.c_char_p, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "opf_tuning_clear": (C.c_int32, []),
    "opf_tuning_load": (C.c_int32, [C.c_char_p, _I]),
    "opf_tuning_lookup": (C.c_int32, [C.c_int32, _I, _I]),
    "opf_destroy": (None, [_P]),
    "opf_batch_create": (C.c_int32, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(C.c_void_p)]),
    "opf_batch_solve": (C.c_int32, [_P, C.POINTER(Params), C.c_int32, _P, C.POINTER(Info)]),
    "opf_batch_destroy": (None, [_P]),
    "opf_batch_capacity": (C.c_int32, [C.c_int32, _I]),
    "opf_batch_engine_for": (C.c_int32, [_P, C.c_int32, _I]),
    "opf_batch_profile_kernels": (C.c_int32, [_P, C.POINTER(Params), C.c_int32, _P, _D]),
    "opf_scenarios_create": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P, C.c_int32, C.c_int32,
                                         C.POINTER(C.c_void_p)]),
    "opf_scenarios_solve": (C.c_int32, [_P, C.POINTER(Params), _P, C.POINTER(Info)]),
    "opf_scenarios_get_state": (C.c_int32, [_P, C.c_int32, _D, _D, _D, _P]),
    "opf_scenarios_dims": (C.c_int32, [_P, _I, _I, C.POINTER(C.c_int64)]),
    "opf_scenarios_profile": (C.c_int32, [_P, C.POINTER(Params), C.c_int32, _P, _D]),
    "opf_scenarios_set_xupdate": (C.c_int32, [_P, C.c_int32]),
    "opf_scenarios_destroy": (None, [_P]),
    "opf_server_config_default": (None, [C.POINTER(ServerConfig)]),
    "opf_server_create": (C.c_int32, [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]),
    "opf_server_submit": (C.c_int32, [_P, _P, C.c_int32, _P, C.c_int32, _P, C.c_int32, _P, C.c_int32,
                                      C.c_int32, C.c_int64, C.POINTER(C.c_int64)]),
    "opf_server_step": (C.c_int32, [_P, _P, _I, _I]),
    "opf_server_poll": (C.c_int32, [_P, C.POINTER(C.c_int64), C.POINTER(Info), C.c_int32, _I]),
    "opf_server_problem": (C.c_int32, [_P, C.c_int64, C.POINTER(C.c_void_p)]),
    "opf_server_get_stats": (C.c_int32, [_P, C.POINTER(ServerStats)]),
    "opf_server_destroy": (None, [_P]),
}
for _name, (_res, _args) in EXPORTS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


# the tuning table written by autotune.py for this package, if there is one
# (entries are keyed by GPU name, so other devices keep the defaults)
_TUNING_PATH = os.path.join(os.path.dirname(_LIB_PATH), "tuning.json")
if os.path.exists(_TUNING_PATH):
    if lib.opf_tuning_load(_TUNING_PATH.encode(), None) != 0:
        import warnings
        warnings.warn(f"{_TUNING_PATH}: {lib.opf_last_error().decode()}; automatic chunking keeps its defaults")


class OpfError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib.opf_last_error().decode()
        super().__init__(f"{where}: {lib.opf_status_string(status).decode()} ({status}): {msg}")


def _check(st: int, where: str) -> int:
    if st < 0:
        raise OpfError(st, where)
    return st


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def default_params(**kw) -> Params:
    p = Params()
    lib.opf_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _stream_handle(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def residuals_noalloc(v, x_local, x_local_prev, lam, rho: float, eps_rel: float, out, stream=None) -> None:
    """Allocation-free residual norms (opf_residuals_noalloc) for callers that
    may not allocate device memory.  All arguments are CUDA tensors of
    float64 (out: 4 elements, receives pres, dres, eps_prim, eps_dual);
    nothing is allocated by the library and the call does not synchronize."""
    n = int(x_local.numel())
    for t in (v, x_local, x_local_prev, lam, out):
        if not t.is_cuda or t.dtype.itemsize != 8 or not t.is_contiguous():
            raise TypeError("expected contiguous float64 CUDA tensors")
    if v.numel() != n or x_local_prev.numel() != n or lam.numel() != n or out.numel() < 4:
        raise ValueError("size mismatch")
    _check(lib.opf_residuals_noalloc(v.data_ptr(), x_local.data_ptr(), x_local_prev.data_ptr(), lam.data_ptr(),
                                     n, rho, eps_rel, out.data_ptr(), _stream_handle(stream)),
           "opf_residuals_noalloc")


def tuning_load(path: str) -> int:
    """Load a tuning table written by autotune.py (opf_tuning_load); returns
    the number of entries read."""
    n = C.c_int32()
    _check(lib.opf_tuning_load(str(path).encode(), C.byref(n)), "opf_tuning_load")
    return n.value


def tuning_set(gpu: str, n_bus_lo: int, n_bus_hi: int, work_per_chunk: int, max_chunks: int) -> None:
    _check(lib.opf_tuning_set(gpu.encode(), int(n_bus_lo), int(n_bus_hi), int(work_per_chunk), int(max_chunks)),
           "opf_tuning_set")


def tuning_clear() -> None:
    lib.opf_tuning_clear()


def tuning_lookup(n_bus: int):
    """(work_per_chunk, max_chunks) that automatic chunking uses for a feeder
    of n_bus buses on the current device."""
    w, m = C.c_int32(), C.c_int32()
    _check(lib.opf_tuning_lookup(int(n_bus), C.byref(w), C.byref(m)), "opf_tuning_lookup")
    return w.value, m.value


def component_operator(A, b):
    """P = -Abar_s and bbar_s of Eq. (closed_2) for caller-given rows A_s, b_s
    after row reduction (opf_component_operator, host only); returns
    (P, bbar, m_reduced)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    m, n = A.shape
    P = np.empty((n, n))
    bbar = np.empty(n)
    mr = C.c_int32()
    _check(lib.opf_component_operator(_dp(A) if m else None, _dp(b) if m else None, m, n, _dp(P), _dp(bbar),
                                      C.byref(mr)), "opf_component_operator")
    return P, bbar, mr.value


class Problem:
    """One feeder: host precompute at construction, device arena from torch."""

    def __init__(self, buses, lines, gens, loads, *, device=None, stream=None, upload=True, chunks: int = 0,
                 decomposition: int = DECOMP_FINE):
        self._h = C.c_void_p()
        # private copies: later record updates (update_lines, set_line_status)
        # must not write into the caller's arrays
        self._arrays = [np.array(a, copy=True, order="C") for a in (buses, lines, gens, loads)]
        for a, dt in zip(self._arrays, (_F.BUS_DTYPE, _F.LINE_DTYPE, _F.GEN_DTYPE, _F.LOAD_DTYPE)):
            if a.dtype != dt:
                raise TypeError(f"record array has dtype {a.dtype}, expected {dt}")
        b, l, g, d = self._arrays
        opts = CreateOptions()
        opts.chunks = int(chunks)
        opts.decomposition = int(decomposition)
        _check(lib.opf_problem_create_ex(b.ctypes.data, len(b), l.ctypes.data, len(l), g.ctypes.data, len(g),
                                         d.ctypes.data, len(d), C.byref(opts), C.byref(self._h)),
               "opf_problem_create_ex")
        self.dims = Dims()
        _check(lib.opf_get_dims(self._h, C.byref(self.dims)), "opf_get_dims")
        self.n_bus, self.n_line, self.n_gen, self.n_load = len(b), len(l), len(g), len(d)
        self._arena = None
        self._device_owned = False
        if upload:
            self.upload(device=device, stream=stream)

    @classmethod
    def from_feeder(cls, f, **kw) -> "Problem":
        return cls(f.buses, f.lines, f.gens, f.loads, **kw)

    @classmethod
    def borrowed(cls, handle, n_bus, n_line, n_gen, n_load) -> "Problem":
        """Non-owning view of a handle owned elsewhere (e.g. a server)."""
        p = cls.__new__(cls)
        p._h = C.c_void_p(handle)
        p._arrays = []
        p.dims = Dims()
        _check(lib.opf_get_dims(p._h, C.byref(p.dims)), "opf_get_dims")
        p.n_bus, p.n_line, p.n_gen, p.n_load = n_bus, n_line, n_gen, n_load
        p._arena = None
        p._device_owned = False
        p._borrowed = True
        return p

    def upload(self, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the solver has no CPU path")
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(dev):
            nbytes = int(self.dims.device_bytes)
            self._arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
            base = self._arena.data_ptr()
            off = (-base) % 256
            _check(lib.opf_problem_upload(self._h, C.c_void_p(base + off), nbytes, _stream_handle(stream)),
                   "opf_problem_upload")

    def solve(self, params: Params | None = None, stream=None, **kw) -> Info:
        p = params if params is not None else default_params()
        for k, v in kw.items():
            setattr(p, k, v)
        info = Info()
        _check(lib.opf_admm_solve(self._h, C.byref(p), _stream_handle(stream), C.byref(info)), "opf_admm_solve")
        return info

    def profile_kernels(self, params: Params | None = None, reps: int = 200, stream=None) -> dict:
        """Average microseconds per launch of each kernel (CUDA events)."""
        p = params if params is not None else default_params()
        us = np.zeros(4)
        _check(lib.opf_profile_kernels(self._h, C.byref(p), reps, _stream_handle(stream), _dp(us)),
               "opf_profile_kernels")
        return dict(z=us[0], x=us[1], x_partials=us[2], finalize=us[3])

    def profile_persistent(self, params: Params | None = None, iters: int = 2000, stream=None) -> dict:
        """Per-iteration microseconds of each persistent-kernel phase (mean, max over CTAs)."""
        p = params if params is not None else default_params()
        out = np.zeros(8)
        _check(lib.opf_profile_persistent(self._h, C.byref(p), int(iters), _stream_handle(stream), _dp(out)),
               "opf_profile_persistent")
        names = ("global_interior", "global_boundary_wait", "local_boundary", "local_interior_check")
        return {"mean": dict(zip(names, out[:4])), "max": dict(zip(names, out[4:]))}

    def profile_persistent_ctas(self, params: Params | None = None, iters: int = 2000, stream=None) -> np.ndarray:
        """Per-CTA microseconds per iteration of each phase, shape (n_blocks, 4)."""
        p = params if params is not None else default_params()
        out = np.zeros((self.dims.n_blocks, 4))
        _check(lib.opf_profile_persistent_ctas(self._h, C.byref(p), int(iters), _stream_handle(stream), _dp(out)),
               "opf_profile_persistent_ctas")
        return out

    CHUNK_STATS = ("tiles", "interior_tiles", "quads", "max_warp_quads", "halo", "boundary_halo", "copies",
                   "external_copies", "neighbours", "locals")

    def chunk_stats(self) -> dict:
        """Per-chunk layout statistics (opf_chunk_stats), one array per name."""
        out = np.zeros((self.dims.n_blocks, len(self.CHUNK_STATS)), dtype=np.int32)
        _check(lib.opf_chunk_stats(self._h, out.ctypes.data_as(_I)), "opf_chunk_stats")
        return {k: out[:, i].copy() for i, k in enumerate(self.CHUNK_STATS)}

    def update_lines(self, idx, records, stream=None):
        """New parameters for in-service lines (same ends, phases, service
        state); operators recomputed on the device, iterate kept."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        rec = np.ascontiguousarray(records)
        if rec.dtype != _F.LINE_DTYPE or len(rec) != len(idx):
            raise TypeError("records must be LINE records, one per index")
        _check(lib.opf_update_lines(self._h, idx.ctypes.data_as(_I), rec.ctypes.data, len(idx),
                                    _stream_handle(stream)), "opf_update_lines")
        for k, e in enumerate(idx):
            self._arrays[1][e] = rec[k]

    def set_line_status(self, line: int, in_service: bool, stream=None) -> int:
        """Switch a line in or out of service (opf_set_line_status): the
        problem is rebuilt on the host (operators recomputed only for the
        touched components, whose count is returned) and, when uploaded, the
        iterate is carried over on the device; the library then owns its
        device arena.  Continue with solve(..., warm_start=1)."""
        n = C.c_int32()
        _check(lib.opf_set_line_status(self._h, int(line), int(bool(in_service)), _stream_handle(stream)
                                       if self._arena is not None or self._device_owned else None, C.byref(n)),
               "opf_set_line_status")
        self._arrays[1]["in_service"][int(line)] = int(bool(in_service))
        _check(lib.opf_get_dims(self._h, C.byref(self.dims)), "opf_get_dims")
        if self._arena is not None:
            self._device_owned = True       # the library allocated a new arena; torch's is free again
            self._arena = None
        return n.value

    def persistent_ok(self, params: Params) -> bool:
        e = C.c_int32()
        _check(lib.opf_engine_for(self._h, params.precision, C.byref(e)), "opf_engine_for")
        return e.value == ENGINE_PERSISTENT

    def debug_config(self, wait_limit_ns: int = 2_000_000_000, withhold_block: int = -1, variant: int = 0):
        _check(lib.opf_debug_config(self._h, int(wait_limit_ns), int(withhold_block), int(variant)),
               "opf_debug_config")

    def state(self, stream=None):
        xg = np.empty(self.dims.n_global)
        xl = np.empty(self.dims.n_local)
        lam = np.empty(self.dims.n_local)
        _check(lib.opf_get_state(self._h, _dp(xg), _dp(xl), _dp(lam), _stream_handle(stream)), "opf_get_state")
        return xg, xl, lam

    def set_state(self, xl, lam, stream=None):
        xl = np.ascontiguousarray(xl, dtype=np.float64)
        lam = np.ascontiguousarray(lam, dtype=np.float64)
        _check(lib.opf_set_state(self._h, _dp(xl), _dp(lam), _stream_handle(stream)), "opf_set_state")

    def structure(self):
        S, nl = self.dims.n_comp, self.dims.n_local
        ptr = np.empty(S + 1, np.int32); kind = np.empty(S, np.int32); idx = np.empty(S, np.int32)
        gidx = np.empty(nl, np.int32); mred = np.empty(S, np.int32)
        ip = lambda a: a.ctypes.data_as(_I)
        _check(lib.opf_get_structure(self._h, ip(ptr), ip(kind), ip(idx), ip(gidx), ip(mred)), "opf_get_structure")
        return dict(comp_ptr=ptr, kind=kind, index=idx, gidx=gidx, m_reduced=mred)

    def operator(self, s: int):
        n = C.c_int32()
        _check(lib.opf_get_operator(self._h, s, None, None, C.byref(n)), "opf_get_operator")
        P = np.empty((n.value, n.value))
        bbar = np.empty(n.value)
        _check(lib.opf_get_operator(self._h, s, _dp(P), _dp(bbar), None), "opf_get_operator")
        return P, bbar

    def solution(self, stream=None) -> dict:
        shp = {"w": self.n_bus, "pg": self.n_gen, "qg": self.n_gen, "p_ij": self.n_line, "q_ij": self.n_line,
               "p_ji": self.n_line, "q_ji": self.n_line, "pd": self.n_load, "qd": self.n_load,
               "pb": self.n_load, "qb": self.n_load}
        out = {k: np.empty((n, 3)) for k, n in shp.items()}
        _check(lib.opf_get_solution(self._h, *[_dp(out[k]) for k in shp], _stream_handle(stream)),
               "opf_get_solution")
        return out

    def close(self):
        if self._h and not getattr(self, "_borrowed", False):
            lib.opf_destroy(self._h)
        self._h = C.c_void_p()
        self._arena = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def batch_capacity(precision: int = FP32) -> int:
    """Co-resident chunks (CTAs) a batch launch can hold on the current device."""
    n = C.c_int32()
    _check(lib.opf_batch_capacity(int(precision), C.byref(n)), "opf_batch_capacity")
    return n.value


class Batch:
    """Several uploaded problems solved in one cooperative launch."""

    def __init__(self, problems):
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p._h.value for p in self.problems])
        self._h = C.c_void_p()
        _check(lib.opf_batch_create(arr, len(self.problems), C.byref(self._h)), "opf_batch_create")

    def solve(self, params, stream=None):
        """params: one Params for all instances or a list (one per instance)."""
        plist = params if isinstance(params, (list, tuple)) else [params]
        arr = (Params * len(plist))(*plist)
        infos = (Info * len(self.problems))()
        _check(lib.opf_batch_solve(self._h, arr, len(plist), _stream_handle(stream), infos), "opf_batch_solve")
        return list(infos)

    def profile_kernels(self, params: Params | None = None, reps: int = 20, stream=None) -> dict:
        """Average microseconds per launch of each batched-graph kernel (CUDA events)."""
        p = params if params is not None else default_params()
        us = np.zeros(4)
        _check(lib.opf_batch_profile_kernels(self._h, C.byref(p), reps, _stream_handle(stream), _dp(us)),
               "opf_batch_profile_kernels")
        return dict(z=us[0], x=us[1], x_partials=us[2], x_chunk=us[3])

    def auto_engine(self, precision: int = FP32) -> int:
        """Engine that ENGINE_AUTO runs for this batch (opf_batch_engine_for)."""
        e = C.c_int32()
        _check(lib.opf_batch_engine_for(self._h, int(precision), C.byref(e)), "opf_batch_engine_for")
        return e.value

    def close(self):
        if self._h:
            lib.opf_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scenarios:
    """Many load scenarios on one topology iterated together (opf_scenarios_*).
    loads: array of shape (n_scenarios, n_load) of LOAD records."""

    def __init__(self, buses, lines, gens, loads, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("CUDA is not available: the solver has no CPU path")
        arrs = [np.ascontiguousarray(a) for a in (buses, lines, gens)]
        ld = np.ascontiguousarray(loads)
        if ld.ndim != 2 or ld.dtype != _F.LOAD_DTYPE:
            raise TypeError("loads must be a (n_scenarios, n_load) array of LOAD records")
        self.n, n_load = ld.shape
        self._keep = arrs + [ld]
        self._h = C.c_void_p()
        _check(lib.opf_scenarios_create(arrs[0].ctypes.data, len(arrs[0]), arrs[1].ctypes.data, len(arrs[1]),
                                        arrs[2].ctypes.data, len(arrs[2]), ld.ctypes.data, n_load, self.n,
                                        C.byref(self._h)), "opf_scenarios_create")
        ng, nl, nb = C.c_int32(), C.c_int32(), C.c_int64()
        _check(lib.opf_scenarios_dims(self._h, C.byref(ng), C.byref(nl), C.byref(nb)), "opf_scenarios_dims")
        self.n_global, self.n_local, self.device_bytes = ng.value, nl.value, nb.value

    @classmethod
    def from_feeder(cls, f, loads, **kw) -> "Scenarios":
        return cls(f.buses, f.lines, f.gens, loads, **kw)

    def solve(self, params: Params, stream=None) -> list:
        infos = (Info * self.n)()
        _check(lib.opf_scenarios_solve(self._h, C.byref(params), _stream_handle(stream), infos),
               "opf_scenarios_solve")
        return list(infos)

    def set_xupdate(self, kind: int) -> None:
        """Small shared-operator local update on CUDA cores (bit-identical to
        single-instance FP32) or on tensor cores (3xTF32)."""
        _check(lib.opf_scenarios_set_xupdate(self._h, int(kind)), "opf_scenarios_set_xupdate")

    def profile(self, params: Params, reps: int = 50, stream=None) -> dict:
        """Per-kernel microseconds of one iteration (opf_scenarios_profile)."""
        us = np.zeros(5)
        _check(lib.opf_scenarios_profile(self._h, C.byref(params), int(reps), _stream_handle(stream), _dp(us)),
               "opf_scenarios_profile")
        return dict(zip(("z", "x_small", "x_large", "x_check", "check"), us.tolist()))

    def state(self, k: int, stream=None):
        xg = np.empty(self.n_global)
        xl = np.empty(self.n_local)
        lam = np.empty(self.n_local)
        _check(lib.opf_scenarios_get_state(self._h, int(k), _dp(xg), _dp(xl), _dp(lam), _stream_handle(stream)),
               "opf_scenarios_get_state")
        return xg, xl, lam

    def close(self):
        if self._h:
            lib.opf_scenarios_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def default_server_config(**kw) -> ServerConfig:
    c = ServerConfig()
    lib.opf_server_config_default(C.byref(c))
    for k, v in kw.items():
        if k in ("device_budget_bytes", "max_active", "round_iters", "max_chunks", "iters_per_bus"):
            setattr(c, k, v)
        else:
            setattr(c.params, k, v)
    return c


class Server:
    """Continuous-batching OPF server (opf_server_*)."""

    def __init__(self, config: ServerConfig | None = None, **kw):
        cfg = config if config is not None else default_server_config(**kw)
        self._h = C.c_void_p()
        _check(lib.opf_server_create(C.byref(cfg), C.byref(self._h)), "opf_server_create")
        self._shapes = {}

    def submit(self, f, warm_from: int = -1, chunks: int = 0) -> int:
        arrs = [np.ascontiguousarray(a) for a in (f.buses, f.lines, f.gens, f.loads)]
        rid = C.c_int64()
        _check(lib.opf_server_submit(self._h, arrs[0].ctypes.data, len(arrs[0]), arrs[1].ctypes.data, len(arrs[1]),
                                     arrs[2].ctypes.data, len(arrs[2]), arrs[3].ctypes.data, len(arrs[3]),
                                     int(chunks), int(warm_from), C.byref(rid)), "opf_server_submit")
        self._shapes[rid.value] = tuple(len(a) for a in arrs)
        return rid.value

    def step(self, stream=None):
        na, npend = C.c_int32(), C.c_int32()
        _check(lib.opf_server_step(self._h, _stream_handle(stream), C.byref(na), C.byref(npend)), "opf_server_step")
        return na.value, npend.value

    def poll(self, cap: int = 1024):
        ids = (C.c_int64 * cap)()
        infos = (Info * cap)()
        n = C.c_int32()
        _check(lib.opf_server_poll(self._h, ids, infos, cap, C.byref(n)), "opf_server_poll")
        return [(ids[k], infos[k]) for k in range(n.value)]

    def problem(self, rid: int) -> Problem:
        h = C.c_void_p()
        _check(lib.opf_server_problem(self._h, int(rid), C.byref(h)), "opf_server_problem")
        return Problem.borrowed(h.value, *self._shapes[rid])

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib.opf_server_get_stats(self._h, C.byref(st)), "opf_server_get_stats")
        return st.as_dict()

    def close(self):
        if self._h:
            lib.opf_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
