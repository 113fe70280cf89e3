"""ctypes binding of libsmnn (include/smnn.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels; this module passes device
pointers of torch tensors, sizes and the current CUDA stream.  There is no CPU path:
if libsmnn.so cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

import torch

from . import _build

_HERE = os.path.dirname(os.path.abspath(__file__))

(SMNN_OK, SMNN_ERR_INVALID_ARG, SMNN_ERR_WORKSPACE, SMNN_ERR_CUDA, SMNN_ERR_UNSUPPORTED,
 SMNN_ERR_TOO_LARGE) = range(6)
F32_REFINED, F32, F64, F32_REFINED_DF = 0, 1, 2, 3
ALGO_AUTO, ALGO_SEQ, ALGO_CR, ALGO_CR_FUSED = 0, 1, 2, 3
SMNN_MAX_R = 3


class SmnnError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_string(status)} (status {status})")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("R_init", ctypes.c_int32), ("T_init", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("max_refine", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("adjoint_refine", ctypes.c_int32), ("w_gov", ctypes.c_double),
                ("w_init", ctypes.c_double), ("w_smooth", ctypes.c_double),
                ("refine_tol", ctypes.c_double), ("num_seq", ctypes.c_int64),
                ("dims_per_seq", ctypes.c_int64), ("T", ctypes.c_int64),
                ("seq_T", ctypes.POINTER(ctypes.c_int64)), ("V", ctypes.c_int32), ("Q", ctypes.c_int32),
                ("per_level_launches", ctypes.c_int32)]


class PlanStats(ctypes.Structure):
    _fields_ = [("num_systems", ctypes.c_int64), ("total_steps", ctypes.c_int64),
                ("num_levels", ctypes.c_int32), ("chunk", ctypes.c_int32 * 8),
                ("kernels_per_solve", ctypes.c_int32), ("workspace_bytes", ctypes.c_size_t),
                ("factor_bytes", ctypes.c_size_t)]


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 48), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


# Every symbol include/smnn.h declares, with (restype, argtypes).
_VP = ctypes.c_void_p
SYMBOLS = {
    "smnn_plan_create": (ctypes.c_int, [ctypes.POINTER(Desc), ctypes.POINTER(_VP)]),
    "smnn_plan_destroy": (ctypes.c_int, [_VP]),
    "smnn_plan_get_stats": (ctypes.c_int, [_VP, ctypes.POINTER(PlanStats)]),
    "smnn_workspace_size": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t),
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "smnn_assemble": (ctypes.c_int, [_VP] + [_VP] * 8 + [_VP]),
    "smnn_factor_solve": (ctypes.c_int, [_VP] + [_VP] * 8 + [_VP]),
    "smnn_backward": (ctypes.c_int, [_VP] + [_VP] * 14 + [_VP]),
    "smnn_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "smnn_launch_count": (ctypes.c_uint64, []),
    "smnn_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "smnn_profile_read": (ctypes.c_int, [ctypes.POINTER(KernelTime), ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int)]),
    "smnn_factor_solve_noalloc": (ctypes.c_int, [ctypes.POINTER(Desc)] + [_VP] * 7),
    "smnn_graph_create": (ctypes.c_int, [_VP] * 16 + [ctypes.POINTER(_VP)]),
    "smnn_graph_launch": (ctypes.c_int, [_VP, _VP]),
    "smnn_graph_destroy": (ctypes.c_int, [_VP]),
    "smnn_fma_rate": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_double), _VP]),
}


def _load() -> ctypes.CDLL:
    path = os.path.join(_HERE, "libsmnn.so")
    if not os.path.exists(path):
        path = _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SYMBOLS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()
LIB_PATH = lib._name


def status_string(status: int) -> str:
    return lib.smnn_status_string(int(status)).decode()


def fma_rate(fp64: bool = False, stream=None) -> float:
    """FMAs per second of the current device in FP32 (or FP64), measured (smnn_fma_rate)."""
    r = ctypes.c_double()
    _check(lib.smnn_fma_rate(1 if fp64 else 0, ctypes.byref(r), _stream(stream)), "smnn_fma_rate")
    return float(r.value)


def launch_count() -> int:
    return int(lib.smnn_launch_count())


def profile_enable(on: bool = True):
    """Start (clearing earlier records) or stop per-launch event timing."""
    _check(lib.smnn_profile_enable(1 if on else 0), "smnn_profile_enable")


def profile_read() -> dict:
    """{kernel name: (launches, total_ms)} of the launches timed since profile_enable."""
    buf = (KernelTime * 64)()
    n = ctypes.c_int()
    _check(lib.smnn_profile_read(buf, 64, ctypes.byref(n)), "smnn_profile_read")
    return {buf[k].name.decode(): (int(buf[k].launches), float(buf[k].total_ms))
            for k in range(min(n.value, 64))}


class StepGraph:
    """A step recorded by smnn_graph_create; launch(stream) replays it (one graph launch)."""

    def __init__(self, plan, bufs):
        self.plan, self.bufs = plan, bufs      # both must outlive the graph
        h = ctypes.c_void_p()
        _check(lib.smnn_graph_create(plan.handle, *[_p(t) for t in bufs], ctypes.byref(h)),
               "smnn_graph_create")
        self.handle = h

    def launch(self, stream=None):
        _check(lib.smnn_graph_launch(self.handle, _stream(stream)), "smnn_graph_launch")

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib.smnn_graph_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(status: int, where: str):
    if status != SMNN_OK:
        raise SmnnError(status, where)


def _p(t: torch.Tensor | None):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Plan:
    """A libsmnn plan: problem constants, batch shape and the level structure."""
    R: int
    R_init: int
    T_init: int
    B: int
    D: int
    T: int | None = None
    seq_T: tuple | None = None
    precision: int = F32_REFINED
    algo: int = ALGO_AUTO
    max_refine: int = 3
    adjoint_refine: int = 2
    chunk: int = 0
    w_gov: float = 1.0
    w_init: float = 1.0
    w_smooth: float = 1.0
    refine_tol: float = 0.0
    V: int = 1
    Q: int = 1
    per_level_launches: int = 0
    handle: ctypes.c_void_p = field(default=None, repr=False)

    def __post_init__(self):
        seq = None
        if self.seq_T is not None:
            self.seq_T = tuple(int(x) for x in self.seq_T)
            seq = (ctypes.c_int64 * len(self.seq_T))(*self.seq_T)
        d = Desc(self.R, self.R_init, self.T_init, self.precision, self.algo, self.max_refine,
                 self.chunk, self.adjoint_refine, self.w_gov, self.w_init, self.w_smooth, self.refine_tol, self.B,
                 self.D, int(self.T or 0), ctypes.cast(seq, ctypes.POINTER(ctypes.c_int64)), self.V, self.Q,
                 self.per_level_launches)
        h = ctypes.c_void_p()
        _check(lib.smnn_plan_create(ctypes.byref(d), ctypes.byref(h)), "smnn_plan_create")
        self.handle = h
        ws, fb = ctypes.c_size_t(), ctypes.c_size_t()
        _check(lib.smnn_workspace_size(h, ctypes.byref(ws), ctypes.byref(fb)), "smnn_workspace_size")
        self.workspace_bytes = int(ws.value)
        self.factor_bytes = int(fb.value)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            try:
                lib.smnn_plan_destroy(h)
            except Exception:  # interpreter shutdown
                pass
            self.handle = None

    @property
    def dtype(self):
        return torch.float64 if self.precision == F64 else torch.float32

    @property
    def S(self) -> int:
        return self.B * self.D

    @property
    def nb(self) -> int:
        """Unknowns per step, V (R+1)."""
        return self.V * (self.R + 1)

    @property
    def steps(self) -> int:
        return self.B * self.D * self.T if self.seq_T is None else self.D * sum(self.seq_T)

    def stats(self) -> PlanStats:
        st = PlanStats()
        _check(lib.smnn_plan_get_stats(self.handle, ctypes.byref(st)), "smnn_plan_get_stats")
        return st

    def workspace(self, device=None) -> torch.Tensor:
        """A fresh device workspace (torch's caching allocator; 256-byte aligned)."""
        return torch.empty(max(self.workspace_bytes, 1), dtype=torch.uint8, device=device or "cuda")

    def factor_buffer(self, device=None) -> torch.Tensor:
        return torch.empty(max(self.factor_bytes, 1), dtype=torch.uint8, device=device or "cuda")

    # ---- compute calls -------------------------------------------------------
    def _args_ok(self, *ts):
        for t in ts:
            if t is not None:
                if not t.is_cuda or not t.is_contiguous():
                    raise ValueError("smnn: every array must be a contiguous CUDA tensor")

    def assemble(self, c, d, s, u, M, N, beta, workspace=None, stream=None):
        workspace = self.workspace(c.device) if workspace is None else workspace
        self._args_ok(c, d, s, u, M, N, beta, workspace)
        _check(lib.smnn_assemble(self.handle, _p(c), _p(d), _p(s), _p(u), _p(M), _p(N), _p(beta),
                                 _p(workspace), _stream(stream)), "smnn_assemble")

    def factor_solve(self, c, d, s, u, y, info, workspace, factor=None, stream=None):
        self._args_ok(c, d, s, u, y, info, workspace, factor)
        _check(lib.smnn_factor_solve(self.handle, _p(c), _p(d), _p(s), _p(u), _p(y), _p(factor),
                                     _p(info), _p(workspace), _stream(stream)), "smnn_factor_solve")

    def backward(self, c, d, s, u, y, gy, gc, gd, gs, gu, info, workspace, factor=None, stream=None,
                 gw=None):
        """gw: optional float64 device tensor of 3 values, receives dl/d(w_gov, w_init, w_smooth)."""
        self._args_ok(c, d, s, u, y, gy, gc, gd, gs, gu, info, workspace, factor)
        if gw is not None and (gw.dtype != torch.float64 or gw.numel() < 3 or not gw.is_cuda):
            raise ValueError("gw must be a CUDA float64 tensor with 3 elements")
        _check(lib.smnn_backward(self.handle, _p(c), _p(d), _p(s), _p(u), _p(y), _p(factor),
                                 _p(gy), _p(gc), _p(gd), _p(gs), _p(gu), _p(gw), _p(info),
                                 _p(workspace), _stream(stream)), "smnn_backward")

    def graph(self, c, d, s, u, y, info, workspace, factor=None, gy=None, gc=None, gd=None,
              gs=None, gu=None, info_b=None, gw=None) -> "StepGraph":
        """Record factor_solve (and, with gy, backward) on these buffers as one CUDA graph
        (smnn_graph_create); the graph keeps references to the tensors."""
        self._args_ok(c, d, s, u, y, info, workspace, factor, gy, gc, gd, gs, gu, info_b, gw)
        return StepGraph(self, (c, d, s, u, y, factor, info, gy, gc, gd, gs, gu, gw, info_b, workspace))
