"""FP64 CPU oracle for the S-MNN least-squares solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may
import this package.  The product library (``paper_2410_06074_b300``) never imports,
loads or calls it, and the two share no code.

The arithmetic lives in ``smnn_oracle.c`` (plain C, FP64); see its header for what it
computes (Sec. 3.1 Eq. 4-9 and App. A.1: explicit rows of A, b, W; Eq. 9 by band or
dense Cholesky, or by Householder QR; Eq. 14 / App. A.3 chain rule for the gradients)
and which pins tie it to the paper.  This module only compiles that file and marshals
numpy arrays into it.

Array conventions (one "system" = one (sequence, dimension) pair of V variables with Q
governing equations per step; nb = V(R+1) unknowns per step, variable-major):
  uniform batch:  c [B, D, T, Q*nb], d [B, D, T, Q], s [B, T], u [B, D, T_init, V*(R_init+1)]
  ragged batch:   c [sum_i T_i, Q*nb], d [sum_i T_i, Q], s [sum_b T_b], u [S, T_init, V*(R_init+1)]
                  with ``seq_T`` giving T_b per sequence; system i = b*D + dd.
  With V = Q = 1 the trailing unit dimensions may be left out (c [..., R+1], d [B, D, T]).
  Solutions y have the layout of c with nb values per step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "smnn_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile smnn_oracle.c into liboracle.so (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("R_init", ctypes.c_int32), ("T_init", ctypes.c_int32),
                ("V", ctypes.c_int32), ("Q", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("w_gov", ctypes.c_double), ("w_init", ctypes.c_double), ("w_smooth", ctypes.c_double)]


@dataclass(frozen=True)
class Params:
    """Problem constants: R (order), R_init, T_init and the unsquared weights (Eq. 9)."""
    R: int = 2
    R_init: int = 1
    T_init: int = 1
    w_gov: float = 1.0
    w_init: float = 1.0
    w_smooth: float = 1.0
    V: int = 1
    Q: int = 1

    @property
    def nb(self) -> int:
        return self.V * (self.R + 1)

    def c(self) -> _Params:
        return _Params(self.R, self.R_init, self.T_init, self.V, self.Q, 0, self.w_gov, self.w_init,
                       self.w_smooth)


_P = ctypes.POINTER
_d = _P(ctypes.c_double)
_i64 = _P(ctypes.c_int64)
_i32 = _P(ctypes.c_int32)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        pp = _P(_Params)
        lib.orc_num_rows.restype = ctypes.c_int64
        lib.orc_num_rows.argtypes = [pp, ctypes.c_int64]
        lib.orc_dense_system.argtypes = [pp, ctypes.c_int64, _d, _d, _d, _d, _d, _d, _d]
        lib.orc_normal_band.argtypes = [pp, ctypes.c_int64, _d, _d, _d, _d, _d, _d]
        lib.orc_band_width.restype = ctypes.c_int
        lib.orc_band_width.argtypes = [pp]
        lib.orc_band_cholesky.restype = ctypes.c_int
        lib.orc_band_cholesky.argtypes = [ctypes.c_int64, ctypes.c_int, _d]
        lib.orc_band_solve.argtypes = [ctypes.c_int64, ctypes.c_int, _d, _d]
        lib.orc_solve_batch.restype = ctypes.c_int
        lib.orc_solve_batch.argtypes = [pp, ctypes.c_int64, _i64, _i64, _i64, _d, _d, _d, _d, _d,
                                        _i32, ctypes.c_int]
        lib.orc_grad_batch.restype = ctypes.c_int
        lib.orc_grad_batch.argtypes = [pp, ctypes.c_int64, _i64, _i64, _i64, _d, _d, _d, _d, _d, _d,
                                       _d, _d, _d, _d, _d, _d, _i32, ctypes.c_int]
        lib.orc_solve_qr_batch.restype = ctypes.c_int
        lib.orc_solve_qr_batch.argtypes = [pp, ctypes.c_int64, _i64, _i64, _i64, _d, _d, _d, _d, _d,
                                           _i32, ctypes.c_int]
        lib.orc_solve_dense_batch.restype = ctypes.c_int
        lib.orc_solve_dense_batch.argtypes = [pp, ctypes.c_int64, _i64, _i64, _i64, _d, _d, _d, _d,
                                              _d, _i32, ctypes.c_int]
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype=ctypes.c_double):
    return a.ctypes.data_as(_P(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def max_threads() -> int:
    return int(_load().orc_max_threads())


# --------------------------------------------------------------------------- layout

@dataclass
class _Layout:
    S: int
    T_sys: np.ndarray   # [S] int64
    off: np.ndarray     # [S] step offset of each system
    soff: np.ndarray    # [S] offset of each system's step sizes in s


def _y_like(p: Params, c, seq_T) -> np.ndarray:
    """Solution array: c's leading (step) dimensions with nb values per step."""
    lead = c.shape[:3] if seq_T is None else c.shape[:1]
    return np.zeros(lead + (p.nb,))


def _layout(c, D: int | None, seq_T) -> _Layout:
    if seq_T is None:  # uniform: c [B, D, T, ...]
        B, Dd, T = c.shape[0], c.shape[1], c.shape[2]
        S = B * Dd
        T_sys = np.full(S, T, np.int64)
        off = np.arange(S, dtype=np.int64) * T
        soff = (np.arange(S, dtype=np.int64) // Dd) * T
        return _Layout(S, T_sys, off, soff)
    seq_T = np.asarray(seq_T, np.int64)
    assert D is not None
    B = seq_T.shape[0]
    seq_off = np.concatenate([[0], np.cumsum(seq_T)[:-1]]).astype(np.int64)
    b_of = np.arange(B * D, dtype=np.int64) // D
    d_of = np.arange(B * D, dtype=np.int64) % D
    T_sys = seq_T[b_of]
    off = D * seq_off[b_of] + d_of * T_sys
    soff = seq_off[b_of]
    return _Layout(B * D, T_sys, off, soff)


# --------------------------------------------------------------------------- API

def num_rows(p: Params, T: int) -> int:
    """m of Eq. 8 (V = Q = 1)."""
    return int(_load().orc_num_rows(ctypes.byref(p.c()), T))


def dense_system(p: Params, c, d, s, u):
    """Explicit (A, b, w) of one system: c [T, R+1], d [T], s [T], u [T_init, R_init+1]."""
    c, d, s, u = _f64(c), _f64(d), _f64(s), _f64(u)
    T = c.shape[0]
    m, n = num_rows(p, T), T * p.nb
    A = np.zeros((m, n)); b = np.zeros(m); w = np.zeros(m)
    _load().orc_dense_system(ctypes.byref(p.c()), T, _ptr(c), _ptr(d), _ptr(s), _ptr(u),
                             _ptr(A), _ptr(b), _ptr(w))
    return A, b, w


def normal_band(p: Params, c, d, s, u):
    """Lower band of M (rows i, offsets i-j = 0..kd) and beta of one system."""
    c, d, s, u = _f64(c), _f64(d), _f64(s), _f64(u)
    T = c.shape[0]
    n = T * p.nb
    kd = int(_load().orc_band_width(ctypes.byref(p.c())))
    band = np.zeros((n, kd + 1)); beta = np.zeros(n)
    _load().orc_normal_band(ctypes.byref(p.c()), T, _ptr(c), _ptr(d), _ptr(s), _ptr(u),
                            _ptr(band), _ptr(beta))
    return band, beta


def band_cholesky_solve(band, rhs):
    """Factor a lower band matrix (as returned by normal_band) and solve with it."""
    band = _f64(band).copy(); x = _f64(rhs).copy()
    n, kd1 = band.shape
    info = _load().orc_band_cholesky(n, kd1 - 1, _ptr(band))
    if info == 0:
        _load().orc_band_solve(n, kd1 - 1, _ptr(band), _ptr(x))
    return x, int(info)


def solve(p: Params, c, d, s, u, *, D: int | None = None, seq_T=None, mode: str = "band",
          nthreads: int = 0):
    """y for every system (Eq. 9).  mode: 'band' (band Cholesky of M, any T), 'band_qr'
    (plane-rotation QR of W^{1/2} A in band storage, any T: no normal equations, for
    ill-conditioned problems), 'dense' (dense Cholesky of M) or 'qr' (Householder QR of
    W^{1/2} A).  Returns (y, info)."""
    c, d, s, u = _f64(c), _f64(d), _f64(s), _f64(u)
    L = _layout(c, D, seq_T)
    y = _y_like(p, c, seq_T)
    info = np.zeros(L.S, np.int32)
    args = (ctypes.byref(p.c()), L.S, _ptr(L.T_sys, ctypes.c_int64), _ptr(L.off, ctypes.c_int64),
            _ptr(L.soff, ctypes.c_int64), _ptr(c), _ptr(d), _ptr(s), _ptr(u), _ptr(y),
            _ptr(info, ctypes.c_int32))
    if mode == "band":
        rc = _load().orc_solve_batch(*args, int(nthreads))
    elif mode == "band_qr":
        rc = _load().orc_solve_qr_batch(*args, int(nthreads))
    elif mode in ("dense", "qr"):
        rc = _load().orc_solve_dense_batch(*args, 0 if mode == "dense" else 1)
    else:
        raise ValueError(mode)
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    return y, info


def gradient(p: Params, c, d, s, u, gy, *, D: int | None = None, seq_T=None, nthreads: int = 0,
             weights: bool = False):
    """(y, gc, gd, gs, gu, info) for dl/dy = gy (Eq. 14 chain rule, App. A.3).  With
    weights=True, (y, gc, gd, gs, gu, gw, info): gw [3] = dl/d(w_gov, w_init, w_smooth),
    the importance weights being shared by every system of the batch (summed in order)."""
    c, d, s, u, gy = _f64(c), _f64(d), _f64(s), _f64(u), _f64(gy)
    L = _layout(c, D, seq_T)
    y = _y_like(p, c, seq_T); gc = np.zeros_like(c); gd = np.zeros_like(d)
    gs = np.zeros_like(s); gu = np.zeros_like(u); gs_sys = np.zeros(int(L.T_sys.sum()))
    gw_sys = np.zeros((L.S, 3))
    info = np.zeros(L.S, np.int32)
    rc = _load().orc_grad_batch(ctypes.byref(p.c()), L.S, _ptr(L.T_sys, ctypes.c_int64),
                                _ptr(L.off, ctypes.c_int64), _ptr(L.soff, ctypes.c_int64),
                                _ptr(c), _ptr(d), _ptr(s), _ptr(u), _ptr(gy), _ptr(y), _ptr(gc),
                                _ptr(gd), _ptr(gs), _ptr(gu), _ptr(gs_sys), _ptr(gw_sys),
                                _ptr(info, ctypes.c_int32), int(nthreads))
    if rc != 0:
        raise ValueError("oracle rejected the parameters")
    if weights:
        gw = np.zeros(3)
        for i in range(L.S):
            gw += gw_sys[i]
        return y, gc, gd, gs, gu, gw, info
    return y, gc, gd, gs, gu, info
