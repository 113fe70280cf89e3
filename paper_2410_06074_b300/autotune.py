"""Autotuner for the level structure of the chunked solve.

For a batch shape (R, number of systems, steps per system) and precision it times the
candidates -- the default plan, one sequential block-Cholesky sweep per system
(SMNN_ALGO_SEQ, Alg. 3/4 as written), the chunked cyclic reduction with level-0 chunks of 8,
16, 32 or 64 steps, and the same reduction in one launch per solve pass (SMNN_ALGO_CR_FUSED,
where every system fits a CTA; the plan is refused otherwise) -- on the caller's inputs,
forward + adjoint, each as replays of the library's CUDA graph of the step (device time, as
a training loop runs it, without the host's launch overhead), after checking that each
candidate reproduces the default plan's solution (so no candidate is ever picked for speed
alone).  Winners are kept in
``autotune_table.json`` next to this file, keyed by R, precision and power-of-two buckets of the
system count and the mean steps per system; ``api.get_plan`` consults the table whenever a
``SolveConfig`` asks for ``ALGO_AUTO`` with ``chunk = 0``.
"""
from __future__ import annotations

import json
import math
import os
import threading
from dataclasses import replace

import torch

from . import binding as B

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_table.json")
_lock = threading.Lock()
_table = None

CANDIDATES = [(B.ALGO_AUTO, 0), (B.ALGO_SEQ, 0)] + [(B.ALGO_AUTO, L) for L in (8, 16, 32, 64)] + \
    [(B.ALGO_CR_FUSED, L) for L in (16, 32, 64)]


def _bucket(x: float) -> int:
    return int(round(math.log2(max(x, 1.0))))


def key(R: int, S: int, steps: int, precision: int) -> str:
    return f"R{R}/P{precision}/S2^{_bucket(S)}/T2^{_bucket(steps / max(S, 1))}"


def table() -> dict:
    global _table
    with _lock:
        if _table is None:
            try:
                with open(TABLE) as f:
                    _table = json.load(f)
            except (OSError, ValueError):
                _table = {}
        return _table


def lookup(R: int, S: int, steps: int, precision: int):
    """(algo, chunk) recorded for this shape bucket, or None."""
    e = table().get(key(R, S, steps, precision))
    return None if e is None else (int(e["algo"]), int(e["chunk"]))


def record(R: int, S: int, steps: int, precision: int, algo: int, chunk: int, ms: float,
           save: bool = True):
    t = table()
    with _lock:
        t[key(R, S, steps, precision)] = {"algo": algo, "chunk": chunk, "ms": round(ms, 4)}
        if save:
            tmp = TABLE + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(t, f, indent=1, sort_keys=True)
            os.replace(tmp, TABLE)


def autotune(c, d, s, u, cfg, gy=None, *, D=None, seq_T=None, repeats: int = 10, tol: float = 1e-6,
             save: bool = True, candidates=CANDIDATES):
    """Time every candidate on these inputs (forward + adjoint when gy is given), keep the
    fastest whose y matches the default plan's within tol (relative L2), record it, and return
    (best SolveConfig, {candidate: ms or None if rejected})."""
    from . import api
    base = replace(cfg, algo=B.ALGO_AUTO, chunk=0)
    shape_key = api._shape_key(c, s, D, seq_T)
    ref_plan = api.get_plan(shape_key, base, tuned=False)
    y_ref = torch.empty_like(c)
    info = torch.empty(ref_plan.S, dtype=torch.int32, device=c.device)
    ref_plan.factor_solve(c, d, s, u, y_ref, info, ref_plan.workspace(c.device))
    results = {}
    best = None
    for algo, chunk in candidates:
        cand = replace(cfg, algo=algo, chunk=chunk)
        try:
            plan = api.get_plan(shape_key, cand, tuned=False)
            ws = plan.workspace(c.device)
            fac = plan.factor_buffer(c.device)
        except (B.SmnnError, torch.OutOfMemoryError):
            results[(algo, chunk)] = None
            continue
        y = torch.empty_like(c)
        plan.factor_solve(c, d, s, u, y, info, ws, factor=fac)
        err = float((y - y_ref).double().norm() / y_ref.double().norm())
        if not err <= tol or int(info.abs().sum()) != 0:
            results[(algo, chunk)] = None
            continue
        g = [torch.empty_like(t) for t in (c, d, s, u)]
        info_b = torch.empty_like(info)
        bw = dict(gy=gy, gc=g[0], gd=g[1], gs=g[2], gu=g[3], info_b=info_b) if gy is not None else {}
        graph = plan.graph(c, d, s, u, y, info, ws, factor=fac, **bw)
        graph.launch()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        for _ in range(repeats):
            graph.launch()
        ev[1].record()
        torch.cuda.synchronize()
        graph.close()
        ms = ev[0].elapsed_time(ev[1]) / repeats
        results[(algo, chunk)] = ms
        if best is None or ms < best[2]:
            best = (algo, chunk, ms)
    if best is None:
        return base, results
    R = c.shape[-1] - 1
    record(R, ref_plan.S, ref_plan.steps, cfg.precision, best[0], best[1], best[2], save=save)
    return replace(cfg, algo=best[0], chunk=best[1]), results
