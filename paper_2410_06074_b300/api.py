"""PyTorch-facing API: plan cache, a functional solve and ``SmnnSolve`` (autograd.Function).

Tensors supply device memory and the current stream; all arithmetic runs in libsmnn's
kernels (binding.py).  Shapes (one system = one (sequence, dimension) pair):
  uniform: c [B, D, T, R+1], d [B, D, T], s [B, T], u [B, D, T_init, R_init+1]
  ragged:  c [N, R+1], d [N], s [sum T_b], u [B*D, T_init, R_init+1], with ``seq_T``
"""
from __future__ import annotations

from dataclasses import dataclass, replace

import torch

from . import binding as B

_PLANS: dict = {}


@dataclass(frozen=True)
class SolveConfig:
    """Problem constants of Eq. 5 and Eq. 9, plus solver options."""
    R_init: int = 1
    T_init: int = 1
    w_gov: float = 1.0
    w_init: float = 1.0
    w_smooth: float = 1.0
    precision: int = B.F32_REFINED_DF
    algo: int = B.ALGO_AUTO
    max_refine: int = 3
    adjoint_refine: int = 3
    chunk: int = 0
    # per-system stop test of the refinement; a system whose estimated error is still above
    # it after the last sweep gets info = -1 (refinement that stagnates is never silent)
    refine_tol: float = 1e-7
    factor_budget_bytes: int = 16 << 30   # store the factor for backward if it fits
    # coupled systems (Sec. 3.1): V variables and Q governing equations per step; c then holds
    # Q*V*(R+1) values per step (equation-major), d Q, u V*(R_init+1) per initial step, and
    # y V*(R+1) (variable-major); built: V = Q = 1; V = 2, R = 1, Q <= 2; V = 3, R = 1, Q = 3;
    # V = 2, R = 2, Q = 2
    V: int = 1
    Q: int = 1
    # nonzero: one launch per level, pass and stop test even where the warp-fused launches
    # apply (the same arithmetic; for comparison)
    per_level_launches: int = 0


def get_plan(shape_key, cfg: SolveConfig, tuned: bool = True) -> B.Plan:
    """shape_key: (R, B, D, T) for uniform batches or (R, B, D, seq_T tuple) for ragged.
    With tuned=True, ALGO_AUTO and chunk=0, the autotuner's table may pick the algorithm and
    the level-0 chunk length for this shape bucket."""
    if tuned and cfg.algo == B.ALGO_AUTO and cfg.chunk == 0 and cfg.V == 1 and cfg.Q == 1:
        from . import autotune
        R, Bn, D, T = shape_key
        S = Bn * D
        steps = S * T if not isinstance(T, tuple) else D * sum(T)
        hit = autotune.lookup(R, S, steps, cfg.precision)
        if hit is not None:
            cfg = replace(cfg, algo=hit[0], chunk=hit[1])
    key = (shape_key, cfg)
    plan = _PLANS.get(key)
    if plan is None:
        R, Bn, D, T = shape_key
        ragged = isinstance(T, tuple)
        plan = B.Plan(R=R, R_init=cfg.R_init, T_init=cfg.T_init, B=Bn, D=D,
                      T=None if ragged else T, seq_T=T if ragged else None,
                      precision=cfg.precision, algo=cfg.algo, max_refine=cfg.max_refine,
                      adjoint_refine=cfg.adjoint_refine,
                      chunk=cfg.chunk, w_gov=cfg.w_gov, w_init=cfg.w_init, w_smooth=cfg.w_smooth,
                      refine_tol=cfg.refine_tol, V=cfg.V, Q=cfg.Q,
                      per_level_launches=cfg.per_level_launches)
        _PLANS[key] = plan
    return plan


def _shape_key(c, s, D=None, seq_T=None, cfg: SolveConfig | None = None):
    vq = 1 if cfg is None else cfg.V * cfg.Q   # c holds Q V (R+1) values per step
    if seq_T is None:
        Bn, Dn, T, k = c.shape
        return (k // vq - 1, Bn, Dn, T)
    seq_T = tuple(int(x) for x in seq_T)
    return (c.shape[-1] // vq - 1, len(seq_T), int(D), seq_T)


def _y_like(c, cfg: SolveConfig):
    """Solution tensor: c's step dimensions with V (R+1) = c.shape[-1] / Q values per step."""
    return c.new_empty(c.shape[:-1] + (c.shape[-1] // cfg.Q,))


def solve(c, d, s, u, cfg: SolveConfig = SolveConfig(), *, D=None, seq_T=None, factor=None,
          workspace=None):
    """Forward solve only: returns (y, info).  ``factor``: optional buffer to keep the factor."""
    plan = get_plan(_shape_key(c, s, D, seq_T, cfg), cfg)
    y = _y_like(c, cfg)
    info = torch.empty(plan.S, dtype=torch.int32, device=c.device)
    ws = plan.workspace(c.device) if workspace is None else workspace
    plan.factor_solve(c, d, s, u, y, info, ws, factor=factor)
    return y, info


def gradients(c, d, s, u, y, gy, cfg: SolveConfig = SolveConfig(), *, D=None, seq_T=None,
              factor=None, workspace=None, weights: bool = False):
    """Backward only: returns (gc, gd, gs, gu, info) for dl/dy = gy; with weights=True,
    (gc, gd, gs, gu, gw, info), gw = dl/d(w_gov, w_init, w_smooth) (float64, 3 values)."""
    plan = get_plan(_shape_key(c, s, D, seq_T, cfg), cfg)
    gc, gd, gs, gu = (torch.empty_like(t) for t in (c, d, s, u))
    info = torch.empty(plan.S, dtype=torch.int32, device=c.device)
    gw = torch.empty(3, dtype=torch.float64, device=c.device) if weights else None
    ws = plan.workspace(c.device) if workspace is None else workspace
    plan.backward(c, d, s, u, y, gy.contiguous(), gc, gd, gs, gu, info, ws, factor=factor, gw=gw)
    if weights:
        return gc, gd, gs, gu, gw, info
    return gc, gd, gs, gu, info


class SmnnSolve(torch.autograd.Function):
    """y = (A^T W A)^{-1} A^T W b (Eq. 9) with the hand-written adjoint of Eq. 14.

    The forward keeps the factor for the backward pass when it fits
    ``cfg.factor_budget_bytes``; otherwise the backward recomputes it.  ``weights``: None, or
    a tensor (w_gov, w_init, w_smooth) that replaces the config's weights and receives
    dl/dw (the weights are plan constants: each new value builds, and caches, a plan)."""

    @staticmethod
    def forward(ctx, c, d, s, u, weights, cfg: SolveConfig, D=None, seq_T=None):
        c, d, s, u = (t.contiguous() for t in (c, d, s, u))
        if weights is not None:
            wg, wi, wsm = (float(v) for v in weights.detach().double().cpu().tolist())
            cfg = replace(cfg, w_gov=wg, w_init=wi, w_smooth=wsm)
        plan = get_plan(_shape_key(c, s, D, seq_T, cfg), cfg)
        factor = plan.factor_buffer(c.device) if plan.factor_bytes <= cfg.factor_budget_bytes else None
        y, info = solve(c, d, s, u, cfg, D=D, seq_T=seq_T, factor=factor)
        ctx.save_for_backward(c, d, s, u, y)
        ctx.cfg, ctx.D, ctx.seq_T, ctx.factor = cfg, D, seq_T, factor
        ctx.w_dtype = None if weights is None else weights.dtype
        ctx.mark_non_differentiable(info)
        return y, info

    @staticmethod
    def backward(ctx, gy, _ginfo):
        c, d, s, u, y = ctx.saved_tensors
        want_w = ctx.w_dtype is not None and ctx.needs_input_grad[4]
        out = gradients(c, d, s, u, y, gy, ctx.cfg, D=ctx.D, seq_T=ctx.seq_T, factor=ctx.factor,
                        weights=want_w)
        gc, gd, gs, gu = out[:4]
        gw = out[4].to(ctx.w_dtype) if want_w else None
        return gc, gd, gs, gu, gw, None, None, None


def smnn_layer(c, d, s, u, cfg: SolveConfig = SolveConfig(), *, D=None, seq_T=None, weights=None):
    """Differentiable S-MNN solve; returns (y, info).  ``weights``: optional tensor
    (w_gov, w_init, w_smooth) to learn; overrides the config's weights."""
    return SmnnSolve.apply(c, d, s, u, weights, cfg, D, seq_T)


class HostPipeline:
    """Forward + adjoint of a uniform batch held in pinned host memory, streamed through the
    GPU in parts of whole sequences.  Part p's host->device copies, solve, backward and
    device->host copies are issued on stream p % 2 with that stream's own device buffers, so
    one part's transfers run on the copy engines while the other part's kernels run on the SMs.
    The systems are independent, so every part is an ordinary solve of its sequences (the
    level structure of a part's plan follows its size).

    run(c, d, s, u, gy, y, gc, gd, gs, gu) takes host tensors in the layouts of ``solve`` and
    ``gradients`` (uniform batch; outputs preallocated, pinned) and returns (info, info_b)
    of the forward and backward passes (device tensors, [B*D]), ordered after the copies on
    the caller's stream."""

    def __init__(self, shape_key, cfg: SolveConfig = SolveConfig(), n_parts: int = 4,
                 device="cuda", dtype=torch.float32):
        R, B, D, T = shape_key
        n_parts = max(1, min(int(n_parts), B))
        step = -(-B // n_parts)
        self.bounds = [(b, min(b + step, B)) for b in range(0, B, step)]
        self.D, self.T, self.nb = D, T, R + 1
        self.plans = {n: get_plan((R, n, D, T), cfg) for n in {b1 - b0 for b0, b1 in self.bounds}}
        big = max(self.plans)
        plan = self.plans[big]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(2)]
        self.bufs = []
        for _ in range(2):
            f = lambda *sh: torch.empty(sh, dtype=dtype, device=device)
            b = dict(c=f(big, D, T, R + 1), d=f(big, D, T), s=f(big, T),
                     u=f(big, D, cfg.T_init, cfg.R_init + 1), gy=f(big, D, T, R + 1))
            b.update(y=torch.empty_like(b["c"]), gc=torch.empty_like(b["c"]), gd=torch.empty_like(b["d"]),
                     gs=torch.empty_like(b["s"]), gu=torch.empty_like(b["u"]),
                     ws=plan.workspace(device), fac=plan.factor_buffer(device))
            self.bufs.append(b)
        self.info = torch.empty(B * D, dtype=torch.int32, device=device)
        self.info_b = torch.empty_like(self.info)

    def run(self, c, d, s, u, gy, y, gc, gd, gs, gu):
        main = torch.cuda.current_stream()
        for st in self.streams:
            st.wait_stream(main)
        for p, (b0, b1) in enumerate(self.bounds):
            st, b = self.streams[p % 2], self.bufs[p % 2]
            n = b1 - b0
            plan = self.plans[n]
            with torch.cuda.stream(st):
                for key, h in (("c", c), ("d", d), ("s", s), ("u", u), ("gy", gy)):
                    b[key][:n].copy_(h[b0:b1], non_blocking=True)
                info = self.info[b0 * self.D:b1 * self.D]
                info_b = self.info_b[b0 * self.D:b1 * self.D]
                plan.factor_solve(b["c"][:n], b["d"][:n], b["s"][:n], b["u"][:n], b["y"][:n], info,
                                  b["ws"], factor=b["fac"], stream=st)
                plan.backward(b["c"][:n], b["d"][:n], b["s"][:n], b["u"][:n], b["y"][:n], b["gy"][:n],
                              b["gc"][:n], b["gd"][:n], b["gs"][:n], b["gu"][:n], info_b, b["ws"],
                              factor=b["fac"], stream=st)
                for h, key in ((y, "y"), (gc, "gc"), (gd, "gd"), (gs, "gs"), (gu, "gu")):
                    h[b0:b1].copy_(b[key][:n], non_blocking=True)
        for st in self.streams:
            main.wait_stream(st)
        return self.info, self.info_b


class HostStream:
    """Forward + adjoint of successive uniform batches held in pinned host memory, with the
    transfers of neighbouring steps overlapped: step k's host->device copy (copy-in stream)
    runs while step k-1 computes (compute stream) and step k-2's device->host copy (copy-out
    stream) drains.  ``n_sets`` device buffer sets rotate between the steps; events order each
    set's reuse after the copy-out of the step that used it before.  With two sets, step k's
    copy-in waits for step k-2's copy-out, so a pair of steps costs copy-in + compute +
    copy-out; with three, the three engines run side by side and a step costs the largest of
    the three.

    submit(c, d, s, u, gy, y, gc, gd, gs, gu): host tensors of one step (layouts of ``solve``
    and ``gradients``; outputs preallocated, pinned).  Returns (info, info_b, done): device
    tensors that hold the step's flags once ``done`` (a CUDA event) has completed; the host
    outputs are complete then too.  wait(stream=None) orders the caller's stream after every
    submitted step."""

    def __init__(self, shape_key, cfg: SolveConfig = SolveConfig(), device="cuda",
                 dtype=torch.float32, n_sets: int = 3):
        R, B, D, T = shape_key
        if n_sets < 1:
            raise ValueError("n_sets >= 1")
        self.plan = get_plan((R, B, D, T), cfg)
        self.s_in, self.s_cmp, self.s_out = (torch.cuda.Stream(device=device) for _ in range(3))
        self.k = 0
        self.sets = []
        for _ in range(n_sets):
            f = lambda *sh: torch.empty(sh, dtype=dtype, device=device)
            b = dict(c=f(B, D, T, R + 1), d=f(B, D, T), s=f(B, T),
                     u=f(B, D, cfg.T_init, cfg.R_init + 1), gy=f(B, D, T, R + 1))
            b.update(y=torch.empty_like(b["c"]), gc=torch.empty_like(b["c"]), gd=torch.empty_like(b["d"]),
                     gs=torch.empty_like(b["s"]), gu=torch.empty_like(b["u"]),
                     info=torch.empty(B * D, dtype=torch.int32, device=device),
                     info_b=torch.empty(B * D, dtype=torch.int32, device=device),
                     freed=None)
            self.sets.append(b)
        self.ws = self.plan.workspace(device)
        self.fac = self.plan.factor_buffer(device)

    def submit(self, c, d, s, u, gy, y, gc, gd, gs, gu):
        b = self.sets[self.k % len(self.sets)]
        self.k += 1
        main = torch.cuda.current_stream()
        self.s_in.wait_stream(main)
        if b["freed"] is not None:               # the set's previous step has been copied out
            self.s_in.wait_event(b["freed"])
        with torch.cuda.stream(self.s_in):
            for key, h in (("c", c), ("d", d), ("s", s), ("u", u), ("gy", gy)):
                b[key].copy_(h, non_blocking=True)
            loaded = torch.cuda.Event()
            loaded.record(self.s_in)
        self.s_cmp.wait_event(loaded)
        p = self.plan
        p.factor_solve(b["c"], b["d"], b["s"], b["u"], b["y"], b["info"], self.ws, factor=self.fac,
                       stream=self.s_cmp)
        p.backward(b["c"], b["d"], b["s"], b["u"], b["y"], b["gy"], b["gc"], b["gd"], b["gs"], b["gu"],
                   b["info_b"], self.ws, factor=self.fac, stream=self.s_cmp)
        solved = torch.cuda.Event()
        solved.record(self.s_cmp)
        self.s_out.wait_event(solved)
        with torch.cuda.stream(self.s_out):
            for h, key in ((y, "y"), (gc, "gc"), (gd, "gd"), (gs, "gs"), (gu, "gu")):
                h.copy_(b[key], non_blocking=True)
            done = torch.cuda.Event()
            done.record(self.s_out)
        b["freed"] = done
        return b["info"], b["info_b"], done

    def wait(self, stream=None):
        st = torch.cuda.current_stream() if stream is None else stream
        for s_ in (self.s_in, self.s_cmp, self.s_out):
            st.wait_stream(s_)
