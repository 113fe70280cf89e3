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


def get_plan(shape_key, cfg: SolveConfig, tuned: bool = True) -> B.Plan:
    """shape_key: (R, B, D, T) for uniform batches or (R, B, D, seq_T tuple) for ragged.
    With tuned=True, ALGO_AUTO and chunk=0, the autotuner's table may pick the algorithm and
    the level-0 chunk length for this shape bucket."""
    if tuned and cfg.algo == B.ALGO_AUTO and cfg.chunk == 0:
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
                      refine_tol=cfg.refine_tol)
        _PLANS[key] = plan
    return plan


def _shape_key(c, s, D=None, seq_T=None):
    if seq_T is None:
        Bn, Dn, T, nb = c.shape
        return (nb - 1, Bn, Dn, T)
    seq_T = tuple(int(x) for x in seq_T)
    return (c.shape[-1] - 1, len(seq_T), int(D), seq_T)


def solve(c, d, s, u, cfg: SolveConfig = SolveConfig(), *, D=None, seq_T=None, factor=None,
          workspace=None):
    """Forward solve only: returns (y, info).  ``factor``: optional buffer to keep the factor."""
    plan = get_plan(_shape_key(c, s, D, seq_T), cfg)
    y = torch.empty_like(c)
    info = torch.empty(plan.S, dtype=torch.int32, device=c.device)
    ws = plan.workspace(c.device) if workspace is None else workspace
    plan.factor_solve(c, d, s, u, y, info, ws, factor=factor)
    return y, info


def gradients(c, d, s, u, y, gy, cfg: SolveConfig = SolveConfig(), *, D=None, seq_T=None,
              factor=None, workspace=None, weights: bool = False):
    """Backward only: returns (gc, gd, gs, gu, info) for dl/dy = gy; with weights=True,
    (gc, gd, gs, gu, gw, info), gw = dl/d(w_gov, w_init, w_smooth) (float64, 3 values)."""
    plan = get_plan(_shape_key(c, s, D, seq_T), cfg)
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
        plan = get_plan(_shape_key(c, s, D, seq_T), cfg)
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
