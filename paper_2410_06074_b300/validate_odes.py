"""Standalone validation on the linear ODEs of App. B.1 (the cases of Table 5).

    python -m paper_2410_06074_b300.validate_odes [--precision F32_REFINED_DF] [--copies N]

Solves the six ODEs (1000 steps of 0.01, Sec. 5.1) on the GPU, in batches of equal order R,
and prints the relative MSE, sum (yhat - y)^2 / sum (y - mean y)^2, of y, y' and y'' against
the closed-form solutions, beside Table 5's printed S-MNN values.  With --copies N every case
is solved N times in one batch and the solve rate is reported as well.
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

import smnn_workloads as W

from . import binding as B
from .api import SolveConfig, solve

# Table 5 (App. B.1), S-MNN rows: relative MSE of y, y', y''
TABLE5 = {"RC": (4.8e-12, 4.8e-12, 2.2e-07), "Population": (9.4e-12, 9.4e-12, 9.6e-08),
          "Language": (2.6e-11, 2.6e-11, 7.1e-07), "Harmonic": (9.5e-08, 7.7e-08, 5.1e-07),
          "Damped": (2.1e-07, 2.3e-07, 4.0e-07), "ThirdOrder": (1.0e-09, 6.8e-10, 4.3e-09)}


def rel_mse(yhat: np.ndarray, y: np.ndarray) -> float:
    return float(np.sum((yhat - y) ** 2) / np.sum((y - y.mean()) ** 2))


def run(precision: int = B.F64, copies: int = 1, device: str = "cuda") -> list[dict]:
    dt = torch.float64 if precision == B.F64 else torch.float32
    rows = []
    for R, R_init in ((2, 0), (3, 1), (3, 2)):
        prob, cases = W.table5_batch(R, R_init)
        rep = lambda a: np.repeat(a, copies, axis=0)
        c, d, s, u = (torch.from_numpy(np.ascontiguousarray(rep(a))).to(device, dt)
                      for a in (prob.c, prob.d, prob.s, prob.u))
        cfg = SolveConfig(R_init=R_init, T_init=1, precision=precision)
        y, info = solve(c, d, s, u, cfg, D=1)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record()
        y, info = solve(c, d, s, u, cfg, D=1)
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1])
        yh = y.double().cpu().numpy()
        for b, cse in enumerate(cases):
            rows.append(dict(name=cse["name"], R=R, info=int(info[b * copies:(b + 1) * copies].abs().max()),
                             rel_mse=[rel_mse(yh[b * copies, 0, :, r], cse["exact"][r]) for r in range(3)],
                             paper=TABLE5[cse["name"]], ms=ms,
                             steps_per_s=c.shape[0] * c.shape[2] / (ms / 1e3)))
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--precision", default="F64", choices=["F64", "F32", "F32_REFINED", "F32_REFINED_DF"],
                    help="F64 by default: with h = 0.01 the highest derivative is fixed only by "
                         "smoothness rows of weight h^(2R), too ill-conditioned for an FP32 factor "
                         "in most cases (those systems report info != 0)")
    ap.add_argument("--copies", type=int, default=1)
    a = ap.parse_args()
    rows = run(getattr(B, a.precision), a.copies)
    print(f"{'ODE':12s} {'R':>2s}  {'rel MSE y':>10s} {'y1':>10s} {'y2':>10s}   {'Table 5 y':>10s} {'y1':>10s} {'y2':>10s}  info")
    for r in rows:
        m, p = r["rel_mse"], r["paper"]
        print(f"{r['name']:12s} {r['R']:2d}  {m[0]:10.2e} {m[1]:10.2e} {m[2]:10.2e}   {p[0]:10.1e} {p[1]:10.1e} {p[2]:10.1e}  {r['info']}")
    if a.copies > 1:
        for R in (2, 3):
            rr = [r for r in rows if r["R"] == R]
            print(f"R={R}: {rr[0]['steps_per_s']:.3e} time-steps/s (forward, {a.copies} copies per case)")


if __name__ == "__main__":
    main()
