"""Populate the autotuner table for the standard workloads on the current GPU.

    python -m paper_2410_06074_b300.tune_tables [--out PATH] [--workloads config2,config4,lorenz]

Each workload's inputs come from ``smnn_workloads``; the refined float-float and FP64
precisions are tuned forward + adjoint and the winners are written to the package's
``autotune_table.json`` (and to --out, if given).  ``lorenz`` tunes the first-order layer of
the coefficient-discovery step (``discovery.Discovery``: R = 1, R_init = 0, three systems per
window) on the batch/length grid of the Lorenz timing (Sec. 5.2, Table 1), refined
float-float only.
"""
from __future__ import annotations

import argparse
import json
import shutil

import numpy as np
import torch

import smnn_workloads as W

from . import autotune, binding as B
from .api import SolveConfig


def tune(name: str, precisions=(B.F32_REFINED_DF, B.F64)):
    prob = getattr(W, name)()
    out = {}
    for prec in precisions:
        dt = np.float64 if prec == B.F64 else np.float32
        c, d, s, u = (torch.from_numpy(np.ascontiguousarray(a, dt)).cuda() for a in (prob.c, prob.d, prob.s, prob.u))
        gy = torch.from_numpy(W.upstream_gradient(prob).astype(dt)).cuda()
        cfg = SolveConfig(R_init=prob.R_init, T_init=prob.T_init, precision=prec)
        best, res = autotune.autotune(c, d, s, u, cfg, gy, D=prob.D,
                                      seq_T=None if prob.seq_T is None else tuple(int(x) for x in prob.seq_T))
        out[f"{name}/P{prec}"] = {"best": [best.algo, best.chunk],
                                  "ms": {f"{a}/{k}": v for (a, k), v in res.items()}}
        print(name, prec, out[f"{name}/P{prec}"], flush=True)
        del c, d, s, u, gy
        torch.cuda.empty_cache()
    return out


LORENZ_GRID = ((512, 50), (512, 5), (512, 500), (64, 50), (4096, 50))


def tune_lorenz(precision=B.F32_REFINED_DF):
    """The discovery layer's shapes: windows of the Lorenz trajectory as the initial values,
    c = (0, 1), s = the sample spacing, d ~ N(0, 10^2) standing in for the library term."""
    tr = W.lorenz_trajectory()
    out = {}
    for Bn, T in LORENZ_GRID:
        _, xb = W.lorenz_chunks(tr, Bn, T, seed=7)
        rng = np.random.Generator(np.random.PCG64(8))
        c = np.zeros((Bn, 3, T, 2), np.float32); c[..., 1] = 1.0
        d = (10.0 * rng.standard_normal((Bn, 3, T))).astype(np.float32)
        s = np.full((Bn, T), W.LORENZ["dt"], np.float32)
        u = np.ascontiguousarray(xb[:, 0, :].reshape(Bn, 3, 1, 1), np.float32)
        gy = rng.standard_normal((Bn, 3, T, 2)).astype(np.float32)
        ct, dt_, st, ut, gt = (torch.from_numpy(a).cuda() for a in (c, d, s, u, gy))
        cfg = SolveConfig(R_init=0, T_init=1, precision=precision)
        best, res = autotune.autotune(ct, dt_, st, ut, cfg, gt, repeats=30)
        out[f"lorenz B={Bn} T={T}/P{precision}"] = {"best": [best.algo, best.chunk],
                                                   "ms": {f"{a}/{k}": v for (a, k), v in res.items()}}
        print(Bn, T, out[f"lorenz B={Bn} T={T}/P{precision}"], flush=True)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    ap.add_argument("--workloads", default="config2,config4")
    args = ap.parse_args()
    log = {}
    for name in args.workloads.split(","):
        log.update(tune_lorenz() if name == "lorenz" else tune(name))
    if args.out:
        shutil.copyfile(autotune.TABLE, args.out)
        with open(args.out + ".log.json", "w") as f:
            json.dump(log, f, indent=1)


if __name__ == "__main__":
    main()
