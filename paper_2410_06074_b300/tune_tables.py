"""Populate the autotuner table for the standard workloads on the current GPU.

    python -m paper_2410_06074_b300.tune_tables [--out PATH] [--workloads config2,config4]

Each workload's inputs come from ``smnn_workloads``; the refined float-float and FP64
precisions are tuned forward + adjoint and the winners are written to the package's
``autotune_table.json`` (and to --out, if given).
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default="")
    ap.add_argument("--workloads", default="config2,config4")
    args = ap.parse_args()
    log = {}
    for name in args.workloads.split(","):
        log.update(tune(name))
    if args.out:
        shutil.copyfile(autotune.TABLE, args.out)
        with open(args.out + ".log.json", "w") as f:
            json.dump(log, f, indent=1)


if __name__ == "__main__":
    main()
