#!/usr/bin/env python
"""Benchmark of the S-MNN batched solve (Scalable Mechanistic Neural Networks, Sec. 3).

One step = one forward solve (assembly, factorisation, substitution, two FP64-residual
refinement sweeps) plus one adjoint pass (re-solve with dl/dy, refined, and the fused
parameter gradients) over the whole workload, inputs resident in HBM.  Metric: time-steps
solved per second (sum over systems of T), forward + adjoint.

Default workload: B=512 sequences x D=8 dimensions x T=1024 steps, R=2 (4,194,304
time-steps), SMNN_F32_REFINED.  Timing: W untimed warm-up steps, then K steps, each bracketed
by CUDA events on the launching stream with a 256 MiB write between steps to flush L2;
barrier + synchronize around the timed region; the max over ranks is reported.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own copy of the workload on its own GPU (systems are
independent: weak scaling, no collective on the data path).  ``--impl reference`` times the
FP64 CPU oracle on the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from smnn_workloads import config2, mse_target, upstream_gradient  # noqa: E402

WORKLOAD = "config2: B=512 D=8 T=1024 R=2, FP32 factor + float-float/FP64-residual refinement, fwd+adjoint"
METRIC = "time-steps solved/s fwd+bwd (FP32-refined, <=1e-6 vs FP64 oracle)"
UNIT = "time-steps/s"
ALGOS = {"auto": 0, "seq": 1, "cr": 2, "fused": 3}   # smnn_algo


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 GPU comparison")
    ap.add_argument("--chunk", type=int, default=0, help="level-0 chunk length (0: plan's table)")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="skip the secondary timings (config 4, config 3b, coupled batch, Lorenz training steps)")
    ap.add_argument("--algo", default="auto", choices=sorted(ALGOS),
                    help="reduction: auto (the plan's choice), seq, cr (a launch per level), "
                         "fused (a launch per solve pass)")
    ap.add_argument("--only", default="", help="comma-separated variants to time (default: all)")
    ap.add_argument("--max-refine", type=int, default=3, help="forward refinement sweeps")
    ap.add_argument("--adjoint-refine", type=int, default=3, help="adjoint refinement sweeps (at most; the stop test skips converged systems)")
    ap.add_argument("--refine-tol", type=float, default=1e-7,
                    help="per-system refinement stop test, the library's default (0: run every "
                         "sweep with no convergence check)")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed

def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        backend = os.environ.get("SMNN_DIST_BACKEND") or ("nccl" if torch.cuda.is_available() else "gloo")
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0])); mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


# ALU peaks.  FP32: 148 SMs x 128 FP32 lanes x 2.032 GHz (maximum SM clock; the clock
# sampled under this benchmark's load) = 38.5e12 FP32 instructions/s, an FMA counted as one
# instruction (a DFMA-chain and FFMA-chain microbenchmark on this B300 measured 34.4e12
# FFMA/s and 0.562e12 DFMA/s).  FP64: ~2 DFMA/clock/SM -> 0.60e12 DP instructions/s.
FP32_PEAK_TOPS = 148 * 128 * 2.032e9 / 1e12
FP64_PEAK_TOPS = 148 * 2 * 2.032e9 / 1e12


# dram__bytes_read.sum + dram__bytes_write.sum of one launch on this workload, from the ncu
# capture summarised in the named file (to be re-taken whenever the kernel changes)
NCU_TRAFFIC = {"k_elim0_res": (452.491776e6 + 44.448512e6, "profiles/k_elim0_res_config2.md"),
               "k_backsub0": (428.012544e6 + 83.223040e6, "profiles/k_backsub0_config2.md")}


def residual_ops(NB: int, explicit_rhs: bool, df: bool) -> float:
    """Arithmetic instructions per time-step of the refinement residual r = rhs - M x
    (governing row, 2(R+1) smoothness rows, accumulation), counted from the formulas in
    csrc/smnn.cu.  Float-float costs per operation (smnn_num.cuh): ff*float 6, ff*ff 7,
    ff+float 10, ff+ff 11 FP32 instructions; in FP64 every operation is one instruction."""
    n = NB
    mf, mm, af, aa = (6, 7, 10, 11) if df else (1, 1, 1, 1)
    half = 2 if df else 1                                # v/2: two exact scalings
    gov = n * (mf + aa) + (mm + n * (mf + af + aa) if explicit_rhs else (af + mm) + n * (mf + aa))
    # smoothness pair in the P F P form: powers s^r, x~ = P x_t and x^ = P x_{t+1}; f, h
    # (F x - ..., n(n-1)/2 additions each plus n subtractions); F^T f, F^T h; D h - F^T f and
    # f - D F^T h; times P and w_s^2.  v/k! costs `half` for k = 2 and a product for k = 3.
    scal = 2 * ((n - 2) * half + max(n - 3, 0) * mm)     # the 1/k! factors of two vectors
    pair = (max(n - 2, 0) * mf + 2 * (mf + (n - 2) * mm)
            + 2 * (n * (n - 1) // 2 * aa) + 2 * n * aa + scal
            + 2 * (n * (n - 1) // 2 * aa) + scal
            + 2 * n * aa + 2 * (mf + (n - 2) * mm) + 2 * n * mm)
    return float(gov + pair + n * aa + n)


def replay_ops(NB: int) -> float:
    """FP32 instructions per time-step of one level-0 replay of the stored factor: z = L^-1 r,
    the fill contribution H^T z, E_t from s_t, X = L^-1 E^T and r_{t+1} -= X^T z."""
    n = NB
    return float(n * n + n * n + (2 * n - 2 + 2 * n * n) + n * n * (n + 1) // 2 + n * n)


def algorithmic_units(name: str, NB: int, D: int, df: bool):
    """Per-step algorithmic work of one launch of a kernel: (bound, amount, unit)."""
    if name == "k_elim0_res":
        if df:
            return "alu", residual_ops(NB, False, True) + replay_ops(NB), "FP32 instr"
        return "alu", residual_ops(NB, False, False), "FP64 instr"
    # memory sweeps: the method's forward bytes per time-step (c, d, s read; y written)
    return "hbm", 8.0 * NB + 4.0 + 4.0 / D, "B"


# ----------------------------------------------------------------------------- our arm

class Variant:
    """One precision mode of the library on the benchmark workload: its plan and buffers."""

    def __init__(self, pk, prob, precision, dev, inputs, factor=True, chunk=0, max_refine=3,
                 adjoint_refine=2, refine_tol=0.0, algo=0):
        import torch
        self.precision = precision
        cfg = pk.SolveConfig(R_init=prob.R_init, T_init=prob.T_init, precision=precision,
                             max_refine=max_refine, adjoint_refine=adjoint_refine, chunk=chunk,
                             algo=algo,
                             refine_tol=refine_tol if precision != pk.F64 else 0.0)
        self.cfg = cfg
        self.plan = pk.get_plan((prob.R, prob.B, prob.D, prob.T), cfg)
        dt = self.plan.dtype
        self.c, self.d, self.s, self.u = (t.to(dt) for t in inputs)
        self.y = torch.empty_like(self.c)
        self.info = torch.empty(self.plan.S, dtype=torch.int32, device=dev)
        self.info_b = torch.empty_like(self.info)
        self.work = self.plan.workspace(dev)
        self.factor = self.plan.factor_buffer(dev) if factor else None
        self.gc, self.gd, self.gs, self.gu = (torch.empty_like(t) for t in (self.c, self.d, self.s, self.u))
        self.gy = None

    def forward(self, c=None, d=None, s=None, u=None):
        self.plan.factor_solve(c if c is not None else self.c, d if d is not None else self.d,
                               s if s is not None else self.s, u if u is not None else self.u,
                               self.y, self.info, self.work, factor=self.factor)

    def backward(self, c=None, d=None, s=None, u=None, gy=None):
        self.plan.backward(c if c is not None else self.c, d if d is not None else self.d,
                           s if s is not None else self.s, u if u is not None else self.u,
                           self.y, gy if gy is not None else self.gy, self.gc, self.gd, self.gs,
                           self.gu, self.info_b, self.work, factor=self.factor)

    def step(self):
        self.forward()
        self.backward()

    def graph(self):
        """The same step recorded once by smnn_graph_create on this variant's buffers."""
        return self.plan.graph(self.c, self.d, self.s, self.u, self.y, self.info, self.work,
                               factor=self.factor, gy=self.gy, gc=self.gc, gd=self.gd, gs=self.gs,
                               gu=self.gu, info_b=self.info_b)


def timed(fn, steps, stream, flush):
    """Sum of per-step CUDA-event durations; a 256 MiB write flushes L2 between steps."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for k in range(steps):
        flush.fill_(k & 0xFF)
        ev[k][0].record(stream)
        fn()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in ev)


def run_ours(args, ws, rank, local):
    import torch
    import paper_2410_06074_b300 as pk
    from paper_2410_06074_b300 import binding as Bd

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    prob = config2()
    p32 = prob.cast(np.float32)
    NB, D = prob.R + 1, prob.D
    steps_per_pass = prob.steps
    inputs = [torch.from_numpy(a).to(dev) for a in (p32.c, p32.d, p32.s, p32.u)]
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    only = set(x for x in args.only.split(",") if x)
    kw = dict(chunk=args.chunk, max_refine=args.max_refine, adjoint_refine=args.adjoint_refine,
              refine_tol=args.refine_tol, algo=ALGOS[args.algo])
    variants = {"F32_REFINED_DF": Variant(pk, prob, pk.F32_REFINED_DF, dev, inputs, **kw)}
    if not only or "F32_REFINED" in only:
        variants["F32_REFINED"] = Variant(pk, prob, pk.F32_REFINED, dev, inputs, **kw)
    # dl/dy of config 2's loss, mean over S*T of (y^(0) - tau)^2, at this workload's y
    v0 = variants["F32_REFINED_DF"]
    v0.forward()
    tau = torch.from_numpy(mse_target(prob).astype(np.float32)).to(dev)
    gy = torch.zeros_like(v0.y)
    gy[..., 0] = 2.0 * (v0.y[..., 0] - tau) / float(steps_per_pass)
    for v in variants.values():
        v.gy = gy
    if not args.no_fp64 and (not only or "F64" in only):
        v64 = Variant(pk, prob, pk.F64, dev, inputs, chunk=args.chunk, algo=ALGOS[args.algo])
        v64.gy = gy.double()
        variants["F64"] = v64
    torch.cuda.synchronize()

    results = {}
    for name, v in variants.items():
        for _ in range(args.warmup):
            v.step()
        torch.cuda.synchronize()
        barrier(ws)
        # the step as a training loop runs it: recorded once by smnn_graph_create on the
        # variant's buffers, replayed by smnn_graph_launch (the same kernels as the eager
        # calls, bit for bit); the eager calls are timed beside it
        gph = v.graph()
        for _ in range(2):
            gph.launch()
        torch.cuda.synchronize()
        barrier(ws)
        with ClockSampler(local) as clk:
            n0 = Bd.launch_count()
            graph_ms = timed(gph.launch, args.steps, stream, flush)
            launches = Bd.launch_count() - n0
            ms = timed(v.step, args.steps, stream, flush)
        gph.close()
        # per-kernel event timing on a further run of the same steps (eager calls), so that
        # the events around every launch do not lengthen the timed runs
        Bd.profile_enable(True)
        ms_prof = timed(v.step, args.steps, stream, flush)
        Bd.profile_enable(False)
        prof = Bd.profile_read()
        ms = max_over_ranks(ms, ws) / args.steps
        graph_ms = max_over_ranks(graph_ms, ws) / args.steps
        fwd_ms = max_over_ranks(timed(v.forward, args.steps, stream, flush), ws) / args.steps
        assert int((v.info != 0).sum()) == 0 and int((v.info_b != 0).sum()) == 0, f"{name}: solver failures"
        results[name] = {"ms_per_step": graph_ms, "value": ws * steps_per_pass / (graph_ms / 1e3),
                         "eager_ms_per_step": ms, "eager_value": ws * steps_per_pass / (ms / 1e3),
                         "fwd_ms_per_step": fwd_ms, "fwd_value": ws * steps_per_pass / (fwd_ms / 1e3),
                         "gpu_launches": launches, "clocks": clk.summary(), "profile": prof,
                         "ms_per_step_profiled": max_over_ranks(ms_prof, ws) / args.steps}
    return prob, p32, variants, results, stream, flush, dev


def other_configs(args, ws, stream, flush):
    """Forward + adjoint time of the other large workloads (library defaults, saved factor,
    L2 flushed between steps): config 4 (4096 ragged systems, T in [32, 65536], R = 2),
    config 3b (4 systems of 2^20 steps, R = 3) and two coupled batches (4096 systems of 1024
    steps with V = 2 variables, R = 1, Q = 2 equations per step, and with V = 3, R = 1, Q = 3
    and a diagonally dominant highest-derivative block) on SMNN_F32_REFINED_DF.
    Secondary lines: their accuracy against the oracle is covered by the parity tests."""
    import torch
    import paper_2410_06074_b300 as pk
    from smnn_workloads import config3b, config4, random_coupled_problem
    out = {}
    coupled = lambda: random_coupled_problem(0, 512, 8, 1024, R=1, V=2, Q=2)   # noqa: E731
    coupled3 = lambda: random_coupled_problem(0, 512, 8, 1024, R=1, V=3, Q=3, lead_cross=0.25)  # noqa: E731
    for name, make in (("config4", config4), ("config3b", config3b), ("coupled_V2_Q2", coupled),
                       ("coupled_V3_Q3", coupled3)):
        prob = make().cast(np.float32)
        seq_T = None if prob.seq_T is None else tuple(int(x) for x in prob.seq_T)
        dev = torch.device("cuda", torch.cuda.current_device())
        c, d, s, u = (torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (prob.c, prob.d, prob.s, prob.u))
        nb = prob.V * (prob.R + 1)
        gy = torch.from_numpy(np.ascontiguousarray(upstream_gradient(prob)[..., :nb]).astype(np.float32)).to(dev)
        cfg = pk.SolveConfig(R_init=prob.R_init, T_init=prob.T_init, precision=pk.F32_REFINED_DF,
                             V=prob.V, Q=prob.Q)
        plan = pk.get_plan(pk.api._shape_key(c, s, prob.D, seq_T, cfg), cfg)
        wsb, fac = plan.workspace(dev), plan.factor_buffer(dev)
        y = pk.api._y_like(c, cfg)
        info, info_b = (torch.empty(plan.S, dtype=torch.int32, device=dev) for _ in range(2))
        g = [torch.empty_like(t) for t in (c, d, s, u)]

        def step():
            plan.factor_solve(c, d, s, u, y, info, wsb, factor=fac)
            plan.backward(c, d, s, u, y, gy, *g, info_b, wsb, factor=fac)
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        barrier(ws)
        ms = max_over_ranks(timed(step, max(3, args.steps // 4), stream, flush), ws) / max(3, args.steps // 4)
        bad = int((info != 0).sum()) + int((info_b != 0).sum())
        st = plan.stats()
        out[name] = {"workload": prob.name, "time_steps_per_pass": prob.steps, "ms_per_step": ms,
                     "value": ws * prob.steps / (ms / 1e3), "unit": UNIT, "flagged_systems": bad,
                     "levels": int(st.num_levels), "chunks": [int(x) for x in st.chunk][:int(st.num_levels)]}
        del c, d, s, u, gy, wsb, fac, y, g
        torch.cuda.empty_cache()
    return out


def e2e_and_roofline(prob, v, res, ws, args, stream, flush):
    """End-to-end rate through the public API with host buffers, and the roofline of the
    dominant kernel of variant v."""
    import torch
    NB, D, steps_per_pass = prob.R + 1, prob.D, prob.steps
    import paper_2410_06074_b300 as pk
    host_in = [t.cpu().pin_memory() for t in (v.c, v.d, v.s, v.u, v.gy)]
    host_out = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (v.y, v.gc, v.gd, v.gs, v.gu)]
    h2d = sum(t.numel() * t.element_size() for t in host_in)
    d2h = sum(t.numel() * t.element_size() for t in host_out)
    # the public API's streaming host path: each step copies its inputs in and its results out;
    # step k+1's copy-in and step k-1's copy-out run on their own streams while step k
    # computes (HostStream, three rotating device buffer sets).  Every step's working set
    # (inputs 120 MB, factor 300 MB, outputs) exceeds L2, so no flush is added between steps.
    pipe = pk.HostStream((prob.R, prob.B, prob.D, prob.T), v.cfg, device=v.c.device, dtype=v.c.dtype)

    def run_steps(n):
        for _ in range(n):
            pipe.submit(*host_in, *host_out)
        pipe.wait(stream)
    run_steps(max(args.warmup, 2))
    torch.cuda.synchronize()
    barrier(ws)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    run_steps(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), ws) / args.steps

    peaks, peak_src = measured_peaks()
    prof = res["profile"]
    name, (nl, tms) = max(prof.items(), key=lambda kv: kv[1][1])
    per_launch_ms = tms / max(nl, 1)
    df = v.precision == 3
    bound, per_step, unit = algorithmic_units(name, NB, D, df)
    if bound == "alu":
        peak = FP32_PEAK_TOPS if df else FP64_PEAK_TOPS
        achieved = per_step * steps_per_pass / (per_launch_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak,
                "unit": "T FP32 instr/s" if df else "T FP64 instr/s", "frac": achieved / peak,
                "peak_source": "derived: 148 SMs x 128 FP32 lanes x 2.032 GHz" if df else
                               "derived: 148 SMs x 2 FP64 lanes x 2.032 GHz"}
    else:
        achieved = per_step * steps_per_pass / (per_launch_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)"}
    tr = NCU_TRAFFIC.get(name)
    roof.update({"traffic": tr[0] if tr else None, "traffic_unit": "B per launch",
                 "traffic_source": tr[1] if tr else None,
                 "per_step": per_step, "per_step_unit": unit,
                 "launch_ms": per_launch_ms,
                 "share": tms / max(sum(x[1] for x in prof.values()), 1e-9)})
    step_bytes = (16 * NB + 8 + 8.0 / D + 8 * NB + 4 + 4.0 / D)
    whole = {"algorithmic_bytes_per_step": step_bytes,
             "algorithmic_GBps": step_bytes * steps_per_pass / (res["ms_per_step"] / 1e3) / 1e9}
    whole["frac_of_hbm"] = whole["algorithmic_GBps"] / peaks["hbm_gbs"]
    e2e = {"value": ws * steps_per_pass / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "path": "HostStream: per step H2D of c, d, s, u, dl/dy and D2H of y and the four "
                   "gradients (pinned host buffers), overlapped with the neighbouring steps' compute"}
    return e2e, roof, whole


# ----------------------------------------------------------------------------- oracle arm

def oracle_timed(prob32, gy, systems, reps_target_s=10.0, cap_s=30.0):
    """Oracle fwd+grad on the first `systems` systems of the FP32-rounded workload, repeated
    until ~reps_target_s of wall time; returns (steps/s, cores, sample description, results)."""
    import oracle as O
    p64 = prob32.as_f64()
    nseq = systems // prob32.D
    sl = slice(0, nseq)
    args = (O.Params(p64.R, p64.R_init, p64.T_init, p64.w_gov, p64.w_init, p64.w_smooth),
            p64.c[sl], p64.d[sl], p64.s[sl], p64.u[sl], gy[sl])
    cores = O.max_threads()
    t0 = time.time()
    res = O.gradient(*args)
    reps, el = 1, time.time() - t0
    while el < reps_target_s and el * (reps + 1) / reps < cap_s:
        O.gradient(*args)
        reps += 1
        el = time.time() - t0
    steps = nseq * prob32.D * prob32.T * reps
    return steps / el, cores, f"{nseq * prob32.D} systems x T={prob32.T}, fwd+grad, {reps} reps, {el:.1f} s", res


def run_reference(args, ws, rank):
    if rank != 0:
        return None
    prob = config2()
    p32 = prob.cast(np.float32)
    from smnn_workloads import upstream_gradient
    gy = np.zeros_like(p32.c, dtype=np.float64)
    gy[..., 0] = upstream_gradient(prob)[..., 0] / prob.steps
    sample_sys = prob.S          # the whole workload per step (~0.3-0.6 s on 8-16 cores)
    import oracle as O
    p64 = p32.as_f64()
    nseq = sample_sys // prob.D
    a = (O.Params(p64.R, p64.R_init, p64.T_init), p64.c[:nseq], p64.d[:nseq], p64.s[:nseq],
         p64.u[:nseq], gy[:nseq])
    for _ in range(args.warmup):
        O.gradient(*a)
    t0 = time.time()
    for _ in range(args.steps):
        O.gradient(*a)
    el = time.time() - t0
    steps = nseq * prob.D * prob.T * args.steps
    v = steps / el
    return {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded config-2 generators)",
            "config": {"workload": WORKLOAD, "B": prob.B, "D": prob.D, "T": prob.T, "R": prob.R,
                       "sample_per_step": f"{nseq * prob.D} of {prob.S} systems"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.max_threads(), "kind": "oracle",
                             "sample": f"{nseq * prob.D} systems x T={prob.T} per step, fwd+grad"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def accuracy(v, oracle_res, S):
    yo, gco, gdo, gso, guo, _ = oracle_res
    def rel(t, ref):
        a = t.double().cpu().numpy().reshape(ref.shape)
        return float(np.linalg.norm((a - ref).ravel()) / np.linalg.norm(ref.ravel()))
    ys = v.y.double().cpu().numpy()
    per = np.linalg.norm((ys - yo).reshape(S, -1), axis=1) / np.linalg.norm(yo.reshape(S, -1), axis=1)
    return {"y_max_rel_l2_per_system": float(per.max()), "gc": rel(v.gc, gco), "gd": rel(v.gd, gdo),
            "gs": rel(v.gs, gso), "gu": rel(v.gu, guo)}


# Sec. 5.2, Table 1: S-MNN time per optimisation step of the Lorenz discovery run on an
# H100 80 GB, by (batch size, sequence length); context only (other hardware, and a whole
# training script around the solver)
LORENZ_PAPER_MS = {(512, 50): 7.4, (512, 5): 5.5, (512, 500): 32.2, (64, 50): 5.5, (4096, 50): 18.3}


def lorenz_training_steps(args, ws, stream):
    """Time per optimisation step of coefficient discovery on the Lorenz trajectory (the
    Sec. 5.2 setting, synthetic RK4 data): B random windows of T samples drawn on the device,
    degree-2 library, first-order layer solve (R = 1, FP32 + float-float refinement), MSE
    loss, adjoint and Adam, the whole step captured in one CUDA graph and replayed.  The
    eager (uncaptured) step is timed beside it.  No L2 flush: a training loop keeps its
    trajectory (10,000 x 3 samples) and parameters resident."""
    import torch
    import paper_2410_06074_b300 as pk
    from paper_2410_06074_b300 import binding as Bd
    from paper_2410_06074_b300.discovery import Discovery, GraphedTrainStep, library_terms
    from smnn_workloads import LORENZ, lorenz_trajectory
    dev = torch.device("cuda", torch.cuda.current_device())
    tr = lorenz_trajectory()
    traj = torch.from_numpy(tr).to(dev)
    terms = library_terms(3, 2)
    scale = Discovery.feature_scale(traj.cpu(), terms)
    cfg = pk.SolveConfig(R_init=0, T_init=1, precision=pk.F32_REFINED_DF)
    reps = max(50, 4 * args.steps)
    out = {}
    for (Bn, T), paper_ms in LORENZ_PAPER_MS.items():
        row = {"batch": Bn, "T": T, "paper_ms_h100": paper_ms}
        for graphed in (True, False):
            torch.manual_seed(0)
            model = Discovery(3, 2, LORENZ["dt"], scale=scale, cfg=cfg, device=dev)
            n0 = Bd.launch_count()
            st = GraphedTrainStep(model, traj, Bn, T, lr=1e-2, warmup=max(args.warmup, 3),
                                  graphed=graphed)
            per_step = (Bd.launch_count() - n0) // (max(args.warmup, 3) + (1 if graphed else 0))
            for _ in range(3):
                st.step()
            torch.cuda.synchronize()
            barrier(ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                st.step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = max_over_ranks(e0.elapsed_time(e1), ws) / reps
            key = "graph" if graphed else "eager"
            row[key + "_ms_per_step"] = ms
            if graphed:
                row["solver_launches_per_step"] = per_step
                row["flagged_solves_last_step"] = int(st.bad)
                row["loss_after"] = float(st.loss)
                row["sequence_steps_per_s"] = ws * Bn * T / (ms / 1e3)
            del st, model
        out[f"B{Bn}_T{T}"] = row
    return out


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        out = run_reference(args, ws, rank)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    prob, p32, variants, results, stream, flush, dev = run_ours(args, ws, rank, local)
    # accuracy of every variant against the FP64 oracle on the full workload (rank 0)
    cpu = None
    acc = {}
    if rank == 0 and not args.no_cpu_baseline:
        gy_np = variants["F32_REFINED_DF"].gy.double().cpu().numpy()
        v_cpu, cores, sample, ores = oracle_timed(p32, gy_np, systems=p32.S)
        cpu = {"value": v_cpu, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
        for name, v in variants.items():
            acc[name] = accuracy(v, ores, p32.S)
    ok = [n for n in ("F32_REFINED_DF", "F32_REFINED")
          if n in acc and max(acc[n].values()) <= 1e-6]
    pool = ok if ok else [n for n in ("F32_REFINED_DF", "F32_REFINED") if n in results]
    head = max(pool, key=lambda n: results[n]["value"])
    r = results[head]
    e2e, roof, whole = e2e_and_roofline(prob, variants[head], r, ws, args, stream, flush)
    others = None if args.no_other_configs else other_configs(args, ws, stream, flush)
    lorenz = None if args.no_other_configs else lorenz_training_steps(args, ws, stream)
    prec_txt = {"F32_REFINED_DF": "FP32 factor + float-float residual refinement",
                "F32_REFINED": "FP32 factor + FP64 residual refinement"}[head]
    out = {
        "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (float-float residual)" if head == "F32_REFINED_DF" else "f32 (f64 residual)",
        "data": "synthetic (seeded config-2 generators: c~N(0,1), c2=1+|N|, d~N(0,1), s~U[0.01,0.1], u~N(0,1))",
        "config": {"workload": WORKLOAD, "B": prob.B, "D": prob.D, "T": prob.T, "R": prob.R,
                   "time_steps_per_pass": prob.steps, "precision": "SMNN_" + head,
                   "solver": prec_txt, "max_refine": args.max_refine,
                   "adjoint_refine": args.adjoint_refine, "refine_tol": args.refine_tol,
                   "algo": args.algo,
                   "factor": "stored in forward, reused in backward",
                   "launch": "one CUDA graph per step (smnn_graph_create once, smnn_graph_launch "
                             "per step); the eager per-kernel calls are in eager_ms_per_step",
                   "l2": "256 MiB write between timed steps (outside the events)",
                   "parallelism": f"replicas x{ws} (independent systems, no collective)"},
        "fwd_only": {"value": r["fwd_value"], "ms_per_step": r["fwd_ms_per_step"]},
        "eager": {"value": r["eager_value"], "ms_per_step": r["eager_ms_per_step"]},
        "e2e": e2e,
        "gpu_launches": r["gpu_launches"],
        "clocks": r["clocks"],
        "roofline": roof,
        "whole_step_hbm": whole,
        "variants": {n: {k: x[k] for k in ("value", "ms_per_step", "eager_value", "eager_ms_per_step",
                                           "fwd_value", "fwd_ms_per_step", "ms_per_step_profiled")}
                     for n, x in results.items()},
        "kernels": {k: {"launches": x[0], "total_ms": x[1]} for k, x in sorted(r["profile"].items())},
        "kernels_note": "per-launch CUDA events on the launching stream over a further timed run "
                        "of the same steps as eager calls (ms_per_step_profiled); the timed runs "
                        "have no events between launches",
        "accuracy_vs_oracle": acc,
    }
    if others is not None:
        out["other_configs"] = others
    if lorenz is not None:
        out["lorenz_training_step"] = lorenz
    if cpu is not None:
        out["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
