"""smnn_factor_solve_noalloc: the forward solve for callers that may not allocate device
memory (an allocator that owns every device byte, a latency-critical loop where cudaMalloc's
synchronisation or failure is not acceptable, or code that cannot keep a plan alive).

It is called here through the C ABI and compared with the planned entry point
(smnn_plan_create + smnn_factor_solve with a caller-allocated workspace) on the same inputs,
several calls in a row: both run the same kernels in the same order, so the outputs must be
identical bit for bit.  This file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from smnn_workloads import random_problem

pytestmark = pytest.mark.gpu



def _desc(B, prob, precision, seq=None, chunk=0):
    return B.Desc(prob.R, prob.R_init, prob.T_init, precision, B.ALGO_AUTO, 3, chunk, 3,
                  prob.w_gov, prob.w_init, prob.w_smooth, 0.0, prob.B, prob.D, int(prob.T or 0),
                  None if seq is None else ctypes.cast(seq, ctypes.POINTER(ctypes.c_int64)))


def _both(B, prob, precision, chunk=0):
    """The no-allocation call and the planned call on the same inputs: (y, info) of each."""
    import torch
    dt = torch.float64 if precision == B.F64 else torch.float32
    c, d, s, u = (torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dt)
                  for a in (prob.c, prob.d, prob.s, prob.u))
    seq_T = None if prob.seq_T is None else tuple(int(x) for x in prob.seq_T)
    plan = B.Plan(R=prob.R, R_init=prob.R_init, T_init=prob.T_init, B=prob.B, D=prob.D,
                  T=None if seq_T else prob.T, seq_T=seq_T, precision=precision,
                  max_refine=3, adjoint_refine=3, chunk=chunk)
    y_ref = torch.empty_like(c)
    info_ref = torch.empty(plan.S, dtype=torch.int32, device="cuda")
    plan.factor_solve(c, d, s, u, y_ref, info_ref, plan.workspace())

    y = torch.full_like(c, float("nan"))
    info = torch.full((plan.S,), 7, dtype=torch.int32, device="cuda")
    seq = None if seq_T is None else (ctypes.c_int64 * len(seq_T))(*seq_T)
    desc = _desc(B, prob, precision, seq, chunk)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = B.lib.smnn_factor_solve_noalloc(ctypes.byref(desc), *(ctypes.c_void_p(t.data_ptr())
                                         for t in (c, d, s, u, y, info)), st)
    assert rc == B.SMNN_OK, B.status_string(rc)
    torch.cuda.synchronize()
    return y.cpu(), info.cpu(), y_ref.cpu(), info_ref.cpu()


def test_noalloc_matches_planned_solve_on_two_calls_in_a_row():
    """Same descriptor, same kernels, same inputs: the outputs must agree bit for bit (a slip in
    binding the tables into the shared scratch, or stale scratch from the previous call, cannot
    hide inside a tolerance).  Two uniform calls in a row, then a ragged batch and the FP64
    path, which lay different tables over the same scratch, and a plan whose refined solve runs
    one warp per system."""
    from paper_2410_06074_b300 import binding as B
    from smnn_workloads import ragged_problem

    cases = [(random_problem(31, 3, 2, 700, 2).cast(np.float32), B.F32_REFINED_DF, 0),
             (random_problem(32, 3, 2, 1500, 2).cast(np.float32), B.F32_REFINED_DF, 0),
             (ragged_problem([1, 5, 64, 65, 1000, 3001], D=2, seed=34).cast(np.float32), B.F32_REFINED_DF, 0),
             (random_problem(35, 2, 3, 900, 2), B.F64, 0),
             (random_problem(36, 4, 2, 1024, 2).cast(np.float32), B.F32_REFINED_DF, 32)]   # one warp per system
    for prob, prec, chunk in cases:
        y, info, y_ref, info_ref = _both(B, prob, prec, chunk)
        assert (info_ref.numpy() == 0).all()
        assert np.array_equal(info.numpy(), info_ref.numpy())
        assert np.array_equal(y.numpy(), y_ref.numpy())


def test_noalloc_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2410_06074_b300 import binding as B

    prob = random_problem(33, 1, 1, 4, 2).cast(np.float32)
    big = _desc(B, prob, B.F32_REFINED_DF)
    big.num_seq, big.dims_per_seq, big.T = 512, 8, 1024     # ~1 GB of workspace
    t = torch.zeros(16, device="cuda")
    info = torch.zeros(4, dtype=torch.int32, device="cuda")
    n0 = B.launch_count()
    rc = B.lib.smnn_factor_solve_noalloc(ctypes.byref(big), *(ctypes.c_void_p(x.data_ptr())
                                         for x in (t, t, t, t, t, info)), None)
    assert rc == B.SMNN_ERR_TOO_LARGE
    assert "static scratch" in B.status_string(rc)
    assert B.launch_count() == n0
