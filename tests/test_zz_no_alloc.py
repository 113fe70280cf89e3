"""smnn_factor_solve_noalloc: the forward solve for callers that may not allocate device
memory (an allocator that owns every device byte, a latency-critical loop where cudaMalloc's
synchronisation or failure is not acceptable, or code that cannot keep a plan alive).

It is called here through the C ABI and compared with the planned entry point
(smnn_plan_create + smnn_factor_solve with a caller-allocated workspace) on the same inputs,
twice in a row, within the refined tolerance the other GPU tests use.  This file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from smnn_workloads import random_problem

pytestmark = pytest.mark.gpu

TOL_REF = 1e-6


def _desc(B, prob, precision):
    return B.Desc(prob.R, prob.R_init, prob.T_init, precision, B.ALGO_AUTO, 3, 0, 3,
                  prob.w_gov, prob.w_init, prob.w_smooth, 0.0, prob.B, prob.D, prob.T, None)


def test_noalloc_matches_planned_solve_on_two_calls_in_a_row():
    import torch
    from paper_2410_06074_b300 import binding as B

    for seed, T in ((31, 700), (32, 1500)):            # two calls, different shapes and data
        prob = random_problem(seed, 3, 2, T, 2).cast(np.float32)
        c, d, s, u = (torch.from_numpy(a).cuda() for a in (prob.c, prob.d, prob.s, prob.u))
        plan = B.Plan(R=2, R_init=1, T_init=1, B=3, D=2, T=T, precision=B.F32_REFINED_DF,
                      max_refine=3, adjoint_refine=3)
        y_ref = torch.empty_like(c)
        info_ref = torch.empty(plan.S, dtype=torch.int32, device="cuda")
        plan.factor_solve(c, d, s, u, y_ref, info_ref, plan.workspace())

        y = torch.full_like(c, float("nan"))
        info = torch.full((plan.S,), 7, dtype=torch.int32, device="cuda")
        desc = _desc(B, prob, B.F32_REFINED_DF)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        rc = B.lib.smnn_factor_solve_noalloc(ctypes.byref(desc), *(ctypes.c_void_p(t.data_ptr())
                                             for t in (c, d, s, u, y, info)), st)
        assert rc == B.SMNN_OK, B.status_string(rc)
        torch.cuda.synchronize()
        assert (info.cpu().numpy() == 0).all() and (info_ref.cpu().numpy() == 0).all()
        a, b = y.double().cpu().numpy(), y_ref.double().cpu().numpy()
        err = np.linalg.norm((a - b).reshape(plan.S, -1), axis=1) / np.linalg.norm(b.reshape(plan.S, -1), axis=1)
        assert err.max() <= TOL_REF, err.max()


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
