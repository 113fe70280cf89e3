"""CUDA path vs the FP64 oracle, element by element, on seeded inputs (GPU required).

Tolerances (relative L2 per system unless stated):
  SMNN_F64             1e-9   (kappa(M) ~ 1e6 on the R=2 generators; FP64 rounding ~ kappa*1e-16)
  SMNN_F32_REFINED     1e-6   (the stated refined target; two FP64-residual sweeps)
  SMNN_F32 unrefined   5e-3   (FP32 factor alone: ~kappa * 2^-24 in practice ~1e-3)
"""
import numpy as np
import pytest

import oracle as O
from smnn_workloads import Problem, config1, ragged_problem, random_problem, upstream_gradient
from _helpers import (assert_grads, gpu_grad, gpu_solve, oracle_grad, oracle_solve, per_system,
                      rel_err, rel_err_per_system, rounded)

pytestmark = pytest.mark.gpu

TOL_F64, TOL_REF, TOL_F32 = 1e-9, 1e-6, 5e-3


def P():
    import paper_2410_06074_b300 as pk
    return pk


# ----------------------------------------------------------------------------- forward

@pytest.mark.parametrize("algo,chunk", [("SEQ", 0), ("CR", 0), ("CR", 4), ("CR", 7)])
def test_config1_fp64_matches_dense_oracle(algo, chunk):
    pk = P()
    prob = config1()
    y, info = gpu_solve(prob, pk.F64, algo=getattr(pk, "ALGO_" + algo), chunk=chunk)
    yo, info_o = O.solve(O.Params(2, 1, 1), prob.c, prob.d, prob.s, prob.u, mode="dense")
    assert (info == 0).all() and (info_o == 0).all()
    for g, r in zip(per_system(y, prob), per_system(yo, prob)):
        assert np.abs(g - r).max() <= TOL_F64 * np.abs(r).max()


REFINED = ["F32_REFINED", "F32_REFINED_DF"]


@pytest.mark.parametrize("prec", REFINED)
@pytest.mark.parametrize("T,algo,chunk", [(1000, "CR", 0), (1000, "CR", 8), (4099, "CR", 64),
                                          (4099, "SEQ", 0), (333, "CR", 2), (64, "CR", 0)])
def test_refined_fp32_forward(T, algo, chunk, prec):
    pk = P()
    prob = random_problem(7, 3, 2, T, 2)
    y, info = gpu_solve(prob, getattr(pk, prec), algo=getattr(pk, "ALGO_" + algo), chunk=chunk)
    yo, _ = oracle_solve(rounded(prob, pk.F32_REFINED))
    assert (info == 0).all()
    assert rel_err_per_system(y, yo, prob).max() <= TOL_REF


@pytest.mark.parametrize("prec", ["F64", "F32", "F32_REFINED", "F32_REFINED_DF"])
@pytest.mark.parametrize("seq_T,D,chunk", [([1024] * 3, 4, 32), ([4099] * 2, 3, 64),
                                           ([1, 2, 3, 5, 64, 65, 1000, 3001], 2, 32),
                                           ([200, 17, 500], 2, 0)])
def test_fused_pass_equals_per_level_launches(seq_T, D, chunk, prec):
    """One launch per solve pass (a CTA runs every level of its systems) performs the same
    operations in the same order as one launch per level: the outputs agree bit for bit,
    forward and adjoint.  ALGO_AUTO (one launch for the levels whose systems fit a CTA, its
    top level a warp-shuffle PCR: another elimination order) agrees with the oracle within
    the precision's tolerance."""
    pk = P()
    prob = ragged_problem(seq_T, D=D, seed=21)
    gy = upstream_gradient(prob)
    p = getattr(pk, prec)
    split = gpu_grad(prob, gy, p, algo=pk.ALGO_CR, chunk=chunk)
    fused = gpu_grad(prob, gy, p, algo=pk.ALGO_CR_FUSED, chunk=chunk)
    for a, b in zip(fused, split):
        np.testing.assert_array_equal(a, b)
    assert (fused[-2] == 0).all() and (fused[-1] == 0).all()
    auto = gpu_grad(prob, gy, p, algo=pk.ALGO_AUTO, chunk=chunk)
    assert (auto[-2] == 0).all() and (auto[-1] == 0).all()
    tol = {"F64": TOL_F64, "F32": TOL_F32}.get(prec, TOL_REF)
    wdt = np.float64 if p == pk.F64 else np.float32
    yo, gco, gdo, gso, guo, _ = oracle_grad(rounded(prob, p), gy.astype(wdt).astype(np.float64))
    assert rel_err_per_system(auto[0], yo, prob).max() <= tol
    if prec != "F32":
        assert_grads(auto, (yo, gco, gdo, gso, guo), prob, tol, 1e-8 if p == pk.F64 else tol)


@pytest.mark.parametrize("prec", REFINED)
@pytest.mark.parametrize("store_factor", [True, False])
@pytest.mark.parametrize("seq_T,D,tol", [([1024] * 6, 2, 1e-7), ([1000, 700, 33, 1024, 97, 1], 3, 1e-7),
                                         ([500, 300, 17], 2, 1e-7), ([1024] * 4, 2, 0.0)])
def test_warp_fused_launches_equal_per_level_launches(seq_T, D, tol, store_factor, prec):
    """Two-level plans (level-0 chunks of 32 steps, a warp-shuffle PCR on top) whose systems
    fit a warp run their refined solves one warp per system, one launch per pass boundary;
    the same plan with per_level_launches runs one launch per level, pass and stop test.  The
    arithmetic and its order are the same: y, every gradient and both info arrays agree bit
    for bit, forward and adjoint, with and without the stop test, with the saved factor and
    with the factor recomputed, for systems of 1 to 32 chunks and PCR groups of 16 and 32."""
    from paper_2410_06074_b300 import binding as Bd
    pk = P()
    prob = ragged_problem(seq_T, D=D, seed=27)
    gy = upstream_gradient(prob).astype(np.float32)
    p = getattr(pk, prec)
    n0 = Bd.launch_count()
    fused = gpu_grad(prob, gy, p, chunk=32, refine_tol=tol, store_factor=store_factor)
    n1 = Bd.launch_count()
    split = gpu_grad(prob, gy, p, chunk=32, refine_tol=tol, store_factor=store_factor, per_level_launches=1)
    n2 = Bd.launch_count()
    assert n1 - n0 < n2 - n1          # the fused launches did run
    for a, b in zip(fused, split):
        np.testing.assert_array_equal(a, b)
    assert (fused[-2] == 0).all() and (fused[-1] == 0).all()
    yo, *_ = oracle_grad(rounded(prob, p), gy.astype(np.float64))
    assert rel_err_per_system(fused[0], yo, prob).max() <= TOL_REF


@pytest.mark.parametrize("T,chunk", [(1000, 0), (2500, 16)])
def test_fp64_forward(T, chunk):
    pk = P()
    prob = random_problem(8, 2, 3, T, 2)
    y, info = gpu_solve(prob, pk.F64, chunk=chunk)
    yo, _ = oracle_solve(prob)
    assert rel_err_per_system(y, yo, prob).max() <= TOL_F64


def test_unrefined_fp32_error_band():
    pk = P()
    prob = random_problem(9, 4, 2, 1024, 2)
    y, info = gpu_solve(prob, pk.F32, max_refine=0)
    yo, _ = oracle_solve(rounded(prob, pk.F32))
    e = rel_err_per_system(y, yo, prob)
    assert e.max() <= TOL_F32
    y1, _ = gpu_solve(prob, pk.F32_REFINED, max_refine=1)
    e1 = rel_err_per_system(y1, yo, prob)
    assert e1.max() < e.max() * 0.05      # one sweep contracts the error by > 20x


@pytest.mark.parametrize("prec", REFINED)
@pytest.mark.parametrize("R", [1, 3])
def test_other_orders(R, prec):
    pk = P()
    prob = random_problem(10, 2, 2, 1500, R, s_lo=0.1, s_hi=0.5)
    y, info = gpu_solve(prob, getattr(pk, prec))
    yo, _ = oracle_solve(rounded(prob, pk.F32_REFINED))
    assert (info == 0).all()
    assert rel_err_per_system(y, yo, prob).max() <= TOL_REF
    y, info = gpu_solve(prob, pk.F64)
    yo, _ = oracle_solve(prob)
    assert rel_err_per_system(y, yo, prob).max() <= TOL_F64


def test_initial_values_over_several_steps_and_weights():
    pk = P()
    prob = random_problem(11, 2, 2, 700, 2, R_init=2, T_init=3, w=(0.7, 1.9, 1.3))
    for prec, tol in ((pk.F64, TOL_F64), (pk.F32_REFINED, TOL_REF)):
        y, info = gpu_solve(prob, prec)
        yo, _ = oracle_solve(rounded(prob, prec))
        assert rel_err_per_system(y, yo, prob).max() <= tol


@pytest.mark.parametrize("seq_T", [[1, 2, 3, 5, 64, 65, 1000, 3001], [4096, 17, 2049]])
def test_ragged_batch(seq_T):
    pk = P()
    prob = ragged_problem(seq_T, D=2)
    for prec, tol in ((pk.F64, TOL_F64), (pk.F32_REFINED, TOL_REF)):
        y, info = gpu_solve(prob, prec)
        yo, info_o = oracle_solve(rounded(prob, prec))
        assert (info == info_o).all()
        assert rel_err_per_system(y, yo, prob).max() <= tol


@pytest.mark.parametrize("chunk,tops", [(8, [1, 2, 3, 5, 8, 13, 16, 17, 31, 32]),
                                        (16, [1, 2, 3, 5, 8, 9, 13, 16])])
def test_pcr_top_level_over_every_size(chunk, tops):
    """ALGO_AUTO solves the top level (<= 32 separators per system) by a warp-shuffle
    parallel cyclic reduction: systems whose top levels hold 1 to 32 (or 1 to 16)
    separators share one plan (groups of 32, or 16 lanes with two systems per warp; rows
    beyond a system's size idle), forward and adjoint against the oracle."""
    pk = P()
    prob = ragged_problem([chunk * p - (p % 3) for p in tops], D=2, seed=33)
    gy = upstream_gradient(prob)
    for prec, tol, gtol in ((pk.F64, TOL_F64, 1e-8), (pk.F32_REFINED_DF, TOL_REF, TOL_REF)):
        wdt = np.float64 if prec == pk.F64 else np.float32
        y, gc, gd, gs, gu, info, info2 = gpu_grad(prob, gy.astype(wdt), prec, algo=pk.ALGO_AUTO,
                                                  chunk=chunk)
        yo, gco, gdo, gso, guo, info_o = oracle_grad(rounded(prob, prec), gy.astype(wdt).astype(np.float64))
        assert (info == 0).all() and (info2 == 0).all() and (info_o == 0).all()
        assert_grads((y, gc, gd, gs, gu), (yo, gco, gdo, gso, guo), prob, tol, gtol)


def test_exact_polynomial_recovery_on_gpu():
    """Degree-<=R polynomial trajectories satisfy every row exactly (any c, any s)."""
    pk = P()
    R, T = 2, 2000
    rng = np.random.Generator(np.random.PCG64(12))
    coef = rng.standard_normal(R + 1)
    s = rng.uniform(0.05, 0.3, T)      # kappa(M) stays ~1e6 (tiny steps make FP64 lose digits)
    tau = np.concatenate([[0.0], np.cumsum(s[:-1])])
    y = np.stack([np.polynomial.polynomial.polyval(tau, np.polynomial.polynomial.polyder(coef, r)
                                                   if r else coef) for r in range(R + 1)], -1)
    c = rng.standard_normal((T, R + 1)); c[:, R] = 1 + np.abs(c[:, R])
    d = np.sum(c * y, axis=1)
    prob = Problem("poly", R, 1, 1, 1, 1, T, c[None, None], d[None, None], s[None],
                   y[None, None, :1, :2])
    yg, info = gpu_solve(prob, pk.F64)
    assert np.abs(yg[0, 0] - y).max() <= 1e-9 * np.abs(y).max()


def test_assemble_matches_appendix_blocks():
    import torch
    from test_oracle_pins import appendix_a2_blocks
    pk = P()
    prob = random_problem(13, 2, 2, 50, 3, R_init=1, T_init=2, w=(1.2, 0.8, 1.5))
    c, d, s, u = (torch.from_numpy(a).cuda() for a in (prob.c, prob.d, prob.s, prob.u))
    cfg = pk.SolveConfig(R_init=1, T_init=2, w_gov=1.2, w_init=0.8, w_smooth=1.5, precision=pk.F64)
    plan = pk.get_plan((3, 2, 2, 50), cfg)
    nb, nt = 4, 10
    M = torch.empty(2, 2, 50, nt, dtype=torch.float64, device="cuda")
    N = torch.empty(2, 2, 50, nb * nb, dtype=torch.float64, device="cuda")
    beta = torch.empty(2, 2, 50, nb, dtype=torch.float64, device="cuda")
    plan.assemble(c, d, s, u, M, N, beta)
    M, N, beta = M.cpu().numpy(), N.cpu().numpy(), beta.cpu().numpy()
    il = np.tril_indices(nb)
    for b in range(2):
        for dd in range(2):
            Ma, Na, ba = appendix_a2_blocks(3, 1, 2, 1.2, 0.8, 1.5, prob.c[b, dd], prob.d[b, dd],
                                            prob.s[b], prob.u[b, dd])
            order = [(i, j) for i in range(nb) for j in range(i + 1)]
            Mp = np.stack([[Ma[t][i, j] for (i, j) in order] for t in range(50)])
            np.testing.assert_allclose(M[b, dd], Mp, rtol=1e-13, atol=1e-14)
            np.testing.assert_allclose(N[b, dd, :49], Na.reshape(49, -1), rtol=1e-13, atol=1e-14)
            assert (N[b, dd, 49] == 0).all()
            np.testing.assert_allclose(beta[b, dd], ba, rtol=1e-13, atol=1e-14)


# ----------------------------------------------------------------------------- failures

def test_info_reports_bad_pivots_and_nan_fills():
    pk = P()
    prob = random_problem(14, 1, 3, 40, 2)
    c = prob.c.copy(); c[0, 1, 9, 0] = np.nan          # system 1: NaN at 1-based step 10
    bad = Problem("nan", 2, 1, 1, 1, 3, 40, c, prob.d, prob.s, prob.u)
    for prec in (pk.F64, pk.F32_REFINED):
        for chunk in (0, 4, 10):
            y, info = gpu_solve(bad, prec, chunk=chunk)
            assert info[1] == 10, (prec, chunk, info)
            assert info[0] == 0 and info[2] == 0
            assert np.isnan(y[0, 1]).all() and np.isfinite(y[0, [0, 2]]).all()
    # T = 1 with c = 0 and w_init = 0: M = 0 exactly
    one = random_problem(15, 1, 1, 1, 2)
    z = Problem("zero", 2, 1, 1, 1, 1, 1, np.zeros_like(one.c), one.d, one.s, one.u, w_init=0.0)
    y, info = gpu_solve(z, pk.F64)
    assert info[0] == 1 and np.isnan(y).all()


# ----------------------------------------------------------------------------- gradients

@pytest.mark.parametrize("store_factor", [True, False])
def test_gradients_fp64_match_oracle(store_factor):
    pk = P()
    prob = random_problem(16, 2, 3, 300, 2, T_init=2, w=(1.1, 0.9, 1.3))
    gy = upstream_gradient(prob)
    y, gc, gd, gs, gu, info, info2 = gpu_grad(prob, gy, pk.F64, store_factor=store_factor, chunk=8)
    yo, gco, gdo, gso, guo, info_o = oracle_grad(prob, gy)
    assert_grads((y, gc, gd, gs, gu), (yo, gco, gdo, gso, guo), prob, 1e-8)


@pytest.mark.parametrize("prec", REFINED)
@pytest.mark.parametrize("T,chunk", [(1024, 0), (777, 16)])
def test_gradients_refined_fp32_match_oracle(T, chunk, prec):
    pk = P()
    prob = random_problem(17, 2, 4, T, 2)
    gy = upstream_gradient(prob)
    r = rounded(prob, pk.F32_REFINED)
    y, gc, gd, gs, gu, info, info2 = gpu_grad(prob, gy.astype(np.float32), getattr(pk, prec), chunk=chunk)
    yo, gco, gdo, gso, guo, _ = oracle_grad(r, gy.astype(np.float32).astype(np.float64))
    assert_grads((y, gc, gd, gs, gu), (yo, gco, gdo, gso, guo), prob, TOL_REF)


@pytest.mark.parametrize("prec", REFINED)
def test_saved_and_recomputed_factor_agree(prec):
    """With the saved factor the backward reuses the forward's refined y; without it the
    factor is recomputed and y refined again.  Both must meet the refined tolerance."""
    pk = P()
    prob = random_problem(18, 2, 2, 900, 2)
    gy = upstream_gradient(prob).astype(np.float32)
    a = gpu_grad(prob, gy, getattr(pk, prec), store_factor=True)
    b = gpu_grad(prob, gy, getattr(pk, prec), store_factor=False)
    ref = oracle_grad(rounded(prob, pk.F32_REFINED), gy.astype(np.float64))
    assert_grads(a, ref, prob, TOL_REF)
    assert_grads(b, ref, prob, TOL_REF)
    assert_grads(a, b, prob, TOL_REF)


def test_gradcheck_config2_slice():
    """torch.autograd.gradcheck of SmnnSolve on the B=2, D=1, T=16 slice, FP64 path."""
    import torch
    from smnn_workloads import config2_slice
    pk = P()
    prob = config2_slice()
    scale = 0.05   # s = scale * z with z ~ 1, so that one eps suits every input
    c, d, z, u = (torch.from_numpy(a).cuda().requires_grad_(True)
                  for a in (prob.c, prob.d, prob.s / scale, prob.u))
    cfg = pk.SolveConfig(R_init=1, T_init=1, precision=pk.F64)
    f = lambda c, d, z, u: pk.smnn_layer(c, d, z * scale, u, cfg)[0]
    # kappa(M) ~ 2e5 here: eps = 1e-6 would leave ~1e-5 finite-difference noise from FP64
    # rounding of the solve itself; eps = 1e-4 keeps both noise and truncation below 1e-7
    assert torch.autograd.gradcheck(f, (c, d, z, u), eps=1e-4, atol=1e-6, rtol=1e-4)


def test_gradcheck_with_learnable_weights():
    """gradcheck of SmnnSolve with (w_gov, w_init, w_smooth) as a differentiable input, FP64."""
    import torch
    from smnn_workloads import config2_slice
    pk = P()
    prob = config2_slice()
    c, d, s, u = (torch.from_numpy(a).cuda() for a in (prob.c, prob.d, prob.s, prob.u))
    w = torch.tensor([0.9, 1.2, 1.1], dtype=torch.float64, device="cuda", requires_grad=True)
    cfg = pk.SolveConfig(R_init=1, T_init=1, precision=pk.F64)
    f = lambda w: pk.smnn_layer(c, d, s, u, cfg, weights=w)[0]
    assert torch.autograd.gradcheck(f, (w,), eps=1e-5, atol=1e-6, rtol=1e-4)


def test_autotuner_checks_candidates_and_picks_a_correct_one():
    import torch
    import paper_2410_06074_b300 as pk
    prob = random_problem(51, 4, 4, 2048, 2).cast(np.float32)
    c, d, s, u = (torch.from_numpy(a).cuda() for a in (prob.c, prob.d, prob.s, prob.u))
    gy = torch.from_numpy(upstream_gradient(prob).astype(np.float32)).cuda()
    cfg = pk.SolveConfig(R_init=1, T_init=1, precision=pk.F32_REFINED_DF)
    best, res = pk.autotune.autotune(c, d, s, u, cfg, gy, save=False)
    assert any(v is not None for v in res.values())
    assert (best.algo, best.chunk) in [k for k, v in res.items() if v is not None]
    y, info = pk.solve(c, d, s, u, best)
    yo, _ = oracle_solve(prob.as_f64())
    assert rel_err_per_system(y.double().cpu().numpy(), yo, prob).max() <= TOL_REF


@pytest.mark.parametrize("prec", REFINED)
def test_adaptive_refinement_stop_test(prec):
    """With refine_tol each system stops once its estimated error is small; results still meet
    the refined tolerance and no system is flagged on a well-conditioned batch."""
    pk = P()
    prob = random_problem(61, 8, 4, 1024, 2)
    y, info = gpu_solve(prob, getattr(pk, prec), max_refine=4, refine_tol=1e-8)
    yo, _ = oracle_solve(rounded(prob, pk.F32_REFINED))
    assert (info == 0).all()
    assert rel_err_per_system(y, yo, prob).max() <= TOL_REF
    gy = upstream_gradient(prob).astype(np.float32)
    out = gpu_grad(prob, gy, getattr(pk, prec), max_refine=4, adjoint_refine=3, refine_tol=1e-8)
    ref = oracle_grad(rounded(prob, pk.F32_REFINED), gy.astype(np.float64))
    assert_grads(out, ref, prob, TOL_REF)
    assert (out[5] == 0).all() and (out[6] == 0).all()


# ----------------------------------------------------------------------------- weight gradients

@pytest.mark.parametrize("prec,tol", [("F64", 1e-9), ("F32_REFINED", 1e-6), ("F32_REFINED_DF", 1e-6)])
@pytest.mark.parametrize("store_factor", [True, False])
def test_weight_gradients_match_oracle(prec, tol, store_factor):
    """dl/d(w_gov, w_init, w_smooth) (shared by the batch) against the oracle's row-wise chain
    rule, on a ragged batch with non-unit weights and several initial steps."""
    import torch
    import paper_2410_06074_b300 as pk
    from paper_2410_06074_b300 import get_plan, gradients, solve
    from paper_2410_06074_b300.api import _shape_key
    from _helpers import cfg_of, dev, np_dtype, oracle_params
    base = ragged_problem([300, 17, 1025, 64], D=3, seed=23)
    prob = Problem("weights", 2, 2, 3, base.B, base.D, None, base.c, base.d, base.s,
                   np.random.Generator(np.random.PCG64(24)).standard_normal((base.S, 3, 3)),
                   seq_T=base.seq_T, w_gov=0.8, w_init=1.7, w_smooth=1.3)
    p = getattr(pk, prec)
    dt = np_dtype(p)
    gy = upstream_gradient(prob).astype(dt)
    c, d, s, u = dev(prob, dt)
    cfg = cfg_of(prob, p)
    plan = get_plan(_shape_key(c, s, prob.D, prob.seq_T), cfg)
    fac = plan.factor_buffer() if store_factor else None
    y, info = solve(c, d, s, u, cfg, D=prob.D, seq_T=prob.seq_T, factor=fac)
    gc, gd, gs, gu, gw, info2 = gradients(c, d, s, u, y, torch.from_numpy(gy).cuda(), cfg, D=prob.D,
                                          seq_T=prob.seq_T, factor=fac, weights=True)
    r = rounded(prob, p)
    *_, gwo, info_o = O.gradient(oracle_params(r), r.c, r.d, r.s, r.u, gy.astype(np.float64),
                                 D=r.D, seq_T=r.seq_T, weights=True)
    assert (info.cpu().numpy() == 0).all() and (info2.cpu().numpy() == 0).all() and (info_o == 0).all()
    gw = gw.cpu().numpy()
    assert np.abs(gw - gwo).max() <= tol * np.abs(gwo).max(), (gw, gwo)
    # the same call without gw leaves the other gradients unchanged
    gc2, gd2, gs2, gu2, _ = gradients(c, d, s, u, y, torch.from_numpy(gy).cuda(), cfg, D=prob.D,
                                      seq_T=prob.seq_T, factor=fac)
    for a, b in ((gc, gc2), (gd, gd2), (gs, gs2), (gu, gu2)):
        assert torch.equal(a, b)


# ----------------------------------------------------------------------------- host pipeline

@pytest.mark.parametrize("n_parts", [1, 3])
def test_host_pipeline_matches_device_calls(n_parts):
    """HostPipeline (pinned host buffers, parts of the batch on two streams) gives the forward
    and adjoint results of one device call on the whole batch."""
    import torch
    import paper_2410_06074_b300 as pk
    prob = random_problem(31, 8, 2, 300, 2).cast(np.float32)
    gy = upstream_gradient(prob).astype(np.float32)
    cfg = pk.SolveConfig(R_init=prob.R_init, T_init=prob.T_init, precision=pk.F32_REFINED_DF)
    host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
            for a in (prob.c, prob.d, prob.s, prob.u, gy)]
    outs = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in (host[0], host[0], host[1], host[2], host[3])]
    pipe = pk.HostPipeline((prob.R, prob.B, prob.D, prob.T), cfg, n_parts=n_parts)
    info, info_b = pipe.run(*host, *outs)
    torch.cuda.synchronize()
    assert (info.cpu() == 0).all() and (info_b.cpu() == 0).all()
    c, d, s, u, g = (t.cuda() for t in host)
    y, _ = pk.solve(c, d, s, u, cfg)
    ref = [y] + list(pk.gradients(c, d, s, u, y, g, cfg)[:4])
    for got, want in zip(outs, ref):
        want = want.cpu().double()
        assert float((got.double() - want).norm() / want.norm()) <= 1e-6


@pytest.mark.parametrize("n_sets", [2, 3])
def test_host_stream_steps_match_device_calls(n_sets):
    """HostStream (three streams, n_sets rotating device buffer sets, the steps' transfers
    overlapped) returns for every step exactly what the device calls return for that step's
    inputs."""
    import torch
    import paper_2410_06074_b300 as pk
    cfg = pk.SolveConfig(R_init=1, T_init=1, precision=pk.F32_REFINED_DF)
    steps = []
    for seed in (41, 42, 43, 44):
        prob = random_problem(seed, 6, 2, 257, 2).cast(np.float32)
        gy = upstream_gradient(prob, seed).astype(np.float32)
        host = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
                for a in (prob.c, prob.d, prob.s, prob.u, gy)]
        outs = [torch.empty(t.shape, dtype=t.dtype).pin_memory()
                for t in (host[0], host[0], host[1], host[2], host[3])]
        steps.append((host, outs))
    hs = pk.HostStream((2, 6, 2, 257), cfg, n_sets=n_sets)
    flags = [hs.submit(*h, *o) for h, o in steps]
    hs.wait()
    torch.cuda.synchronize()
    for info, info_b, _ in flags[-n_sets:]:   # a set's flags are reused n_sets steps later
        assert (info.cpu() == 0).all() and (info_b.cpu() == 0).all()
    fac = pk.get_plan((2, 6, 2, 257), cfg).factor_buffer()   # the saved-factor path, as HostStream
    for h, o in steps:
        c, d, s, u, g = (t.cuda() for t in h)
        y, _ = pk.solve(c, d, s, u, cfg, factor=fac)
        ref = [y] + list(pk.gradients(c, d, s, u, y, g, cfg, factor=fac)[:4])
        for got, want in zip(o, ref):
            assert torch.equal(got, want.cpu())


# ----------------------------------------------------------------------------- coupled systems

@pytest.mark.parametrize("prec,tol", [("F64", 1e-9), ("F32_REFINED_DF", 1e-6), ("F32_REFINED", 1e-6)])
@pytest.mark.parametrize("Q,T,algo,chunk", [(2, 1000, "AUTO", 0), (2, 777, "CR", 16), (2, 300, "CR_FUSED", 8),
                                            (1, 400, "AUTO", 0)])
def test_coupled_systems_match_oracle(Q, T, algo, chunk, prec, tol):
    """V = 2 variables (R = 1: 4 unknowns per step) with Q governing equations per step
    (Sec. 3.1, Eq. 4-7), forward and adjoint, against the oracle's coupled rows."""
    import paper_2410_06074_b300 as pk
    from smnn_workloads import random_coupled_problem
    prob = random_coupled_problem(60 + Q, 3, 2, T, R=1, V=2, Q=Q, T_init=2, w=(0.9, 1.1, 1.2))
    p = getattr(pk, prec)
    gy = upstream_gradient(prob)[..., :4]
    y, gc, gd, gs, gu, info, info2 = gpu_grad(prob, gy.astype(np.float64 if p == pk.F64 else np.float32), p,
                                              algo=getattr(pk, "ALGO_" + algo), chunk=chunk)
    r = rounded(prob, p)
    g64 = gy.astype(np.float64 if p == pk.F64 else np.float32).astype(np.float64)
    yo, gco, gdo, gso, guo, info_o = oracle_grad(r, g64)
    assert (info == 0).all() and (info2 == 0).all() and (info_o == 0).all()
    assert y.shape == (3, 2, T, 4)
    assert_grads((y, gc, gd, gs, gu), (yo, gco, gdo, gso, guo), prob, tol, 1e-8 if p == pk.F64 else tol)


@pytest.mark.parametrize("prec,tol", [("F64", 1e-9), ("F32_REFINED_DF", 1e-6)])
@pytest.mark.parametrize("V,R,Q", [(3, 1, 3), (2, 2, 2)])
@pytest.mark.parametrize("T,algo,chunk", [(1000, "AUTO", 0), (333, "CR", 8), (200, "CR_FUSED", 8),
                                          (150, "SEQ", 0)])
def test_coupled_six_wide_blocks_match_oracle(V, R, Q, T, algo, chunk, prec, tol):
    """Steps of n_b = V(R+1) = 6 unknowns: three first-order variables with three equations,
    and two second-order variables with two equations (Sec. 3.1), forward and adjoint,
    against the oracle's coupled rows.  The highest-derivative block of each step is made
    diagonally dominant (lead_cross), so that the FP32 factor's refinement converges."""
    import paper_2410_06074_b300 as pk
    from smnn_workloads import random_coupled_problem
    prob = random_coupled_problem(80 + V, 3, 2, T, R=R, V=V, Q=Q, T_init=2, w=(1.1, 0.9, 1.05),
                                  lead_cross=0.5 / (V - 1))
    p = getattr(pk, prec)
    nb = V * (R + 1)
    gy = upstream_gradient(prob)[..., :nb]
    wdt = np.float64 if p == pk.F64 else np.float32
    y, gc, gd, gs, gu, info, info2 = gpu_grad(prob, gy.astype(wdt), p,
                                              algo=getattr(pk, "ALGO_" + algo), chunk=chunk)
    r = rounded(prob, p)
    yo, gco, gdo, gso, guo, info_o = oracle_grad(r, gy.astype(wdt).astype(np.float64))
    assert (info == 0).all() and (info2 == 0).all() and (info_o == 0).all()
    assert y.shape == (3, 2, T, nb)
    assert_grads((y, gc, gd, gs, gu), (yo, gco, gdo, gso, guo), prob, tol, 1e-8 if p == pk.F64 else tol)


@pytest.mark.parametrize("prec,tol", [("F64", 1e-9), ("F32_REFINED_DF", 1e-6)])
@pytest.mark.parametrize("T,algo,chunk", [(600, "AUTO", 0), (257, "CR", 8), (120, "SEQ", 0)])
def test_coupled_nine_wide_blocks_match_oracle(T, algo, chunk, prec, tol):
    """Steps of n_b = V(R+1) = 9 unknowns: three coupled second-order states with three
    governing equations per step (Sec. 3.1, Eq. 4-8), forward and adjoint, against the
    oracle's coupled rows.  Each step's highest-derivative block is kept diagonally dominant
    (lead_cross), so that the FP32 factor's refinement converges."""
    import paper_2410_06074_b300 as pk
    from smnn_workloads import random_coupled_problem
    V, R, Q = 3, 2, 3
    prob = random_coupled_problem(90, 2, 2, T, R=R, V=V, Q=Q, T_init=2, w=(1.05, 0.95, 1.1),
                                  lead_cross=0.5 / (V - 1))
    p = getattr(pk, prec)
    nb = V * (R + 1)
    gy = upstream_gradient(prob)[..., :nb]
    wdt = np.float64 if p == pk.F64 else np.float32
    y, gc, gd, gs, gu, info, info2 = gpu_grad(prob, gy.astype(wdt), p,
                                              algo=getattr(pk, "ALGO_" + algo), chunk=chunk)
    r = rounded(prob, p)
    yo, gco, gdo, gso, guo, info_o = oracle_grad(r, gy.astype(wdt).astype(np.float64))
    assert (info == 0).all() and (info2 == 0).all() and (info_o == 0).all()
    assert y.shape == (2, 2, T, nb)
    assert_grads((y, gc, gd, gs, gu), (yo, gco, gdo, gso, guo), prob, tol, 1e-8 if p == pk.F64 else tol)


def test_coupled_decoupled_equations_equal_independent_gpu_solves():
    """On the GPU too: two variables whose equations do not couple them solve as two scalar
    systems (FP64)."""
    import paper_2410_06074_b300 as pk
    from smnn_workloads import random_coupled_problem
    R, T = 1, 500
    prob = random_coupled_problem(70, 2, 1, T, R, V=2, Q=2)
    c = prob.c.reshape(2, 1, T, 2, 2, R + 1).copy()
    c[:, :, :, 0, 1, :] = 0.0
    c[:, :, :, 1, 0, :] = 0.0
    cp = Problem("decoupled", R, prob.R_init, 1, 2, 1, T, c.reshape(2, 1, T, -1), prob.d, prob.s,
                 prob.u, V=2, Q=2)
    y, info = gpu_solve(cp, pk.F64)
    assert (info == 0).all()
    ui = prob.u.reshape(2, 1, 1, 2, prob.R_init + 1)
    for v in range(2):
        one = Problem("one", R, prob.R_init, 1, 2, 1, T, np.ascontiguousarray(c[:, :, :, v, v, :]),
                      np.ascontiguousarray(prob.d[..., v]), prob.s, np.ascontiguousarray(ui[:, :, :, v, :]))
        yv, iv = gpu_solve(one, pk.F64)
        assert (iv == 0).all()
        np.testing.assert_allclose(y[..., v * (R + 1):(v + 1) * (R + 1)], yv, rtol=1e-10, atol=1e-12)
