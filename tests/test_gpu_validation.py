"""App. B.1's standalone ODEs (the cases of Table 5) through the CUDA path (GPU required):
each batch agrees with the FP64 oracle, and the relative MSE against the closed-form
solutions reproduces Table 5's first-order rows to the printed digits and stays below the
paper's 1e-6 bound for the oscillators."""
import math
import os

import numpy as np
import pytest

import smnn_workloads as W
from _helpers import gpu_solve, oracle_solve, rel_err_per_system, rounded

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rel_mse(yhat, y):
    return float(np.sum((yhat - y) ** 2) / np.sum((y - y.mean()) ** 2))


def _gold():
    out = {}
    with open(os.path.join(GOLDEN, "table5_first_order.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                parts = line.split()
                out[parts[0]] = [float(v) for v in parts[1:]]
    return out


# Parity tolerance of two FP64 solvers ~ kappa(M) * 1e-16: with h = 0.01 the smoothness rows
# of the highest order weigh h^{2R} against the governing rows, so kappa grows like h^{-2R}
# (R = 2: measured agreement ~1e-11; R = 3 oscillators: 1.9e-7).  The third-order ODE has
# c_0 = 0, so y itself is fixed only by the initial values and the smoothness rows: the two
# FP64 solvers agree to 6e-4 there, and its relative MSE (1.3e-6 in the oracle at R = 3) is
# checked against a bound only.
@pytest.mark.parametrize("R,R_init,tol,rtol", [(2, 0, 1e-9, 0.01), (3, 1, 1e-6, 0.01), (3, 2, 1e-3, None)])
def test_table5_cases_on_gpu_fp64(R, R_init, tol, rtol):
    import paper_2410_06074_b300 as pk
    prob, cases = W.table5_batch(R, R_init)
    y, info = gpu_solve(prob, pk.F64)
    yo, info_o = oracle_solve(prob)
    assert (info == 0).all() and (info_o == 0).all()
    assert rel_err_per_system(y, yo, prob).max() <= tol
    if rtol is None:
        for b, cse in enumerate(cases):
            assert max(_rel_mse(y[b, 0, :, r], cse["exact"][r]) for r in range(3)) < 1e-5
    else:
        _check_against_closed_forms(y, yo, cases, rtol=rtol)


# With h = 0.01 the highest derivative is fixed only by smoothness rows of weight h^{2R}
# (1e-8 for R = 2, 1e-12 for R = 3), so kappa(M) is far beyond an FP32 factorisation for
# most of these cases: the refined FP32 paths solve RC and language death, and must flag
# (info != 0) every system they do not solve -- a breakdown (> 0) or a refinement that
# does not converge (-1) -- instead of returning it silently.
@pytest.mark.parametrize("prec", ["F32_REFINED", "F32_REFINED_DF"])
@pytest.mark.parametrize("R,R_init", [(2, 0), (3, 1), (3, 2)])
def test_table5_cases_on_gpu_refined_fp32(R, R_init, prec):
    import paper_2410_06074_b300 as pk
    prob, cases = W.table5_batch(R, R_init)
    p = getattr(pk, prec)
    y, info = gpu_solve(prob, p, refine_tol=1e-6)
    yo, _ = oracle_solve(rounded(prob, p))
    err = rel_err_per_system(y, yo, prob)
    for b, cse in enumerate(cases):
        if cse["name"] in ("RC", "Language"):
            assert info[b] == 0, (cse["name"], info[b])
        assert info[b] != 0 or err[b] <= 1e-6, (cse["name"], info[b], err[b])
    ok = [b for b in range(len(cases)) if info[b] == 0]
    _check_against_closed_forms(y[ok], yo[ok], [cases[b] for b in ok], exact_inputs=False, rtol=0.1)


def _check_against_closed_forms(y, yo, cases, exact_inputs=True, rtol=0.01):
    """Relative MSE against the closed forms: Table 5's printed first-order rows (only with
    the exact inputs: FP32 rounds h = 0.01, which shifts the time grid by ~2e-8 relative and
    moves the second printed digit), the paper's 1e-6 bound for the oscillators, and, for
    every case, the oracle's own relative MSE on the same inputs within rtol."""
    gold = _gold()
    for b, cse in enumerate(cases):
        got = [_rel_mse(y[b, 0, :, r], cse["exact"][r]) for r in range(3)]
        ref = [_rel_mse(yo[b, 0, :, r], cse["exact"][r]) for r in range(3)]
        if cse["name"] in gold and exact_inputs:      # printed to two significant digits
            for g, v in zip(got, gold[cse["name"]]):
                assert abs(g - v) <= 0.051 * 10 ** math.floor(math.log10(v)) * 1.0001, (cse["name"], g, v)
        elif cse["name"] in ("Harmonic", "Damped"):
            assert max(got) < 1e-6, (cse["name"], got)
        for g, r in zip(got, ref):
            assert abs(g - r) <= rtol * r + 1e-15, (cse["name"], g, r)
