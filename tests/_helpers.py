"""Shared test plumbing: move a seeded Problem to the GPU, call the library through its
binding, call the oracle on the same (rounded) inputs, and compare."""
import numpy as np

import oracle as O


def oracle_params(prob):
    return O.Params(prob.R, prob.R_init, prob.T_init, prob.w_gov, prob.w_init, prob.w_smooth,
                    V=prob.V, Q=prob.Q)


def dev(prob, dtype):
    import torch
    tt = torch.float64 if dtype == np.float64 else torch.float32
    return tuple(torch.from_numpy(np.ascontiguousarray(a, dtype)).to("cuda", tt)
                 for a in (prob.c, prob.d, prob.s, prob.u))


def cfg_of(prob, precision, **kw):
    from paper_2410_06074_b300 import SolveConfig
    kw.setdefault("V", prob.V)
    kw.setdefault("Q", prob.Q)
    return SolveConfig(R_init=prob.R_init, T_init=prob.T_init, w_gov=prob.w_gov,
                       w_init=prob.w_init, w_smooth=prob.w_smooth, precision=precision, **kw)


def np_dtype(precision):
    from paper_2410_06074_b300 import F64
    return np.float64 if precision == F64 else np.float32


def gpu_solve(prob, precision, **kw):
    from paper_2410_06074_b300 import solve
    dt = np_dtype(precision)
    c, d, s, u = dev(prob, dt)
    y, info = solve(c, d, s, u, cfg_of(prob, precision, **kw), D=prob.D, seq_T=prob.seq_T)
    return y.double().cpu().numpy(), info.cpu().numpy()


def gpu_grad(prob, gy, precision, store_factor=True, **kw):
    import torch
    from paper_2410_06074_b300 import get_plan, gradients, solve
    from paper_2410_06074_b300.api import _shape_key
    dt = np_dtype(precision)
    c, d, s, u = dev(prob, dt)
    cfg = cfg_of(prob, precision, **kw)
    plan = get_plan(_shape_key(c, s, prob.D, prob.seq_T, cfg), cfg)
    fac = plan.factor_buffer() if store_factor else None
    y, info = solve(c, d, s, u, cfg, D=prob.D, seq_T=prob.seq_T, factor=fac)
    gyt = torch.from_numpy(np.ascontiguousarray(gy, dt)).cuda()
    gc, gd, gs, gu, info2 = gradients(c, d, s, u, y, gyt, cfg, D=prob.D, seq_T=prob.seq_T, factor=fac)
    out = [t.double().cpu().numpy() for t in (y, gc, gd, gs, gu)]
    return out + [info.cpu().numpy(), info2.cpu().numpy()]


def rounded(prob, precision):
    """The problem as the GPU sees it (inputs rounded to the working precision)."""
    return prob.cast(np_dtype(precision)).as_f64()


def oracle_solve(prob, nthreads=0):
    return O.solve(oracle_params(prob), prob.c, prob.d, prob.s, prob.u, D=prob.D,
                   seq_T=prob.seq_T, nthreads=nthreads)


def oracle_grad(prob, gy, nthreads=0):
    return O.gradient(oracle_params(prob), prob.c, prob.d, prob.s, prob.u, gy, D=prob.D,
                      seq_T=prob.seq_T, nthreads=nthreads)


def per_system(a, prob):
    """Split a per-step array (uniform or ragged layout) into one flat vector per system."""
    if prob.seq_T is None:
        S = prob.B * prob.D
        return [x.reshape(-1) for x in a.reshape(S, prob.T, -1)]
    out, pos = [], 0
    for Tb in prob.seq_T:
        for _ in range(prob.D):
            out.append(a[pos:pos + Tb].reshape(-1))
            pos += Tb
    return out


def rel_err_per_system(got, ref, prob):
    return np.array([np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)
                     for g, r in zip(per_system(got, prob), per_system(ref, prob))])


def rel_err(got, ref):
    return float(np.linalg.norm((got - ref).reshape(-1)) / max(np.linalg.norm(ref.reshape(-1)), 1e-300))


def per_sequence(a, prob):
    """Split a per-sequence array (s and dl/ds: uniform [B, T], ragged [sum T_b]) by sequence."""
    if prob.seq_T is None:
        return [x.reshape(-1) for x in a.reshape(prob.B, -1)]
    off = np.concatenate([[0], np.cumsum(prob.seq_T)])
    return [a[off[b]:off[b + 1]].reshape(-1) for b in range(prob.B)]


def _rel_parts(got, ref):
    return np.array([np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300) for g, r in zip(got, ref)])


def grad_errs(got, ref, prob):
    """Largest relative L2 error over the batch, per system for y, dl/dc, dl/dd and dl/du, and
    per sequence for dl/ds (which sums over the D systems of a sequence): a gradient wrong on
    one system is not diluted by the others.  got, ref: (y, gc, gd, gs, gu)."""
    S = prob.B * prob.D
    y, gc, gd, gs, gu = got[:5]
    yo, gco, gdo, gso, guo = ref[:5]
    return {"y": float(rel_err_per_system(y, yo, prob).max()),
            "gc": float(rel_err_per_system(gc, gco, prob).max()),
            "gd": float(rel_err_per_system(gd, gdo, prob).max()),
            "gs": float(_rel_parts(per_sequence(gs, prob), per_sequence(gso, prob)).max()),
            "gu": float(_rel_parts(list(gu.reshape(S, -1)), list(guo.reshape(S, -1))).max())}


def assert_grads(got, ref, prob, tol, gtol=None):
    """y within tol and every gradient within gtol (default tol), system by system."""
    e = grad_errs(got, ref, prob)
    gtol = tol if gtol is None else gtol
    assert e["y"] <= tol and max(e[k] for k in ("gc", "gd", "gs", "gu")) <= gtol, e
    return e
