"""Seeded synthetic inputs for the S-MNN batched solve.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic.  Both the oracle (tests, CPU baseline) and the CUDA path
(tests, bench) take their inputs from here, so both see identical bytes: every
generator draws in float64 from ``numpy.random.Generator(PCG64(seed))`` in a fixed
order, and ``Problem.cast`` rounds once to the working dtype; the oracle then gets
those rounded values promoted exactly to float64.

Workloads (one "system" = one (sequence b, dimension dd) pair, index i = b*D + dd;
the step sizes s are per sequence and shared by its D systems):

  config1   B=4,   D=2,  T=64,      R=2  -- FP64 forward solve
  config2   B=512, D=8,  T=1024,    R=2  -- FP32 refined forward + adjoint
  config3   B=1,   D=4,  T=2**20,   R=3, s~U[0.001,0.01]  (variant 3b: s~U[0.1,0.5])
  config4   4096 sequences, D=1, T_b = round(exp(U[ln 32, ln 65536])), R=2, ragged
  config5   B=256, D=32, T=8192,    R=2, c and d from a seeded 2-layer tanh MLP
            (width 128) applied to a sum of 8 sinusoids plus N(0, 0.05) noise

Coefficient generator (configs 1-4): c_{t,r} ~ N(0,1) with the leading coefficient
c_{t,R} = 1 + |N(0,1)|, d_t ~ N(0,1), s_t ~ U[lo, hi] per (sequence, step), initial
values u ~ N(0,1) for orders 0..R_init at step 1 (T_init = 1), unit weights.
"""
from __future__ import annotations

import math
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field, replace

import numpy as np

__all__ = ["Problem", "config1", "config2", "config2_slice", "config3", "config3b", "config4",
           "config5", "random_problem", "ragged_problem", "upstream_gradient", "mse_target", "CONFIGS",
           "table5_odes", "table5_batch", "ODE_T", "ODE_H", "random_coupled_problem",
           "LORENZ", "lorenz_trajectory", "lorenz_chunks"]


@dataclass
class Problem:
    """One batch of systems.  Uniform layout when ``seq_T`` is None:
    c [B, D, T, R+1], d [B, D, T], s [B, T], u [B, D, T_init, R_init+1].
    Ragged layout (``seq_T`` = int64 [B] steps per sequence): c [N, R+1], d [N], s [sum T_b],
    u [B*D, T_init, R_init+1], with N = D * sum T_b and the D systems of sequence b stored
    one after another (system i = b*D + dd starts at step D*sum_{b'<b} T_b' + dd*T_b)."""
    name: str
    R: int
    R_init: int
    T_init: int
    B: int
    D: int
    T: int | None
    c: np.ndarray
    d: np.ndarray
    s: np.ndarray
    u: np.ndarray
    seq_T: np.ndarray | None = None
    w_gov: float = 1.0
    w_init: float = 1.0
    w_smooth: float = 1.0
    meta: dict = field(default_factory=dict)
    V: int = 1   # variables per step (Sec. 3.1); c then holds Q*V*(R+1) values per step,
    Q: int = 1   # d holds Q, u holds V*(R_init+1) per initial step (variable-major)

    @property
    def S(self) -> int:
        return self.B * self.D

    @property
    def steps(self) -> int:
        """Time-steps solved per pass: sum over systems of T_i."""
        if self.seq_T is None:
            return self.B * self.D * self.T
        return int(self.D * np.sum(self.seq_T))

    def cast(self, dtype) -> "Problem":
        """The same problem with every array rounded once to ``dtype``."""
        return replace(self, c=self.c.astype(dtype), d=self.d.astype(dtype),
                       s=self.s.astype(dtype), u=self.u.astype(dtype))

    def as_f64(self) -> "Problem":
        return self.cast(np.float64)


def _coeffs(rng, shape_steps, R):
    c = rng.standard_normal(shape_steps + (R + 1,))
    c[..., R] = 1.0 + np.abs(c[..., R])
    return c


def random_problem(seed: int = 0, B: int = 4, D: int = 2, T: int = 64, R: int = 2,
                   R_init: int | None = None, T_init: int = 1, s_lo: float = 0.01,
                   s_hi: float = 0.1, name: str = "random", w=(1.0, 1.0, 1.0)) -> Problem:
    """Uniform batch with the coefficient generator above (draw order: c, d, s, u)."""
    if R_init is None:
        R_init = max(R - 1, 0)
    rng = np.random.Generator(np.random.PCG64(seed))
    c = _coeffs(rng, (B, D, T), R)
    d = rng.standard_normal((B, D, T))
    s = rng.uniform(s_lo, s_hi, (B, T))
    u = rng.standard_normal((B, D, T_init, R_init + 1))
    return Problem(name, R, R_init, T_init, B, D, T, c, d, s, u,
                   w_gov=w[0], w_init=w[1], w_smooth=w[2])


def ragged_problem(seq_T, D: int = 1, R: int = 2, seed: int = 5, s_lo: float = 0.01,
                   s_hi: float = 0.1) -> Problem:
    """Ragged batch (packed layout) with the coefficient generator above: sequence b has
    seq_T[b] steps; draw order c, d, s, u over the packed steps; R_init = R - 1, T_init = 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    seq_T = np.asarray(seq_T, np.int64)
    N = int(D * seq_T.sum())
    c = _coeffs(rng, (N,), R)
    d = rng.standard_normal(N)
    s = rng.uniform(s_lo, s_hi, int(seq_T.sum()))
    u = rng.standard_normal((len(seq_T) * D, 1, R))
    return Problem("ragged", R, R - 1, 1, len(seq_T), D, None, c, d, s, u, seq_T=seq_T)


def config1() -> Problem:
    return random_problem(0, 4, 2, 64, 2, name="config1: B=4 D=2 T=64 R=2 (FP64)")


def config2() -> Problem:
    return random_problem(0, 512, 8, 1024, 2, name="config2: B=512 D=8 T=1024 R=2")


def config2_slice() -> Problem:
    """The gradcheck slice of config 2: B=2, D=1, T=16."""
    return random_problem(0, 2, 1, 16, 2, name="config2 slice: B=2 D=1 T=16 R=2")


def config3(T: int = 1 << 20) -> Problem:
    return random_problem(0, 1, 4, T, 3, R_init=2, s_lo=0.001, s_hi=0.01,
                          name=f"config3: B=1 D=4 T={T} R=3 s~U[0.001,0.01]")


def config3b(T: int = 1 << 20) -> Problem:
    return random_problem(0, 1, 4, T, 3, R_init=2, s_lo=0.1, s_hi=0.5,
                          name=f"config3b: B=1 D=4 T={T} R=3 s~U[0.1,0.5]")


def config4(n_seq: int = 4096, T_lo: int = 32, T_hi: int = 65536, seed: int = 0) -> Problem:
    """Ragged batch: T_b = round(exp(U[ln T_lo, ln T_hi])), D = 1, packed with offsets.
    Draw order: T_b, then c, d, s, u over the packed steps."""
    rng = np.random.Generator(np.random.PCG64(seed))
    seq_T = np.rint(np.exp(rng.uniform(math.log(T_lo), math.log(T_hi), n_seq))).astype(np.int64)
    N = int(seq_T.sum())
    c = _coeffs(rng, (N,), 2)
    d = rng.standard_normal(N)
    s = rng.uniform(0.01, 0.1, N)
    u = rng.standard_normal((n_seq, 1, 2))
    return Problem(f"config4: {n_seq} ragged systems T in [{T_lo},{T_hi}] R=2", 2, 1, 1, n_seq, 1,
                   None, c, d, s, u, seq_T=seq_T)


def _mlp_apply(x: np.ndarray, W1, b1, W2, b2, block: int = 1 << 16) -> np.ndarray:
    """tanh MLP on a flat float32 vector of scalars -> [len(x), out] (float32)."""
    out = np.empty((x.shape[0], W2.shape[1]), np.float32)

    def work(lo):
        hi = min(lo + block, x.shape[0])
        h = np.tanh(x[lo:hi, None] * W1[None, :] + b1[None, :])
        out[lo:hi] = h @ W2 + b2[None, :]

    with ThreadPoolExecutor(max_workers=8) as ex:
        list(ex.map(work, range(0, x.shape[0], block)))
    return out


def config5(B: int = 256, D: int = 32, T: int = 8192, seed: int = 0) -> Problem:
    """Training-step shape.  Signal per (b, dd): sum of 8 sinusoids with amplitude
    ~U[0.1,1], frequency ~U[0.5,20] cycles over the sequence, phase ~U[0,2pi], on
    t_k = k/T, plus N(0, 0.05) noise.  A 2-layer MLP Linear(1,128)-tanh-Linear(128,4)
    with weights and biases ~U(-1/sqrt(fan_in), 1/sqrt(fan_in)) maps each sample to
    (c0, c1, c2_raw, d), and c2 = 1 + |c2_raw|.  s ~ U[0.01,0.1] and u ~ N(0,1) as in
    config 1.  Draw order: MLP (W1, b1, W2, b2), sinusoid parameters, noise, s, u."""
    R = 2
    rng = np.random.Generator(np.random.PCG64(seed))
    W1 = rng.uniform(-1.0, 1.0, 128)                     # fan_in 1
    b1 = rng.uniform(-1.0, 1.0, 128)
    k2 = 1.0 / math.sqrt(128.0)
    W2 = rng.uniform(-k2, k2, (128, R + 2))
    b2 = rng.uniform(-k2, k2, R + 2)
    amp = rng.uniform(0.1, 1.0, (B, D, 8))
    freq = rng.uniform(0.5, 20.0, (B, D, 8))
    phase = rng.uniform(0.0, 2 * math.pi, (B, D, 8))
    tgrid = np.arange(T, dtype=np.float64) / T
    x = np.zeros((B, D, T), np.float32)
    for b in range(B):
        arg = 2 * math.pi * freq[b, :, :, None] * tgrid[None, None, :] + phase[b, :, :, None]
        x[b] = np.sum(amp[b, :, :, None] * np.sin(arg), axis=1)
    x += rng.standard_normal((B, D, T), dtype=np.float32) * np.float32(0.05)
    out = _mlp_apply(x.reshape(-1), W1.astype(np.float32), b1.astype(np.float32),
                     W2.astype(np.float32), b2.astype(np.float32)).reshape(B, D, T, R + 2)
    c = out[..., :R + 1].astype(np.float64)
    c[..., R] = 1.0 + np.abs(c[..., R])
    d = out[..., R + 1].astype(np.float64)
    s = rng.uniform(0.01, 0.1, (B, T))
    u = rng.standard_normal((B, D, 1, 2))
    return Problem(f"config5: B={B} D={D} T={T} R=2 MLP coefficients", R, 1, 1, B, D, T, c, d, s, u)


def upstream_gradient(prob: Problem, seed: int = 2) -> np.ndarray:
    """A seeded dl/dy with the shape of y (N(0,1) entries), float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(prob.c.shape)


def mse_target(prob: Problem, seed: int = 1) -> np.ndarray:
    """Target tau ~ N(0,1) for the order-0 component, shape of d (config 2's loss)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(prob.d.shape)


CONFIGS = {"config1": config1, "config2": config2, "config3": config3, "config3b": config3b,
           "config4": config4, "config5": config5}


# ----------------------------------------------------------------------------- App. B.1 ODEs

ODE_T, ODE_H = 1000, 0.01   # Sec. 5.1 standalone setting: 1000 steps of 0.01


def table5_odes(T: int = ODE_T, h: float = ODE_H) -> list[dict]:
    """The six linear ODEs of App. B.1 with their closed-form solutions (Table 5's cases).

    Each case: name, order R of the solve (R = 2 for the first-order ODEs, whose Table 5
    columns include y''; R = 3 for the second- and third-order ones, the largest order the
    GPU path supports), R_init, coefficients c_0..c_R of sum_r c_r y^(r) = rhs, rhs, initial
    values u (orders 0..R_init at t = 0), and ``exact`` = [y, y', y''] on t_k = k h."""
    t = np.arange(T) * h
    out = []
    c0, c1, c2, u0 = 0.7, 1.2, 2.31, 10.0                 # RC circuit: y/c1 + c2 y' = c0
    k = 1.0 / (c1 * c2)
    a = u0 - c0 * c1
    out.append(dict(name="RC", R=2, coeffs=[1.0 / c1, c2, 0.0], rhs=c0, u=[u0],
                    exact=[c0 * c1 + a * np.exp(-k * t), -k * a * np.exp(-k * t),
                           k * k * a * np.exp(-k * t)]))
    c0, u0 = 0.23, 4.78                                   # population growth: c0 y - y' = 0
    out.append(dict(name="Population", R=2, coeffs=[c0, -1.0, 0.0], rhs=0.0, u=[u0],
                    exact=[u0 * np.exp(c0 * t) * c0 ** r for r in range(3)]))
    c0, c1, u0 = 0.32, 0.28, 0.14                         # language death: (c0+c1) y + y' = c0
    kk = c0 + c1
    A0 = c0 / kk
    out.append(dict(name="Language", R=2, coeffs=[kk, 1.0, 0.0], rhs=c0, u=[u0],
                    exact=[A0 - (A0 - u0) * np.exp(-kk * t), kk * (A0 - u0) * np.exp(-kk * t),
                           -kk * kk * (A0 - u0) * np.exp(-kk * t)]))
    c0 = 2.1                                              # harmonic oscillator: c0 y + y'' = 0
    u0, u1 = 0.4, -0.03
    wq = math.sqrt(c0)
    y0 = u0 * np.cos(wq * t) + u1 / wq * np.sin(wq * t)
    out.append(dict(name="Harmonic", R=3, coeffs=[c0, 0.0, 1.0, 0.0], rhs=0.0, u=[u0, u1],
                    exact=[y0, -u0 * wq * np.sin(wq * t) + u1 * np.cos(wq * t), -c0 * y0]))
    c0, c1 = 4.5, 0.43                                    # damped oscillator: c0 y + c1 y' + y'' = 0
    u0, u1 = 0.12, 0.043
    om = math.sqrt(4 * c0 - c1 ** 2) / 2
    lam = -c1 / 2 + 1j * om
    z = np.exp(lam * t) * (u0 - 1j * (c1 * u0 + 2 * u1) / (2 * om))   # y = Re z
    out.append(dict(name="Damped", R=3, coeffs=[c0, c1, 1.0, 0.0], rhs=0.0, u=[u0, u1],
                    exact=[np.real(z), np.real(lam * z), np.real(lam * lam * z)]))
    u0, u1, u2 = 0.0, -1.0, 1.0                           # third order: y' + y'' + y''' = 0
    lam = -0.5 + 1j * math.sqrt(3) / 2
    z = np.exp(lam * t) * (-(u1 + u2) - 1j * math.sqrt(3) / 3 * (u1 - u2))
    out.append(dict(name="ThirdOrder", R=3, coeffs=[0.0, 1.0, 1.0, 1.0], rhs=0.0, u=[u0, u1, u2],
                    exact=[u0 + u1 + u2 + np.real(z), np.real(lam * z), np.real(lam * lam * z)]))
    for cse in out:
        cse["R_init"] = len(cse["u"]) - 1
    return out


def table5_batch(R: int, R_init: int, T: int = ODE_T, h: float = ODE_H) -> tuple[Problem, list[dict]]:
    """The App. B.1 cases of order R with R_init + 1 initial values, as one uniform batch
    (one system per case, D = 1, constant step h, unit weights, T_init = 1)."""
    cases = [cse for cse in table5_odes(T, h) if cse["R"] == R and cse["R_init"] == R_init]
    B = len(cases)
    c = np.zeros((B, 1, T, R + 1))
    d = np.zeros((B, 1, T))
    u = np.zeros((B, 1, 1, R_init + 1))
    for b, cse in enumerate(cases):
        c[b, 0, :, :] = np.asarray(cse["coeffs"], float)[: R + 1]
        d[b, 0, :] = cse["rhs"]
        u[b, 0, 0, :] = cse["u"]
    s = np.full((B, T), h)
    return Problem(f"App. B.1 ODEs R={R}", R, R_init, 1, B, 1, T, c, d, s, u), cases


def random_coupled_problem(seed: int = 0, B: int = 2, D: int = 2, T: int = 64, R: int = 1,
                           V: int = 2, Q: int = 2, R_init: int | None = None, T_init: int = 1,
                           s_lo: float = 0.01, s_hi: float = 0.1, w=(1.0, 1.0, 1.0),
                           lead_cross: float | None = None) -> Problem:
    """Uniform batch of coupled systems (Sec. 3.1 with V variables and Q governing equations
    per step): c [B, D, T, Q*V*(R+1)] ~ N(0,1) with the coefficient of each equation's own
    variable's highest derivative (variable q mod V) set to 1 + |N(0,1)|, d [B, D, T, Q] ~ N(0,1),
    s ~ U[s_lo, s_hi] per (sequence, step), u [B, D, T_init, V*(R_init+1)] ~ N(0,1).
    Draw order: c, d, s, u.

    ``lead_cross``: if set, an equation's coefficients on the OTHER variables' highest
    derivatives become lead_cross * tanh(N) (same draws), so that with
    lead_cross <= 1 / (V - 1) the highest derivatives are pinned by a diagonally dominant
    block; left unset, those coefficients are plain N(0,1) and a step's block can come
    arbitrarily close to singular (the highest derivatives then rest on smoothness rows of
    weight s^{2R} alone)."""
    if R_init is None:
        R_init = max(R - 1, 0)
    nb = V * (R + 1)
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.standard_normal((B, D, T, Q, nb))
    for q in range(Q):
        k = (q % V) * (R + 1) + R
        c[..., q, k] = 1.0 + np.abs(c[..., q, k])
        if lead_cross is not None:
            for v in range(V):
                if v != q % V:
                    kv = v * (R + 1) + R
                    c[..., q, kv] = lead_cross * np.tanh(c[..., q, kv])
    d = rng.standard_normal((B, D, T, Q))
    s = rng.uniform(s_lo, s_hi, (B, T))
    u = rng.standard_normal((B, D, T_init, V * (R_init + 1)))
    return Problem(f"coupled: B={B} D={D} T={T} V={V} R={R} Q={Q}", R, R_init, T_init, B, D, T,
                   c.reshape(B, D, T, Q * nb),
                   d, s, u, w_gov=w[0], w_init=w[1], w_smooth=w[2], V=V, Q=Q)


# ----------------------------------------------------------------------------- Lorenz data

# Sec. 5.2: the standard Lorenz parameters, start (1, 1, 1), 10,000 samples 0.01 apart
LORENZ = dict(sigma=10.0, rho=28.0, beta=8.0 / 3.0, x0=(1.0, 1.0, 1.0), n_steps=10000, dt=0.01)


def lorenz_trajectory(n_steps: int = LORENZ["n_steps"], dt: float = LORENZ["dt"],
                      x0=LORENZ["x0"], sigma: float = LORENZ["sigma"], rho: float = LORENZ["rho"],
                      beta: float = LORENZ["beta"], substeps: int = 10) -> np.ndarray:
    """The Lorenz trajectory of Sec. 5.2 as [n_steps, 3] float64 samples dt apart (row 0 = x0).

    dx/dt = sigma (y - x), dy/dt = x (rho - z) - y, dz/dt = x y - beta z, integrated by the
    classical fourth-order Runge-Kutta method with ``substeps`` equal sub-steps per sample
    (a fixed-step stand-in for the adaptive integrator the paper names; deterministic, no
    random numbers)."""
    h = dt / substeps
    x, y, z = (float(v) for v in x0)
    out = np.empty((n_steps, 3))
    out[0] = (x, y, z)

    def f(x, y, z):
        return sigma * (y - x), x * (rho - z) - y, x * y - beta * z

    for i in range(1, n_steps):
        for _ in range(substeps):
            a1, b1, c1 = f(x, y, z)
            a2, b2, c2 = f(x + 0.5 * h * a1, y + 0.5 * h * b1, z + 0.5 * h * c1)
            a3, b3, c3 = f(x + 0.5 * h * a2, y + 0.5 * h * b2, z + 0.5 * h * c2)
            a4, b4, c4 = f(x + h * a3, y + h * b3, z + h * c3)
            x += h / 6.0 * (a1 + 2.0 * a2 + 2.0 * a3 + a4)
            y += h / 6.0 * (b1 + 2.0 * b2 + 2.0 * b3 + b4)
            z += h / 6.0 * (c1 + 2.0 * c2 + 2.0 * c3 + c4)
        out[i] = (x, y, z)
    return out


def lorenz_chunks(traj: np.ndarray, B: int, T: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """B random windows of T consecutive samples of ``traj`` (App. B.2's batches): returns
    (starts [B] int64, chunks [B, T, n]).  Start indices ~ U{0, ..., len(traj) - T}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    starts = rng.integers(0, traj.shape[0] - T + 1, B).astype(np.int64)
    return starts, traj[starts[:, None] + np.arange(T)[None, :]]
