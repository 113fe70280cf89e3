"""Governing-equation discovery through the S-MNN layer (Sec. 2's discovery example; the
Lorenz experiment of Sec. 5.2).

Every state variable v of an observed trajectory x_1..x_T is modelled as a first-order ODE

    y_v'(t) = d_v(t),   d_v(t) = sum_k Xi[v, k] phi_k(x_t),

with phi a polynomial library in the observed state.  In the layer's terms (Eq. 4-7, R = 1):
c puts coefficient 1 on the first derivative and 0 on y itself, the initial value of order
0 at the first step is the first observation (T_init = 1, R_init = 0), and s is the sample
spacing.  The loss is the mean squared difference between the order-0 solution and the
observations; Xi is learned by gradient descent through ``SmnnSolve``.

The state variables are independent systems here (D = n_state, one variable and one
equation per system): d depends on the observations, not on y, so the coupled form with
V = Q = n_state would have a block-diagonal M and separate into the same solves.

Features are divided by fixed scales (their root mean square over the training trajectory)
so that one learning rate suits every term; ``coefficients()`` returns Xi in the original
units.  ``GraphedTrainStep`` captures a whole optimisation step (window sampling, library,
solve, loss, adjoint, Adam update) in one CUDA graph.
"""
from __future__ import annotations

import itertools

import torch

from . import binding as B
from .api import SolveConfig, smnn_layer


def library_terms(n_state: int = 3, degree: int = 2, names: str = "xyz") -> list[tuple[int, ...]]:
    """Monomials of the library as tuples of state indices: () is the constant, (0,) is x,
    (0, 2) is x z, ...; all monomials of total degree <= ``degree``, by degree then index."""
    out: list[tuple[int, ...]] = [()]
    for k in range(1, degree + 1):
        out += list(itertools.combinations_with_replacement(range(n_state), k))
    return out


def term_name(term: tuple[int, ...], names: str = "xyz") -> str:
    return "1" if not term else "".join(names[i] for i in term)


def library(x: torch.Tensor, terms) -> torch.Tensor:
    """phi(x): [..., n_state] -> [..., len(terms)]."""
    cols = []
    for term in terms:
        if not term:
            cols.append(torch.ones_like(x[..., 0]))
        else:
            v = x[..., term[0]]
            for i in term[1:]:
                v = v * x[..., i]
            cols.append(v)
    return torch.stack(cols, dim=-1)


class Discovery(torch.nn.Module):
    """Learnable library coefficients for an n_state-dimensional first-order system.

    forward(x) with x [B, T, n_state] (observations at spacing dt) returns (loss, y, info):
    y [B, n_state, T, 2] the layer's solution (order 0 and 1), info [B * n_state]."""

    def __init__(self, n_state: int = 3, degree: int = 2, dt: float = 0.01, scale=None,
                 cfg: SolveConfig | None = None, dtype=torch.float32, device="cuda"):
        super().__init__()
        self.n_state, self.dt = n_state, float(dt)
        self.terms = library_terms(n_state, degree)
        K = len(self.terms)
        self.cfg = cfg if cfg is not None else SolveConfig(R_init=0, T_init=1)
        if self.cfg.R_init != 0 or self.cfg.T_init != 1 or self.cfg.V != 1 or self.cfg.Q != 1:
            raise ValueError("discovery uses R_init = 0, T_init = 1 and one variable per system")
        if self.cfg.precision == B.F64:
            dtype = torch.float64
        self.xi = torch.nn.Parameter(torch.zeros(n_state, K, dtype=dtype, device=device))
        sc = torch.ones(K, dtype=dtype) if scale is None else torch.as_tensor(scale, dtype=dtype)
        self.register_buffer("scale", sc.to(device))
        self._static: dict = {}

    @staticmethod
    def feature_scale(traj: torch.Tensor, terms) -> torch.Tensor:
        """Root mean square of each library term over a trajectory [N, n_state]."""
        return library(traj.double(), terms).pow(2).mean(0).sqrt()

    def coefficients(self) -> torch.Tensor:
        """Xi in the units of the unscaled library: [n_state, K]."""
        return (self.xi / self.scale).detach()

    def _constants(self, Bn: int, T: int, device):
        key = (Bn, T, str(device))
        hit = self._static.get(key)
        if hit is None:
            dt = self.xi.dtype
            c = torch.zeros(Bn, self.n_state, T, 2, dtype=dt, device=device)
            c[..., 1] = 1.0
            s = torch.full((Bn, T), self.dt, dtype=dt, device=device)
            hit = self._static[key] = (c, s)
        return hit

    def forward(self, x: torch.Tensor):
        Bn, T, n = x.shape
        c, s = self._constants(Bn, T, x.device)
        phi = library(x, self.terms) / self.scale                        # [B, T, K]
        d = torch.einsum("btk,vk->bvt", phi, self.xi).contiguous()        # [B, n, T]
        u = x[:, 0, :].reshape(Bn, n, 1, 1).contiguous()
        y, info = smnn_layer(c, d, s, u, self.cfg)
        loss = (y[..., 0] - x.transpose(1, 2)).pow(2).mean()
        return loss, y, info


class GraphedTrainStep:
    """One optimisation step of ``Discovery`` on B random windows of T samples of a
    device-resident trajectory, captured in a CUDA graph (``step()`` replays it).

    Each replay draws new window starts on the device (torch's generator, graph-safe),
    gathers the windows, runs forward, loss, adjoint and Adam (capturable) without a host
    synchronisation.  With ``resample=False`` the windows stay those of ``starts``.  The
    warm-up steps that precede the capture are undone (parameters and Adam state restored),
    so replay k is optimisation step k from the model's state at construction.  With
    ``graphed=False`` ``step()`` runs the same body eagerly instead."""

    def __init__(self, model: Discovery, traj: torch.Tensor, Bn: int, T: int, lr: float = 1e-2,
                 starts: torch.Tensor | None = None, resample: bool = True, warmup: int = 3,
                 graphed: bool = True):
        self.model, self.Bn, self.T, self.resample = model, Bn, T, resample
        dev = traj.device
        self.traj = traj.to(model.xi.dtype).contiguous()
        self.n_start = traj.shape[0] - T + 1
        if self.n_start < 1:
            raise ValueError("trajectory shorter than one window")
        self.offs = torch.arange(T, device=dev)
        self.starts = (torch.zeros(Bn, dtype=torch.int64, device=dev) if starts is None
                       else starts.to(dev, torch.int64).clone())
        self.opt = torch.optim.Adam(model.parameters(), lr=lr, capturable=True)
        self.loss = torch.zeros((), dtype=model.xi.dtype, device=dev)
        self.bad = torch.zeros((), dtype=torch.int32, device=dev)
        params0 = [p.detach().clone() for p in model.parameters()]
        starts0 = self.starts.clone()
        side = torch.cuda.Stream(device=dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            for _ in range(max(warmup, 1)):
                self._body()
        torch.cuda.current_stream(dev).wait_stream(side)
        self.graph = None
        if graphed:
            self.graph = torch.cuda.CUDAGraph()
            self.opt.zero_grad(set_to_none=True)
            with torch.cuda.graph(self.graph):
                self._body()
        with torch.no_grad():   # undo the warm-up steps
            for p, p0 in zip(model.parameters(), params0):
                p.copy_(p0)
                if p.grad is not None:
                    p.grad.zero_()
            for st in self.opt.state.values():
                for v in st.values():
                    if torch.is_tensor(v):
                        v.zero_()
            self.starts.copy_(starts0)

    def _body(self):
        if self.resample:
            self.starts.random_(0, self.n_start)
        x = self.traj[self.starts[:, None] + self.offs[None, :]]
        loss, _, info = self.model(x)
        loss.backward()
        self.opt.step()
        self.opt.zero_grad(set_to_none=False)
        self.loss.copy_(loss.detach())
        self.bad.copy_((info != 0).sum())

    def step(self):
        if self.graph is not None:
            self.graph.replay()
        else:
            self._body()
