"""Seeded request streams for the solver service (the serving workload).

Each request is one all-at-once backward-Euler problem (eq. 2):
- kind: 1D heat, 1D advection-diffusion (a = 1, upwind), or 2D heat;
- n_x uniform in {127..4095} (2D: grid side in {63, 127, 255}, the sides this build's DST
  accepts);
- n_t a power of two in {32..2048}, T = 1;
- diffusion nu log-uniform in [1e-4, 1];
- forcing of 16 space-time sine modes with N(0, 1) amplitudes, as in the 1D heat workload heat1d_1023x1024 (2D: a
  product sine in x and y);
- arrival times of a Poisson process of the given rate.

A request carries only these parameters.  Its right-hand side G is synthesised from
them, by `request_problem` (numpy, for the oracle) or by `rhs_device` (torch on the
GPU, for the server): the same formulas in both.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional

import numpy as np

from .gen import Problem, SplitMix64, _grid, advdiff1d_operator, heat1d_operator

KINDS = ("heat1d", "advdiff1d", "heat2d")
SIDES_2D = (63, 127, 255)


@dataclass
class Request:
    rid: int
    arrival: float  # seconds after the start of the stream
    kind: str
    nx: int
    ny: int
    nt: int
    nu: float
    seed: int
    T: float = 1.0
    # filled in by the server
    start: Optional[float] = None
    done: Optional[float] = None
    batch: int = 0
    joined_running: bool = False  # admitted into a batch that was already being solved
    error: Optional[str] = None
    result: Optional[np.ndarray] = None  # final state u_l (n_x * n_y), when kept

    @property
    def dim(self) -> int:
        return 2 if self.kind == "heat2d" else 1

    @property
    def tau(self) -> float:
        return self.T / self.nt

    @property
    def unknowns(self) -> int:
        return self.nx * self.ny * self.nt


def request_stream(n: int, rate: float, seed: int = 0, kinds=KINDS, nx_range=(127, 4095),
                   nt_choices=(32, 64, 128, 256, 512, 1024, 2048), sides_2d=SIDES_2D) -> list:
    """n requests with exponential inter-arrival times of mean 1/rate seconds."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += -math.log(1.0 - rng.uniform()) / rate
        kind = kinds[rng.randint(0, len(kinds) - 1)]
        if kind == "heat2d":
            nx = ny = sides_2d[rng.randint(0, len(sides_2d) - 1)]
        else:
            nx, ny = rng.randint(nx_range[0], nx_range[1]), 1
        nt = nt_choices[rng.randint(0, len(nt_choices) - 1)]
        nu = 10.0 ** (-4.0 + 4.0 * rng.uniform())
        out.append(Request(rid=i, arrival=t, kind=kind, nx=nx, ny=ny, nt=nt, nu=nu,
                           seed=int(rng.next_u64() & 0x7FFFFFFF)))
    return out


def operator(req: Request):
    """(lo, diag, up) of K, and of T_y in 2D (K = I (x) T_x + T_y (x) I)."""
    if req.kind == "advdiff1d":
        return advdiff1d_operator(req.nx, 1.0, req.nu), None
    lo, di, up = heat1d_operator(req.nx)
    kx = (req.nu * lo, req.nu * di, req.nu * up)
    if req.kind == "heat1d":
        return kx, None
    lo, di, up = heat1d_operator(req.ny)
    return kx, (req.nu * lo, req.nu * di, req.nu * up)


def forcing(req: Request, terms: int = 16):
    """Amplitudes a_q ~ N(0, 1) and integer wave numbers (k_q, l_q, p_q)."""
    rng = SplitMix64(req.seed)
    amps = rng.normals(terms, std=1.0)
    ks = [rng.randint(1, min(64, req.nx)) for _ in range(terms)]
    ls = [rng.randint(1, min(64, req.ny)) for _ in range(terms)]
    ps = [rng.randint(1, 16) for _ in range(terms)]
    return amps, ks, ls, ps


def request_problem(req: Request) -> Problem:
    """The request as a workloads.Problem with G in host memory (numpy)."""
    amps, ks, ls, ps = forcing(req)
    x = _grid(req.nx)
    t = req.tau * np.arange(1, req.nt + 1)
    y = _grid(req.ny) if req.dim == 2 else None
    G = np.zeros((req.nt, req.nx * req.ny))
    for a, k, l, p in zip(amps, ks, ls, ps):
        sx = np.sin(k * np.pi * x)
        space = np.outer(np.sin(l * np.pi * y), sx).reshape(-1) if req.dim == 2 else sx
        G += a * np.outer(np.sin(p * np.pi * t), space)
    G *= req.tau
    kx, ky = operator(req)
    P = Problem(name=f"req{req.rid}_{req.kind}", dim=req.dim, nx=req.nx, ny=req.ny, nt=req.nt, T=req.T,
                tau=req.tau, k_lo=kx[0], k_diag=kx[1], k_up=kx[2], G=G, seed=req.seed,
                recipe="serving request: 16 seeded space-time sine modes, nu log-uniform")
    if ky is not None:
        P.k_lo_y, P.k_diag_y, P.k_up_y = ky
    return P


def rhs_device(req: Request, torch, device, out=None):
    """G of `request_problem` built on the device with torch (same formulas), written
    into out[:, :n_x n_y] when out (nt, >= n_x n_y) is given."""
    amps, ks, ls, ps = forcing(req)
    f64 = torch.float64
    x = (torch.arange(1, req.nx + 1, dtype=f64, device=device)) / (req.nx + 1)
    t = req.tau * torch.arange(1, req.nt + 1, dtype=f64, device=device)
    y = (torch.arange(1, req.ny + 1, dtype=f64, device=device)) / (req.ny + 1) if req.dim == 2 else None
    # G = tau * S_t^T diag(a) S_x: one small matrix product over the 16 terms
    st = torch.stack([torch.sin(p * math.pi * t) for p in ps], dim=1)  # (nt, terms)
    cols = []
    for k, l in zip(ks, ls):
        sx = torch.sin(k * math.pi * x)
        cols.append(torch.outer(torch.sin(l * math.pi * y), sx).reshape(-1) if req.dim == 2 else sx)
    sp = torch.stack(cols, dim=0) * torch.tensor(amps, dtype=f64, device=device)[:, None]
    G = (st @ sp) * req.tau
    if out is None:
        return G
    out[:, : G.shape[1]].copy_(G)
    return out


@dataclass
class SlotOperator:
    """The operator fields of a problem (no right-hand side), for batched plans; 2D slots
    also carry T_y."""

    dim: int
    nx: int
    nt: int
    tau: float
    k_lo: np.ndarray
    k_diag: np.ndarray
    k_up: np.ndarray
    ny: int = 1
    k_lo_y: Optional[np.ndarray] = None
    k_diag_y: Optional[np.ndarray] = None
    k_up_y: Optional[np.ndarray] = None


def request_problem_operator_only(req: Request, slot_nx: int) -> SlotOperator:
    if req.dim == 2:  # 2D slots are the request's own grid
        if req.nx != slot_nx:
            raise ValueError("a 2D request of the slot's grid is needed")
        (lo, di, up), (ylo, ydi, yup) = operator(req)
        return SlotOperator(2, req.nx, req.nt, req.tau, lo, di, up, req.ny, ylo, ydi, yup)
    if req.nx > slot_nx:
        raise ValueError("a 1D request no longer than the slot is needed")
    (lo, di, up), _ = operator(req)
    return SlotOperator(1, req.nx, req.nt, req.tau, lo, di, up)


def empty_slot(nt: int, nx: int = 1, ny: int = 1) -> SlotOperator:
    """An unused slot of a batch, zero right-hand side: one decoupled row (1D), or the 2D
    heat operator on the batch's grid (2D: ny > 1)."""
    if ny > 1:
        lo, di, up = heat1d_operator(nx)
        ylo, ydi, yup = heat1d_operator(ny)
        return SlotOperator(2, nx, nt, 1.0 / nt, lo, di, up, ny, ylo, ydi, yup)
    return SlotOperator(1, 1, nt, 1.0 / nt, np.zeros(1), np.ones(1), np.zeros(1))
