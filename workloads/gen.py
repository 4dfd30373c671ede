"""Seeded inputs for the all-at-once system (I + tau K) U - U Sigma_1^T = G (eq. 2).

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) -> 53-bit uniforms in [0, 1) -> Box-Muller
normals.  Everything is plain Python/numpy so that the bytes are identical on
every host.

Layout of G and U: row-major (n_t, n_bar) float64 with the spatial index
contiguous; row j holds time t_{j+1} = (j+1) tau.  In 2D the spatial index is
iy * nx + ix (x fastest), matching K = I_ny (x) T_x + T_y (x) I_nx (Sec. 6.1).
Row 0 of G is u_0 + tau f_1 and row j >= 1 is tau f_{j+1} (eq. 2).

Spatial operators use second-order finite differences on (0, 1) with n
interior nodes, h = 1/(n+1) (Sec. 6.1) and homogeneous Dirichlet boundaries.
Tridiagonal coefficients are stored as three length-n arrays (lo, diag, up):
row i of K is lo[i] u[i-1] + diag[i] u[i] + up[i] u[i+1]; lo[0] and up[n-1]
are zero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_MASK = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 stream (Steele et al. 2014), one 64-bit output per call."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """53-bit uniform in [0, 1)."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)

    def normals(self, n: int, std: float = 1.0) -> np.ndarray:
        """Box-Muller pairs: r = sqrt(-2 ln(1-u1)), (r cos 2 pi u2, r sin 2 pi u2)."""
        out = np.empty(n, dtype=np.float64)
        i = 0
        while i < n:
            u1 = 1.0 - self.uniform()  # in (0, 1]
            u2 = self.uniform()
            r = math.sqrt(-2.0 * math.log(u1))
            out[i] = r * math.cos(2.0 * math.pi * u2)
            if i + 1 < n:
                out[i + 1] = r * math.sin(2.0 * math.pi * u2)
            i += 2
        return out * std

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in {lo, ..., hi}."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)

    def distinct_ints(self, count: int, lo: int, hi: int) -> list:
        if count > hi - lo + 1:
            raise ValueError("not enough distinct integers in range")
        got: list = []
        while len(got) < count:
            k = self.randint(lo, hi)
            if k not in got:
                got.append(k)
        return got


@dataclass
class Problem:
    """One instance of eq. (2): operator K, step tau, n_t steps, right-hand side G."""

    name: str
    dim: int
    nx: int
    ny: int
    nt: int
    T: float
    tau: float
    k_lo: np.ndarray
    k_diag: np.ndarray
    k_up: np.ndarray
    G: np.ndarray
    seed: int
    recipe: str
    k_lo_y: Optional[np.ndarray] = None
    k_diag_y: Optional[np.ndarray] = None
    k_up_y: Optional[np.ndarray] = None
    m_diag: Optional[np.ndarray] = None  # diagonal mass matrix (1D), None = identity
    extra: dict = field(default_factory=dict)

    @property
    def nbar(self) -> int:
        return self.nx * self.ny

    @property
    def unknowns(self) -> int:
        return self.nx * self.ny * self.nt


def _grid(n: int) -> np.ndarray:
    h = 1.0 / (n + 1)
    return h * np.arange(1, n + 1, dtype=np.float64)


def heat1d_operator(n: int):
    """K = tridiag(-1, 2, -1) / h^2, h = 1/(n+1) (Sec. 6.1, one axis)."""
    h = 1.0 / (n + 1)
    s = 1.0 / (h * h)
    lo = np.full(n, -s)
    up = np.full(n, -s)
    diag = np.full(n, 2.0 * s)
    lo[0] = 0.0
    up[-1] = 0.0
    return lo, diag, up


heat2d_axis_operator = heat1d_operator


def advdiff1d_operator(n: int, a: float, nu: float):
    """K for u_t + a u_x = nu u_xx: nu tridiag(-1,2,-1)/h^2 + (a/h) tridiag(-1,1,0).

    First-order upwind advection for a > 0 plus central diffusion; K is
    nonsymmetric tridiagonal.
    """
    h = 1.0 / (n + 1)
    d = nu / (h * h)
    lo = np.full(n, -d - a / h)
    diag = np.full(n, 2.0 * d + a / h)
    up = np.full(n, -d)
    lo[0] = 0.0
    up[-1] = 0.0
    return lo, diag, up


def advdiff1d_centred_operator(n: int, a: float, nu: float):
    """K for u_t + a u_x = nu u_xx with centred differences for both terms (the discretisation
    of the paper's Sec. 6.2 example, in 1D): nu tridiag(-1,2,-1)/h^2 + (a/(2h)) tridiag(-1,0,1).
    Weakly diagonally dominant exactly when the cell Peclet number |a| h / nu is at most 2."""
    h = 1.0 / (n + 1)
    d = nu / (h * h)
    lo = np.full(n, -d - a / (2.0 * h))
    diag = np.full(n, 2.0 * d)
    up = np.full(n, -d + a / (2.0 * h))
    lo[0] = 0.0
    up[-1] = 0.0
    return lo, diag, up


def build_rhs(u0: np.ndarray, f, tau: float, m_diag=None) -> np.ndarray:
    """Right-hand side G of the all-at-once system (eq. 2) from an initial value and a forcing.

    u0: (n_x,) initial value.  f: (n_t, n_x) forcing sampled at t_1..t_l (zeros for f = 0).
    tau: time step.
    m_diag: optional (n_x,) diagonal mass matrix.  Returns G with G_1 = M u0 + tau f_1 and
    G_j = tau f_j for j > 1, so that (M + tau K) u_j = M u_{j-1} + G_j with u_0 = 0 steps the
    scheme.  The right-hand side printed with eq. 4 drops the factor tau on f; eq. 2 carries it.
    """
    f = np.asarray(f, dtype=np.float64)
    if f.ndim != 2:
        raise ValueError("f must be (n_t, n_x)")
    u0 = np.asarray(u0, dtype=np.float64).reshape(-1)
    if u0.shape[0] != f.shape[1]:
        raise ValueError("u0 and f disagree on n_x")
    G = tau * f
    G[0] += u0 if m_diag is None else np.asarray(m_diag, dtype=np.float64) * u0
    return G


def heat1d_sine_modes(n: int = 127, nt: int = 64, T: float = 1.0, seed: int = 0,
                      modes: int = 8) -> Problem:
    """1D heat, f = 0, u0 = sin(pi x) + sum_q a_q sin(k_q pi x), a_q ~ N(0, 0.1).

    k_q are distinct, uniform in {2, ..., min(32, n)}.
    """
    rng = SplitMix64(seed)
    x = _grid(n)
    kmax = min(32, n)
    ks = rng.distinct_ints(min(modes, kmax - 1), 2, kmax)
    amps = rng.normals(len(ks), std=0.1)
    u0 = np.sin(np.pi * x)
    for a, k in zip(amps, ks):
        u0 = u0 + a * np.sin(k * np.pi * x)
    tau = T / nt
    lo, diag, up = heat1d_operator(n)
    G = np.zeros((nt, n))
    G[0] = u0
    return Problem(name=f"heat1d_sine_n{n}_nt{nt}", dim=1, nx=n, ny=1, nt=nt, T=T,
                   tau=tau, k_lo=lo, k_diag=diag, k_up=up, G=G, seed=seed,
                   recipe="1D heat, f=0, u0 = sin(pi x) + 8 seeded sine modes, a~N(0,0.1)",
                   extra={"modes": [1] + list(ks), "amps": [1.0] + list(amps)})


def heat1d_forced(n: int = 1023, nt: int = 1024, T: float = 1.0, seed: int = 0,
                  terms: int = 16) -> Problem:
    """1D heat, u0 = 0, f = sum_q a_q sin(k_q pi x) sin(p_q pi t), a_q ~ N(0,1).

    k_q uniform in {1..min(64, n)}, p_q uniform in {1..16}; G_j = tau f(., t_j).
    """
    rng = SplitMix64(seed)
    x = _grid(n)
    tau = T / nt
    t = tau * np.arange(1, nt + 1)
    kmax = min(64, n)
    amps = rng.normals(terms, std=1.0)
    ks = [rng.randint(1, kmax) for _ in range(terms)]
    ps = [rng.randint(1, 16) for _ in range(terms)]
    G = np.zeros((nt, n))
    for a, k, p in zip(amps, ks, ps):
        G += a * np.outer(np.sin(p * np.pi * t), np.sin(k * np.pi * x))
    G *= tau
    lo, diag, up = heat1d_operator(n)
    return Problem(name=f"heat1d_forced_n{n}_nt{nt}", dim=1, nx=n, ny=1, nt=nt, T=T,
                   tau=tau, k_lo=lo, k_diag=diag, k_up=up, G=G, seed=seed,
                   recipe="1D heat, u0=0, f = 16 seeded space-time sine modes, a~N(0,1)",
                   extra={"amps": list(amps), "k": ks, "p": ps})


def heat2d_smooth(n: int = 255, nt: int = 256, T: float = 0.1, seed: int = 0,
                  modes: int = 32) -> Problem:
    """2D heat on (0,1)^2, f = 0, u0 = sum_{k,l} a_kl/(k^2+l^2) sin(k pi x) sin(l pi y).

    a_kl ~ N(0,1) drawn with k outer, l inner, k, l = 1..min(32, n).
    """
    rng = SplitMix64(seed)
    x = _grid(n)
    M = min(modes, n)
    amps = rng.normals(M * M, std=1.0).reshape(M, M)
    kk = np.arange(1, M + 1)
    sx = np.sin(np.pi * np.outer(kk, x))  # (M, n) rows = k
    coef = amps / (kk[:, None] ** 2 + kk[None, :] ** 2)  # (k, l)
    # u0[iy, ix] = sum_{k,l} coef[k,l] sin(k pi x_ix) sin(l pi y_iy)
    u0 = sx.T @ coef @ sx  # (ix, iy)
    u0 = u0.T  # (iy, ix): x fastest
    tau = T / nt
    lo, diag, up = heat1d_operator(n)
    G = np.zeros((nt, n * n))
    G[0] = u0.reshape(-1)
    return Problem(name=f"heat2d_n{n}_nt{nt}", dim=2, nx=n, ny=n, nt=nt, T=T, tau=tau,
                   k_lo=lo.copy(), k_diag=diag.copy(), k_up=up.copy(),
                   k_lo_y=lo.copy(), k_diag_y=diag.copy(), k_up_y=up.copy(), G=G,
                   seed=seed,
                   recipe="2D heat, f=0, u0 = 32x32 seeded product sine modes, a/(k^2+l^2)")


def advdiff1d_pulse(n: int = 4095, nt: int = 2048, T: float = 1.0, seed: int = 0,
                    a: float = 1.0, nu: float = 1e-3) -> Problem:
    """1D advection-diffusion, f = 0, u0 = exp(-(x-0.3)^2 / (2 0.05^2)) + N(0, 1e-3)."""
    rng = SplitMix64(seed)
    x = _grid(n)
    u0 = np.exp(-((x - 0.3) ** 2) / (2 * 0.05 ** 2)) + rng.normals(n, std=1e-3)
    tau = T / nt
    lo, diag, up = advdiff1d_operator(n, a, nu)
    G = np.zeros((nt, n))
    G[0] = u0
    return Problem(name=f"advdiff1d_n{n}_nt{nt}", dim=1, nx=n, ny=1, nt=nt, T=T, tau=tau,
                   k_lo=lo, k_diag=diag, k_up=up, G=G, seed=seed,
                   recipe="1D adv-diff a=1 nu=1e-3 upwind, Gaussian pulse + N(0,1e-3) noise",
                   extra={"a": a, "nu": nu})


def advdiff1d_centred(n: int = 255, nt: int = 64, T: float = 1.0, peclet: float = 1.5, nu: float = 1e-2,
                      seed: int = 0) -> Problem:
    """1D advection-diffusion with centred advection at cell Peclet number `peclet`
    (a = peclet nu / h), f = 0, u0 = Gaussian pulse at x = 0.3 (std 0.05) + N(0, 1e-3) noise."""
    rng = SplitMix64(seed)
    h = 1.0 / (n + 1)
    a = peclet * nu / h
    lo, diag, up = advdiff1d_centred_operator(n, a, nu)
    x = _grid(n)
    u0 = np.exp(-((x - 0.3) ** 2) / (2 * 0.05 ** 2)) + rng.normals(n, 1e-3)
    tau = T / nt
    G = build_rhs(u0, np.zeros((nt, n)), tau)
    return Problem(name=f"advdiff1d_centred_n{n}_nt{nt}_pe{peclet:g}", dim=1, nx=n, ny=1, nt=nt, T=T, tau=tau,
                   k_lo=lo, k_diag=diag, k_up=up, G=G, seed=seed,
                   recipe=f"1D adv-diff, centred advection at cell Peclet {peclet:g}, nu={nu:g}, Gaussian pulse",
                   extra={"a": a, "nu": nu, "peclet": peclet})


def random_tridiag_problem(n: int, nt: int, T: float = 1.0, seed: int = 0,
                           symmetric: bool = False) -> Problem:
    """Random tridiagonal K with nonnegative diagonal dominance and random G ~ N(0,1).

    K = s * tri(lo, diag, up) with lo, up in -[0.2, 1.2], diag = |lo|+|up| + U(0.1, 1),
    s = (n+1)^2, so I + tau K is strictly diagonally dominant.  Used for ragged and
    degenerate sizes (n = 1, 2, 3, ...).
    """
    rng = SplitMix64(seed)
    s = float((n + 1) ** 2)
    lo = -(0.2 + rng.uniforms(n))
    up = lo.copy() if symmetric else -(0.2 + rng.uniforms(n))
    if symmetric:
        up = np.concatenate([lo[1:], [0.0]])
    lo[0] = 0.0
    up[-1] = 0.0
    diag = np.abs(lo) + np.abs(up) + 0.1 + 0.9 * rng.uniforms(n)
    G = rng.normals(nt * n).reshape(nt, n)
    return Problem(name=f"random_tridiag_n{n}_nt{nt}", dim=1, nx=n, ny=1, nt=nt, T=T,
                   tau=T / nt, k_lo=s * lo, k_diag=s * diag, k_up=s * up, G=G, seed=seed,
                   recipe="random diagonally dominant tridiagonal K, G ~ N(0,1)")


def with_mass(P: Problem, seed: int = 0, lo: float = 0.5, hi: float = 2.0) -> Problem:
    """A copy of the 1D problem P with a diagonal mass matrix, entries uniform in [lo, hi)
    (a lumped mass of a non-uniform mesh); G is kept as the right-hand side of
    (M + tau K) u_j = M u_{j-1} + G_j."""
    if P.dim != 1:
        raise ValueError("mass matrices are generated for 1D problems")
    rng = SplitMix64(seed)
    m = lo + (hi - lo) * rng.uniforms(P.nx)
    return Problem(name=f"{P.name}_mass{seed}", dim=1, nx=P.nx, ny=1, nt=P.nt, T=P.T, tau=P.tau,
                   k_lo=P.k_lo.copy(), k_diag=P.k_diag.copy(), k_up=P.k_up.copy(), G=P.G.copy(), seed=P.seed,
                   recipe=P.recipe + f"; diagonal mass matrix U[{lo}, {hi}) (seed {seed})", m_diag=m)


def heat1d_127x64(seed: int = 0) -> Problem:
    """1D heat, n_x = 127, n_t = 64, T = 1, f = 0, sine-mode u0 (FP64 everywhere)."""
    return heat1d_sine_modes(127, 64, 1.0, seed)


def heat1d_1023x1024(seed: int = 0) -> Problem:
    """1D heat, n_x = 1023, n_t = 1024, T = 1, 16 space-time sine-mode forcing terms."""
    return heat1d_forced(1023, 1024, 1.0, seed)


def heat2d_255x255x256(seed: int = 0) -> Problem:
    """2D heat, 255 x 255 interior grid, n_t = 256, T = 0.1, smooth random u0."""
    return heat2d_smooth(255, 256, 0.1, seed)


def advdiff1d_4095x2048(seed: int = 0) -> Problem:
    """1D advection-diffusion a = 1, nu = 1e-3, n_x = 4095, n_t = 2048, T = 1."""
    return advdiff1d_pulse(4095, 2048, 1.0, seed)


_BY_NAME = {f.__name__: f for f in (heat1d_127x64, heat1d_1023x1024, heat2d_255x255x256, advdiff1d_4095x2048)}


def by_name(name: str, seed: int = 0) -> Problem:
    return _BY_NAME[name](seed)
