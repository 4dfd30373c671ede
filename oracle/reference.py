"""FP64 CPU oracle for the new ParaDiag method (Gander & Palitta, arXiv 2304.12597).

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in __graft_entry__ and
the CPU-baseline leg of bench.py may import this module.  It shares no code
with the CUDA path; the two meet only in the seeded inputs of `workloads`.

What each function follows (paper sections/equations):

* ``be_solve``          eq. (2) by its plain definition: sequential backward Euler
                        (C routines in be_oracle.c).  ParaDiag with alpha = 1 and
                        exact inner solves reaches exactly this solution.  With a
                        diagonal mass matrix M (``problem.m_diag``) each step solves
                        (M + tau K) u_j = M u_{j-1} + G_j, the all-at-once system
                        (B (x) M + I (x) K) u = f of the method's general form.
* ``be_solve_refined``  ``be_solve`` plus one correction on its extended-precision
                        residual (the reference for FP64 comparisons).
* ``aao_apply``         left-hand side of eq. (2), (I + tau K) U - U Sigma_1^T (M in place
                        of I when the problem has a mass matrix).
* ``sigma1``, ``c_alpha``  Sigma_1 and the (alpha-)circulant C_alpha, eqs. (3), (15).
* ``dft_matrix``        F, F_{jk} = omega^{(j-1)(k-1)}, omega = exp(-2 pi i / l)
                        (appendix, proof of Theorem 3.1).
* ``circulant_eigs``    pi = F C_1 e_1 and gamma = F^{-T} e_l (Algorithm 1, first step).
* ``dft_time``/``idft_time``  U F^T and U F^{-T} along time (eq. 5, Sec. 2 end).
* ``paradiag``          Algorithm 1: parallel-in-time solves, b = L F^{-T} e_l (eq. 7),
                        Algorithm 2 for eq. (8), correction W, U = (L - W) F^{-T}.
* ``fom_like``          Algorithm 2 with the Arnoldi relation (10), the shifted
                        relation (11), the projected system (12) and residual (13).
* ``j_dense``           J_l of eq. (8), formed densely (tiny sizes only).
* ``periodic_solve_dense``  P^{-1} of Sec. 2 mapped back to time: the circulant
                        all-at-once system (I + tau K) U - U C_1^T = R.
* ``kappa_bound``       eq. (14), Theorem 3.1.
* ``alpha_quantities``, ``paradiag_alpha``, ``j_alpha_dense``  Algorithm 3 and
                        eqs. (15)-(17) (alpha-circulant C_alpha, scaled DFT), with
                        the U_1 early exit and the fixed-loop variants of Table 3.
* ``j_extreme_eigs``    the extreme eigenvalues of J_l for SPD K (Sec. 6.1).

Readings of points where the paper is silent or inconsistent:

1. eq. (11)-(13) and Algorithm 2 write t_{m+1,m} where the shifted Arnoldi
   relation for (1 - pi_i) I + tau K carries tau * t_{m+1,m}; the factor tau is
   kept here.  (Without it eq. (13) does not equal the explicit residual.)
2. The residual-norm line of Algorithm 2 omits gamma_i; eq. (13) has it: kept.
3. Algorithm 2 starts with ||r|| = 1; here ||r|| starts at beta = ||b||, the
   residual of x_0 = 0, so that at least one iteration runs whenever b != 0.
4. Breakdown t_{m+1,m} ~ 0 (silent in the paper): K_m(K, b) is invariant, the
   t-term of eq. (12) vanishes, the residual is zero and the iteration stops.
5. U = Re((L - W) F^{-T}); the imaginary part is roundoff for real data.
6. Frozen residual (q > 1, Sec. 3): the paper checks only at m mod q = 0; a step
   also checks at m = maxit and at a breakdown, so a run always ends on a checked
   step and x_m = V_m y_m uses that step's y_m.
7. Fixed-loop variants (Sec. 6, Table 3): two loops take x_m = b (the inner matrix
   of eq. (17) replaced by the identity); one loop returns U_1.
"""
from __future__ import annotations

import numpy as np

from . import native

# ----------------------------------------------------------------------------
# Operators (the problem definition; built independently of the CUDA path)
# ----------------------------------------------------------------------------


class TridiagOp:
    """Tridiagonal real K given by (lo, diag, up); row i = lo[i], diag[i], up[i]."""

    def __init__(self, lo, diag, up):
        self.lo = np.asarray(lo, dtype=np.float64)
        self.diag = np.asarray(diag, dtype=np.float64)
        self.up = np.asarray(up, dtype=np.float64)
        self.n = self.diag.size

    def matvec(self, v):
        w = self.diag * v
        w[1:] += self.lo[1:] * v[:-1]
        w[:-1] += self.up[:-1] * v[1:]
        return w

    def dense(self):
        n = self.n
        K = np.diag(self.diag)
        if n > 1:
            K += np.diag(self.lo[1:], -1) + np.diag(self.up[:-1], 1)
        return K

    def shifted_solve(self, s, tau, r):
        """((s) I + tau K)^{-1} r, complex shift s."""
        return native.shifted_tridiag_solve(s, tau, self.lo, self.diag, self.up,
                                            np.asarray(r, dtype=np.complex128))


class DenseOp:
    """Any real K held densely (used for the 2D operator at tiny sizes)."""

    def __init__(self, K):
        self.K = np.asarray(K, dtype=np.float64)
        self.n = self.K.shape[0]

    def matvec(self, v):
        return self.K @ v

    def dense(self):
        return self.K

    def shifted_solve(self, s, tau, r):
        return np.linalg.solve(s * np.eye(self.n) + tau * self.K, np.asarray(r, dtype=np.complex128))


def k_dense(problem):
    """K of the problem as a dense matrix.  2D: K = I (x) T_x + T_y (x) I (Sec. 6.1)."""
    Tx = TridiagOp(problem.k_lo, problem.k_diag, problem.k_up).dense()
    if problem.dim == 1:
        return Tx
    Ty = TridiagOp(problem.k_lo_y, problem.k_diag_y, problem.k_up_y).dense()
    return np.kron(np.eye(problem.ny), Tx) + np.kron(Ty, np.eye(problem.nx))


def k_band(problem):
    """Row-major band storage of K (kl = ku = 1 in 1D, nx in 2D, x fastest)."""
    nx, ny = problem.nx, problem.ny
    if problem.dim == 1:
        B = np.zeros((nx, 3))
        B[:, 0] = problem.k_lo
        B[:, 1] = problem.k_diag
        B[:, 2] = problem.k_up
        B[0, 0] = 0.0
        B[-1, 2] = 0.0
        return 1, 1, B
    n = nx * ny
    w = 2 * nx + 1
    B = np.zeros((n, w))
    for iy in range(ny):
        for ix in range(nx):
            i = iy * nx + ix
            B[i, nx] = problem.k_diag[ix] + problem.k_diag_y[iy]
            if ix > 0:
                B[i, nx - 1] = problem.k_lo[ix]
            if ix < nx - 1:
                B[i, nx + 1] = problem.k_up[ix]
            if iy > 0:
                B[i, 0] = problem.k_lo_y[iy]
            if iy < ny - 1:
                B[i, 2 * nx] = problem.k_up_y[iy]
    return nx, nx, B


def operator(problem, dense_limit: int = 4096):
    if problem.dim == 1:
        return TridiagOp(problem.k_lo, problem.k_diag, problem.k_up)
    if problem.nbar > dense_limit:
        raise ValueError("2D oracle operator is dense; use a small grid")
    return DenseOp(k_dense(problem))


# ----------------------------------------------------------------------------
# eq. (2): definition and sequential solution
# ----------------------------------------------------------------------------


def be_solve(problem, G=None, mdiag=None):
    """Exact solution of eq. (2): sequential backward Euler, u_0 := 0, G_1 = u0 + tau f_1
    (G_1 = M u0 + tau f_1 with a mass matrix)."""
    G = problem.G if G is None else G
    if mdiag is None:
        mdiag = getattr(problem, "m_diag", None)
    if problem.dim == 1:
        return native.be_tridiag(problem.tau, problem.k_lo, problem.k_diag, problem.k_up, G, mdiag)
    kl, ku, B = k_band(problem)
    return native.be_banded(problem.tau, kl, ku, B, G, mdiag)


def residual_extended(problem, U, G=None):
    """G - [(I + tau K) U - U Sigma_1^T] (eq. 2) with every operation in numpy.longdouble
    (64-bit mantissa on x86-64, IEEE quad on aarch64), rounded to float64 at the end."""
    L = np.longdouble
    G = problem.G if G is None else G
    Ul = np.asarray(U, dtype=np.float64).astype(L)
    nt = Ul.shape[0]
    if problem.dim == 1:
        KU = problem.k_diag.astype(L)[None, :] * Ul
        KU[:, 1:] += problem.k_lo[1:].astype(L)[None, :] * Ul[:, :-1]
        KU[:, :-1] += problem.k_up[:-1].astype(L)[None, :] * Ul[:, 1:]
    else:
        nx, ny = problem.nx, problem.ny
        X = Ul.reshape(nt, ny, nx)
        KU = (problem.k_diag.astype(L)[None, None, :] + problem.k_diag_y.astype(L)[None, :, None]) * X
        KU[:, :, 1:] += problem.k_lo[1:].astype(L)[None, None, :] * X[:, :, :-1]
        KU[:, :, :-1] += problem.k_up[:-1].astype(L)[None, None, :] * X[:, :, 1:]
        KU[:, 1:, :] += problem.k_lo_y[1:].astype(L)[None, :, None] * X[:, :-1, :]
        KU[:, :-1, :] += problem.k_up_y[:-1].astype(L)[None, :, None] * X[:, 1:, :]
        KU = KU.reshape(nt, -1)
    md = getattr(problem, "m_diag", None)
    MU = Ul if md is None else np.asarray(md, dtype=np.float64).astype(L)[None, :] * Ul
    Rl = np.asarray(G, dtype=np.float64).astype(L) - (MU + L(problem.tau) * KU)
    Rl[1:] += MU[:-1]
    return Rl.astype(np.float64)


def be_solve_refined(problem, G=None):
    """be_solve plus one correction solve on its extended-precision residual.

    The sequential solve is backward stable, so its forward error is bounded by
    about kappa(all-at-once operator) * eps; one refinement step with a residual
    carried in extended precision removes most of it.  This is the reference for
    FP64 comparisons on ill-conditioned workloads (e.g. 2D heat with T = 0.1,
    where the plain FP64 oracle is off by ~2e-12 relative)."""
    U = be_solve(problem, G)
    r = residual_extended(problem, U, G)
    return U + be_solve(problem, G=r)


def aao_apply(problem, U):
    """(I + tau K) U - U Sigma_1^T of eq. (2) in the row layout (row j = u_{j+1}).

    Column j of U Sigma_1^T is u_{j-1} (Sigma_1 has ones on the first
    subdiagonal, eq. 3), and u_0 contributes nothing.
    """
    U = np.asarray(U, dtype=np.float64)
    tau = problem.tau
    if problem.dim == 1:
        op = TridiagOp(problem.k_lo, problem.k_diag, problem.k_up)
        KU = np.stack([op.matvec(u) for u in U])
    else:
        nx, ny = problem.nx, problem.ny
        X = U.reshape(U.shape[0], ny, nx)
        KU = problem.k_diag[None, None, :] * X + problem.k_diag_y[None, :, None] * X
        KU[:, :, 1:] += problem.k_lo[None, None, 1:] * X[:, :, :-1]
        KU[:, :, :-1] += problem.k_up[None, None, :-1] * X[:, :, 1:]
        KU[:, 1:, :] += problem.k_lo_y[None, 1:, None] * X[:, :-1, :]
        KU[:, :-1, :] += problem.k_up_y[None, :-1, None] * X[:, 1:, :]
        KU = KU.reshape(U.shape)
    md = getattr(problem, "m_diag", None)
    MU = U if md is None else np.asarray(md, dtype=np.float64)[None, :] * U
    R = MU + tau * KU
    R[1:] -= MU[:-1]
    return R


def sigma1(ell):
    """Sigma_1: zeros with ones on the first subdiagonal (eq. 3)."""
    return np.eye(ell, k=-1)


def c_alpha(ell, alpha=1.0):
    """C_alpha = Sigma_1 + alpha e_1 e_l^T (eq. 15; alpha = 1 gives C_1 of eq. 3)."""
    C = sigma1(ell)
    C[0, ell - 1] = alpha
    return C


# ----------------------------------------------------------------------------
# Fourier quantities (Sec. 2 and the appendix)
# ----------------------------------------------------------------------------


def dft_matrix(ell):
    """F with F_{jk} = omega^{jk} (0-based), omega = exp(-2 pi i / l).  Exponents are
    reduced mod l before the exponential so every entry is an exact root of unity."""
    j = np.arange(ell)
    e = np.outer(j, j) % ell
    return np.exp(-2j * np.pi * e / ell)


def circulant_eigs(ell):
    """Algorithm 1, first step: pi = F C_1 e_1 and gamma = F^{-T} e_l."""
    F = dft_matrix(ell)
    pi = F @ c_alpha(ell, 1.0)[:, 0]
    e_ell = np.zeros(ell)
    e_ell[-1] = 1.0
    gamma = np.linalg.solve(F.T, e_ell.astype(np.complex128))
    return pi, gamma


def dft_time(X):
    """Row layout of U F^T: hat X[k] = sum_j omega^{jk} X[j] (forward DFT along time)."""
    X = np.asarray(X)
    return dft_matrix(X.shape[0]) @ X


def idft_time(Xhat):
    """Row layout of Y F^{-T}: F^{-1} Y (F is symmetric)."""
    Xhat = np.asarray(Xhat)
    return np.linalg.solve(dft_matrix(Xhat.shape[0]), Xhat)


# ----------------------------------------------------------------------------
# Algorithm 2 (FOM-like method for eq. 8)
# ----------------------------------------------------------------------------


def fom_like(op, tau, b, pi, gamma, eps=1e-8, maxit=50, q=1, breakdown_tol=1e-14,
             keep_tau=True, keep_gamma_in_residual=True, weight=1.0):
    """Algorithm 2 for J_l x = b with J_l = I + sum_i gamma_i ((1-pi_i) I + tau K)^{-1}.

    ``weight`` = alpha^{1/l} gives the variant Algorithm 3 applies to
    I + alpha^{1/l} sum_i gamma_i ((1-pi_i) I + tau K)^{-1} (eq. 17): the weight
    multiplies the sum in the projected system (12) and in the residual (13).

    Krylov space K_m(K, b) (eq. 9), Arnoldi by modified Gram-Schmidt (eq. 10).
    Every q iterations: h_i = ((1-pi_i) I + tau K)^{-1} v_{m+1},
    S_i = ((1-pi_i) I_m + tau T_m)^{-1}, y_m from eq. (12), ||r_m|| from eq. (13).
    Returns (x_m, info) with info = dict(m, y, resnorms, breakdown, T, V).
    ``keep_tau``/``keep_gamma_in_residual`` exist only so tests can show that the
    literal (tau-less / gamma-less) forms disagree with the explicit residual.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    ell = pi.size
    beta = float(np.linalg.norm(b))
    info = {"m": 0, "y": np.zeros(0), "resnorms": [], "breakdown": False, "beta": beta}
    if beta == 0.0:
        return np.zeros(n), info
    V = np.zeros((maxit + 1, n))
    T = np.zeros((maxit + 1, maxit))
    V[0] = b / beta
    m = 0
    r = beta
    y = None
    tfac = tau if keep_tau else 1.0
    while r > eps * beta and m < maxit:
        m += 1
        w = op.matvec(V[m - 1])
        wnorm0 = float(np.linalg.norm(w))
        for k in range(m):
            T[k, m - 1] = V[k] @ w
            w = w - T[k, m - 1] * V[k]
        t = float(np.linalg.norm(w))
        T[m, m - 1] = t
        breakdown = t <= breakdown_tol * max(wnorm0, 1e-300)
        if not breakdown:
            V[m] = w / t
        if m % q == 0 or breakdown or m == maxit:
            Tm = T[:m, :m]
            Vm = V[:m]
            Msys = np.eye(m, dtype=np.complex128)
            S = []
            H = []
            for i in range(ell):
                Si = np.linalg.inv((1.0 - pi[i]) * np.eye(m) + tau * Tm)
                S.append(Si)
                if breakdown:
                    Msys += weight * gamma[i] * Si
                else:
                    hi = op.shifted_solve(1.0 - pi[i], tau, V[m])
                    H.append(hi)
                    gi = Vm @ hi  # V_m^T h_i
                    # (I - tau t V_m^T h_i e_m^T) S_i = S_i - tau t g_i (e_m^T S_i)
                    Msys += weight * gamma[i] * (Si - tfac * t * np.outer(gi, Si[m - 1, :]))
            rhs = np.zeros(m, dtype=np.complex128)
            rhs[0] = beta
            y = np.linalg.solve(Msys, rhs)
            if breakdown:
                r = 0.0
            else:
                z = np.zeros(n, dtype=np.complex128)
                for i in range(ell):
                    c = S[i][m - 1, :] @ y
                    g = gamma[i] if keep_gamma_in_residual else 1.0
                    z += weight * g * H[i] * c
                proj = z - Vm.T @ (Vm @ z)
                r = abs(tfac * t) * float(np.linalg.norm(proj))
            info["resnorms"].append(r)
        if breakdown:
            info["breakdown"] = True
            break
    x = V[:m].T @ y
    info.update(m=m, y=y, T=T[: m + 1, :m], V=V[: m + 1], x_imag=float(np.linalg.norm(x.imag)))
    return x.real, info


# ----------------------------------------------------------------------------
# Algorithm 1 (new ParaDiag with backward Euler)
# ----------------------------------------------------------------------------


def paradiag(problem, G=None, eps=1e-8, maxit=50, q=1, op=None, **kw):
    """Algorithm 1 end to end on the row layout.  Returns (U, info).

    info holds pi, gamma, Ghat (= rows of G F^T), L, b, x, the Algorithm-2 info
    and the imaginary part discarded from U.
    """
    G = problem.G if G is None else np.asarray(G, dtype=np.float64)
    op = operator(problem) if op is None else op
    ell = G.shape[0]
    tau = problem.tau
    pi, gamma = circulant_eigs(ell)
    Ghat = dft_time(G)  # rows: [u0 + tau f_1, ..., tau f_l] F^T e_i
    L = np.stack([op.shifted_solve(1.0 - pi[i], tau, Ghat[i]) for i in range(ell)])
    b_c = gamma @ L  # L F^{-T} e_l  (sum_i gamma_i L e_i)
    b = b_c.real
    x, kinfo = fom_like(op, tau, b, pi, gamma, eps=eps, maxit=maxit, q=q, **kw)
    W = np.stack([op.shifted_solve(1.0 - pi[i], tau, x) for i in range(ell)])
    Uc = idft_time(L - W)
    info = {"pi": pi, "gamma": gamma, "Ghat": Ghat, "L": L, "b": b,
            "b_imag": float(np.linalg.norm(b_c.imag)), "x": x, "krylov": kinfo,
            "U_imag": float(np.linalg.norm(Uc.imag))}
    return Uc.real, info


# ----------------------------------------------------------------------------
# Algorithm 3 (alpha-acceleration, Sec. 4)
# ----------------------------------------------------------------------------


def alpha_quantities(ell, alpha):
    """Algorithm 3, first step: pi = alpha^{1/l} F C_1 e_1, gamma = F^{-T} e_l and
    the diagonal of D_alpha = diag(1, alpha^{1/l}, ..., alpha^{(l-1)/l})."""
    pi1, gamma = circulant_eigs(ell)
    a = alpha ** (1.0 / ell)
    d = alpha ** (np.arange(ell) / ell)
    return a * pi1, gamma, d


def paradiag_alpha(problem, alpha, G=None, eps=1e-8, maxit=50, q=1, op=None, early_exit_eps=None, loops=None,
                   **kw):
    """Algorithm 3 on the row layout (row j of G = column j of [u0 + tau f_1, ...]).
    Returns (U, info).  early_exit_eps: the optional residual test on U_1 of the
    algorithm (None = always run the correction).

    loops: the fixed-cost variants the paper compares at equal numbers of
    parallel-in-time loops (Sec. 6, Table 3).  1 returns U_1 (one loop, no correction);
    2 skips Algorithm 2 and takes x_m = b, i.e. the inner matrix of eq. (17) approximated
    by the identity (two loops); None runs Algorithm 3 in full."""
    G = problem.G if G is None else np.asarray(G, dtype=np.float64)
    op = operator(problem) if op is None else op
    ell = G.shape[0]
    tau = problem.tau
    pi, gamma, d = alpha_quantities(ell, alpha)
    a = alpha ** (1.0 / ell)
    Ghat = dft_time(d[:, None] * G)  # rows of [u0 + tau f_1, ...] D_alpha F^T
    L = np.stack([op.shifted_solve(1.0 - pi[i], tau, Ghat[i]) for i in range(ell)])
    U1 = (idft_time(L) / d[:, None])  # L F^{-T} D_alpha^{-1}
    info = {"pi": pi, "gamma": gamma, "d": d, "L": L, "exited_early": False}
    if loops == 1:
        return U1.real, info
    if early_exit_eps is not None:
        res = np.linalg.norm(aao_apply(problem, U1.real) - G)
        if res <= early_exit_eps * np.linalg.norm(U1.real):
            info["exited_early"] = True
            return U1.real, info
    b_c = gamma @ L  # L F^{-T} e_l
    b = b_c.real
    if loops == 2:
        x, kinfo = b.copy(), {"m": 0}
    else:
        x, kinfo = fom_like(op, tau, b, pi, gamma, eps=eps, maxit=maxit, q=q, weight=a, **kw)
    W = np.stack([op.shifted_solve(1.0 - pi[i], tau, x) for i in range(ell)])
    Uc = U1 - a * idft_time(W) / d[:, None]
    info.update(b=b, x=x, krylov=kinfo, U_imag=float(np.linalg.norm(Uc.imag)))
    return Uc.real, info


def j_alpha_dense(K, tau, ell, alpha):
    """I + alpha^{1/l} sum_i gamma_i ((1 - pi_i) I + tau K)^{-1} (eq. 17), densely."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    pi, gamma, _ = alpha_quantities(ell, alpha)
    a = alpha ** (1.0 / ell)
    J = np.eye(n, dtype=np.complex128)
    for i in range(ell):
        J += a * gamma[i] * np.linalg.inv((1.0 - pi[i]) * np.eye(n) + tau * K)
    return J


# ----------------------------------------------------------------------------
# Dense objects for pins (tiny sizes)
# ----------------------------------------------------------------------------


def j_dense(K, tau, ell):
    """J_l = I + sum_i gamma_i ((1 - pi_i) I + tau K)^{-1} (eq. 8), formed densely."""
    K = np.asarray(K, dtype=np.float64)
    n = K.shape[0]
    pi, gamma = circulant_eigs(ell)
    J = np.eye(n, dtype=np.complex128)
    for i in range(ell):
        J += gamma[i] * np.linalg.inv((1.0 - pi[i]) * np.eye(n) + tau * K)
    return J


def aao_matrix(K, tau, ell, circulant=False):
    """I_l (x) (I + tau K) - Sigma_1 (x) I on vec(U) (C_1 instead of Sigma_1 if circulant)."""
    n = K.shape[0]
    S = c_alpha(ell, 1.0) if circulant else sigma1(ell)
    return np.kron(np.eye(ell), np.eye(n) + tau * K) - np.kron(S, np.eye(n))


def aao_matrix_mass(K, tau, ell, mdiag):
    """I_l (x) (M + tau K) - Sigma_1 (x) M on vec(U): eq. (2) with a diagonal mass matrix."""
    n = K.shape[0]
    M = np.diag(np.asarray(mdiag, dtype=np.float64))
    return np.kron(np.eye(ell), M + tau * np.asarray(K)) - np.kron(sigma1(ell), M)


def periodic_solve_dense(K, tau, R):
    """Solve the circulant system (I + tau K) U - U C_1^T = R (row layout) densely."""
    R = np.asarray(R)
    ell, n = R.shape
    A = aao_matrix(np.asarray(K), tau, ell, circulant=True)
    return np.linalg.solve(A, R.reshape(-1)).reshape(ell, n)


def kappa_bound(tau, lam_min):
    """eq. (14): kappa(J_l) <= 1 + 1 / (tau lambda_min(K))."""
    return 1.0 + 1.0 / (tau * lam_min)


def j_extreme_eigs(tau, ell, lam_min, lam_max):
    """Sec. 6.1: lambda_min(J) = 1 + sum_i gamma_i / (1 - pi_i + tau lambda_max(K)),
    lambda_max(J) = 1 + sum_i gamma_i / (1 - pi_i + tau lambda_min(K))."""
    pi, gamma = circulant_eigs(ell)
    lo = 1.0 + np.sum(gamma / (1.0 - pi + tau * lam_max))
    hi = 1.0 + np.sum(gamma / (1.0 - pi + tau * lam_min))
    return lo, hi


def rel_err(A, B):
    """||A - B||_F / ||B||_F."""
    A = np.asarray(A)
    B = np.asarray(B)
    nb = np.linalg.norm(B)
    return float(np.linalg.norm(A - B) / (nb if nb > 0 else 1.0))
