"""Pins of the CPU oracle against facts fixed by the paper and the mathematics.

Each test checks the oracle against something other than itself: a closed
form, a dense direct solve, an algebraic identity, a library routine, or a
value printed in the paper (tests/golden/, with citations).
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import reference as R

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sine_eig(k, h):
    """Eigenvalue of tridiag(-1,2,-1)/h^2 for sin(k pi x): (4/h^2) sin^2(k pi h / 2)."""
    return 4.0 / h ** 2 * np.sin(k * np.pi * h / 2.0) ** 2


# ----------------------------------------------------------------------------
# Sequential backward Euler (the definition of eq. 2) against closed forms
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("n,nt", [(127, 64), (31, 16), (255, 8)])
def test_be_sine_mode_decay(n, nt):
    """u0 in sine eigenmodes, f = 0: u_j = sum_k a_k (1 + tau mu_k)^{-j} sin(k pi x)."""
    P = W.heat1d_sine_modes(n, nt, 1.0, seed=5)
    U = R.be_solve(P)
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    j = np.arange(1, nt + 1)[:, None]
    Uc = np.zeros((nt, n))
    for k, a in zip(P.extra["modes"], P.extra["amps"]):
        Uc += a * (1.0 + P.tau * _sine_eig(k, h)) ** (-j) * np.sin(k * np.pi * x)[None, :]
    assert R.rel_err(U, Uc) < 1e-12


def test_be_forced_sine_modes_recurrence():
    """Forcing in sine modes: each mode obeys c_j = (c_{j-1} + g_j) / (1 + tau mu_k)."""
    n, nt = 63, 64
    P = W.heat1d_forced(n, nt, 1.0, seed=11)
    U = R.be_solve(P)
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    t = P.tau * np.arange(1, nt + 1)
    Uc = np.zeros((nt, n))
    for k in sorted(set(P.extra["k"])):
        g = np.zeros(nt)
        for a, kq, pq in zip(P.extra["amps"], P.extra["k"], P.extra["p"]):
            if kq == k:
                g += P.tau * a * np.sin(pq * np.pi * t)
        c, coef = 0.0, np.zeros(nt)
        for jj in range(nt):
            c = (c + g[jj]) / (1.0 + P.tau * _sine_eig(k, h))
            coef[jj] = c
        Uc += np.outer(coef, np.sin(k * np.pi * x))
    assert R.rel_err(U, Uc) < 1e-12


def _tiny_problems():
    return [
        W.random_tridiag_problem(6, 5, seed=1),
        W.random_tridiag_problem(1, 4, seed=2),
        W.random_tridiag_problem(9, 8, seed=3, symmetric=True),
        W.advdiff1d_pulse(9, 8, 1.0, seed=4),
        W.heat2d_smooth(3, 4, 0.1, seed=5),
        W.heat2d_smooth(4, 6, 0.1, seed=6),
    ]


@pytest.mark.parametrize("P", _tiny_problems(), ids=lambda p: p.name)
def test_be_equals_dense_all_at_once_solve(P):
    """Dense LU (numpy.linalg.solve) of I_l (x) (I + tau K) - Sigma_1 (x) I equals the oracle."""
    K = R.k_dense(P)
    A = R.aao_matrix(K, P.tau, P.nt)
    Ud = np.linalg.solve(A, P.G.reshape(-1)).reshape(P.nt, P.nbar)
    assert R.rel_err(R.be_solve(P), Ud) < 1e-13


@pytest.mark.parametrize("name", ["heat1d_127x64", "heat1d_1023x1024", "advdiff1d_4095x2048"])
def test_be_solution_satisfies_eq2(name):
    """The oracle's U makes the left side of eq. (2) equal G (full-size 1D configs)."""
    P = W.by_name(name)
    U = R.be_solve(P)
    res = R.aao_apply(P, U) - P.G
    scale = np.linalg.norm(U) * (1.0 + P.tau * np.abs(P.k_diag).max() * 2) + np.linalg.norm(P.G)
    assert np.linalg.norm(res) / scale < 1e-15


def test_be_2d_satisfies_eq2():
    P = W.heat2d_smooth(31, 16, 0.1, seed=2)
    U = R.be_solve(P)
    res = R.aao_apply(P, U) - P.G
    assert np.linalg.norm(res) / np.linalg.norm(P.G) < 1e-13


# ----------------------------------------------------------------------------
# Sigma_1 = C_1 - e_1 e_l^T (eq. 3) and the B = (I - Sigma_1)/tau form
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("ell", [2, 3, 8, 17])
def test_sigma1_circulant_plus_rank_one(ell):
    S = R.sigma1(ell)
    C1 = R.c_alpha(ell, 1.0)
    e1 = np.eye(ell)[:, [0]]
    el = np.eye(ell)[:, [ell - 1]]
    assert np.array_equal(S, C1 - e1 @ el.T)
    # C_1 is circulant: every column is a cyclic shift of the first.
    for j in range(ell):
        assert np.array_equal(C1[:, j], np.roll(C1[:, 0], j))
    tau = 0.37
    B = (np.eye(ell) - S) / tau
    C = (np.eye(ell) - C1) / tau
    assert np.allclose(B, C + (e1 @ el.T) / tau, atol=0, rtol=0)
    # The "B = C - (1/tau) e_1 e_l^T" form holds for the skew-circulant C_{-1} (alpha = -1, eq. 15).
    Cm = (np.eye(ell) - R.c_alpha(ell, -1.0)) / tau
    assert np.allclose(B, Cm - (e1 @ el.T) / tau, atol=1e-15)
    if ell > 1:
        assert not np.allclose(B, C - (e1 @ el.T) / tau)


@pytest.mark.parametrize("P", _tiny_problems()[:4], ids=lambda p: p.name)
def test_oracle_solves_kron_form(P):
    """(B (x) I + I (x) K) u = G / tau with B = C + (1/tau) e_1 e_l^T, C = (I - C_1)/tau."""
    K = R.k_dense(P)
    ell, n = P.nt, P.nbar
    C = (np.eye(ell) - R.c_alpha(ell, 1.0)) / P.tau
    E = np.zeros((ell, ell))
    E[0, ell - 1] = 1.0
    B = C + E / P.tau
    A = np.kron(B, np.eye(n)) + np.kron(np.eye(ell), K)
    U = R.be_solve(P)
    assert np.linalg.norm(A @ U.reshape(-1) - P.G.reshape(-1) / P.tau) <= 1e-12 * np.linalg.norm(P.G / P.tau)


# ----------------------------------------------------------------------------
# Fourier objects (Sec. 2, appendix)
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("ell", [1, 2, 4, 6, 16, 64])
def test_dft_matches_numpy_fft(ell):
    rng = np.random.default_rng(ell)
    X = rng.standard_normal((ell, 5)) + 1j * rng.standard_normal((ell, 5))
    assert np.allclose(R.dft_time(X), np.fft.fft(X, axis=0), rtol=0, atol=1e-12 * ell)
    assert np.allclose(R.idft_time(X), np.fft.ifft(X, axis=0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("ell", [2, 3, 8, 32])
def test_circulant_eigs(ell):
    """F C_1 F^{-1} = diag(pi), pi_i = omega^i, gamma = F^{-T} e_l = pi / l (appendix)."""
    F = R.dft_matrix(ell)
    pi, gamma = R.circulant_eigs(ell)
    D = F @ R.c_alpha(ell, 1.0) @ np.linalg.inv(F)
    assert np.allclose(D, np.diag(pi), atol=1e-12)
    assert np.allclose(pi, np.exp(-2j * np.pi * np.arange(ell) / ell), atol=1e-13)
    assert np.allclose(gamma, pi / ell, atol=1e-13)


# ----------------------------------------------------------------------------
# Table 1 and the Sec. 6.1 heat claims
# ----------------------------------------------------------------------------


def _read_table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                nbar, ell, val = line.split()
                rows.append((int(nbar), int(ell), float(val)))
    return rows


@pytest.mark.parametrize("nbar,ell,val", _read_table1())
def test_table1_bound(nbar, ell, val):
    """eq. (14) evaluated with lambda_min(K) of the generator's 2D operator matches Table 1."""
    n = int(round(np.sqrt(nbar)))
    if n <= 512:
        lo, diag, up = W.heat2d_axis_operator(n)
        T = np.diag(diag) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)
        lam_T = np.linalg.eigvalsh(T)[0]
    else:  # the same eigenvalue in closed form (Sec. 6.1) for the largest grid
        h = 1.0 / (n + 1)
        lam_T = 4.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    lam = 2.0 * lam_T  # K = I (x) T + T (x) I
    h = 1.0 / (n + 1)
    assert abs(lam - 8.0 / h ** 2 * np.sin(np.pi / (2 * (n + 1))) ** 2) < 1e-9 * lam
    assert abs(R.kappa_bound(1.0 / ell, lam) - val) <= 1.0e-3


def _read_claims():
    d = {}
    with open(os.path.join(GOLDEN, "heat_claims.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                d[k] = float(v)
    return d


@pytest.mark.parametrize("nbar,ell", [(r[0], r[1]) for r in _read_table1()])
def test_heat_spectrum_of_J(nbar, ell):
    """[lambda_min(J), lambda_max(J)] in [1, 1.004] (Sec. 6.1), and equal to the closed
    form z^l / (z^l - 1), z = 1 + tau lambda (geometric sum over the l-th roots of unity)."""
    c = _read_claims()
    n = int(round(np.sqrt(nbar)))
    h = 1.0 / (n + 1)
    tau = 1.0 / ell
    lam_min = 8.0 / h ** 2 * np.sin(np.pi * h / 2) ** 2
    lam_max = 8.0 / h ** 2 * np.cos(np.pi * h / 2) ** 2
    lo, hi = R.j_extreme_eigs(tau, ell, lam_min, lam_max)
    for val, lam in ((lo, lam_max), (hi, lam_min)):
        w = np.exp(-ell * np.log1p(tau * lam))  # z^{-l}, z = 1 + tau lambda
        assert abs(val.imag) < 1e-12
        assert abs(val.real - (1.0 + w / (1.0 - w))) < 1e-12
    assert c["spec_lo"] <= lo.real <= hi.real <= c["spec_hi"]


def test_mcdonald_example_one_iteration():
    """Algorithm 1 on f = 0, u0 = x y (x-1)(1-y): one Algorithm-2 iteration reaches
    relative residual < 1e-8 (Sec. 6.1), here on a 15 x 15 grid with l = 16, 32."""
    c = _read_claims()
    for ell in (16, 32):
        P = W.heat2d_smooth(15, ell, 1.0, seed=0)
        h = 1.0 / 16
        x = h * np.arange(1, 16)
        X, Y = np.meshgrid(x, x)  # (iy, ix)
        G = np.zeros_like(P.G)
        G[0] = (X * Y * (X - 1) * (1 - Y)).reshape(-1)
        U, info = R.paradiag(P, G=G, eps=c["eps"], maxit=20)
        k = info["krylov"]
        assert k["m"] == int(c["iterations"])
        assert k["resnorms"][0] < c["eps"] * k["beta"]
        assert R.rel_err(U, R.be_solve(P, G=G)) < 1e-7


# ----------------------------------------------------------------------------
# Theorem 3.1 and the capacitance operator J_l (eq. 8)
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("n,ell", [(8, 8), (8, 16), (5, 7)])
def test_theorem31_hpd_and_bound(n, ell):
    P = W.random_tridiag_problem(n, ell, seed=n + ell, symmetric=True)
    K = R.k_dense(P)
    J = R.j_dense(K, P.tau, ell)
    assert np.allclose(J, J.conj().T, atol=1e-13)
    ev = np.linalg.eigvalsh(J)
    assert ev.min() > 0
    lam = np.linalg.eigvalsh(K)
    assert ev.max() / ev.min() <= R.kappa_bound(P.tau, lam.min()) + 1e-12
    z = 1.0 + P.tau * lam
    assert np.allclose(np.sort(ev), np.sort(z ** ell / (z ** ell - 1.0)), rtol=1e-12)


# ----------------------------------------------------------------------------
# Algorithm 2: eq. (13) against the explicit residual, x = u_l, b = periodic u_l
# ----------------------------------------------------------------------------


def _slow_problems():
    return [W.heat2d_smooth(5, 8, 0.05, seed=3), W.advdiff1d_pulse(31, 16, 0.2, seed=1),
            W.random_tridiag_problem(12, 8, 0.1, seed=9)]


@pytest.mark.parametrize("P", _slow_problems(), ids=lambda p: p.name)
def test_eq13_equals_explicit_residual(P):
    """||r_m|| of eq. (13), with tau * t_{m+1,m}, equals ||J_l x_m - b|| at every m;
    the literal tau-less form does not."""
    op = R.operator(P)
    K = R.k_dense(P)
    J = R.j_dense(K, P.tau, P.nt)
    pi, gamma = R.circulant_eigs(P.nt)
    b = np.random.default_rng(0).standard_normal(P.nbar)
    mismatch_without_tau = 0.0
    for m in range(1, 6):
        x, info = R.fom_like(op, P.tau, b, pi, gamma, eps=0.0, maxit=m)
        if info["breakdown"]:
            break
        explicit = np.linalg.norm(J @ x - b)
        assert abs(info["resnorms"][-1] - explicit) <= 1e-9 * np.linalg.norm(b) + 1e-6 * explicit
        # Galerkin condition V_m^T r_m = 0
        assert np.linalg.norm(info["V"][:m] @ (J @ x - b).real) <= 1e-10 * np.linalg.norm(b)
        _, info2 = R.fom_like(op, P.tau, b, pi, gamma, eps=0.0, maxit=m, keep_tau=False)
        x2 = info2["V"][:m].T @ info2["y"]
        mismatch_without_tau = max(mismatch_without_tau,
                                   abs(info2["resnorms"][-1] - np.linalg.norm(J @ x2 - b)) / np.linalg.norm(b))
    assert mismatch_without_tau > 1e-6


@pytest.mark.parametrize("P", _tiny_problems()[:5] + _slow_problems(), ids=lambda p: p.name)
def test_b_is_periodic_final_state_and_x_is_u_ell(P):
    """b = L F^{-T} e_l (eq. 7) is the last time slice of the circulant (periodic) solution,
    and the exact solution x of eq. (8) is the true final state u_l."""
    K = R.k_dense(P)
    U_per = R.periodic_solve_dense(K, P.tau, P.G)
    U, info = R.paradiag(P, eps=1e-14, maxit=60)
    assert np.linalg.norm(info["b"] - U_per[-1].real) <= 1e-12 * max(1.0, np.linalg.norm(U_per[-1]))
    assert info["b_imag"] <= 1e-12 * max(1.0, np.linalg.norm(info["b"]))
    Ube = R.be_solve(P)
    assert np.linalg.norm(info["x"] - Ube[-1]) <= 1e-11 * max(1.0, np.linalg.norm(Ube[-1]))


@pytest.mark.parametrize("name,size", [("heat1d_sine_modes", (63, 32)), ("heat1d_forced", (127, 64)),
                                       ("advdiff1d_pulse", (255, 64)), ("heat2d_smooth", (7, 16))])
def test_algorithm1_equals_sequential(name, size):
    P = getattr(W, name)(*size)
    U, info = R.paradiag(P, eps=1e-13, maxit=60)
    assert R.rel_err(U, R.be_solve(P)) < 1e-12
    assert info["U_imag"] < 1e-12 * np.linalg.norm(U)


# ----------------------------------------------------------------------------
# A diagonal mass matrix M: (B (x) M + I (x) K) u = f, step (M + tau K) u_j = M u_{j-1} + G_j
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("P", [W.random_tridiag_problem(7, 5, seed=1), W.heat1d_forced(15, 8, seed=2),
                               W.random_tridiag_problem(1, 4, seed=3), W.advdiff1d_pulse(12, 6, seed=4)],
                         ids=lambda p: p.name)
def test_mass_matrix_oracle_equals_dense_all_at_once(P):
    """Dense LU of I_l (x) (M + tau K) - Sigma_1 (x) M equals the sequential oracle."""
    Q = W.with_mass(P, seed=3)
    A = R.aao_matrix_mass(R.k_dense(Q), Q.tau, Q.nt, Q.m_diag)
    Ud = np.linalg.solve(A, Q.G.reshape(-1)).reshape(Q.nt, Q.nbar)
    assert R.rel_err(R.be_solve(Q), Ud) < 1e-13
    # and M actually changes the answer
    assert R.rel_err(R.be_solve(P), Ud) > 1e-3


def test_constant_mass_matrix_is_a_rescaled_step():
    """M = c I: (c I + tau K) u_j = c u_{j-1} + G_j is the unit-mass problem with tau / c and G / c."""
    P = W.heat1d_forced(63, 16, seed=2)
    c = 2.5
    Q = W.with_mass(P, seed=1)
    Q.m_diag = np.full(P.nx, c)
    P2 = W.heat1d_forced(63, 16, seed=2)
    P2.tau, P2.G = P.tau / c, P.G / c
    assert R.rel_err(R.be_solve(Q), R.be_solve(P2)) < 1e-14


def test_mass_matrix_residual_vanishes_at_the_solution():
    """aao_apply and the extended residual carry M: the refined solution leaves ~1e-16."""
    Q = W.with_mass(W.heat1d_forced(127, 32, seed=5), seed=2)
    U = R.be_solve_refined(Q)
    assert np.linalg.norm(R.residual_extended(Q, U)) / np.linalg.norm(Q.G) < 1e-14
    assert np.linalg.norm(R.aao_apply(Q, U) - Q.G) / np.linalg.norm(Q.G) < 1e-13


# The refined reference (one correction on an extended-precision residual)
# ----------------------------------------------------------------------------


def test_refined_oracle_closed_form():
    """With the extended residual the sine-mode closed form is met to ~1e-15."""
    n, nt = 255, 64
    P = W.heat1d_sine_modes(n, nt, 1.0, seed=5)
    h = 1.0 / (n + 1)
    x = h * np.arange(1, n + 1)
    j = np.arange(1, nt + 1)[:, None]
    Uc = np.zeros((nt, n))
    for k, a in zip(P.extra["modes"], P.extra["amps"]):
        Uc += a * (1.0 + P.tau * _sine_eig(k, h)) ** (-j) * np.sin(k * np.pi * x)[None, :]
    assert R.rel_err(R.be_solve_refined(P), Uc) < 2e-15


@pytest.mark.parametrize("P", [W.heat2d_smooth(63, 64, 0.1, seed=1), W.heat1d_1023x1024(), W.advdiff1d_pulse(511, 256, seed=2)],
                         ids=lambda p: p.name)
def test_refined_oracle_converges(P):
    """A second correction on the extended residual is negligible next to the first
    (the refinement has converged to working precision)."""
    U = R.be_solve(P)
    d1 = R.be_solve(P, G=R.residual_extended(P, U))
    d2 = R.be_solve(P, G=R.residual_extended(P, U + d1))
    n = np.linalg.norm(U)
    assert np.linalg.norm(d1) / n < 1e-10
    assert np.linalg.norm(d2) / n < 1e-15
    assert np.linalg.norm(d2) <= 0.05 * np.linalg.norm(d1) + 1e-16 * n


def test_extended_residual_matches_float64_residual():
    P = W.heat2d_smooth(7, 8, 0.1, seed=2)
    U = np.random.default_rng(1).standard_normal(P.G.shape)
    assert np.allclose(R.residual_extended(P, U), P.G - R.aao_apply(P, U), rtol=1e-13, atol=1e-13)


# ----------------------------------------------------------------------------
# Algorithm 3 (alpha-acceleration, Sec. 4)
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("ell,alpha", [(8, 0.3), (16, 1e-3), (5, 1.0)])
def test_c_alpha_is_diagonalised_by_the_scaled_dft(ell, alpha):
    """eq. (15)-(16): C_alpha = D_alpha^{-1} F^{-1} diag(pi) F D_alpha with pi of Algorithm 3."""
    pi, _, d = R.alpha_quantities(ell, alpha)
    F = R.dft_matrix(ell)
    C = np.diag(1.0 / d) @ np.linalg.solve(F, np.diag(pi) @ F @ np.diag(d))
    assert np.allclose(C, R.c_alpha(ell, alpha), atol=1e-13 / alpha)
    # and Sigma_1 = C_alpha - alpha e_1 e_l^T (eq. 15)
    E = np.zeros((ell, ell))
    E[0, -1] = alpha
    assert np.array_equal(R.c_alpha(ell, alpha) - E, R.sigma1(ell))


@pytest.mark.parametrize("alpha", [1.0, 0.2, 1e-4])
def test_alpha_inner_matrix_eigenvalues(alpha):
    """eq. (17) for SPD K: I + alpha^{1/l} sum_i gamma_i (1 - pi_i + tau lambda)^{-1} has
    the eigenvalue z^l / (z^l - alpha), z = 1 + tau lambda (the identity
    sum_i omega^i / (z - a omega^i) = l a^{l-1} / (z^l - a^l) summed over the roots of
    unity); alpha = 1 is Theorem 3.1's z^l / (z^l - 1)."""
    n, ell, tau = 12, 16, 0.05
    K = (np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)) * (n + 1) ** 2 / 50.0
    lam = np.linalg.eigvalsh(K)
    z = 1.0 + tau * lam
    expect = np.sort(z ** ell / (z ** ell - alpha))
    got = np.sort(np.linalg.eigvals(R.j_alpha_dense(K, tau, ell, alpha)).real)
    assert np.allclose(got, expect, rtol=1e-10)


@pytest.mark.parametrize("alpha", [1.0, 0.1, 1e-3, 1e-6])
def test_algorithm3_equals_sequential_stepping(alpha):
    """Algorithm 3 with an exact inner solve reaches eq. (2)'s solution; the error grows
    like kappa(F D_alpha) = alpha^{-(l-1)/l} times the rounding unit (Sec. 4)."""
    P = W.heat1d_forced(15, 16, seed=1)
    U, info = R.paradiag_alpha(P, alpha, eps=1e-14, maxit=40)
    kappa = alpha ** (-(P.nt - 1) / P.nt)
    assert R.rel_err(U, R.be_solve(P)) <= 50 * kappa * 2.2e-16
    assert info["U_imag"] <= 1e-10 * np.linalg.norm(U)


def test_algorithm3_with_alpha_one_is_algorithm1():
    P = W.advdiff1d_pulse(31, 16, 0.2, seed=1)
    U3, i3 = R.paradiag_alpha(P, 1.0, eps=1e-13, maxit=40)
    U1, i1 = R.paradiag(P, eps=1e-13, maxit=40)
    assert R.rel_err(U3, U1) <= 1e-13
    assert i3["krylov"]["m"] == i1["krylov"]["m"]


def test_small_alpha_accelerates_the_inner_solve():
    """Sec. 4: the inner matrix is a small perturbation of I for alpha << 1, so FOM needs
    fewer iterations; here slow diffusion (nu = 1e-3) makes J_l far from I at alpha = 1."""
    lo, di, up = W.heat1d_operator(63)
    P = W.heat1d_forced(63, 32, seed=3)
    P.k_lo, P.k_diag, P.k_up = 1e-3 * lo, 1e-3 * di, 1e-3 * up
    ref = R.be_solve(P)
    U1, i1 = R.paradiag_alpha(P, 1.0, eps=1e-6, maxit=60)
    U4, i4 = R.paradiag_alpha(P, 1e-4, eps=1e-6, maxit=60)
    U6, i6 = R.paradiag_alpha(P, 1e-6, eps=1e-6, maxit=60)
    assert i6["krylov"]["m"] < i4["krylov"]["m"] < i1["krylov"]["m"]
    assert i6["krylov"]["m"] <= 2
    # the correction is weighted by alpha^{1/l}: the same inner tolerance leaves a
    # far smaller error in U
    assert R.rel_err(U4, ref) <= 1e-2 * R.rel_err(U1, ref)


def test_algorithm3_early_exit_on_u1():
    """For small alpha the first term U_1 alone passes the residual test of Algorithm 3
    (the correction is O(alpha)); far smaller alpha loses that to kappa(F D_alpha)."""
    P = W.heat1d_forced(31, 16, seed=4)
    U, info = R.paradiag_alpha(P, 1e-6, early_exit_eps=1e-6)
    assert info["exited_early"]
    assert R.rel_err(U, R.be_solve(P)) <= 1e-6
    _, info = R.paradiag_alpha(P, 1e-12, early_exit_eps=1e-6)
    assert not info["exited_early"]


@pytest.mark.parametrize("mass", [False, True])
def test_build_rhs_steps_backward_euler(mass):
    """G from build_rhs (eq. 2: G_1 = M u0 + tau f_1, G_j = tau f_j) makes the oracle's solve
    equal to backward Euler stepped by hand from u0 with dense solves of (M + tau K)."""
    P = W.random_tridiag_problem(23, 12, seed=4)
    rng = np.random.default_rng(8)
    u0, f = rng.standard_normal(P.nx), rng.standard_normal((P.nt, P.nx))
    m = 0.5 + 1.5 * rng.random(P.nx) if mass else None
    Mm = np.diag(m) if mass else np.eye(P.nx)
    A = Mm + P.tau * R.k_dense(P)
    u, Ue = u0, np.empty((P.nt, P.nx))
    for j in range(P.nt):
        u = np.linalg.solve(A, Mm @ u + P.tau * f[j])
        Ue[j] = u
    G = W.build_rhs(u0, f, P.tau, m)
    assert R.rel_err(R.be_solve(P, G=G, mdiag=m), Ue) < 1e-13
    # the generators' f = 0 right-hand sides are build_rhs of their initial values
    S = W.heat1d_sine_modes(31, 8)
    assert np.array_equal(W.build_rhs(S.G[0], np.zeros_like(S.G), S.tau), S.G)


def test_backward_euler_is_causal_under_time_padding():
    """Rows 1..l of the all-at-once solution depend on rows 1..l of G only: extending G by
    zero rows leaves those rows of the oracle's solution unchanged (the reading that lets
    a batch carry problems of fewer time steps), and the dense all-at-once solve agrees."""
    P = W.random_tridiag_problem(9, 8, seed=11)
    U = R.be_solve(P)
    Q = W.random_tridiag_problem(9, 8, seed=11)
    Q.nt, Q.G = 32, np.vstack([P.G, np.zeros((24, P.nx))])
    V = R.be_solve(Q)
    assert np.array_equal(V[:8], U)
    A = R.aao_matrix_mass(R.k_dense(Q), Q.tau, Q.nt, np.ones(Q.nx))
    Vd = np.linalg.solve(A, Q.G.reshape(-1)).reshape(Q.nt, Q.nx)
    assert R.rel_err(Vd[:8], U) < 1e-13


def _slow_krylov_heat(n=127, nt=64, c=1e-4):
    """1D heat with K scaled by c: tau lambda_min(K) ~ 1.5e-6, so J_l is far from I and
    Algorithm 2 needs about a dozen steps (the bound of eq. 14)."""
    P = W.heat1d_forced(n, nt, seed=1)
    P.k_lo, P.k_diag, P.k_up = P.k_lo * c, P.k_diag * c, P.k_up * c
    return P


@pytest.mark.parametrize("q", [2, 3, 5])
def test_frozen_residual_stops_at_the_first_checked_step(q):
    """Sec. 3, frozen residual: y_m and ||r_m|| of step m do not depend on q, so checking
    only every q steps stops at the first multiple of q (or maxit) whose q = 1 residual is
    <= eps beta, with the same x_m as a q = 1 run stopped there."""
    P = _slow_krylov_heat()
    eps, maxit = 1e-10, 32
    _, full = R.paradiag(P, eps=0.0, maxit=maxit, q=1)
    r1 = full["krylov"]["resnorms"]  # r_1 .. r_maxit
    beta = full["krylov"]["beta"]
    want = next(m for m in range(1, maxit + 1) if (m % q == 0 or m == maxit) and r1[m - 1] <= eps * beta)
    Uq, iq = R.paradiag(P, eps=eps, maxit=maxit, q=q)
    assert iq["krylov"]["m"] == want
    # one residual per checked step, equal to the q = 1 residual there
    checked = [m for m in range(1, want + 1) if m % q == 0 or m == want]
    assert np.allclose(iq["krylov"]["resnorms"], [r1[m - 1] for m in checked], rtol=1e-12, atol=0)
    U1, _ = R.paradiag(P, eps=0.0, maxit=want, q=1)
    assert R.rel_err(Uq, U1) < 1e-15
    assert R.rel_err(Uq, R.be_solve(P)) < 1e-9


@pytest.mark.parametrize("alpha", [1e-2, 0.3, 1.0])
def test_fixed_loop_variants_equal_their_dense_forms(alpha):
    """Sec. 6, Table 3 variants of Algorithm 3, against the dense operators.  With
    A = I (x) (I + tau K) - Sigma_1 (x) I and P_alpha = A - alpha (e_1 e_l^T (x) I) (the
    alpha-circulant of eq. 15), Sherman-Morrison-Woodbury gives
    A^{-1} g = U_1 - alpha P^{-1} E_1 (I + alpha E_l^T P^{-1} E_1)^{-1} E_l^T U_1 with
    U_1 = P^{-1} g: one loop returns U_1, and two loops (x_m = b) drop the inner inverse."""
    P = W.random_tridiag_problem(5, 8, seed=3)
    n, ell = P.nx, P.nt
    A = R.aao_matrix_mass(R.k_dense(P), P.tau, ell, np.ones(n))
    E = np.zeros((ell, ell))
    E[0, ell - 1] = 1.0
    Pa = A - alpha * np.kron(E, np.eye(n))
    U1 = np.linalg.solve(Pa, P.G.reshape(-1)).reshape(ell, n)
    r = np.zeros((ell, n))
    r[0] = U1[-1]
    U2 = U1 - alpha * np.linalg.solve(Pa, r.reshape(-1)).reshape(ell, n)
    V1, _ = R.paradiag_alpha(P, alpha, loops=1)
    V2, info = R.paradiag_alpha(P, alpha, loops=2)
    assert R.rel_err(V1, U1) < 1e-13 and R.rel_err(V2, U2) < 1e-13
    assert info["krylov"]["m"] == 0
    # the full method recovers the exact solution; the variants are approximations of it
    assert R.rel_err(R.paradiag_alpha(P, alpha, eps=1e-14)[0], R.be_solve(P)) < 1e-11
    assert R.rel_err(V2, R.be_solve(P)) > 1e-14


@pytest.mark.parametrize("nu", [1e-1, 1e-2, 1e-3])
def test_fixed_loop_variants_reach_table3_orders(nu):
    """Table 3's orders of magnitude, on 1D advection-diffusion (the paper's problem is 2D):
    two loops at alpha = 1e-4 leave a relative residual of at most 1e-8, one loop at
    alpha = 1e-6 one in 1e-9 .. 1e-6, and two loops are the more accurate."""
    P = W.advdiff1d_pulse(255, 32, nu=nu, seed=1)
    rr = lambda U: np.linalg.norm(R.residual_extended(P, U)) / np.linalg.norm(P.G)
    r2 = rr(R.paradiag_alpha(P, 1e-4, loops=2)[0])
    r1 = rr(R.paradiag_alpha(P, 1e-6, loops=1)[0])
    assert r2 <= 1e-8 and 1e-9 <= r1 <= 1e-6 and r2 < r1


def test_algorithm3_reproduces_figure1_trends():
    """Sec. 6, Fig. 1 (one FOM step, maxit = 1), on 1D advection-diffusion with the figure's
    nu = 2^-5 and l = 64 (its 2D operator is not separable):
    - ||U_1|| hardly moves with alpha, ||U_2|| follows alpha;
    - the error and residual of U = U_1 + U_2 scale like alpha^2, the residual of U_1 like alpha;
    - alpha ~ 1e-7 leaves U_1 alone a residual of order 1e-7;
    - below alpha ~ 1e-4 the conditioning of F D_alpha takes over and the error grows again."""
    P = W.advdiff1d_pulse(511, 64, nu=2.0 ** -5, seed=1)
    ex = R.be_solve_refined(P)
    rr = lambda X: np.linalg.norm(R.residual_extended(P, X)) / np.linalg.norm(P.G)
    alphas = [1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-10]
    n1, n2, err, res, res1 = {}, {}, {}, {}, {}
    for a in alphas:
        U, _ = R.paradiag_alpha(P, a, eps=0.0, maxit=1)
        U1, _ = R.paradiag_alpha(P, a, loops=1)
        n1[a], n2[a] = np.linalg.norm(U1), np.linalg.norm(U - U1)
        err[a], res[a], res1[a] = R.rel_err(U, ex), rr(U), rr(U1)
    assert max(n1.values()) / min(n1.values()) < 1.02
    c2 = [n2[a] / a for a in alphas if a <= 1e-1]
    assert max(c2) / min(c2) < 1.05
    for d in (err, res):  # alpha^2 while rounding is negligible
        q = [d[a] / a ** 2 for a in (1.0, 1e-1, 1e-2)]
        assert max(q) / min(q) < 1.1
    q1 = [res1[a] / a for a in (1.0, 1e-1, 1e-2, 1e-3, 1e-4, 1e-5)]
    assert max(q1) / min(q1) < 1.05
    assert 1e-8 < res1[1e-7] < 1e-6
    best = min(alphas, key=lambda a: err[a])
    assert 1e-4 <= best <= 1e-2
    assert err[1e-10] > 100 * err[best] and err[1e-6] > err[1e-4]
