"""The relation behind the final loop by linearity, checked on the oracle (CPU).

Algorithm 2's Arnoldi process on K (eq. 10) gives tau K V_m = V_m (tau T_m) + tau t_{m+1,m}
v_{m+1} e_m^T, so for every shift s_i = 1 - pi_i and A_i = s_i I + tau K

    A_i^{-1} V_m y = V_m S_i y - tau t_{m+1,m} (e_m^T S_i y) A_i^{-1} v_{m+1},
    S_i = (s_i I_m + tau T_m)^{-1}.

With m = 1 this is A_i^{-1} x_1 = phi_i v_1 - psi_i h_i, phi_i = y_1 / (s_i + tau t_11),
psi_i = tau t_21 phi_i, h_i = A_i^{-1} v_2: the form the GPU path's inverse DFT uses for
Algorithm 1's final loop, Y_i = L_i - A_i^{-1} x_m.  The oracle's own Arnoldi basis,
Hessenberg matrix and shifted solves must satisfy it to rounding, and a dropped t-term or a
transposed T_m must not.
"""
import numpy as np
import pytest

import workloads as W
from oracle import reference as R


def _krylov(P, maxit):
    op = R.operator(P)
    ell = P.G.shape[0]
    pi, gamma = R.circulant_eigs(ell)
    _, info = R.paradiag(P, eps=1e-30, maxit=maxit, op=op)
    return op, pi, info["krylov"]


@pytest.mark.parametrize("make", [lambda: W.heat1d_forced(63, 16, seed=1),
                                  lambda: W.advdiff1d_pulse(127, 16, nu=1e-2, seed=2)],
                         ids=["heat1d", "advdiff1d"])
@pytest.mark.parametrize("m", [1, 3])
def test_shifted_solve_of_krylov_combination(make, m):
    P = make()
    op, pi, k = _krylov(P, m)
    assert k["m"] == m and not k["breakdown"]
    V, T, y = k["V"], k["T"], k["y"]  # V: (m+1, n), T: (m+1, m)
    x = V[:m].T @ y
    tau = P.tau
    t = T[m, m - 1]
    for i in range(len(pi)):
        s = 1.0 - pi[i]
        direct = op.shifted_solve(s, tau, x.astype(np.complex128))
        Si = np.linalg.inv(s * np.eye(m) + tau * T[:m, :m])
        sy = Si @ y
        h = op.shifted_solve(s, tau, V[m].astype(np.complex128))
        via = V[:m].T @ sy - tau * t * sy[m - 1] * h
        assert R.rel_err(via, direct) < 1e-12, (i, R.rel_err(via, direct))
        if m == 1:  # the scalar form with phi_i and psi_i
            phi = y[0] / (s + tau * T[0, 0])
            psi = tau * t * phi
            assert R.rel_err(phi * V[0] - psi * h, direct) < 1e-12
        # plausible slips fail: the t-term dropped, or T_m transposed (nonsymmetric K)
        assert R.rel_err(V[:m].T @ sy, direct) > 1e-6
        if m > 1 and not np.allclose(T[:m, :m], T[:m, :m].T):
            St = np.linalg.inv(s * np.eye(m) + tau * T[:m, :m].T)
            wrong = V[:m].T @ (St @ y) - tau * t * (St @ y)[m - 1] * h
            assert R.rel_err(wrong, direct) > 1e-6


def test_final_loop_by_linearity_reproduces_algorithm1():
    """Algorithm 1 with its final loop replaced by L_i - (phi_i v_1 - psi_i h_i) (m = 1)
    equals the oracle's Algorithm 1, whose final loop solves for x_1 directly."""
    P = W.heat1d_forced(63, 16, seed=4)
    op = R.operator(P)
    U_ref, info = R.paradiag(P, eps=1e-30, maxit=1, op=op)
    k = info["krylov"]
    V, T, y = k["V"], k["T"], k["y"]
    pi, L = info["pi"], info["L"]
    rows = []
    for i in range(len(pi)):
        s = 1.0 - pi[i]
        h = op.shifted_solve(s, P.tau, V[1].astype(np.complex128))
        phi = y[0] / (s + P.tau * T[0, 0])
        rows.append(L[i] - (phi * V[0] - P.tau * T[1, 0] * phi * h))
    U = R.idft_time(np.stack(rows)).real
    assert R.rel_err(U, U_ref) < 1e-12
