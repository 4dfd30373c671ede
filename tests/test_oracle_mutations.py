"""Planted mistakes in the CPU oracle must be caught by its pins.

Each case copies the oracle, plants one plausible mistake (a wrong sign, a
transposed operand, a dropped term, a mismatched convention) and checks that
at least one pin from test_oracle_pins.py's families fails on the mutant.
Mutants live only in pytest's temporary directories.
"""
import os
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import native
from oracle import reference as R

SRC = os.path.join(os.path.dirname(native.__file__), "be_oracle.c")


def _closed_form_err(lib):
    P = W.heat1d_sine_modes(63, 16, 1.0, seed=5)
    U = np.empty_like(P.G)
    d = native._p
    lib.or_be_tridiag(P.nx, P.nt, P.tau, d(P.k_lo), d(P.k_diag), d(P.k_up), None, d(P.G), d(U))
    h = 1.0 / (P.nx + 1)
    x = h * np.arange(1, P.nx + 1)
    j = np.arange(1, P.nt + 1)[:, None]
    Uc = np.zeros_like(U)
    for k, a in zip(P.extra["modes"], P.extra["amps"]):
        mu = 4.0 / h ** 2 * np.sin(k * np.pi * h / 2) ** 2
        Uc += a * (1.0 + P.tau * mu) ** (-j) * np.sin(k * np.pi * x)[None, :]
    return R.rel_err(U, Uc)


def _dense_err(lib, banded=False, problem=None):
    P = problem or W.advdiff1d_pulse(9, 8, 1.0, seed=4)
    K = R.k_dense(P)
    Ud = np.linalg.solve(R.aao_matrix(K, P.tau, P.nt), P.G.reshape(-1)).reshape(P.nt, P.nbar)
    U = np.empty_like(P.G)
    d = native._p
    if banded:
        kl, ku, B = R.k_band(P)
        B = np.ascontiguousarray(B)
        lib.or_be_banded(P.nbar, kl, ku, P.tau, d(B), None, P.nt, d(P.G), d(U))
    else:
        lib.or_be_tridiag(P.nx, P.nt, P.tau, d(P.k_lo), d(P.k_diag), d(P.k_up), None, d(P.G), d(U))
    return R.rel_err(U, Ud)


def _shifted_err(lib):
    P = W.advdiff1d_pulse(15, 8, 1.0, seed=1)
    K = R.k_dense(P)
    s = 1.0 - np.exp(-2j * np.pi / 8)
    r = np.random.default_rng(0).standard_normal(15) + 1j * np.random.default_rng(1).standard_normal(15)
    xd = np.linalg.solve(s * np.eye(15) + P.tau * K, r)
    x = np.empty(15, dtype=np.complex128)
    d = native._p
    lib.or_shifted_tridiag_solve(15, s.real, s.imag, P.tau, d(P.k_lo), d(P.k_diag), d(P.k_up),
                                 d(r.view(np.float64)), d(x.view(np.float64)))
    return R.rel_err(x, xd)


def _mutant(tmp_path, old, new, count=1):
    src = open(SRC).read()
    assert src.count(old) >= count, old
    src = src.replace(old, new, count)
    c = tmp_path / "mut.c"
    c.write_text(src)
    so = tmp_path / "mut.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", str(c), "-o", str(so), "-lm"])
    return native.load(str(so))


def test_unmutated_copy_passes(tmp_path):
    lib = _mutant(tmp_path, "#include <math.h>", "#include <math.h>")
    assert _closed_form_err(lib) < 1e-12
    assert _dense_err(lib) < 1e-13
    assert _dense_err(lib, banded=True, problem=W.heat2d_smooth(3, 4, 0.1, seed=5)) < 1e-13
    assert _shifted_err(lib) < 1e-13


C_MUTATIONS = [
    # wrong sign of the u_{j-1} coupling (Sigma_1 term)
    ("if (uprev) r += (mdiag ? mdiag[i] : 1.0) * uprev[i];\n      y[i]",
     "if (uprev) r -= (mdiag ? mdiag[i] : 1.0) * uprev[i];\n      y[i]", "tridiag"),
    # transposed operand in the factorisation (lo and up swapped)
    ("b -= mul[i] * tau * up[i - 1];", "b -= mul[i] * tau * lo[i];", "tridiag"),
    # dropped tau on the super-diagonal in the back substitution
    ("u[i] = (y[i] - tau * up[i] * u[i + 1]) / piv[i];", "u[i] = (y[i] - up[i] * u[i + 1]) / piv[i];", "tridiag"),
    # dropped identity in M + tau K (banded)
    ("A[i * w + kl] += mdiag ? mdiag[i] : 1.0;", "A[i * w + kl] += 0.0;", "banded"),
    # off-by-one band index in the banded elimination
    ("A[i * w + (j - i + kl)] -= l * A[k * w + (j - k + kl)];",
     "A[i * w + (j - i + kl)] -= l * A[k * w + (j - k + kl - 1)];", "banded"),
    # wrong sign of the complex shift
    ("double complex b = s + tau * diag[i];", "double complex b = -s + tau * diag[i];", "shifted"),
    # conjugated shift
    ("double complex s = s_re + I * s_im;", "double complex s = s_re - I * s_im;", "shifted"),
]


@pytest.mark.parametrize("old,new,kind", C_MUTATIONS, ids=[m[2] + str(i) for i, m in enumerate(C_MUTATIONS)])
def test_c_mutation_is_caught(tmp_path, old, new, kind):
    lib = _mutant(tmp_path, old, new)
    if kind == "tridiag":
        assert _closed_form_err(lib) > 1e-6 or _dense_err(lib) > 1e-6
    elif kind == "banded":
        assert _dense_err(lib, banded=True, problem=W.heat2d_smooth(3, 4, 0.1, seed=5)) > 1e-6
    else:
        assert _shifted_err(lib) > 1e-6


def test_py_mutation_gamma_convention(monkeypatch):
    """gamma taken with the conjugate convention (pi-bar / l) breaks Algorithm 1."""
    P = W.heat1d_forced(31, 16, 1.0, seed=2)
    good = R.circulant_eigs

    def bad(ell):
        pi, gamma = good(ell)
        return pi, np.conj(gamma)

    monkeypatch.setattr(R, "circulant_eigs", bad)
    U, _ = R.paradiag(P, eps=1e-13, maxit=40)
    assert R.rel_err(U, R.be_solve(P)) > 1e-6


def test_py_mutation_dropped_correction(monkeypatch):
    """Without the SMW correction W, U is the periodic solution, not eq. (2)'s."""
    P = W.heat1d_forced(31, 16, 1.0, seed=2)
    monkeypatch.setattr(R, "fom_like", lambda op, tau, b, *a, **k: (np.zeros_like(b), {"m": 0}))
    U, _ = R.paradiag(P)
    assert R.rel_err(U, R.be_solve(P)) > 1e-6


def test_py_mutation_transposed_krylov_operator(monkeypatch):
    """Building the Krylov space with K^T (nonsymmetric K) breaks eq. (11) and the result."""
    P = W.advdiff1d_pulse(31, 16, 0.2, seed=1)
    op = R.operator(P)
    Kt = R.k_dense(P).T
    monkeypatch.setattr(op, "matvec", lambda v: Kt @ v)
    U, info = R.paradiag(P, op=op, eps=1e-13, maxit=12)
    K = R.k_dense(P)
    J = R.j_dense(K, P.tau, P.nt)
    explicit = np.linalg.norm(J @ info["x"] - info["b"])
    reported = info["krylov"]["resnorms"][-1]
    assert abs(explicit - reported) > 1e-6 * np.linalg.norm(info["b"]) or R.rel_err(U, R.be_solve(P)) > 1e-6


def test_py_mutation_alpha_weight_dropped(monkeypatch):
    """Algorithm 3 without the weight alpha^{1/l} on the inner sum (eq. 17) misses eq. (2)."""
    P = W.heat1d_forced(15, 16, seed=1)
    good = R.fom_like

    def unweighted(*a, **k):
        k["weight"] = 1.0
        return good(*a, **k)

    monkeypatch.setattr(R, "fom_like", unweighted)
    alpha = 1e-2
    U, _ = R.paradiag_alpha(P, alpha, eps=1e-14, maxit=40)
    kappa = alpha ** (-(P.nt - 1) / P.nt)
    # the bound test_algorithm3_equals_sequential_stepping holds the unmutated oracle to
    assert R.rel_err(U, R.be_solve(P)) > 1e3 * 50 * kappa * 2.2e-16


def _mutant_reference(old, new):
    """A copy of oracle/reference.py with one planted mistake, loaded as a module of the
    oracle package (so its relative imports resolve); the file on disk is not touched."""
    import types

    src = open(R.__file__).read()
    assert src.count(old) == 1, old
    mod = types.ModuleType("oracle._mutant_reference")
    mod.__package__ = "oracle"
    mod.__file__ = R.__file__
    exec(compile(src.replace(old, new), R.__file__, "exec"), mod.__dict__)
    return mod


def test_py_mutation_frozen_check_off_by_one():
    """Checking at m mod q = 1 instead of 0 is caught by the frozen-residual pin: the q-run no
    longer stops at the first multiple of q whose q = 1 residual is below eps beta."""
    M = _mutant_reference("if m % q == 0 or breakdown or m == maxit:",
                          "if (m - 1) % q == 0 or breakdown or m == maxit:")
    P = W.heat1d_forced(127, 64, seed=1)
    P.k_lo, P.k_diag, P.k_up = P.k_lo * 1e-4, P.k_diag * 1e-4, P.k_up * 1e-4
    eps, maxit, q = 1e-10, 32, 3
    _, full = M.paradiag(P, eps=0.0, maxit=maxit, q=1)
    r1, beta = full["krylov"]["resnorms"], full["krylov"]["beta"]
    want = next(m for m in range(1, maxit + 1) if (m % q == 0 or m == maxit) and r1[m - 1] <= eps * beta)
    _, iq = M.paradiag(P, eps=eps, maxit=maxit, q=q)
    assert iq["krylov"]["m"] != want


def _dense_variants(P, alpha):
    n, ell = P.nx, P.nt
    A = R.aao_matrix_mass(R.k_dense(P), P.tau, ell, np.ones(n))
    E = np.zeros((ell, ell))
    E[0, ell - 1] = 1.0
    Pa = A - alpha * np.kron(E, np.eye(n))
    U1 = np.linalg.solve(Pa, P.G.reshape(-1)).reshape(ell, n)
    r = np.zeros((ell, n))
    r[0] = U1[-1]
    return U1, U1 - alpha * np.linalg.solve(Pa, r.reshape(-1)).reshape(ell, n)


def test_py_mutation_two_loop_weight_dropped():
    """The correction without its weight alpha^{1/l} fails the dense SMW pin of two loops."""
    M = _mutant_reference("Uc = U1 - a * idft_time(W) / d[:, None]", "Uc = U1 - idft_time(W) / d[:, None]")
    P = W.random_tridiag_problem(5, 8, seed=3)
    _, U2 = _dense_variants(P, 1e-2)
    V2, _ = M.paradiag_alpha(P, 1e-2, loops=2)
    assert R.rel_err(V2, U2) > 1e-6


def test_py_mutation_u1_without_d_alpha_inverse():
    """U_1 without D_alpha^{-1} after the inverse DFT fails the dense pin of one loop."""
    M = _mutant_reference("U1 = (idft_time(L) / d[:, None])", "U1 = idft_time(L)")
    P = W.random_tridiag_problem(5, 8, seed=3)
    U1, _ = _dense_variants(P, 1e-2)
    V1, _ = M.paradiag_alpha(P, 1e-2, loops=1)
    assert R.rel_err(V1, U1) > 1e-6
