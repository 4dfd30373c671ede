"""Algorithm 1's final loop formed by linearity (GPU, through the C ABI).

Arnoldi's relation (eq. 10) gives A_k^{-1} V_m = [V_m - tau t_{m+1,m} h_k e_m^T] S_k with
h_k = A_k^{-1} v_{m+1} the last step's stored solves and S_k = (s_k I + tau T_m)^{-1}, so the
final loop Y_k = A_k^{-1}(G^_k - a x_m) equals L_k - V_m s_k + c_k h_k, s_k = a S_k y_m,
c_k = tau t_{m+1,m} (e_m^T s_k), with L_k = A_k^{-1} G^_k from the first loop.  One
elementwise pass forms it over the spectrum for 1 <= m <= 16, and the third set of shifted
solves is skipped.  Solves with m > 16, or with the binary32 path's FP64 zero-frequency lane,
run the final loop's solves as before.  Both ways must meet the oracle's bars (1e-12 FP64,
1e-10 mixed), and the statistics must say which solves skipped the loop.
"""
import numpy as np
import pytest

import workloads as W
from oracle import reference as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}
OFF = {"final_loop": -1}


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as entry

    entry.build()
    import paper_2304_12597_gb300 as pkg

    return pkg


def dev():
    return torch.device("cuda:0")


def _solve(pd, P, prec, tune=None, **kw):
    with pd.Plan.from_problem(P, precision=prec, tune=tune, device=dev(), **kw) as plan:
        U, st = plan.solve(torch.from_numpy(np.ascontiguousarray(P.G)).to(dev()))
        b, x = plan.last_vectors()
        return U.cpu().numpy(), st, b.cpu().numpy(), x.cpu().numpy()


MAXM = 16


def _comb_solves(st, prec="mixed"):
    """Solves expected to form the final loop by linearity (none in binary32 plans whose
    zero frequency runs in the FP64 lane)."""
    if prec == "mixed" and st["zero_freq_fp64"]:
        return 0
    n = st["refine_sweeps"]
    return sum(1 for m in st["sweep_krylov_iters"][:n] if 1 <= m <= MAXM)


CASES = [
    ("heat1d_127x64", lambda: W.heat1d_sine_modes(127, 64, 1.0, seed=0)),
    ("heat1d_1023x256", lambda: W.heat1d_forced(1023, 256, seed=5)),
    ("advdiff1d_4095x128", lambda: W.advdiff1d_pulse(4095, 128, seed=6)),
    ("heat2d_63x63x32", lambda: W.heat2d_smooth(63, 32, seed=3)),
    ("heat2d_127x127x64", lambda: W.heat2d_smooth(127, 64, seed=4)),
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_final_loop_by_linearity_matches_oracle(pd, name, make, prec):
    P = make()
    ref = R.be_solve_refined(P)
    U, st, b, x = _solve(pd, P, prec)
    U0, st0, b0, x0 = _solve(pd, P, prec, tune=OFF)
    e, e0 = R.rel_err(U, ref), R.rel_err(U0, ref)
    assert e <= TOL[prec] and e0 <= TOL[prec], (name, e, e0, st, st0)
    # every solve whose Algorithm 2 stopped at 1 <= m <= 16 skipped the final loop's solves
    assert st0["final_by_linearity"] == 0
    assert st["final_by_linearity"] == _comb_solves(st, prec), st
    assert st["shifted_sweeps"] == st["pint_loops"] - st["final_by_linearity"]
    # x_m of the first solve (paradiag_last_vectors) is formed either way
    assert R.rel_err(x, x0) <= (1e-12 if prec == "fp64" else 1e-5), (R.rel_err(x, x0))
    assert R.rel_err(b, b0) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("c", [1e-2, 1e-3, 1e-4])
def test_final_loop_with_several_krylov_steps(pd, prec, c):
    """J_l far from I (K scaled by c): Algorithm 2 takes several steps (FP64 about 20 at
    c = 1e-4, above 16: that solve runs the final loop's solves), and the final loop by
    linearity needs S_k of the last eq. (12) system and all of V_m."""
    P = W.heat1d_forced(300, 32, seed=3)
    P.k_lo, P.k_diag, P.k_up = P.k_lo * c, P.k_diag * c, P.k_up * c
    U, st, _, x = _solve(pd, P, prec, maxit=32)
    U0, st0, _, x0 = _solve(pd, P, prec, tune=OFF, maxit=32)
    ref = R.be_solve_refined(P)
    assert R.rel_err(U, ref) <= TOL[prec] and R.rel_err(U0, ref) <= TOL[prec], (st, st0)
    assert st["sweep_krylov_iters"][0] > 1
    assert st["final_by_linearity"] == _comb_solves(st, prec), st
    assert R.rel_err(x, x0) <= (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("q", [2, 3])
def test_final_loop_with_frozen_residual(pd, q):
    """q > 1 (Sec. 3): Algorithm 2 stops only at a checked step, whose h_k and S_k the final
    loop by linearity uses."""
    P = W.heat1d_forced(300, 32, seed=3)
    c = 1e-2
    P.k_lo, P.k_diag, P.k_up = P.k_lo * c, P.k_diag * c, P.k_up * c
    U, st, _, _ = _solve(pd, P, "fp64", q=q, maxit=32)
    assert st["final_by_linearity"] == _comb_solves(st, "fp64") >= 1, st
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL["fp64"], st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_final_loop_after_breakdown(pd, prec):
    """n = 1: t_21 = 0 at the first step (breakdown), so Y_k = L_k - phi_k v_1 without the
    h_k term (no h_k was formed)."""
    P = W.random_tridiag_problem(1, 16, seed=3)
    U, st, _, _ = _solve(pd, P, prec)
    assert st["breakdown"] == 1 and st["krylov_iters"] == 1
    assert st["final_by_linearity"] >= 1
    assert R.rel_err(U, R.be_solve(P)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("alpha", [1e-2, 1e-4])
def test_final_loop_with_alpha(pd, prec, alpha):
    """Algorithm 3: the shifts s_k = 1 - alpha^{1/l} pi_k and the weight a = alpha^{1/l} enter
    phi_k."""
    P = W.heat1d_forced(255, 64, seed=11)
    U, st, _, _ = _solve(pd, P, prec, alpha=alpha)
    assert st["final_by_linearity"] >= 1
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL[prec], st


@pytest.mark.parametrize("tune,kw", [({"persistent": 1}, {}), ({}, {"no_graph": True}),
                                     ({"krylov_cluster": -1}, {})], ids=["persistent", "host_loop", "one_cta"])
def test_final_loop_in_every_launch_mode(pd, tune, kw):
    P = W.heat1d_forced(1023, 64, seed=5)
    U, st, _, _ = _solve(pd, P, "mixed", tune=tune, **kw)
    assert st["final_by_linearity"] == _comb_solves(st) >= 1
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL["mixed"], st


def test_zero_frequency_lane_keeps_the_final_loop(pd):
    P = W.heat1d_forced(255, 64, seed=2)
    U, st, _, _ = _solve(pd, P, "mixed", tune={"zero_lane": 1})
    assert st["zero_freq_fp64"] == 1 and st["final_by_linearity"] == 0
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL["mixed"]


def test_u1_exit_with_the_final_loop_by_linearity(pd):
    """Algorithm 3's U_1 test forms U_1 from the L the first loop stores for the final loop;
    when it passes (alpha = 1e-6, eps ten times U_1's residual ratio) no final loop runs."""
    P = W.advdiff1d_pulse(511, 64, nu=2.0 ** -5, seed=1)
    alpha = 1e-6
    U1, _ = R.paradiag_alpha(P, alpha, loops=1)
    r1 = np.linalg.norm(R.residual_extended(P, U1)) / np.linalg.norm(U1)
    U, st, _, _ = _solve(pd, P, "fp64", alpha=alpha, early_exit_eps=10.0 * r1)
    assert st["early_exit"] == 1 and st["final_by_linearity"] == 0
    # U = U_1 within kappa(F D_alpha) (about 1/alpha) times the FP64 rounding of the loop
    assert R.rel_err(U, U1) <= 1e-6, R.rel_err(U, U1)
