"""The persistent form of an Algorithm-2 step (GPU, through the C ABI).

After a step's shifted solves (h_k = A_k^{-1} v_m and their dots), one cooperative launch
runs the eq. (12) terms and system, z = sum_k gamma_k h_k c_k, the eq. (13) residual with
the stopping decision, and the next Arnoldi step (eq. 10), with grid barriers between the
phases.  Results must match the oracle to the same bars as the per-phase launches (1e-12
FP64, 1e-10 mixed), for the vector phases in one CTA (n_bar <= 8192) and spread over the
grid, in the graph and in the host-driven loop, with frozen steps (q > 1) and at a
breakdown.  Every grid barrier waits a bounded number of polls: with barrier_extra = 1 each
barrier waits for a CTA that does not exist, every wait runs out, and the solve must come
back with PD_ERR_TIMEOUT (no hang), the plan still usable.
"""
import numpy as np
import pytest

import workloads as W
from oracle import reference as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}
ON = {"persistent": 1}
OFF = {"persistent": -1}


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


def _solve(pd, P, prec, tune, G=None, **kw):
    G = P.G if G is None else G
    with pd.Plan.from_problem(P, precision=prec, tune=tune, device=dev(), **kw) as plan:
        plan.set_timing(kw.get("no_graph", False))
        U, st = plan.solve(torch.from_numpy(G).to(dev()))
        fams = {k["name"] for k in plan.kernel_times()} if kw.get("no_graph", False) else set()
    return U.cpu().numpy(), st, fams


CASES = [
    ("heat1d_127x64", lambda: W.heat1d_sine_modes(127, 64, 1.0, seed=0)),
    ("heat1d_1023x64", lambda: W.heat1d_forced(1023, 64, seed=5)),
    ("advdiff1d_4095x64", lambda: W.advdiff1d_pulse(4095, 64, seed=6)),
    ("heat2d_63x63x32", lambda: W.heat2d_smooth(63, 32, seed=3)),     # vectors in CTA 0
    ("heat2d_127x127x16", lambda: W.heat2d_smooth(127, 16, seed=4)),  # n_bar 16129: over the grid
]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_persistent_step_matches_oracle(pd, name, make, prec):
    P = make()
    ref = R.be_solve_refined(P)
    U, st, _ = _solve(pd, P, prec, ON)
    # the same Algorithm-2 run with one launch per phase (z summed in another order)
    U0, st0, _ = _solve(pd, P, prec, OFF)
    e, e0 = R.rel_err(U, ref), R.rel_err(U0, ref)
    assert st["graph"] == 1 and st["persistent_step"] == 1 and st0["persistent_step"] == 0
    assert e <= TOL[prec] and e0 <= TOL[prec], (name, e, e0, st, st0)
    assert abs(st["krylov_iters_total"] - st0["krylov_iters_total"]) <= max(1, st0["krylov_iters_total"] // 4), (st, st0)


@pytest.mark.parametrize("name,make", [CASES[1], CASES[4]], ids=[CASES[1][0], CASES[4][0]])
def test_persistent_step_in_host_loop(pd, name, make):
    """The host-driven loop (timing mode) launches the same persistent kernel each step."""
    P = make()
    U, st, fams = _solve(pd, P, "mixed", ON, no_graph=True)
    assert st["graph"] == 0
    assert "krylov_step" in fams and "capacitance" not in fams and "zsum" not in fams, fams
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL["mixed"], st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_step_frozen_residual(pd, prec):
    """q = 3 (Sec. 3): the persistent launch of a frozen step only advances m and runs the
    next Arnoldi step; checks fall on multiples of q, maxit or a breakdown."""
    P = W.heat1d_forced(300, 32, seed=3)
    c = 1e-4  # J_l far from I: Algorithm 2 takes many steps
    P.k_lo, P.k_diag, P.k_up = P.k_lo * c, P.k_diag * c, P.k_up * c
    U, st, _ = _solve(pd, P, prec, ON, q=3, maxit=32)
    assert st["persistent_step"] == 1
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL[prec], st
    ms = st["sweep_krylov_iters"][: st["refine_sweeps"]]
    assert max(ms) > 3
    for m in ms:
        assert m % 3 == 0 or m == 32 or st["breakdown"], ms


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_persistent_step_breakdown(pd, prec):
    """n = 1: t_{2,1} = 0 at the first Arnoldi step (run before the loop); the persistent
    step then solves eq. (12) without its t-term and stops with ||r_1|| = 0."""
    P = W.random_tridiag_problem(1, 16, seed=3)
    U, st, _ = _solve(pd, P, prec, ON)
    assert st["persistent_step"] == 1
    assert st["breakdown"] == 1 and st["krylov_iters"] == 1
    assert R.rel_err(U, R.be_solve(P)) <= TOL[prec]


@pytest.mark.parametrize("ctas", [1, 8, 40])
def test_persistent_step_grid_sizes(pd, ctas):
    """Any co-resident grid gives the oracle's result (z tiles and capacitance partials are
    spread over however many CTAs there are; the vector phases need the grid's registers
    for n_bar = 16129 only when the grid has >= 8 CTAs, so one CTA falls back)."""
    P = W.heat2d_smooth(127, 16, seed=4)
    U, st, _ = _solve(pd, P, "mixed", {"persistent": 1, "persist_ctas": ctas})
    assert st["persistent_step"] == (0 if ctas == 1 else 1)
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL["mixed"], st


@pytest.mark.parametrize("no_graph", [False, True])
@pytest.mark.parametrize("name,make", [CASES[1], CASES[4]], ids=[CASES[1][0], CASES[4][0]])
def test_barrier_timeout_returns_status(pd, name, make, no_graph):
    """barrier_extra = 1: every grid barrier of the persistent step waits for one CTA more
    than the launch has, so no barrier can complete.  Each wait gives up after
    barrier_polls polls, the kernel returns, the loops stop, and the solve reports
    PD_ERR_TIMEOUT.  The plan stays usable (a second solve times out the same way), and a
    plan without the phantom CTA then solves to the oracle's bar on the same context."""
    P = make()
    G = torch.from_numpy(P.G).to(dev())
    with pd.Plan.from_problem(P, precision="mixed", tune=ON, barrier_extra=1, barrier_polls=2000,
                              no_graph=no_graph, device=dev()) as plan:
        for _ in range(2):
            with pytest.raises(pd.ParadiagError) as e:
                plan.solve(G)
            assert e.value.status_name == "PD_ERR_TIMEOUT", str(e.value)
    torch.cuda.synchronize()
    U, st, _ = _solve(pd, P, "mixed", ON)
    assert R.rel_err(U, R.be_solve_refined(P)) <= TOL["mixed"], st


def test_persistent_step_applies_to_single_problems_only(pd):
    """Batches keep the per-phase launches (one Algorithm 2 per problem) even on request."""
    probs = [W.heat1d_forced(255, 32, seed=s) for s in range(3)]
    with pd.Plan.from_problems(probs, precision="mixed", no_graph=True, tune=ON, device=dev()) as plan:
        plan.set_timing(True)
        Gs = plan.stack([p.G for p in probs])
        plan.solve(torch.from_numpy(Gs).to(dev()))
        fams = {k["name"] for k in plan.kernel_times()}
    assert "krylov_step" not in fams and "capacitance" in fams, fams
