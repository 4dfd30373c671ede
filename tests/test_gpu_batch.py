"""Batched plans (GPU, through the C ABI): many 1D problems (uneven n_x; fewer time steps
padded causally to the plan's n_t) solved as one block-diagonal problem must give, for every problem, the oracle's solution of that
problem alone, within the same tolerances as single solves (1e-12 FP64, 1e-10 mixed),
whatever the mix of sizes, time steps and magnitudes in the batch.

Every problem runs its own Algorithm 2, so heterogeneous batches are covered with
Algorithm 1 (alpha = 1) and Algorithm 3 (alpha = 1e-4) in both precisions.
"""
import numpy as np
import pytest

import workloads as W
from oracle import reference as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-10}


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


def _scaled(P, s):
    P.G = P.G * s
    return P


def _mix(nt):
    """Uneven n_x, different T (so different tau), operators and magnitudes 1e-6..1e4."""
    return [
        _scaled(W.heat1d_forced(255, nt, seed=1), 1.0),
        _scaled(W.heat1d_forced(127, nt, T=0.5, seed=2), 1e-6),
        _scaled(W.advdiff1d_pulse(300, nt, seed=3), 1e4),
        W.random_tridiag_problem(33, nt, seed=4),
        _scaled(W.heat1d_sine_modes(63, nt, seed=5), 3e-3),
        W.random_tridiag_problem(1, nt, seed=6),
    ]


MIXES = [("fp64", 1.0), ("fp64", 1e-4), ("mixed", 1.0), ("mixed", 1e-4)]


@pytest.mark.parametrize("prec,alpha", MIXES)
def test_batch_matches_oracle_per_problem(pd, prec, alpha):
    probs = _mix(64)
    with pd.Plan.from_problems(probs, precision=prec, alpha=alpha, device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, st = plan.solve(G)
        parts = plan.unstack(U.cpu().numpy(), [P.nx for P in probs])
    for P, Ub in zip(probs, parts):
        err = R.rel_err(Ub, R.be_solve_refined(P))
        assert err <= TOL[prec], (P.name, err, st)


@pytest.mark.parametrize("prec,alpha", MIXES)
def test_batch_member_equals_its_single_solve(pd, prec, alpha):
    probs = _mix(128)
    with pd.Plan.from_problems(probs, precision=prec, alpha=alpha, device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, _ = plan.solve(G)
        parts = plan.unstack(U.cpu().numpy(), [P.nx for P in probs])
    for P, Ub in zip(probs, parts):
        with pd.Plan.from_problem(P, precision=prec, alpha=alpha, device=dev()) as single:
            Us, _ = single.solve(torch.from_numpy(P.G).to(dev()))
        Us = Us.cpu().numpy()
        assert R.rel_err(Ub, Us) <= 2 * TOL[prec], P.name


@pytest.mark.parametrize("scales", [(1.0,) * 6, (1e-3, 1.0, 1e3, 1e-2, 10.0, 0.5)])
def test_mixed_batch_of_one_operator(pd, scales):
    """Algorithm 1 in mixed precision on a batch that shares one operator (uneven n_x,
    magnitudes 1e-3..1e3): every problem within 1e-10."""
    probs = [_scaled(W.heat1d_forced(n, 128, seed=10 + i), s) for i, (n, s) in enumerate(zip(
        (255, 255, 200, 255, 100, 255), scales))]
    for P in probs:  # one operator: the n_x = 255 heat operator, truncated
        P.k_lo, P.k_diag, P.k_up = [a[: P.nx].copy() for a in W.heat1d_operator(255)]
        P.k_up[-1] = 0.0
    with pd.Plan.from_problems(probs, precision="mixed", device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, st = plan.solve(G)
        parts = plan.unstack(U.cpu().numpy(), [P.nx for P in probs])
    for P, Ub in zip(probs, parts):
        err = R.rel_err(Ub, R.be_solve_refined(P))
        assert err <= TOL["mixed"], (P.name, err, st)


def test_batch_zero_problem_and_padding_stay_zero(pd):
    probs = _mix(32)
    probs[3].G = np.zeros_like(probs[3].G)
    with pd.Plan.from_problems(probs, precision="mixed", alpha=1e-4, device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, _ = plan.solve(G)
        V = U.cpu().numpy().reshape(plan.nt, plan.batch, plan.nx)
    assert not np.any(V[:, 3, :])
    for b, P in enumerate(probs):
        assert not np.any(V[:, b, P.nx:])  # padding rows


def test_batch_of_identical_problems_is_deterministic(pd):
    P = W.heat1d_forced(1023, 256, seed=7)
    probs = [P] * 8
    with pd.Plan.from_problems(probs, precision="mixed", device=dev()) as plan:
        G = torch.from_numpy(plan.stack([Q.G for Q in probs])).to(dev())
        U1, _ = plan.solve(G)
        U1 = U1.cpu().numpy()
        U2, _ = plan.solve(G)
        U2 = U2.cpu().numpy()
    assert np.array_equal(U1, U2)
    parts = plan.unstack(U1, [P.nx] * 8)
    ref = R.be_solve_refined(P)
    for Ub in parts:
        assert R.rel_err(Ub, ref) <= TOL["mixed"]


def _uneven_nt_mix():
    """Uneven n_x and n_t (16..256) with different tau, operators and magnitudes."""
    return [
        _scaled(W.heat1d_forced(255, 256, seed=1), 1.0),
        _scaled(W.heat1d_forced(127, 64, T=0.5, seed=2), 1e-6),
        _scaled(W.advdiff1d_pulse(300, 128, seed=3), 1e4),
        W.random_tridiag_problem(33, 16, seed=4),
        _scaled(W.heat1d_sine_modes(63, 32, seed=5), 3e-3),
        W.random_tridiag_problem(1, 256, seed=6),
    ]


@pytest.mark.parametrize("prec,alpha", MIXES)
def test_batch_of_uneven_nt_matches_oracle_per_problem(pd, prec, alpha):
    """Problems with fewer time steps ride in the longest problem's plan (zero rows of G
    past their n_t, causality of backward Euler): each one's first n_t,b rows match the
    oracle on its own n_t,b."""
    probs = _uneven_nt_mix()
    with pd.Plan.from_problems(probs, precision=prec, alpha=alpha, device=dev()) as plan:
        assert plan.nt == 256
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, st = plan.solve(G)
        parts = plan.unstack(U.cpu().numpy(), [P.nx for P in probs], [P.nt for P in probs])
    for P, Ub in zip(probs, parts):
        assert Ub.shape == (P.nt, P.nx)
        err = R.rel_err(Ub, R.be_solve_refined(P))
        assert err <= TOL[prec], (P.name, err, st)


# ----------------------------------------------------------------------------
# 2D batches: problems of one grid stacked along y (nx x (batch ny)); each keeps its own
# T_x, T_y (diffusion nu_b) and tau_b, its own DST blocks and its own Algorithm 2
# ----------------------------------------------------------------------------


def _heat2d(n, nt, T, seed, nu=1.0, scale=1.0):
    P = W.heat2d_smooth(n, nt, T=T, seed=seed)
    for name in ("k_lo", "k_diag", "k_up", "k_lo_y", "k_diag_y", "k_up_y"):
        setattr(P, name, getattr(P, name) * nu)
    P.G = P.G * scale
    return P


def _mix2d(nt, n=31):
    """One grid, different T (tau), diffusion (1e-3..1), magnitudes (1e-5..1e3) and steps."""
    return [
        _heat2d(n, nt, 0.1, seed=1),
        _heat2d(n, nt, 0.5, seed=2, nu=1e-2, scale=1e-5),
        _heat2d(n, nt // 2, 0.05, seed=3, nu=0.3, scale=1e3),
        _heat2d(n, nt, 1.0, seed=4, nu=1e-3),
    ]


@pytest.mark.parametrize("prec,alpha", MIXES)
def test_batch_2d_matches_oracle_per_problem(pd, prec, alpha):
    probs = _mix2d(32)
    with pd.Plan.from_problems(probs, precision=prec, alpha=alpha, device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, st = plan.solve(G)
        parts = plan.unstack(U.cpu().numpy(), [P.nx * P.ny for P in probs], [P.nt for P in probs])
    for P, Ub in zip(probs, parts):
        err = R.rel_err(Ub, R.be_solve_refined(P))
        assert err <= TOL[prec], (P.name, err, st)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_2d_member_equals_its_single_solve(pd, prec):
    """A 63 x 63 problem (its Algorithm 2 on 3969 entries in one CTA) gives the same U in a
    batch as alone."""
    probs = [_heat2d(63, 32, 0.1, seed=7), _heat2d(63, 32, 0.2, seed=8, nu=0.05)]
    with pd.Plan.from_problems(probs, precision=prec, device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, _ = plan.solve(G)
        parts = plan.unstack(U.cpu().numpy(), [P.nx * P.ny for P in probs])
    for P, Ub in zip(probs, parts):
        with pd.Plan.from_problem(P, precision=prec, device=dev()) as single:
            Us, _ = single.solve(torch.from_numpy(P.G).to(dev()))
        assert R.rel_err(Ub, Us.cpu().numpy()) <= 2 * TOL[prec], P.name
        assert R.rel_err(Ub, R.be_solve_refined(P)) <= TOL[prec], P.name


@pytest.mark.parametrize("dim", [1, 2])
def test_unused_slots_leave_the_refinement_decision_alone(pd, dim):
    """An unused slot (zero right-hand side) is solved exactly by zero; the rounding-level
    values the paired real DFTs leave in its columns must not enter the refinement decision:
    a problem with an unused slot beside it refines like the problem alone (same sweeps,
    same recorded updates) and its slot stays exactly zero."""
    import workloads.serving as S

    if dim == 1:
        P = W.heat1d_forced(1023, 256, seed=1)
        empty = S.empty_slot(P.nt)
        kw = {"nx": P.nx}
    else:
        P = _heat2d(63, 32, 0.1, seed=9, nu=0.1)
        empty = S.empty_slot(P.nt, P.nx, P.ny)
        kw = {}
    with pd.Plan.from_problem(P, precision="mixed", device=dev()) as plan:
        _, st1 = plan.solve(torch.from_numpy(P.G).to(dev()))
    with pd.Plan.from_problems([P, empty], precision="mixed", device=dev(), **kw) as plan:
        G = torch.from_numpy(plan.stack([P.G])).to(dev())
        U, st = plan.solve(G)
        Ub = U.cpu().numpy().reshape(plan.nt, 2, plan.slot)
    assert R.rel_err(Ub[:, 0, :P.nx * P.ny], R.be_solve_refined(P)) <= TOL["mixed"], st
    assert not np.any(Ub[:, 1])
    n = st["refine_sweeps"]
    upd, upd1 = st["sweep_rel_update"][:n], st1["sweep_rel_update"][:st1["refine_sweeps"]]
    assert n <= st1["refine_sweeps"] + 1, (upd, upd1)
    # each refinement sweep records the problem's own contraction (the unused slot's
    # rounding noise, relative to its own noise, would record ~1 and stall the decision)
    assert all(u < 1e-2 for u in upd[1:]), (upd, upd1)
