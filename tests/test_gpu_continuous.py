"""Problems joining a running batched solve (paradiag_batch_advance; GPU, through the C ABI).

A batched plan advances every problem by refinement sweeps, one call at a time; a problem
joins between calls (its slot of U restarts at zero, its refinement counts from its own
first solve) and leaves once its state says converged.  Every problem's result must meet
the oracle's bar (1e-10 mixed, 1e-12 FP64) and equal the same problem solved alone within
twice that, whenever it joined and whoever shared the batch with it.
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


def _problems(nt=64):
    return [W.heat1d_forced(255, nt, seed=1), W.advdiff1d_pulse(200, nt, seed=2),
            W.heat1d_forced(127, nt, T=0.5, seed=3), W.random_tridiag_problem(33, nt, seed=4),
            W.heat1d_sine_modes(63, nt, seed=5)]


def _alone(pd, P, prec):
    with pd.Plan.from_problem(P, precision=prec, device=dev()) as plan:
        U, _ = plan.solve(torch.from_numpy(P.G).to(dev()))
    return U.cpu().numpy()


def _put(plan, G, b, P):
    """Problem P's right-hand side into slot b of G (zero-padded), or zeros if P is None."""
    V = G.view(plan.nt, plan.batch, plan.slot)
    V[:, b, :] = 0.0
    if P is not None:
        V[:P.nt, b, :P.nx] = torch.from_numpy(P.G).to(dev())


def _slot(plan, U, b, P):
    return U.view(plan.nt, plan.batch, plan.slot)[:P.nt, b, :P.nx].cpu().numpy()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_problems_join_and_leave_a_running_batch(pd, prec):
    """Slots 0 and 1 start; slot 2 joins after one sweep; when slot 0's problem has
    converged it leaves and a new problem (another operator, swapped in with
    set_problems) takes its slot; every result meets the bars."""
    A, B, C, D, E = _problems()
    results = {}
    with pd.Plan.from_problems([A, B, C, D], precision=prec, device=dev()) as plan:
        G = torch.zeros((plan.nt, plan.nbar), dtype=torch.float64, device=dev())
        U = torch.zeros_like(G)
        occupant = [A, B, None, None]
        _put(plan, G, 0, A)
        _put(plan, G, 1, B)
        join = [1, 1, 0, 0]
        e_joined = False
        for call in range(1, 41):
            state, st = plan.advance(G, U, join, steps=1)
            assert st["refine_sweeps"] == 1
            join = [0] * plan.batch
            for b, P in enumerate(occupant):
                assert P is None or state[b] != 2, (b, state)
                if P is not None and state[b] == 1:
                    results[P.name] = _slot(plan, U, b, P)
                    occupant[b] = None
                    _put(plan, G, b, None)  # it leaves: the slot is unused from the next call
            if call == 1:  # C joins a batch whose problems have had one solve
                occupant[2] = C
                _put(plan, G, 2, C)
                join[2] = 1
            if occupant[0] is None and not e_joined:  # E takes A's slot, with its own operator
                plan.set_problems([E, B, C, D])
                occupant[0] = E
                _put(plan, G, 0, E)
                join[0] = 1
                e_joined = True
            if e_joined and all(o is None for o in occupant):
                break
    assert set(results) == {A.name, B.name, C.name, E.name}, list(results)
    for P in (A, B, C, E):
        U_b = results[P.name]
        assert R.rel_err(U_b, R.be_solve_refined(P)) <= TOL[prec], P.name
        assert R.rel_err(U_b, _alone(pd, P, prec)) <= 2 * TOL[prec], P.name


def test_join_equals_batch_solve(pd):
    """All problems joining at the first call and advanced to convergence give what one
    paradiag_solve of the batch gives, within the bar."""
    probs = _problems()[:4]
    with pd.Plan.from_problems(probs, precision="mixed", device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U = torch.zeros_like(G)
        join = [1] * plan.batch
        for _ in range(20):
            state, _ = plan.advance(G, U, join, steps=2)
            join = [0] * plan.batch
            if all(s == 1 for s in state):
                break
        assert all(s == 1 for s in state), state
        U1, _ = plan.solve(G)
        for b, P in enumerate(probs):
            assert R.rel_err(_slot(plan, U, b, P), _slot(plan, U1, b, P)) <= 2 * TOL["mixed"], P.name


def test_member_gives_up_after_its_solves(pd):
    """max_refine = 1: a problem may take two solves; the mixed path needs three to meet
    refine_tol, so its state turns 2 at its second call, counted from its own join."""
    probs = _problems()[:2]
    with pd.Plan.from_problems(probs, precision="mixed", max_refine=1, device=dev()) as plan:
        G = torch.zeros((plan.nt, plan.nbar), dtype=torch.float64, device=dev())
        U = torch.zeros_like(G)
        _put(plan, G, 0, probs[0])
        s1, _ = plan.advance(G, U, [1, 0], steps=1)
        _put(plan, G, 1, probs[1])
        s2, _ = plan.advance(G, U, [0, 1], steps=1)
        s3, _ = plan.advance(G, U, [0, 0], steps=1)
    assert s1[0] == 0 and s2[0] == 2 and s2[1] == 0 and s3[1] == 2, (s1, s2, s3)


def test_advance_rejects_single_problems_and_bad_steps(pd):
    P = _problems()[0]
    G = torch.from_numpy(P.G).to(dev())
    U = torch.zeros_like(G)
    with pd.Plan.from_problem(P, precision="mixed", device=dev()) as plan:
        with pytest.raises(ValueError):
            plan.advance(G, U, [1, 0], steps=1)
        with pytest.raises(pd.ParadiagError) as e:
            plan.advance(G, U, [1], steps=1)
        assert e.value.status_name == "PD_ERR_INVALID_ARG"
    probs = _problems()[:2]
    with pd.Plan.from_problems(probs, precision="mixed", device=dev()) as plan:
        G = torch.zeros((plan.nt, plan.nbar), dtype=torch.float64, device=dev())
        with pytest.raises(pd.ParadiagError) as e:
            plan.advance(G, torch.zeros_like(G), [1, 1], steps=0)
        assert e.value.status_name == "PD_ERR_INVALID_ARG"
