"""A diagonal mass matrix M on the GPU (through the C ABI): (B (x) M + I (x) K) u = f, each
step (M + tau K) u_j = M u_{j-1} + G_j.  The plan solves for w = M^{1/2} u with
K' = M^{-1/2} K M^{-1/2}; the result must equal the oracle's sequential solve with M
(which handles M directly), within 1e-12 (FP64) and 1e-10 (mixed)."""
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


def _problems():
    return [W.with_mass(W.random_tridiag_problem(300, 16, seed=1), seed=2),
            W.with_mass(W.heat1d_forced(1023, 64, seed=3), seed=4, lo=0.25, hi=4.0),
            W.with_mass(W.advdiff1d_pulse(511, 32, seed=5), seed=6),
            W.with_mass(W.random_tridiag_problem(1, 4, seed=7), seed=8)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("P", _problems(), ids=lambda p: p.name)
def test_mass_matrix_solve_matches_oracle(pd, prec, P):
    ref = R.be_solve_refined(P)
    with pd.Plan.from_problem(P, precision=prec, device=dev()) as plan:
        U, st = plan.solve(torch.from_numpy(P.G).to(dev()))
        U = U.cpu().numpy()
    assert R.rel_err(U, ref) <= TOL[prec], st
    # M matters: the unit-mass solution is far from it (well beyond the tolerance)
    Q = W.with_mass(P, seed=0)
    Q.m_diag = None
    assert R.rel_err(U, R.be_solve(Q)) > 1e4 * TOL[prec]


@pytest.mark.parametrize("prec,alpha", [("mixed", 1.0), ("fp64", 1e-4)])
def test_mass_matrix_batch_matches_oracle_per_problem(pd, prec, alpha):
    probs = [W.with_mass(W.heat1d_forced(255, 64, seed=1), seed=1),
             W.heat1d_forced(200, 64, T=0.5, seed=2),  # no mass matrix: identity in its slot
             W.with_mass(W.advdiff1d_pulse(300, 64, seed=3), seed=3, lo=0.2, hi=3.0)]
    with pd.Plan.from_problems(probs, precision=prec, alpha=alpha, device=dev()) as plan:
        G = torch.from_numpy(plan.stack([P.G for P in probs])).to(dev())
        U, st = plan.solve(G)
        parts = plan.unstack(U.cpu().numpy(), [P.nx for P in probs])
    for P, Ub in zip(probs, parts):
        assert R.rel_err(Ub, R.be_solve_refined(P)) <= TOL[prec], (P.name, st)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_set_operator_swaps_the_mass_matrix(pd, prec):
    A = W.with_mass(W.heat1d_forced(255, 64, seed=1), seed=1)
    B = W.with_mass(W.heat1d_forced(255, 64, seed=2), seed=9, lo=0.3, hi=3.0)
    with pd.Plan.from_problem(A, precision=prec, device=dev()) as plan:
        Ua, _ = plan.solve(torch.from_numpy(A.G).to(dev()))
        plan.set_operator(tau=B.tau, k_lo=B.k_lo, k_diag=B.k_diag, k_up=B.k_up, m_diag=B.m_diag)
        Ub, st = plan.solve(torch.from_numpy(B.G).to(dev()))
        # no mass matrix in the descriptor: identity
        C = W.heat1d_forced(255, 64, seed=2)
        plan.set_operator(tau=C.tau, k_lo=C.k_lo, k_diag=C.k_diag, k_up=C.k_up)
        Uc, _ = plan.solve(torch.from_numpy(C.G).to(dev()))
    assert R.rel_err(Ua.cpu().numpy(), R.be_solve_refined(A)) <= TOL[prec]
    assert R.rel_err(Ub.cpu().numpy(), R.be_solve_refined(B)) <= TOL[prec], st
    assert R.rel_err(Uc.cpu().numpy(), R.be_solve_refined(C)) <= TOL[prec]


def test_mass_matrix_host_io(pd):
    P = W.with_mass(W.heat1d_forced(127, 32, seed=4), seed=5)
    with pd.Plan.from_problem(P, precision="mixed", host_io=True, device=dev()) as plan:
        Gh = torch.from_numpy(P.G.copy()).pin_memory()
        Uh = torch.empty_like(Gh).pin_memory()
        plan.solve_host(Gh, Uh)
    assert R.rel_err(Uh.numpy(), R.be_solve_refined(P)) <= TOL["mixed"]
