"""The solver service on the GPU: requests of mixed kind and size, arriving together,
are batched and run on two streams, and requests join running batches between sweeps;
every request's result must equal the result of the same request solved alone, and the
oracle's, within the mixed-precision tolerance 1e-10."""
import numpy as np
import pytest

import workloads.serving as S
from oracle import reference as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as entry

    entry.build()
    import paper_2304_12597_gb300 as pkg

    return pkg


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("alpha", [1e-4, 1.0])
def test_served_results_equal_alone_and_oracle(pd, alpha):
    """Algorithm 3 (alpha = 1e-4, the service's default) and Algorithm 1 (alpha = 1).  The
    whole trajectory U of every request is compared (relative Frobenius norm, the accuracy
    contract of the mixed path)."""
    from paper_2304_12597_gb300.serve import Server

    reqs = S.request_stream(24, 1e5, seed=11, nx_range=(127, 700), nt_choices=(32, 64))
    server = Server(device="cuda:0", workers=2, max_batch=8, keep_results="full", budget_bytes=8 << 30, alpha=alpha)
    stats = server.run(reqs)
    server.close()
    summ = stats.summary()
    assert summ["failed"] == 0, [r.error for r in reqs if r.error]
    assert max(r.batch for r in reqs) > 1  # some requests shared a batch
    dev = torch.device("cuda:0")
    for r in reqs:
        P = S.request_problem(r)
        with pd.Plan.from_problem(P, precision="mixed", alpha=server.alpha, device=dev) as plan:
            U, _ = plan.solve(S.rhs_device(r, torch, dev).contiguous())
            alone = U.cpu().numpy().reshape(r.result.shape)
        assert _rel(r.result, alone) <= 2 * TOL, (r.rid, r.kind, r.batch)
    for r in reqs[:6]:
        P = S.request_problem(r)
        ref = R.be_solve_refined(P).reshape(r.result.shape)
        assert _rel(r.result, ref) <= TOL, (r.rid, r.kind)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


def test_served_2d_requests_share_a_batch(pd):
    """2D requests on one 63 x 63 grid (different nu, n_t and forcing) share a batched plan;
    each request's trajectory equals its solve alone and the oracle's."""
    from paper_2304_12597_gb300.serve import Server

    reqs = S.request_stream(6, 1e5, seed=21, kinds=("heat2d",), nt_choices=(32,), sides_2d=(63,))
    server = Server(device="cuda:0", workers=1, max_batch=8, keep_results="full", budget_bytes=8 << 30, alpha=1.0)
    stats = server.run(reqs)
    server.close()
    assert stats.summary()["failed"] == 0, [r.error for r in reqs if r.error]
    assert max(r.batch for r in reqs) > 1
    dev = torch.device("cuda:0")
    for r in reqs:
        P = S.request_problem(r)
        with pd.Plan.from_problem(P, precision="mixed", alpha=1.0, device=dev) as plan:
            U, _ = plan.solve(S.rhs_device(r, torch, dev).contiguous())
        assert _rel(r.result, U.cpu().numpy().reshape(r.result.shape)) <= 2 * TOL, (r.rid, r.batch)
        ref = R.be_solve_refined(P).reshape(r.result.shape)
        assert _rel(r.result, ref) <= TOL, r.rid



@pytest.mark.parametrize("kind,side", [("heat1d", 0), ("heat2d", 63)])
def test_requests_join_a_running_batch(pd, kind, side):
    """One worker and batches of two: the first two requests start a batch, and the others
    (same shape, queued behind them) join it as its problems converge and leave, between
    sweeps, instead of waiting for it to end.  Every trajectory equals its solve alone and
    the oracle's."""
    from paper_2304_12597_gb300.serve import Server

    kw = dict(kinds=(kind,), nt_choices=(64,))
    if kind == "heat2d":
        kw["sides_2d"] = (side,)
    else:
        kw["nx_range"] = (200, 250)
    reqs = S.request_stream(5, 1e5, seed=41, **kw)
    server = Server(device="cuda:0", workers=1, max_batch=2, keep_results="full", budget_bytes=8 << 30, alpha=1.0)
    stats = server.run(reqs)
    server.close()
    assert stats.summary()["failed"] == 0, [r.error for r in reqs if r.error]
    assert stats.batches == 1, stats.batches  # one running batch served all five
    assert sum(r.joined_running for r in reqs) >= 3  # at most two started it
    dev = torch.device("cuda:0")
    for r in reqs:
        P = S.request_problem(r)
        with pd.Plan.from_problem(P, precision="mixed", alpha=1.0, device=dev) as plan:
            U, _ = plan.solve(S.rhs_device(r, torch, dev).contiguous())
        assert _rel(r.result, U.cpu().numpy().reshape(r.result.shape)) <= 2 * TOL, (r.rid, r.joined_running)
        ref = R.be_solve_refined(P).reshape(r.result.shape)
        assert _rel(r.result, ref) <= TOL, r.rid
