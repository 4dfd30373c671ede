"""Host logic of the solver service (no GPU): request streams and the scheduler's
grouping and admission rules."""
import workloads.serving as S
from paper_2304_12597_gb300.serve import NX_CLASSES, BatchKey, Scheduler, capacity_for, key_of, size_class


def test_request_stream_is_seeded_and_in_range():
    a = S.request_stream(200, 500.0, seed=3)
    b = S.request_stream(200, 500.0, seed=3)
    assert [(r.kind, r.nx, r.nt, r.nu, r.seed, r.arrival) for r in a] == \
           [(r.kind, r.nx, r.nt, r.nu, r.seed, r.arrival) for r in b]
    assert all(a[i].arrival < a[i + 1].arrival for i in range(len(a) - 1))
    for r in a:
        assert r.nt in (32, 64, 128, 256, 512, 1024, 2048)
        assert 1e-4 <= r.nu <= 1.0
        if r.kind == "heat2d":
            assert r.nx == r.ny and r.nx in S.SIDES_2D
        else:
            assert 127 <= r.nx <= 4095 and r.ny == 1
    # mean inter-arrival ~ 1/rate
    assert abs(a[-1].arrival / len(a) - 1 / 500.0) < 0.5 / 500.0


def test_size_classes_and_capacity():
    assert size_class(127) == 128 and size_class(128) == 128 and size_class(129) == 256
    assert size_class(4095) == NX_CLASSES[-1]
    assert [capacity_for(c, 32) for c in (1, 2, 3, 5, 16, 17, 40)] == [2, 2, 4, 8, 16, 32, 32]


def _req(rid, kind, nx, nt, t):
    ny = nx if kind == "heat2d" else 1
    return S.Request(rid=rid, arrival=t, kind=kind, nx=nx, ny=ny, nt=nt, nu=0.1, seed=rid)


def test_scheduler_groups_by_key_in_arrival_order():
    sch = Scheduler(budget=1 << 40, workspace_bytes=lambda k, c: 1000, max_batch=4)
    reqs = [_req(0, "heat1d", 300, 64, 0.0), _req(1, "heat1d", 500, 64, 0.1), _req(2, "advdiff1d", 260, 64, 0.2),
            _req(3, "heat2d", 63, 64, 0.3), _req(4, "heat1d", 400, 128, 0.4), _req(5, "heat1d", 511, 64, 0.5),
            _req(6, "heat1d", 270, 64, 0.6), _req(7, "heat1d", 290, 64, 0.7), _req(8, "heat1d", 280, 64, 0.8)]
    for r in reqs:
        sch.add(r)
    b1 = sch.next_batch()
    # key of request 0: 1D, nt 64, class 512 -> 0, 1, 2, 5 (first four of that key)
    assert b1.key == BatchKey(1, 64, 512, 1) and [r.rid for r in b1.requests] == [0, 1, 2, 5] and b1.cap == 4
    b2 = sch.next_batch()
    # a 63 x 63 grid shares a batched plan (capacity 2 at least); 127 x 127 runs alone
    assert b2.key.dim == 2 and [r.rid for r in b2.requests] == [3] and b2.cap == 2
    b3 = sch.next_batch()
    assert [r.rid for r in b3.requests] == [4] and b3.cap == 2
    b4 = sch.next_batch()
    assert [r.rid for r in b4.requests] == [6, 7, 8] and b4.cap == 4
    assert sch.next_batch() is None
    for b in (b1, b2, b3, b4):
        sch.release(b)
    assert sch.in_flight == 0


def test_scheduler_admission_waits_for_memory():
    per = lambda k, c: 10_000  # noqa: E731
    sch = Scheduler(budget=1, workspace_bytes=per, max_batch=8)  # nothing fits beside another batch
    for i in range(3):
        sch.add(_req(i, "heat1d", 200, 32, 0.01 * i))
    b1 = sch.next_batch()  # an idle device always takes the head batch
    assert b1 is not None and len(b1.requests) == 3
    sch.add(_req(9, "heat1d", 200, 32, 1.0))
    assert sch.next_batch() is None  # budget exhausted while b1 is in flight
    sch.release(b1)
    b2 = sch.next_batch()
    assert [r.rid for r in b2.requests] == [9]


def test_key_of():
    assert key_of(_req(0, "heat2d", 127, 256, 0)) == BatchKey(2, 256, 127, 127)
    assert key_of(_req(0, "advdiff1d", 1025, 256, 0)) == BatchKey(1, 256, 2048, 1)


def test_device_rhs_equals_the_host_problem():
    """The service builds G with torch on its device; on the CPU device it must equal the
    numpy right-hand side of request_problem (which the parity tests give the oracle), for
    every request kind, also when written into the first columns of a wider buffer."""
    import numpy as np
    import torch

    reqs = [_req(1, "heat1d", 300, 32, 0.0), _req(2, "advdiff1d", 257, 64, 0.0), _req(3, "heat2d", 63, 32, 0.0)]
    for r in reqs:
        G = S.request_problem(r).G
        Gd = S.rhs_device(r, torch, torch.device("cpu")).numpy()
        assert Gd.shape == G.shape
        assert np.linalg.norm(Gd - G) <= 1e-13 * np.linalg.norm(G)
        out = torch.full((r.nt, G.shape[1] + 5), 7.0, dtype=torch.float64)
        S.rhs_device(r, torch, torch.device("cpu"), out=out)
        assert np.linalg.norm(out[:, : G.shape[1]].numpy() - G) <= 1e-13 * np.linalg.norm(G)
        assert bool((out[:, G.shape[1]:] == 7.0).all())  # columns past the request untouched


def test_slot_operators():
    r = _req(4, "heat1d", 200, 64, 0.0)
    op = S.request_problem_operator_only(r, 256)
    assert (op.nx, op.nt) == (200, 64) and op.k_diag.shape == (200,)
    import pytest

    with pytest.raises(ValueError):
        S.request_problem_operator_only(r, 128)
    e = S.empty_slot(64)
    assert (e.nx, e.nt) == (1, 64) and e.k_diag[0] == 1.0 and e.k_lo[0] == 0.0 and e.k_up[0] == 0.0
    r2 = _req(5, "heat2d", 63, 32, 0.0)
    op2 = S.request_problem_operator_only(r2, 63)
    assert (op2.dim, op2.nx, op2.ny) == (2, 63, 63) and op2.k_diag_y.shape == (63,)
    with pytest.raises(ValueError):
        S.request_problem_operator_only(r2, 127)
    e2 = S.empty_slot(32, 63, 63)
    assert (e2.dim, e2.nx, e2.ny, e2.nt) == (2, 63, 63, 32) and e2.k_diag_y.shape == (63,)


def test_scheduler_batches_small_2d_grids_only():
    from paper_2304_12597_gb300.serve import Scheduler

    sch = Scheduler(budget=1 << 40, workspace_bytes=lambda k, c: 1000, max_batch=8)
    for i, side in enumerate((63, 127, 63, 127, 63)):
        sch.add(_req(i, "heat2d", side, 32, 0.1 * i))
    b1 = sch.next_batch()
    assert [r.rid for r in b1.requests] == [0, 2, 4] and b1.cap == 4
    b2 = sch.next_batch()
    assert [r.rid for r in b2.requests] == [1] and b2.cap == 1  # 16129 points: one per plan
    b3 = sch.next_batch()
    assert [r.rid for r in b3.requests] == [3] and b3.cap == 1


def test_scheduler_take_hands_same_key_requests_to_a_running_batch():
    """Requests joining a running batch: take(key, n) removes up to n waiting requests of
    that key, in arrival order, and leaves every other request (and the memory count) as
    it was."""
    sched = Scheduler(budget=1 << 40, workspace_bytes=lambda k, c: 1000, max_batch=4)
    reqs = [_req(0, "heat1d", 200, 64, 0.0), _req(1, "heat1d", 900, 64, 0.1), _req(2, "heat1d", 210, 64, 0.2),
            _req(3, "heat1d", 220, 64, 0.3), _req(4, "heat1d", 230, 128, 0.4)]
    for r in reqs:
        sched.add(r)
    key = key_of(reqs[0])
    before = sched.in_flight
    got = sched.take(key, 2)
    assert [r.rid for r in got] == [0, 2]
    assert [r.rid for r in sched.waiting] == [1, 3, 4]
    assert sched.take(key, 0) == [] and sched.in_flight == before
    assert [r.rid for r in sched.take(key, 5)] == [3]
    assert [r.rid for r in sched.waiting] == [1, 4]
