"""Host logic of the service's continuous batching (CPU, no GPU): a stand-in plan whose
problems converge a fixed number of calls after they join lets the tests follow which
request sits in which slot, when waiting requests join a running batch, that every request
finishes exactly once, and that a failing call fails its batch without stopping the
service."""
import threading
from collections import OrderedDict
from dataclasses import dataclass

import pytest

import workloads.serving as S
from paper_2304_12597_gb300 import serve as SV

torch = pytest.importorskip("torch")


class FakePlan:
    """Slots converge `need` calls after they join; optional failures on a given call."""

    def __init__(self, cap, need=3, fail_advance_at=None, fail_set_at=None):
        self.cap, self.need = cap, need
        self.age = [None] * cap
        self.calls = 0
        self.sets = 0
        self.fail_advance_at, self.fail_set_at = fail_advance_at, fail_set_at
        self.closed = False
        self.log = []

    def set_problems(self, probs):
        self.sets += 1
        if self.fail_set_at is not None and self.sets == self.fail_set_at:
            raise RuntimeError("set_operator failed")
        assert len(probs) == self.cap

    def advance(self, G, U, join, steps=1):
        self.calls += 1
        if self.fail_advance_at is not None and self.calls == self.fail_advance_at:
            raise RuntimeError("advance failed")
        Gv = G.view(G.shape[0], self.cap, -1)
        state = []
        for b in range(self.cap):
            occupied = bool(Gv[:, b, :].abs().sum() > 0)
            if join[b]:
                assert occupied, "a joining slot has its right-hand side"
                self.age[b] = 0
            if not occupied:
                self.age[b] = None
            if self.age[b] is not None:
                self.age[b] += 1
                U.view(U.shape[0], self.cap, -1)[:, b, :] = Gv[:, b, :]  # "solution": a copy of G
            state.append(1 if self.age[b] is not None and self.age[b] >= self.need else 0)
        self.log.append((list(join), state))
        return state, {"refine_sweeps": 1}

    def close(self):
        self.closed = True


@dataclass
class FakeSlot:
    plan: object
    G: object
    U: object
    bytes: int


def _server(monkeypatch, plans, **kw):
    server = SV.Server(device="cpu", workers=kw.pop("workers", 1), keep_results="full", **kw)
    server._workers = [(None, OrderedDict()) for _ in range(server.workers)]
    monkeypatch.setattr(server, "_workspace_bytes", lambda key, cap: 1000)

    def slot(cache, batch, stream):
        k = (batch.key, batch.cap)
        if k not in cache:
            width = batch.key.nx * batch.key.ny
            G = torch.zeros((batch.key.nt, batch.cap * width), dtype=torch.float64)
            plan = plans(batch.cap)
            cache[k] = FakeSlot(plan, G, torch.zeros_like(G), batch.bytes)
            return cache[k], True
        return cache[k], False

    monkeypatch.setattr(server, "_slot", slot)
    return server


def _same_key_requests(n):
    reqs = S.request_stream(n, 1e6, seed=3, kinds=("heat1d",), nx_range=(200, 250), nt_choices=(32,))
    for r in reqs:
        r.arrival = 0.0
    return reqs


def _run_with_deadline(server, reqs, seconds=30):
    out = {}
    t = threading.Thread(target=lambda: out.setdefault("stats", server.run(reqs)), daemon=True)
    t.start()
    t.join(seconds)
    assert not t.is_alive(), "the service did not finish"
    return out["stats"]


def test_waiting_requests_join_the_running_batch(monkeypatch):
    plans = []
    server = _server(monkeypatch, lambda cap: plans.append(FakePlan(cap)) or plans[-1], max_batch=2)
    reqs = _same_key_requests(6)
    stats = _run_with_deadline(server, reqs)
    summ = stats.summary()
    assert summ["failed"] == 0 and summ["requests"] == 6
    assert stats.batches == 1 and len(plans) == 1  # one running batch served all six
    assert summ["joined_running"] == 4
    for r in reqs:  # every result is its own right-hand side (the stand-in's "solution")
        G = S.rhs_device(r, torch, "cpu").numpy()
        assert r.result.shape == (r.nt, r.nx) and (r.result == G).all(), r.rid
    # a slot is joined only when free, and a joining slot starts its own count
    p = plans[0]
    assert p.log[0][0] == [1, 1]
    assert any(j == [1, 1] for j, _ in p.log[1:])


def test_failed_call_fails_its_batch_and_the_service_goes_on(monkeypatch):
    plans = []
    # the first plan fails at its second call; the plan that replaces it works
    make = lambda cap: plans.append(FakePlan(cap, fail_advance_at=2 if not plans else None)) or plans[-1]  # noqa
    server = _server(monkeypatch, make, max_batch=2)
    reqs = _same_key_requests(5)
    stats = _run_with_deadline(server, reqs)
    summ = stats.summary()
    assert summ["requests"] == 5
    failed = [r for r in reqs if r.error]
    assert len(failed) == 2 and all("advance failed" in r.error for r in failed)
    assert plans[0].closed and len(plans) == 2  # the plan that failed is dropped and replaced
    assert all(r.done is not None for r in reqs)
    assert all(r.result is not None for r in reqs if not r.error)


def test_failed_operator_swap_fails_the_joining_requests(monkeypatch):
    plans = []
    make = lambda cap: plans.append(FakePlan(cap, fail_set_at=2 if not plans else None)) or plans[-1]  # noqa
    server = _server(monkeypatch, make, max_batch=2)
    reqs = _same_key_requests(4)
    stats = _run_with_deadline(server, reqs)
    assert stats.summary()["requests"] == 4
    failed = [r for r in reqs if r.error]
    assert failed and all("service:" in r.error and r.joined_running for r in failed)
    assert all(r.done is not None for r in reqs)
