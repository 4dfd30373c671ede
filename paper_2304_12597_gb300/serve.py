"""A continuous-batching solver service on top of the C ABI.

Requests (workloads.serving.Request: kind, n_x, n_y, n_t, nu, forcing seed) arrive
over time.  The scheduler groups the waiting ones into batches, and worker threads
(one CUDA stream each) run them, so several batches are on the device at once:
- 1D requests with one n_t and n_x in one size class share a batched plan (problem b in
  slot b, zero-padded to the class's n_x);
- 2D requests with one n_t and grid share a batched plan when the grid has at most 8192
  points (each problem's Algorithm 2 then runs in one CTA); larger grids run one per plan.
A batched plan is advanced one refinement sweep at a time (paradiag_batch_advance): between
sweeps, problems that have converged leave their slots and waiting requests of the same
shape join the running batch in the free slots (continuous batching); other requests
start a new batch as soon as a worker and enough device memory are free.  Large 2D
grids run one per plan, solved whole.  Admission is by an HBM budget that counts
the workspace, G and U of every batch in flight; idle cached plans (up to
plan_cache_bytes, half the budget by default) come on top of it, so the service can hold
about 1.5 times budget_bytes of device memory.

Plans are cached per (shape, capacity) and worker; a new batch swaps its operators in
with paradiag_set_operator, so the workspace and the captured CUDA graph are reused.
Requests span diffusion coefficients down to 1e-4, where Algorithm 1's inner system is
ill-conditioned (kappa <= 1 + 1/(tau lambda_min), Theorem 3.1); the service therefore
runs Algorithm 3 with alpha = 1e-4 by default (mixed precision refines away the
kappa(F D_alpha) loss).
All arithmetic of a solve runs in the library's kernels; this module only schedules.
"""
from __future__ import annotations

import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np

NX_CLASSES = (128, 256, 512, 1024, 2048, 4096)
GRID_2D_BATCHED = 8192  # largest 2D grid (n_x n_y) that shares a batched plan


def size_class(nx: int) -> int:
    for c in NX_CLASSES:
        if nx <= c:
            return c
    raise ValueError(f"n_x = {nx} is above the largest size class")


def next_pow2(v: int) -> int:
    p = 1
    while p < v:
        p <<= 1
    return p


@dataclass(frozen=True)
class BatchKey:
    dim: int
    nt: int
    nx: int  # slot length (1D: size class; 2D: grid side)
    ny: int


def key_of(req) -> BatchKey:
    if req.dim == 2:
        return BatchKey(2, req.nt, req.nx, req.ny)
    return BatchKey(1, req.nt, size_class(req.nx), 1)


def capacity_for(count: int, max_batch: int) -> int:
    """Slots of the plan that serves `count` 1D requests (a power of two >= 2, so that
    one plan shape serves a range of batch sizes)."""
    return max(2, min(next_pow2(count), max_batch))


def batch_bytes(key: BatchKey, cap: int, workspace_bytes: Callable[[BatchKey, int], int]) -> int:
    """Device bytes of one batch in flight: workspace plus G and U."""
    return workspace_bytes(key, cap) + 2 * 8 * key.nt * key.nx * key.ny * cap


@dataclass
class Batch:
    key: BatchKey
    cap: int
    requests: list
    bytes: int


class Scheduler:
    """Waiting requests and the admission rule (host logic only; no GPU).

    next_batch() takes the oldest waiting request, collects up to `max_batch` waiting
    requests of its key in arrival order (2D: one), and admits the batch if the bytes
    in flight stay within `budget`; otherwise nothing is admitted (the oldest request
    keeps its place at the head of the queue).
    """

    def __init__(self, budget: int, workspace_bytes: Callable[[BatchKey, int], int], max_batch: int = 32):
        self.budget = budget
        self.workspace_bytes = workspace_bytes
        self.max_batch = max_batch
        self.waiting: list = []
        self.in_flight = 0

    def add(self, req) -> None:
        self.waiting.append(req)

    def next_batch(self) -> Optional[Batch]:
        if not self.waiting:
            return None
        head = self.waiting[0]
        key = key_of(head)
        if key.dim == 2 and key.nx * key.ny > GRID_2D_BATCHED:
            group = [head]
            cap = 1
        else:
            group = [r for r in self.waiting if key_of(r) == key][: self.max_batch]
            cap = capacity_for(len(group), self.max_batch)
        need = batch_bytes(key, cap, self.workspace_bytes)
        if self.in_flight > 0 and self.in_flight + need > self.budget:
            return None  # wait for memory (a batch that fits nowhere still runs alone)
        ids = {id(r) for r in group}
        self.waiting = [r for r in self.waiting if id(r) not in ids]
        self.in_flight += need
        return Batch(key, cap, group, need)

    def take(self, key: BatchKey, n: int) -> list:
        """Up to n waiting requests of `key` in arrival order, removed from the queue (they
        join a running batch, whose memory is already counted)."""
        if n <= 0:
            return []
        group = [r for r in self.waiting if key_of(r) == key][:n]
        ids = {id(r) for r in group}
        self.waiting = [r for r in self.waiting if id(r) not in ids]
        return group

    def release(self, batch: Batch) -> None:
        self.in_flight -= batch.bytes


@dataclass
class _Slot:
    plan: object
    G: object
    U: object
    bytes: int


@dataclass
class ServeStats:
    requests: int = 0
    failed: int = 0
    batches: int = 0
    elapsed_s: float = 0.0
    unknowns: int = 0
    joined: int = 0  # requests admitted into a batch that was already running
    latencies_ms: list = field(default_factory=list)

    def summary(self) -> dict:
        lat = np.array(self.latencies_ms) if self.latencies_ms else np.zeros(1)
        return {"requests": self.requests, "failed": self.failed, "batches": self.batches, "joined_running": self.joined,
                "mean_batch": self.requests / max(self.batches, 1), "elapsed_s": self.elapsed_s,
                "solves_per_s": self.requests / max(self.elapsed_s, 1e-9),
                "unknowns_per_s": self.unknowns / max(self.elapsed_s, 1e-9),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "max_ms": float(lat.max())}


class Server:
    """Runs a request stream in real time on one GPU with `workers` CUDA streams."""

    def __init__(self, device=None, precision="mixed", workers=2, budget_bytes=40 << 30, max_batch=32,
                 keep_results=False, plan_cache_bytes=None, alpha=1e-4, continuous=True):
        import torch

        from . import _binding as B
        from .plan import Plan

        self.torch, self.B, self.Plan = torch, B, Plan
        self.device = torch.device(device) if device is not None else torch.device("cuda", 0)
        self.precision = precision
        self.alpha = alpha  # Algorithm 3: slow diffusion (nu ~ 1e-4) needs it (Sec. 4)
        self.workers = workers
        self.keep_results = keep_results
        # batched plans advance sweep by sweep and take new requests into free slots
        self.continuous = continuous
        self.plan_cache_bytes = plan_cache_bytes if plan_cache_bytes is not None else budget_bytes // 2
        self._ws_cache: dict = {}
        self.sched = Scheduler(budget_bytes, self._workspace_bytes, max_batch)
        self.cv = threading.Condition()
        self._workers: list = []  # (stream, plan cache) per worker, kept across runs

    def close(self) -> None:
        """Release every cached plan."""
        for _, cache in self._workers:
            for s in cache.values():
                s.plan.close()
            cache.clear()

    def warmup(self, n: int = 300, seed: int = 987654321) -> None:
        """Serve a throw-away stream (all arriving at once) so that kernel modules are
        loaded, per-thread library state exists and the plan caches hold the common
        shapes before a measured run."""
        import workloads.serving as S

        self.run(S.request_stream(n, 1e6, seed=seed))

    # -- sizes ------------------------------------------------------------------------
    def _desc_for(self, key: BatchKey, cap: int):
        B = self.B
        d = B.PdDesc()
        d.abi_version = B.PD_ABI_VERSION
        d.dim, d.nx, d.ny, d.nt, d.tau = key.dim, key.nx, key.ny, key.nt, 1.0 / key.nt
        d.precision = B.PD_MIXED if self.precision == "mixed" else B.PD_FP64
        d.q, d.alpha = 1, 1.0
        d.batch = cap if (key.dim == 1 or cap > 1) else 0
        return d

    def _workspace_bytes(self, key: BatchKey, cap: int) -> int:
        k = (key, cap)
        if k not in self._ws_cache:
            n = key.nx * cap  # T_x of every problem
            # a placeholder operator of the right shape (the size depends on the shape only);
            # tridiag(-1, 2, -1) passes the plan's diagonal-dominance check
            off, two = -np.ones(n), np.full(n, 2.0)
            d = self._desc_for(key, cap)
            p = lambda a: a.ctypes.data_as(self.B.ctypes.POINTER(self.B.ctypes.c_double))  # noqa: E731
            d.k_lo, d.k_diag, d.k_up = p(off), p(two), p(off)
            if key.dim == 2:  # T_y of every problem
                yoff, ytwo = -np.ones(key.ny * cap), np.full(key.ny * cap, 2.0)
                d.k_lo_y, d.k_diag_y, d.k_up_y = p(yoff), p(ytwo), p(yoff)
            self._ws_cache[k] = self.B.paradiag_workspace_size(d)
        return self._ws_cache[k]

    # -- one batch ----------------------------------------------------------------------
    def _slot(self, cache: OrderedDict, batch: Batch, stream):
        torch = self.torch
        k = (batch.key, batch.cap)
        if k in cache:
            cache.move_to_end(k)
            return cache[k], False
        # evict least recently used plans beyond this worker's share of the cache budget
        share = self.plan_cache_bytes // max(self.workers, 1)
        while cache and sum(s.bytes for s in cache.values()) + batch.bytes > share:
            _, old = cache.popitem(last=False)
            old.plan.close()
        # the plan's workspace is allocated on the worker's stream, the stream its
        # kernels run on, so the allocator reuses it in stream order
        with torch.cuda.stream(stream):
            plan, nb = self._new_plan(batch, stream)
            G = torch.zeros((batch.key.nt, nb), dtype=torch.float64, device=self.device)
            U = torch.empty_like(G)
        slot = _Slot(plan, G, U, batch.bytes)
        cache[k] = slot
        return slot, True

    def _new_plan(self, batch: Batch, stream):
        import workloads.serving as S

        r0 = batch.requests[0]
        if batch.key.dim == 1 or batch.cap > 1:
            plan = self.Plan.from_problems(self._slot_problems(batch, batch.requests), nx=batch.key.nx,
                                           precision=self.precision, alpha=self.alpha, device=self.device,
                                           stream=stream)
            nb = batch.cap * batch.key.nx * batch.key.ny
        else:
            kx, ky = S.operator(r0)
            plan = self.Plan(dim=2, nx=r0.nx, ny=r0.ny, nt=r0.nt, tau=r0.tau, k_lo=kx[0], k_diag=kx[1],
                             k_up=kx[2], k_lo_y=ky[0], k_diag_y=ky[1], k_up_y=ky[2], precision=self.precision,
                             alpha=self.alpha, device=self.device, stream=stream)
            nb = r0.nx * r0.ny
        return plan, nb

    @staticmethod
    def _slot_problems(batch: Batch, reqs):
        """The operators of a batched plan's slots: the requests' (None: an empty slot),
        then empty slots."""
        import workloads.serving as S

        k = batch.key
        empty = lambda: S.empty_slot(k.nt, k.nx, k.ny) if k.dim == 2 else S.empty_slot(k.nt)  # noqa: E731
        probs = [S.request_problem_operator_only(r, k.nx) if r is not None else empty() for r in reqs]
        probs += [empty() for _ in range(batch.cap - len(probs))]
        return probs

    def _run(self, batch: Batch, cache: OrderedDict, stream) -> None:
        import workloads.serving as S

        torch = self.torch
        slot, fresh = self._slot(cache, batch, stream)
        reqs = batch.requests
        batched = batch.key.dim == 1 or batch.cap > 1
        width = batch.key.nx * batch.key.ny  # unknowns per slot
        host = None
        with torch.cuda.stream(stream):
            try:  # a failed solve fails its requests, not the service
                if batched:
                    if not fresh:
                        slot.plan.set_problems(self._slot_problems(batch, reqs))
                    slot.G.zero_()
                    Gv = slot.G.view(batch.key.nt, batch.cap, width)
                    for b, r in enumerate(reqs):
                        S.rhs_device(r, torch, self.device, out=Gv[:, b, :])
                else:
                    r0 = reqs[0]
                    if not fresh:
                        kx, ky = S.operator(r0)
                        slot.plan.set_operator(tau=r0.tau, k_lo=kx[0], k_diag=kx[1], k_up=kx[2], k_lo_y=ky[0],
                                               k_diag_y=ky[1], k_up_y=ky[2])
                    S.rhs_device(r0, torch, self.device, out=slot.G)
                slot.plan.solve(slot.G, slot.U)
                err = None
                if self.keep_results == "full":  # the whole trajectory U (nt, n_bar) of each request
                    host = slot.U.view(batch.key.nt, batch.cap, width).cpu().numpy()
                elif self.keep_results:  # the final state u_l of each request
                    host = slot.U[-1].view(1, batch.cap, width).cpu().numpy()
            except Exception as e:
                err = str(e)
                self._drop_plan(cache, batch)
        now = time.perf_counter() - self.t0
        for b, r in enumerate(reqs):
            r.done, r.batch, r.error = now, len(reqs), err
            if host is not None:
                res = host[:, b, : r.nx * r.ny]
                r.result = (res if self.keep_results == "full" else res[0]).copy()

    def _finish(self, r, host_slot, err, now, occupancy):
        r.done, r.batch, r.error = now, occupancy, err
        if host_slot is not None:
            res = host_slot[:, : r.nx * r.ny]
            r.result = (res if self.keep_results == "full" else res[-1]).copy()

    def _drop_plan(self, cache: OrderedDict, batch: Batch) -> None:
        """Forget a cached plan after an error (it may be unusable)."""
        slot = cache.pop((batch.key, batch.cap), None)
        if slot is not None:
            try:
                slot.plan.close()
            except Exception:
                pass

    def _run_continuous(self, batch: Batch, cache: OrderedDict, stream) -> list:
        """Advance a batched plan one refinement sweep at a time; converged problems leave
        and waiting requests of the same key join in the free slots.  Returns every request
        finished here (the batch's and those that joined it), each counted once as done."""
        import workloads.serving as S

        torch = self.torch
        key, cap = batch.key, batch.cap
        width = key.nx * key.ny
        occ = list(batch.requests) + [None] * (cap - len(batch.requests))
        finished, counted = [], [0]

        def count():  # finished requests are counted as they finish
            with self.cv:
                self._done_count[0] += len(finished) - counted[0]
                counted[0] = len(finished)
                self.cv.notify_all()

        try:
            slot, _ = self._slot(cache, batch, stream)
            with torch.cuda.stream(stream):
                plan = slot.plan
                Gv = slot.G.view(key.nt, cap, width)
                Uv = slot.U.view(key.nt, cap, width)
                plan.set_problems(self._slot_problems(batch, occ))
                slot.G.zero_()
                for b, r in enumerate(occ):
                    if r is not None:
                        S.rhs_device(r, torch, self.device, out=Gv[:, b, :])
                join = [1 if r is not None else 0 for r in occ]
                while any(r is not None for r in occ):
                    try:
                        state, _ = plan.advance(slot.G, slot.U, join, steps=1)
                        err = None
                    except Exception as e:  # a failed call fails the requests in the batch
                        state, err = [2] * cap, str(e)
                    join = [0] * cap
                    now = time.perf_counter() - self.t0
                    occupancy = sum(r is not None for r in occ)
                    for b, r in enumerate(occ):
                        if r is None or state[b] == 0:
                            continue
                        host = None
                        if err is None and self.keep_results == "full":
                            host = Uv[:, b, :].cpu().numpy()
                        elif err is None and self.keep_results:
                            host = Uv[-1:, b, :].cpu().numpy()
                        self._finish(r, host, err or (None if state[b] == 1 else "refinement did not converge"),
                                     now, occupancy)
                        finished.append(r)
                        occ[b] = None
                        Gv[:, b, :].zero_()  # the slot is unused from the next sweep
                    if err is not None:
                        self._drop_plan(cache, batch)
                        break
                    free = [b for b, r in enumerate(occ) if r is None]
                    with self.cv:
                        new = self.sched.take(key, len(free))
                    count()
                    if new:
                        t_join = time.perf_counter() - self.t0
                        for b, r in zip(free, new):
                            occ[b] = r
                            r.start, r.joined_running = t_join, True
                        plan.set_problems(self._slot_problems(batch, occ))
                        for b, r in zip(free, new):
                            S.rhs_device(r, torch, self.device, out=Gv[:, b, :])
                            join[b] = 1
        except Exception as e:  # the service keeps running; this batch's requests fail
            now = time.perf_counter() - self.t0
            done = {id(r) for r in finished}
            for r in occ:
                if r is not None and id(r) not in done:
                    self._finish(r, None, f"service: {e}", now, 0)
                    finished.append(r)
            self._drop_plan(cache, batch)
        count()
        return finished

    # -- the run ------------------------------------------------------------------------
    def run(self, requests: list) -> ServeStats:
        torch = self.torch
        reqs = sorted(requests, key=lambda r: r.arrival)
        stats = ServeStats()
        pending = list(reqs)
        lock = self.cv
        done_count = [0]
        self._done_count = done_count
        self.t0 = time.perf_counter()

        def feeder():
            for r in pending:
                delay = r.arrival - (time.perf_counter() - self.t0)
                if delay > 0:
                    time.sleep(delay)
                with lock:
                    self.sched.add(r)
                    lock.notify_all()

        def worker(w):
            stream, cache = self._workers[w]
            while True:
                with lock:
                    while True:
                        if done_count[0] >= len(reqs):
                            return
                        batch = self.sched.next_batch()
                        if batch is not None:
                            break
                        lock.wait(timeout=0.05)
                t_start = time.perf_counter() - self.t0
                for r in batch.requests:
                    r.start = t_start
                if self.continuous and (batch.key.dim == 1 or batch.cap > 1):
                    self._run_continuous(batch, cache, stream)  # counts its requests itself
                    with lock:
                        self.sched.release(batch)
                        stats.batches += 1
                        lock.notify_all()
                    continue
                try:
                    self._run(batch, cache, stream)
                except Exception as e:  # (plan creation failed) the service keeps running
                    for r in batch.requests:
                        r.done, r.error = time.perf_counter() - self.t0, f"service: {e}"
                with lock:
                    self.sched.release(batch)
                    done_count[0] += len(batch.requests)
                    stats.batches += 1
                    lock.notify_all()

        if not self._workers:
            self._workers = [(torch.cuda.Stream(device=self.device), OrderedDict()) for _ in range(self.workers)]
        threads = [threading.Thread(target=feeder)] + [threading.Thread(target=worker, args=(w,))
                                                        for w in range(self.workers)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        stats.elapsed_s = max(r.done for r in reqs) - min(r.arrival for r in reqs) if reqs else 0.0
        for r in reqs:
            stats.requests += 1
            stats.failed += 1 if r.error else 0
            stats.joined += 1 if r.joined_running else 0
            stats.unknowns += r.unknowns
            stats.latencies_ms.append((r.done - r.arrival) * 1e3)
        return stats
