"""Launch-geometry autotuner for one plan shape.

Coordinate descent over the `tune_*` fields of pd_desc: rows per thread and teams per
CTA of the shifted-solve kernel, columns per CTA and the first-stage radix (one radix-16
stage in registers, or radix-4 passes only) of the time FFTs and the DST along y, CTAs of
the capacitance-term kernel and of the Krylov vector kernels.  Each candidate plan solves
the caller's right-hand side; its time is the median of CUDA-event timed solves with an
L2 flush before each, and a candidate whose result differs from the default plan's by
more than the precision's tolerance is rejected.  Geometries the library refuses
(PD_ERR_UNSUPPORTED / PD_ERR_INVALID_ARG) are skipped.  Results can be kept in a JSON
cache file keyed by the plan shape and the GPU, so a shape is tuned once per machine.
The tuner only chooses launch parameters; every solve runs in the library's kernels.
"""
from __future__ import annotations

import json
import os
import statistics

from ._binding import ParadiagError

TOL = {"fp64": 1e-12, "mixed": 1e-10}


def _candidates(plan_kw, nf):
    mixed = plan_kw.get("precision", "mixed") == "mixed"
    return [
        ("pint_rows", [0, 4, 8] + ([16] if mixed else [])),
        ("pint_teams", [0, 1, 2, 4]),
        ("fft_cols", [0, 2, 4, 8, 16]),
        ("fft_radix", [0, 4, 16]),
        ("cap_ctas", sorted({0, max(1, (nf + 7) // 8), max(1, (nf + 3) // 4), max(1, (nf + 1) // 2)})),
        ("krylov_ctas", [0, 8, 16]),
        ("pint_factor", [0, 1, -1]),
        ("krylov_cluster", [0, -1, 16]), ("krylov_tails", [0, 1]),
    ]


def plan_key(plan) -> str:
    """Cache key of a plan's shape: dimension, sizes, batch, precision and alpha, and the GPU
    model (launch geometry depends on all of them)."""
    import torch

    d = plan.desc
    return json.dumps({"dim": plan.dim, "nx": plan.nx, "ny": plan.ny, "nt": plan.nt, "batch": plan.batch,
                       "precision": plan.precision, "alpha": float(d.alpha) or 1.0,
                       "gpu": torch.cuda.get_device_name(plan.device)}, sort_keys=True)


def _cache_load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _cache_store(path, key, entry):
    data = _cache_load(path)
    data[key] = entry
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def autotune(make_plan, G, reps=5, flush_bytes=256 << 20, log=None, cache=None):
    """Tune the launch geometry of the plans `make_plan(tune=...)` builds for right-hand side G
    (a device tensor of the plan's shape).  Returns (best tune dict, best ms, default ms).

    make_plan: callable taking tune=dict and returning a paper_2304_12597_gb300.Plan (used
    as a context manager).
    cache: optional path of a JSON file.  A stored result for this plan's shape and GPU
    (plan_key) is returned without tuning; a new result is added to the file."""
    import torch

    key = None
    if cache is not None:
        with make_plan(tune={}) as p0:
            key = plan_key(p0)
        hit = _cache_load(cache).get(key)
        if hit is not None:
            return dict(hit["tune"]), hit["ms"], hit["default_ms"]

    dev = G.device
    flush = torch.empty(flush_bytes // 4, dtype=torch.float32, device=dev)

    def run(tune):
        U = torch.empty_like(G)
        with make_plan(tune=tune) as plan:
            prec = plan.precision
            for _ in range(2):
                plan.solve(G, U)
            ts = []
            for _ in range(reps):
                flush.add_(1.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                plan.solve(G, U)
                e1.record()
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            nf = plan.nt // 2 + 1
        return statistics.median(ts), U, prec, nf

    base_ms, U0, prec, nf = run({})
    best, best_ms = {}, base_ms
    with make_plan(tune={}) as p0:
        kw = {"precision": p0.precision}
    for name, values in _candidates(kw, nf):
        for v in values:
            if v == best.get(name, 0):
                continue
            trial = dict(best)
            if v:
                trial[name] = v
            else:
                trial.pop(name, None)
            try:
                ms, U, _, _ = run(trial)
            except ParadiagError:
                continue
            diff = float(torch.linalg.norm(U - U0) / torch.linalg.norm(U0))
            if log is not None:
                log.append({"tune": dict(trial), "ms": ms, "diff": diff})
            if diff <= 2 * TOL[prec] and ms < best_ms:
                best, best_ms = trial, ms
    if cache is not None:
        _cache_store(cache, key, {"tune": best, "ms": best_ms, "default_ms": base_ms})
    return best, best_ms, base_ms
