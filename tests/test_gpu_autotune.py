"""The launch-geometry autotuner: the tuned plan solves to the oracle's tolerance and is not
slower than the default plan (within timing noise)."""
import pytest

import workloads as W
from oracle import reference as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as entry

    entry.build()
    import paper_2304_12597_gb300 as pkg

    return pkg


def test_autotune_keeps_accuracy_and_speed(pd, tmp_path):
    from paper_2304_12597_gb300.autotune import autotune

    P = W.heat1d_forced(511, 256, seed=3)
    dev = torch.device("cuda:0")
    G = torch.from_numpy(P.G).to(dev)
    log = []
    cache = str(tmp_path / "tuned.json")
    make = lambda tune: pd.Plan.from_problem(P, precision="mixed", device=dev, tune=tune)  # noqa: E731
    best, best_ms, base_ms = autotune(make, G, reps=3, log=log, cache=cache)
    assert len(log) >= 8 and best_ms <= base_ms * 1.05
    assert any("fft_radix" in e["tune"] for e in log)  # the first-stage radix is a coordinate
    # the cache file returns the stored result without tuning again
    log2 = []
    again = autotune(make, G, reps=3, log=log2, cache=cache)
    assert again == (best, best_ms, base_ms) and not log2
    with pd.Plan.from_problem(P, precision="mixed", device=dev, tune=best) as plan:
        U, _ = plan.solve(G)
    assert R.rel_err(U.cpu().numpy(), R.be_solve_refined(P)) <= 1e-10
