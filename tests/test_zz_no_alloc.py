"""paradiag_smw_rhs_noalloc against paradiag_shifted_solve (GPU, through the C ABI).

paradiag_smw_rhs_noalloc serves callers that cannot allocate device memory when
they need the first parallel-in-time loop (a pool or arena that owns all device
memory, a real-time loop, a host that forbids allocation after start-up): its
scratch is a static device array instead of a plan workspace.  It must give the
same Y and b (eq. 7) as the plan-based entry point, call after call, within the
FP64 shifted-solve tolerance used by the other GPU tests.  This file is named so
that pytest collects it last.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FWD_TOL = 1e-10  # FP64 shifted solves and b, as in test_gpu_parity.py


@pytest.fixture(scope="module")
def pd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as entry

    entry.build()
    import paper_2304_12597_gb300 as pkg

    return pkg


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _compare(pd, P):
    dev = torch.device("cuda:0")
    with pd.Plan.from_problem(P, precision="fp64", device=dev) as plan:
        R = plan.time_dft(torch.from_numpy(P.G).to(dev))
        Y_ref, b_ref = plan.shifted_solve(R)
    k = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (P.k_lo, P.k_diag, P.k_up)]
    Y = torch.empty_like(R)
    b = torch.empty(P.nbar, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    pd._binding.paradiag_smw_rhs_noalloc(P.nt, P.nbar, P.tau, k[0].data_ptr(), k[1].data_ptr(), k[2].data_ptr(),
                                         R.data_ptr(), Y.data_ptr(), b.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    assert _rel(Y, Y_ref) <= FWD_TOL
    assert _rel(b, b_ref) <= FWD_TOL


def test_noalloc_matches_plan_entry_point_call_after_call(pd):
    # several calls in a row share the static scratch; sizes change between calls
    _compare(pd, W.heat1d_forced(1023, 64, seed=1))
    _compare(pd, W.advdiff1d_pulse(4095, 16, seed=2))
    _compare(pd, W.heat1d_forced(1023, 64, seed=1))


def _periodic_last_slice(P, sweeps=8):
    """b of eq. (7), the last slice of the periodic (circulant) solution, from the oracle's
    sequential backward Euler: the periodic solution is the one whose start value is its own
    final state, u_0 = u_l, the fixed point of u_l <- BE(G with u_0 = u_l)[-1] (G_1 carries
    u_0), a contraction by ||(I + tau K)^{-l}|| = (1 + tau lambda_min)^{-l}."""
    from oracle import reference as R

    y = np.zeros(P.nbar)
    for _ in range(sweeps):
        G = P.G.copy()
        G[0] += y
        y = R.be_solve(P, G=G)[-1]
    return y


def test_noalloc_clamped_partial_rows_match_plan_and_oracle(pd):
    """n near the limit and a long time axis (n = 4095, l = 4096): the per-team partial rows
    of b no longer fit the static scratch at the default split, so the entry point clamps the
    number of frequency ranges; Y and b still equal the plan entry point's, and b equals the
    oracle's eq. (7) vector."""
    P = W.heat1d_forced(4095, 4096, seed=3)
    _compare(pd, P)
    dev = torch.device("cuda:0")
    with pd.Plan.from_problem(P, precision="fp64", device=dev) as plan:
        R = plan.time_dft(torch.from_numpy(P.G).to(dev))
    k = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (P.k_lo, P.k_diag, P.k_up)]
    b = torch.empty(P.nbar, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    pd._binding.paradiag_smw_rhs_noalloc(P.nt, P.nbar, P.tau, k[0].data_ptr(), k[1].data_ptr(), k[2].data_ptr(),
                                         R.data_ptr(), 0, b.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    ref = _periodic_last_slice(P)
    assert np.linalg.norm(b.cpu().numpy() - ref) <= FWD_TOL * np.linalg.norm(ref)


def test_noalloc_rejects_sizes_beyond_its_scratch(pd):
    dev = torch.device("cuda:0")
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    with pytest.raises(pd.ParadiagError) as e:
        pd._binding.paradiag_smw_rhs_noalloc(16, 5000, 0.1, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr(),
                                             x.data_ptr(), x.data_ptr(), 0)
    assert e.value.status_name == "PD_ERR_UNSUPPORTED"
    assert "static scratch" in str(e.value)
