"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (relative Frobenius norm against the oracle, as the method's
accuracy contract states them): 1e-12 for the FP64 path and 1e-10 for the
mixed path after refinement.  Stage tests compare each step of the path with
the oracle's definition of that step.
"""
import numpy as np
import pytest

import workloads as W
from oracle import native
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


def _solve(pd, P, prec, G=None, **kw):
    G = P.G if G is None else G
    with pd.Plan.from_problem(P, precision=prec, device=dev(), **kw) as plan:
        U, st = plan.solve(torch.from_numpy(np.ascontiguousarray(G)).to(dev()))
        b, x = plan.last_vectors()
        return U.cpu().numpy(), st, b.cpu().numpy(), x.cpu().numpy()


# ----------------------------------------------------------------------------
# Stage a1 / a5: time DFTs
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("nt,nbar", [(1, 5), (2, 3), (8, 17), (64, 100), (1024, 33), (4096, 3)])
def test_time_dft_matches_definition(pd, prec, nt, nbar):
    P = W.random_tridiag_problem(nbar, nt, seed=nt + nbar)
    X = P.G
    ref = R.dft_time(X)[: nt // 2 + 1 if nt > 1 else 1]
    with pd.Plan.from_problem(P, precision=prec, device=dev()) as plan:
        Xh = plan.time_dft(torch.from_numpy(X).to(dev())).cpu().numpy()
        err = np.linalg.norm(Xh - ref) / np.linalg.norm(ref)
        assert err < (1e-14 * max(1, np.log2(nt)) if prec == "fp64" else 2e-7 * max(1, np.log2(nt)))
        # inverse of the half spectrum of real data returns the data
        Xb = plan.time_idft(torch.from_numpy(ref.astype(Xh.dtype)).to(dev())).cpu().numpy()
        err2 = np.linalg.norm(Xb - X) / np.linalg.norm(X)
        assert err2 < (1e-14 * max(1, np.log2(nt)) if prec == "fp64" else 2e-7 * max(1, np.log2(nt)))


# ----------------------------------------------------------------------------
# Stage a2: shifted solves and b (eq. 7)
# ----------------------------------------------------------------------------


def _stage_problems():
    return [W.heat1d_forced(127, 64, seed=1), W.heat1d_forced(1023, 32, seed=2),
            W.advdiff1d_pulse(255, 16, seed=3), W.advdiff1d_pulse(4095, 8, seed=4),
            W.random_tridiag_problem(1, 8, seed=5), W.random_tridiag_problem(2, 4, seed=6),
            W.random_tridiag_problem(3, 2, seed=7), W.random_tridiag_problem(33, 16, seed=8),
            W.random_tridiag_problem(129, 16, seed=9), W.random_tridiag_problem(200, 1, seed=10)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("P", _stage_problems(), ids=lambda p: p.name)
def test_shifted_solves_and_b(pd, prec, P):
    ell = P.nt
    nf = ell // 2 + 1 if ell > 1 else 1
    pi, gamma = R.circulant_eigs(ell)
    Rfull = R.dft_time(P.G)
    op = R.operator(P)
    L = np.stack([op.shifted_solve(1.0 - pi[i], P.tau, Rfull[i]) for i in range(ell)])
    b_ref = (gamma @ L).real
    K = R.k_dense(P) if P.nbar <= 1200 else None
    ctype = np.complex128 if prec == "fp64" else np.complex64
    with pd.Plan.from_problem(P, precision=prec, device=dev()) as plan:
        Y, b = plan.shifted_solve(torch.from_numpy(Rfull[:nf].astype(ctype)).to(dev()))
        Y = Y.cpu().numpy().astype(np.complex128)
        b = b.cpu().numpy()
    # backward error of every shifted system, and forward agreement with the oracle
    for k in range(nf):
        if K is not None:
            A = (1.0 - pi[k]) * np.eye(P.nbar) + P.tau * K
            bw = np.linalg.norm(A @ Y[k] - Rfull[k]) / (np.linalg.norm(A, 2) * np.linalg.norm(Y[k]) + 1e-300)
            assert bw < (1e-13 if prec == "fp64" else 1e-4), (k, bw)
    fwd = np.linalg.norm(Y - L[:nf]) / np.linalg.norm(L[:nf])
    assert fwd < (1e-10 if prec == "fp64" else 5e-3)
    assert np.linalg.norm(b - b_ref) / max(np.linalg.norm(b_ref), 1e-300) < (1e-10 if prec == "fp64" else 5e-3)


# ----------------------------------------------------------------------------
# Full path (Algorithm 1 + 2, and refinement) against the oracle
# ----------------------------------------------------------------------------


def _full_problems():
    return [
        W.heat1d_127x64(),
        W.heat1d_forced(255, 128, seed=3),
        W.advdiff1d_pulse(511, 256, seed=4),
        W.random_tridiag_problem(1, 1, seed=1),
        W.random_tridiag_problem(1, 16, seed=2),
        W.random_tridiag_problem(2, 2, seed=3),
        W.random_tridiag_problem(3, 64, seed=4),
        W.random_tridiag_problem(7, 8, seed=5, symmetric=True),
        W.random_tridiag_problem(33, 32, seed=6),
        W.random_tridiag_problem(130, 4, seed=7),
        W.random_tridiag_problem(4096, 8, seed=8),
        W.heat2d_smooth(7, 8, 0.1, seed=1),
        W.heat2d_smooth(15, 16, 0.1, seed=2),
        W.heat2d_smooth(31, 32, 0.1, seed=3),
        W.heat2d_smooth(1, 4, 0.1, seed=4),
        # centred advection (the paper's Sec. 6.2 discretisation, in 1D) at cell Peclet 1.5 and 2:
        # weakly diagonally dominant, so the plan accepts it (above 2 it is rejected, see
        # test_abi_cpu.py)
        W.advdiff1d_centred(255, 64, 0.1, peclet=1.5, seed=5),
        W.advdiff1d_centred(127, 32, 0.1, peclet=2.0, nu=1e-3, seed=6),
    ]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("P", _full_problems(), ids=lambda p: p.name)
def test_solve_matches_oracle(pd, prec, P):
    Uref = R.be_solve_refined(P)
    U, st, b, x = _solve(pd, P, prec)
    assert R.rel_err(U, Uref) <= TOL[prec], st
    if prec == "fp64" and st["refine_sweeps"] == 1:
        # x_m of Algorithm 2 is the true final state u_l (Sec. 2: W = P^{-1} M x)
        nl = max(np.linalg.norm(Uref[-1]), 1e-300)
        assert np.linalg.norm(x - Uref[-1]) / nl < 1e-10


@pytest.mark.parametrize("P", [W.random_tridiag_problem(12, 8, seed=3), W.heat1d_forced(31, 16, seed=1),
                               W.heat2d_smooth(3, 4, 0.1, seed=1)], ids=lambda p: p.name)
def test_b_is_last_slice_of_periodic_solution(pd, P):
    K = R.k_dense(P)
    Uper = R.periodic_solve_dense(K, P.tau, P.G).real
    _, _, b, _ = _solve(pd, P, "fp64")
    assert np.linalg.norm(b - Uper[-1]) <= 1e-12 * max(1.0, np.linalg.norm(Uper[-1]))


def test_krylov_iterations_match_oracle_algorithm2(pd):
    P = W.advdiff1d_pulse(63, 32, 0.3, seed=2)
    _, info = R.paradiag(P, eps=1e-13, maxit=32)
    U, st, _, _ = _solve(pd, P, "fp64", eps_krylov=1e-13)
    assert R.rel_err(U, R.be_solve(P)) <= 1e-12
    if st["refine_sweeps"] == 1:  # Algorithm 2 reached eps in one solve, like the oracle
        assert abs(st["krylov_iters"] - info["krylov"]["m"]) <= 1
        assert st["krylov_rel_resnorm"] <= 1e-13
        assert st["pint_loops"] == st["krylov_iters"] + 2


def test_one_eigenmode_needs_one_iteration(pd):
    """G = one sine eigenmode of K: b is a multiple of that mode, K_1(K, b) is invariant, and
    one Algorithm-2 step solves eq. (8) exactly.  In floating point b carries rounding noise
    in every mode, of size about eps ||L_k|| (b is the weighted sum of the shifted solutions
    L_k, eq. 7), and v_2 is that noise.  With mode 1 at T = 0.05 the final state is hardly
    decayed (||b|| ~ ||u_0||), so the noise stays at rounding level and one step meets the
    FP64 tolerance: one solve, m = 1, two parallel-in-time loops."""
    n, nt = 63, 16
    P = W.heat1d_sine_modes(n, nt, 0.05, seed=0)
    x = np.arange(1, n + 1) / (n + 1)
    G = np.zeros_like(P.G)
    G[0] = np.sin(np.pi * x)
    U, st, _, _ = _solve(pd, P, "fp64", G=G)
    assert st["refine_sweeps"] == 1 and st["krylov_iters"] == 1 and st["pint_loops"] == 3, st
    assert st["krylov_rel_resnorm"] <= 1e-13
    assert R.rel_err(U, R.be_solve_refined(P, G=G)) <= 1e-12


def test_decayed_eigenmode_invariance_is_limited_by_rounding(pd):
    """Mode 3 over T = 1 decays to ||u_l|| ~ (1 + tau mu_3)^{-l} ||u_0|| ~ 1e-13 ||u_0||, so b
    (~ u_l, eq. 7) is a sum of O(||G||) terms that cancel to 1e-13 and its rounding noise is
    large relative to b itself.  K_1(K, b) is then invariant only to that noise level: the
    eq. (13) residual after one Algorithm-2 step stands at the noise level (3e-8 of ||b||
    measured), stalls there instead of reaching 1e-13 (a few steps, not maxit), and FP64
    refinement sweeps finish the solve to the FP64 bar."""
    n, nt = 63, 16
    P = W.heat1d_sine_modes(n, nt, 1.0, seed=0)
    x = np.arange(1, n + 1) / (n + 1)
    G = np.zeros_like(P.G)
    G[0] = np.sin(3 * np.pi * x)
    _, st1, _, _ = _solve(pd, P, "fp64", G=G, maxit=1)
    assert st1["sweep_krylov_iters"][0] == 1 and st1["sweep_krylov_rel_resnorm"][0] <= 1e-6
    U, st, _, _ = _solve(pd, P, "fp64", G=G)
    assert st["sweep_krylov_iters"][0] <= 5, st  # stalled at the noise level
    assert R.rel_err(U, R.be_solve_refined(P, G=G)) <= 1e-12, st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_breakdown_on_invariant_krylov_space(pd, prec):
    """n = 1: K v_1 is exactly parallel to v_1, t_{2,1} = 0 and Algorithm 2 breaks down."""
    P = W.random_tridiag_problem(1, 16, seed=3)
    U, st, _, _ = _solve(pd, P, prec)
    assert st["breakdown"] == 1 and st["krylov_iters"] == 1
    assert R.rel_err(U, R.be_solve(P)) <= TOL[prec]


def test_zero_rhs_gives_zero(pd):
    P = W.random_tridiag_problem(40, 8, seed=1)
    for prec in ("fp64", "mixed"):
        U, st, _, _ = _solve(pd, P, prec, G=np.zeros_like(P.G))
        assert np.all(U == 0.0)


def test_nonfinite_input_is_reported(pd):
    P = W.random_tridiag_problem(40, 8, seed=1)
    G = P.G.copy()
    G[3, 5] = np.nan
    with pytest.raises(pd.ParadiagError) as e:
        _solve(pd, P, "fp64", G=G)
    assert e.value.status_name == "PD_ERR_NONFINITE"


def test_fp64_solve_is_deterministic(pd):
    P = W.heat1d_forced(255, 64, seed=9)
    with pd.Plan.from_problem(P, precision="fp64", device=dev()) as plan:
        G = torch.from_numpy(P.G).to(dev())
        U1, _ = plan.solve(G)
        U2, _ = plan.solve(G)
        assert torch.equal(U1, U2)


def test_host_io_matches_device_solve(pd):
    P = W.heat1d_forced(127, 64, seed=2)
    with pd.Plan.from_problem(P, precision="mixed", device=dev(), host_io=True) as plan:
        Gd = torch.from_numpy(P.G).to(dev())
        Ud, _ = plan.solve(Gd)
        Gh = torch.from_numpy(P.G.copy()).pin_memory()
        Uh = torch.empty_like(Gh).pin_memory()
        plan.solve_host(Gh, Uh)
        assert torch.equal(Ud.cpu(), Uh)


def test_dst_y_matches_definition(pd):
    P = W.heat2d_smooth(15, 4, 0.1, seed=1)
    n = 15
    j = np.arange(1, n + 1)
    S = np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(j, j) / (n + 1))
    X = np.random.default_rng(0).standard_normal((4, n * n))
    ref = np.einsum("ly,tyx->tlx", S, X.reshape(4, n, n)).reshape(4, -1)
    with pd.Plan.from_problem(P, precision="fp64", device=dev()) as plan:
        Y = plan.dst_y(torch.from_numpy(X).to(dev())).cpu().numpy()
    assert np.linalg.norm(Y - ref) / np.linalg.norm(ref) < 1e-14


# ----------------------------------------------------------------------------
# The benchmark workloads at full size
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("name", ["heat1d_1023x1024", "advdiff1d_4095x2048"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_1d_workloads(pd, name, prec):
    P = W.by_name(name)
    Uref = R.be_solve_refined(P)
    U, st, _, x = _solve(pd, P, prec)
    assert R.rel_err(U, Uref) <= TOL[prec], st
    if prec == "mixed":  # J_l's zero-frequency term is small here: no FP64 lane
        assert st["zero_freq_fp64"] == 0 and st["zero_freq_weight"] < 4, st["zero_freq_weight"]


@pytest.fixture(scope="module")
def heat2d_ref():
    P = W.heat2d_255x255x256()
    return P, R.be_solve_refined(P)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_2d_heat(pd, heat2d_ref, prec):
    P, Uref = heat2d_ref
    U, st, _, _ = _solve(pd, P, prec)
    assert R.rel_err(U, Uref) <= TOL[prec], st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("P", [W.heat1d_forced(255, 64, seed=4), W.heat2d_smooth(15, 16, 0.1, seed=2),
                               W.advdiff1d_pulse(127, 32, 0.3, seed=5)], ids=lambda p: p.name)
def test_graph_solve_equals_host_driven_solve(pd, prec, P):
    """One CUDA-graph launch with device-side loop control runs exactly the kernels the
    host-driven loops run: identical U and statistics."""
    G = torch.from_numpy(P.G).to(dev())
    with pd.Plan.from_problem(P, precision=prec, device=dev()) as pg, \
            pd.Plan.from_problem(P, precision=prec, device=dev(), no_graph=True) as ph:
        Ug, sg = pg.solve(G)
        Ug2, sg2 = pg.solve(G)  # graph reused
        Uh, sh = ph.solve(G)
    assert sg["graph"] == 1 and sg2["graph"] == 1 and sh["graph"] == 0
    assert torch.equal(Ug, Uh) and torch.equal(Ug2, Uh)
    for key in ("refine_sweeps", "krylov_iters_total", "sweep_krylov_iters", "kernel_launches"):
        assert sg[key] == sh[key], key
    assert R.rel_err(Ug.cpu().numpy(), R.be_solve_refined(P)) <= TOL[prec]


# ----------------------------------------------------------------------------
# Factored shifted systems (factors computed once per operator) against the oracle
# ----------------------------------------------------------------------------


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("factor", [-1, 1])
@pytest.mark.parametrize("P", [W.random_tridiag_problem(129, 16, seed=9), W.heat1d_forced(255, 128, seed=3),
                               W.random_tridiag_problem(4096, 8, seed=8), W.heat2d_smooth(15, 16, 0.1, seed=2),
                               W.random_tridiag_problem(3, 64, seed=4)], ids=lambda p: p.name)
def test_factored_and_eliminating_loops_match_oracle(pd, prec, factor, P):
    """Both forms of the parallel-in-time loop: eliminating in every loop (-1) and
    solving with factors stored per operator (1), in both precisions."""
    Uref = R.be_solve_refined(P)
    U, st, _, _ = _solve(pd, P, prec, tune={"pint_factor": factor})
    assert R.rel_err(U, Uref) <= TOL[prec], st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_factored_shifted_solves_match_definition(pd, prec):
    """The factored shifted solves of every frequency against the oracle's (1 - pi_k) I + tau K."""
    P = W.random_tridiag_problem(200, 32, seed=12)
    ell = P.nt
    nf = ell // 2 + 1
    pi, _ = R.circulant_eigs(ell)
    Rfull = R.dft_time(P.G)
    op = R.operator(P)
    L = np.stack([op.shifted_solve(1.0 - pi[i], P.tau, Rfull[i]) for i in range(nf)])
    ctype = np.complex128 if prec == "fp64" else np.complex64
    with pd.Plan.from_problem(P, precision=prec, device=dev(), tune={"pint_factor": 1}) as plan:
        Y, _ = plan.shifted_solve(torch.from_numpy(Rfull[:nf].astype(ctype)).to(dev()))
        Y = Y.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(Y - L) / np.linalg.norm(L) < (1e-10 if prec == "fp64" else 5e-3)


@pytest.mark.parametrize("prec,factor", [("fp64", 0), ("mixed", 1), ("mixed", 0)])
def test_set_operator_refactors(pd, prec, factor):
    """paradiag_set_operator swaps K (and tau): the next solve is the new problem's
    (the stored factors are recomputed)."""
    A = W.heat1d_forced(255, 64, seed=1)
    B = W.advdiff1d_pulse(255, 64, seed=2)
    with pd.Plan.from_problem(A, precision=prec, device=dev(), tune={"pint_factor": factor}) as plan:
        Ua, _ = plan.solve(torch.from_numpy(A.G).to(dev()))
        plan.set_operator(tau=B.tau, k_lo=B.k_lo, k_diag=B.k_diag, k_up=B.k_up)
        Ub, st = plan.solve(torch.from_numpy(B.G).to(dev()))
        Ub = Ub.cpu().numpy()
    assert R.rel_err(Ua.cpu().numpy(), R.be_solve_refined(A)) <= TOL[prec]
    assert R.rel_err(Ub, R.be_solve_refined(B)) <= TOL[prec], st


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("tune", [{"krylov_cluster": -1, "persistent": -1}, {"krylov_cluster": 4, "persistent": -1},
                                  {"krylov_cluster": 16, "persistent": -1}, {"krylov_ctas": 8, "persistent": -1},
                                  {"persistent": 1}],
                         ids=lambda t: "-".join(f"{k}{v}" for k, v in t.items()))
@pytest.mark.parametrize("P", [W.heat1d_forced(1023, 64, seed=5), W.advdiff1d_pulse(2047, 32, seed=6),
                               W.random_tridiag_problem(300, 16, seed=13)], ids=lambda p: p.name)
def test_krylov_variants_match_oracle(pd, prec, tune, P):
    """The Algorithm-2 vector steps in one CTA, in clusters of 4 and 16 CTAs (one per SM,
    reductions through distributed shared memory), on a cooperative grid (one launch per
    phase of a step), and in the persistent step."""
    Uref = R.be_solve_refined(P)
    U, st, _, _ = _solve(pd, P, prec, tune=tune)
    assert R.rel_err(U, Uref) <= TOL[prec], st


# ----------------------------------------------------------------------------
# The binary32 reciprocal of the mixed-precision shifted solves
# ----------------------------------------------------------------------------


def _ulp_distance(a, b):
    """|a - b| in units in the last place of binary32 (same-sign finite values)."""
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def test_binary32_reciprocal_within_one_ulp(pd):
    """The complex division 1/a = conj(a) / |a|^2 of the binary32 shifted solves takes 1/|a|^2
    from the hardware approximation plus one Newton-Raphson step.  Over normal-range operands
    (2^-120 .. 2^120, random mantissas, both signs) it is within 1 ulp of the correctly
    rounded reciprocal (numpy's IEEE binary32 division), and exact on powers of two."""
    rng = np.random.default_rng(7)
    n = 1 << 22
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-120, 121, n)
    x = (np.ldexp(mant, expo) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    x[:241] = np.ldexp(1.0, np.arange(-120, 121)).astype(np.float32)  # powers of two
    xd = torch.from_numpy(x).to(dev())
    rd = torch.empty_like(xd)
    stream = torch.cuda.current_stream(dev())
    pd._binding.paradiag_recip_f32(xd.data_ptr(), rd.data_ptr(), n, stream.cuda_stream)
    r = rd.cpu().numpy()
    ref = (np.float32(1.0) / x).astype(np.float32)  # correctly rounded (IEEE division)
    d = _ulp_distance(r, ref)
    assert d.max() <= 1, (d.max(), x[np.argmax(d)])
    assert np.array_equal(r[:241], ref[:241])
    assert np.mean(d == 0) > 0.5  # mostly correctly rounded; the rest one ulp off
