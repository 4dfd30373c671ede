"""Host-side checks of the C ABI (no GPU needed, no compute calls).

The library must build for sm_103a here, load, export every symbol that
include/paradiag.h declares, agree with the ctypes struct layouts, and reject
bad descriptors in its pure-host argument validation.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import __graft_entry__ as entry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "paradiag.h")


@pytest.fixture(scope="module")
def B():
    entry.build()
    from paper_2304_12597_gb300 import _binding

    return _binding


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"\b(paradiag_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(B):
    names = _declared()
    assert len(names) >= 10
    lib = ctypes.CDLL(B.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.SIGNATURES) == names
    nm = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (paradiag_\w+)", nm))
    assert exported == set(names)


def test_struct_layouts_match_header(B, tmp_path):
    prog = tmp_path / "sz.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "paradiag.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu\\n\", sizeof(pd_desc), sizeof(pd_stats),"
        " sizeof(pd_kernel_time), offsetof(pd_desc, stream), offsetof(pd_desc, precision),"
        " offsetof(pd_stats, kernel_launches), offsetof(pd_stats, sweep_rel_update));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(prog), "-o", str(exe)])
    vals = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert vals == [ctypes.sizeof(B.PdDesc), ctypes.sizeof(B.PdStats), ctypes.sizeof(B.PdKernelTime),
                    B.PdDesc.stream.offset, B.PdDesc.precision.offset, B.PdStats.kernel_launches.offset,
                    B.PdStats.sweep_rel_update.offset]


def _desc(B, **kw):
    n = kw.pop("n", 31)
    lo = np.full(n, -1.0)
    di = np.full(n, 2.0)
    up = np.full(n, -1.0)
    if "k" in kw:  # (lo, diag, up) of K
        lo, di, up = (np.ascontiguousarray(a, dtype=np.float64) for a in kw.pop("k"))
        n = len(di)
    keep = [lo, di, up]
    d = B.PdDesc()
    d.abi_version = 1
    d.dim = 1
    d.nx = n
    d.ny = 1
    d.nt = 16
    d.tau = 0.1
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))  # noqa: E731
    d.k_lo, d.k_diag, d.k_up = p(lo), p(di), p(up)
    d.precision = 0
    for k, v in kw.items():
        if k.startswith("y_") or k in ("batch_nx", "batch_tau", "batch_k", "mass"):
            continue
        setattr(d, k, v)
    if kw.get("batch", 0) > 1:  # K arrays hold batch * nx rows
        B = kw["batch"]
        lo, di, up = np.tile(lo, B), np.tile(di, B), np.tile(up, B)
        keep += [lo, di, up]
        d.k_lo, d.k_diag, d.k_up = p(lo), p(di), p(up)
        if "batch_nx" in kw:
            bn = np.asarray(kw["batch_nx"], dtype=np.int64)
            keep.append(bn)
            d.batch_nx = bn.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        if "batch_tau" in kw:
            bt = np.asarray(kw["batch_tau"], dtype=np.float64)
            keep.append(bt)
            d.batch_tau = p(bt)
    if "mass" in kw:  # diagonal mass matrix, one entry per row (of every slot)
        m = np.asarray(kw["mass"], dtype=np.float64)
        keep.append(m)
        d.m_diag = p(m)
    if kw.get("dim") == 2:
        ny = kw.get("ny", 7)
        nb = max(kw.get("batch", 1), 1)  # T_y of every problem of a batch
        ylo = kw.get("y_lo", np.full(ny * nb, -1.0))
        ydi = kw.get("y_diag", np.full(ny * nb, 2.0))
        yup = kw.get("y_up", np.full(ny * nb, -1.0))
        keep += [ylo, ydi, yup]
        d.k_lo_y, d.k_diag_y, d.k_up_y = p(ylo), p(ydi), p(yup)
    d._keep = keep
    return d


def _size_status(B, d):
    n = ctypes.c_size_t(0)
    return B.load().paradiag_workspace_size(ctypes.byref(d), ctypes.byref(n)), n.value


def test_valid_descriptors_have_a_workspace(B):
    for kw in ({}, {"precision": 1}, {"nt": 1}, {"n": 1}, {"n": 4096, "nt": 2048, "precision": 1},
               {"precision": 1, "tune_pint_rows": 16, "tune_pint_teams": 2, "tune_krylov_ctas": 8,
                "tune_cap_ctas": 3, "tune_fft_cols": 2},
               {"tune_krylov_cluster": 16}, {"tune_krylov_cluster": -1}, {"tune_krylov_ctas": 1, "n": 4095},
               {"tune_pint_factor": 1, "precision": 1}, {"tune_pint_factor": -1},
               {"mass": np.full(31, 0.5)}, {"mass": np.linspace(0.5, 2.0, 62), "batch": 2},
               {"batch": 3, "batch_nx": [31, 5, 1], "batch_tau": [0.1, 0.2, 1e-3]}, {"batch": 4},
               {"alpha": 1e-4}, {"alpha": 0.5, "precision": 1}, {"q": 3}, {"q": 32, "precision": 1}, {"tune_krylov_tails": 1}, {"tune_krylov_tails": -1},
               {"dim": 2, "ny": 7}, {"dim": 2, "ny": 255, "n": 255, "nt": 256, "precision": 1}):
        st, n = _size_status(B, _desc(B, **kw))
        assert st == 0, (kw, B.last_error())
        assert n > 0 and n % 256 == 0


@pytest.mark.parametrize("kw,code", [
    ({"abi_version": 2}, 1),
    ({"dim": 3}, 1),
    ({"nx": 0}, 1),
    ({"nt": 3}, 2),
    ({"nt": 16384}, 2),
    ({"tau": 0.0}, 1),
    ({"tau": float("nan")}, 1),
    ({"precision": 7}, 1),
    ({"maxit": 40}, 2),
    ({"q": 2, "batch": 2}, 2),             # frozen residual: single problems only
    ({"q": 33}, 1),
    ({"q": -1}, 1),
    ({"alpha": 1.5}, 1),
    ({"alpha": -0.1}, 1),
    ({"alpha": float("nan")}, 1),
    ({"n": 5000}, 2),
    ({"dim": 2, "ny": 6}, 2),
    ({"dim": 2, "ny": 7, "y_diag": np.array([2, 2, 2, 3, 2, 2, 2.0])}, 2),
    ({"dim": 2, "ny": 7, "y_up": np.array([-1, -1, -0.5, -1, -1, -1, -1.0])}, 2),
    ({"tune_pint_rows": 5}, 1),
    ({"tune_pint_rows": 16}, 2),              # 16 rows per thread: PD_MIXED only
    ({"tune_pint_rows": 4, "n": 4095}, 2),    # 1024 threads per team
    ({"tune_pint_teams": 3}, 1),
    ({"tune_krylov_ctas": -1}, 1),
    ({"tune_krylov_ctas": 1, "n": 4095, "batch": 3}, 2),   # one CTA holds <= 8192 entries
    ({"tune_krylov_cluster": 2}, 1),
    ({"tune_pint_factor": 2}, 1),
    ({"tune_krylov_tails": 2}, 1),
    ({"mass": np.full(31, 1.0), "dim": 2, "ny": 7}, 2),        # mass matrices: 1D only
    ({"mass": np.concatenate([np.ones(30), [0.0]])}, 1),       # entries must be > 0
    ({"mass": np.concatenate([np.ones(30), [np.nan]])}, 1),
    ({"tune_krylov_cluster": 32}, 1),
    ({"tune_cap_ctas": 5000}, 1),
    ({"tune_fft_cols": 6}, 1),
    ({"batch": -1}, 1),
    ({"batch": 2, "dim": 2, "n": 127, "ny": 127}, 2),         # 2D batches: nx ny <= 8192
    ({"batch": 3, "batch_nx": [31, 32, 1]}, 1),
    ({"batch": 3, "batch_nx": [31, 0, 1]}, 1),
    ({"batch": 2, "batch_tau": [0.1, 0.0]}, 1),
    ({"batch": 2, "batch_tau": [0.1, float("inf")]}, 1),
])
def test_bad_descriptors_are_rejected(B, kw, code):
    st, _ = _size_status(B, _desc(B, **kw))
    assert st == code, B.last_error()
    assert B.last_error()


def _centred_advdiff(n, peclet, nu=1e-2):
    """1D advection-diffusion nu u_xx - a u_x by centred differences (the discretisation of
    the paper's Sec. 6.2 example, in 1D) at cell Peclet number a h / nu = peclet."""
    h = 1.0 / (n + 1)
    a = peclet * nu / h
    lo = np.full(n, -nu / h**2 - a / (2 * h))
    di = np.full(n, 2 * nu / h**2)
    up = np.full(n, -nu / h**2 + a / (2 * h))
    lo[0] = up[-1] = 0.0
    return lo, di, up


def test_pivot_free_elimination_needs_dominance_or_spd(B):
    """The shifted solves eliminate without pivoting.  The plan accepts K when each block is
    weakly diagonally dominant by rows or symmetric positive definite (in the solve basis)
    and rejects it otherwise with PD_ERR_UNSUPPORTED: centred advection at cell Peclet
    number 4 is neither; at 1.5 (and at exactly 2) it is dominant."""
    st, _ = _size_status(B, _desc(B, k=_centred_advdiff(63, 4.0)))
    assert st == 2 and "diagonally dominant" in B.last_error()
    for pe in (1.5, 2.0):
        st, _ = _size_status(B, _desc(B, k=_centred_advdiff(63, pe)))
        assert st == 0, (pe, B.last_error())
    # symmetric positive definite but not dominant: accepted
    n = 40
    lo, di, up = np.full(n, -1.0), np.full(n, 1.999), np.full(n, -1.0)  # eigenvalues 1.999 - 2 cos(j pi/41) > 0
    lo[0] = up[-1] = 0.0
    assert np.linalg.eigvalsh(np.diag(di) + np.diag(lo[1:], -1) + np.diag(up[:-1], 1)).min() > 0
    st, _ = _size_status(B, _desc(B, k=(lo, di, up)))
    assert st == 0, B.last_error()
    # symmetric but indefinite (and not dominant): rejected
    di2 = np.full(n, 1.99)
    st, _ = _size_status(B, _desc(B, k=(lo, di2, up)))
    assert st == 2
    # a diagonal mass matrix keeps (1 - pi_k) M + tau K dominant: accepted with a dominant K
    # (even where the symmetrically scaled operator is not), rejected with a bad one
    st, _ = _size_status(B, _desc(B, k=_centred_advdiff(31, 1.0), mass=np.linspace(0.5, 2.0, 31)))
    assert st == 0, B.last_error()
    st, _ = _size_status(B, _desc(B, k=_centred_advdiff(31, 3.0), mass=np.linspace(0.5, 2.0, 31)))
    assert st == 2
    # one bad slot of a batch is found
    good, bad = _centred_advdiff(31, 1.0), _centred_advdiff(31, 3.0)
    kk = [np.concatenate([g, b]) for g, b in zip(good, bad)]
    d = _desc(B, k=kk)
    d.nx, d.batch = 31, 2
    st, _ = _size_status(B, d)
    assert st == 2 and "row 3" in B.last_error()
    # 2D: T_x dominant only with the smallest eigenvalue of T_y added (2 - 2 cos(pi/8) = 0.152)
    lo2, di2, up2 = np.full(7, -1.0), np.full(7, 1.9), np.full(7, -1.0)
    lo2[0] = up2[-1] = 0.0
    lo2[3] = -1.05  # non-symmetric, so only dominance can accept it
    st, _ = _size_status(B, _desc(B, k=(lo2, di2, up2), dim=2, ny=7))
    assert st == 0, B.last_error()
    st, _ = _size_status(B, _desc(B, k=(lo2, di2 - 0.2, up2), dim=2, ny=7))
    assert st == 2


def test_null_arguments_are_rejected(B):
    L = B.load()
    assert L.paradiag_workspace_size(None, None) == 1
    assert L.paradiag_solve(None, None, None, None) == 1
    assert L.paradiag_destroy(None) == 0
    assert "sm_103a" in B.paradiag_version()


def test_mass_matrix_adds_its_scaling_buffers(B):
    """A mass matrix adds M^{-1/2} and a scaled copy of G to the workspace."""
    st0, n0 = _size_status(B, _desc(B))
    st1, n1 = _size_status(B, _desc(B, mass=np.full(31, 2.0)))
    assert st0 == 0 and st1 == 0
    assert n1 >= n0 + (16 * 31 + 31) * 8


def test_batch_stack_pads_time_and_unstack_cuts_it():
    """Host side of uneven-n_t batches: stack zero-pads each problem's G past its n_t and
    n_x; unstack returns each problem's first n_t,b rows and n_x,b columns."""
    from types import SimpleNamespace
    from paper_2304_12597_gb300.plan import Plan
    slots = SimpleNamespace(nt=8, batch=3, nx=5, slot=5)  # slot: unknowns per problem (1D: n_x)
    arrays = [np.full((8, 5), 1.0), np.full((2, 3), 2.0), np.full((4, 1), 3.0)]
    S = Plan.stack(slots, arrays)
    assert S.shape == (8, 15)
    V = S.reshape(8, 3, 5)
    assert np.all(V[:, 0] == 1.0)
    assert np.all(V[:2, 1, :3] == 2.0) and not np.any(V[2:, 1]) and not np.any(V[:, 1, 3:])
    assert np.all(V[:4, 2, :1] == 3.0) and not np.any(V[4:, 2]) and not np.any(V[:, 2, 1:])
    parts = Plan.unstack(slots, S, [5, 3, 1], [8, 2, 4])
    for a, b in zip(arrays, parts):
        assert np.array_equal(a, b)
    with pytest.raises(ValueError):
        Plan.stack(slots, [np.zeros((9, 5))])



def test_2d_batch_limits_are_checked(B):
    """2D batches share one grid (batch_nx must be NULL) and run each problem's Algorithm 2
    in one CTA (nx ny <= 8192); both are checked before any device work, and T_y must be
    symmetric Toeplitz in every problem."""
    st, _ = _size_status(B, _desc(B, dim=2, n=127, ny=127, batch=2, precision=1))
    assert st == 2 and "8192" in B.last_error()
    st, _ = _size_status(B, _desc(B, dim=2, n=31, ny=31, batch=2, batch_nx=[31, 31]))
    assert st == 2 and "batch_nx" in B.last_error()
    y_diag = np.concatenate([np.full(7, 2.0), np.full(7, 3.0)])
    y_diag[10] = 3.5  # problem 1's T_y is not Toeplitz
    st, _ = _size_status(B, _desc(B, dim=2, n=31, ny=7, batch=2, y_diag=y_diag))
    assert st == 2 and "Toeplitz" in B.last_error()
    st, n = _size_status(B, _desc(B, dim=2, n=63, ny=63, batch=3, batch_tau=[0.1, 0.2, 0.3], precision=1))
    assert st == 0 and n > 0, B.last_error()


def test_u1_test_limits_are_checked(B):
    """The residual test on U_1 needs a single problem that runs Algorithm 2."""
    assert _size_status(B, _desc(B, early_exit_eps=1e-6, alpha=1e-4))[0] == 0, B.last_error()
    st, _ = _size_status(B, _desc(B, early_exit_eps=1e-6, batch=2))
    assert st == 2 and "early_exit_eps" in B.last_error()
    st, _ = _size_status(B, _desc(B, early_exit_eps=1e-6, loops=1))
    assert st == 2
    st, _ = _size_status(B, _desc(B, early_exit_eps=-1.0))
    assert st == 1
