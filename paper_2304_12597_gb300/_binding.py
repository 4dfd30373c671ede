"""ctypes binding of the C ABI in include/paradiag.h (argument marshalling only).

Names and argument order follow the C entry points.  Every step of the solve
runs in the CUDA library; nothing here computes.  If the library has not been
built the import of this module fails loudly: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libparadiag_gb300.so")

PD_ABI_VERSION = 1
PD_FP64 = 0
PD_MIXED = 1

STATUS = {
    0: "PD_OK",
    1: "PD_ERR_INVALID_ARG",
    2: "PD_ERR_UNSUPPORTED",
    3: "PD_ERR_OOM",
    4: "PD_ERR_CUDA",
    5: "PD_ERR_NOT_CONVERGED",
    6: "PD_ERR_NONFINITE",
    7: "PD_ERR_TIMEOUT",
}

_dp = ctypes.POINTER(ctypes.c_double)


class PdDesc(ctypes.Structure):
    _fields_ = [
        ("abi_version", ctypes.c_int32),
        ("dim", ctypes.c_int32),
        ("nx", ctypes.c_int64),
        ("ny", ctypes.c_int64),
        ("nt", ctypes.c_int64),
        ("tau", ctypes.c_double),
        ("k_lo", _dp),
        ("k_diag", _dp),
        ("k_up", _dp),
        ("k_lo_y", _dp),
        ("k_diag_y", _dp),
        ("k_up_y", _dp),
        ("m_diag", _dp),
        ("precision", ctypes.c_int32),
        ("maxit", ctypes.c_int32),
        ("eps_krylov", ctypes.c_double),
        ("q", ctypes.c_int32),
        ("max_refine", ctypes.c_int32),
        ("refine_tol", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("stream", ctypes.c_void_p),
        ("host_io", ctypes.c_int32),
        ("no_graph", ctypes.c_int32),
        ("loops", ctypes.c_int32),
        ("tune_pint_rows", ctypes.c_int32),
        ("tune_pint_teams", ctypes.c_int32),
        ("tune_krylov_ctas", ctypes.c_int32),
        ("tune_cap_ctas", ctypes.c_int32),
        ("tune_fft_cols", ctypes.c_int32),
        ("tune_no_pdl", ctypes.c_int32),
        ("tune_krylov_cluster", ctypes.c_int32),
        ("tune_pint_factor", ctypes.c_int32),
        ("tune_krylov_tails", ctypes.c_int32),
        ("batch", ctypes.c_int32),
        ("batch_nx", ctypes.POINTER(ctypes.c_int64)),
        ("batch_tau", ctypes.POINTER(ctypes.c_double)),
        ("tune_fft_radix", ctypes.c_int32),
        ("tune_persistent", ctypes.c_int32),
        ("barrier_polls", ctypes.c_int64),
        ("tune_persist_ctas", ctypes.c_int32),
        ("barrier_extra", ctypes.c_int32),
        ("tune_zero_lane", ctypes.c_int32),
        ("early_exit_eps", ctypes.c_double),
        ("eps_krylov_refine", ctypes.c_double),
        ("tune_final_loop", ctypes.c_int32),
    ]


class PdStats(ctypes.Structure):
    _fields_ = [
        ("krylov_iters", ctypes.c_int32),
        ("krylov_iters_total", ctypes.c_int32),
        ("pint_loops", ctypes.c_int32),
        ("shifted_sweeps", ctypes.c_int32),
        ("refine_sweeps", ctypes.c_int32),
        ("breakdown", ctypes.c_int32),
        ("graph", ctypes.c_int32),
        ("kernel_launches", ctypes.c_int64),
        ("beta", ctypes.c_double),
        ("krylov_rel_resnorm", ctypes.c_double),
        ("rel_update", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("sweep_krylov_iters", ctypes.c_int32 * 16),
        ("sweep_krylov_rel_resnorm", ctypes.c_double * 16),
        ("sweep_rel_update", ctypes.c_double * 16),
        ("zero_freq_fp64", ctypes.c_int32),
        ("zero_freq_weight", ctypes.c_double),
        ("persistent_step", ctypes.c_int32),
        ("early_exit", ctypes.c_int32),
        ("u1_rel_residual", ctypes.c_double),
        ("final_by_linearity", ctypes.c_int32),
    ]

    def as_dict(self):
        d = {}
        n = self.refine_sweeps
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v)[: min(n, 16)] if name.startswith("sweep_") else v
        return d


class PdKernelTime(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("launches", ctypes.c_int64),
        ("total_ms", ctypes.c_double),
        ("bytes", ctypes.c_double),
    ]


class ParadiagError(RuntimeError):
    def __init__(self, func, status, message):
        self.status = status
        self.status_name = STATUS.get(status, str(status))
        super().__init__(f"{func}: {self.status_name}: {message}")


# Every exported symbol with (restype, argtypes); the tests compare this table
# with the declarations in include/paradiag.h.
SIGNATURES = {
    "paradiag_workspace_size": (ctypes.c_int, [ctypes.POINTER(PdDesc), ctypes.POINTER(ctypes.c_size_t)]),
    "paradiag_plan": (ctypes.c_int, [ctypes.POINTER(PdDesc), ctypes.c_void_p, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "paradiag_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(PdStats)]),
    "paradiag_solve_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.POINTER(PdStats)]),
    "paradiag_batch_advance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(PdStats)]),
    "paradiag_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "paradiag_set_operator": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PdDesc)]),
    "paradiag_last_error": (ctypes.c_char_p, []),
    "paradiag_version": (ctypes.c_char_p, []),
    "paradiag_time_dft": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "paradiag_time_idft": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "paradiag_shifted_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "paradiag_dst_y": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "paradiag_recip_f32": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "paradiag_last_vectors": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "paradiag_smw_rhs_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "paradiag_set_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "paradiag_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(PdKernelTime), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the CUDA library and declare every signature.  Raises if it is missing."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"paradiag CUDA library not found at {path}; build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _lib = L
    return L


def last_error() -> str:
    return load().paradiag_last_error().decode()


def check(func: str, status: int, allow=()):
    if status != 0 and status not in allow:
        raise ParadiagError(func, status, last_error())
    return status


def paradiag_workspace_size(desc: PdDesc) -> int:
    n = ctypes.c_size_t(0)
    check("paradiag_workspace_size", load().paradiag_workspace_size(ctypes.byref(desc), ctypes.byref(n)))
    return n.value


def paradiag_plan(desc: PdDesc, workspace_ptr: int, workspace_bytes: int) -> int:
    h = ctypes.c_void_p(0)
    check("paradiag_plan", load().paradiag_plan(ctypes.byref(desc), ctypes.c_void_p(workspace_ptr or None),
                                                workspace_bytes, ctypes.byref(h)))
    return h.value


def paradiag_solve(plan: int, G_ptr: int, U_ptr: int, allow_not_converged=False) -> PdStats:
    st = PdStats()
    allow = (5,) if allow_not_converged else ()
    check("paradiag_solve", load().paradiag_solve(plan, G_ptr, U_ptr, ctypes.byref(st)), allow)
    return st


def paradiag_solve_host(plan: int, G_host_ptr: int, U_host_ptr: int, allow_not_converged=False) -> PdStats:
    st = PdStats()
    allow = (5,) if allow_not_converged else ()
    check("paradiag_solve_host", load().paradiag_solve_host(plan, G_host_ptr, U_host_ptr, ctypes.byref(st)), allow)
    return st


def paradiag_batch_advance(plan: int, G_ptr: int, U_ptr: int, join, steps: int):
    """Advance a batched solve by up to `steps` refinement sweeps; join[b] != 0 starts
    problem b.  Returns (state per problem: 1 converged, 2 gave up, 0 running; PdStats)."""
    n = len(join)
    jarr = (ctypes.c_int32 * n)(*[1 if j else 0 for j in join])
    sarr = (ctypes.c_int32 * n)()
    st = PdStats()
    check("paradiag_batch_advance", load().paradiag_batch_advance(plan, G_ptr, U_ptr, jarr, int(steps), sarr,
                                                                  ctypes.byref(st)))
    return [int(v) for v in sarr], st


def paradiag_destroy(plan: int) -> None:
    check("paradiag_destroy", load().paradiag_destroy(plan))


def paradiag_set_operator(plan: int, desc: PdDesc) -> None:
    check("paradiag_set_operator", load().paradiag_set_operator(plan, ctypes.byref(desc)))


def paradiag_time_dft(plan: int, X_ptr: int, Xhat_ptr: int) -> None:
    check("paradiag_time_dft", load().paradiag_time_dft(plan, X_ptr, Xhat_ptr))


def paradiag_time_idft(plan: int, Y_ptr: int, X_ptr: int) -> None:
    check("paradiag_time_idft", load().paradiag_time_idft(plan, Y_ptr, X_ptr))


def paradiag_shifted_solve(plan: int, R_ptr: int, Y_ptr, b_ptr) -> None:
    check("paradiag_shifted_solve", load().paradiag_shifted_solve(plan, R_ptr, Y_ptr, b_ptr))


def paradiag_dst_y(plan: int, X_ptr: int, Y_ptr: int) -> None:
    check("paradiag_dst_y", load().paradiag_dst_y(plan, X_ptr, Y_ptr))


def paradiag_recip_f32(x_ptr: int, r_ptr: int, n: int, stream_ptr) -> None:
    check("paradiag_recip_f32", load().paradiag_recip_f32(x_ptr, r_ptr, n, stream_ptr))


def paradiag_last_vectors(plan: int, b_ptr, x_ptr) -> None:
    check("paradiag_last_vectors", load().paradiag_last_vectors(plan, b_ptr, x_ptr))


def paradiag_smw_rhs_noalloc(nt: int, n: int, tau: float, k_lo_ptr: int, k_diag_ptr: int, k_up_ptr: int,
                             R_ptr: int, Y_ptr, b_ptr: int, stream_ptr) -> None:
    """Allocation-free first parallel-in-time loop and b (eq. 7); see include/paradiag.h.
    For callers that cannot allocate device memory: scratch is a static device array."""
    check("paradiag_smw_rhs_noalloc", load().paradiag_smw_rhs_noalloc(nt, n, tau, k_lo_ptr, k_diag_ptr, k_up_ptr,
                                                                      R_ptr, Y_ptr, b_ptr, stream_ptr))


def paradiag_set_timing(plan: int, enable: bool) -> None:
    check("paradiag_set_timing", load().paradiag_set_timing(plan, 1 if enable else 0))


def paradiag_kernel_times(plan: int):
    n = ctypes.c_int(0)
    buf = (PdKernelTime * 64)()
    check("paradiag_kernel_times", load().paradiag_kernel_times(plan, buf, 64, ctypes.byref(n)))
    return [{"name": buf[i].name.decode(), "launches": buf[i].launches, "total_ms": buf[i].total_ms,
             "bytes": buf[i].bytes} for i in range(min(n.value, 64))]


def paradiag_version() -> str:
    return load().paradiag_version().decode()
