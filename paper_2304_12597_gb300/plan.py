"""Python wrapper of one ParaDiag plan: torch supplies device memory and the stream.

A ``Plan`` holds the C plan handle, its device workspace (a torch uint8
tensor) and the host copies of the operator it was built from.  All arithmetic
happens in the CUDA library behind ``paradiag_*``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _binding as B


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Plan:
    """All-at-once backward-Euler solver (Algorithm 1 + Algorithm 2) for one problem shape.

    Parameters mirror ``pd_desc`` in include/paradiag.h.  ``precision`` is
    "fp64" or "mixed".  ``tune`` maps launch-geometry names (pint_rows, pint_teams,
    krylov_ctas, cap_ctas, fft_cols) to values; 0 or absent = built-in choice.
    G and U passed to ``solve`` are (nt, nx*ny) float64 CUDA
    tensors, row j = time step j+1, spatial index contiguous.
    """

    def __init__(self, *, dim, nx, nt, tau, k_lo, k_diag, k_up, ny=1, k_lo_y=None, k_diag_y=None,
                 k_up_y=None, m_diag=None, precision="mixed", maxit=0, eps_krylov=0.0, max_refine=0, refine_tol=0.0,
                 alpha=1.0, q=1, loops=0, host_io=False, no_graph=False, tune=None, batch=1, batch_nx=None, batch_tau=None,
                 barrier_polls=0, barrier_extra=0, eps_krylov_refine=0.0, early_exit_eps=0.0, device=None,
                 stream=None, workspace="torch"):
        import torch

        self._torch = torch
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.dim, self.nx, self.ny, self.nt = int(dim), int(nx), int(ny if dim == 2 else 1), int(nt)
        self.batch = max(int(batch), 1)
        self.nbar = self.nx * self.ny * self.batch
        self.precision = precision
        self._arrays = [_f64(k_lo), _f64(k_diag), _f64(k_up), _f64(k_lo_y), _f64(k_diag_y), _f64(k_up_y),
                        _f64(m_diag)]
        self._batch_nx = None if batch_nx is None else np.ascontiguousarray(batch_nx, dtype=np.int64)
        self._batch_tau = _f64(batch_tau)
        d = B.PdDesc()
        d.abi_version = B.PD_ABI_VERSION
        d.dim = self.dim
        d.nx = self.nx
        d.ny = self.ny
        d.nt = self.nt
        d.tau = float(tau)
        d.k_lo, d.k_diag, d.k_up, d.k_lo_y, d.k_diag_y, d.k_up_y, d.m_diag = [_ptr(a) for a in self._arrays]
        d.precision = {"fp64": B.PD_FP64, "mixed": B.PD_MIXED}[precision]
        d.maxit = int(maxit)
        d.eps_krylov = float(eps_krylov)
        d.q = int(q)  # Algorithm 2 checks its residual every q steps (frozen residual, Sec. 3)
        d.max_refine = int(max_refine)
        d.refine_tol = float(refine_tol)
        d.alpha = float(alpha)
        d.stream = ctypes.c_void_p(self.stream.cuda_stream)
        d.host_io = 1 if host_io else 0
        d.no_graph = 1 if no_graph else 0
        d.loops = int(loops)  # 1: U = U_1; 2: x_m = b (fixed-cost variants, Table 3)
        for key, val in (tune or {}).items():  # launch geometry: pint_rows, pint_teams, krylov_ctas, ...
            setattr(d, "tune_" + key, int(val))
        # bounded waits of the persistent Algorithm-2 step; barrier_extra > 0 only to test them
        d.barrier_polls = int(barrier_polls)
        d.barrier_extra = int(barrier_extra)
        d.eps_krylov_refine = float(eps_krylov_refine)
        d.early_exit_eps = float(early_exit_eps)  # Algorithm 3's residual test on U_1 (0 = off)
        d.batch = self.batch if self.batch > 1 else 0
        if self._batch_nx is not None:
            d.batch_nx = self._batch_nx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        if self._batch_tau is not None:
            d.batch_tau = _ptr(self._batch_tau)
        self.desc = d
        self.workspace_bytes = B.paradiag_workspace_size(d)
        self.handle = None
        with torch.cuda.device(self.device):
            if workspace == "torch":
                self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
                base = self._ws.data_ptr()
                ptr = (base + 255) // 256 * 256
                self.handle = B.paradiag_plan(d, ptr, self.workspace_bytes)
            else:
                self._ws = None
                self.handle = B.paradiag_plan(d, 0, 0)

    @classmethod
    def from_problems(cls, problems, **kw):
        """One batched plan for a list of problems (fields of workloads.Problem).  1D: slot b
        holds problem b, padded to the largest n_x (or to the keyword nx, if larger).  2D:
        every problem has the same nx x ny grid (nx ny <= 8192), its own T_x, T_y and tau,
        and slot b is its nx ny unknowns.

        The plan's n_t is the largest n_t,b.  Backward Euler is causal: rows 1..l_b of the
        all-at-once solution depend only on rows 1..l_b of G.  So a problem with fewer time
        steps is solved exactly by the longer system with its G extended by zero rows
        (stack), and its answer is the first n_t,b rows of its slot (unstack)."""
        nt = max(P.nt for P in problems)
        dims = {P.dim for P in problems}
        if dims == {2}:
            return cls._from_problems_2d(problems, nt, **kw)
        if dims != {1}:
            raise ValueError("a batch needs problems of one dimension")
        nx = max(max(P.nx for P in problems), int(kw.pop("nx", 0) or 0))  # slot length
        B = len(problems)
        lo, di, up = np.zeros((B, nx)), np.ones((B, nx)), np.zeros((B, nx))
        md = np.ones((B, nx))
        for b, P in enumerate(problems):
            lo[b, :P.nx], di[b, :P.nx], up[b, :P.nx] = P.k_lo, P.k_diag, P.k_up
            if getattr(P, "m_diag", None) is not None:
                md[b, :P.nx] = P.m_diag
        any_mass = any(getattr(P, "m_diag", None) is not None for P in problems)
        args = dict(dim=1, nx=nx, nt=nt, tau=problems[0].tau, k_lo=lo.ravel(), k_diag=di.ravel(), k_up=up.ravel(),
                    m_diag=md.ravel() if any_mass else None,
                    batch=B, batch_nx=[P.nx for P in problems], batch_tau=[P.tau for P in problems])
        args.update(kw)
        return cls(**args)

    @classmethod
    def _from_problems_2d(cls, problems, nt, **kw):
        nx, ny = problems[0].nx, problems[0].ny
        kw.pop("nx", None)  # the slot is the grid itself
        if any(P.nx != nx or P.ny != ny for P in problems):
            raise ValueError("a 2D batch needs problems of one grid size")
        cat = lambda name: np.concatenate([np.asarray(getattr(P, name), dtype=np.float64) for P in problems])
        args = dict(dim=2, nx=nx, ny=ny, nt=nt, tau=problems[0].tau, k_lo=cat("k_lo"), k_diag=cat("k_diag"),
                    k_up=cat("k_up"), k_lo_y=cat("k_lo_y"), k_diag_y=cat("k_diag_y"), k_up_y=cat("k_up_y"),
                    batch=len(problems), batch_tau=[P.tau for P in problems])
        args.update(kw)
        return cls(**args)

    @property
    def slot(self):
        """Unknowns per problem slot of a batched plan (n_x in 1D, n_x n_y in 2D)."""
        return self.nx * self.ny

    def stack(self, arrays):
        """(nt, batch * slot) float64 array with array b (n_t,b, n_x,b) in slot b, zero-padded
        in space and, past row n_t,b, in time (2D: arrays of n_x n_y columns)."""
        out = np.zeros((self.nt, self.batch, self.slot))
        for b, a in enumerate(arrays):
            if a.shape[0] > self.nt or a.shape[1] > self.slot:
                raise ValueError("array does not fit its slot")
            out[:a.shape[0], b, :a.shape[1]] = a
        return out.reshape(self.nt, self.batch * self.slot)

    def unstack(self, U, nxs, nts=None):
        """Slot b of a (nt, batch * slot) array, cut to n_x,b columns (2D: n_x n_y) and its
        first n_t,b rows (all rows when nts is None)."""
        V = U.reshape(self.nt, self.batch, self.slot)
        nts = [self.nt] * len(nxs) if nts is None else nts
        return [V[:t, b, :n] for b, (n, t) in enumerate(zip(nxs, nts))]

    @classmethod
    def from_problem(cls, problem, **kw):
        """Build from any object with the fields of workloads.Problem."""
        args = dict(dim=problem.dim, nx=problem.nx, ny=problem.ny, nt=problem.nt, tau=problem.tau,
                    k_lo=problem.k_lo, k_diag=problem.k_diag, k_up=problem.k_up,
                    k_lo_y=problem.k_lo_y, k_diag_y=problem.k_diag_y, k_up_y=problem.k_up_y,
                    m_diag=getattr(problem, "m_diag", None))
        args.update(kw)
        return cls(**args)

    def set_operator(self, *, tau, k_lo, k_diag, k_up, k_lo_y=None, k_diag_y=None, k_up_y=None, m_diag=None,
                     batch_nx=None, batch_tau=None):
        """Swap in a new operator (and mass matrix) of the same shape (paradiag_set_operator)."""
        arrays = [_f64(k_lo), _f64(k_diag), _f64(k_up), _f64(k_lo_y), _f64(k_diag_y), _f64(k_up_y), _f64(m_diag)]
        bnx = None if batch_nx is None else np.ascontiguousarray(batch_nx, dtype=np.int64)
        btau = _f64(batch_tau)
        d = B.PdDesc()
        ctypes.pointer(d)[0] = self.desc  # copy of the plan's descriptor
        d.tau = float(tau)
        d.k_lo, d.k_diag, d.k_up, d.k_lo_y, d.k_diag_y, d.k_up_y, d.m_diag = [_ptr(a) for a in arrays]
        d.batch_nx = bnx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if bnx is not None else None
        d.batch_tau = _ptr(btau) if btau is not None else None
        B.paradiag_set_operator(self.handle, d)
        self._arrays, self._batch_nx, self._batch_tau = arrays, bnx, btau
        self.desc = d

    def set_problems(self, problems):
        """Swap in the operators of a list of problems (same batch size, n_t,b <= the plan's
        n_t; 1D: n_x,b <= its slot length; 2D: the plan's grid); see from_problems."""
        if self.dim == 2:
            if len(problems) != self.batch or any(P.dim != 2 or P.nt > self.nt or P.nx != self.nx or P.ny != self.ny
                                                  for P in problems):
                raise ValueError("problems do not fit this plan's slots")
            cat = lambda name: np.concatenate([np.asarray(getattr(P, name), dtype=np.float64) for P in problems])
            self.set_operator(tau=problems[0].tau, k_lo=cat("k_lo"), k_diag=cat("k_diag"), k_up=cat("k_up"),
                              k_lo_y=cat("k_lo_y"), k_diag_y=cat("k_diag_y"), k_up_y=cat("k_up_y"),
                              batch_tau=[P.tau for P in problems])
            return
        if len(problems) != self.batch or any(P.dim != 1 or P.nt > self.nt or P.nx > self.nx for P in problems):
            raise ValueError("problems do not fit this plan's slots")
        nx = self.nx
        lo, di, up = np.zeros((self.batch, nx)), np.ones((self.batch, nx)), np.zeros((self.batch, nx))
        for b, P in enumerate(problems):
            lo[b, :P.nx], di[b, :P.nx], up[b, :P.nx] = P.k_lo, P.k_diag, P.k_up
        self.set_operator(tau=problems[0].tau, k_lo=lo.ravel(), k_diag=di.ravel(), k_up=up.ravel(),
                          batch_nx=[P.nx for P in problems], batch_tau=[P.tau for P in problems])

    # -- helpers -------------------------------------------------------------------
    def _check(self, t, dtype, shape):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or t.device != self.device or t.dtype != dtype:
            raise ValueError(f"expected a {dtype} tensor on {self.device}")
        if tuple(t.shape) != tuple(shape) or not t.is_contiguous():
            raise ValueError(f"expected a contiguous tensor of shape {shape}, got {tuple(t.shape)}")

    @property
    def spectrum_dtype(self):
        torch = self._torch
        return torch.complex128 if self.precision == "fp64" else torch.complex64

    # -- main entry points ---------------------------------------------------------
    def solve(self, G, U=None, allow_not_converged=False):
        """U = solution of eq. (2) for right-hand side G.  Returns (U, stats dict)."""
        torch = self._torch
        shape = (self.nt, self.nbar)
        self._check(G, torch.float64, shape)
        if U is None:
            U = torch.empty_like(G)
        self._check(U, torch.float64, shape)
        st = B.paradiag_solve(self.handle, G.data_ptr(), U.data_ptr(), allow_not_converged)
        return U, st.as_dict()

    def advance(self, G, U, join, steps=1):
        """Batched plans: advance every problem by up to `steps` refinement sweeps on U (in
        place); join[b] starts problem b (its slot of U restarts from zero).  Returns
        (state per slot: 1 converged, 2 gave up, 0 running; stats dict of this call)."""
        torch = self._torch
        shape = (self.nt, self.nbar)
        self._check(G, torch.float64, shape)
        self._check(U, torch.float64, shape)
        if len(join) != self.batch:
            raise ValueError("join needs one flag per slot")
        state, st = B.paradiag_batch_advance(self.handle, G.data_ptr(), U.data_ptr(), join, steps)
        return state, st.as_dict()

    def solve_host(self, G_host, U_host, allow_not_converged=False):
        """Host-buffer variant: G_host, U_host are CPU tensors (pinned preferred)."""
        torch = self._torch
        for t in (G_host, U_host):
            if t.device.type != "cpu" or t.dtype != torch.float64 or not t.is_contiguous():
                raise ValueError("host buffers must be contiguous CPU float64 tensors")
            if tuple(t.shape) != (self.nt, self.nbar):
                raise ValueError("host buffer has the wrong shape")
        st = B.paradiag_solve_host(self.handle, G_host.data_ptr(), U_host.data_ptr(), allow_not_converged)
        return U_host, st.as_dict()

    # -- stage entry points --------------------------------------------------------
    def time_dft(self, X):
        torch = self._torch
        self._check(X, torch.float64, (self.nt, self.nbar))
        nf = self.nt // 2 + 1 if self.nt > 1 else 1
        Xhat = torch.empty((nf, self.nbar), dtype=self.spectrum_dtype, device=self.device)
        B.paradiag_time_dft(self.handle, X.data_ptr(), Xhat.data_ptr())
        return Xhat

    def time_idft(self, Y):
        torch = self._torch
        nf = self.nt // 2 + 1 if self.nt > 1 else 1
        self._check(Y, self.spectrum_dtype, (nf, self.nbar))
        X = torch.empty((self.nt, self.nbar), dtype=torch.float64, device=self.device)
        B.paradiag_time_idft(self.handle, Y.data_ptr(), X.data_ptr())
        return X

    def shifted_solve(self, R, want_y=True, want_b=True):
        torch = self._torch
        nf = self.nt // 2 + 1 if self.nt > 1 else 1
        self._check(R, self.spectrum_dtype, (nf, self.nbar))
        Y = torch.empty_like(R) if want_y else None
        b = torch.empty(self.nbar, dtype=torch.float64, device=self.device) if want_b else None
        B.paradiag_shifted_solve(self.handle, R.data_ptr(), Y.data_ptr() if Y is not None else None,
                                 b.data_ptr() if b is not None else None)
        return Y, b

    def dst_y(self, X):
        torch = self._torch
        self._check(X, torch.float64, (self.nt, self.nbar))
        Y = torch.empty_like(X)
        B.paradiag_dst_y(self.handle, X.data_ptr(), Y.data_ptr())
        return Y

    def last_vectors(self):
        torch = self._torch
        b = torch.empty(self.nbar, dtype=torch.float64, device=self.device)
        x = torch.empty_like(b)
        B.paradiag_last_vectors(self.handle, b.data_ptr(), x.data_ptr())
        return b, x

    def set_timing(self, enable=True):
        B.paradiag_set_timing(self.handle, enable)

    def kernel_times(self):
        return B.paradiag_kernel_times(self.handle)

    def close(self):
        if self.handle:
            B.paradiag_destroy(self.handle)
            self.handle = None
        self._ws = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
