/*
 * paradiag.h — C ABI of the GB300 (sm_103a) implementation of the new ParaDiag
 * method of Gander & Palitta, "A new ParaDiag time-parallel time integration
 * method" (arXiv 2304.12597).
 *
 * The library solves the all-at-once backward-Euler system (Sec. 1, eq. 2)
 *
 *     (I + tau K) U - U Sigma_1^T = G,     U = [u_1, ..., u_l],
 *
 * by Algorithm 1 (Sec. 2): Sigma_1 = C_1 - e_1 e_l^T (eq. 3), the circulant
 * part is diagonalised by an FFT along time (eq. 5), the block-diagonal
 * shifted systems ((1 - pi_i) I + tau K) are solved in parallel, and the
 * rank-one Sherman-Morrison-Woodbury correction (eqs. 6-8) is resolved by the
 * FOM-like Krylov method of Algorithm 2 (Sec. 3, eqs. 9-13).
 *
 * Conventions used by every entry point:
 *  - n_bar = nx * ny spatial unknowns, l = nt time steps, tau = T / l.
 *  - G and U are row-major (nt, n_bar) float64 arrays with the spatial index
 *    contiguous; row j is time step j+1 (the paper's column-major U in R^{n_bar x l}).
 *    Row 0 of G is u_0 + tau f_1, row j >= 1 is tau f_{j+1} (eq. 2).
 *  - In 2D the spatial index is iy * nx + ix and K = I_ny (x) T_x + T_y (x) I_nx
 *    (Sec. 6.1).
 *  - "device" pointers are CUDA global-memory addresses on the current device
 *    (e.g. torch tensor data pointers); "host" pointers are ordinary memory.
 *  - No entry point throws; each returns a pd_status.  After PD_ERR_CUDA the
 *    plan must be destroyed.  paradiag_last_error() returns a thread-local
 *    message for the last failure on the calling thread.
 *  - A plan is not thread safe: one solve at a time per plan.
 */
#ifndef PARADIAG_H
#define PARADIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PD_ABI_VERSION 1

typedef enum pd_status {
  PD_OK = 0,
  PD_ERR_INVALID_ARG = 1,   /* bad size, pointer, alignment or parameter */
  PD_ERR_UNSUPPORTED = 2,   /* valid request outside what this build implements */
  PD_ERR_OOM = 3,           /* workspace too small or device allocation failed */
  PD_ERR_CUDA = 4,          /* a CUDA runtime call failed; destroy the plan */
  PD_ERR_NOT_CONVERGED = 5, /* Krylov or refinement limit reached; U holds the last iterate */
  PD_ERR_NONFINITE = 6,     /* NaN/Inf met in the input or an intermediate norm */
  PD_ERR_TIMEOUT = 7        /* a bounded device-side wait (a grid barrier of the persistent
                               Algorithm-2 step) ran out; U is unspecified, the plan stays
                               usable */
} pd_status;

typedef enum pd_precision {
  PD_FP64 = 0,  /* every step in IEEE binary64 */
  PD_MIXED = 1  /* FFTs and shifted solves in complex binary32; Krylov, capacitance
                   system, all-at-once residual and the solution update in binary64;
                   iterative refinement recovers FP64 accuracy */
} pd_precision;

/* Problem and solver description.  Host arrays are copied at plan time and may be
 * freed afterwards.  Fill unused fields with 0 / NULL. */
typedef struct pd_desc {
  int32_t abi_version;   /* must be PD_ABI_VERSION */
  int32_t dim;           /* 1 or 2 */
  int64_t nx;            /* 1D: n_bar; 2D: grid points along x (contiguous) */
  int64_t ny;            /* 1D: 1;     2D: grid points along y */
  int64_t nt;            /* l, number of time steps: a power of two, 1 <= l <= 8192 */
  double tau;            /* time step tau = T / l > 0 */
  /* K (1D) or T_x (2D): tridiagonal, row i = lo[i] u[i-1] + diag[i] u[i] + up[i] u[i+1];
   * lo[0] and up[n-1] are ignored.  Length nx, host memory.  The shifted systems are
   * eliminated without pivoting, so every block must be weakly diagonally dominant by rows
   * (diag[i] >= |lo[i]| + |up[i]|; in 2D with the smallest eigenvalue of T_y added to
   * diag) or symmetric positive definite; otherwise PD_ERR_UNSUPPORTED (e.g. centred
   * advection at cell Peclet number > 2). */
  const double *k_lo, *k_diag, *k_up;
  /* 2D only: T_y, length ny, host memory.  This build requires T_y to be symmetric
   * Toeplitz (constant diagonal and constant off-diagonal) and ny + 1 to be a power
   * of two <= 4096, so that T_y is diagonalised by the orthonormal DST-I. */
  const double *k_lo_y, *k_diag_y, *k_up_y;
  /* Diagonal mass matrix M (1D only; NULL = identity), host memory, length nx (batch *
   * nx for a batch, one entry per row of every slot), every entry > 0 and finite.  The
   * system is then (B (x) M + I (x) K) u = f: each step solves (M + tau K) u_j =
   * M u_{j-1} + G_j, with G_1 = M u_0 + tau f_1.  The plan solves for w = M^{1/2} u with
   * K' = M^{-1/2} K M^{-1/2} (symmetric scaling, so K' stays tridiagonal and Algorithm 1
   * applies unchanged) and scales G and U on the device.  The stage entry points work
   * in those scaled variables. */
  const double *m_diag;
  int32_t precision;     /* pd_precision */
  int32_t maxit;         /* Algorithm 2 iteration limit, 1 <= maxit <= 32 (0 = 32) */
  double eps_krylov;     /* Algorithm 2 tolerance epsilon (stop when ||r|| <= eps * ||b||);
                            0 = 1e-13 for PD_FP64 (1e-5 for PD_FP64 batches and alpha < 1,
                            which always refine and leave a stalled step at any level),
                            1e-4 for the first solve of PD_MIXED
                            (its refinement sweeps use max(eps_krylov, eps_krylov_refine)).
                            Both also stop when ||r|| stalls near the precision floor (no
                            halving over 1 iteration in PD_MIXED once ||r|| <= 1e-3 ||b||, and
                            over 2 once ||r|| <= 10 eps_krylov_refine ||b|| in its refinement
                            sweeps; over 3 iterations in PD_FP64 once ||r|| <= 1e-6 ||b||) */
  int32_t q;             /* residual check period of Algorithm 2 (Sec. 3, the frozen residual):
                            the shifted solves h_k, eq. (12) and eq. (13) run only at steps
                            m with m mod q = 0, at m = maxit and at a breakdown, so a solve
                            runs about m/q + 2 parallel-in-time loops.  0 or 1 = every step;
                            at most 32; q > 1 is built for single problems (batch <= 1) */
  int32_t max_refine;    /* refinement sweeps after the first solve (0 = 8, 16 for batches,
                            which stop only when every problem has converged).  PD_MIXED always
                            refines; PD_FP64 refines when Algorithm 2 stopped short of
                            eps_krylov (stall or maxit) or when eps_krylov > 1e-10, since the
                            residual of eq. (2) left by an inexact x_m is exactly -r_m in the
                            first time step */
  double refine_tol;     /* refinement stops when the predicted remaining relative error,
                            (||delta_s|| / ||delta_{s-1}||) * ||delta_s|| / ||U||, is <= refine_tol
                            (0 = 1e-14 for PD_FP64, 1e-11 for PD_MIXED) */
  double alpha;          /* alpha of Sec. 4 in (0, 1] (0 = 1): 1 runs Algorithm 1, alpha < 1
                            Algorithm 3 (alpha-circulant C_alpha, eq. 15: pi_k = alpha^{1/l}
                            omega^k, time rows scaled by D_alpha before the DFT and by
                            D_alpha^{-1} after the inverse, the inner system of eq. 17 and
                            the correction weighted by alpha^{1/l}).  Every solve then loses up
                            to kappa(F D_alpha) = alpha^{-(l-1)/l}, so alpha < 1 always
                            refines (PD_FP64 too).  The stage entry points keep the plain
                            DFT; paradiag_shifted_solve uses the plan's shifts. */
  void *stream;          /* cudaStream_t every launch is ordered on (NULL = legacy stream) */
  int32_t host_io;       /* nonzero: reserve device staging for paradiag_solve_host */
  int32_t no_graph;      /* nonzero: drive the Algorithm-2 and refinement loops from the host
                            instead of running each solve as one CUDA graph with device-side
                            conditionals (also the behaviour while kernel timing is enabled) */
  int32_t loops;         /* fixed-cost variants of Algorithms 1 and 3 (Sec. 6, Table 3), one
                            solve with no refinement and no Algorithm 2: 2 = x_m = b (the
                            inner matrix of eq. 17 approximated by the identity: the b loop
                            and the final loop); 1 = U = U_1 (the first loop alone, no
                            correction).  The result is the variant's approximation, so the
                            solve returns PD_OK without a convergence test.  0 = the full
                            method.  Single problems only (batch <= 1) */
  /* Launch geometry; 0 selects the built-in choice (paradiag_autotune fills these). */
  int32_t tune_pint_rows;    /* rows per thread of the shifted-solve kernel: 4, 8, or 16
                                (16 with PD_MIXED only) */
  int32_t tune_pint_teams;   /* teams (one tridiagonal block each) per CTA of that kernel:
                                a power of two with teams * threads-per-team <= 512
                                (<= 256 with 16 rows per thread) */
  int32_t tune_krylov_ctas;  /* CTAs of the Krylov vector kernels: 1 = one 512-thread CTA
                                (n_bar <= 8192), > 1 = cooperative launch of 512-thread CTAs
                                (<= SM count) */
  int32_t tune_cap_ctas;     /* CTAs of the capacitance-term kernel, 1 .. 1024 */
  int32_t tune_fft_cols;     /* columns per CTA of the time FFTs: 2, 4, 8 or 16 */
  int32_t tune_no_pdl;       /* nonzero: launch kernels without programmatic dependent launch
                                (by default a kernel may be scheduled while its predecessor
                                drains; it waits for it before reading anything) */
  int32_t tune_krylov_cluster; /* where one CTA would run the Krylov vector kernels: -1 =
                                keep that single CTA; 4 .. 16 = spread them over a
                                thread-block cluster of that many CTAs, one per SM, with the
                                reductions through distributed shared memory */
  int32_t tune_pint_factor;  /* 1: factor every shifted system once per operator (plan
                                creation, paradiag_set_operator) and keep the factors (at
                                most 4 GiB), so each parallel-in-time loop only solves; -1:
                                eliminate in every loop; 0: factor PD_FP64 plans only (FP64
                                elimination is costly on GB300; binary32 elimination costs
                                less than streaming its factors) */
  int32_t tune_krylov_tails; /* single-CTA vector work (the start of Algorithm 2: beta and v_1;
                                the eq. (13) projection and decision) in the last CTA of the
                                reduction before it (b, z) instead of separate launches: 1 =
                                also when the Arnoldi step runs on a cluster; -1 = only with
                                the single CTA; 0 = built-in choice */
  /* Batching (1D only): `batch` independent problems are solved together as one
   * block-diagonal problem (their DFTs, shifted solves and refinement sweeps are shared,
   * each problem runs its own Algorithm 2, and the blocks never couple).  A problem with
   * fewer time steps nt_b < nt rides along exactly: backward Euler is causal, so rows
   * 1..nt_b of the solution depend on rows 1..nt_b of G alone; give it zero rows
   * nt_b+1..nt in G and read the first nt_b rows of U.  Problem b occupies slot b:
   * columns [b*nx, b*nx + nx_b) of G and U, rows [b*nx, b*nx + nx_b) of k_lo/k_diag/
   * k_up (so those arrays have length batch*nx); columns nx_b..nx-1 of a slot must be
   * zero in G and are returned as zero.  Each problem is scaled to unit Frobenius norm
   * on the device before the solve and scaled back after it, so the stopping rules
   * hold for every problem, not just for the stack.  0 or 1 = a single problem. */
  int32_t batch;
  const int64_t *batch_nx;   /* host, length batch: rows of problem b, 1 <= nx_b <= nx
                                (NULL = nx for all) */
  const double *batch_tau;   /* host, length batch: time step of problem b (NULL = tau) */
  int32_t tune_fft_radix;    /* first stages of the time DFTs and the DST along y: 16 = one
                                radix-16 stage in registers (n >= 16), then radix-4 passes in
                                shared memory; 4 = radix-4 (and one radix-2) passes only;
                                0 = built-in choice (16 for binary32 transforms of n >= 16, 4
                                otherwise; the residual-on-load DFT always uses 4) */
  int32_t tune_persistent;   /* single problems: run each Algorithm-2 step after its shifted
                                solves as one persistent cooperative launch (the eq. (12)
                                terms and system, z, eq. (13) with the stopping decision, and
                                the next Arnoldi step, separated by grid barriers whose waits
                                are bounded, see barrier_polls) instead of one launch per
                                phase: 1 = on where it applies, -1 or 0 = off (the built-in
                                choice: inside one CUDA graph the per-phase launches overlap
                                their launch latency with programmatic dependent launch, and
                                measured 1-11 % faster per solve on GB300).  Batches always
                                use the per-phase launches. */
  int64_t barrier_polls;     /* polls of a grid barrier of the persistent step before it gives
                                up: the solve then returns PD_ERR_TIMEOUT (0 = 4194304, some
                                seconds) */
  int32_t tune_persist_ctas; /* CTAs of the persistent step, 1 .. one per SM (0 = one per SM) */
  int32_t barrier_extra;     /* testing the bounded wait: every grid barrier of the persistent
                                step waits for this many more CTAs than the launch has, so no
                                barrier completes and every wait runs out; 0 in normal use */
  int32_t tune_zero_lane;    /* PD_MIXED: solve the zero frequency in FP64 inside the binary32
                                loops: 1 = always, -1 = never, 0 = built-in choice (see
                                pd_stats.zero_freq_fp64) */
  double early_exit_eps;     /* Algorithm 3's optional test on U_1 (single problems, loops = 0):
                                after the first parallel-in-time loop, U_1 = L F^{-T} D_alpha^{-1}
                                is formed and, if ||(I + tau K) U_1 - U_1 Sigma_1^T - G||_F <=
                                early_exit_eps ||U_1||_F, the solve returns U = U_1 without
                                Algorithm 2, the final loop or refinement (pd_stats.early_exit).
                                0 = off (the test costs an inverse DFT and a residual pass) */
  double eps_krylov_refine;  /* PD_MIXED: Algorithm 2 tolerance of the refinement sweeps (0 = 3e-3);
                                a sweep's Algorithm 2 also leaves once its residual is below
                                10 eps_krylov_refine and stops halving */
  int32_t tune_final_loop;   /* single problems, loops = 0: when Algorithm 2 stops at 1 <= m <= 16,
                                form Algorithm 1's final loop by linearity instead of a third set
                                of shifted solves: Y_k = L_k - V_m s_k + c_k h_k, where
                                L_k = A_k^{-1} G^_k is stored by the first loop, h_k = A_k^{-1}
                                v_{m+1} by Algorithm 2's last step, s_k = alpha^{1/l} S_k y_m with
                                S_k = (sigma_k I + tau T_m)^{-1} from the last eq. (12) system
                                (sigma_k = 1 - alpha^{1/l} pi_k the frequency's shift), and
                                c_k = tau t_{m+1,m} (e_m^T s_k) (eq. 10's relation
                                tau K V_m = V_m tau T_m + tau t_{m+1,m} v_{m+1} e_m^T), formed by
                                one elementwise pass over the spectrum.  0 = on where it applies
                                (costs one spectrum-sized buffer), -1 = always run the final
                                loop's solves.  Not used with the binary32 path's FP64
                                zero-frequency lane. */
} pd_desc;

/* Statistics of the last paradiag_solve / paradiag_solve_host. */
typedef struct pd_stats {
  int32_t krylov_iters;        /* m of the last Algorithm-2 run */
  int32_t krylov_iters_total;  /* sum of m over all refinement sweeps */
  int32_t pint_loops;          /* parallel-in-time loops in the paper's count, m/q + 2 per solve */
  int32_t shifted_sweeps;      /* passes over all l/2+1 shifted systems executed (h_k is stored,
                                  so the residual of eq. (13) needs no second pass) */
  int32_t refine_sweeps;       /* solves performed (first solve + refinement sweeps) */
  int32_t breakdown;           /* 1 if Algorithm 2 met an invariant Krylov space */
  int32_t graph;               /* 1 if the solve ran as one CUDA-graph launch */
  int64_t kernel_launches;     /* this library's kernel launches during the solve */
  double beta;                 /* ||b|| of the last Algorithm-2 run */
  double krylov_rel_resnorm;   /* eq. (13) residual / ||b|| at exit of the last run */
  double rel_update;           /* ||delta||_F / ||U||_F of the last refinement sweep (0 if none) */
  double ms_total;             /* wall time of the solve measured with CUDA events */
  /* per solve (first solve, then each refinement sweep; first 16): */
  int32_t sweep_krylov_iters[16];        /* m of Algorithm 2 */
  double sweep_krylov_rel_resnorm[16];   /* eq. (13) residual / ||b|| at exit */
  double sweep_rel_update[16];           /* ||delta_s||_F / ||delta_0||_F */
  /* PD_MIXED: 1 if the zero frequency (the shifted system (1 - alpha^{1/l}) I + tau K) was
     solved in FP64 inside the binary32 loops, which the plan chooses when J_l's
     zero-frequency term is large: zero_freq_weight = ||(l A_0)^{-1}||_inf (estimated) > 4,
     about 1 / (T lambda_min(K)) for Algorithm 1 (Theorem 3.1), where binary32 solves of A_0
     would keep refinement from contracting */
  int32_t zero_freq_fp64;
  double zero_freq_weight;
  int32_t persistent_step;  /* 1 if each Algorithm-2 step ran as the persistent launch
                               (pd_desc.tune_persistent) */
  int32_t early_exit;       /* 1 if Algorithm 3's test on U_1 passed and U = U_1 */
  double u1_rel_residual;   /* ||(I + tau K) U_1 - U_1 Sigma_1^T - G||_F / ||U_1||_F of that test
                               (0 when early_exit_eps = 0) */
  int32_t final_by_linearity;  /* solves whose final loop was formed by linearity
                                  (pd_desc.tune_final_loop); shifted_sweeps excludes them */
} pd_stats;

typedef struct pd_plan pd_plan;

/* Device workspace a plan for *desc needs (bytes).  Pure host computation.
 * Errors: PD_ERR_INVALID_ARG / PD_ERR_UNSUPPORTED for a bad or unbuilt desc. */
pd_status paradiag_workspace_size(const pd_desc *desc, size_t *bytes);

/* Build a plan: validate desc, copy the operator, compute pi_i = omega^{i},
 * gamma_i = pi_i / l (Algorithm 1, first step; appendix), the FFT twiddles and the
 * per-axis transforms, and upload them.  workspace: device memory of at least
 * paradiag_workspace_size() bytes, 256-byte aligned, owned by the caller and kept
 * alive until paradiag_destroy; NULL asks the plan to cudaMalloc its own.
 * *out receives the plan.  Runs synchronously on desc->stream. */
pd_status paradiag_plan(const pd_desc *desc, void *workspace, size_t workspace_bytes,
                        pd_plan **out);

/* Solve eq. (2) for one right-hand side: Algorithm 1 with Algorithm 2 (PD_FP64), or
 * iterative refinement around it (PD_MIXED).  G_dev: device, (nt, n_bar) float64,
 * read only.  U_dev: device, (nt, n_bar) float64, overwritten; must not alias G_dev.
 * Both 8-byte aligned.  stats (host, may be NULL) is filled on return.  The call
 * enqueues on the plan's stream and returns after it has synchronised with it, so U_dev
 * is complete on return.  By default the whole solve is one CUDA-graph launch whose
 * loops are decided on the device (the graph is built on the first solve for a given
 * (G_dev, U_dev) pair and reused while both pointers stay the same).
 * PD_ERR_NOT_CONVERGED: limits reached; U_dev holds the last iterate. */
pd_status paradiag_solve(pd_plan *plan, const double *G_dev, double *U_dev, pd_stats *stats);

/* Batched plans: advance the solve of every problem by up to `steps` refinement sweeps
 * (solves of eq. 2's FP64 residual by Algorithm 1, as paradiag_solve's sweeps), so that
 * problems can join a batch while the others are being solved: the continuous batching
 * of a solve service.  Not part of the paper.
 * G_dev: device, (nt, n_bar), each problem's right-hand side in its slot (zero slots are
 * unused).  U_dev: device, (nt, n_bar), the current iterates, updated in place.
 * join (host, length batch): nonzero for a problem that starts with this call; its U slot
 * is set to zero and its refinement state reset, so its first sweep is its first solve
 * (with the refinement sweeps' Algorithm-2 tolerance).  The other problems continue from
 * U_dev and their own count of solves.
 * state (host, length batch, out): 1 = the problem met refine_tol (its slot of U_dev is
 * its solution; later calls keep refining it while it stays), 2 = it took max_refine + 1
 * solves without meeting it, 0 = still running (or an unused slot).
 * Each problem decides convergence by the same rules as in paradiag_solve, counted from
 * its own first solve.  The sweeps run as host-driven loops on the plan's stream; the call
 * returns after synchronising with it.  stats: this call's sweeps.
 * Errors: PD_ERR_INVALID_ARG (not a batched plan, steps outside [1, 64], NULL or aliasing
 * arguments), PD_ERR_UNSUPPORTED (fixed-loop variants, mass matrices), PD_ERR_NONFINITE. */
pd_status paradiag_batch_advance(pd_plan *plan, const double *G_dev, double *U_dev, const int32_t *join,
                                 int32_t steps, int32_t *state, pd_stats *stats);

/* Same as paradiag_solve with G and U in host memory (pinned memory gives the best
 * copy rate).  The host-to-device copy of G and the device-to-host copy of U are
 * part of the call.  Requires desc->host_io != 0 at plan time. */
pd_status paradiag_solve_host(pd_plan *plan, const double *G_host, double *U_host,
                              pd_stats *stats);

/* Replace the operator of an existing plan: desc must describe the plan's shape (dim,
 * nx, ny, nt, batch, precision); its K arrays, tau, batch_nx and batch_tau are
 * uploaded in place (host-synchronous; it first waits for the plan's stream), so the
 * plan's workspace and, unless a single problem's tau changes, its captured CUDA
 * graph are reused.  Errors: PD_ERR_INVALID_ARG for a different shape, and the
 * validation errors of paradiag_plan.  Not part of the paper: it lets a solver
 * service reuse plans across requests of one shape. */
pd_status paradiag_set_operator(pd_plan *plan, const pd_desc *desc);

/* Release the plan and, if the plan allocated it, its workspace.  NULL is a no-op. */
pd_status paradiag_destroy(pd_plan *plan);

/* Thread-local description of the last error on this thread ("" if none). */
const char *paradiag_last_error(void);

/* Library version string. */
const char *paradiag_version(void);

/* ---- Stage entry points (single steps of the path, for verification) ----------
 * They run the same kernels paradiag_solve runs, on caller-provided device arrays.
 * Spectra are (nt/2 + 1, n_bar) row-major complex arrays, interleaved (re, im), of
 * the plan's compute type: complex128 for PD_FP64 plans, complex64 for PD_MIXED.
 * In 2D they act in the basis where T_y is diagonal (after paradiag_dst_y). */

/* Forward DFT along time, X (nt, n_bar) float64 -> Xhat (nt/2+1, n_bar):
 * Xhat[k] = sum_j omega^{jk} X[j], omega = exp(-2 pi i / l); the rows of X F^T (eq. 5). */
pd_status paradiag_time_dft(pd_plan *plan, const double *X_dev, void *Xhat_dev);

/* Inverse DFT along time, Y (nt/2+1, n_bar) -> X (nt, n_bar) float64,
 * X[j] = Re((1/l) sum_k omega^{-jk} Y[k]) with Y[l-k] = conj(Y[k]): the rows of Y F^{-T}. */
pd_status paradiag_time_idft(pd_plan *plan, const void *Y_dev, double *X_dev);

/* The first parallel-in-time loop of Algorithm 1: Y[k] = ((1 - pi_k) I + tau K)^{-1} R[k]
 * for k = 0..nt/2 (Y_dev may be NULL to skip the store), and, if b_dev != NULL, the SMW
 * right-hand side b = sum_{i=0}^{l-1} gamma_i Y_i (eq. 7) over the full spectrum,
 * using Y_{l-k} = conj(Y_k); b is float64 of length n_bar. */
pd_status paradiag_shifted_solve(pd_plan *plan, const void *R_dev, void *Y_dev, double *b_dev);

/* 2D only: the orthonormal DST-I along y of a (nt, ny, nx) float64 array (its own
 * inverse).  This is the transform that diagonalises T_y (Sec. 6.1 operator). */
pd_status paradiag_dst_y(pd_plan *plan, const double *X_dev, double *Y_dev);

/* After a solve: the SMW right-hand side b (eq. 7) for G and the Algorithm-2 solution
 * x_m of eq. (8) from the first solve (before any refinement sweep), float64 length
 * n_bar, device.  Either may be NULL. */
pd_status paradiag_last_vectors(pd_plan *plan, double *b_dev, double *x_dev);

/* The binary32 reciprocal 1/v that the PD_MIXED shifted solves use inside the complex
 * division 1/a = conj(a) / |a|^2 (Smith-free: the operands are bounded away from zero and
 * overflow): the hardware approximation refined by one Newton-Raphson step.  It is within
 * 1 ulp of 1/v for normal-range v, not always correctly rounded, and flushes subnormals to
 * zero.  x, r: device, n float32 each (r[i] = that reciprocal of x[i]); stream: cudaStream_t.
 * Returns after the stream has synchronised.  A verification entry point: the paper's
 * arithmetic is not specified to this level. */
pd_status paradiag_recip_f32(const float *x, float *r, int64_t n, void *stream);

/* ---- Allocation-free variant ---------------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * call cudaMalloc when they need this step (an arena or pool that owns all device
 * memory, a real-time loop where an allocation would stall, a host application that
 * forbids allocation after start-up).  It computes what paradiag_shifted_solve computes
 * with b requested (the first parallel-in-time loop of Algorithm 1 and b of eq. 7), in
 * FP64, without a plan and without allocating anything: its scratch is a file-scope
 * __device__ array of PD_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds
 * until the process exits.
 *   nt      time steps l (power of two, 1 <= nt <= 8192), n rows of K (1 <= n <= 4096);
 *           larger sizes return PD_ERR_UNSUPPORTED with a message in paradiag_last_error().
 *   tau     time step; k_lo, k_diag, k_up: device, length n, the tridiagonal K
 *           (k_lo[0], k_up[n-1] ignored); K must be weakly diagonally dominant by rows or
 *           symmetric positive definite, as for paradiag_plan (not checked here: the
 *           arrays are on the device).
 *   R       device, (nt/2+1, n) complex128 right-hand sides (half spectrum of real data).
 *   Y       device, (nt/2+1, n) complex128 solutions, or NULL to skip the store.
 *   b       device, length n float64: b = sum_{i=0}^{l-1} gamma_i Y_i.
 *   stream  cudaStream_t the work is enqueued on; the call returns without waiting.
 * The first call on each device looks up the device address of the scratch array
 * (cudaGetSymbolAddress, with that device current); make that first call before any
 * stream capture.  All calls share the one array and each rewrites every word it reads,
 * so calls that overlap on the GPU race: serialise them. */
#define PD_NOALLOC_SCRATCH_BYTES (4u * 1024u * 1024u)
pd_status paradiag_smw_rhs_noalloc(int64_t nt, int64_t n, double tau, const double *k_lo,
                                   const double *k_diag, const double *k_up, const void *R, void *Y,
                                   double *b, void *stream);

/* ---- Kernel timing (tracing) ------------------------------------------------------ */

typedef struct pd_kernel_time {
  char name[32];       /* kernel family */
  int64_t launches;    /* launches recorded since timing was enabled */
  double total_ms;     /* summed CUDA-event durations on the plan's stream */
  double bytes;        /* summed algorithmic bytes of those launches */
} pd_kernel_time;

/* Enable (1) or disable (0) per-launch CUDA-event timing on the plan's stream;
 * enabling resets the counters. */
pd_status paradiag_set_timing(pd_plan *plan, int enable);

/* Copy up to max_entries kernel-family records into out; *n_out = families present. */
pd_status paradiag_kernel_times(pd_plan *plan, pd_kernel_time *out, int max_entries, int *n_out);

#ifdef __cplusplus
}
#endif

#endif /* PARADIAG_H */
