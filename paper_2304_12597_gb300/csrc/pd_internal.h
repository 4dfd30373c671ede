// Internal host-side interfaces shared by the .cu files of the library:
// launch context with per-kernel CUDA-event tracing, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <utility>
#include <string>
#include <vector>

#include "pd_common.cuh"

namespace pd {

// Device control block layout (the plan's `flags` int array and `scal` double array).
enum FlagIndex {
  F_BREAK = 0,    // Algorithm 2 met an invariant Krylov space
  F_BZERO = 1,    // ||b|| == 0
  F_NONFIN = 2,   // a non-finite value was met
  F_CAPCNT = 3,   // completion counter of the capacitance kernel
  F_KSTOP = 4,    // Algorithm 2 loop finished
  F_M = 5,        // completed Algorithm-2 iterations m of the current solve
  F_SWEEP = 6,    // completed solves (first solve + refinement sweeps)
  F_RCONV = 7,    // refinement reached its tolerance
  F_KCONV = 8,    // Algorithm 2 reached eps (or b == 0, or breakdown)
  F_RSTOP = 9,    // refinement loop finished
  F_MTOT = 10,    // sum of m over the solves
  F_C2RCNT = 11,  // completion counter of the inverse DFT's finishing epilogue
  F_ACCCNT = 12,  // completion counter of the b reduction (runs the start of Algorithm 2)
  F_ZCNT = 13,    // completion counter of the z reduction (runs eq. 13 and the decision)
  F_MEMCNT = 14,  // batched plans: members done in a per-member Algorithm-2 step
  F_RNCNT = 15,   // completion counter of the forward DFT's right-hand-side norm
  F_SWM = 16,     // [16, 32): m of each solve
  F_FROZEN = 32,  // this Algorithm-2 step skips the residual check (q > 1, Sec. 3)
  F_NOH = 33,     // this step forms no h_k: breakdown or a frozen step
  F_TIMEOUT = 34, // a bounded device-side wait ran out (persistent Algorithm-2 step)
  F_BARCNT = 35,  // grid barrier of the persistent step: arrivals
  F_BARGEN = 36,  // grid barrier of the persistent step: generation
  F_EARLY = 37,   // Algorithm 3's residual test on U_1 passed: U = U_1
  F_EARLYCNT = 38,  // completion counter of that test
  F_COMB = 39,    // this solve forms its final loop by linearity (1; 2 with the h_k term), 0 = solves
  F_COMBCNT = 40, // solves whose final loop was formed by linearity
  kFlagWords = 64
};
// CTA size of the cooperative Krylov vector kernels (pd_krylov.cuh, kCoop mode).
constexpr int kBlas = 512;

enum ScalIndex {
  S_BETA = 0,     // ||b|| of the current solve
  S_T = 1,        // t_{m+1,m}
  S_RES = 2,      // ||r_m|| of eq. (13)
  S_KNORM = 3,    // ||K v_m|| (breakdown reference)
  S_D2 = 4,       // ||delta||_F^2 of the last solve's output
  S_REF2 = 5,     // ||delta_0||_F^2
  S_PREV = 6,     // previous relative update
  S_UPD = 7,      // last relative update
  S_RNORM = 8,    // ||R||_F of the current solve's right-hand side (G, or the residual)
  S_U1RES = 9,    // ||(I + tau K) U_1 - U_1 Sigma_1^T - G||_F (Algorithm 3's test on U_1)
  S_U1NORM = 10,  // ||U_1||_F
  S_HIST = 16,    // [16, 49): ||r_m|| history of the current solve
  S_SWRES = 64,   // [64, 80): eq. (13) residual / ||b|| at exit of each solve
  S_SWUPD = 80,   // [80, 96): ||delta_s|| / ||delta_0|| of each solve
  S_SWBETA = 96,  // [96, 112): ||b|| of each solve
  kScalWords = 128
};

// Launch context: the stream every kernel is ordered on, a launch counter, and
// optional per-launch timing with CUDA events recorded on that same stream.
// Launch `kern` on stream s, with programmatic stream serialization when pdl is set:
// the kernel may then be scheduled while its predecessor drains; it waits for it in
// grid_dep_wait() before reading anything.
template <typename... KArgs, typename... Args>
cudaError_t pdl_launch(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

struct Ctx {
  cudaStream_t stream = nullptr;
  bool pdl = true;   // programmatic dependent launch between consecutive kernels
  int fft_cols = 0;  // columns per CTA of the time FFTs (0 = choose per launch)
  int fft_radix = 0;  // first stage of the FFTs: 16, 4, or 0 = built-in (fft.cu: use_r16)
  bool timing = false;
  int64_t launches = 0;
  cudaError_t err = cudaSuccess;
  const char *err_where = "";

  struct Family {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
  };
  struct Pending {
    int fam;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Family> fams;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;

  int family(const char *name);
  cudaEvent_t event();
  // Launch through f(); records events around it when timing is on.
  void launch(const char *fam, double bytes, const std::function<void()> &f);
  // Resolve recorded events (call after the stream has been synchronised).
  void collect();
  void release();
};

int sm_count();
size_t smem_optin();
// Lets kernel fn take as much dynamic shared memory per CTA as its static arrays leave of
// smem_optin(); returns that limit (0 if it could not be set).  The value is the same for
// every call (set once per kernel): host threads that launch one kernel with different
// shared-memory sizes (plans solved concurrently with host-driven loops) cannot lower the
// limit another thread needs between its setting and its launch.
int allow_dyn_smem(const void *fn);
// Sets the thread-local message returned by paradiag_last_error().
void set_last_error(const char *msg);

// Device-side control of Algorithm 2 and of the refinement loop (control.cu).
struct KrylovCtl {
  double eps;          // stop when ||r_m|| <= eps * ref, ref = beta (or ||R||_F with rrel)
  double stall_floor;  // stall exit only once ||r_m|| <= stall_floor * ref
  int rrel;            // 1: ref = ||R||_F of the solve's right-hand side (refining plans;
                       // see krylov_decide)
  int win;             // stall: no halving over `win` checks
  int maxit;
  int q;               // residual check every q steps (and at maxit or a breakdown)
};
struct RefineCtl {
  int fp64;
  double eps_first, eps_refine;  // Algorithm-2 tolerances of the first solve / sweeps
  double refine_tol;
  int max_refine;
  // batched plans: each problem's own count of solves (msw[b]; its refinement rules count
  // from there, so a problem can join a running batch with msw[b] = 0), and its state after
  // this decision (mconv[b]: 1 converged, 2 gave up after member_solves solves, 0 running)
  int *msw;
  int *mconv;
  int member_solves;  // 0 = no per-problem limit (the plan's max_refine bounds the batch)
};
// ---- time FFT / DST (fft.cu) ----------------------------------------------------
// Forward DFT along time of real (n, ncols) rows -> half spectrum (n/2+1, ncols).
// rs (may be null): row j of X is multiplied by rs[j] on load (the D_alpha of
// Algorithm 3); rsi in the inverse: output row j multiplied by rsi[j].
// rn (optional): ||X||_F (or ||R||_F) of the transformed data, reduced over the CTAs by
// the last one to finish into *rn.dst (before the D_alpha scaling).
struct RhsNorm {
  double *part;  // one partial sum of squares per CTA
  int *counter;  // zero on entry; reset by the last CTA
  double *dst;
};
template <typename T, typename Tin>
void launch_fft_r2c(Ctx &c, const Tin *X, int64_t ldx, int64_t ncols, int n, const cpx<T> *tw,
                    cpx<T> *S, int64_t lds, const T *rs = nullptr, const RhsNorm *rn = nullptr);
// Forward DFT along time of the FP64 all-at-once residual
// R = G - [(I + tau K) U - U Sigma_1^T] (1D), computed on load: R is never stored.
// mex/mnx (batched plans): column c is scaled by 2^mex[c / mnx], undone by the inverse.
template <typename T>
void launch_fft_r2c_residual(Ctx &c, const double *G, const double *U, int64_t ncols, int n,
                             const double *rxl, const double *rxd, const double *rxu, const cpx<T> *tw,
                             cpx<T> *S, int64_t lds, const T *rs = nullptr, const int *mex = nullptr,
                             int mnx = 1, const RhsNorm *rn = nullptr);
// Optional epilogue of the inverse DFT: the last CTA to finish sums the per-CTA
// squares into scal[S_D2] and runs the refinement decision.
struct StepFinish {
  int enabled;
  int *counter;  // zero on entry; reset by the last CTA
  double *scal;
  int *flags;
  RefineCtl rc;
  int use_handle;
  cudaGraphConditionalHandle h;
};
// Inverse DFT along time of a half spectrum; mode 0: store double, 1: add into
// double, 2: store float.  norm_part (may be null) receives per-CTA sums of the
// squared output values; *nparts = number of CTAs.  colsum (may be null) receives
// per-column sums of the squared output values (ncols doubles).
template <typename T>
void launch_fft_c2r(Ctx &c, const cpx<T> *S, int64_t lds, int64_t ncols, int n, const cpx<T> *tw,
                    void *out, int64_t ldo, int mode, double *norm_part, int *nparts,
                    const StepFinish *fin = nullptr, const T *rsi = nullptr, double *colsum = nullptr,
                    const int *mex = nullptr, int mnx = 1, const int *skip = nullptr);
// Orthonormal DST-I along the middle axis of (nt, ny, nx); ny + 1 a power of two.
// mode 0: store, 1: add into (double output only).
template <typename Tin, typename Tout, typename T>
void launch_dst_y(Ctx &c, const Tin *X, Tout *Y, int64_t nt, int64_t ny, int64_t nx,
                  const cpx<T> *tw, int mode, const int *skip = nullptr);
// The same transform of the FP64 all-at-once residual of the 2D path, formed while each tile
// loads (nt time rows of batch problems, nym rows of T_y each, stacked along y; rx
// per problem, ry over the stacked rows; mex: the batches' residual scaling, or null):
// the residual and the DST in one pass.  rx = (tau lo_x, 1 + tau diag_x, tau up_x),
// ry = (tau lo_y, tau diag_y, tau up_y).
template <typename T>
void launch_dst_y_residual(Ctx &c, const double *G, const double *U, T *Y, int64_t nt, int batch, int64_t nym,
                           int64_t nx, const double *rxl, const double *rdd, const double *rxu, const double *ryl,
                           const double *ryu, const int *mex, const cpx<T> *tw);

// ---- shifted tridiagonal solves (pint.cu) ------------------------------------------
struct PintGeom {
  int nf;        // frequencies k = 0..nf-1 (half spectrum)
  int nblk;      // independent tridiagonal blocks per frequency
  int blen;      // rows per block
  int P;         // threads per team (power of two, >= 32)
  int R;         // k-range splits: teams = nblk * R
  int teams_per_cta;
  int M;         // rows per thread (template value)
  int cta_sum;   // 1: the teams of a CTA add their partial rows (nblk == 1)
  int acc_rows;  // partial rows per block in acc_part (R, or CTAs when cta_sum)
  int stage;     // 1: tau K staged in shared memory once per launch
};
// m_req / teams_req: rows per thread and teams per CTA requested by the caller (0 = choose);
// fact: the loops will use stored factors (a smaller shared-memory footprint)
PintGeom pint_geometry(int nf, int nblk, int blen, int target_teams, int elem_bytes, int m_req = 0,
                       int teams_req = 0, bool fact = false);
void set_acc_rows(PintGeom &g);  // recompute cta_sum / acc_rows after changing R

template <typename T>
struct PintArgs {
  const int *mcount;       // device m (completed Algorithm-2 steps), or null: when set the
                           // right-hand side is V[m+1] and the dots use V[0..m]
  int want_dots;           // with mcount: compute g_k = V^T y_k
  int mdots_max;           // with mcount: largest possible number of dots (smem sizing)
  const int *xm_count;     // if set: subtract x_m = sum_{q < m} y_q V[q] (m = *xm_count), formed
  const double *xm_y;      // per team from y (xm_y) and V (a.V, ldv) instead of rvec; the teams
  const double *xm_Vd;     // starting at k = 0 also store x_m in FP64 (from xm_Vd) into xm_out
  double *xm_out;
  const double2 *shift;    // s_k = 1 - pi_k, length nf
  const cpx<T> *shift_t;   // the same in the compute type (binary32 plans; null = convert)
  const cpx<T> *omega_t;   // omega in the compute type (null = convert)
  const T *tlo, *tdiag, *tup;  // tau * K (block-decoupled), length nblk*blen
  const cpx<T> *R;         // spectrum right-hand sides (nf, ldr) or null
  int64_t ldr;
  const T *rvec;           // real vector: the right-hand side when R is null,
                           // subtracted from every R[k] otherwise (may be null)
  cpx<T> *Y;               // solution store (nf, ldy) or null
  int64_t ldy;
  const double2 *omega;    // accumulation weights: acc += Re(omega_k y_k) (summed in T per
                           // team, over that team's few frequencies), or null
  double *acc_part;        // (teams, blen) partial sums when omega != null
  const T *V;              // Krylov basis rows in the compute type (ldv stride) for dots, or null
  int64_t ldv;
  int mdots;               // number of basis vectors dotted with y_k
  double2 *gpart;          // (nf, nblk, mdots) dot products y_k . V[q]
  const int *skip_flag;    // if non-null and *skip_flag != 0 the kernel does nothing
  const int *skip_flag2;   // a second such flag (the final loop formed by linearity)
  double xm_scale;         // with xm_count: subtract xm_scale * x_m (alpha^{1/l} in Algorithm 3)
  int64_t xm_ldy;          // block blk takes y_m from xm_y + blk * xm_ldy (0: one y_m)
  int xm_bpm;              // blocks per batch member (2D batches: the modes of its T_y; 0 = 1)
  const cpx<T> *fac_in;    // precomputed factors of every (k, block) system (pint.cu), or null
  cpx<T> *fac_out;         // factor pass: store those factors (R, rvec, Y, omega, V unused)
  // Zero-frequency lane of the binary32 path.  A_0 = (1 - pi_0) I + tau K has the real
  // shift 1 - alpha^{1/l} (0 for Algorithm 1) and is the only ill-conditioned shifted
  // system (|1 - pi_k| >= 2 sin(pi / l) for k >= 1); its inverse (norm up to
  // 1 / (tau lambda_min(K))) dominates b (eq. 7) and J_l (eq. 8).  With k0_fp64 the team
  // owning k = 0 solves it in FP64 from FP64 coefficients (tlo_d, ...), takes v_{m+1} and
  // x_m from the FP64 basis Vd, and writes its FP64 share of b into acc0 (added by the
  // reduction), h_0 into h0 (added by the z sum) and its dots g_0 in FP64.
  int k0_fp64;
  const double *tlo_d, *tdiag_d, *tup_d;
  const double *Vd;
  double *acc0;            // (nblk * blen) omega_0 y_0 of the acc pass, or null
  double *h0;              // (nblk * blen) h_0 of the dots pass, or null
  const double *fac0_in;   // the lane's stored FP64 factors (pint_k0_factor_elems), or null
  double *fac0_out;        // factor pass of the lane: store them (frequency 0 only)
};
// Doubles of the zero-frequency lane's factors (one real system per block).
size_t pint_k0_factor_elems(const PintGeom &g);
// Complex elements of the factor array of one plan geometry (pint.cu: fac_slots).
size_t pint_factor_elems(const PintGeom &g);
template <typename T>
void launch_pint(Ctx &c, const PintGeom &g, const PintArgs<T> &a);
void launch_recip_f32(cudaStream_t s, const float *x, float *r, int64_t n);
struct InitTail;  // pd_krylov.cuh: the start of Algorithm 2 run by a reduction's last CTA
struct ProjTail;  // pd_krylov.cuh: eq. 13 and the step decision run by the z reduction's last CTA
// z[j] = sum_k Re(omega_k H[k][j]) over stored h_k (nf rows, leading dimension ldh);
// with tail, the last CTA then projects z and decides the Algorithm-2 step.
// h0 (or null): the FP64 h_0 of the zero-frequency lane, which replaces row 0 of H.
template <typename T>
void launch_zsum(Ctx &c, int nf, int64_t n, const cpx<T> *H, int64_t ldh, const double2 *omega, double *z,
                 const int *skip_flag, const ProjTail *tail = nullptr, int mlen = 0, const double *h0 = nullptr);
// Batched plans (batch.cu): Gs = G with slot b scaled by 2^ex[b] ~ 1/||slot b||_F
// (part: batch * nc doubles of scratch; zero[b] = 1 marks an all-zero slot), and the
// inverse scaling of U in place with the columns past problem b's nxb[b] rows, and every
// column of an all-zero problem, set to zero.
void launch_batch_normalize(Ctx &c, const double *G, double *Gs, int64_t nt, int batch, int nxm, int nc,
                            double *part, int *ex, int *zero);
// Problems joining a running batched solve (paradiag_batch_advance): for join[b] != 0 the
// slot's U is zeroed and its refinement state reset (msw, mprev, mref2, mex, mconv); unused
// slots (zero[b]) start from U = 0 as well; the other slots' U is scaled by 2^ex[b] into
// the solve's units (exact).
void launch_member_join(Ctx &c, double *U, int64_t nt, int batch, int nxm, const int *ex, const int *join,
                        const int *zero, int *msw, double *prev, double *ref2, int *mex, int *mconv);
void launch_batch_unscale(Ctx &c, double *U, int64_t nt, int batch, int nxm, const int *ex, const int *nxb,
                          const int *zero);
// out[t][j] = in[t][j] * s[j] over nt rows of nb columns (in place allowed; batch.cu)
void launch_col_scale(Ctx &c, const double *in, double *out, int64_t nt, int64_t nb, const double *s);
// Batched plans: per-problem ||delta||^2 from the inverse DFT's per-column sums, then the
// refinement decision over all problems but the all-zero ones (zero[b]; control.cu).
void launch_member_decide(Ctx &c, const double *colsum, int nxm, const int *nxb, int nmem, double *d2, double *ref2,
                          double *prev, int *mex, const int *zero, double *scal, int *flags, const RefineCtl &r,
                          int use_handle, cudaGraphConditionalHandle h);

// out[j] = sum_r acc_part[(blk*R + r)*blen + e] (+ extra[j]), j = blk*blen + e; with tail,
// the last CTA then computes beta = ||out|| and v_1 (the start of Algorithm 2).
void launch_acc_reduce(Ctx &c, const PintGeom &g, const double *acc_part, double *out, const int *skip_flag,
                       const InitTail *tail = nullptr, const double *extra = nullptr);

// ---- Krylov / small systems / residual (krylov.cu) -----------------------------------
struct KrylovBufs {
  int n;              // vector length n_bar
  int maxit;
  const double *klo, *kdiag, *kup;  // K (block-decoupled tridiagonal), unscaled
  double *V;          // (maxit+1, n)
  float *Vf;          // binary32 copy of V for the mixed-precision shifted solves, or null
  double *T;          // (maxit+1, maxit) upper Hessenberg, row-major T[q*maxit + c]
  double *w;          // work vector (n)
  double *part;       // per-CTA partials (grid, maxit+2)
  int grid;           // CTAs of the BLAS-1 kernels
  double *scal;       // scalar block (see krylov.cu)
  int *flags;         // flag block (see krylov.cu)
  int cluster;        // grid == 1 only: > 0 runs the vector kernels on a cluster of this many CTAs
  // Batched plans: `members` problems of `mlen` rows each run their own Algorithm 2
  // (0 = one Algorithm 2 over the whole vector).  Member b's control blocks are
  // mscal + b kScalWords and mflags + b kFlagWords, its T_m is T + b (maxit+1) maxit, its
  // y_m is y + b (maxit+1); scal/flags above then hold the batch totals and the loop
  // control, and `counter` counts the members done in a step.
  int members, mlen;
  double *mscal;
  int *mflags;
  double *y;
  int *counter;
  int q;             // residual check period of Algorithm 2 (single problems; batches use 1)
};
// All Algorithm-2 kernels read m from flags[F_M] (completed steps), so one captured
// iteration serves every m.  `use_handle` / `h`: set a CUDA-graph conditional.
void launch_vec_norm_init(Ctx &c, KrylovBufs &k, const double *b, int use_handle,
                          cudaGraphConditionalHandle h);  // also zeroes T
void launch_arnoldi(Ctx &c, KrylovBufs &k);
// Largest cluster size <= want (halving, >= 4) the device can co-schedule for the
// cluster variant of the vector kernels (one CTA per SM); 0 if none.
int krylov_cluster_size(int want);
void launch_capacitance(Ctx &c, KrylovBufs &k, int nf, double tau, const double2 *shift,
                        const double2 *wg, const double2 *gpart, int nblk, double *msys_part,
                        int k5_grid, double2 *srow, double2 *omega, double *y, int members = 0, int bpm = 1,
                        double2 *sinv = nullptr);
// Batched plans, one Algorithm 2 per member (one CTA each; krylov_members.cu): the
// start (beta_b, v_1), an Arnoldi step, and eq. (13) with the per-member decision; the
// last member of the start and of eq. (13) sets the batch's control block and the
// WHILE conditional (run while any member runs).
void launch_member_init(Ctx &c, KrylovBufs &k, const double *b, int use_handle, cudaGraphConditionalHandle h);
void launch_member_arnoldi(Ctx &c, KrylovBufs &k);
void launch_member_project(Ctx &c, KrylovBufs &k, const double *z, double tau, const KrylovCtl &kc,
                           int use_handle, cudaGraphConditionalHandle h);
// Persistent form of one Algorithm-2 step (single problems): one cooperative launch runs
// the eq. (12) terms and system, z = sum_k gamma_k h_k c_k, eq. (13) with the stopping
// decision and, unless Algorithm 2 stops there, the next Arnoldi step (eq. 10), with
// grid barriers between the phases instead of kernel boundaries.  The shifted solves of
// the step (h_k and their dots) stay a launch of their own, with their own CTA shape.
// Every barrier waits at most bar_polls polls; one that runs out sets flags[F_TIMEOUT],
// sets the WHILE conditional to 0 and the kernel returns (the solve then reports
// PD_ERR_TIMEOUT).  bar_extra > 0 makes every barrier wait for that many CTAs that do
// not exist (a wait that cannot complete: the bounded wait's own test).
template <typename TC>
struct StepArgs {
  // Algorithm 2 state (as KrylovBufs)
  int n, maxit, q, ld;
  const double *klo, *kdiag, *kup;
  double *V, *w, *T, *part, *scal, *z;
  float *Vf;
  int *flags;
  double tau;
  KrylovCtl kc;
  // eq. (12)
  int nf, nblk;
  const double2 *shift, *wg, *gpart;
  double *msys_part, *y;
  double2 *srow, *omega;
  double2 *sinv;  // (nf, m, m) S_k of the step, or null (the final loop by linearity)
  // z from the stored h_k (the zero frequency from the FP64 lane h0 when it is on)
  const cpx<TC> *H;
  int64_t ldh;
  const double *h0;
  int zrg;  // row groups of the z sum (power of two <= 64)
  int nv;   // CTAs of the vector phases (eq. 13, Arnoldi): the first nv of the grid
  // launch
  size_t smem;  // dynamic shared memory of the launch
  long long bar_polls;
  int bar_extra;
  int use_handle;
  cudaGraphConditionalHandle h;
};
// grid = co-resident CTAs of 512 threads; the vector phases hold E entries per thread over
// a.nv of them.
template <typename T>
void launch_step_tail(Ctx &c, const StepArgs<T> &a, int grid, int E);
// Dynamic shared memory and the largest co-resident grid of the persistent step (0 if it
// cannot run: its shared memory does not fit).
size_t step_tail_smem(int maxit, int nf, int elem_bytes);
int step_tail_max_grid(int nv, int E, int elem_bytes, size_t smem);

// Algorithm 3's optional test on U_1: r = ||(I + tau K) U_1 - U_1 Sigma_1^T - G||_F against
// eps ||U_1||_F (the residual of the original system, as in the refinement).  If it passes,
// flags[F_EARLY] is set, Algorithm 2 does not run (flags[F_KSTOP], F_M = 0, the WHILE
// conditional set to 0) and the final loop and inverse transforms are skipped: U = U_1.
// part: 2 * (4 * SMs) doubles of scratch.  Coefficients: (tau lo_x, 1 + tau d_x, tau up_x)
// and (tau lo_y, tau d_y, tau up_y) (1D: ryl == null, ny = 1).
void launch_early_check(Ctx &c, const double *G, const double *U, int64_t nt, int64_t ny, int64_t nx,
                        const double *rxl, const double *rxd, const double *rxu, const double *ryl,
                        const double *ryd, const double *ryu, int64_t nym, double eps, double *part, double *scal,
                        int *flags, int use_handle, cudaGraphConditionalHandle h);
// After the (skipped) final loop: with flags[F_EARLY], record the solve and stop the
// refinement loop.
void launch_early_finish(Ctx &c, double *scal, int *flags, int use_handle, cudaGraphConditionalHandle h);

// eq. (13) and the Algorithm-2 stopping decision (krylov_decide) in one kernel
void launch_project_resnorm(Ctx &c, KrylovBufs &k, const double *z, double tau, const KrylovCtl &kc,
                            int use_handle, cudaGraphConditionalHandle h);
void launch_xm(Ctx &c, KrylovBufs &k, const double *y, double *x, float *xf);
// Algorithm 1's final loop by linearity (k_final_comb): when Algorithm 2 stopped at
// 1 <= m <= maxm and U_1 was not taken, flags[F_COMB] != 0 and the spectrum S becomes
// Y_k = L_k - V_m s_k + c_k h_k, s_k = a S_k y_m, c_k = tau t_{m+1,m} (e_m^T s_k) (L from the
// first loop, h_k in H, both (nf, lds); S_k in sinv, (nf, m, m), for m > 1), so the final
// loop's solves are skipped (PintArgs.skip_flag2); else flags[F_COMB] = 0 and S is left for
// them.  Vb: the basis in the compute type (rows of n).  Also x = x_m = sum_{q<m} y_q V[q] in
// FP64 (length n) for any m.
constexpr int kCombMaxM = 16;  // largest m whose final loop is formed by linearity
template <typename T>
void launch_final_comb(Ctx &c, int nf, int64_t n, int64_t lds, double tau, double aroot, const double2 *shift,
                       const double *Tm, const double *y, const double *V, const T *Vb, const double *scal,
                       int *flags, const double2 *sinv, int maxm, const cpx<T> *L, const cpx<T> *H, cpx<T> *S,
                       double *x);


void launch_solve_reset(Ctx &c, double *scal, int *flags);
void launch_krylov_decide(Ctx &c, double *scal, int *flags, const KrylovCtl &k, int use_handle,
                          cudaGraphConditionalHandle h);
void launch_inner_fixed(Ctx &c, double *scal, int *flags, double *y, int loops, int use_handle,
                        cudaGraphConditionalHandle h);  // Table 3 variants: no Algorithm 2
void launch_refine_decide(Ctx &c, double *scal, int *flags, const RefineCtl &r, int use_handle,
                          cudaGraphConditionalHandle h);
void launch_sumsq(Ctx &c, const double *part, int nparts, double *dst);


}  // namespace pd
