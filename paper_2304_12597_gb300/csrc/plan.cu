// Host orchestration of Algorithm 1 (with Algorithm 2 inside) and of the mixed-
// precision refinement around it, plus the C ABI declared in include/paradiag.h.
//
// Solve basis: in 1D the spatial operator is K itself.  In 2D,
// K = I (x) T_x + T_y (x) I with T_y symmetric Toeplitz; the orthonormal DST-I
// along y (S, S = S^T = S^{-1}) turns it into the block-diagonal
// K~ = I (x) T_x + diag(mu_l) (x) I, mu_l = d + 2 c cos(pi l / (ny + 1)).  S acts
// on space only, so it commutes with the time DFT, and since it is orthogonal
// the Arnoldi process of Algorithm 2 run on (K~, S b) produces S V_m and the same
// T_m: Algorithm 1 is carried out unchanged in that basis, between one DST of
// the input and one DST of the output.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <string>
#include <vector>

#include "../../include/paradiag.h"
#include "pd_internal.h"
#include "pd_krylov.cuh"

using pd::cpx;

namespace {

thread_local std::string g_err;

pd_status fail(pd_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

// Serialises the heavy host-side paths of different plans (plan building, graph
// capture and instantiation, operator upload, destruction) so that callers may drive
// plans from several threads; solves themselves run concurrently.
std::recursive_mutex &host_mutex() {  // recursive: a failing paradiag_plan destroys its plan
  static std::recursive_mutex m;
  return m;
}

// Bump allocator over the workspace; the same sequence of take() calls is run
// once for sizing (base == nullptr) and once for assignment.
struct Arena {
  unsigned char *base = nullptr;
  size_t off = 0;
  template <typename X>
  X *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    X *p = base ? reinterpret_cast<X *>(base + off) : nullptr;
    off += count * sizeof(X);
    return p;
  }
};

}  // namespace

namespace pd {

void set_last_error(const char *msg) { g_err = msg ? msg : ""; }

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  }
  return n;
}

size_t smem_optin() {
  static int v = 0;
  if (v == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
      v = 227 * 1024;
  }
  return (size_t)v;
}

int allow_dyn_smem(const void *fn) {
  // the opt-in limit covers static and dynamic shared memory together: a kernel's limit is
  // what its static arrays leave (one value per kernel, set once)
  static std::mutex mu;
  static std::unordered_map<const void *, int> done;
  std::lock_guard<std::mutex> lk(mu);
  auto it = done.find(fn);
  if (it != done.end()) return it->second;
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
    cudaGetLastError();  // leave no error for the next launch to pick up
    return 0;
  }
  const int lim = (int)smem_optin() - (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  done[fn] = lim;
  return lim;
}

int Ctx::family(const char *name) {
  for (size_t i = 0; i < fams.size(); ++i)
    if (fams[i].name == name) return (int)i;
  fams.push_back(Family{name, 0, 0.0, 0.0});
  return (int)fams.size() - 1;
}

cudaEvent_t Ctx::event() {
  if (!free_events.empty()) {
    cudaEvent_t e = free_events.back();
    free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void Ctx::launch(const char *fam, double bytes, const std::function<void()> &f) {
  if (err != cudaSuccess) return;
  cudaEvent_t a = nullptr, b = nullptr;
  int fi = -1;
  if (timing) {
    fi = family(fam);
    a = event();
    b = event();
    cudaEventRecord(a, stream);
  }
  f();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess && err == cudaSuccess) {
    err = e;
    err_where = fam;
  }
  ++launches;
  if (timing) {
    cudaEventRecord(b, stream);
    pending.push_back(Pending{fi, a, b, bytes});
  }
}

void Ctx::collect() {
  for (auto &p : pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      fams[p.fam].ms += ms;
      fams[p.fam].launches += 1;
      fams[p.fam].bytes += p.bytes;
    }
    free_events.push_back(p.a);
    free_events.push_back(p.b);
  }
  pending.clear();
}

void Ctx::release() {
  collect();
  for (auto e : free_events) cudaEventDestroy(e);
  free_events.clear();
}

}  // namespace pd

struct pd_plan {
  pd::Ctx ctx;
  int dim = 1;
  int64_t nx = 0, ny = 1, nbar = 0, nt = 0;
  int nf = 0;
  double tau = 0.0;
  double alpha = 1.0;  // Algorithm 3: C_alpha instead of C_1 (1 = Algorithm 1)
  bool refined64 = false;  // FP64 plan that always refines (alpha < 1, or a batch)
  double aroot = 1.0;  // alpha^{1/l}
  int precision = PD_FP64;
  int maxit = 32;
  int q = 1;  // Algorithm 2 checks its residual every q steps (Sec. 3)
  int loops = 0;  // fixed-cost variant (Table 3): 2 = x_m = b, 1 = U_1; 0 = the full method
  double eps = 1e-13;
  double eps_refine = 3e-3;  // PD_MIXED: Algorithm 2 tolerance of the refinement sweeps
  double early_eps = 0.0;    // Algorithm 3's residual test on U_1 (0 = off)
  // the final loop by linearity when Algorithm 2 stops at m = 1 (k_final_comb): the first
  // loop stores L_k in lbuf
  bool comb = false;
  void *lbuf = nullptr;
  double2 *sinv = nullptr;  // S_k of the last eq. (12) system (nf, m, m), m <= maxit
  int max_refine = 6;
  double refine_tol = 1e-13;
  int host_io = 0;
  bool own_ws = false;
  void *ws = nullptr;
  size_t ws_bytes = 0;

  int nblk = 1, blen = 0;
  // batched plans: `batch` problems of up to nxm unknowns (slot b = columns [b nxm, (b+1) nxm));
  // in 2D every problem is nx x nym and the stacked grid is nx x (batch nym), ny = batch nym
  int batch = 1;
  int64_t nym = 1;   // rows of T_y per problem (the DST length); 1 in 1D
  int64_t nrx = 0;   // length of the x-coefficient arrays: T_x of every problem
  int64_t nxd = 0;   // the descriptor's nx
  int64_t nxm = 0;
  int bnc = 0;                  // time-row groups of the per-problem norm pass
  double *Gs = nullptr;         // G with every problem scaled to unit norm
  double *bpart = nullptr;      // norm partials (batch * bnc)
  int *bex = nullptr;           // per-problem power-of-two scale exponents
  int *bzero = nullptr;         // per-problem flag: all-zero right-hand side (unused slot)
  int *bnx = nullptr;           // rows of each problem
  double *colsum = nullptr;     // per-column ||delta||^2 of the last solve
  double *md2 = nullptr, *mref2 = nullptr, *mprev = nullptr;  // per-problem refinement state
  int *mex = nullptr;  // per-problem residual scaling 2^mex of the next refinement sweep
  int *msw = nullptr, *mconv = nullptr, *mjoin = nullptr;  // per-problem solves, state, join flags
  int member_solves = 0;  // paradiag_batch_advance: solves a problem may take (0 = no limit)
  int members = 0;     // batched plans: one Algorithm 2 per problem (0 = one for the plan)
  bool mass = false;   // diagonal mass matrix: solve for w = M^{1/2} u with K' = M^{-1/2} K M^{-1/2}
  double *msc = nullptr;  // M^{-1/2} (n_bar)
  double *Gm = nullptr;   // M^{-1/2} G (nt, n_bar)
  bool factored = false;  // the shifted systems are factored once per operator (fac)
  void *fac = nullptr;
  double *mscal = nullptr;  // per-problem Algorithm-2 scalar and flag blocks
  int *mflags = nullptr;
  pd::PintGeom geom{};
  int blas_grid = 1, k5_grid = 1;
  int k5_grid_members = 1;  // capacitance CTAs per problem of a batched plan
  int blas_cluster = 0;  // CTAs of the cluster variant of the one-CTA Krylov kernels (0 = off)
  bool krylov_tails = false;  // beta / v_1 and eq. (13) in the last CTA of the b and z reductions
  // persistent Algorithm-2 step (single problems): one cooperative launch after each
  // step's shifted solves (see pd::StepArgs)
  bool persist = false;
  int persist_grid = 0;     // CTAs (co-resident)
  int persist_nv = 1;       // CTAs of the vector phases (the first of the grid)
  int persist_E = 1;        // vector entries per thread
  int persist_zrg = 1;      // row groups of the z sum
  size_t persist_smem = 0;  // dynamic shared memory
  long long bar_polls = 0;  // bounded wait of its grid barriers
  int bar_extra = 0;        // test only: arrivals that never come
  int64_t lds = 0;

  // device buffers
  double2 *shift = nullptr, *wg = nullptr;
  cpx<float> *shift_f = nullptr, *wg_f = nullptr;  // binary32 copies for the shifted solves
  double2 *wga = nullptr;  // alpha^{1/l} w_k gamma_k: weights of the inner system (eq. 17)
  double *ts_d = nullptr, *tsi_d = nullptr;  // D_alpha and D_alpha^{-1} (time rows)
  float *ts_f = nullptr, *tsi_f = nullptr;
  double *klo = nullptr, *kdiag = nullptr, *kup = nullptr;
  double *tlo_d = nullptr, *tdiag_d = nullptr, *tup_d = nullptr;
  float *tlo_f = nullptr, *tdiag_f = nullptr, *tup_f = nullptr;
  double *xlo = nullptr, *xdiag = nullptr, *xup = nullptr, *ylo = nullptr, *ydiag = nullptr, *yup = nullptr;
  // residual coefficients: (tau lo_x, 1 + tau diag_x, tau up_x) and (tau lo_y, tau diag_y, tau up_y)
  double *rxl = nullptr, *rxd = nullptr, *rxu = nullptr, *ryl = nullptr, *ryd = nullptr, *ryu = nullptr;
  double *rdd = nullptr;  // 2D: rxd + ryd at every point of the grid (n_bar), one FP64 add less per point
  cpx<double> *tw_d = nullptr, *twy_d = nullptr;
  cpx<float> *tw_f = nullptr, *twy_f = nullptr;
  void *spec = nullptr;
  void *hbuf = nullptr;  // h_k of the current Algorithm-2 step (same shape as the spectrum)
  double *V = nullptr, *T = nullptr, *w = nullptr, *part = nullptr, *scal = nullptr;
  float *Vf = nullptr, *xf = nullptr;  // binary32 copies of V and x_m (mixed precision)
  int *flags = nullptr;
  double *b = nullptr, *z = nullptr, *x = nullptr, *y = nullptr;
  double *b0 = nullptr, *x0 = nullptr;  // b and x_m of the first solve (for paradiag_last_vectors)
  double *acc_part = nullptr;
  double *acc0 = nullptr, *h0 = nullptr;  // PD_MIXED: FP64 zero-frequency lane outputs (b share, h_0)
  double *fac0 = nullptr;                 // PD_MIXED: the lane's FP64 factors (per operator)
  bool lane = false;                      // PD_MIXED: the zero frequency runs in the FP64 lane
  double nu0 = 0.0;                       // ||(l A_0)^{-1}||_inf estimate (lane criterion)
  double2 *gpart = nullptr, *srow = nullptr, *omega = nullptr;
  double *msys_part = nullptr;
  double *norm_part = nullptr;
  float *tmp_f = nullptr;
  double *tmp_d = nullptr;
  double *G_stage = nullptr, *U_stage = nullptr;
  // paradiag_solve_host: the device-to-host copy of U, queued behind a graph solve's
  // control-block read so that one host synchronisation covers both
  void *tail_dst = nullptr;
  const void *tail_src = nullptr;
  size_t tail_bytes = 0;
  bool tail_done = false;
  // pinned host mirrors of the scalar and flag blocks
  double *h_scal = nullptr;
  int *h_flags = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  pd_stats last{};
  // CUDA graph of the whole solve, built for one (G, U) pair
  int use_graphs = 1;
  bool graph_failed = false;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};  // capture streams (top level, bodies)
  cudaGraphExec_t gexec = nullptr;
  const double *g_G = nullptr;
  double *g_U = nullptr;
  struct {
    int64_t pre0 = 0, iter0 = 0, post0 = 0, pre1 = 0, iter1 = 0, post1 = 0;
  } seg;  // kernel launches per segment (for the launch count of graph solves)
};

namespace {

// Host copies of the operator in the solve basis.
struct HostOp {
  std::vector<double> lo, diag, up;  // K~ (length nbar), block-decoupled
  std::vector<double> xlo, xdiag, xup, ylo, ydiag, yup;
};

// The shifted solves eliminate without pivoting (partitioned Thomas + PCR).  Every
// shift of Algorithms 1 and 3 has Re(1 - pi_k) >= 0 (|pi_k| = alpha^{1/l} <= 1).  Either
// of two conditions on each block of K then makes elimination in any order safe for
// every shifted matrix (1 - pi_k) I + tau K (in 2D, after the DST along y, the blocks
// T_x + mu_j I with mu_j = d_y + 2 c_y cos(j pi / (ny + 1)); the smallest mu_j is added
// to the diagonal of T_x):
//  (a) weak row diagonal dominance, k_ii >= |lo_i| + |up_i|: the shifted matrix is
//      dominant as well, |(1 - pi_k) + tau k_ii| >= tau k_ii;
//  (b) K symmetric positive definite: the Hermitian part Re(1 - pi_k) I + tau K is
//      positive definite, a property every Schur complement keeps, so every pivot has a
//      real part at least the corresponding pivot of the real LDL^T of tau K.
// A diagonal mass matrix changes neither: (1 - pi_k) M + tau K is dominant when K is
// (and has a positive definite Hermitian part when K is SPD), and the plan's symmetric
// scaling M^{-1/2} (.) M^{-1/2} only rescales the rows and columns of its LU factors.
// A centred advection term at cell Peclet number above 2 satisfies neither condition;
// such operators are rejected rather than solved without pivoting.  The relative slack
// 1e-12 absorbs the rounding of operators that are dominant with equality (upwind).
pd_status check_dominance(const pd_desc *d) {
  const int nb = d->batch > 1 ? d->batch : 1;
  for (int b = 0; b < nb; ++b) {
    double mu = 0.0;  // smallest eigenvalue of the problem's T_y (2D)
    if (d->dim == 2) {
      const double dy = d->k_diag_y[(int64_t)b * d->ny], cy = d->ny > 1 ? d->k_up_y[(int64_t)b * d->ny] : 0.0;
      mu = dy - 2.0 * std::fabs(cy) * std::cos(M_PI / (double)(d->ny + 1));
    }
    const int64_t n = (nb > 1 && d->batch_nx) ? d->batch_nx[b] : d->nx;
    const double *lo = d->k_lo + (int64_t)b * d->nx, *di = d->k_diag + (int64_t)b * d->nx,
                 *up = d->k_up + (int64_t)b * d->nx;
    bool dominant = true, symmetric = true;
    int64_t bad = -1;
    double bad_off = 0.0, bad_di = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      const double l = i > 0 ? lo[i] : 0.0, u = i + 1 < n ? up[i] : 0.0, dd = di[i] + mu;
      if (!std::isfinite(dd) || !std::isfinite(l) || !std::isfinite(u))
        return fail(PD_ERR_INVALID_ARG, "K has a non-finite coefficient in row %lld", (long long)(b * d->nx + i));
      const double off = std::fabs(l) + std::fabs(u);
      if (dominant && dd < off - 1e-12 * (std::fabs(dd) + off)) {
        dominant = false;
        bad = (int64_t)b * d->nx + i;
        bad_off = off;
        bad_di = dd;
      }
      if (i + 1 < n && std::fabs(lo[i + 1] - u) > 1e-12 * (std::fabs(lo[i + 1]) + std::fabs(u))) symmetric = false;
    }
    if (dominant) continue;
    bool spd = symmetric;
    double h = 0.0;  // LDL^T pivots of the symmetric block
    for (int64_t i = 0; spd && i < n; ++i) {
      const double dd = di[i] + mu;
      h = i == 0 ? dd : dd - lo[i] * lo[i] / h;
      if (!(h > 1e-13 * std::fabs(dd))) spd = false;
    }
    if (!spd)
      return fail(PD_ERR_UNSUPPORTED,
                  "K is neither diagonally dominant (row %lld: |lo| + |up| = %.17g > diag = %.17g%s) nor symmetric "
                  "positive definite: the shifted systems are eliminated without pivoting, which needs one of the two",
                  (long long)bad, bad_off, bad_di, d->dim == 2 ? " incl. the smallest eigenvalue of T_y" : "");
  }
  return PD_OK;
}

pd_status validate(const pd_desc *d) {
  if (!d) return fail(PD_ERR_INVALID_ARG, "desc is NULL");
  if (d->abi_version != PD_ABI_VERSION)
    return fail(PD_ERR_INVALID_ARG, "abi_version %d, library expects %d", d->abi_version, PD_ABI_VERSION);
  if (d->dim != 1 && d->dim != 2) return fail(PD_ERR_INVALID_ARG, "dim must be 1 or 2 (got %d)", d->dim);
  if (d->nx < 1) return fail(PD_ERR_INVALID_ARG, "nx must be >= 1");
  if (d->dim == 1 && d->ny != 1 && d->ny != 0) return fail(PD_ERR_INVALID_ARG, "1D problems need ny == 1");
  if (d->dim == 2 && d->ny < 1) return fail(PD_ERR_INVALID_ARG, "ny must be >= 1");
  if (!is_pow2(d->nt) || d->nt > 8192)
    return fail(PD_ERR_UNSUPPORTED, "nt must be a power of two in [1, 8192] (got %lld)", (long long)d->nt);
  if (!(d->tau > 0.0) || !std::isfinite(d->tau)) return fail(PD_ERR_INVALID_ARG, "tau must be finite and > 0");
  if (!d->k_lo || !d->k_diag || !d->k_up) return fail(PD_ERR_INVALID_ARG, "K coefficient arrays are NULL");
  if (d->precision != PD_FP64 && d->precision != PD_MIXED) return fail(PD_ERR_INVALID_ARG, "bad precision");
  if (d->maxit < 0 || d->maxit > 32) return fail(PD_ERR_UNSUPPORTED, "maxit must be in [1, 32]");
  if (d->q < 0 || d->q > 32) return fail(PD_ERR_INVALID_ARG, "q must be in [0, 32] (0 = 1)");
  if (d->loops < 0 || d->loops > 2) return fail(PD_ERR_INVALID_ARG, "loops must be 0, 1 or 2");
  if (d->loops > 0 && d->batch > 1)
    return fail(PD_ERR_UNSUPPORTED, "the fixed-loop variants (loops > 0) are built for single problems");
  if (d->q > 1 && d->batch > 1)
    return fail(PD_ERR_UNSUPPORTED, "a frozen residual (q > 1) is built for single problems, not batches");
  if (!(d->alpha >= 0.0 && d->alpha <= 1.0)) return fail(PD_ERR_INVALID_ARG, "alpha must be in (0, 1] (0 = 1)");
  if (d->eps_krylov < 0.0 || d->refine_tol < 0.0 || d->max_refine < 0 || !(d->eps_krylov_refine >= 0.0))
    return fail(PD_ERR_INVALID_ARG, "negative tolerance or sweep count");
  const int64_t blen = d->nx;
  if (blen > 4096) return fail(PD_ERR_UNSUPPORTED, "tridiagonal blocks longer than 4096 rows are not built");
  if (d->m_diag) {  // diagonal mass matrix: symmetric scaling keeps K tridiagonal (1D only)
    if (d->dim != 1)
      return fail(PD_ERR_UNSUPPORTED, "a mass matrix is built for 1D problems (2D needs M (x) structure for the DST)");
    const int64_t nm = d->nx * (d->batch > 1 ? d->batch : 1);
    for (int64_t i = 0; i < nm; ++i)
      if (!(d->m_diag[i] > 0.0) || !std::isfinite(d->m_diag[i]))
        return fail(PD_ERR_INVALID_ARG, "m_diag[%lld] = %g must be finite and > 0", (long long)i, d->m_diag[i]);
  }
  if (d->dim == 2) {
    if (!d->k_lo_y || !d->k_diag_y || !d->k_up_y) return fail(PD_ERR_INVALID_ARG, "T_y arrays are NULL");
    if (!is_pow2(d->ny + 1) || d->ny + 1 > 4096)
      return fail(PD_ERR_UNSUPPORTED, "2D needs ny + 1 to be a power of two <= 4096 (DST-I by FFT)");
    for (int b = 0; b < (d->batch > 1 ? d->batch : 1); ++b) {  // T_y of every problem
      const double *ylo = d->k_lo_y + (int64_t)b * d->ny, *ydi = d->k_diag_y + (int64_t)b * d->ny,
                   *yup = d->k_up_y + (int64_t)b * d->ny;
      const double dd = ydi[0];
      const double c = d->ny > 1 ? yup[0] : 0.0;
      const double tol = 1e-12 * (std::fabs(dd) + std::fabs(c));
      for (int64_t i = 0; i < d->ny; ++i) {
        if (!std::isfinite(ydi[i]) || std::fabs(ydi[i] - dd) > tol)
          return fail(PD_ERR_UNSUPPORTED, "T_y must be Toeplitz");
        if (i + 1 < d->ny && (std::fabs(yup[i] - c) > tol || std::fabs(ylo[i + 1] - c) > tol))
          return fail(PD_ERR_UNSUPPORTED, "T_y must be symmetric Toeplitz");
      }
    }
  }
  if (d->tune_pint_rows != 0 && d->tune_pint_rows != 4 && d->tune_pint_rows != 8 && d->tune_pint_rows != 16)
    return fail(PD_ERR_INVALID_ARG, "tune_pint_rows must be 0, 4, 8 or 16");
  if (d->tune_pint_rows == 16 && d->precision != PD_MIXED)
    return fail(PD_ERR_UNSUPPORTED, "16 rows per thread are built for PD_MIXED only");
  if (d->tune_pint_rows) {  // one team of P threads must fit one CTA
    int64_t P = 32;
    while (P * d->tune_pint_rows < d->nx) P <<= 1;
    if (P > (d->tune_pint_rows == 16 ? 256 : 512))
      return fail(PD_ERR_UNSUPPORTED, "tune_pint_rows %d is too few rows per thread for blocks of %lld rows",
                  d->tune_pint_rows, (long long)d->nx);
  }
  if (d->tune_pint_teams < 0 || (d->tune_pint_teams && !is_pow2(d->tune_pint_teams)) || d->tune_pint_teams > 16)
    return fail(PD_ERR_INVALID_ARG, "tune_pint_teams must be 0 or a power of two <= 16");
  if (d->tune_krylov_ctas < 0 || d->tune_krylov_ctas > 1024 || d->tune_cap_ctas < 0 || d->tune_cap_ctas > 1024)
    return fail(PD_ERR_INVALID_ARG, "tune_krylov_ctas and tune_cap_ctas must be in [0, 1024]");
  if (d->tune_pint_factor < -1 || d->tune_pint_factor > 1)
    return fail(PD_ERR_INVALID_ARG, "tune_pint_factor must be -1, 0 or 1");
  if (d->tune_krylov_tails < -1 || d->tune_krylov_tails > 1)
    return fail(PD_ERR_INVALID_ARG, "tune_krylov_tails must be -1, 0 or 1");
  if (d->tune_krylov_cluster != 0 && d->tune_krylov_cluster != -1 &&
      (d->tune_krylov_cluster < 4 || d->tune_krylov_cluster > 16))
    return fail(PD_ERR_INVALID_ARG, "tune_krylov_cluster must be 0, -1 or in [4, 16]");
  {  // one CTA (or one cluster) holds at most 16 vector entries per thread
    const int64_t nbar = d->nx * (d->dim == 2 ? d->ny : 1) * (d->batch > 1 ? d->batch : 1);
    if (d->tune_krylov_ctas == 1 && nbar > 8192)
      return fail(PD_ERR_UNSUPPORTED, "tune_krylov_ctas = 1 (one CTA) needs n_bar <= 8192, got %lld",
                  (long long)nbar);
  }
  if (d->tune_fft_cols != 0 && d->tune_fft_cols != 2 && d->tune_fft_cols != 4 && d->tune_fft_cols != 8 &&
      d->tune_fft_cols != 16)
    return fail(PD_ERR_INVALID_ARG, "tune_fft_cols must be 0, 2, 4, 8 or 16");
  if (d->tune_fft_radix != 0 && d->tune_fft_radix != 4 && d->tune_fft_radix != 16)
    return fail(PD_ERR_INVALID_ARG, "tune_fft_radix must be 0, 4 or 16");
  if (!(d->early_exit_eps >= 0.0) || !std::isfinite(d->early_exit_eps))
    return fail(PD_ERR_INVALID_ARG, "early_exit_eps must be finite and >= 0");
  if (d->early_exit_eps > 0.0 && (d->batch > 1 || d->loops > 0))
    return fail(PD_ERR_UNSUPPORTED, "the residual test on U_1 (early_exit_eps) is built for single problems that "
                                    "run Algorithm 2 (no batch, loops = 0)");
  if (d->tune_zero_lane < -1 || d->tune_zero_lane > 1)
    return fail(PD_ERR_INVALID_ARG, "tune_zero_lane must be -1, 0 or 1");
  if (d->tune_persistent < -1 || d->tune_persistent > 1)
    return fail(PD_ERR_INVALID_ARG, "tune_persistent must be -1, 0 or 1");
  if (d->barrier_polls < 0 || d->tune_persist_ctas < 0 || d->barrier_extra < 0 || d->barrier_extra > 1024)
    return fail(PD_ERR_INVALID_ARG, "barrier_polls, tune_persist_ctas must be >= 0; barrier_extra in 0..1024");
  if (d->batch < 0) return fail(PD_ERR_INVALID_ARG, "batch must be >= 0");
  if (d->batch > 1) {
    if (d->dim == 2) {  // every problem nx x ny; its Algorithm 2 runs in one CTA
      if (d->batch_nx) return fail(PD_ERR_UNSUPPORTED, "2D batches share nx and ny (batch_nx must be NULL)");
      if (d->nx * d->ny > 8192)
        return fail(PD_ERR_UNSUPPORTED, "2D batches need nx * ny <= 8192 per problem (got %lld)",
                    (long long)(d->nx * d->ny));
    }
    if (d->batch > 65535) return fail(PD_ERR_UNSUPPORTED, "at most 65535 problems per batch");
    for (int b = 0; b < d->batch; ++b) {
      if (d->batch_nx && (d->batch_nx[b] < 1 || d->batch_nx[b] > d->nx))
        return fail(PD_ERR_INVALID_ARG, "batch_nx[%d] = %lld is outside [1, nx]", b, (long long)d->batch_nx[b]);
      if (d->batch_tau && !(d->batch_tau[b] > 0.0 && std::isfinite(d->batch_tau[b])))
        return fail(PD_ERR_INVALID_ARG, "batch_tau[%d] must be finite and > 0", b);
    }
  }
  const int64_t nbar = d->nx * (d->dim == 2 ? d->ny : 1) * (d->batch > 1 ? d->batch : 1);
  if (nbar > (int64_t)1 << 28 || d->nt * nbar > (int64_t)1 << 34)
    return fail(PD_ERR_UNSUPPORTED, "problem too large for this build");
  return check_dominance(d);
}

void fill_geometry(pd_plan *p, const pd_desc *d) {
  p->dim = d->dim;
  p->batch = d->batch > 1 ? d->batch : 1;
  p->nxd = d->nx;
  p->nrx = d->nx * p->batch;
  if (d->dim == 2) {  // problems stacked along y: nx x (batch ny)
    p->nym = d->ny;
    p->nxm = d->nx * d->ny;
    p->nx = d->nx;
  } else {
    p->nym = 1;
    p->nxm = d->nx;
    p->nx = d->nx * p->batch;  // 1D: the stacked spatial length
  }
  p->ny = d->dim == 2 ? d->ny * p->batch : 1;
  p->nbar = p->nx * p->ny;
  p->nt = d->nt;
  p->nf = (int)(d->nt / 2 + 1);
  if (d->nt == 1) p->nf = 1;
  // a batch folds each problem's time step into its block of K (tau = 1 below)
  p->tau = p->batch > 1 ? 1.0 : d->tau;
  p->alpha = d->alpha > 0.0 ? d->alpha : 1.0;
  p->aroot = std::pow(p->alpha, 1.0 / (double)d->nt);
  p->refined64 = d->precision == PD_FP64 && (p->alpha < 1.0 || d->batch > 1);
  p->precision = d->precision;
  p->maxit = d->maxit ? d->maxit : 32;
  p->q = d->q > 1 ? d->q : 1;
  // PD_MIXED: a binary32 solve is accurate to ~1e-4 whatever Algorithm 2 does past that
  // (measured: tighter tolerances add Krylov steps, not accuracy), so the first solve's
  // Algorithm 2 stops at 1e-4; refinement does the rest
  p->eps = d->eps_krylov > 0 ? d->eps_krylov : (d->precision == PD_FP64 ? 1e-13 : 1e-4);
  // FP64 plans that refine anyway use a loose tolerance per solve: Algorithm 3 loses
  // up to kappa(F D_alpha) per solve, and a batch runs until its slowest problem's
  // Algorithm 2 has converged (one problem that needs 30 steps at 1e-13 holds all of
  // them), so FP64 refinement sweeps with a few Krylov steps each beat one tight solve
  if (p->refined64 && !(d->eps_krylov > 0)) p->eps = 1e-5;
  // batches stop only when their slowest problem has converged: allow more sweeps
  p->max_refine = d->max_refine ? d->max_refine : (d->batch > 1 ? 16 : 8);
  p->loops = d->loops;
  if (p->loops) p->max_refine = 0;  // one solve: the variant's approximation
  p->refine_tol = d->refine_tol > 0 ? d->refine_tol : (d->precision == PD_FP64 ? 1e-14 : 1e-11);
  p->eps_refine = d->eps_krylov_refine > 0 ? d->eps_krylov_refine : 3e-3;
  p->early_eps = d->early_exit_eps;
  p->comb = d->tune_final_loop >= 0 && p->batch == 1 && d->loops == 0;
  p->host_io = d->host_io;
  // tridiagonal blocks of nx rows: one per problem (1D) or per mode of T_y (2D)
  p->nblk = p->dim == 2 ? (int)p->ny : p->batch;
  p->blen = (int)d->nx;
  p->bnc = (int)std::min<int64_t>(p->nt, 64);
  p->lds = (p->nbar + 31) / 32 * 32;
  const int sms = pd::sm_count();
  const int esz = d->precision == PD_FP64 ? 16 : 8;
  // factored loops (FP64 by default) need one PCR exchange buffer, eliminating loops two
  const bool want_fac = d->tune_pint_factor == 1 || (d->tune_pint_factor == 0 && d->precision == PD_FP64);
  pd::PintGeom g0 =
      pd::pint_geometry(p->nf, p->nblk, p->blen, 1, esz, d->tune_pint_rows, d->tune_pint_teams, want_fac);
  // one wave of resident teams: occupancy estimated from shared memory and threads
  const size_t team_bytes = (size_t)g0.P * (g0.M + 1) * esz + (size_t)2 * g0.P * ((want_fac || g0.P < 64) ? 5 : 8) * esz +
                            (size_t)g0.P * g0.M * 8 +
                            (size_t)(g0.P / 32) * 33 * 16;
  const size_t cta_bytes = team_bytes * g0.teams_per_cta;
  int by_smem = (int)std::max<size_t>(1, (228 * 1024) / (cta_bytes + 1024));
  int by_threads = std::max(1, 2048 / (g0.P * g0.teams_per_cta));
  const int ctas_per_sm = std::max(1, std::min(by_smem, by_threads));
  const int target = sms * ctas_per_sm * g0.teams_per_cta;
  p->geom =
      pd::pint_geometry(p->nf, p->nblk, p->blen, target, esz, d->tune_pint_rows, d->tune_pint_teams, want_fac);
  // Krylov vector kernels: vectors up to 8192 entries run in one 512-thread CTA or (see
  // below) a cluster; beyond, cooperative 64-thread CTAs, at most one per SM (co-resident)
  p->blas_grid =
      p->nbar <= 8192 ? 1 : (int)std::max<int64_t>(1, std::min<int64_t>((p->nbar + pd::kBlas - 1) / pd::kBlas, (int64_t)sms));
  // capacitance terms: one frequency per warp (four warps per CTA; a thread per
  // frequency when m = 1)
  p->k5_grid = std::max(1, std::min((p->nf + 3) / 4, 1024));
  if (d->tune_krylov_ctas) p->blas_grid = std::min(d->tune_krylov_ctas, sms);
  // Vectors one CTA would hold: a cluster of 8 (n_bar <= 2048) or 16 CTAs, one per SM,
  // spreads their FP64 work (GB300 runs FP64 at ~1/64 of the FP32 rate) over as many
  // SMs, with reductions through distributed shared memory
  p->blas_cluster = 0;
  // batched plans: one Algorithm 2 per problem, one CTA each (see krylov_members.cu)
  p->members = p->batch > 1 ? p->batch : 0;
  if (!p->members && p->blas_grid == 1 && d->tune_krylov_cluster >= 0 && p->nbar >= 256) {
    const int want = d->tune_krylov_cluster > 0 ? d->tune_krylov_cluster : (p->nbar <= 2048 ? 8 : 16);
    p->blas_cluster = pd::krylov_cluster_size(want);
    if (p->blas_cluster < 4) p->blas_cluster = 0;
  }
  // the start of Algorithm 2 and its eq. (13) decision are single-CTA work: with one CTA
  // they run in the last CTA of the reduction before them; with a cluster, on request
  p->krylov_tails = !p->members && p->blas_grid == 1 && d->tune_krylov_tails >= 0 &&
                    (p->blas_cluster == 0 || d->tune_krylov_tails == 1);
  if (d->tune_cap_ctas) p->k5_grid = d->tune_cap_ctas;
  // batched plans run one capacitance system per problem: about two waves of CTAs over
  // all problems (each CTA sized for maxit-step Gauss-Jordan holds one SM), so a warp
  // takes several frequencies instead of the grid taking many waves
  p->k5_grid_members = p->k5_grid;
  if (p->batch > 1 && !d->tune_cap_ctas)
    p->k5_grid_members = std::max(1, std::min(p->k5_grid, (2 * sms + p->batch - 1) / p->batch));
  p->ctx.fft_cols = d->tune_fft_cols;
  p->ctx.fft_radix = d->tune_fft_radix;
  p->mass = d->m_diag != nullptr;
  {  // factors of the shifted systems: computed once per operator, read by every loop
    const size_t esz = p->precision == PD_MIXED ? sizeof(cpx<float>) : sizeof(cpx<double>);
    const size_t fbytes = pd::pint_factor_elems(p->geom) * esz;
    p->factored = want_fac && fbytes <= ((size_t)4 << 30);
  }
  p->ctx.pdl = d->tune_no_pdl == 0;
  // persistent Algorithm-2 step: single problems that run Algorithm 2.  The vector phases
  // take one entry per thread on as few CTAs as that needs (up to four entries once the
  // grid is full): few CTAs keep their barriers short, one entry per thread spreads the
  // FP64 work over as many SMs as there are 512-entry slices.
  p->persist = false;
  p->persist_grid = std::max(1, std::min(d->tune_persist_ctas > 0 ? d->tune_persist_ctas : sms, sms));
  p->bar_polls = d->barrier_polls > 0 ? (long long)d->barrier_polls : (1LL << 22);
  p->bar_extra = d->barrier_extra;
  if (!p->members && !p->loops && d->tune_persistent > 0) {
    const int elem = p->precision == PD_MIXED ? 4 : 8;
    const int G = p->persist_grid;
    const int64_t slices = (p->nbar + 511) / 512;
    p->persist_nv = (int)std::min<int64_t>(slices, G);
    p->persist_E = pd::reg_elems((int)p->nbar, p->persist_nv * 512);
    const bool fits = p->nbar <= (int64_t)p->persist_nv * 512 * 4;
    p->persist_smem = pd::step_tail_smem(p->maxit, p->nf, elem);
    if (fits && p->persist_smem <= 180 * 1024 &&
        pd::step_tail_max_grid(p->persist_nv, p->persist_E, elem, p->persist_smem) >= G)
      p->persist = true;
    // z sum: the row-group count that needs the fewest dependent memory round trips per
    // CTA (tiles per CTA x batches of 16 loads per tile)
    int64_t best = -1;
    for (int rg = 1; rg <= 64; rg <<= 1) {
      const int64_t cw = 512 / rg, tiles = (p->nbar + cw - 1) / cw;
      const int64_t rows = (p->nf + rg - 1) / rg;
      const int64_t cost = ((tiles + G - 1) / G) * ((rows + 15) / 16);
      if (best < 0 || cost < best) {
        best = cost;
        p->persist_zrg = rg;
      }
    }
  }
}

// Assign (or size) every device buffer.
size_t layout(pd_plan *p, unsigned char *base) {
  Arena A;
  A.base = base;
  const int64_t nbar = p->nbar, nt = p->nt;
  const int nf = p->nf, mx = p->maxit;
  const bool mixed = p->precision == PD_MIXED;
  p->shift = A.take<double2>(nf);
  p->wg = A.take<double2>(nf);
  if (mixed) {
    p->shift_f = A.take<cpx<float>>(nf);
    p->wg_f = A.take<cpx<float>>(nf);
  }
  p->wga = A.take<double2>(nf);
  p->ts_d = A.take<double>(nt);
  p->tsi_d = A.take<double>(nt);
  if (mixed) {
    p->ts_f = A.take<float>(nt);
    p->tsi_f = A.take<float>(nt);
  }
  p->klo = A.take<double>(nbar);
  p->kdiag = A.take<double>(nbar);
  p->kup = A.take<double>(nbar);
  p->tlo_d = A.take<double>(nbar);
  p->tdiag_d = A.take<double>(nbar);
  p->tup_d = A.take<double>(nbar);
  if (mixed) {
    p->tlo_f = A.take<float>(nbar);
    p->tdiag_f = A.take<float>(nbar);
    p->tup_f = A.take<float>(nbar);
  }
  p->xlo = A.take<double>(p->nrx);
  p->xdiag = A.take<double>(p->nrx);
  p->xup = A.take<double>(p->nrx);
  p->rxl = A.take<double>(p->nrx);
  p->rxd = A.take<double>(p->nrx);
  p->rxu = A.take<double>(p->nrx);
  if (p->dim == 2) {
    p->ylo = A.take<double>(p->ny);
    p->ydiag = A.take<double>(p->ny);
    p->yup = A.take<double>(p->ny);
    p->ryl = A.take<double>(p->ny);
    p->ryd = A.take<double>(p->ny);
    p->rdd = A.take<double>(p->nbar);
    p->ryu = A.take<double>(p->ny);
  }
  const int ntw = std::max<int>(1, (int)(nt / 2));
  p->tw_d = A.take<cpx<double>>(ntw);
  if (mixed) p->tw_f = A.take<cpx<float>>(ntw);
  if (p->dim == 2) {
    p->twy_d = A.take<cpx<double>>(p->nym + 1);
    if (mixed) p->twy_f = A.take<cpx<float>>(p->nym + 1);
  }
  p->spec = mixed ? (void *)A.take<cpx<float>>((size_t)nf * p->lds) : (void *)A.take<cpx<double>>((size_t)nf * p->lds);
  p->hbuf = mixed ? (void *)A.take<cpx<float>>((size_t)nf * p->lds) : (void *)A.take<cpx<double>>((size_t)nf * p->lds);
  if (p->comb) {
    p->lbuf = mixed ? (void *)A.take<cpx<float>>((size_t)nf * p->lds) : (void *)A.take<cpx<double>>((size_t)nf * p->lds);
    const int mc = std::min(mx, pd::kCombMaxM);
    p->sinv = A.take<double2>((size_t)nf * mc * mc);
  }
  if (p->factored)
    p->fac = mixed ? (void *)A.take<cpx<float>>(pd::pint_factor_elems(p->geom))
                   : (void *)A.take<cpx<double>>(pd::pint_factor_elems(p->geom));
  p->V = A.take<double>((size_t)(mx + 1) * nbar);
  if (mixed) {
    p->Vf = A.take<float>((size_t)(mx + 1) * nbar);
    p->xf = A.take<float>(nbar);
  }
  const int nmem = std::max(1, p->members);  // Algorithm-2 states (one per batch member)
  p->T = A.take<double>((size_t)(mx + 1) * mx * nmem);
  p->w = A.take<double>(nbar);
  p->part = A.take<double>((size_t)3 * std::max(p->blas_grid, p->persist_grid) * (mx + 2));
  p->scal = A.take<double>(pd::kScalWords);
  p->flags = A.take<int>(pd::kFlagWords);
  p->b = A.take<double>(nbar);
  p->z = A.take<double>(nbar);
  p->x = A.take<double>(nbar);
  p->b0 = A.take<double>(nbar);
  p->x0 = A.take<double>(nbar);
  p->y = A.take<double>((size_t)(mx + 1) * nmem);
  p->acc_part = A.take<double>((size_t)p->geom.nblk * p->geom.R * p->geom.blen);
  if (mixed) {
    p->acc0 = A.take<double>(nbar);
    p->h0 = A.take<double>(nbar);
    p->fac0 = A.take<double>(pd::pint_k0_factor_elems(p->geom));
  }
  p->gpart = A.take<double2>((size_t)nf * p->nblk * mx);
  p->srow = A.take<double2>((size_t)nf * mx * nmem);
  p->omega = A.take<double2>((size_t)nf * nmem);
  p->msys_part = A.take<double>((size_t)std::max(p->k5_grid, p->persist_grid) * mx * mx * nmem);
  if (p->members) {
    p->mscal = A.take<double>((size_t)pd::kScalWords * nmem);
    p->mflags = A.take<int>((size_t)pd::kFlagWords * nmem);
  }
  p->norm_part = A.take<double>((size_t)std::max<int64_t>(nbar / 2 + 2, 8 * (int64_t)pd::sm_count()));
  if (mixed && p->dim == 2) p->tmp_f = A.take<float>((size_t)nt * nbar);
  if (!mixed && p->dim == 2) p->tmp_d = A.take<double>((size_t)nt * nbar);
  if (p->mass) {
    p->msc = A.take<double>(nbar);
    p->Gm = A.take<double>((size_t)nt * nbar);
  }
  if (p->batch > 1) {
    p->Gs = A.take<double>((size_t)nt * nbar);
    p->bpart = A.take<double>((size_t)p->batch * p->bnc);
    p->bex = A.take<int>(p->batch);
    p->bzero = A.take<int>(p->batch);
    p->bnx = A.take<int>(p->batch);
    p->colsum = A.take<double>(nbar);
    p->md2 = A.take<double>(p->batch);
    p->mref2 = A.take<double>(p->batch);
    p->mprev = A.take<double>(p->batch);
    p->mex = A.take<int>(p->batch);
    p->msw = A.take<int>(p->batch);
    p->mconv = A.take<int>(p->batch);
    p->mjoin = A.take<int>(p->batch);
  }
  if (p->host_io) {
    p->G_stage = A.take<double>((size_t)nt * nbar);
    p->U_stage = A.take<double>((size_t)nt * nbar);
  }
  return (A.off + 255) & ~(size_t)255;
}

// 2D batch: problem b is nx x ny with its own T_x, T_y and tau_b, stacked along y (rows
// [b ny, (b+1) ny) of the nx x (batch ny) grid).  Its blocks (one per mode l of its T_y)
// carry tau_b (T_x + mu_{b,l} I); the stacked T_y has no coupling across problems.
HostOp build_batched_operator_2d(const pd_desc *d) {
  HostOp h;
  const int64_t nx = d->nx, ny = d->ny, B = d->batch;
  h.xlo.assign(nx * B, 0.0);
  h.xdiag.assign(nx * B, 1.0);
  h.xup.assign(nx * B, 0.0);
  h.ylo.assign(ny * B, 0.0);
  h.ydiag.assign(ny * B, 0.0);
  h.yup.assign(ny * B, 0.0);
  h.lo.resize(nx * ny * B);
  h.diag.resize(nx * ny * B);
  h.up.resize(nx * ny * B);
  for (int64_t b = 0; b < B; ++b) {
    const double tb = d->batch_tau ? d->batch_tau[b] : d->tau;
    for (int64_t i = 0; i < nx; ++i) {
      const int64_t j = b * nx + i;
      h.xlo[j] = i > 0 ? tb * d->k_lo[j] : 0.0;
      h.xdiag[j] = tb * d->k_diag[j];
      h.xup[j] = i + 1 < nx ? tb * d->k_up[j] : 0.0;
    }
    const double dd = d->k_diag_y[b * ny], c = ny > 1 ? d->k_up_y[b * ny] : 0.0;
    for (int64_t l = 0; l < ny; ++l) {
      const int64_t r = b * ny + l;
      h.ylo[r] = l > 0 ? tb * d->k_lo_y[r] : 0.0;
      h.ydiag[r] = tb * d->k_diag_y[r];
      h.yup[r] = l + 1 < ny ? tb * d->k_up_y[r] : 0.0;
      const double mu = tb * (dd + 2.0 * c * std::cos(M_PI * (double)(l + 1) / (double)(ny + 1)));
      for (int64_t ix = 0; ix < nx; ++ix) {
        const int64_t j = r * nx + ix;
        h.lo[j] = h.xlo[b * nx + ix];
        h.diag[j] = h.xdiag[b * nx + ix] + mu;
        h.up[j] = h.xup[b * nx + ix];
      }
    }
  }
  return h;
}

// Batched plans: K~ = diag(tau_b K_b), each block padded to nx rows with decoupled
// identity rows (their unknowns are zero); blocks never couple.
HostOp build_batched_operator(const pd_desc *d) {
  if (d->dim == 2) return build_batched_operator_2d(d);
  HostOp h;
  const int64_t nx = d->nx, B = d->batch, n = nx * B;
  h.xlo.assign(n, 0.0);
  h.xdiag.assign(n, 1.0);
  h.xup.assign(n, 0.0);
  for (int64_t b = 0; b < B; ++b) {
    const int64_t nb = d->batch_nx ? d->batch_nx[b] : nx;
    const double tb = d->batch_tau ? d->batch_tau[b] : d->tau;
    for (int64_t i = 0; i < nb; ++i) {
      const int64_t j = b * nx + i;
      h.xlo[j] = i > 0 ? tb * d->k_lo[j] : 0.0;
      h.xdiag[j] = tb * d->k_diag[j];
      h.xup[j] = i + 1 < nb ? tb * d->k_up[j] : 0.0;
    }
  }
  h.lo = h.xlo;
  h.diag = h.xdiag;
  h.up = h.xup;
  return h;
}

// K' = M^{-1/2} K M^{-1/2} for a diagonal mass matrix (1D rows; the batch's blocks stay
// decoupled since only existing couplings are scaled).
void scale_by_mass(HostOp &h, const double *m) {
  const int64_t n = (int64_t)h.xdiag.size();
  std::vector<double> s(n);
  for (int64_t j = 0; j < n; ++j) s[j] = 1.0 / std::sqrt(m[j]);
  for (int64_t j = 0; j < n; ++j) {
    h.xdiag[j] *= s[j] * s[j];
    if (j > 0) h.xlo[j] *= s[j] * s[j - 1];
    if (j + 1 < n) h.xup[j] *= s[j] * s[j + 1];
  }
  h.lo = h.xlo;
  h.diag = h.xdiag;
  h.up = h.xup;
}

HostOp build_operator_plain(const pd_desc *d);

HostOp build_operator(const pd_desc *d) {
  HostOp h = build_operator_plain(d);
  if (d->m_diag && d->dim == 1) scale_by_mass(h, d->m_diag);
  return h;
}

HostOp build_operator_plain(const pd_desc *d) {
  if (d->batch > 1) return build_batched_operator(d);
  HostOp h;
  const int64_t nx = d->nx, ny = d->dim == 2 ? d->ny : 1;
  h.xlo.assign(d->k_lo, d->k_lo + nx);
  h.xdiag.assign(d->k_diag, d->k_diag + nx);
  h.xup.assign(d->k_up, d->k_up + nx);
  h.xlo[0] = 0.0;
  h.xup[nx - 1] = 0.0;
  h.lo.resize(nx * ny);
  h.diag.resize(nx * ny);
  h.up.resize(nx * ny);
  std::vector<double> mu(ny, 0.0);
  if (d->dim == 2) {
    h.ylo.assign(d->k_lo_y, d->k_lo_y + ny);
    h.ydiag.assign(d->k_diag_y, d->k_diag_y + ny);
    h.yup.assign(d->k_up_y, d->k_up_y + ny);
    h.ylo[0] = 0.0;
    h.yup[ny - 1] = 0.0;
    const double dd = d->k_diag_y[0];
    const double c = ny > 1 ? d->k_up_y[0] : 0.0;
    for (int64_t l = 0; l < ny; ++l) mu[l] = dd + 2.0 * c * std::cos(M_PI * (double)(l + 1) / (double)(ny + 1));
  }
  for (int64_t l = 0; l < ny; ++l)
    for (int64_t ix = 0; ix < nx; ++ix) {
      const int64_t j = l * nx + ix;
      h.lo[j] = h.xlo[ix];
      h.diag[j] = h.xdiag[ix] + mu[l];
      h.up[j] = h.xup[ix];
    }
  return h;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(PD_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename X>
pd_status upload(X *dst, const X *src, size_t n, cudaStream_t s) {
  if (!dst || n == 0) return PD_OK;
  CK(cudaMemcpyAsync(dst, src, n * sizeof(X), cudaMemcpyHostToDevice, s));
  return PD_OK;
}

// K in the solve basis and every array derived from it (tau K in both precisions,
// the residual coefficients, the per-problem row counts of a batch), uploaded on the
// plan's stream.  Shared by paradiag_plan and paradiag_set_operator.
// The binary32 path solves the zero frequency in FP64 (the lane, pint.cu) when J_l's
// zero-frequency term gamma_0 A_0^{-1}, A_0 = (1 - alpha^{1/l}) I + tau K, is large:
// nu_0 = ||(l A_0)^{-1}|| ~ 1 / (T lambda_min(K)) for Algorithm 1 (its eigenvalue
// z^l / (z^l - 1) - 1, z = 1 + tau lambda_min, Theorem 3.1).  Then A_0^{-1} dominates b
// (eq. 7) and J_l (eq. 8), and binary32 solves of A_0 (relative error kappa(A_0) eps)
// would keep refinement from contracting.  Every other shift has |1 - pi_k| >= 2 sin(pi/l)
// and a well-conditioned system.  nu_0 is estimated per block by FP64 Thomas solves of
// A_0 x = 1 and A_0 x = (-1)^i (exact for M-matrices such as the heat and upwind operators,
// whose inverses are nonnegative), the largest |x_i| over the blocks, divided by l.
constexpr double kLaneWeight = 4.0;
double zero_frequency_weight(const pd_plan *p, const std::vector<double> &tlo, const std::vector<double> &tdiag,
                             const std::vector<double> &tup) {
  const double s0 = 1.0 - p->aroot;  // 1 - pi_0
  const int64_t nb = p->nblk, bl = p->blen;
  std::vector<double> cp(bl), dp(bl);
  double worst = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    const int64_t o = b * bl;
    for (int sign = 0; sign < 2; ++sign) {
      for (int64_t i = 0; i < bl; ++i) {
        const double lo = i > 0 ? tlo[o + i] : 0.0, up = i + 1 < bl ? tup[o + i] : 0.0;
        const double r = (sign && (i & 1)) ? -1.0 : 1.0;
        const double m = s0 + tdiag[o + i] - (i > 0 ? lo * cp[i - 1] : 0.0);
        cp[i] = up / m;
        dp[i] = (r - (i > 0 ? lo * dp[i - 1] : 0.0)) / m;
      }
      double x = dp[bl - 1];
      worst = std::max(worst, std::fabs(x));
      for (int64_t i = bl - 2; i >= 0; --i) {
        x = dp[i] - cp[i] * x;
        worst = std::max(worst, std::fabs(x));
      }
    }
  }
  return std::isfinite(worst) ? worst / (double)p->nt : 1e300;
}

pd_status upload_operator(pd_plan *p, const pd_desc *desc) {
  pd_status st = PD_OK;
  HostOp h = build_operator(desc);
  const int64_t nbar = p->nbar;
  std::vector<double> tlo(nbar), tdiag(nbar), tup(nbar);
  std::vector<float> flo(nbar), fdiag(nbar), fup(nbar);
  for (int64_t j = 0; j < nbar; ++j) {
    tlo[j] = p->tau * h.lo[j];
    tdiag[j] = p->tau * h.diag[j];
    tup[j] = p->tau * h.up[j];
    flo[j] = (float)tlo[j];
    fdiag[j] = (float)tdiag[j];
    fup[j] = (float)tup[j];
  }
  std::vector<double> rxl(p->nrx), rxd(p->nrx), rxu(p->nrx), ryl(p->ny), ryd(p->ny), ryu(p->ny);
  for (int64_t i = 0; i < p->nrx; ++i) {
    rxl[i] = p->tau * h.xlo[i];
    rxd[i] = 1.0 + p->tau * h.xdiag[i];
    rxu[i] = p->tau * h.xup[i];
  }
  if (p->dim == 2)
    for (int64_t i = 0; i < p->ny; ++i) {
      ryl[i] = p->tau * h.ylo[i];
      ryd[i] = p->tau * h.ydiag[i];
      ryu[i] = p->tau * h.yup[i];
    }
  if (p->precision == PD_MIXED) {
    p->nu0 = zero_frequency_weight(p, tlo, tdiag, tup);
    p->lane = desc->tune_zero_lane > 0 || (desc->tune_zero_lane == 0 && p->nu0 > kLaneWeight);
  }
  cudaStream_t s = p->ctx.stream;
  if ((st = upload(p->klo, h.lo.data(), nbar, s)) || (st = upload(p->kdiag, h.diag.data(), nbar, s)) ||
      (st = upload(p->kup, h.up.data(), nbar, s)) || (st = upload(p->tlo_d, tlo.data(), nbar, s)) ||
      (st = upload(p->tdiag_d, tdiag.data(), nbar, s)) || (st = upload(p->tup_d, tup.data(), nbar, s)) ||
      (st = upload(p->tlo_f, flo.data(), nbar, s)) || (st = upload(p->tdiag_f, fdiag.data(), nbar, s)) ||
      (st = upload(p->tup_f, fup.data(), nbar, s)) || (st = upload(p->xlo, h.xlo.data(), p->nrx, s)) ||
      (st = upload(p->xdiag, h.xdiag.data(), p->nrx, s)) || (st = upload(p->xup, h.xup.data(), p->nrx, s)) ||
      (st = upload(p->rxl, rxl.data(), p->nrx, s)) || (st = upload(p->rxd, rxd.data(), p->nrx, s)) ||
      (st = upload(p->rxu, rxu.data(), p->nrx, s)))
    return st;
  std::vector<double> rdd(p->dim == 2 ? p->nbar : 0);
  if (p->dim == 2)  // row iy of the stacked grid belongs to problem iy / nym (its x-coefficients)
    for (int64_t iy = 0; iy < p->ny; ++iy)
      for (int64_t x = 0; x < p->nx; ++x) rdd[iy * p->nx + x] = rxd[(iy / p->nym) * p->nx + x] + ryd[iy];
  if (p->dim == 2 && ((st = upload(p->rdd, rdd.data(), p->nbar, s)) ||
                      (st = upload(p->ryl, ryl.data(), p->ny, s)) || (st = upload(p->ryd, ryd.data(), p->ny, s)) ||
                      (st = upload(p->ryu, ryu.data(), p->ny, s)) || (st = upload(p->ylo, h.ylo.data(), p->ny, s)) ||
                      (st = upload(p->ydiag, h.ydiag.data(), p->ny, s)) || (st = upload(p->yup, h.yup.data(), p->ny, s))))
    return st;
  if (p->batch > 1) {
    std::vector<int> bnx(p->batch);
    // unknowns of problem b inside its slot (2D: the whole nx x ny grid)
    for (int b = 0; b < p->batch; ++b)
      bnx[b] = p->dim == 2 ? (int)p->nxm : (int)(desc->batch_nx ? desc->batch_nx[b] : desc->nx);
    if ((st = upload(p->bnx, bnx.data(), p->batch, s))) return st;
  }
  std::vector<double> msc;
  if (p->mass) {  // M^{-1/2}; identity when the descriptor carries no mass matrix
    msc.assign(nbar, 1.0);
    if (desc->m_diag)
      for (int64_t j = 0; j < nbar; ++j) msc[j] = 1.0 / std::sqrt(desc->m_diag[j]);
    if ((st = upload(p->msc, msc.data(), nbar, s))) return st;
  }
  // the host vectors die on return: wait for the copies
  if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PD_ERR_CUDA, "operator upload failed");
  return PD_OK;
}

pd_status ctx_status(pd_plan *p) {
  if (p->ctx.err != cudaSuccess)
    return fail(PD_ERR_CUDA, "kernel launch failed in %s: %s", p->ctx.err_where, cudaGetErrorString(p->ctx.err));
  return PD_OK;
}

pd_status sync_read(pd_plan *p, bool with_tail = false) {
  CK(cudaMemcpyAsync(p->h_scal, p->scal, pd::kScalWords * sizeof(double), cudaMemcpyDeviceToHost, p->ctx.stream));
  CK(cudaMemcpyAsync(p->h_flags, p->flags, pd::kFlagWords * sizeof(int), cudaMemcpyDeviceToHost, p->ctx.stream));
  if (with_tail && p->tail_dst) {
    CK(cudaMemcpyAsync(p->tail_dst, p->tail_src, p->tail_bytes, cudaMemcpyDeviceToHost, p->ctx.stream));
    p->tail_done = true;
  }
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
}

// The final loop by linearity applies to single problems of the full method whose zero
// frequency runs in binary32 like the others (the FP64 lane keeps the final loop's solves).
bool use_comb(const pd_plan *p) { return p->comb && !(p->precision == PD_MIXED && p->lane); }

template <typename T>
const cpx<T> *time_tw(pd_plan *p);
template <>
const cpx<double> *time_tw<double>(pd_plan *p) { return p->tw_d; }
template <>
const cpx<float> *time_tw<float>(pd_plan *p) { return p->tw_f; }
// D_alpha and D_alpha^{-1} on the time rows (Algorithm 3), or null for alpha = 1
template <typename T>
const T *row_scale(pd_plan *p, bool inverse);
template <>
const double *row_scale<double>(pd_plan *p, bool inverse) {
  return p->alpha == 1.0 ? nullptr : (inverse ? p->tsi_d : p->ts_d);
}
template <>
const float *row_scale<float>(pd_plan *p, bool inverse) {
  return p->alpha == 1.0 ? nullptr : (inverse ? p->tsi_f : p->ts_f);
}

template <typename T>
const T *vbasis(pd_plan *p);
template <>
const double *vbasis<double>(pd_plan *p) { return p->V; }
template <>
const float *vbasis<float>(pd_plan *p) { return p->Vf; }
template <typename T>
const T *xvec(pd_plan *p);
template <>
const double *xvec<double>(pd_plan *p) { return p->x; }
template <>
const float *xvec<float>(pd_plan *p) { return p->xf; }

template <typename T>
pd::PintArgs<T> base_args(pd_plan *p);
template <>
pd::PintArgs<double> base_args<double>(pd_plan *p) {
  pd::PintArgs<double> a{};
  if (p->precision == PD_FP64) a.fac_in = reinterpret_cast<const cpx<double> *>(p->fac);
  a.xm_scale = p->aroot;
  a.shift = p->shift;
  a.tlo = p->tlo_d;
  a.tdiag = p->tdiag_d;
  a.tup = p->tup_d;
  return a;
}
template <>
pd::PintArgs<float> base_args<float>(pd_plan *p) {
  pd::PintArgs<float> a{};
  if (p->precision == PD_MIXED) a.fac_in = reinterpret_cast<const cpx<float> *>(p->fac);
  a.xm_scale = p->aroot;
  a.shift = p->shift;
  a.shift_t = p->shift_f;
  a.tlo = p->tlo_f;
  a.tdiag = p->tdiag_f;
  a.tup = p->tup_f;
  // the zero frequency, whose shifted system carries the ill-conditioning of tau K, in FP64
  a.k0_fp64 = p->lane ? 1 : 0;
  a.tlo_d = p->tlo_d;
  a.tdiag_d = p->tdiag_d;
  a.tup_d = p->tup_d;
  a.Vd = p->V;
  a.fac0_in = p->lane ? p->fac0 : nullptr;
  return a;
}
// FP64 zero-frequency lane outputs of the binary32 path (null for FP64 plans and when the
// lane is off)
template <typename T>
double *lane_acc0(pd_plan *p) {
  return (sizeof(T) == 4 && p->lane) ? p->acc0 : nullptr;
}
template <typename T>
double *lane_h0(pd_plan *p) {
  return (sizeof(T) == 4 && p->lane) ? p->h0 : nullptr;
}

// Factor every (k, block) shifted system of the plan (after the operator changed).
pd_status factorize(pd_plan *p) {
  if (p->precision == PD_MIXED && p->lane) {  // the FP64 factors of the zero-frequency lane
    pd::PintArgs<float> a = base_args<float>(p);
    a.fac_in = nullptr;
    a.fac0_in = nullptr;
    a.fac0_out = p->fac0;
    pd::launch_pint<float>(p->ctx, p->geom, a);
  }
  if (!p->fac) return ctx_status(p);
  if (p->precision == PD_MIXED) {
    pd::PintArgs<float> a = base_args<float>(p);
    a.fac_in = nullptr;
    a.k0_fp64 = 0;  // every frequency's binary32 factors are stored
    a.fac0_in = nullptr;
    a.fac_out = reinterpret_cast<cpx<float> *>(p->fac);
    pd::launch_pint<float>(p->ctx, p->geom, a);
  } else {
    pd::PintArgs<double> a = base_args<double>(p);
    a.fac_in = nullptr;
    a.fac_out = reinterpret_cast<cpx<double> *>(p->fac);
    pd::launch_pint<double>(p->ctx, p->geom, a);
  }
  return ctx_status(p);
}

template <typename T>
T *tmp_buf(pd_plan *p);
template <>
double *tmp_buf<double>(pd_plan *p) { return p->tmp_d; }
template <>
float *tmp_buf<float>(pd_plan *p) { return p->tmp_f; }
template <typename T>
const cpx<T> *dst_tw(pd_plan *p);
template <>
const cpx<double> *dst_tw<double>(pd_plan *p) { return p->twy_d; }
template <>
const cpx<float> *dst_tw<float>(pd_plan *p) { return p->twy_f; }

template <typename T>
pd::KrylovBufs kbufs(pd_plan *p) {
  return pd::KrylovBufs{(int)p->nbar, p->maxit, p->klo, p->kdiag, p->kup, p->V, sizeof(T) == 4 ? p->Vf : nullptr,
                        p->T, p->w, p->part, p->blas_grid, p->scal, p->flags, p->blas_cluster,
                        p->members, (int)p->nxm, p->mscal, p->mflags, p->y, p->flags + pd::F_MEMCNT, p->q};
}

// Algorithm-2 stopping parameters of the first solve (kind 0) and of refinement
// sweeps (kind 1).  Algorithm 2 stops at eps * beta or maxit (Sec. 3), and also once
// the eq. (13) residual stops halving near the precision floor: in binary32 it
// levels off at the rounding noise of the shifted solves, and in FP64 the polynomial
// space K_m(K, b) can stall for many steps when J_l is far from I.  A binary32
// refinement sweep contracts the error by ~1e-3 at best (rounding noise of the
// residual, amplified by the solution operator), so its Algorithm 2 asks for 1e-3; FOM
// residuals are not monotone, so it leaves on a stall only after two checks without
// halving and once ||r_m|| <= 1e-2 ref (far above the binary32 noise floor of eq. 13, far
// below a residual that would keep the refinement from contracting).  FP64 refinement
// sweeps (only after a stall) ask for 1e-8.
pd::KrylovCtl krylov_ctl(pd_plan *p, int kind) {
  const bool fp64 = p->precision == PD_FP64;
  pd::KrylovCtl k;
  k.eps = kind == 0 ? p->eps : std::max(p->eps, fp64 ? 1e-8 : p->eps_refine);
  k.stall_floor = fp64 ? 1e-6 : (kind == 0 ? 1e-3 : 10.0 * p->eps_refine);
  k.win = fp64 ? 3 : (kind == 0 ? 1 : 2);
  if (p->refined64) {  // refined FP64 plans: leave a stalled step at any level
    k.eps = std::max(p->eps, 1e-8);
    k.stall_floor = 1.0;
    k.win = 2;
  } else if (fp64 && kind == 1) {  // an FP64 refinement sweep only needs a contraction
    k.stall_floor = 1.0;
    k.win = 2;
  }
  // plans that refine measure ||r_m|| against ||R||_F of the solve's right-hand side
  // (krylov_decide); single problems only (batches keep each problem's beta)
  k.rrel = (!p->members && (!fp64 || p->refined64 || kind == 1)) ? 1 : 0;
  k.maxit = p->maxit;
  k.q = p->q;
  return k;
}

pd::RefineCtl refine_ctl(pd_plan *p) {
  const bool fp64 = p->precision == PD_FP64;
  pd::RefineCtl r;
  // refined FP64 plans stop like the mixed ones (by the contraction of the updates)
  r.fp64 = (fp64 && !p->refined64) ? 1 : 0;
  r.eps_first = p->eps;
  r.eps_refine = p->refined64 ? std::max(p->eps, 1e-8) : std::max(p->eps, fp64 ? 1e-8 : p->eps_refine);
  r.refine_tol = p->refine_tol;
  r.max_refine = p->max_refine;
  r.msw = p->batch > 1 ? p->msw : nullptr;
  r.mconv = p->batch > 1 ? p->mconv : nullptr;
  r.member_solves = p->member_solves;
  return r;
}

// ---- the three segments of one solve -------------------------------------------
// kind 0: the first solve, for G (Algorithm 1).  kind 1: a refinement sweep, for the
// FP64 all-at-once residual G - [(I + tau K) U - U Sigma_1^T], added into U.  If
// Algorithm 2 stops with ||r_m|| > 0, the U it produces satisfies eq. (2) up to
// exactly -r_m in the first time step (its last slice is x_m - r_m while the
// correction used x_m), so a sweep on that residual corrects precisely the Krylov
// error.  In 2D every solve runs between one DST along y of its input and one of
// its output.

// forward DFT (eq. 5), first parallel-in-time loop with b = L F^{-T} e_l (eq. 7),
// beta = ||b|| and v_1 (Algorithm 2, first step)
template <typename T>
pd_status emit_pre(pd_plan *p, int kind, const double *G, double *U, int use_handle,
                   cudaGraphConditionalHandle hk) {
  pd::Ctx &c = p->ctx;
  cpx<T> *S = reinterpret_cast<cpx<T> *>(p->spec);
  const int nt = (int)p->nt;
  T *tmp = tmp_buf<T>(p);
  // ||R||_F of this solve's right-hand side, the reference of the refining plans' Algorithm-2
  // stop (krylov_decide); batches measure each problem against its own beta instead
  const pd::RhsNorm rn{p->norm_part, p->flags + pd::F_RNCNT, p->scal + pd::S_RNORM};
  const pd::RhsNorm *rnp = p->members ? nullptr : &rn;
  if (kind == 0) {
    if (p->dim == 1) {
      pd::launch_fft_r2c<T, double>(c, G, p->nbar, p->nbar, nt, time_tw<T>(p), S, p->lds, row_scale<T>(p, false),
                                    rnp);
    } else {
      pd::launch_dst_y<double, T, T>(c, G, tmp, p->nt * p->batch, p->nym, p->nx, dst_tw<T>(p), 0);
      pd::launch_fft_r2c<T, T>(c, tmp, p->nbar, p->nbar, nt, time_tw<T>(p), S, p->lds, row_scale<T>(p, false), rnp);
    }
  } else {
    if (p->dim == 1) {  // the FP64 residual is formed while the DFT loads its tiles
      pd::launch_fft_r2c_residual<T>(c, G, U, p->nbar, nt, p->rxl, p->rxd, p->rxu, time_tw<T>(p), S, p->lds,
                                     row_scale<T>(p, false), p->batch > 1 ? p->mex : nullptr, (int)p->nxm, rnp);
    } else {
      // the FP64 residual is formed while the DST along y loads its tiles
      pd::launch_dst_y_residual<T>(c, G, U, tmp, p->nt, p->batch, p->nym, p->nx, p->rxl, p->rdd, p->rxu, p->ryl,
                                   p->ryu, p->batch > 1 ? p->mex : nullptr, dst_tw<T>(p));
      pd::launch_fft_r2c<T, T>(c, tmp, p->nbar, p->nbar, nt, time_tw<T>(p), S, p->lds, row_scale<T>(p, false), rnp);
    }
  }
  if (p->loops == 1) {  // U = U_1: no b and no Algorithm 2; the final loop runs with x_m = 0
    pd::launch_inner_fixed(c, p->scal, p->flags, p->y, 1, use_handle, hk);
    return PD_OK;
  }
  // Algorithm 3's test on U_1 (first solve) forms U_1 from L
  const bool early = kind == 0 && p->early_eps > 0.0;
  // L_k = A_k^{-1} G^_k: kept for the final loop by linearity, or for U_1 (then in the h_k
  // buffer, free until Algorithm 2 starts)
  const bool comb = use_comb(p);
  cpx<T> *L = reinterpret_cast<cpx<T> *>(comb ? p->lbuf : p->hbuf);
  pd::PintArgs<T> a = base_args<T>(p);
  a.R = S;
  a.ldr = p->lds;
  a.omega = p->wg;
  if constexpr (sizeof(T) == 4) a.omega_t = reinterpret_cast<const cpx<T> *>(p->wg_f);
  a.acc_part = p->acc_part;
  a.acc0 = lane_acc0<T>(p);
  if (early || comb) {
    a.Y = L;
    a.ldy = p->lds;
  }
  pd::launch_pint<T>(c, p->geom, a);
  pd::KrylovBufs kb = kbufs<T>(p);
  double *acc0 = lane_acc0<T>(p);
  if (kb.members) {
    pd::launch_acc_reduce(c, p->geom, p->acc_part, p->b, nullptr, nullptr, acc0);
    pd::launch_member_init(c, kb, p->b, use_handle, hk);
  } else if (p->krylov_tails) {  // beta and v_1 in the b reduction's last CTA
    const pd::InitTail t{1, p->flags + pd::F_ACCCNT, kb.n, kb.maxit + 2, (kb.maxit + 1) * kb.maxit, use_handle,
                         kb.part, kb.V, kb.scal, kb.T, kb.Vf, kb.flags, hk};
    pd::launch_acc_reduce(c, p->geom, p->acc_part, p->b, nullptr, &t, acc0);
  } else {
    pd::launch_acc_reduce(c, p->geom, p->acc_part, p->b, nullptr, nullptr, acc0);
    pd::launch_vec_norm_init(c, kb, p->b, use_handle, hk);
  }
  // x_m = b: the inner matrix of eq. (17) taken as I (two loops in all)
  if (p->loops == 2) pd::launch_inner_fixed(c, p->scal, p->flags, p->y, 2, use_handle, hk);
  if (early) {  // U_1 = L F^{-T} D_alpha^{-1} into U, then its residual against eps ||U_1||
    int nparts = 0;
    if (p->dim == 1) {
      pd::launch_fft_c2r<T>(c, L, p->lds, p->nbar, nt, time_tw<T>(p), U, p->nbar, 0, nullptr, &nparts, nullptr,
                            row_scale<T>(p, true));
    } else {
      pd::launch_fft_c2r<T>(c, L, p->lds, p->nbar, nt, time_tw<T>(p), tmp, p->nbar, sizeof(T) == 8 ? 0 : 2, nullptr,
                            &nparts, nullptr, row_scale<T>(p, true));
      pd::launch_dst_y<T, double, T>(c, tmp, U, p->nt, p->nym, p->nx, dst_tw<T>(p), 0);
    }
    pd::launch_early_check(c, G, U, p->nt, p->ny, p->nx, p->rxl, p->rxd, p->rxu, p->ryl, p->ryd, p->ryu, p->nym,
                           p->early_eps, p->norm_part, p->scal, p->flags, use_handle, hk);
  }
  // the persistent step ends with the next step's Arnoldi step: the first one runs here
  if (p->persist) pd::launch_arnoldi(c, kb);
  return PD_OK;
}

template <typename T>
pd::StepArgs<T> step_args(pd_plan *p, int kind, int use_handle, cudaGraphConditionalHandle hk) {
  pd::StepArgs<T> a{};
  a.n = (int)p->nbar;
  a.maxit = p->maxit;
  a.q = p->q;
  a.ld = p->maxit + 2;
  a.klo = p->klo;
  a.kdiag = p->kdiag;
  a.kup = p->kup;
  a.V = p->V;
  a.w = p->w;
  a.T = p->T;
  a.part = p->part;
  a.scal = p->scal;
  a.z = p->z;
  a.Vf = sizeof(T) == 4 ? p->Vf : nullptr;
  a.flags = p->flags;
  a.tau = p->tau;
  a.kc = krylov_ctl(p, kind);
  a.nf = p->nf;
  a.nblk = p->nblk;
  a.shift = p->shift;
  a.wg = p->wga;
  a.gpart = p->gpart;
  a.msys_part = p->msys_part;
  a.y = p->y;
  a.srow = p->srow;
  a.omega = p->omega;
  a.sinv = use_comb(p) ? p->sinv : nullptr;
  a.H = reinterpret_cast<const cpx<T> *>(p->hbuf);
  a.ldh = p->lds;
  a.h0 = lane_h0<T>(p);
  a.zrg = p->persist_zrg;
  a.nv = p->persist_nv;
  a.smem = p->persist_smem;
  a.bar_polls = p->bar_polls;
  a.bar_extra = p->bar_extra;
  a.use_handle = use_handle;
  a.h = hk;
  return a;
}

// one step of Algorithm 2 (m read on the device)
template <typename T>
pd_status emit_iter(pd_plan *p, int kind, int use_handle, cudaGraphConditionalHandle hk) {
  pd::Ctx &c = p->ctx;
  pd::KrylovBufs kb = kbufs<T>(p);
  if (kb.members)
    pd::launch_member_arnoldi(c, kb);
  else if (!p->persist)  // the persistent step ran this Arnoldi step at its end
    pd::launch_arnoldi(c, kb);
  cpx<T> *H = reinterpret_cast<cpx<T> *>(p->hbuf);
  // no h_k at a breakdown (eq. 12 loses its t-term) or on a frozen step (q > 1); batches
  // run q = 1 and read the batch-level breakdown flag
  const int *noh = kb.members ? p->flags + pd::F_BREAK : p->flags + pd::F_NOH;
  {  // h_k = ((1 - pi_k) I + tau K)^{-1} v_{m+1} (stored) and g_k = V_m^T h_k
    pd::PintArgs<T> a = base_args<T>(p);
    a.mcount = p->flags + pd::F_M;
    a.want_dots = 1;
    a.mdots_max = p->maxit;
    a.V = vbasis<T>(p);
    a.ldv = p->nbar;
    a.gpart = p->gpart;
    a.Y = H;
    a.ldy = p->lds;
    a.skip_flag = noh;
    a.h0 = lane_h0<T>(p);
    pd::launch_pint<T>(c, p->geom, a);
  }
  if (p->persist) {
    pd::launch_step_tail<T>(c, step_args<T>(p, kind, use_handle, hk), p->persist_grid, p->persist_E);
    return PD_OK;
  }
  const double *h0 = lane_h0<T>(p);
  pd::launch_capacitance(c, kb, p->nf, p->tau, p->shift, p->wga, p->gpart, p->nblk, p->msys_part,
                         kb.members ? p->k5_grid_members : p->k5_grid,
                         p->srow, p->omega, p->y, kb.members, (int)p->nym, use_comb(p) ? p->sinv : nullptr);
  // z = sum_i gamma_i h_i (e_m^T S_i y_m) from the stored h_i, then eq. (13)
  if (kb.members) {
    pd::launch_zsum<T>(c, p->nf, p->nbar, H, p->lds, p->omega, p->z, noh, nullptr, kb.mlen, h0);
    pd::launch_member_project(c, kb, p->z, p->tau, krylov_ctl(p, kind), use_handle, hk);
  } else if (p->krylov_tails) {  // eq. (13) and the decision in the z reduction's last CTA
    const pd::ProjTail t{1, p->flags + pd::F_ZCNT, kb.n, kb.maxit + 2, use_handle, kb.V, p->tau, kb.part, kb.scal,
                         kb.flags, krylov_ctl(p, kind), hk};
    pd::launch_zsum<T>(c, p->nf, p->nbar, H, p->lds, p->omega, p->z, noh, &t, 0, h0);
  } else {
    pd::launch_zsum<T>(c, p->nf, p->nbar, H, p->lds, p->omega, p->z, noh, nullptr, 0, h0);
    pd::launch_project_resnorm(c, kb, p->z, p->tau, krylov_ctl(p, kind), use_handle, hk);
  }
  return PD_OK;
}

// x_m = V_m y_m; final parallel-in-time loop Y_k = A_k^{-1} (G^_k - x_m) (L - W fused);
// U = (L - W) F^{-T}; ||delta||^2; refinement decision
template <typename T>
pd_status emit_post(pd_plan *p, int kind, double *U, int use_handle, cudaGraphConditionalHandle hr) {
  pd::Ctx &c = p->ctx;
  cpx<T> *S = reinterpret_cast<cpx<T> *>(p->spec);
  const int nt = (int)p->nt;
  const bool fp64 = sizeof(T) == 8;
  pd::PintArgs<T> a = base_args<T>(p);
  a.R = S;
  a.ldr = p->lds;
  a.xm_count = p->flags + pd::F_M;  // x_m = V_m y_m formed by each team
  a.xm_y = p->y;
  a.xm_ldy = p->members ? p->maxit + 1 : 0;  // batch member: its own y_m
  a.xm_bpm = (int)p->nym;                     // blocks per member (2D: one per mode of T_y)
  a.V = vbasis<T>(p);
  a.ldv = p->nbar;
  a.xm_Vd = p->V;
  a.xm_out = p->x;
  a.Y = S;
  a.ldy = p->lds;
  const bool early = kind == 0 && p->early_eps > 0.0;
  const int *skip = early ? p->flags + pd::F_EARLY : nullptr;  // U = U_1 already
  a.skip_flag = skip;
  // after one Algorithm-2 step the final loop is formed by linearity (into S), and its
  // shifted solves skip
  if (use_comb(p)) {
    pd::launch_final_comb<T>(c, p->nf, p->nbar, p->lds, p->tau, p->aroot, p->shift, p->T, p->y, p->V, vbasis<T>(p),
                             p->scal, p->flags, p->sinv, std::min(p->maxit, pd::kCombMaxM),
                             reinterpret_cast<const cpx<T> *>(p->lbuf), reinterpret_cast<const cpx<T> *>(p->hbuf), S,
                             p->x);
    a.skip_flag2 = p->flags + pd::F_COMB;
  }
  pd::launch_pint<T>(c, p->geom, a);
  if (kind == 0) {
    CK(cudaMemcpyAsync(p->b0, p->b, sizeof(double) * p->nbar, cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaMemcpyAsync(p->x0, p->x, sizeof(double) * p->nbar, cudaMemcpyDeviceToDevice, c.stream));
  }
  // inverse DFT; its last CTA sums ||delta||^2 and takes the refinement decision
  pd::StepFinish fin{};
  fin.enabled = 1;
  fin.counter = p->flags + pd::F_C2RCNT;
  fin.scal = p->scal;
  fin.flags = p->flags;
  fin.rc = refine_ctl(p);
  fin.use_handle = use_handle;
  fin.h = hr;
  int nparts = 0;
  if (p->batch > 1) {  // per-problem norms and decision (every problem must converge)
    if (p->dim == 2) {  // the DST is orthonormal: the column norms of its input are delta's
      T *tmp = tmp_buf<T>(p);
      pd::launch_fft_c2r<T>(c, S, p->lds, p->nbar, nt, time_tw<T>(p), tmp, p->nbar, fp64 ? 0 : 2, nullptr, &nparts,
                            nullptr, row_scale<T>(p, true), p->colsum, kind == 0 ? nullptr : p->mex, (int)p->nxm);
      pd::launch_dst_y<T, double, T>(c, tmp, U, p->nt * p->batch, p->nym, p->nx, dst_tw<T>(p), kind == 0 ? 0 : 1);
    } else {
      pd::launch_fft_c2r<T>(c, S, p->lds, p->nbar, nt, time_tw<T>(p), U, p->nbar, kind == 0 ? 0 : 1, nullptr,
                            &nparts, nullptr, row_scale<T>(p, true), p->colsum, kind == 0 ? nullptr : p->mex,
                            (int)p->nxm);
    }
    pd::launch_member_decide(c, p->colsum, (int)p->nxm, p->bnx, p->batch, p->md2, p->mref2, p->mprev, p->mex, p->bzero,
                             p->scal, p->flags, refine_ctl(p), use_handle, hr);
  } else if (p->dim == 1) {
    pd::launch_fft_c2r<T>(c, S, p->lds, p->nbar, nt, time_tw<T>(p), U, p->nbar, kind == 0 ? 0 : 1, p->norm_part,
                          &nparts, &fin, row_scale<T>(p, true), nullptr, nullptr, 1, skip);
  } else {
    T *tmp = tmp_buf<T>(p);
    pd::launch_fft_c2r<T>(c, S, p->lds, p->nbar, nt, time_tw<T>(p), tmp, p->nbar, fp64 ? 0 : 2, p->norm_part,
                          &nparts, &fin, row_scale<T>(p, true), nullptr, nullptr, 1, skip);
    pd::launch_dst_y<T, double, T>(c, tmp, U, p->nt, p->nym, p->nx, dst_tw<T>(p), kind == 0 ? 0 : 1, skip);
  }
  if (early) pd::launch_early_finish(c, p->scal, p->flags, use_handle, hr);
  return PD_OK;
}

pd_status timeout_status(pd_plan *p) {
  return fail(PD_ERR_TIMEOUT,
              "a grid barrier of the persistent Algorithm-2 step waited %lld polls without the other CTAs; "
              "U is unspecified, the plan stays usable",
              p->bar_polls);
}

// Host-driven loops (timing mode, or when graphs are unavailable): the same kernels,
// with the host reading the control block after each step.
template <typename T>
pd_status solve_hostloop(pd_plan *p, const double *G, double *U) {
  pd::Ctx &c = p->ctx;
  pd_status st;
  pd::launch_solve_reset(c, p->scal, p->flags);
  for (int kind = 0;; kind = 1) {
    if ((st = emit_pre<T>(p, kind, G, U, 0, 0)) != PD_OK) return st;
    if ((st = sync_read(p)) != PD_OK) return st;
    while (!p->h_flags[pd::F_KSTOP]) {
      if ((st = emit_iter<T>(p, kind, 0, 0)) != PD_OK) return st;
      if ((st = sync_read(p)) != PD_OK) return st;
      if (p->h_flags[pd::F_TIMEOUT]) return timeout_status(p);
    }
    if ((st = emit_post<T>(p, kind, U, 0, 0)) != PD_OK) return st;
    if ((st = sync_read(p)) != PD_OK) return st;
    if (p->h_flags[pd::F_RSTOP]) break;
  }
  return ctx_status(p);
}

// Refinement sweeps only, on the U given (paradiag_batch_advance): the same kernels as the
// host-driven loop, every solve a sweep on the FP64 residual, until the decision stops.
template <typename T>
pd_status solve_continue(pd_plan *p, const double *G, double *U) {
  pd::Ctx &c = p->ctx;
  pd_status st;
  pd::launch_solve_reset(c, p->scal, p->flags);
  for (;;) {
    if ((st = emit_pre<T>(p, 1, G, U, 0, 0)) != PD_OK) return st;
    if ((st = sync_read(p)) != PD_OK) return st;
    while (!p->h_flags[pd::F_KSTOP]) {
      if ((st = emit_iter<T>(p, 1, 0, 0)) != PD_OK) return st;
      if ((st = sync_read(p)) != PD_OK) return st;
      if (p->h_flags[pd::F_TIMEOUT]) return timeout_status(p);
    }
    if ((st = emit_post<T>(p, 1, U, 0, 0)) != PD_OK) return st;
    if ((st = sync_read(p)) != PD_OK) return st;
    if (p->h_flags[pd::F_RSTOP]) break;
  }
  return ctx_status(p);
}

// ---- CUDA graph of the whole solve -------------------------------------------------
// top:   reset, pre(0), WHILE_k0 { iter(0) }, post(0),
//        WHILE_R { pre(1), WHILE_k1 { iter(1) }, post(1) }
// The conditionals are set on the device by the init / decide kernels, so one graph
// launch runs the solve with a single host synchronisation at the end.

#define GK(call)                   \
  do {                             \
    cudaError_t e_ = (call);       \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

// Append a WHILE node after the capture frontier of `s`; return its body graph.
cudaError_t splice_while(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraph_t *body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t *deps = nullptr;
  size_t nd = 0;
  GK(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  GK(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
  *body = np.conditional.phGraph_out[0];
  GK(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  return cudaSuccess;
}

template <typename T>
cudaError_t capture_iter_body(pd_plan *p, cudaGraph_t body, cudaStream_t s, int kind, cudaGraphConditionalHandle hk) {
  GK(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  cudaStream_t keep = p->ctx.stream;
  p->ctx.stream = s;
  const pd_status st = emit_iter<T>(p, kind, 1, hk);
  p->ctx.stream = keep;
  cudaGraph_t out = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &out);
  if (st != PD_OK || p->ctx.err != cudaSuccess) return cudaErrorUnknown;
  return e;
}

template <typename T>
cudaError_t build_graph(pd_plan *p, const double *G, double *U, cudaGraph_t *gout) {
  cudaStream_t s0 = p->cap[0], s1 = p->cap[1], s2 = p->cap[2];
  cudaStream_t keep = p->ctx.stream;
  cudaGraph_t g = nullptr;
  GK(cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed));
  cudaError_t err = cudaSuccess;
  do {
    cudaStreamCaptureStatus cs;
    if ((err = cudaStreamGetCaptureInfo(s0, &cs, nullptr, &g, nullptr, nullptr, nullptr)) != cudaSuccess) break;
    cudaGraphConditionalHandle hk0, hR, hk1;
    if ((err = cudaGraphConditionalHandleCreate(&hk0, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    if ((err = cudaGraphConditionalHandleCreate(&hR, g, 0, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    p->ctx.stream = s0;
    int64_t l0 = p->ctx.launches;
    pd::launch_solve_reset(p->ctx, p->scal, p->flags);
    if (emit_pre<T>(p, 0, G, U, 1, hk0) != PD_OK) { err = cudaErrorUnknown; break; }
    p->seg.pre0 = p->ctx.launches - l0;
    cudaGraph_t body = nullptr;
    if ((err = splice_while(s0, hk0, &body)) != cudaSuccess) break;
    l0 = p->ctx.launches;
    if ((err = capture_iter_body<T>(p, body, s1, 0, hk0)) != cudaSuccess) break;
    p->seg.iter0 = p->ctx.launches - l0;
    p->ctx.stream = s0;
    l0 = p->ctx.launches;
    if (emit_post<T>(p, 0, U, 1, hR) != PD_OK) { err = cudaErrorUnknown; break; }
    p->seg.post0 = p->ctx.launches - l0;
    cudaGraph_t bodyR = nullptr;
    if ((err = splice_while(s0, hR, &bodyR)) != cudaSuccess) break;
    if ((err = cudaGraphConditionalHandleCreate(&hk1, bodyR, 1, cudaGraphCondAssignDefault)) != cudaSuccess) break;
    // refinement body: pre(1), WHILE_k1 { iter(1) }, post(1), captured on s1
    if ((err = cudaStreamBeginCaptureToGraph(s1, bodyR, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed)) !=
        cudaSuccess)
      break;
    p->ctx.stream = s1;
    l0 = p->ctx.launches;
    bool ok = emit_pre<T>(p, 1, G, U, 1, hk1) == PD_OK;
    p->seg.pre1 = p->ctx.launches - l0;
    cudaGraph_t body1 = nullptr;
    if (ok) ok = splice_while(s1, hk1, &body1) == cudaSuccess;
    l0 = p->ctx.launches;
    if (ok) ok = capture_iter_body<T>(p, body1, s2, 1, hk1) == cudaSuccess;
    p->seg.iter1 = p->ctx.launches - l0;
    p->ctx.stream = s1;
    l0 = p->ctx.launches;
    if (ok) ok = emit_post<T>(p, 1, U, 1, hR) == PD_OK;
    p->seg.post1 = p->ctx.launches - l0;
    cudaGraph_t outR = nullptr;
    const cudaError_t e1 = cudaStreamEndCapture(s1, &outR);
    if (!ok || e1 != cudaSuccess || p->ctx.err != cudaSuccess) {
      err = cudaErrorUnknown;
      break;
    }
  } while (false);
  p->ctx.stream = keep;
  cudaGraph_t out = nullptr;
  const cudaError_t e0 = cudaStreamEndCapture(s0, &out);
  if (err == cudaSuccess) err = e0;
  if (err != cudaSuccess) {
    if (out) cudaGraphDestroy(out);
    return err;
  }
  *gout = out;
  return cudaSuccess;
}

void drop_graph(pd_plan *p) {
  if (p->gexec) cudaGraphExecDestroy(p->gexec);
  p->gexec = nullptr;
  p->g_G = nullptr;
  p->g_U = nullptr;
}

template <typename T>
pd_status solve_graph(pd_plan *p, const double *G, double *U, bool *used) {
  *used = false;
  if (p->graph_failed || p->ctx.timing) return PD_OK;
  if (!p->gexec || p->g_G != G || p->g_U != U) {
    std::lock_guard<std::recursive_mutex> lk(host_mutex());  // one capture at a time in the process
    drop_graph(p);
    const int64_t l0 = p->ctx.launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = build_graph<T>(p, G, U, &g);
    p->ctx.launches = l0;  // capture launches nothing
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || p->ctx.err != cudaSuccess) {
      // graphs unavailable here: use the host-driven loops from now on
      cudaGetLastError();
      p->ctx.err = cudaSuccess;
      p->gexec = nullptr;
      p->graph_failed = true;
      return PD_OK;
    }
    p->g_G = G;
    p->g_U = U;
  }
  CK(cudaGraphLaunch(p->gexec, p->ctx.stream));
  pd_status st = sync_read(p, true);
  if (st != PD_OK) return st;
  // kernels run = fixed segments + m steps of Algorithm 2 per solve
  const int sweeps = p->h_flags[pd::F_SWEEP];
  int64_t n = p->seg.pre0 + p->seg.post0 + (int64_t)p->seg.iter0 * p->h_flags[pd::F_SWM];
  for (int s = 1; s < sweeps && s < 16; ++s)
    n += p->seg.pre1 + p->seg.post1 + (int64_t)p->seg.iter1 * p->h_flags[pd::F_SWM + s];
  p->ctx.launches += n;
  *used = true;
  return PD_OK;
}

template <typename T>
pd_status solve_refined(pd_plan *p, const double *G, double *U, pd_stats &s) {
  bool used = false;
  pd_status st = p->use_graphs ? solve_graph<T>(p, G, U, &used) : PD_OK;
  if (st != PD_OK) return st;
  if (!used) {
    if ((st = solve_hostloop<T>(p, G, U)) != PD_OK) return st;
  }
  const int *f = p->h_flags;
  const double *sc = p->h_scal;
  const int sweeps = f[pd::F_SWEEP];
  const int last = std::min(std::max(sweeps - 1, 0), 15);
  s.refine_sweeps = sweeps;
  s.krylov_iters = f[pd::F_SWM + last];
  s.krylov_iters_total = f[pd::F_MTOT];
  s.pint_loops = 0;
  s.shifted_sweeps = 0;
  for (int i = 0; i < sweeps && i < 16; ++i) {
    s.sweep_krylov_iters[i] = f[pd::F_SWM + i];
    s.sweep_krylov_rel_resnorm[i] = sc[pd::S_SWRES + i];
    s.sweep_rel_update[i] = sc[pd::S_SWUPD + i];
    // a residual check (one pass over the shifted systems) every q steps and at the last
    // step, plus the b and final passes
    const int checks = (f[pd::F_SWM + i] + p->q - 1) / p->q;
    s.pint_loops += p->loops ? p->loops : checks + 2;
    s.shifted_sweeps += p->loops ? p->loops : checks + 2;
    if (p->loops) s.sweep_krylov_iters[i] = 0;  // m = 1 only carries x_m = b
  }
  s.final_by_linearity = f[pd::F_COMBCNT];
  s.shifted_sweeps -= f[pd::F_COMBCNT];
  s.breakdown = f[pd::F_BREAK];
  s.beta = sc[pd::S_SWBETA + last];
  s.krylov_rel_resnorm = sc[pd::S_SWRES + last];
  s.rel_update = sweeps > 1 ? sc[pd::S_UPD] : 0.0;
  s.graph = used ? 1 : 0;
  s.zero_freq_fp64 = p->lane ? 1 : 0;
  s.zero_freq_weight = p->nu0;
  s.persistent_step = p->persist ? 1 : 0;
  s.early_exit = f[pd::F_EARLY];
  s.u1_rel_residual = sc[pd::S_U1NORM] > 0.0 ? sc[pd::S_U1RES] / sc[pd::S_U1NORM] : 0.0;
  if (f[pd::F_EARLY]) {  // U = U_1: one parallel-in-time loop, no Algorithm 2
    s.pint_loops = s.shifted_sweeps = 1;
    s.krylov_iters = s.krylov_iters_total = 0;
    s.sweep_krylov_iters[0] = 0;
  }
  if (f[pd::F_TIMEOUT]) return timeout_status(p);
  if (f[pd::F_NONFIN]) return fail(PD_ERR_NONFINITE, "non-finite value met (input contains NaN/Inf?)");
  if (p->loops) {  // the variant's approximation: no convergence claim
    s.krylov_iters = s.krylov_iters_total = 0;
    return PD_OK;
  }
  return f[pd::F_RCONV] ? PD_OK
                        : fail(PD_ERR_NOT_CONVERGED, "refinement did not reach refine_tol in %d solves", sweeps);
}

pd_status check_plan(pd_plan *p) {
  if (!p) return fail(PD_ERR_INVALID_ARG, "plan is NULL");
  if (p->ctx.err != cudaSuccess) return fail(PD_ERR_CUDA, "plan is in an error state; destroy it");
  return PD_OK;
}

}  // namespace

extern "C" {

const char *paradiag_last_error(void) { return g_err.c_str(); }

const char *paradiag_version(void) { return "paradiag-gb300 0.1 (sm_103a)"; }

pd_status paradiag_workspace_size(const pd_desc *desc, size_t *bytes) {
  pd_status st = validate(desc);
  if (st != PD_OK) return st;
  if (!bytes) return fail(PD_ERR_INVALID_ARG, "bytes is NULL");
  pd_plan tmp;
  fill_geometry(&tmp, desc);
  *bytes = layout(&tmp, nullptr);
  return PD_OK;
}

pd_status paradiag_plan(const pd_desc *desc, void *workspace, size_t workspace_bytes, pd_plan **out) {
  std::lock_guard<std::recursive_mutex> lk(host_mutex());
  g_err.clear();
  pd_status st = validate(desc);
  if (st != PD_OK) return st;
  if (!out) return fail(PD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (workspace && ((uintptr_t)workspace & 255)) return fail(PD_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  pd_plan *p = new pd_plan();
  fill_geometry(p, desc);
  p->ctx.stream = (cudaStream_t)desc->stream;
  const size_t need = layout(p, nullptr);
  if (workspace) {
    if (workspace_bytes < need) {
      delete p;
      return fail(PD_ERR_OOM, "workspace of %zu bytes is smaller than the %zu bytes needed", workspace_bytes, need);
    }
    p->ws = workspace;
  } else {
    cudaError_t e = cudaMalloc(&p->ws, need);
    if (e != cudaSuccess) {
      delete p;
      return fail(PD_ERR_OOM, "cudaMalloc(%zu) failed: %s", need, cudaGetErrorString(e));
    }
    p->own_ws = true;
  }
  p->ws_bytes = need;
  layout(p, reinterpret_cast<unsigned char *>(p->ws));
  auto cleanup = [&](pd_status s) {
    paradiag_destroy(p);
    return s;
  };
  if (cudaMallocHost(&p->h_scal, pd::kScalWords * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&p->h_flags, pd::kFlagWords * sizeof(int)) != cudaSuccess)
    return cleanup(fail(PD_ERR_OOM, "cudaMallocHost failed"));
  std::memset(p->h_scal, 0, pd::kScalWords * sizeof(double));
  std::memset(p->h_flags, 0, pd::kFlagWords * sizeof(int));
  for (int i = 0; i < 3; ++i)
    if (cudaStreamCreateWithFlags(&p->cap[i], cudaStreamNonBlocking) != cudaSuccess)
      return cleanup(fail(PD_ERR_CUDA, "cudaStreamCreateWithFlags failed"));
  p->use_graphs = desc->no_graph ? 0 : 1;
  if (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess)
    return cleanup(fail(PD_ERR_CUDA, "cudaEventCreate failed"));

  // Algorithm 1, first step: pi_k = omega^k, gamma_k = omega^k / l; shifts s_k = 1 - pi_k;
  // half-spectrum weights w_k (1 for k = 0 and k = l/2, 2 otherwise).  Algorithm 3:
  // pi_k = alpha^{1/l} omega^k, the same gamma_k, D_alpha = diag(alpha^{j/l}), and the
  // inner system weighted by alpha^{1/l} (wga).
  const int nf = p->nf;
  const int64_t nt = p->nt;
  const double a = p->aroot;
  std::vector<double2> shift(nf), wg(nf), wga(nf);
  std::vector<cpx<float>> shift_f(nf), wg_f(nf);
  for (int k = 0; k < nf; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)nt;
    const double pr = std::cos(ang), pi_ = std::sin(ang);
    const double wk = (k == 0 || 2 * (int64_t)k == nt) ? 1.0 : 2.0;
    shift[k] = make_double2(1.0 - a * pr, -a * pi_);
    wg[k] = make_double2(wk * pr / (double)nt, wk * pi_ / (double)nt);
    wga[k] = make_double2(a * wg[k].x, a * wg[k].y);
    shift_f[k] = pd::mk<float>((float)shift[k].x, (float)shift[k].y);
    wg_f[k] = pd::mk<float>((float)wg[k].x, (float)wg[k].y);
  }
  std::vector<double> ts(nt), tsi(nt);
  std::vector<float> tsf(nt), tsif(nt);
  for (int64_t j = 0; j < nt; ++j) {
    ts[j] = std::pow(p->alpha, (double)j / (double)nt);
    tsi[j] = 1.0 / ts[j];
    tsf[j] = (float)ts[j];
    tsif[j] = (float)tsi[j];
  }
  const int ntw = std::max<int>(1, (int)(nt / 2));
  std::vector<cpx<double>> tw(ntw);
  std::vector<cpx<float>> twf(ntw);
  for (int k = 0; k < ntw; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)nt;
    tw[k] = pd::mk<double>(std::cos(ang), std::sin(ang));
    twf[k] = pd::mk<float>((float)tw[k].x, (float)tw[k].y);
  }
  cudaStream_t s = p->ctx.stream;
  if ((st = upload(p->shift, shift.data(), nf, s)) || (st = upload(p->wg, wg.data(), nf, s)) ||
      (st = upload(p->wga, wga.data(), nf, s)) || (st = upload(p->tw_d, tw.data(), ntw, s)) ||
      (st = upload(p->tw_f, twf.data(), ntw, s)) || (st = upload(p->ts_d, ts.data(), nt, s)) ||
      (st = upload(p->tsi_d, tsi.data(), nt, s)) || (st = upload(p->ts_f, tsf.data(), nt, s)) ||
      (st = upload(p->tsi_f, tsif.data(), nt, s)) || (st = upload(p->shift_f, shift_f.data(), nf, s)) ||
      (st = upload(p->wg_f, wg_f.data(), nf, s)))
    return cleanup(st);
  if (p->dim == 2) {
    const int N = (int)(2 * (p->nym + 1));
    std::vector<cpx<double>> ty(N / 2);
    std::vector<cpx<float>> tyf(N / 2);
    for (int k = 0; k < N / 2; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)N;
      ty[k] = pd::mk<double>(std::cos(ang), std::sin(ang));
      tyf[k] = pd::mk<float>((float)ty[k].x, (float)ty[k].y);
    }
    if ((st = upload(p->twy_d, ty.data(), N / 2, s)) || (st = upload(p->twy_f, tyf.data(), N / 2, s)))
      return cleanup(st);
  }
  if ((st = upload_operator(p, desc)) != PD_OK) return cleanup(st);
  if ((st = factorize(p)) != PD_OK) return cleanup(st);
  if (cudaMemsetAsync(p->flags, 0, pd::kFlagWords * sizeof(int), s) != cudaSuccess)
    return cleanup(fail(PD_ERR_CUDA, "plan upload failed"));
  if (cudaStreamSynchronize(s) != cudaSuccess) return cleanup(fail(PD_ERR_CUDA, "plan upload failed"));
  *out = p;
  return PD_OK;
}

pd_status paradiag_set_operator(pd_plan *p, const pd_desc *desc) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if ((st = validate(desc)) != PD_OK) return st;
  const int batch = desc->batch > 1 ? desc->batch : 1;
  const int64_t ny = desc->dim == 2 ? desc->ny : 1;
  if (desc->dim != p->dim || desc->nx != p->nxd || ny != p->nym || desc->nt != p->nt || batch != p->batch ||
      desc->precision != p->precision)
    return fail(PD_ERR_INVALID_ARG, "paradiag_set_operator: desc has a different shape or precision than the plan");
  if (desc->m_diag && !p->mass)
    return fail(PD_ERR_INVALID_ARG, "paradiag_set_operator: the plan was built without a mass matrix");
  if (batch == 1 && desc->tau != p->tau) {  // tau reaches some kernels by value: re-capture
    if (p->ctx.stream) cudaStreamSynchronize(p->ctx.stream);
    drop_graph(p);
    p->tau = desc->tau;
  }
  if (p->ctx.stream) cudaStreamSynchronize(p->ctx.stream);  // no solve may still read the old operator
  std::lock_guard<std::recursive_mutex> lk(host_mutex());
  const bool lane_before = p->lane;
  if ((st = upload_operator(p, desc)) != PD_OK) return st;
  if (p->lane != lane_before) drop_graph(p);  // the lane's arguments are captured in the graph
  if ((st = factorize(p)) != PD_OK) return st;
  if (p->ctx.stream && cudaStreamSynchronize(p->ctx.stream) != cudaSuccess)
    return fail(PD_ERR_CUDA, "operator factorisation failed");
  return PD_OK;
}

pd_status paradiag_destroy(pd_plan *p) {
  if (!p) return PD_OK;
  std::lock_guard<std::recursive_mutex> lk(host_mutex());
  if (p->ctx.stream) cudaStreamSynchronize(p->ctx.stream);
  drop_graph(p);
  for (int i = 0; i < 3; ++i)
    if (p->cap[i]) cudaStreamDestroy(p->cap[i]);
  p->ctx.release();
  if (p->own_ws && p->ws) cudaFree(p->ws);
  if (p->h_scal) cudaFreeHost(p->h_scal);
  if (p->h_flags) cudaFreeHost(p->h_flags);
  if (p->ev0) cudaEventDestroy(p->ev0);
  if (p->ev1) cudaEventDestroy(p->ev1);
  delete p;
  return PD_OK;
}

pd_status paradiag_solve(pd_plan *p, const double *G, double *U, pd_stats *stats) {
  cudaGetLastError();  // an error an earlier call of this thread left is not this call's
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (!G || !U) return fail(PD_ERR_INVALID_ARG, "G and U must be device pointers");
  if (((uintptr_t)G & 7) || ((uintptr_t)U & 7)) return fail(PD_ERR_INVALID_ARG, "G and U must be 8-byte aligned");
  const size_t bytes = (size_t)p->nt * p->nbar * sizeof(double);
  const char *g0 = reinterpret_cast<const char *>(G), *u0 = reinterpret_cast<const char *>(U);
  if (g0 < u0 + bytes && u0 < g0 + bytes) return fail(PD_ERR_INVALID_ARG, "U must not alias G");
  const int64_t l0 = p->ctx.launches;
  CK(cudaEventRecord(p->ev0, p->ctx.stream));
  pd_stats s{};
  const double *Gin = G;
  if (p->mass) {  // G' = M^{-1/2} G: the system for w = M^{1/2} u
    pd::launch_col_scale(p->ctx, G, p->Gm, p->nt, p->nbar, p->msc);
    Gin = p->Gm;
  }
  if (p->batch > 1) {  // every problem of the batch scaled to unit norm (exactly, by 2^k)
    pd::launch_batch_normalize(p->ctx, Gin, p->Gs, p->nt, p->batch, (int)p->nxm, p->bnc, p->bpart, p->bex, p->bzero);
    Gin = p->Gs;
    CK(cudaMemsetAsync(p->msw, 0, sizeof(int) * p->batch, p->ctx.stream));  // every problem starts here
  }
  st = p->precision == PD_FP64 ? solve_refined<double>(p, Gin, U, s) : solve_refined<float>(p, Gin, U, s);
  if (st == PD_ERR_CUDA) return st;
  if (p->batch > 1) pd::launch_batch_unscale(p->ctx, U, p->nt, p->batch, (int)p->nxm, p->bex, p->bnx, p->bzero);
  if (p->mass) pd::launch_col_scale(p->ctx, U, U, p->nt, p->nbar, p->msc);  // u = M^{-1/2} w
  CK(cudaEventRecord(p->ev1, p->ctx.stream));
  CK(cudaEventSynchronize(p->ev1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  s.ms_total = ms;
  s.kernel_launches = p->ctx.launches - l0;
  if (p->ctx.timing) p->ctx.collect();
  p->last = s;
  if (stats) *stats = s;
  pd_status cs = ctx_status(p);
  return cs != PD_OK ? cs : st;
}

pd_status paradiag_batch_advance(pd_plan *p, const double *G, double *U, const int32_t *join, int32_t steps,
                                 int32_t *state, pd_stats *stats) {
  cudaGetLastError();  // an error an earlier call of this thread left is not this call's
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (p->batch < 2) return fail(PD_ERR_INVALID_ARG, "paradiag_batch_advance needs a batched plan");
  if (p->loops || p->mass)
    return fail(PD_ERR_UNSUPPORTED, "paradiag_batch_advance: no fixed-loop variants or mass matrices");
  if (!G || !U || !join || !state) return fail(PD_ERR_INVALID_ARG, "G, U, join and state must not be NULL");
  if (((uintptr_t)G & 7) || ((uintptr_t)U & 7)) return fail(PD_ERR_INVALID_ARG, "G and U must be 8-byte aligned");
  if (steps < 1 || steps > 64) return fail(PD_ERR_INVALID_ARG, "steps must be in [1, 64] (got %d)", steps);
  const size_t bytes = (size_t)p->nt * p->nbar * sizeof(double);
  const char *g0 = reinterpret_cast<const char *>(G), *u0 = reinterpret_cast<const char *>(U);
  if (g0 < u0 + bytes && u0 < g0 + bytes) return fail(PD_ERR_INVALID_ARG, "U must not alias G");
  const int64_t l0 = p->ctx.launches;
  CK(cudaEventRecord(p->ev0, p->ctx.stream));
  CK(cudaMemcpyAsync(p->mjoin, join, sizeof(int32_t) * p->batch, cudaMemcpyHostToDevice, p->ctx.stream));
  pd::launch_batch_normalize(p->ctx, G, p->Gs, p->nt, p->batch, (int)p->nxm, p->bnc, p->bpart, p->bex, p->bzero);
  pd::launch_member_join(p->ctx, U, p->nt, p->batch, (int)p->nxm, p->bex, p->mjoin, p->bzero, p->msw, p->mprev,
                         p->mref2, p->mex, p->mconv);
  const int keep_max = p->max_refine;
  p->max_refine = steps - 1;         // this call's sweeps
  p->member_solves = keep_max + 1;   // each problem's own limit, counted over calls
  st = p->precision == PD_FP64 ? solve_continue<double>(p, p->Gs, U) : solve_continue<float>(p, p->Gs, U);
  p->max_refine = keep_max;
  p->member_solves = 0;
  if (st == PD_ERR_CUDA) return st;
  pd::launch_batch_unscale(p->ctx, U, p->nt, p->batch, (int)p->nxm, p->bex, p->bnx, p->bzero);
  CK(cudaMemcpyAsync(state, p->mconv, sizeof(int32_t) * p->batch, cudaMemcpyDeviceToHost, p->ctx.stream));
  CK(cudaEventRecord(p->ev1, p->ctx.stream));
  CK(cudaEventSynchronize(p->ev1));
  pd_stats s{};
  const int *f = p->h_flags;
  s.refine_sweeps = f[pd::F_SWEEP];
  s.krylov_iters_total = f[pd::F_MTOT];
  for (int i = 0; i < s.refine_sweeps && i < 16; ++i) {
    s.sweep_krylov_iters[i] = f[pd::F_SWM + i];
    s.sweep_krylov_rel_resnorm[i] = p->h_scal[pd::S_SWRES + i];
    s.sweep_rel_update[i] = p->h_scal[pd::S_SWUPD + i];
  }
  float ms = 0.f;
  cudaEventElapsedTime(&ms, p->ev0, p->ev1);
  s.ms_total = ms;
  s.kernel_launches = p->ctx.launches - l0;
  p->last = s;
  if (stats) *stats = s;
  if (st != PD_OK) return st;
  if (f[pd::F_NONFIN]) return fail(PD_ERR_NONFINITE, "non-finite value met (input contains NaN/Inf?)");
  return ctx_status(p);
}

pd_status paradiag_solve_host(pd_plan *p, const double *G_host, double *U_host, pd_stats *stats) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (!p->host_io) return fail(PD_ERR_INVALID_ARG, "plan was built without host_io staging");
  if (!G_host || !U_host) return fail(PD_ERR_INVALID_ARG, "G_host and U_host must be non-NULL");
  const size_t bytes = (size_t)p->nt * p->nbar * sizeof(double);
  CK(cudaMemcpyAsync(p->G_stage, G_host, bytes, cudaMemcpyHostToDevice, p->ctx.stream));
  if (p->batch <= 1 && !p->mass) {  // no kernel follows the graph: its final read can carry U back
    p->tail_dst = U_host;
    p->tail_src = p->U_stage;
    p->tail_bytes = bytes;
    p->tail_done = false;
  }
  st = paradiag_solve(p, p->G_stage, p->U_stage, stats);
  const bool done = p->tail_done;
  p->tail_dst = nullptr;
  p->tail_src = nullptr;
  p->tail_done = false;
  if (st != PD_OK && st != PD_ERR_NOT_CONVERGED) return st;
  if (!done) {
    CK(cudaMemcpyAsync(U_host, p->U_stage, bytes, cudaMemcpyDeviceToHost, p->ctx.stream));
    CK(cudaStreamSynchronize(p->ctx.stream));
  }
  return st;
}

pd_status paradiag_time_dft(pd_plan *p, const double *X, void *Xhat) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (!X || !Xhat) return fail(PD_ERR_INVALID_ARG, "NULL pointer");
  if (p->precision == PD_FP64)
    pd::launch_fft_r2c<double, double>(p->ctx, X, p->nbar, p->nbar, (int)p->nt, p->tw_d,
                                       reinterpret_cast<cpx<double> *>(Xhat), p->nbar);
  else
    pd::launch_fft_r2c<float, double>(p->ctx, X, p->nbar, p->nbar, (int)p->nt, p->tw_f,
                                      reinterpret_cast<cpx<float> *>(Xhat), p->nbar);
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
}

pd_status paradiag_time_idft(pd_plan *p, const void *Y, double *X) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (!X || !Y) return fail(PD_ERR_INVALID_ARG, "NULL pointer");
  int np = 0;
  if (p->precision == PD_FP64)
    pd::launch_fft_c2r<double>(p->ctx, reinterpret_cast<const cpx<double> *>(Y), p->nbar, p->nbar, (int)p->nt,
                               p->tw_d, X, p->nbar, 0, nullptr, &np);
  else
    pd::launch_fft_c2r<float>(p->ctx, reinterpret_cast<const cpx<float> *>(Y), p->nbar, p->nbar, (int)p->nt,
                              p->tw_f, X, p->nbar, 0, nullptr, &np);
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
}

pd_status paradiag_shifted_solve(pd_plan *p, const void *R, void *Y, double *b) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (!R) return fail(PD_ERR_INVALID_ARG, "R is NULL");
  if (p->precision == PD_FP64) {
    pd::PintArgs<double> a = base_args<double>(p);
    a.R = reinterpret_cast<const cpx<double> *>(R);
    a.ldr = p->nbar;
    a.Y = reinterpret_cast<cpx<double> *>(Y);
    a.ldy = p->nbar;
    if (b) {
      a.omega = p->wg;
      a.acc_part = p->acc_part;
    }
    pd::launch_pint<double>(p->ctx, p->geom, a);
  } else {
    pd::PintArgs<float> a = base_args<float>(p);
    a.k0_fp64 = 0;  // the stage entry point solves every frequency of arbitrary complex data in binary32
    a.R = reinterpret_cast<const cpx<float> *>(R);
    a.ldr = p->nbar;
    a.Y = reinterpret_cast<cpx<float> *>(Y);
    a.ldy = p->nbar;
    if (b) {
      a.omega = p->wg;
      a.acc_part = p->acc_part;
    }
    pd::launch_pint<float>(p->ctx, p->geom, a);
  }
  if (b) pd::launch_acc_reduce(p->ctx, p->geom, p->acc_part, b, nullptr);
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
}

pd_status paradiag_dst_y(pd_plan *p, const double *X, double *Y) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (p->dim != 2) return fail(PD_ERR_INVALID_ARG, "paradiag_dst_y needs a 2D plan");
  if (!X || !Y) return fail(PD_ERR_INVALID_ARG, "NULL pointer");
  pd::launch_dst_y<double, double, double>(p->ctx, X, Y, p->nt * p->batch, p->nym, p->nx, p->twy_d, 0);
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
}

pd_status paradiag_last_vectors(pd_plan *p, double *b, double *x) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  const double *src[2] = {p->b0, p->x0};
  double *dst[2] = {b, x};
  for (int i = 0; i < 2; ++i) {
    if (!dst[i]) continue;
    if (p->dim == 1) {
      CK(cudaMemcpyAsync(dst[i], src[i], sizeof(double) * p->nbar, cudaMemcpyDeviceToDevice, p->ctx.stream));
    } else {
      pd::launch_dst_y<double, double, double>(p->ctx, src[i], dst[i], p->batch, p->nym, p->nx, p->twy_d, 0);
    }
  }
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
}

pd_status paradiag_recip_f32(const float *x, float *r, int64_t n, void *stream) {
  if (n < 0) return fail(PD_ERR_INVALID_ARG, "n must be >= 0");
  if (n > 0 && (!x || !r)) return fail(PD_ERR_INVALID_ARG, "NULL pointer");
  if (n > ((int64_t)1 << 31) * 256) return fail(PD_ERR_UNSUPPORTED, "n too large");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  pd::launch_recip_f32(s, x, r, n);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return PD_OK;
}

pd_status paradiag_set_timing(pd_plan *p, int enable) {
  if (!p) return fail(PD_ERR_INVALID_ARG, "plan is NULL");
  if (p->ctx.stream) cudaStreamSynchronize(p->ctx.stream);
  p->ctx.collect();
  for (auto &f : p->ctx.fams) {
    f.launches = 0;
    f.ms = 0.0;
    f.bytes = 0.0;
  }
  p->ctx.timing = enable != 0;
  return PD_OK;
}

pd_status paradiag_kernel_times(pd_plan *p, pd_kernel_time *out, int max_entries, int *n_out) {
  if (!p) return fail(PD_ERR_INVALID_ARG, "plan is NULL");
  if (p->ctx.stream) cudaStreamSynchronize(p->ctx.stream);
  p->ctx.collect();
  int n = (int)p->ctx.fams.size();
  if (n_out) *n_out = n;
  for (int i = 0; i < n && i < max_entries && out; ++i) {
    std::memset(&out[i], 0, sizeof(pd_kernel_time));
    std::strncpy(out[i].name, p->ctx.fams[i].name.c_str(), sizeof(out[i].name) - 1);
    out[i].launches = p->ctx.fams[i].launches;
    out[i].total_ms = p->ctx.fams[i].ms;
    out[i].bytes = p->ctx.fams[i].bytes;
  }
  return PD_OK;
}

}  // extern "C"
