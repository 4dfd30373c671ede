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
#include <string>
#include <vector>

#include "../../include/paradiag.h"
#include "pd_internal.h"

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
  int precision = PD_FP64;
  int maxit = 32;
  double eps = 1e-13;
  int max_refine = 6;
  double refine_tol = 1e-13;
  int host_io = 0;
  bool own_ws = false;
  void *ws = nullptr;
  size_t ws_bytes = 0;

  int nblk = 1, blen = 0;
  pd::PintGeom geom{};
  int blas_grid = 1, k5_grid = 1;
  int64_t lds = 0;

  // device buffers
  double2 *shift = nullptr, *wg = nullptr;
  double *klo = nullptr, *kdiag = nullptr, *kup = nullptr;
  double *tlo_d = nullptr, *tdiag_d = nullptr, *tup_d = nullptr;
  float *tlo_f = nullptr, *tdiag_f = nullptr, *tup_f = nullptr;
  double *xlo = nullptr, *xdiag = nullptr, *xup = nullptr, *ylo = nullptr, *ydiag = nullptr, *yup = nullptr;
  cpx<double> *tw_d = nullptr, *twy_d = nullptr;
  cpx<float> *tw_f = nullptr, *twy_f = nullptr;
  void *spec = nullptr;
  double *V = nullptr, *T = nullptr, *w = nullptr, *part = nullptr, *scal = nullptr;
  float *Vf = nullptr, *xf = nullptr;  // binary32 copies of V and x_m (mixed precision)
  int *flags = nullptr;
  double *b = nullptr, *z = nullptr, *x = nullptr, *y = nullptr;
  double *b0 = nullptr, *x0 = nullptr;  // b and x_m of the first solve (for paradiag_last_vectors)
  double *acc_part = nullptr;
  double2 *gpart = nullptr, *srow = nullptr, *omega = nullptr;
  double *msys_part = nullptr;
  double *norm_part = nullptr;
  float *res_f = nullptr, *tmp_f = nullptr;
  double *res_d = nullptr, *tmp_d = nullptr;
  double *G_stage = nullptr, *U_stage = nullptr;
  // pinned host mirrors of the scalar and flag blocks
  double *h_scal = nullptr;
  int *h_flags = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  pd_stats last{};
};

namespace {

// Host copies of the operator in the solve basis.
struct HostOp {
  std::vector<double> lo, diag, up;  // K~ (length nbar), block-decoupled
  std::vector<double> xlo, xdiag, xup, ylo, ydiag, yup;
};

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
  if (d->q != 0 && d->q != 1) return fail(PD_ERR_UNSUPPORTED, "only q = 1 (residual check every iteration) is built");
  if (d->alpha != 0.0 && d->alpha != 1.0) return fail(PD_ERR_UNSUPPORTED, "only alpha = 1 (Algorithm 1) is built");
  if (d->eps_krylov < 0.0 || d->refine_tol < 0.0 || d->max_refine < 0)
    return fail(PD_ERR_INVALID_ARG, "negative tolerance or sweep count");
  const int64_t blen = d->nx;
  if (blen > 4096) return fail(PD_ERR_UNSUPPORTED, "tridiagonal blocks longer than 4096 rows are not built");
  if (d->dim == 2) {
    if (!d->k_lo_y || !d->k_diag_y || !d->k_up_y) return fail(PD_ERR_INVALID_ARG, "T_y arrays are NULL");
    if (!is_pow2(d->ny + 1) || d->ny + 1 > 4096)
      return fail(PD_ERR_UNSUPPORTED, "2D needs ny + 1 to be a power of two <= 4096 (DST-I by FFT)");
    const double dd = d->k_diag_y[0];
    const double c = d->ny > 1 ? d->k_up_y[0] : 0.0;
    const double tol = 1e-12 * (std::fabs(dd) + std::fabs(c));
    for (int64_t i = 0; i < d->ny; ++i) {
      if (std::fabs(d->k_diag_y[i] - dd) > tol) return fail(PD_ERR_UNSUPPORTED, "T_y must be Toeplitz");
      if (i + 1 < d->ny && (std::fabs(d->k_up_y[i] - c) > tol || std::fabs(d->k_lo_y[i + 1] - c) > tol))
        return fail(PD_ERR_UNSUPPORTED, "T_y must be symmetric Toeplitz");
    }
  }
  const int64_t nbar = d->nx * (d->dim == 2 ? d->ny : 1);
  if (nbar > (int64_t)1 << 28 || d->nt * nbar > (int64_t)1 << 34)
    return fail(PD_ERR_UNSUPPORTED, "problem too large for this build");
  return PD_OK;
}

void fill_geometry(pd_plan *p, const pd_desc *d) {
  p->dim = d->dim;
  p->nx = d->nx;
  p->ny = d->dim == 2 ? d->ny : 1;
  p->nbar = p->nx * p->ny;
  p->nt = d->nt;
  p->nf = (int)(d->nt / 2 + 1);
  if (d->nt == 1) p->nf = 1;
  p->tau = d->tau;
  p->precision = d->precision;
  p->maxit = d->maxit ? d->maxit : 32;
  p->eps = d->eps_krylov > 0 ? d->eps_krylov : (d->precision == PD_FP64 ? 1e-13 : 1e-5);
  p->max_refine = d->max_refine ? d->max_refine : 8;
  p->refine_tol = d->refine_tol > 0 ? d->refine_tol : (d->precision == PD_FP64 ? 1e-14 : 1e-11);
  p->host_io = d->host_io;
  p->nblk = (int)p->ny;
  p->blen = (int)p->nx;
  p->lds = (p->nbar + 31) / 32 * 32;
  const int sms = pd::sm_count();
  const int esz = d->precision == PD_FP64 ? 16 : 8;
  pd::PintGeom g0 = pd::pint_geometry(p->nf, p->nblk, p->blen, 1, esz);
  // one wave of resident teams: occupancy estimated from shared memory and threads
  const size_t team_bytes = (size_t)g0.P * (g0.M + 1) * esz + (size_t)2 * g0.P * 5 * esz + (size_t)g0.P * g0.M * 8 +
                            (size_t)(g0.P / 32) * 33 * 16;
  const size_t cta_bytes = team_bytes * g0.teams_per_cta;
  int by_smem = (int)std::max<size_t>(1, (228 * 1024) / (cta_bytes + 1024));
  int by_threads = std::max(1, 2048 / (g0.P * g0.teams_per_cta));
  const int ctas_per_sm = std::max(1, std::min(by_smem, by_threads));
  const int target = sms * ctas_per_sm * g0.teams_per_cta;
  p->geom = pd::pint_geometry(p->nf, p->nblk, p->blen, target, esz);
  // cooperative Krylov kernels: at most one 256-thread CTA per SM (always co-resident)
  p->blas_grid = (int)std::max<int64_t>(1, std::min<int64_t>((p->nbar + 255) / 256, (int64_t)sms));
  // capacitance terms: a few frequencies per warp keeps the partial reduction short
  p->k5_grid = std::max(1, std::min((p->nf + 15) / 16, 64));
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
  p->xlo = A.take<double>(p->nx);
  p->xdiag = A.take<double>(p->nx);
  p->xup = A.take<double>(p->nx);
  if (p->dim == 2) {
    p->ylo = A.take<double>(p->ny);
    p->ydiag = A.take<double>(p->ny);
    p->yup = A.take<double>(p->ny);
  }
  const int ntw = std::max<int>(1, (int)(nt / 2));
  p->tw_d = A.take<cpx<double>>(ntw);
  if (mixed) p->tw_f = A.take<cpx<float>>(ntw);
  if (p->dim == 2) {
    p->twy_d = A.take<cpx<double>>(p->ny + 1);
    if (mixed) p->twy_f = A.take<cpx<float>>(p->ny + 1);
  }
  p->spec = mixed ? (void *)A.take<cpx<float>>((size_t)nf * p->lds) : (void *)A.take<cpx<double>>((size_t)nf * p->lds);
  p->V = A.take<double>((size_t)(mx + 1) * nbar);
  if (mixed) {
    p->Vf = A.take<float>((size_t)(mx + 1) * nbar);
    p->xf = A.take<float>(nbar);
  }
  p->T = A.take<double>((size_t)(mx + 1) * mx);
  p->w = A.take<double>(nbar);
  p->part = A.take<double>((size_t)3 * p->blas_grid * (mx + 2));
  p->scal = A.take<double>(16);
  p->flags = A.take<int>(16);
  p->b = A.take<double>(nbar);
  p->z = A.take<double>(nbar);
  p->x = A.take<double>(nbar);
  p->b0 = A.take<double>(nbar);
  p->x0 = A.take<double>(nbar);
  p->y = A.take<double>(mx + 1);
  p->acc_part = A.take<double>((size_t)p->geom.nblk * p->geom.R * p->geom.blen);
  p->gpart = A.take<double2>((size_t)nf * p->nblk * mx);
  p->srow = A.take<double2>((size_t)nf * mx);
  p->omega = A.take<double2>(nf);
  p->msys_part = A.take<double>((size_t)p->k5_grid * mx * mx);
  p->norm_part = A.take<double>((size_t)std::max<int64_t>(nbar / 2 + 2, 8 * (int64_t)pd::sm_count()));
  if (mixed) p->res_f = A.take<float>((size_t)nt * nbar);
  if (mixed && p->dim == 2) p->tmp_f = A.take<float>((size_t)nt * nbar);
  if (!mixed) p->res_d = A.take<double>((size_t)nt * nbar);
  if (!mixed && p->dim == 2) p->tmp_d = A.take<double>((size_t)nt * nbar);
  if (p->host_io) {
    p->G_stage = A.take<double>((size_t)nt * nbar);
    p->U_stage = A.take<double>((size_t)nt * nbar);
  }
  return (A.off + 255) & ~(size_t)255;
}

HostOp build_operator(const pd_desc *d) {
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

pd_status ctx_status(pd_plan *p) {
  if (p->ctx.err != cudaSuccess)
    return fail(PD_ERR_CUDA, "kernel launch failed in %s: %s", p->ctx.err_where, cudaGetErrorString(p->ctx.err));
  return PD_OK;
}

pd_status sync_read(pd_plan *p) {
  CK(cudaMemcpyAsync(p->h_scal, p->scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, p->ctx.stream));
  CK(cudaMemcpyAsync(p->h_flags, p->flags, 16 * sizeof(int), cudaMemcpyDeviceToHost, p->ctx.stream));
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
}

template <typename T>
const cpx<T> *time_tw(pd_plan *p);
template <>
const cpx<double> *time_tw<double>(pd_plan *p) { return p->tw_d; }
template <>
const cpx<float> *time_tw<float>(pd_plan *p) { return p->tw_f; }

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
  a.shift = p->shift;
  a.tlo = p->tlo_d;
  a.tdiag = p->tdiag_d;
  a.tup = p->tup_d;
  return a;
}
template <>
pd::PintArgs<float> base_args<float>(pd_plan *p) {
  pd::PintArgs<float> a{};
  a.shift = p->shift;
  a.tlo = p->tlo_f;
  a.tdiag = p->tdiag_f;
  a.tup = p->tup_f;
  return a;
}

struct SolveInfo {
  int m = 0;
  int pint_loops = 0;
  int sweeps_exec = 0;
  bool breakdown = false;
  bool converged = true;
  double beta = 0.0;
  double rel_res = 0.0;
};

// Algorithm 1 in the solve basis on real input X (nt, nbar); the result is
// written by the inverse DFT in `out_mode` (0 store double, 1 add double,
// 2 store float) and ||result||_F^2 is left in scal[4].
template <typename T, typename Tin>
pd_status run_paradiag(pd_plan *p, const Tin *X, void *out, int out_mode, SolveInfo &info, double eps,
                       double stall_floor) {
  pd::Ctx &c = p->ctx;
  cpx<T> *S = reinterpret_cast<cpx<T> *>(p->spec);
  const int nt = (int)p->nt;
  // forward DFT along time: rows of G F^T (eq. 5)
  pd::launch_fft_r2c<T, Tin>(c, X, p->nbar, p->nbar, nt, time_tw<T>(p), S, p->lds);
  // first parallel-in-time loop and b = L F^{-T} e_l (eq. 7)
  {
    pd::PintArgs<T> a = base_args<T>(p);
    a.R = S;
    a.ldr = p->lds;
    a.omega = p->wg;
    a.acc_part = p->acc_part;
    pd::launch_pint<T>(c, p->geom, a);
    pd::launch_acc_reduce(c, p->geom, p->acc_part, p->b, nullptr);
  }
  info.pint_loops += 1;
  info.sweeps_exec += 1;
  // Algorithm 2 on J_l x = b (eq. 8)
  pd::KrylovBufs kb{(int)p->nbar, p->maxit, p->klo, p->kdiag, p->kup, p->V, sizeof(T) == 4 ? p->Vf : nullptr,
                    p->T, p->w, p->part, p->blas_grid, p->scal, p->flags};
  CK(cudaMemsetAsync(p->T, 0, sizeof(double) * (p->maxit + 1) * p->maxit, c.stream));
  pd::launch_vec_norm_init(c, kb, p->b);
  pd_status st = sync_read(p);
  if (st != PD_OK) return st;
  const double beta = p->h_scal[0];
  info.beta = beta;
  info.m = 0;
  info.breakdown = false;
  if (!std::isfinite(beta) || p->h_flags[2]) return fail(PD_ERR_NONFINITE, "non-finite ||b|| (input contains NaN/Inf?)");
  int m = 0;
  double res = beta;
  double hist[40];
  hist[0] = beta;
  // Algorithm 2 stops at eps * beta or maxit (Sec. 3), and here also once the eq. (13)
  // residual stops halving: in binary32 it levels off at the rounding-noise floor of
  // the shifted solves, and in FP64 the polynomial space K_m(K, b) can stall for
  // many steps when J_l is far from I.  The refinement sweeps recover the rest.
  // Window: 1 iteration in binary32 (the floor is flat), 3 in FP64 (FOM residuals
  // are not monotone, so a single non-halving step is not yet a stall).  The stall
  // exit only applies once ||r|| <= stall_floor * beta: above it a slow phase is
  // convergence, not noise.
  const int win = p->precision == PD_MIXED ? 1 : 3;
  if (beta > 0.0) {
    while (res > eps * beta && m < p->maxit) {
      if (m >= win + 1 && res <= stall_floor * beta && res > 0.5 * hist[m - win]) break;
      ++m;
      pd::launch_arnoldi(c, kb, m);
      // h_k = ((1 - pi_k) I + tau K)^{-1} v_{m+1} and g_k = V_m^T h_k
      {
        pd::PintArgs<T> a = base_args<T>(p);
        a.rvec = vbasis<T>(p) + (size_t)m * p->nbar;
        a.V = vbasis<T>(p);
        a.ldv = p->nbar;
        a.mdots = m;
        a.gpart = p->gpart;
        a.skip_flag = p->flags;
        pd::launch_pint<T>(c, p->geom, a);
      }
      pd::launch_capacitance(c, kb, m, p->nf, p->tau, p->shift, p->wg, p->gpart, p->nblk, p->msys_part, p->k5_grid,
                             p->srow, p->omega, p->y);
      // z = sum_i gamma_i h_i (e_m^T S_i y_m), then eq. (13)
      {
        pd::PintArgs<T> a = base_args<T>(p);
        a.rvec = vbasis<T>(p) + (size_t)m * p->nbar;
        a.omega = p->omega;
        a.acc_part = p->acc_part;
        a.skip_flag = p->flags;
        pd::launch_pint<T>(c, p->geom, a);
        pd::launch_acc_reduce(c, p->geom, p->acc_part, p->z, p->flags);
      }
      info.sweeps_exec += 2;
      info.pint_loops += 1;
      pd::launch_project_resnorm(c, kb, m, p->z, p->tau);
      st = sync_read(p);
      if (st != PD_OK) return st;
      res = p->h_scal[2];
      hist[m] = res;
      if (p->h_flags[2] || !std::isfinite(res)) return fail(PD_ERR_NONFINITE, "non-finite value in Algorithm 2");
      if (p->h_flags[0]) {
        info.breakdown = true;
        break;
      }
    }
    pd::launch_xm(c, kb, m, p->y, p->x, sizeof(T) == 4 ? p->xf : nullptr);
  } else {
    CK(cudaMemsetAsync(p->x, 0, sizeof(double) * p->nbar, c.stream));
    if (p->xf) CK(cudaMemsetAsync(p->xf, 0, sizeof(float) * p->nbar, c.stream));
  }
  info.m = m;
  info.rel_res = beta > 0 ? res / beta : 0.0;
  info.converged = (beta == 0.0) || info.breakdown || res <= eps * beta;
  // final parallel-in-time loop: Y_k = A_k^{-1} (G^_k - x_m), i.e. L - W fused
  {
    pd::PintArgs<T> a = base_args<T>(p);
    a.R = S;
    a.ldr = p->lds;
    a.rvec = xvec<T>(p);
    a.Y = S;
    a.ldy = p->lds;
    pd::launch_pint<T>(c, p->geom, a);
  }
  info.pint_loops += 1;
  info.sweeps_exec += 1;
  // U = (L - W) F^{-T}
  int nparts = 0;
  pd::launch_fft_c2r<T>(c, S, p->lds, p->nbar, nt, time_tw<T>(p), out, p->nbar, out_mode, p->norm_part, &nparts);
  pd::launch_sumsq(c, p->norm_part, nparts, p->scal + 4);
  return ctx_status(p);
}

template <typename T>
T *res_buf(pd_plan *p);
template <>
double *res_buf<double>(pd_plan *p) { return p->res_d; }
template <>
float *res_buf<float>(pd_plan *p) { return p->res_f; }
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

// Iterative refinement around Algorithm 1 on the all-at-once residual.
// Sweep 0 solves eq. (2) for G; sweep s >= 1 solves it for the FP64 residual
// G - [(I + tau K) U - U Sigma_1^T] and adds the correction to U (FP64).
// If Algorithm 2 stops with ||r_m|| > 0, the U it produces satisfies eq. (2)
// up to exactly -r_m in the first time step (its last slice is x_m - r_m while
// the correction used x_m), so a sweep on that residual corrects precisely the
// Krylov error.  T = compute type of the FFTs and shifted solves (double for
// PD_FP64, float for PD_MIXED); residuals are stored in T.
template <typename T>
pd_status solve_refined(pd_plan *p, const double *G, double *U, pd_stats &s) {
  const bool fp64 = sizeof(T) == 8;
  const int out_mode_2d = fp64 ? 0 : 2;  // inverse DFT into the 2D temporary buffer
  T *res = res_buf<T>(p);
  T *tmp = tmp_buf<T>(p);
  double ref2 = 0.0, rel_update = 1.0;
  int total_m = 0, loops = 0, execs = 0, sweeps = 0;
  SolveInfo info;
  bool conv = false;
  for (int sweep = 0; sweep <= p->max_refine; ++sweep) {
    SolveInfo si;
    pd_status st;
    // A binary32 refinement sweep contracts the error by ~1e-3 at best (rounding
    // noise of the residual, amplified by the solution operator), so its inner
    // Algorithm 2 needs no more than that; the first solve uses eps_krylov.
    // FP64 refinement sweeps (only after Algorithm 2 stalled) ask for 1e-8: the error
    // they leave is about that times their (already small) update.
    const double eps = sweep == 0 ? p->eps : std::max(p->eps, fp64 ? 1e-8 : 1e-3);
    // Stall exit: FP64 near its floor (1e-6 beta); binary32 first solve once below
    // 1e-3 beta; binary32 refinement sweeps at any level (their residuals are
    // rounding noise and the eq. (13) estimate levels off at 1e-3..1e-2).
    const double stall_floor = fp64 ? 1e-6 : (sweep == 0 ? 1e-3 : 1.0);
    if (sweep == 0) {
      if (p->dim == 1) {
        st = run_paradiag<T, double>(p, G, U, 0, si, eps, stall_floor);
      } else {
        pd::launch_dst_y<double, T, T>(p->ctx, G, tmp, p->nt, p->ny, p->nx, dst_tw<T>(p), 0);
        st = run_paradiag<T, T>(p, tmp, tmp, out_mode_2d, si, eps, stall_floor);
        if (st == PD_OK) pd::launch_dst_y<T, double, T>(p->ctx, tmp, U, p->nt, p->ny, p->nx, dst_tw<T>(p), 0);
      }
    } else {
      int np = 0;
      pd::launch_residual<T>(p->ctx, G, U, res, p->nt, p->ny, p->nx, p->tau, p->xlo, p->xdiag, p->xup, p->ylo,
                             p->ydiag, p->yup, nullptr, &np);
      if (p->dim == 1) {
        st = run_paradiag<T, T>(p, res, U, 1, si, eps, stall_floor);
      } else {
        pd::launch_dst_y<T, T, T>(p->ctx, res, tmp, p->nt, p->ny, p->nx, dst_tw<T>(p), 0);
        st = run_paradiag<T, T>(p, tmp, tmp, out_mode_2d, si, eps, stall_floor);
        if (st == PD_OK) pd::launch_dst_y<T, double, T>(p->ctx, tmp, U, p->nt, p->ny, p->nx, dst_tw<T>(p), 1);
      }
    }
    if (st != PD_OK) return st;
    if (sweep == 0) {
      CK(cudaMemcpyAsync(p->b0, p->b, sizeof(double) * p->nbar, cudaMemcpyDeviceToDevice, p->ctx.stream));
      CK(cudaMemcpyAsync(p->x0, p->x, sizeof(double) * p->nbar, cudaMemcpyDeviceToDevice, p->ctx.stream));
    }
    st = sync_read(p);
    if (st != PD_OK) return st;
    const double d2 = p->h_scal[4];
    if (!std::isfinite(d2)) return fail(PD_ERR_NONFINITE, "non-finite update in refinement sweep %d", sweep);
    if (sweeps < 16) {
      s.sweep_krylov_iters[sweeps] = si.m;
      s.sweep_rel_update[sweeps] = ref2 > 0 || sweep == 0 ? (sweep == 0 ? 1.0 : std::sqrt(d2 / ref2)) : 0.0;
      s.sweep_krylov_rel_resnorm[sweeps] = si.rel_res;
    }
    ++sweeps;
    total_m += si.m;
    loops += si.pint_loops;
    execs += si.sweeps_exec;
    info = si;
    if (sweep == 0) ref2 = d2;
    const double prev_update = rel_update;
    rel_update = ref2 > 0 ? std::sqrt(d2 / ref2) : 0.0;
    if (ref2 == 0.0) {
      conv = true;
      break;
    }
    // FP64: Algorithm 2 met its tolerance, so this sweep's correction is exact to
    // working accuracy (sweep 0: the paper's Algorithm 1 itself); a refinement sweep
    // leaves about eps * ||delta_s||.
    if (fp64 && si.converged && (sweep == 0 || eps * rel_update <= p->refine_tol)) {
      conv = true;
      break;
    }
    // Each refinement sweep contracts the error by rho ~ ||delta_s|| / ||delta_{s-1}||
    // (s >= 2: delta_1 / delta_0 is the first solve's error, not a contraction), so
    // the error left after sweep s is about rho * ||delta_s||: stop once that
    // predicted remainder (relative to ||U|| ~ ||delta_0||) is below refine_tol and
    // the last update itself is small.
    if (sweep > 0) {
      const double rho = prev_update > 0 ? rel_update / prev_update : 0.0;
      if ((sweep >= 2 && rho * rel_update <= p->refine_tol && rel_update <= 1e-7) || rel_update <= 1e-15) {
        conv = true;
        break;
      }
      // No longer contracting: the rounding floor of the residual is reached.
      if (sweep > 1 && rho > 0.5) {
        conv = rel_update <= 1e-10;
        break;
      }
    }
  }
  s.krylov_iters = info.m;
  s.krylov_iters_total = total_m;
  s.pint_loops = loops;
  s.shifted_sweeps = execs;
  s.refine_sweeps = sweeps;
  s.breakdown = info.breakdown;
  s.beta = info.beta;
  s.krylov_rel_resnorm = info.rel_res;
  s.rel_update = sweeps > 1 ? rel_update : 0.0;
  return conv ? PD_OK : fail(PD_ERR_NOT_CONVERGED, "refinement did not reach refine_tol in %d sweeps", sweeps);
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
  if (cudaMallocHost(&p->h_scal, 16 * sizeof(double)) != cudaSuccess ||
      cudaMallocHost(&p->h_flags, 16 * sizeof(int)) != cudaSuccess)
    return cleanup(fail(PD_ERR_OOM, "cudaMallocHost failed"));
  if (cudaEventCreate(&p->ev0) != cudaSuccess || cudaEventCreate(&p->ev1) != cudaSuccess)
    return cleanup(fail(PD_ERR_CUDA, "cudaEventCreate failed"));

  // Algorithm 1, first step: pi_k = omega^k, gamma_k = pi_k / l; shifts s_k = 1 - pi_k;
  // half-spectrum weights w_k (1 for k = 0 and k = l/2, 2 otherwise).
  const int nf = p->nf;
  const int64_t nt = p->nt;
  std::vector<double2> shift(nf), wg(nf);
  for (int k = 0; k < nf; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)nt;
    const double pr = std::cos(ang), pi_ = std::sin(ang);
    const double wk = (k == 0 || 2 * (int64_t)k == nt) ? 1.0 : 2.0;
    shift[k] = make_double2(1.0 - pr, -pi_);
    wg[k] = make_double2(wk * pr / (double)nt, wk * pi_ / (double)nt);
  }
  const int ntw = std::max<int>(1, (int)(nt / 2));
  std::vector<cpx<double>> tw(ntw);
  std::vector<cpx<float>> twf(ntw);
  for (int k = 0; k < ntw; ++k) {
    const double ang = -2.0 * M_PI * (double)k / (double)nt;
    tw[k] = pd::mk<double>(std::cos(ang), std::sin(ang));
    twf[k] = pd::mk<float>((float)tw[k].x, (float)tw[k].y);
  }
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
  cudaStream_t s = p->ctx.stream;
  if ((st = upload(p->shift, shift.data(), nf, s)) || (st = upload(p->wg, wg.data(), nf, s)) ||
      (st = upload(p->klo, h.lo.data(), nbar, s)) || (st = upload(p->kdiag, h.diag.data(), nbar, s)) ||
      (st = upload(p->kup, h.up.data(), nbar, s)) || (st = upload(p->tlo_d, tlo.data(), nbar, s)) ||
      (st = upload(p->tdiag_d, tdiag.data(), nbar, s)) || (st = upload(p->tup_d, tup.data(), nbar, s)) ||
      (st = upload(p->tlo_f, flo.data(), nbar, s)) || (st = upload(p->tdiag_f, fdiag.data(), nbar, s)) ||
      (st = upload(p->tup_f, fup.data(), nbar, s)) || (st = upload(p->xlo, h.xlo.data(), p->nx, s)) ||
      (st = upload(p->xdiag, h.xdiag.data(), p->nx, s)) || (st = upload(p->xup, h.xup.data(), p->nx, s)) ||
      (st = upload(p->tw_d, tw.data(), ntw, s)) || (st = upload(p->tw_f, twf.data(), ntw, s)))
    return cleanup(st);
  if (p->dim == 2) {
    const int N = (int)(2 * (p->ny + 1));
    std::vector<cpx<double>> ty(N / 2);
    std::vector<cpx<float>> tyf(N / 2);
    for (int k = 0; k < N / 2; ++k) {
      const double ang = -2.0 * M_PI * (double)k / (double)N;
      ty[k] = pd::mk<double>(std::cos(ang), std::sin(ang));
      tyf[k] = pd::mk<float>((float)ty[k].x, (float)ty[k].y);
    }
    if ((st = upload(p->ylo, h.ylo.data(), p->ny, s)) || (st = upload(p->ydiag, h.ydiag.data(), p->ny, s)) ||
        (st = upload(p->yup, h.yup.data(), p->ny, s)) || (st = upload(p->twy_d, ty.data(), N / 2, s)) ||
        (st = upload(p->twy_f, tyf.data(), N / 2, s)))
      return cleanup(st);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return cleanup(fail(PD_ERR_CUDA, "plan upload failed"));
  *out = p;
  return PD_OK;
}

pd_status paradiag_destroy(pd_plan *p) {
  if (!p) return PD_OK;
  if (p->ctx.stream) cudaStreamSynchronize(p->ctx.stream);
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
  st = p->precision == PD_FP64 ? solve_refined<double>(p, G, U, s) : solve_refined<float>(p, G, U, s);
  if (st == PD_ERR_CUDA) return st;
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

pd_status paradiag_solve_host(pd_plan *p, const double *G_host, double *U_host, pd_stats *stats) {
  pd_status st = check_plan(p);
  if (st != PD_OK) return st;
  if (!p->host_io) return fail(PD_ERR_INVALID_ARG, "plan was built without host_io staging");
  if (!G_host || !U_host) return fail(PD_ERR_INVALID_ARG, "G_host and U_host must be non-NULL");
  const size_t bytes = (size_t)p->nt * p->nbar * sizeof(double);
  CK(cudaMemcpyAsync(p->G_stage, G_host, bytes, cudaMemcpyHostToDevice, p->ctx.stream));
  st = paradiag_solve(p, p->G_stage, p->U_stage, stats);
  if (st != PD_OK && st != PD_ERR_NOT_CONVERGED) return st;
  CK(cudaMemcpyAsync(U_host, p->U_stage, bytes, cudaMemcpyDeviceToHost, p->ctx.stream));
  CK(cudaStreamSynchronize(p->ctx.stream));
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
  pd::launch_dst_y<double, double, double>(p->ctx, X, Y, p->nt, p->ny, p->nx, p->twy_d, 0);
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
      pd::launch_dst_y<double, double, double>(p->ctx, src[i], dst[i], 1, p->ny, p->nx, p->twy_d, 0);
    }
  }
  CK(cudaStreamSynchronize(p->ctx.stream));
  return ctx_status(p);
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
