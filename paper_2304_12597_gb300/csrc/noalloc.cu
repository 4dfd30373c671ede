// paradiag_smw_rhs_noalloc: the first parallel-in-time loop and the SMW
// right-hand side b, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need this step:
// code running under a memory pool or arena that owns every byte of the device
// (so a stray allocation would break its accounting or fail outright), real-time
// loops where an allocation would stall or synchronise the device, and plugins
// whose host application forbids allocation after start-up.  They can hand us
// their input and output buffers, but not the scratch the parallel-in-time loop
// needs for its per-team partial sums.  This entry point therefore keeps that
// scratch in the file-scope __device__ array below: a fixed 4 MiB that every
// GPU which loads this library holds until the process exits.  Nothing here
// calls cudaMalloc, cudaFree or an allocating library routine.
//
// The array is shared by every call, so calls that overlap on the GPU (on
// different streams, or from different threads) race on it and must be
// serialised by the caller.  Each call writes every scratch word it later reads
// (coefficients, shifts, weights and every team's partial sums), so nothing has
// to be cleared between calls.
#include <cstdio>
#include <mutex>

#include "../../include/paradiag.h"
#include "pd_internal.h"

using pd::cpx;

namespace {

constexpr size_t kScratchBytes = (size_t)PD_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxN = 4096;                           // rows per tridiagonal system
constexpr int kMaxNf = 8192 / 2 + 1;                  // half-spectrum length for nt <= 8192
constexpr size_t kFixedBytes = 256 * 1024;            // shifts, weights and tau*K
constexpr size_t kAccDoubles = (kScratchBytes - kFixedBytes) / sizeof(double);
static_assert(2 * kMaxNf * sizeof(double2) + 3 * kMaxN * sizeof(double) <= kFixedBytes, "layout");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[128] = {};  // device address of g_scratch, per device ordinal

// 1 - pi_k and w_k gamma_k (Algorithm 1, first step), and tau K with the ignored
// end couplings zeroed, written into the scratch array.
__global__ void k_noalloc_coeffs(int nf, int64_t nt, int64_t n, double tau, const double *__restrict__ lo,
                                 const double *__restrict__ diag, const double *__restrict__ up, double2 *shift,
                                 double2 *wg, double *tlo, double *tdiag, double *tup) {
  pd::grid_dep_wait();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nf) {
    double s, c;
    sincospi(-2.0 * (double)i / (double)nt, &s, &c);  // pi_i = exp(-2 pi i / nt)
    const double wk = (i == 0 || 2 * i == nt) ? 1.0 : 2.0;
    shift[i] = make_double2(1.0 - c, -s);
    wg[i] = make_double2(wk * c / (double)nt, wk * s / (double)nt);
  }
  if (i < n) {
    tlo[i] = i > 0 ? tau * lo[i] : 0.0;
    tdiag[i] = tau * diag[i];
    tup[i] = i + 1 < n ? tau * up[i] : 0.0;
  }
}

pd_status reject(pd_status st, const char *fmt, long long a = 0, long long b = 0, int c = 0) {
  char msg[256];
  snprintf(msg, sizeof(msg), fmt, a, b, c);
  pd::set_last_error(msg);
  return st;
}

}  // namespace

extern "C" pd_status paradiag_smw_rhs_noalloc(int64_t nt, int64_t n, double tau, const double *k_lo,
                                              const double *k_diag, const double *k_up, const void *R, void *Y,
                                              double *b, void *stream) {
  if (nt < 1 || (nt & (nt - 1)) != 0 || nt > 8192 || n < 1 || n > kMaxN) {
    return reject(PD_ERR_UNSUPPORTED,
                  "paradiag_smw_rhs_noalloc: nt = %lld, n = %lld exceed the static scratch limits "
                  "(nt a power of two <= 8192, n <= %d)", (long long)nt, (long long)n, kMaxN);
  }
  if (!(tau > 0.0) || !k_lo || !k_diag || !k_up || !R || !b) {
    return reject(PD_ERR_INVALID_ARG, "paradiag_smw_rhs_noalloc: tau must be > 0 and K, R, b non-NULL");
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
    return reject(PD_ERR_CUDA, "paradiag_smw_rhs_noalloc: no usable current CUDA device");
  }
  void *base = nullptr;
  {
    // Set-up once per device, with that device current: the host-side symbol
    // g_scratch is only a stand-in, the kernels need its device address.
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) {
        char msg[256];
        snprintf(msg, sizeof(msg), "paradiag_smw_rhs_noalloc: cudaGetSymbolAddress failed: %s",
                 cudaGetErrorString(e));
        pd::set_last_error(msg);
        return PD_ERR_CUDA;
      }
      g_scratch_ptr[dev] = p;
    }
    base = g_scratch_ptr[dev];
  }
  unsigned char *sc = static_cast<unsigned char *>(base);
  const int nf = nt > 1 ? (int)(nt / 2 + 1) : 1;
  double2 *shift = reinterpret_cast<double2 *>(sc);
  double2 *wg = shift + kMaxNf;
  double *tlo = reinterpret_cast<double *>(wg + kMaxNf);
  double *tdiag = tlo + kMaxN;
  double *tup = tdiag + kMaxN;
  double *acc = reinterpret_cast<double *>(sc + kFixedBytes);

  pd::Ctx c;
  c.stream = static_cast<cudaStream_t>(stream);
  const int64_t cover = nf > n ? nf : n;
  c.launch("noalloc_coeffs", 0.0, [&] {
    pd::pdl_launch(c.pdl, k_noalloc_coeffs, dim3((unsigned)((cover + 255) / 256)), dim3(256), 0, c.stream, nf, nt, n, tau,
                 k_lo, k_diag, k_up,
                                                                            shift, wg, tlo, tdiag, tup);
  });
  pd::PintGeom g = pd::pint_geometry(nf, 1, (int)n, 4 * pd::sm_count(), 16);
  const int rmax = (int)(kAccDoubles / (size_t)n);
  if (g.R > rmax) g.R = rmax;
  pd::set_acc_rows(g);
  pd::PintArgs<double> a{};
  a.shift = shift;
  a.tlo = tlo;
  a.tdiag = tdiag;
  a.tup = tup;
  a.R = static_cast<const cpx<double> *>(R);
  a.ldr = n;
  a.Y = static_cast<cpx<double> *>(Y);
  a.ldy = n;
  a.omega = wg;
  a.acc_part = acc;
  pd::launch_pint<double>(c, g, a);
  pd::launch_acc_reduce(c, g, acc, b, nullptr);
  if (c.err != cudaSuccess) {
    char msg[256];
    snprintf(msg, sizeof(msg), "paradiag_smw_rhs_noalloc: launch failed in %s: %s", c.err_where,
             cudaGetErrorString(c.err));
    pd::set_last_error(msg);
    return PD_ERR_CUDA;
  }
  return PD_OK;
}
