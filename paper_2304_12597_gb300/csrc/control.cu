// Device-side control of the solve: the stopping tests of Algorithm 2 (Sec. 3:
// ||r_m|| <= eps ||b|| or m = maxit, plus the stall and breakdown exits) and the
// refinement stopping rule run in single-thread kernels that write the control
// block and, inside a CUDA graph, set the conditional of the enclosing WHILE node.
// The same kernels run when the host drives the loops (it then reads the flags).
#include <cmath>

#include "pd_internal.h"

namespace pd {

__global__ void k_solve_reset(double *scal, int *flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < kFlagWords; ++i) flags[i] = 0;
  for (int i = 0; i < kScalWords; ++i) scal[i] = 0.0;
  scal[S_PREV] = 1.0;
}

// After an Algorithm-2 step: record ||r_m||, decide whether to continue.
__global__ void k_krylov_decide(double *scal, int *flags, KrylovCtl k, int use_handle,
                                cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = flags[F_M] + 1;
  const double res = scal[S_RES], beta = scal[S_BETA];
  if (m < 33) scal[S_HIST + m] = res;
  bool nonfinite = flags[F_NONFIN] || !isfinite(res);
  if (nonfinite) flags[F_NONFIN] = 1;
  const bool conv = flags[F_BREAK] || res <= k.eps * beta;
  const bool stall = m >= k.win + 1 && res <= k.stall_floor * beta && res > 0.5 * scal[S_HIST + m - k.win];
  const bool stop = nonfinite || conv || stall || m >= k.maxit;
  flags[F_M] = m;
  flags[F_KCONV] = conv ? 1 : 0;
  flags[F_KSTOP] = stop ? 1 : 0;
  if (use_handle) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// After a solve (first or refinement sweep) has produced ||delta_s||^2 in
// scal[S_D2]: record the sweep and decide whether another refinement sweep runs.
__global__ void k_refine_decide(double *scal, int *flags, RefineCtl r, int use_handle,
                                cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int s = flags[F_SWEEP];
  const double d2 = scal[S_D2];
  if (s == 0) scal[S_REF2] = d2;
  const double ref2 = scal[S_REF2];
  const double prev = scal[S_PREV];
  const double rel = ref2 > 0.0 ? sqrt(d2 / ref2) : 0.0;
  const double beta = scal[S_BETA];
  if (s < 16) {
    flags[F_SWM + s] = flags[F_M];
    scal[S_SWRES + s] = beta > 0.0 ? scal[S_RES] / beta : 0.0;
    scal[S_SWUPD + s] = rel;
    scal[S_SWBETA + s] = beta;
  }
  flags[F_MTOT] += flags[F_M];
  bool conv = false, stop = false;
  if (!isfinite(d2) || flags[F_NONFIN]) {
    flags[F_NONFIN] = 1;
    stop = true;
  } else if (ref2 == 0.0) {
    conv = stop = true;
  } else {
    const double eps = s == 0 ? r.eps_first : r.eps_refine;
    // FP64: Algorithm 2 met its tolerance, so this sweep's correction is exact to
    // working accuracy (s = 0: the paper's Algorithm 1 itself); a refinement sweep
    // leaves about eps * ||delta_s||.
    if (r.fp64 && flags[F_KCONV] && (s == 0 || eps * rel <= r.refine_tol)) conv = stop = true;
    // Refinement contracts the error by rho ~ ||delta_s|| / ||delta_{s-1}|| (s >= 2:
    // delta_1 / delta_0 is the first solve's error, not a contraction), so about
    // rho * ||delta_s|| remains after sweep s.
    if (!stop && s > 0) {
      const double rho = prev > 0.0 ? rel / prev : 0.0;
      if ((s >= 2 && rho * rel <= r.refine_tol && rel <= 1e-7) || rel <= 1e-15) {
        conv = stop = true;
      } else if (s > 1 && rho > 0.5) {  // no longer contracting: rounding floor reached
        conv = rel <= 1e-10;
        stop = true;
      }
    }
    if (!stop && s + 1 > r.max_refine) stop = true;
  }
  scal[S_PREV] = rel;
  scal[S_UPD] = rel;
  flags[F_SWEEP] = s + 1;
  flags[F_RCONV] = conv ? 1 : 0;
  flags[F_RSTOP] = stop ? 1 : 0;
  if (use_handle) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

void launch_solve_reset(Ctx &c, double *scal, int *flags) {
  c.launch("control", 0.0, [&] { k_solve_reset<<<1, 32, 0, c.stream>>>(scal, flags); });
}

void launch_krylov_decide(Ctx &c, double *scal, int *flags, const KrylovCtl &k, int use_handle,
                          cudaGraphConditionalHandle h) {
  c.launch("control", 0.0, [&] { k_krylov_decide<<<1, 32, 0, c.stream>>>(scal, flags, k, use_handle, h); });
}

void launch_refine_decide(Ctx &c, double *scal, int *flags, const RefineCtl &r, int use_handle,
                          cudaGraphConditionalHandle h) {
  c.launch("control", 0.0, [&] { k_refine_decide<<<1, 32, 0, c.stream>>>(scal, flags, r, use_handle, h); });
}

}  // namespace pd
