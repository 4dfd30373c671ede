// Device-side stopping logic of Algorithm 2 and of the refinement loop, shared
// by the kernels that finish a step (the eq. (13) projection, the inverse DFT).
// Internal header; single-thread functions, called by one thread of one CTA.
#pragma once

#include <cuda_runtime.h>

#include "pd_internal.h"

namespace pd {

// After an Algorithm-2 step (Sec. 3): record ||r_m||, decide whether to continue:
// stop at ||r_m|| <= eps ref, at maxit, at a breakdown, or at a stall near the
// precision floor (no halving over `win` checks once ||r_m|| <= stall_floor ref).
// ref = beta = ||b|| as in the paper; plans that refine (k.rrel) use ||R||_F, the norm of
// the solve's right-hand side (G, or the residual a refinement sweep corrects): the
// residual of eq. (2) a solve leaves behind is exactly -r_m in the first time step, so
// a sweep contracts by about ||r_m|| / ||R||.  Measured against beta this can fail both
// ways: for damped problems ||b|| (~ the final state) << ||R|| and the steps past
// eps ||R|| buy nothing; when J_l is ill-conditioned (Theorem 3.1: kappa up to
// 1 + 1/(tau lambda_min)) b lies along its large eigenvalues, ||b|| >> ||R||, and eps beta
// would leave ||r_m|| as large as the sweep's input.
// A frozen step (q > 1, flags[F_FROZEN]) has no residual: it only advances m.
__device__ __forceinline__ void krylov_decide(double *scal, int *flags, const KrylovCtl &k, int use_handle,
                                              cudaGraphConditionalHandle h) {
  const int m = flags[F_M] + 1;
  if (flags[F_FROZEN]) {
    flags[F_M] = m;
    flags[F_KCONV] = 0;
    flags[F_KSTOP] = 0;
    if (use_handle) cudaGraphSetConditional(h, 1u);
    return;
  }
  const double res = scal[S_RES], beta = scal[S_BETA];
  const double rn = scal[S_RNORM];
  const double ref = (k.rrel && rn > 0.0) ? rn : beta;
  if (m < 33) scal[S_HIST + m] = res;
  const bool nonfinite = flags[F_NONFIN] || !isfinite(res);
  if (nonfinite) flags[F_NONFIN] = 1;
  const bool conv = flags[F_BREAK] || res <= k.eps * ref;
  // checks are q steps apart (the last one may be closer: maxit or a breakdown)
  const int back = k.win * (k.q > 1 ? k.q : 1);
  const bool stall = m >= back + 1 && m % (k.q > 1 ? k.q : 1) == 0 && res <= k.stall_floor * ref &&
                     res > 0.5 * scal[S_HIST + m - back];
  const bool stop = nonfinite || conv || stall || m >= k.maxit;
  flags[F_M] = m;
  flags[F_KCONV] = conv ? 1 : 0;
  flags[F_KSTOP] = stop ? 1 : 0;
  if (use_handle) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// After a solve (first or refinement sweep) has produced ||delta_s||^2 in
// scal[S_D2]: record the sweep and decide whether another refinement sweep runs.
__device__ __forceinline__ void refine_decide(double *scal, int *flags, const RefineCtl &r, int use_handle,
                                              cudaGraphConditionalHandle h) {
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
  if (flags[F_TIMEOUT]) {  // a bounded wait of the persistent step ran out: stop
    stop = true;
  } else if (!isfinite(d2) || flags[F_NONFIN]) {
    flags[F_NONFIN] = 1;
    stop = true;
  } else if (ref2 == 0.0) {
    conv = stop = true;
  } else {
    const double eps = s == 0 ? r.eps_first : r.eps_refine;
    // FP64: Algorithm 2 met its tolerance.  With a tight tolerance the first solve is
    // exact to working accuracy (the paper's Algorithm 1 itself); otherwise each sweep
    // leaves about eps * ||delta_s|| (relative) behind.
    if (r.fp64 && flags[F_KCONV] && (s == 0 ? eps <= 1e-10 : eps * rel <= r.refine_tol)) conv = stop = true;
    // Refinement contracts the error by rho ~ ||delta_s|| / ||delta_{s-1}|| (s >= 2:
    // delta_1 / delta_0 is the first solve's error, not a contraction), so about
    // rho * ||delta_s|| remains after sweep s.  The contraction varies from sweep to sweep
    // (each sweep's Algorithm 2 stops at a different point), so the prediction takes the
    // larger of the last two ratios where there are two.
    if (!stop && s > 0) {
      const double rho = prev > 0.0 ? rel / prev : 0.0;
      const double pp = (s >= 3 && s < 16) ? scal[S_SWUPD + s - 2] : 0.0;
      const double rho_pred = pp > 0.0 ? fmax(rho, prev / pp) : rho;
      if ((s >= 2 && rho_pred * rel <= r.refine_tol && rel <= 1e-7) || rel <= 1e-15) {
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

// Batched plans: the same rule per problem.  d2[b] = ||delta_s||^2 of problem b,
// ref2[b] its ||delta_0||^2 (set at s = 0), prev[b] its previous relative update.
// Refinement stops when every problem meets the predicted-error rule (a problem with
// a zero first solve, or an all-zero right-hand side, is done), or when any problem stops
// contracting (then it has
// converged if every problem's update is at the rounding floor).  The recorded
// update of the sweep is the largest over the problems.  mex[b] receives the power of
// two that scales problem b's residual in the next sweep, 2^-round(log2 ||delta_s||):
// every problem's residual enters the binary32 DFTs and shifted solves, and its own
// Algorithm 2, near unit norm however far its earlier sweeps have shrunk it.
// Run by every thread of one CTA (red: blockDim.x doubles of shared memory): the
// problems are spread over the threads, so the per-problem loads overlap instead of
// following one another through L2; the batch totals are then reduced in a fixed order.
__device__ __forceinline__ void refine_decide_members(double *scal, int *flags, const RefineCtl &r, int nmem,
                                                      const double *d2, double *ref2, double *prev, int *mex,
                                                      const int *zero, int use_handle, cudaGraphConditionalHandle h,
                                                      double *red) {
  const int s = flags[F_SWEEP];
  bool nonfinite = flags[F_NONFIN] != 0, all_conv = true, any_stall = false, all_floor = true;
  double relmax = 0.0, d2sum = 0.0;
  for (int b = threadIdx.x; b < nmem; b += blockDim.x) {
    if (zero[b]) {  // an all-zero problem (an unused slot): solved exactly by U = 0
      ref2[b] = 0.0;
      prev[b] = 0.0;
      mex[b] = 0;
      if (r.msw) r.msw[b] = 0;
      if (r.mconv) r.mconv[b] = 0;
      continue;
    }
    const int sb = r.msw ? r.msw[b] : s;  // this problem's solves before this one
    const double d = d2[b];
    d2sum += d;
    if (!isfinite(d)) nonfinite = true;
    if (sb == 0) ref2[b] = d;
    const double rf = ref2[b];
    const double rel = rf > 0.0 ? sqrt(d / rf) : 0.0;
    bool conv_b = true;
    if (rf > 0.0) {
      relmax = fmax(relmax, rel);
      const double rho = prev[b] > 0.0 ? rel / prev[b] : 0.0;
      const bool floor_b = sb > 1 && rho > 0.5;  // no longer contracting: rounding floor
      conv_b = sb > 0 &&
               ((sb >= 2 && rho * rel <= r.refine_tol && rel <= 1e-7) || rel <= 1e-15 || (floor_b && rel <= 1e-10));
      if (!conv_b) all_conv = false;
      if (!conv_b && floor_b) any_stall = true;  // stuck above the floor
      if (rel > 1e-10) all_floor = false;
    }
    if (r.msw) r.msw[b] = sb + 1;
    if (r.mconv) r.mconv[b] = conv_b ? 1 : ((r.member_solves > 0 && sb + 1 >= r.member_solves) ? 2 : 0);
    prev[b] = rel;
    int e = 0;
    if (d > 0.0 && isfinite(d)) {
      int e2;
      frexp(d, &e2);  // ||delta_s|| ~ 2^(e2/2)
      e = max(-100, min(100, -(e2 / 2)));
    }
    mex[b] = e;
  }
  nonfinite = __syncthreads_or(nonfinite);
  all_conv = __syncthreads_and(all_conv);
  any_stall = __syncthreads_or(any_stall);
  all_floor = __syncthreads_and(all_floor);
  // relmax: a maximum (order-free); d2sum: a fixed-order tree over the threads
  red[threadIdx.x] = relmax;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  relmax = red[0];
  __syncthreads();
  red[threadIdx.x] = d2sum;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  d2sum = red[0];
  if (threadIdx.x != 0) return;
  const double beta = scal[S_BETA];
  if (s < 16) {
    flags[F_SWM + s] = flags[F_M];
    scal[S_SWRES + s] = beta > 0.0 ? scal[S_RES] / beta : 0.0;
    scal[S_SWUPD + s] = s == 0 ? 1.0 : relmax;
    scal[S_SWBETA + s] = beta;
  }
  flags[F_MTOT] += flags[F_M];
  bool conv = false, stop = false;
  if (nonfinite) {
    flags[F_NONFIN] = 1;
    stop = true;
  } else if (r.fp64 && flags[F_KCONV] && (s == 0 ? r.eps_first <= 1e-10 : r.eps_refine * relmax <= r.refine_tol)) {
    // FP64, every problem's Algorithm 2 met its tolerance (as for a single problem)
    conv = stop = true;
  } else if (all_conv && (s > 0 || relmax == 0.0)) {
    conv = stop = true;
  } else if (any_stall) {
    conv = all_floor;
    stop = true;
  }
  if (!stop && s + 1 > r.max_refine) stop = true;
  scal[S_D2] = d2sum;
  scal[S_UPD] = relmax;
  scal[S_PREV] = relmax;
  flags[F_SWEEP] = s + 1;
  flags[F_RCONV] = conv ? 1 : 0;
  flags[F_RSTOP] = stop ? 1 : 0;
  if (use_handle) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

}  // namespace pd
