// Device-side control of the solve: the stopping tests of Algorithm 2 (Sec. 3:
// ||r_m|| <= eps ||b|| or m = maxit, plus the stall and breakdown exits) and the
// refinement stopping rule run in single-thread kernels that write the control
// block and, inside a CUDA graph, set the conditional of the enclosing WHILE node.
// The same kernels run when the host drives the loops (it then reads the flags).
#include <cmath>

#include "pd_control.cuh"

namespace pd {

__global__ void k_solve_reset(double *scal, int *flags) {
  grid_dep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < kFlagWords; ++i) flags[i] = 0;
  for (int i = 0; i < kScalWords; ++i) scal[i] = 0.0;
  scal[S_PREV] = 1.0;
}

__global__ void k_krylov_decide(double *scal, int *flags, KrylovCtl k, int use_handle,
                                cudaGraphConditionalHandle h) {
  grid_dep_wait();
  if (threadIdx.x == 0 && blockIdx.x == 0) krylov_decide(scal, flags, k, use_handle, h);
}

// The fixed-cost variants of Table 3 run no Algorithm 2.  loops = 2: x_m = b, i.e. the
// inner matrix of eq. (17) taken as I, which the final loop forms as V_1 y_1 with
// v_1 = b / beta from the initialisation and y_1 = beta; loops = 1: x_m = 0, so the final
// loop returns U_1.  Closes the Algorithm-2 loop before it starts.
__global__ void k_inner_fixed(double *scal, int *flags, double *y, int loops, int use_handle,
                              cudaGraphConditionalHandle h) {
  grid_dep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double beta = scal[S_BETA];
  const bool take_b = loops == 2 && !flags[F_BZERO] && isfinite(beta) && beta > 0.0;
  y[0] = take_b ? beta : 0.0;
  flags[F_M] = take_b ? 1 : 0;
  flags[F_KSTOP] = 1;
  flags[F_KCONV] = 1;
  if (use_handle) cudaGraphSetConditional(h, 0u);
}

__global__ void k_refine_decide(double *scal, int *flags, RefineCtl r, int use_handle,
                                cudaGraphConditionalHandle h) {
  grid_dep_wait();
  if (threadIdx.x == 0 && blockIdx.x == 0) refine_decide(scal, flags, r, use_handle, h);
}

// Batched plans: block b sums the per-column squares of problem b's n_x columns
// (fixed order), and the last block to finish (counter; no block waits) takes the
// refinement decision over all problems.
__global__ void __launch_bounds__(256) k_member_decide(const double *__restrict__ colsum, int nxm,
                                                       const int *__restrict__ nxb, int nmem, double *d2,
                                                       double *ref2, double *prev, int *mex,
                                                       const int *__restrict__ zero, int *counter, double *scal,
                                                       int *flags, RefineCtl rc, int use_handle,
                                                       cudaGraphConditionalHandle h) {
  grid_dep_wait();
  __shared__ double red[256];
  const int b = blockIdx.x;
  const int n = nxb[b];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += colsum[(int64_t)b * nxm + i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  __shared__ int last;
  if (threadIdx.x == 0) {
    d2[b] = red[0];
    __threadfence();
    last = atomicAdd(counter, 1) == nmem - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    if (threadIdx.x == 0) *counter = 0;
    __syncthreads();  // red is reused
    refine_decide_members(scal, flags, rc, nmem, d2, ref2, prev, mex, zero, use_handle, h, red);
  }
}

void launch_member_decide(Ctx &c, const double *colsum, int nxm, const int *nxb, int nmem, double *d2, double *ref2,
                          double *prev, int *mex, const int *zero, double *scal, int *flags, const RefineCtl &r,
                          int use_handle, cudaGraphConditionalHandle h) {
  int *counter = flags + F_C2RCNT;
  c.launch("control", 0.0, [&] {
    pdl_launch(c.pdl, k_member_decide, dim3(nmem), dim3(256), 0, c.stream, colsum, nxm, nxb, nmem, d2, ref2, prev, mex,
               zero, counter, scal, flags, r, use_handle, h);
  });
}

// Algorithm 3's U_1 exit: the solve is U_1 itself; record it as one solve with no
// Algorithm-2 step and stop the refinement loop (the inverse DFT, which otherwise
// decides, was skipped).
__global__ void k_early_finish(double *scal, int *flags, int use_handle, cudaGraphConditionalHandle h) {
  grid_dep_wait();
  if (threadIdx.x != 0 || blockIdx.x != 0 || !flags[F_EARLY]) return;
  flags[F_SWM] = 0;
  scal[S_SWRES] = 0.0;
  scal[S_SWUPD] = 1.0;
  scal[S_SWBETA] = scal[S_BETA];
  scal[S_UPD] = 0.0;
  flags[F_SWEEP] = 1;
  flags[F_RCONV] = 1;
  flags[F_RSTOP] = 1;
  if (use_handle) cudaGraphSetConditional(h, 0u);
}

void launch_early_finish(Ctx &c, double *scal, int *flags, int use_handle, cudaGraphConditionalHandle h) {
  c.launch("control", 0.0, [&] { pdl_launch(c.pdl, k_early_finish, dim3(1), dim3(32), 0, c.stream, scal, flags, use_handle, h); });
}

void launch_solve_reset(Ctx &c, double *scal, int *flags) {
  c.launch("control", 0.0, [&] { pdl_launch(c.pdl, k_solve_reset, dim3(1), dim3(32), 0, c.stream, scal, flags); });
}

void launch_krylov_decide(Ctx &c, double *scal, int *flags, const KrylovCtl &k, int use_handle,
                          cudaGraphConditionalHandle h) {
  c.launch("control", 0.0, [&] { pdl_launch(c.pdl, k_krylov_decide, dim3(1), dim3(32), 0, c.stream, scal, flags, k, use_handle, h); });
}

void launch_inner_fixed(Ctx &c, double *scal, int *flags, double *y, int loops, int use_handle,
                        cudaGraphConditionalHandle h) {
  c.launch("control", 0.0, [&] { pdl_launch(c.pdl, k_inner_fixed, dim3(1), dim3(32), 0, c.stream, scal, flags, y, loops, use_handle, h); });
}

void launch_refine_decide(Ctx &c, double *scal, int *flags, const RefineCtl &r, int use_handle,
                          cudaGraphConditionalHandle h) {
  c.launch("control", 0.0, [&] { pdl_launch(c.pdl, k_refine_decide, dim3(1), dim3(32), 0, c.stream, scal, flags, r, use_handle, h); });
}

}  // namespace pd
