// Device-side control of the solve: the stopping tests of Algorithm 2 (Sec. 3:
// ||r_m|| <= eps ||b|| or m = maxit, plus the stall and breakdown exits) and the
// refinement stopping rule run in single-thread kernels that write the control
// block and, inside a CUDA graph, set the conditional of the enclosing WHILE node.
// The same kernels run when the host drives the loops (it then reads the flags).
#include <cmath>

#include "pd_control.cuh"

namespace pd {

__global__ void k_solve_reset(double *scal, int *flags) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < kFlagWords; ++i) flags[i] = 0;
  for (int i = 0; i < kScalWords; ++i) scal[i] = 0.0;
  scal[S_PREV] = 1.0;
}

__global__ void k_krylov_decide(double *scal, int *flags, KrylovCtl k, int use_handle,
                                cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) krylov_decide(scal, flags, k, use_handle, h);
}

__global__ void k_refine_decide(double *scal, int *flags, RefineCtl r, int use_handle,
                                cudaGraphConditionalHandle h) {
  if (threadIdx.x == 0 && blockIdx.x == 0) refine_decide(scal, flags, r, use_handle, h);
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
