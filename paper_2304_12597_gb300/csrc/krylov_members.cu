// One Algorithm 2 per member of a batched plan.  K is block diagonal over the
// members (member b owns rows [b len, (b+1) len) and never couples to another), so
// each member runs the paper's Algorithm 2 on its own part b_b of b = sum_i gamma_i L_i
// (eq. 7): its own Krylov space K_m(K_b, b_b), Hessenberg T_m (eq. 10), capacitance
// system (eq. 12), residual estimate and stopping decision (eq. 13), exactly as if it
// were solved alone.  The members share the kernel launches, the stored shifted
// solves h_k and the basis array V (member b's entries in its own rows).
//
// One CTA per member holds that member's vectors in registers (len <= 8192 entries).
// A member whose Algorithm 2 has stopped keeps its y_m and writes zero rows into V
// from then on, so the shared shifted solves return zero there and x_m = V y_m stays
// each member's own; the step loop runs while any member runs.  The last member to
// finish the start or eq. (13) writes the batch totals and the loop decision.
#include "pd_internal.h"
#include "pd_krylov.cuh"

namespace pd {

struct MemberView {
  double *scal;
  int *flags;
  double *T, *y;
  int64_t off;
};

__device__ __forceinline__ MemberView member_view(const KrylovBufs &k, int b) {
  MemberView v;
  v.scal = k.mscal + (int64_t)b * kScalWords;
  v.flags = k.mflags + (int64_t)b * kFlagWords;
  v.T = k.T + (int64_t)b * (k.maxit + 1) * k.maxit;
  v.y = k.y + (int64_t)b * (k.maxit + 1);
  v.off = (int64_t)b * k.mlen;
  return v;
}

// Batch totals after every member has finished a step (run by the last CTA):
// ||b|| and ||r_m|| as root sums of squares over the members, the loop flags, and the
// WHILE conditional (continue while any member runs).  start: after the first step.
// red: kRedWords doubles of shared memory.
__device__ void member_totals(const KrylovBufs &k, bool start, int use_handle, cudaGraphConditionalHandle h,
                              double *red) {
  __shared__ double out[2];
  double s[2] = {0.0, 0.0};
  int run = 0, conv = 1, nonfin = 0, zero = 1;
  for (int b = threadIdx.x; b < k.members; b += blockDim.x) {
    const double *sb = k.mscal + (int64_t)b * kScalWords;
    const int *fb = k.mflags + (int64_t)b * kFlagWords;
    s[0] += sb[S_BETA] * sb[S_BETA];
    s[1] += sb[S_RES] * sb[S_RES];
    run |= fb[F_KSTOP] ? 0 : 1;
    conv &= fb[F_KCONV] ? 1 : 0;
    nonfin |= fb[F_NONFIN] ? 1 : 0;
    zero &= fb[F_BZERO] ? 1 : 0;
  }
  run = __syncthreads_or(run);
  conv = __syncthreads_and(conv);
  nonfin = __syncthreads_or(nonfin);
  zero = __syncthreads_and(zero);
  block_sums(s, 2, red, out);
  if (threadIdx.x == 0) {
    double *scal = k.scal;
    int *flags = k.flags;
    if (nonfin) flags[F_NONFIN] = 1;
    scal[S_RES] = sqrt(out[1]);
    if (start) {
      scal[S_BETA] = sqrt(out[0]);
      scal[S_T] = 0.0;
      flags[F_BREAK] = 0;  // a member's breakdown only stops that member
      flags[F_BZERO] = zero;
      flags[F_CAPCNT] = 0;
      flags[F_M] = 0;
    } else {
      flags[F_M] += 1;
    }
    const bool stop = !run || nonfin || flags[F_M] >= k.maxit;
    flags[F_KSTOP] = stop ? 1 : 0;
    flags[F_KCONV] = conv;
    if (use_handle) cudaGraphSetConditional(h, stop ? 0u : 1u);
    *k.counter = 0;
  }
}

// Start of Algorithm 2 for member blockIdx.x: beta_b = ||b_b||, v_1 = b_b / beta_b, its
// T_m and y_m cleared, its control block reset.
template <int E>
__global__ void __launch_bounds__(kBlasSingle) k_member_init(KrylovBufs k, const double *__restrict__ b,
                                                            int use_handle, cudaGraphConditionalHandle h) {
  grid_dep_wait();
  __shared__ double red[kRedWords];
  __shared__ double c[34];
  const MemberView mv = member_view(k, blockIdx.x);
  const int len = k.mlen;
  for (int i = threadIdx.x; i < (k.maxit + 1) * k.maxit; i += blockDim.x) mv.T[i] = 0.0;
  for (int i = threadIdx.x; i <= k.maxit; i += blockDim.x) mv.y[i] = 0.0;
  double x[E];
  reg_load<kSingle, E>(len, b + mv.off, x);
  const double beta = sqrt(reg_norm2<kSingle, E>(x, nullptr, 0, red, c));
  const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = threadIdx.x + e * blockDim.x;
    if (j < len) {
      const double v = x[e] * ib;
      k.V[mv.off + j] = v;
      if (k.Vf) k.Vf[mv.off + j] = (float)v;
    }
  }
  if (threadIdx.x == 0) {
    const bool finite = isfinite(beta), zero = !(beta > 0.0);
    double *scal = mv.scal;
    int *flags = mv.flags;
    scal[S_BETA] = beta;
    scal[S_T] = 0.0;
    scal[S_RES] = beta;
    scal[S_HIST] = beta;
    flags[F_BREAK] = 0;
    flags[F_BZERO] = zero ? 1 : 0;
    flags[F_NONFIN] = finite ? 0 : 1;
    flags[F_CAPCNT] = 0;
    flags[F_M] = 0;
    flags[F_FROZEN] = 0;  // no step is frozen until an Arnoldi step says so (q > 1)
    flags[F_NOH] = 0;
    flags[F_KSTOP] = (finite && !zero) ? 0 : 1;
    flags[F_KCONV] = zero ? 1 : 0;
  }
  if (last_cta_done(k.counter)) member_totals(k, true, use_handle, h, red);
}

// One Arnoldi step (eq. 10) for member blockIdx.x, as in the single-problem kernel;
// a member that has stopped writes a zero row instead.
template <int E>
__global__ void __launch_bounds__(kBlasSingle) k_member_arnoldi(KrylovBufs k) {
  grid_dep_wait();
  __shared__ double red[kRedWords];
  __shared__ double c[34];
  const MemberView mv = member_view(k, blockIdx.x);
  const int len = k.mlen, ldT = k.maxit;
  const int64_t ldv = k.n;
  const int m = k.flags[F_M] + 1;  // the step computed here produces row m of V
  double *vm = k.V + m * ldv + mv.off;
  float *vmf = k.Vf ? k.Vf + m * ldv + mv.off : nullptr;
  if (mv.flags[F_KSTOP]) {
    for (int j = threadIdx.x; j < len; j += blockDim.x) {
      vm[j] = 0.0;
      if (vmf) vmf[j] = 0.0f;
    }
    return;
  }
  const double *Vb = k.V + mv.off;
  const double *v = Vb + (m - 1) * ldv;
  const double *klo = k.klo + mv.off, *kdiag = k.kdiag + mv.off, *kup = k.kup + mv.off;
  double x[E];
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = threadIdx.x + e * blockDim.x;
    double a = 0.0;
    if (j < len) {
      a = kdiag[j] * v[j];
      if (j > 0) a += klo[j] * v[j - 1];
      if (j + 1 < len) a += kup[j] * v[j + 1];
    }
    x[e] = a;
  }
  const bool wr = (int)threadIdx.x < m;  // writes column m-1 of T
  reg_dots<kSingle, E>(len, m, Vb, ldv, x, nullptr, 0, red, c);
  const double knorm = sqrt(c[m]);
  const double tq = wr ? c[threadIdx.x] : 0.0;
  reg_axpy<kSingle, E>(len, m, Vb, ldv, x, c);
  __syncthreads();  // c is rewritten next
  reg_dots<kSingle, E>(len, m, Vb, ldv, x, nullptr, 0, red, c);
  if (wr) mv.T[(int64_t)threadIdx.x * ldT + (m - 1)] = tq + c[threadIdx.x];
  reg_axpy<kSingle, E>(len, m, Vb, ldv, x, c);
  __syncthreads();
  const double t = sqrt(cgs2_norm2<kSingle, E>(m, x, c, nullptr, 0, red));
  const bool bd = !(t > 1e-14 * knorm);
  const double it = bd ? 0.0 : 1.0 / t;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = threadIdx.x + e * blockDim.x;
    if (j < len) {
      const double y = x[e] * it;
      vm[j] = y;
      if (vmf) vmf[j] = (float)y;
    }
  }
  if (threadIdx.x == 0) {
    mv.T[(int64_t)m * ldT + (m - 1)] = bd ? 0.0 : t;
    mv.scal[S_T] = bd ? 0.0 : t;
    mv.scal[S_KNORM] = knorm;
    mv.flags[F_BREAK] = bd ? 1 : 0;
    if (!isfinite(t)) mv.flags[F_NONFIN] = 1;
  }
}

// eq. (13) for member blockIdx.x (two CGS passes of its part of z against its basis)
// and its stopping decision; members that had stopped keep their state.
template <int E>
__global__ void __launch_bounds__(kBlasSingle) k_member_project(KrylovBufs k, const double *__restrict__ z,
                                                               double tau, KrylovCtl kc, int use_handle,
                                                               cudaGraphConditionalHandle h) {
  grid_dep_wait();
  __shared__ double red[kRedWords];
  __shared__ double c[34];
  const MemberView mv = member_view(k, blockIdx.x);
  const int len = k.mlen;
  const int64_t ldv = k.n;
  if (!mv.flags[F_KSTOP]) {  // the same for every thread of the CTA
    const int m = mv.flags[F_M] + 1;
    const double *Vb = k.V + mv.off;
    double x[E];
    reg_load<kSingle, E>(len, z + mv.off, x);
    reg_dots<kSingle, E>(len, m, Vb, ldv, x, nullptr, 0, red, c);
    reg_axpy<kSingle, E>(len, m, Vb, ldv, x, c);
    __syncthreads();  // c is rewritten next
    reg_dots<kSingle, E>(len, m, Vb, ldv, x, nullptr, 0, red, c);
    reg_axpy<kSingle, E>(len, m, Vb, ldv, x, c);
    __syncthreads();
    const double zz = cgs2_norm2<kSingle, E>(m, x, c, nullptr, 0, red);
    if (threadIdx.x == 0) {
      mv.scal[S_RES] = mv.flags[F_BREAK] ? 0.0 : fabs(tau * mv.scal[S_T]) * sqrt(zz);
      krylov_decide(mv.scal, mv.flags, kc, 0, h);
    }
  }
  if (last_cta_done(k.counter)) member_totals(k, false, use_handle, h, red);
}

static void member_launch(Ctx &c, const char *fam, double bytes, const void *fn, int members, void **args) {
  c.launch(fam, bytes, [&] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)members);
    cfg.blockDim = dim3(kBlasSingle);
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = c.pdl ? 1 : 0;
    cudaLaunchKernelExC(&cfg, fn, args);
  });
}

#define PD_MEMBER_BY_E(E, KERNEL)                                                                    \
  ((E) <= 1 ? (const void *)KERNEL<1>                                                               \
            : (E) == 2 ? (const void *)KERNEL<2>                                                    \
                       : (E) == 4 ? (const void *)KERNEL<4>                                         \
                                  : (E) == 8 ? (const void *)KERNEL<8> : (const void *)KERNEL<16>)

void launch_member_init(Ctx &c, KrylovBufs &k, const double *b, int use_handle, cudaGraphConditionalHandle h) {
  void *args[] = {&k, (void *)&b, &use_handle, &h};
  member_launch(c, "krylov_init", (double)k.n * 16, PD_MEMBER_BY_E(reg_elems(k.mlen, kBlasSingle), k_member_init),
                k.members, args);
}

void launch_member_arnoldi(Ctx &c, KrylovBufs &k) {
  void *args[] = {&k};
  member_launch(c, "krylov_arnoldi", (double)k.n * 8.0 * 8,
                PD_MEMBER_BY_E(reg_elems(k.mlen, kBlasSingle), k_member_arnoldi), k.members, args);
}

void launch_member_project(Ctx &c, KrylovBufs &k, const double *z, double tau, const KrylovCtl &kc0, int use_handle,
                           cudaGraphConditionalHandle h) {
  KrylovCtl kc = kc0;
  void *args[] = {&k, (void *)&z, &tau, &kc, &use_handle, &h};
  member_launch(c, "krylov_project", (double)k.n * 8.0 * 6,
                PD_MEMBER_BY_E(reg_elems(k.mlen, kBlasSingle), k_member_project), k.members, args);
}

}  // namespace pd
