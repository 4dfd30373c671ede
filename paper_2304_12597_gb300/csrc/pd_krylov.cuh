// Vector building blocks of Algorithm 2 (FP64): fixed-order CTA reductions, the CGS
// dot products and updates, and the bodies of the steps that start Algorithm 2
// (beta = ||b||, v_1) and finish each of its iterations (eq. 13 and the stopping
// decision).  Internal header, included by the Krylov kernels and by the kernels
// that run those bodies in their last CTA.
//
// MODE kCoop: the vectors are spread over a cooperative grid of kBlas-thread CTAs (at
// most one per SM), partial sums meet in a global panel after a grid barrier; with E >= 1
// each thread holds its E entries in registers through a step (as in the cluster mode),
// with E = 0 (vectors longer than the grid's registers hold) they stream from memory.  kCluster: they are spread over one thread-block
// cluster (the whole grid), each CTA keeps its partial sums in shared memory and the
// others read them through distributed shared memory after a cluster barrier, so the
// FP64 work of a vector step runs on several SMs without grid-wide barriers.
// kTail: one CTA, streaming the vectors from memory with few registers (the tail
// of another kernel, which keeps that kernel's register budget).
// kSingle: one CTA owns the whole vector (short
// vectors); it may be any CTA of a larger launch, since these bodies then ignore the
// block index.
#pragma once

#include <cooperative_groups.h>

#include "pd_control.cuh"

namespace pd {

constexpr int kBlasSingle = 512;   // threads of the one-CTA variants (short vectors)
constexpr int kBlasCluster = 128;  // threads per CTA of the cluster variants
constexpr int kRedQ = 4;           // sums reduced side by side
constexpr int kRedWords = kRedQ * kBlasSingle;
constexpr int kSingle = 0, kCoop = 1, kCluster = 2, kTail = 3;  // MODE of the vector steps
// kPersist: as kCoop (register-resident entries over a cooperative grid), inside the
// persistent Algorithm-2 step, whose grid barriers wait a bounded number of polls
constexpr int kPersist = 4;

// Grid barrier with a bounded wait (cooperative launches of the persistent step).  Every
// CTA arrives on flags[F_BARCNT]; the last of `expect` arrivals resets the count and bumps
// the generation flags[F_BARGEN]; the others poll the generation at most `limit` times.  A
// wait that runs out records flags[F_TIMEOUT], sets the step's WHILE conditional to 0 and
// marks the CTA failed: its later barriers return false at once, and the kernel leaves
// after the phase it is in.  The counters start at zero in every solve (k_solve_reset),
// and no launch of the persistent step runs once flags[F_TIMEOUT] is set.
struct BarCtx {
  int *flags;
  long long limit;
  int expect;  // arrivals that complete a barrier: the grid, plus any test-only phantoms
  int nv;      // CTAs of the vector phases (kPersist), the first nv of the grid
  int use_handle;
  cudaGraphConditionalHandle h;
  int failed;
};
__device__ __forceinline__ BarCtx &bar_ctx() {
  __shared__ BarCtx c;
  return c;
}
// wait = false: arrive only (a CTA with nothing left to do after this barrier).
__device__ inline bool bounded_grid_sync(bool wait = true) {
  BarCtx &bc = bar_ctx();
  __syncthreads();
  if (threadIdx.x == 0 && !bc.failed) {
    volatile int *gen = bc.flags + F_BARGEN;
    const int g = *gen;
    __threadfence();
    const int arrived = atomicAdd(bc.flags + F_BARCNT, 1) + 1;
    if (arrived == bc.expect) {
      bc.flags[F_BARCNT] = 0;
      __threadfence();
      atomicAdd(bc.flags + F_BARGEN, 1);
    } else if (wait) {
      long long polls = 0;
      while (*gen == g && polls < bc.limit) ++polls;
      if (*gen == g) {
        bc.failed = 1;
        atomicExch(bc.flags + F_TIMEOUT, 1);
        if (bc.use_handle) cudaGraphSetConditional(bc.h, 0u);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return !bc.failed;
}
constexpr int kSlot = 36;  // doubles per cluster-mode partial slot (m + 1 <= 33 sums)

template <int MODE>
__device__ __forceinline__ int g_first() {
  if constexpr (MODE == kCoop || MODE == kCluster || MODE == kPersist) return blockIdx.x * blockDim.x + threadIdx.x;
  return threadIdx.x;
}
template <int MODE>
__device__ __forceinline__ int g_stride() {
  if constexpr (MODE == kCoop || MODE == kCluster) return gridDim.x * blockDim.x;
  if constexpr (MODE == kPersist) return bar_ctx().nv * blockDim.x;
  return blockDim.x;
}
// CTAs that hold partials of a grid reduction (one panel row each)
template <int MODE>
__device__ __forceinline__ int g_ctas() {
  if constexpr (MODE == kCoop) return gridDim.x;
  if constexpr (MODE == kPersist) return bar_ctx().nv;
  return 1;
}
template <int MODE>
__device__ __forceinline__ bool g_leader() {
  if constexpr (MODE == kCoop || MODE == kCluster || MODE == kPersist) return blockIdx.x == 0 && threadIdx.x == 0;
  return threadIdx.x == 0;
}

// out[i] = sum over the CTA of s[i], i < nq <= kRedQ (shared `out`, valid for every
// thread on return).  The partials go through shared memory and warp i adds column
// i (also i + warps, ... when the CTA has fewer warps than sums), so each sum costs
// blockDim/32 + 5 dependent FP64 adds on one warp instead of a shuffle tree on every
// warp (GB300's FP64 rate makes the instruction count matter).
// red: kRedWords doubles of shared memory; blockDim.x <= kBlasSingle.
__device__ __forceinline__ void block_sums(const double *s, int nq, double *red, double *out) {
  const int nt = blockDim.x, tid = threadIdx.x;
  for (int i = 0; i < nq; ++i) red[i * nt + tid] = s[i];
  __syncthreads();
  const int l = tid & 31, nw = nt >> 5;
  for (int w = tid >> 5; w < nq; w += nw) {  // fewer warps than sums: warps take several
    double t = 0.0;
    for (int i = l; i < nt; i += 32) t += red[w * nt + i];
    t = warp_sum(t);
    if (l == 0) out[w] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ double block_sum(double v, double *red) {
  __shared__ double out1[1];
  block_sums(&v, 1, red, out1);
  return out1[0];  // valid in every thread
}

// part_row[q] = sum over this CTA's slice of V[q][j] x[j] (q < m); part_row[m] = ||x||^2
// (into the shared c_local instead when it is given).  kRedQ sums per pass over x.
template <int MODE>
__device__ __forceinline__ void cta_dots(int n, int m, const double *__restrict__ V, const double *__restrict__ x,
                                         double *part_row, double *red, double *c_local) {
  __shared__ double out[kRedQ];
  for (int q0 = 0; q0 <= m; q0 += kRedQ) {
    const int nq = min(kRedQ, m + 1 - q0);
    double s[kRedQ];
#pragma unroll
    for (int i = 0; i < kRedQ; ++i) s[i] = 0.0;
    for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) {
      const double xj = x[j];
#pragma unroll
      for (int i = 0; i < kRedQ; ++i) {
        const int q = q0 + i;
        if (i < nq) s[i] += (q < m ? V[(int64_t)q * n + j] : xj) * xj;
      }
    }
    block_sums(s, nq, red, out);
    if ((int)threadIdx.x < nq) (c_local ? c_local : part_row)[q0 + threadIdx.x] = out[threadIdx.x];
  }
}

// c[q] = sum_cta panel[cta][q], q <= m, then a CTA barrier.  Warp w sums column q = w
// (w + warps, ...): its lanes load the CTAs' partials side by side and a fixed-order warp
// sum adds them, so the panel is read in one round trip rather than one per partial.
__device__ __forceinline__ void cta_gather(const double *panel, int ld, int nparts, int m, double *c) {
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = threadIdx.x >> 5; q <= m; q += nw) {
    double s = 0.0;
    for (int i = lane; i < nparts; i += 32) s += panel[i * ld + q];
    s = warp_sum(s);
    if (lane == 0) c[q] = s;
  }
  __syncthreads();
}

// c[q] = sum over the cluster's CTAs of slot[q] (q < cnt; `slot` is this CTA's shared
// slot, the same offset in every CTA), rank order fixed; then a CTA barrier.  The
// cluster barrier's release/acquire makes every CTA's slot (and earlier global writes,
// after a fence) visible.  A slot must not be rewritten in the same launch.
__device__ __forceinline__ void cluster_gather(double *slot, int cnt, double *c) {
  cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
  cl.sync();
  if ((int)threadIdx.x < cnt) {
    double s = 0.0;
    const int nb = (int)cl.num_blocks();
    for (int r = 0; r < nb; ++r) s += cl.map_shared_rank(slot, r)[threadIdx.x];
    c[threadIdx.x] = s;
  }
  __syncthreads();
}

// c[q] = V[q] . x over the grid (q < m), c[m] = ||x||^2; shared c, valid in every thread
// on return.  Cooperative grids combine per-CTA partials through `panel` after a grid
// barrier; clusters through `panel` = a shared slot of kSlot doubles (cluster_gather);
// a single CTA keeps the totals in shared memory.
template <int MODE>
__device__ __forceinline__ void grid_dots(int n, int m, const double *__restrict__ V, const double *__restrict__ x,
                                          double *panel, int ld, double *red, double *c) {
  if constexpr (MODE == kCoop) {
    cta_dots<kCoop>(n, m, V, x, panel + (size_t)blockIdx.x * ld, red, nullptr);
    cooperative_groups::this_grid().sync();
    cta_gather(panel, ld, gridDim.x, m, c);
  } else if constexpr (MODE == kCluster) {
    cta_dots<kCluster>(n, m, V, x, nullptr, red, panel);
    cluster_gather(panel, m + 1, c);
  } else {
    cta_dots<MODE>(n, m, V, x, nullptr, red, c);
    __syncthreads();
  }
}

// The grid total of one value per thread (valid in every thread).
template <int MODE>
__device__ __forceinline__ double grid_sum(double s, double *panel, int ld, double *red, double *c) {
  s = block_sum(s, red);
  if constexpr (MODE == kCoop || MODE == kPersist) {
    if (threadIdx.x == 0) panel[(size_t)blockIdx.x * ld] = s;
    if constexpr (MODE == kCoop)
      cooperative_groups::this_grid().sync();
    else
      bounded_grid_sync();
    cta_gather(panel, ld, g_ctas<MODE>(), 0, c);
    return c[0];
  } else if constexpr (MODE == kCluster) {
    if (threadIdx.x == 0) panel[0] = s;
    cluster_gather(panel, 1, c);
    return c[0];
  } else {
    return s;
  }
}

// Cluster mode: no CTA may exit while another can still read its shared slots.
template <int MODE>
__device__ __forceinline__ void cluster_exit() {
  if constexpr (MODE == kCluster) cooperative_groups::this_cluster().sync();
}

// x -= sum_{q<m} c[q] V[q] over this CTA's slice.
template <int MODE>
__device__ __forceinline__ void cta_axpy(int n, int m, const double *__restrict__ V, double *x, const double *c) {
  for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) {
    double xj = x[j];
    for (int q = 0; q < m; ++q) xj -= c[q] * V[(int64_t)q * n + j];
    x[j] = xj;
  }
}

// Register-resident vectors (single CTA and cluster modes): thread entries
// j = g_first + e * g_stride, e < E, held in registers for the whole step, so a step
// reads its input vector once and the basis V through the read-only cache.  E (at most
// kEMax) is the smallest power of two that covers n; each E is its own kernel, so the
// unrolled loops stay as short as the vector needs.
constexpr int kEMax = 16;

// Entries per thread of the register-resident variants: the smallest power of two
// with E * threads >= n (the plan keeps n <= 8192 = 16 * 512 there).
inline int reg_elems(int n, int threads) {
  int e = 1;
  while (e < kEMax && e * threads < n) e <<= 1;
  return e;
}

template <int MODE, int E>
__device__ __forceinline__ void reg_load(int n, const double *__restrict__ x, double (&r)[E]) {
  const int f = g_first<MODE>(), st = g_stride<MODE>();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = f + e * st;
    r[e] = j < n ? x[j] : 0.0;
  }
}

// c[q] = V[q] . x over the grid (q < m), c[m] = ||x||^2 (shared c, valid in every
// thread on return); cluster mode combines the CTAs' sums through the shared `slot`.
// slot: cluster mode, this CTA's shared slot; cooperative mode, the global panel whose row
// blockIdx.x (leading dimension ld) receives this CTA's partials.
template <int MODE, int E>
__device__ __forceinline__ void reg_dots(int n, int m, const double *V, int64_t ldv, const double (&x)[E], double *slot,
                                         int ld, double *red, double *c) {
  static_assert(MODE == kSingle || MODE == kCluster || MODE == kCoop || MODE == kPersist, "register-resident steps");
  __shared__ double out[kRedQ];
  const int f = g_first<MODE>(), st = g_stride<MODE>();
  double *dst = MODE == kCluster ? slot : (MODE == kCoop || MODE == kPersist) ? slot + (size_t)blockIdx.x * ld : c;
  for (int q0 = 0; q0 <= m; q0 += kRedQ) {
    const int nq = min(kRedQ, m + 1 - q0);
    double s[kRedQ];
#pragma unroll
    for (int i = 0; i < kRedQ; ++i) s[i] = 0.0;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = f + e * st;
      if (j < n) {
#pragma unroll
        for (int i = 0; i < kRedQ; ++i) {
          const int q = q0 + i;
          if (i < nq) s[i] += (q < m ? __ldg(V + q * ldv + j) : x[e]) * x[e];
        }
      }
    }
    block_sums(s, nq, red, out);
    if ((int)threadIdx.x < nq) dst[q0 + threadIdx.x] = out[threadIdx.x];
  }
  if constexpr (MODE == kCluster) {
    cluster_gather(slot, m + 1, c);
  } else if constexpr (MODE == kCoop) {
    cooperative_groups::this_grid().sync();
    cta_gather(slot, ld, gridDim.x, m, c);
  } else if constexpr (MODE == kPersist) {
    bounded_grid_sync();
    cta_gather(slot, ld, g_ctas<MODE>(), m, c);
  } else {
    __syncthreads();
  }
}

// x -= sum_{q<m} c[q] V[q] on this thread's entries.
template <int MODE, int E>
__device__ __forceinline__ void reg_axpy(int n, int m, const double *V, int64_t ldv, double (&x)[E], const double *c) {
  const int f = g_first<MODE>(), st = g_stride<MODE>();
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int j = f + e * st;
    if (j < n) {
      double xj = x[e];
      for (int q = 0; q < m; ++q) xj -= c[q] * __ldg(V + q * ldv + j);
      x[e] = xj;
    }
  }
}

template <int MODE, int E>
__device__ __forceinline__ double reg_norm2(const double (&x)[E], double *slot, int ld, double *red, double *c) {
  double s = 0.0;
#pragma unroll
  for (int e = 0; e < E; ++e) s += x[e] * x[e];  // entries past n are zero
  return grid_sum<MODE>(s, slot, ld, red, c);
}

// ||x2||^2 after the second Gram-Schmidt pass x2 = x1 - V c, from that pass's dots
// (c[q] = V_q . x1, c[m] = ||x1||^2): ||x2||^2 = ||x1||^2 - sum_q c[q]^2 for orthonormal
// V, which saves a reduction.  The second pass removes only rounding-level components, so
// the difference keeps its digits; if it removed more than 1e-4 of ||x1||^2 the explicit
// reduction runs instead (every thread and CTA holds the same c: a uniform branch).
template <int MODE, int E>
__device__ __forceinline__ double cgs2_norm2(int m, const double (&x)[E], double *c, double *slot, int ld,
                                             double *red) {
  double r = 0.0;
  for (int q = 0; q < m; ++q) r += c[q] * c[q];
  const double a = c[m];
  if (r <= 1e-4 * a) return a - r;
  return reg_norm2<MODE, E>(x, slot, ld, red, c);
}

// Algorithm 2, first step: beta = ||b||, V[0] = b / beta (and its binary32 copy), T_m
// cleared, the control block reset, and the WHILE conditional set to run the loop
// unless b is zero or not finite.
template <int MODE, int E = 1>
__device__ __forceinline__ void init_v0_body(const double *__restrict__ b, int n, double *part, int ld, double *V,
                                             float *Vf, double *scal, int *flags, int use_handle,
                                             cudaGraphConditionalHandle h, double *T, int nT) {
  __shared__ double red[kRedWords];
  __shared__ double c[34];
  __shared__ double cslot[MODE == kCluster ? kSlot : 1];
  for (int i = g_first<MODE>(); i < nT; i += g_stride<MODE>()) T[i] = 0.0;
  double beta;
  if constexpr ((MODE == kCoop && E == 0) || MODE == kTail) {
    double s = 0.0;
    for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) s += b[j] * b[j];
    beta = sqrt(grid_sum<MODE>(s, part, ld, red, c));
    const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
    for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) {
      V[j] = b[j] * ib;
      if (Vf) Vf[j] = (float)V[j];
    }
  } else {
    double x[E > 0 ? E : 1];
    reg_load<MODE, E>(n, b, x);
    beta = sqrt(reg_norm2<MODE, E>(x, (MODE == kCoop || MODE == kPersist) ? part : cslot, ld, red, c));
    const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
    const int f = g_first<MODE>(), st = g_stride<MODE>();
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = f + e * st;
      if (j < n) {
        const double v = x[e] * ib;
        V[j] = v;
        if (Vf) Vf[j] = (float)v;
      }
    }
  }
  const bool zero = !(beta > 0.0);
  if (g_leader<MODE>()) {
    const bool finite = isfinite(beta);
    scal[S_BETA] = beta;
    scal[S_T] = 0.0;
    scal[S_RES] = beta;
    scal[S_HIST] = beta;
    flags[F_BREAK] = 0;
    flags[F_BZERO] = zero ? 1 : 0;
    if (!finite) flags[F_NONFIN] = 1;
    flags[F_CAPCNT] = 0;
    flags[F_M] = 0;
    flags[F_FROZEN] = 0;  // no step is frozen until an Arnoldi step says so (q > 1)
    flags[F_NOH] = 0;
    const bool run = finite && !zero;
    flags[F_KSTOP] = run ? 0 : 1;
    flags[F_KCONV] = zero ? 1 : 0;
    if (use_handle) cudaGraphSetConditional(h, run ? 1u : 0u);
  }
  cluster_exit<MODE>();
}

// eq. (13): ||r_m|| = |tau t_{m+1,m}| ||(I - V_m V_m^T) z|| with two CGS passes (zero
// after a breakdown), then the stopping decision.  The cooperative variant overwrites z
// with its projection.
template <int MODE, int E = 1>
__device__ __forceinline__ void project_body(int n, const double *__restrict__ V, double *z, double tau, double *part,
                                             int ld, double *scal, int *flags, const KrylovCtl &kc, int use_handle,
                                             cudaGraphConditionalHandle h) {
  __shared__ double red[kRedWords];
  __shared__ double c[34];
  const int m = flags[F_M] + 1;
  __shared__ double cslot[MODE == kCluster ? 3 * kSlot : 1];
  const int G = g_ctas<MODE>();
  double *pa = part, *pb = part + (size_t)G * ld, *pc = part + (size_t)2 * G * ld;
  if constexpr (MODE == kCluster) {
    pa = cslot;
    pb = cslot + kSlot;
    pc = cslot + 2 * kSlot;
  }
  double zz = 0.0;
  // a frozen step (q > 1) forms no z: the decision only advances m (uniform over the grid)
  const bool frozen = flags[F_FROZEN] != 0;
  if (frozen) {
  } else if constexpr ((MODE == kCoop && E == 0) || MODE == kTail) {
    grid_dots<MODE>(n, m, V, z, pa, ld, red, c);
    cta_axpy<MODE>(n, m, V, z, c);
    __syncthreads();  // c is rewritten next
    grid_dots<MODE>(n, m, V, z, pb, ld, red, c);
    cta_axpy<MODE>(n, m, V, z, c);
    __syncthreads();
    double s = 0.0;
    for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) s += z[j] * z[j];
    zz = grid_sum<MODE>(s, pc, ld, red, c);
  } else {  // z projected in registers (z itself is left as it is)
    double x[E > 0 ? E : 1];
    reg_load<MODE, E>(n, z, x);
    reg_dots<MODE, E>(n, m, V, n, x, pa, ld, red, c);
    reg_axpy<MODE, E>(n, m, V, n, x, c);
    __syncthreads();  // c is rewritten next
    reg_dots<MODE, E>(n, m, V, n, x, pb, ld, red, c);
    reg_axpy<MODE, E>(n, m, V, n, x, c);
    __syncthreads();
    zz = cgs2_norm2<MODE, E>(m, x, c, pc, ld, red);
  }
  if (g_leader<MODE>()) {
    if (!frozen) scal[S_RES] = flags[F_BREAK] ? 0.0 : fabs(tau * scal[S_T]) * sqrt(zz);
    krylov_decide(scal, flags, kc, use_handle, h);
  }
  cluster_exit<MODE>();
}

// Argument bundles of those bodies when they run in the last CTA of another kernel.
struct InitTail {
  int enabled;
  int *counter;  // zero on entry; reset by the last CTA
  int n, ld, nT, use_handle;
  double *part, *V, *scal, *T;
  float *Vf;
  int *flags;
  cudaGraphConditionalHandle h;
};
struct ProjTail {
  int enabled;
  int *counter;
  int n, ld, use_handle;
  const double *V;
  double tau;
  double *part, *scal;
  int *flags;
  KrylovCtl kc;
  cudaGraphConditionalHandle h;
};

// Last-block-done: every CTA calls this after its share of the work; the last one to
// arrive (no CTA waits for another) returns true with all other CTAs' writes visible.
__device__ __forceinline__ bool last_cta_done(int *counter) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) last = atomicAdd(counter, 1) == (int)(gridDim.x * gridDim.y) - 1;
  __syncthreads();
  if (last) __threadfence();
  return last;
}

}  // namespace pd
