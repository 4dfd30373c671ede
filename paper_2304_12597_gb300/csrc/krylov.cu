// Algorithm 2 (FOM-like method for J_l x = b, eq. 8) on the device, in FP64:
//  - Arnoldi in K (eqs. 9-10): w = K v_m, two classical Gram-Schmidt passes
//    (CGS2) against V_m, t_{m+1,m} = ||w||, v_{m+1} = w / t_{m+1,m};
//  - the projected m x m system of eq. (12): for every frequency k a warp forms
//    S_k = ((1 - pi_k) I_m + tau T_m)^{-1} by Gauss-Jordan elimination with
//    partial pivoting (a thread per frequency when m = 1) and accumulates
//    w_k Re(gamma_k (S_k - tau t g_k e_m^T S_k)); the last CTA then solves for y_m and
//    forms c_k = e_m^T S_k y_m;
//  - the residual norm of eq. (13): ||r_m|| = |tau t_{m+1,m}| ||(I - V_m V_m^T) z||,
//    z = sum_i gamma_i h_i c_i (z itself is accumulated by the shifted-solve pass);
//  - x_m = V_m y_m;
//  - the FP64 all-at-once residual G - [(I + tau K) U - U Sigma_1^T] used by the
//    mixed-precision refinement.
// The vector steps (init, Arnoldi, eq. 13) run in one CTA, one thread-block cluster
// or a cooperative grid (pd_krylov.cuh); batched plans run one CTA per problem
// (krylov_members.cu).  Cross-CTA reductions write one partial per CTA (or per
// cluster rank); every consumer sums the partials in the same fixed order, so results
// do not depend on scheduling.
//
// Scalar block `scal`: [0] beta = ||b||, [1] t_{m+1,m}, [2] ||r_m|| (eq. 13),
// [3] ||K v_m|| (breakdown reference), [4] last sum-of-squares result.
// Flag block `flags`: [0] breakdown (invariant Krylov space), [1] beta == 0,
// [2] non-finite value met, [3] completion counter of k_capacitance_terms.
#include <algorithm>
#include <cmath>

#include "pd_krylov.cuh"

namespace pd {

// beta = ||b||, V[0] = b / beta; resets scal/flags.
template <int MODE, int E>
__global__ void __launch_bounds__(MODE == kCoop ? kBlas : MODE == kCluster ? kBlasCluster : kBlasSingle)
    k_init_v0_coop(const double *__restrict__ b, int n, double *part, int ld, double *V, float *Vf, double *scal,
                   int *flags, int use_handle, cudaGraphConditionalHandle h, double *T, int nT) {
  grid_dep_wait();
  init_v0_body<MODE, E>(b, n, part, ld, V, Vf, scal, flags, use_handle, h, T, nT);
}

// One Arnoldi step (eq. 10): w = K v_{m-1}; two classical Gram-Schmidt passes
// against v_0..v_{m-1} (their coefficients summed into column m-1 of T_m);
// t = ||w||; v_m = w / t, or breakdown when t <= 1e-14 ||K v_{m-1}||.  With q > 1
// (Sec. 3: the residual is frozen for q steps) the step is marked frozen unless
// m is a multiple of q, m = maxit or the space broke down; a frozen step forms no
// h_k, no eq. (12) system and no eq. (13) residual.
template <int MODE, int E>
__device__ __forceinline__ void arnoldi_body(int n, const double *__restrict__ klo, const double *__restrict__ kdiag,
                                             const double *__restrict__ kup, double *V, float *Vf, double *w,
                                             double *T, int ldT, double *part, int ld, double *scal, int *flags,
                                             int q, int maxit) {
  __shared__ double red[kRedWords];
  __shared__ double c[34];
  const int m = flags[F_M] + 1;  // the step computed here produces v_m
  __shared__ double cslot[MODE == kCluster ? 3 * kSlot : 1];
  const int G = g_ctas<MODE>();
  double *pa = part, *pb = part + (size_t)G * ld, *pc = part + (size_t)2 * G * ld;
  if constexpr (MODE == kCluster) {
    pa = cslot;
    pb = cslot + kSlot;
    pc = cslot + 2 * kSlot;
  }
  const double *v = V + (int64_t)(m - 1) * n;
  double knorm, t;
  bool bd;
  if constexpr (MODE == kCoop && E == 0) {
    for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) {
      double x = kdiag[j] * v[j];
      if (j > 0) x += klo[j] * v[j - 1];
      if (j + 1 < n) x += kup[j] * v[j + 1];
      w[j] = x;
    }
    grid_dots<MODE>(n, m, V, w, pa, ld, red, c);
    knorm = sqrt(c[m]);
    if (blockIdx.x == 0 && (int)threadIdx.x < m) T[(int64_t)threadIdx.x * ldT + (m - 1)] = c[threadIdx.x];
    cta_axpy<MODE>(n, m, V, w, c);
    __syncthreads();  // c is rewritten next
    grid_dots<MODE>(n, m, V, w, pb, ld, red, c);
    if (blockIdx.x == 0 && (int)threadIdx.x < m) T[(int64_t)threadIdx.x * ldT + (m - 1)] += c[threadIdx.x];
    cta_axpy<MODE>(n, m, V, w, c);
    __syncthreads();
    double s = 0.0;
    for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) s += w[j] * w[j];
    t = sqrt(grid_sum<MODE>(s, pc, ld, red, c));
    bd = !(t > 1e-14 * knorm);
    const double it = bd ? 0.0 : 1.0 / t;
    double *vm = V + (int64_t)m * n;
    float *vmf = Vf ? Vf + (int64_t)m * n : nullptr;
    for (int j = g_first<MODE>(); j < n; j += g_stride<MODE>()) {
      vm[j] = w[j] * it;
      if (vmf) vmf[j] = (float)vm[j];
    }
  } else {  // w = K v_m held in registers through both CGS passes
    const int f = g_first<MODE>(), st = g_stride<MODE>();
    double x[E > 0 ? E : 1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = f + e * st;
      double a = 0.0;
      if (j < n) {
        a = kdiag[j] * v[j];
        if (j > 0) a += klo[j] * v[j - 1];
        if (j + 1 < n) a += kup[j] * v[j + 1];
      }
      x[e] = a;
    }
    // writes column m-1 of T
    const bool wr = (MODE == kSingle || MODE == kTail || blockIdx.x == 0) && (int)threadIdx.x < m;
    reg_dots<MODE, E>(n, m, V, n, x, pa, ld, red, c);
    knorm = sqrt(c[m]);
    double tq = wr ? c[threadIdx.x] : 0.0;
    reg_axpy<MODE, E>(n, m, V, n, x, c);
    __syncthreads();  // c is rewritten next
    reg_dots<MODE, E>(n, m, V, n, x, pb, ld, red, c);
    if (wr) T[(int64_t)threadIdx.x * ldT + (m - 1)] = tq + c[threadIdx.x];
    reg_axpy<MODE, E>(n, m, V, n, x, c);
    __syncthreads();
    t = sqrt(cgs2_norm2<MODE, E>(m, x, c, pc, ld, red));
    bd = !(t > 1e-14 * knorm);
    const double it = bd ? 0.0 : 1.0 / t;
    double *vm = V + (int64_t)m * n;
    float *vmf = Vf ? Vf + (int64_t)m * n : nullptr;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int j = f + e * st;
      if (j < n) {
        const double y = x[e] * it;
        vm[j] = y;
        if (vmf) vmf[j] = (float)y;
      }
    }
  }
  if (g_leader<MODE>()) {
    T[(int64_t)m * ldT + (m - 1)] = bd ? 0.0 : t;
    scal[S_T] = bd ? 0.0 : t;
    scal[S_KNORM] = knorm;
    flags[F_BREAK] = bd ? 1 : 0;
    const bool frozen = !bd && q > 1 && m % q != 0 && m < maxit;
    flags[F_FROZEN] = frozen ? 1 : 0;
    flags[F_NOH] = (bd || frozen) ? 1 : 0;
    if (!isfinite(t)) flags[F_NONFIN] = 1;
  }
  cluster_exit<MODE>();
}

// The Arnoldi step as a kernel of its own (nothing to do once Algorithm 2 has stopped:
// the first step of the persistent form follows the start unconditionally).
template <int MODE, int E>
__global__ void __launch_bounds__(MODE == kCoop ? kBlas : MODE == kCluster ? kBlasCluster : kBlasSingle) k_arnoldi_coop(int n, const double *__restrict__ klo,
                                                        const double *__restrict__ kdiag,
                                                        const double *__restrict__ kup, double *V, float *Vf,
                                                        double *w, double *T, int ldT, double *part, int ld,
                                                        double *scal, int *flags, int q, int maxit) {
  grid_dep_wait();
  if (flags[F_KSTOP]) return;  // uniform over the grid (and the cluster)
  arnoldi_body<MODE, E>(n, klo, kdiag, kup, V, Vf, w, T, ldT, part, ld, scal, flags, q, maxit);
}

// eq. (13) and the stopping decision (project_body).
template <int MODE, int E>
__global__ void __launch_bounds__(MODE == kCoop ? kBlas : MODE == kCluster ? kBlasCluster : kBlasSingle)
    k_project_coop(int n, const double *__restrict__ V, double *z, double tau, double *part, int ld, double *scal,
                   int *flags, KrylovCtl kc, int use_handle, cudaGraphConditionalHandle h) {
  grid_dep_wait();
  project_body<MODE, E>(n, V, z, tau, part, ld, scal, flags, kc, use_handle, h);
}

// ---- eq. (12): capacitance-system terms, one warp per frequency -----------------

// Gauss-Jordan inversion of the m x m complex matrix H (row-major, ld m) into X
// (initialised here), partial pivoting on rows; lane c owns column c; m <= 32.
__device__ void warp_gj_inverse(cpx<double> *H, cpx<double> *X, cpx<double> *fcol, int m) {
  const int lane = threadIdx.x & 31;
  for (int q = 0; q < m; ++q)
    if (lane < m) X[q * m + lane] = mk<double>(q == lane ? 1.0 : 0.0, 0.0);
  __syncwarp();
  for (int p = 0; p < m; ++p) {
    double v = (lane >= p && lane < m) ? abs2(H[lane * m + p]) : -1.0;
    int idx = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int oi = __shfl_xor_sync(0xffffffffu, idx, o);
      if (ov > v || (ov == v && oi < idx)) {
        v = ov;
        idx = oi;
      }
    }
    if (idx != p && lane < m) {
      cpx<double> h = H[p * m + lane];
      H[p * m + lane] = H[idx * m + lane];
      H[idx * m + lane] = h;
      cpx<double> x = X[p * m + lane];
      X[p * m + lane] = X[idx * m + lane];
      X[idx * m + lane] = x;
    }
    __syncwarp();
    const cpx<double> inv = recip(H[p * m + p]);
    __syncwarp();
    if (lane < m) {
      H[p * m + lane] = mul(H[p * m + lane], inv);
      X[p * m + lane] = mul(X[p * m + lane], inv);
    }
    __syncwarp();
    if (lane < m) fcol[lane] = H[lane * m + p];
    __syncwarp();
    if (lane < m) {
      const cpx<double> hp = H[p * m + lane], xp = X[p * m + lane];
      for (int i = 0; i < m; ++i) {
        if (i == p) continue;
        const cpx<double> f = fcol[i];
        H[i * m + lane] = fnms(H[i * m + lane], f, hp);
        X[i * m + lane] = fnms(X[i * m + lane], f, xp);
      }
    }
    __syncwarp();
  }
}

constexpr int kK5Warps = 4;

__device__ void capacitance_solve_cta(int nf, int m, int nparts, const double *msys_part,
                                      const double2 *__restrict__ srow, double2 *omega, double *y,
                                      const double *scal, unsigned char *smem);

// Per-warp shared-memory slice, rounded up to 16 bytes so that every warp's
// complex (16-byte) arrays stay aligned for any m.
__host__ __device__ inline size_t k5a_warp_bytes(int m) {
  const size_t b = (size_t)(2 * m * m + 2 * m) * sizeof(cpx<double>) + (size_t)m * m * sizeof(double);
  return (b + 15) & ~(size_t)15;
}

// The eq. (12) terms of CTA `cta` of `ncta`: each of its first `nwk` warps owns a
// shared-memory slice of k5a_warp_bytes(m) bytes at smraw and accumulates the terms of
// its frequencies there (a thread per frequency, every warp, when m = 1); the CTA's sum
// over those warps (fixed order) goes to row `cta` of msys_part.  `mb` selects a batch
// member's blocks of partial dots (members != 0; bpm blocks per member).  Ends with a CTA
// barrier.
__device__ void capacitance_terms_body(int cta, int ncta, int nwk, int m, int nf, int maxit, double tau,
                                       const double *__restrict__ T, const double2 *__restrict__ shift,
                                       const double2 *__restrict__ wg, const double2 *__restrict__ gpart,
                                       int nblk, double *msys_part, double2 *srow, const double *scal,
                                       const int *flags, int members, int mb, unsigned char *smraw, int bpm = 1,
                                       double2 *sinv = nullptr) {
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t wb = k5a_warp_bytes(m);
  const bool busy = wid < nwk;
  unsigned char *base = smraw + (busy ? wid : 0) * wb;
  cpx<double> *H = reinterpret_cast<cpx<double> *>(base);
  cpx<double> *X = H + m * m;
  cpx<double> *fcol = X + m * m;
  cpx<double> *gq = fcol + m;
  double *msw = reinterpret_cast<double *>(gq + m);
  const double tt = flags[F_BREAK] ? 0.0 : tau * scal[S_T];
  if (busy)
    for (int i = lane; i < m * m; i += 32) msw[i] = 0.0;
  __syncwarp();
  // g_k = sum over blocks of the partial dots; after a breakdown the dot pass was skipped
  // and the t-term vanishes; a batch member takes only its own blocks' dots (bpm of them)
  const int b0 = members ? mb * bpm : 0, b1 = flags[F_BREAK] ? b0 : (members ? b0 + bpm : nblk);
  if (m == 1) {
    // one step (the common case): S_k = 1 / ((1 - pi_k) + tau t_11) is a scalar, so a
    // thread takes a frequency (a warp of GJ per frequency would leave 31 lanes idle on
    // GB300's slow FP64 pipe)
    const double t11 = tau * T[0];
    double acc = 0.0;
    auto term = [&](int k, double gx, double gy) {
      const double2 sk = shift[k];
      const cpx<double> X1 = recip(mk<double>(t11 + sk.x, sk.y));
      const double2 w = wg[k];
      const cpx<double> wk = mk<double>(w.x, w.y);
      const cpx<double> ws = mul(wk, X1);
      srow[k] = make_double2(ws.x, ws.y);
      const cpx<double> gs = mul(mk<double>(gx, gy), X1);
      return mul(wk, mk<double>(X1.x - tt * gs.x, X1.y - tt * gs.y)).x;
    };
    if (b1 - b0 >= 32) {
      // many blocks (2D: one per mode of T_y): a warp per frequency, its lanes split the
      // blocks' partial dots, so the loads are in flight together rather than one after
      // another along a chain of adds
      const int gw = cta * nwk + wid, nw = ncta * nwk;
      for (int k = gw; busy && k < nf; k += nw) {
        double gx = 0.0, gy = 0.0;
        for (int b = b0 + lane; b < b1; b += 32) {
          const double2 v = gpart[(int64_t)k * nblk + b];
          gx += v.x;
          gy += v.y;
        }
        gx = warp_sum(gx);
        gy = warp_sum(gy);
        if (lane == 0) acc += term(k, gx, gy);
      }
    } else {
      for (int k = cta * blockDim.x + threadIdx.x; busy && k < nf; k += ncta * blockDim.x) {
        double gx = 0.0, gy = 0.0;
        for (int b = b0; b < b1; ++b) {
          const double2 v = gpart[(int64_t)k * nblk + b];
          gx += v.x;
          gy += v.y;
        }
        acc += term(k, gx, gy);
      }
    }
    acc = warp_sum(acc);
    if (busy && lane == 0) msw[0] = acc;
  } else if (busy) {
    const int gw = cta * nwk + wid, nw = ncta * nwk;
    for (int k = gw; k < nf; k += nw) {
      const double2 sk = shift[k];
      if (lane < m) {
        for (int q = 0; q < m; ++q) {
          const double tq = (q <= lane + 1) ? T[(int64_t)q * maxit + lane] : 0.0;
          H[q * m + lane] = mk<double>(tau * tq + (q == lane ? sk.x : 0.0), q == lane ? sk.y : 0.0);
        }
      }
      if (b1 - b0 >= 32) {  // many blocks: the lanes split them, one warp sum per dot
        for (int q = 0; q < m; ++q) {
          double gx = 0.0, gy = 0.0;
          for (int b = b0 + lane; b < b1; b += 32) {
            const double2 v = gpart[((int64_t)k * nblk + b) * m + q];
            gx += v.x;
            gy += v.y;
          }
          gx = warp_sum(gx);
          gy = warp_sum(gy);
          if (lane == 0) gq[q] = mk<double>(gx, gy);
        }
      } else if (lane < m) {
        double gx = 0.0, gy = 0.0;
        for (int b = b0; b < b1; ++b) {
          const double2 v = gpart[((int64_t)k * nblk + b) * m + lane];
          gx += v.x;
          gy += v.y;
        }
        gq[lane] = mk<double>(gx, gy);
      }
      __syncwarp();
      warp_gj_inverse(H, X, fcol, m);
      if (sinv && m <= kCombMaxM && lane < m)  // S_k = (s_k I + tau T_m)^{-1}, for the final loop
        for (int q = 0; q < m; ++q)
          sinv[((int64_t)k * m + q) * m + lane] = make_double2(X[q * m + lane].x, X[q * m + lane].y);
      const double2 w = wg[k];
      const cpx<double> wk = mk<double>(w.x, w.y);
      if (lane < m) {
        const cpx<double> sl = X[(m - 1) * m + lane];  // e_m^T S_k, column `lane`
        const cpx<double> ws = mul(wk, sl);  // w_k gamma_k (e_m^T S_k): omega_k = this . y_m
        srow[(int64_t)k * m + lane] = make_double2(ws.x, ws.y);
        for (int q = 0; q < m; ++q) {
          const cpx<double> gs = mul(gq[q], sl);
          const cpx<double> val = mk<double>(X[q * m + lane].x - tt * gs.x, X[q * m + lane].y - tt * gs.y);
          const cpx<double> c = mul(wk, val);
          msw[q * m + lane] += c.x;
        }
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // CTA partial = sum over its warps (fixed order)
  const size_t msw_off = (size_t)(2 * m * m + 2 * m) * sizeof(cpx<double>);
  for (int i = threadIdx.x; i < m * m; i += blockDim.x) {
    double s = 0.0;
    for (int wv = 0; wv < nwk; ++wv) s += reinterpret_cast<double *>(smraw + wv * wb + msw_off)[i];
    msys_part[(int64_t)cta * m * m + i] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kK5Warps * 32) k_capacitance_terms(
    int nf, int maxit, double tau, const double *__restrict__ T, const double2 *__restrict__ shift,
    const double2 *__restrict__ wg, const double2 *__restrict__ gpart, int nblk, double *msys_part,
    double2 *srow, const double *scal, int *flags, double2 *omega, double *y, int members, int bpm,
    double2 *sinv) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smraw[];
  if (members) {  // member blockIdx.y of a batch: its own Algorithm-2 state (strided views)
    const int mb = blockIdx.y;
    T += (int64_t)mb * (maxit + 1) * maxit;
    msys_part += (int64_t)mb * gridDim.x * maxit * maxit;
    srow += (int64_t)mb * nf * maxit;
    omega += (int64_t)mb * nf;
    y += (int64_t)mb * (maxit + 1);
    scal += (int64_t)mb * kScalWords;
    flags += (int64_t)mb * kFlagWords;
    if (flags[F_KSTOP]) return;  // this member's Algorithm 2 has stopped (whole CTA)
  } else if (flags[F_FROZEN]) {
    return;  // a frozen step (q > 1): no eq. (12) system (every CTA leaves; the counter stays 0)
  }
  const int m = flags[F_M] + 1;
  capacitance_terms_body(blockIdx.x, gridDim.x, kK5Warps, m, nf, maxit, tau, T, shift, wg, gpart, nblk, msys_part,
                         srow, scal, flags, members, (int)blockIdx.y, smraw, bpm, members ? nullptr : sinv);
  // The last CTA to finish (counted in flags[F_CAPCNT]; no CTA waits for another) sums the
  // partials and solves the m x m system, then resets the counter.
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&flags[F_CAPCNT], 1) == (int)gridDim.x - 1;
  __syncthreads();
  if (last) {
    __threadfence();
    capacitance_solve_cta(nf, m, gridDim.x, msys_part, srow, omega, y, scal, smraw);
    if (members)  // x_m = V y_m then runs over every step of the batch: zero the rest
      for (int q = m + threadIdx.x; q <= maxit; q += blockDim.x) y[q] = 0.0;
    if (threadIdx.x == 0) flags[F_CAPCNT] = 0;
  }
}

// M = I + sum of the per-CTA partials; y = beta M^{-1} e_1; omega_k = w_k gamma_k
// (e_m^T S_k y), with srow already holding the rows w_k gamma_k e_m^T S_k.  Run by one
// CTA; smem holds H, X (m x m complex), fcol and y.  GB300 issues FP64 at ~1/64 of the
// FP32 rate, so this serial tail keeps its FP64 instruction count small.
__device__ void capacitance_solve_cta(int nf, int m, int nparts, const double *msys_part,
                                      const double2 *__restrict__ srow, double2 *omega, double *y,
                                      const double *scal, unsigned char *smem) {
  cpx<double> *H = reinterpret_cast<cpx<double> *>(smem);
  cpx<double> *X = H + m * m;
  cpx<double> *fcol = X + m * m;
  double *ys = reinterpret_cast<double *>(fcol + m);
  // M = I + sum of the per-CTA partials: one warp per entry, lanes stride over CTAs
  {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = wid; i < m * m; i += nw) {
      double s = 0.0;
#pragma unroll 4
      for (int p = lane; p < nparts; p += 32) s += msys_part[(int64_t)p * m * m + i];
      s = warp_sum(s);
      if (lane == 0) H[i] = mk<double>(s + (((i / m) == (i % m)) ? 1.0 : 0.0), 0.0);
    }
  }
  __syncthreads();
  const double beta = scal[S_BETA];
  if (m == 1) {  // M is 1 x 1 (the common case): no elimination
    if (threadIdx.x == 0) {
      ys[0] = beta / H[0].x;
      y[0] = ys[0];
    }
  } else {
    if (threadIdx.x < 32) warp_gj_inverse(H, X, fcol, m);
    __syncthreads();
    if ((int)threadIdx.x < m) {
      ys[threadIdx.x] = beta * X[threadIdx.x * m + 0].x;
      y[threadIdx.x] = ys[threadIdx.x];
    }
  }
  __syncthreads();
  // srow holds w_k gamma_k (e_m^T S_k): two FP64 operations per step and frequency
#pragma unroll 4
  for (int k = threadIdx.x; k < nf; k += blockDim.x) {
    double cx = 0.0, cy = 0.0;
    for (int q = 0; q < m; ++q) {
      const double2 sv = srow[(int64_t)k * m + q];
      cx += sv.x * ys[q];
      cy += sv.y * ys[q];
    }
    omega[k] = make_double2(cx, cy);
  }
}

// x = sum_q y_q V[q] (and its binary32 copy xf when requested)
__global__ void k_xm(int n, const int *flags, const double *__restrict__ V, const double *__restrict__ y, double *x,
                     float *xf) {
  grid_dep_wait();
  __shared__ double ys[33];
  const int m = flags[F_M];  // 0 when b == 0: x = 0
  if (threadIdx.x < m) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < m; ++q) s += ys[q] * V[(int64_t)q * n + j];
    x[j] = s;
    if (xf) xf[j] = (float)s;
  }
}

// *dst = sum of part[0..nparts) (one warp, fixed order)
// The final parallel-in-time loop by linearity.  Arnoldi's relation (eq. 10),
// tau K V_m = V_m (tau T_m) + tau t_{m+1,m} v_{m+1} e_m^T, gives for A_k = s_k I + tau K
//   A_k^{-1} V_m = [V_m - tau t_{m+1,m} h_k e_m^T] S_k,  S_k = (s_k I + tau T_m)^{-1},
// with h_k = A_k^{-1} v_{m+1} the last step's stored shifted solves.  The final loop
// Y_k = A_k^{-1}(G^_k - a x_m), x_m = V_m y_m (a = alpha^{1/l}, 1 for Algorithm 1), is then
//   Y_k = L_k - V_m s_k + c_k h_k,  s_k = a S_k y_m,  c_k = tau t_{m+1,m} (e_m^T s_k),
// with L_k = A_k^{-1} G^_k stored by the first loop: an elementwise pass over the spectrum
// instead of a third set of shifted solves.  m = 1: s_k = a y_1 / (s_k + tau t_11); m > 1:
// S_k as the last eq. (12) system stored it (sinv).  Mode (the same in every CTA): 2, or 1
// without the h_k term after a breakdown (t_{m+1,m} = 0, no h_k formed), when Algorithm 2
// stopped at 1 <= m <= maxm and U_1 was not taken; else 0 and S is left to the final loop.
// CTAs with blockIdx.x = k < nf write row k of S (kCombCols columns each, blockIdx.y the
// chunk); blockIdx.x = nf forms x = x_m in FP64 for any m (paradiag_last_vectors).
constexpr int kCombCols = 1024;
template <typename T>
__global__ void __launch_bounds__(256) k_final_comb(int nf, int64_t n, int64_t lds, double tau, double aroot,
                                                    const double2 *__restrict__ shift, const double *__restrict__ Tm,
                                                    const double *__restrict__ y, const double *__restrict__ V,
                                                    const T *__restrict__ Vb, const double *__restrict__ scal,
                                                    int *flags, const double2 *__restrict__ sinv, int maxm,
                                                    const cpx<T> *__restrict__ L, const cpx<T> *__restrict__ H,
                                                    cpx<T> *__restrict__ S, double *x) {
  grid_dep_wait();
  __shared__ cpx<T> sc[kCombMaxM + 1];  // s_k, then c_k
  const int m = flags[F_M];
  const int mode = (m >= 1 && m <= maxm && !flags[F_EARLY] && !flags[F_TIMEOUT]) ? (flags[F_NOH] ? 1 : 2) : 0;
  const int k = blockIdx.x;
  const int64_t cstride = (int64_t)gridDim.y * kCombCols;  // chunks beyond 65535 loop
  if (k == nf) {  // x_m in FP64
    if (blockIdx.y == 0 && threadIdx.x == 0) {
      flags[F_COMB] = mode;
      if (mode) flags[F_COMBCNT] += 1;
    }
    for (int64_t c0 = (int64_t)blockIdx.y * kCombCols; c0 < n; c0 += cstride)
      for (int64_t j = c0 + threadIdx.x; j < n && j < c0 + kCombCols; j += blockDim.x) {
        double v = 0.0;
        for (int q = 0; q < m; ++q) v += y[q] * V[(int64_t)q * n + j];
        x[j] = v;
      }
    return;
  }
  if (!mode) return;
  __shared__ double2 sd[kCombMaxM];
  const int i = threadIdx.x;
  if (i < m) {  // s_k[i] = a (S_k y_m)_i
    double2 v;
    if (m == 1) {
      const double2 sk = shift[k];
      const cpx<double> r = recip(mk<double>(sk.x + tau * Tm[0], sk.y));
      v = make_double2(r.x * y[0], r.y * y[0]);
    } else {
      const double2 *X = sinv + ((int64_t)k * m + i) * m;
      v = make_double2(0.0, 0.0);
      for (int q = 0; q < m; ++q) {
        const double2 xq = X[q];
        v.x += xq.x * y[q];
        v.y += xq.y * y[q];
      }
    }
    v.x *= aroot;
    v.y *= aroot;
    sd[i] = v;
    sc[i] = mk<T>((T)v.x, (T)v.y);
  }
  __syncthreads();
  if (i == 0) {
    const double tt = mode == 2 ? tau * scal[S_T] : 0.0;
    sc[m] = mk<T>((T)(tt * sd[m - 1].x), (T)(tt * sd[m - 1].y));
  }
  __syncthreads();
  const cpx<T> ck = sc[m];
  constexpr int kE = kCombCols / 256;
  const int64_t o = (int64_t)k * lds;
  for (int64_t c0 = (int64_t)blockIdx.y * kCombCols; c0 < n; c0 += cstride) {
    cpx<T> acc[kE], h[kE];
#pragma unroll
    for (int e = 0; e < kE; ++e) {  // all loads in flight before any use
      const int64_t j = c0 + threadIdx.x + e * 256;
      const bool in = j < n;
      acc[e] = in ? L[o + j] : mk<T>(T(0), T(0));
      h[e] = (in && mode == 2) ? H[o + j] : mk<T>(T(0), T(0));
    }
    for (int q = 0; q < m; ++q) {  // - V_m s_k
      T v[kE];
#pragma unroll
      for (int e = 0; e < kE; ++e) {
        const int64_t j = c0 + threadIdx.x + e * 256;
        v[e] = j < n ? Vb[(int64_t)q * n + j] : T(0);
      }
      const cpx<T> sq = sc[q];
#pragma unroll
      for (int e = 0; e < kE; ++e) {
        acc[e].x -= sq.x * v[e];
        acc[e].y -= sq.y * v[e];
      }
    }
#pragma unroll
    for (int e = 0; e < kE; ++e) {
      const int64_t j = c0 + threadIdx.x + e * 256;
      if (j < n)
        S[o + j] = mk<T>(acc[e].x + ck.x * h[e].x - ck.y * h[e].y, acc[e].y + ck.x * h[e].y + ck.y * h[e].x);
    }
  }
}

__global__ void k_sumsq_final(const double *part, int nparts, double *dst) {
  grid_dep_wait();
  double s = 0.0;
  for (int i = threadIdx.x; i < nparts; i += 32) s += part[i];
  s = warp_sum(s);
  if (threadIdx.x == 0) *dst = s;
}

// Algorithm 3's test on U_1 (see launch_early_check): a grid-stride pass over the residual
// r = G_t + u_{t-1} - [(I + tau T_x) u_t (+ tau T_y u_t)] (the refinement's stencil), sums of
// r^2 and u^2 per CTA in FP64, combined in a fixed order by the last CTA to finish, which
// takes the decision.
template <bool TWO_D>
__global__ void __launch_bounds__(256) k_early_check(const double *__restrict__ G, const double *__restrict__ U,
                                                     int64_t nt, int nb, int nx, const double *__restrict__ rxl,
                                                     const double *__restrict__ rxd, const double *__restrict__ rxu,
                                                     const double *__restrict__ ryl, const double *__restrict__ ryd,
                                                     const double *__restrict__ ryu, int ny, int nym, double eps,
                                                     double *part, double *scal, int *flags, int use_handle,
                                                     cudaGraphConditionalHandle h) {
  grid_dep_wait();
  double rr = 0.0, uu = 0.0;
  const int64_t total = nt * nb;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = idx / nb;
    const int j = (int)(idx - t * nb);
    const double *u = U + t * nb;
    const int iy = TWO_D ? j / nx : 0;
    const int ix = TWO_D ? j - iy * nx : j;
    const int cx = TWO_D ? (iy / nym) * nx + ix : ix;
    const double uj = u[j];
    double r = G[idx];
    if (t > 0) r += U[idx - nb];
    r = fma(-(TWO_D ? rxd[cx] + ryd[iy] : rxd[cx]), uj, r);
    if (ix > 0) r = fma(-rxl[cx], u[j - 1], r);
    if (ix + 1 < nx) r = fma(-rxu[cx], u[j + 1], r);
    if (TWO_D) {
      if (iy > 0) r = fma(-ryl[iy], u[j - nx], r);
      if (iy + 1 < ny) r = fma(-ryu[iy], u[j + nx], r);
    }
    rr = fma(r, r, rr);
    uu = fma(uj, uj, uu);
  }
  __shared__ double red[kRedWords];
  __shared__ double out[2];
  const double s2[2] = {rr, uu};
  block_sums(s2, 2, red, out);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = out[0];
    part[2 * blockIdx.x + 1] = out[1];
  }
  if (!last_cta_done(flags + F_EARLYCNT)) return;
  if (threadIdx.x == 0) {
    double r2 = 0.0, u2 = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      r2 += __ldcg(part + 2 * b);
      u2 += __ldcg(part + 2 * b + 1);
    }
    const double res = sqrt(r2), un = sqrt(u2);
    scal[S_U1RES] = res;
    scal[S_U1NORM] = un;
    const bool exit = isfinite(res) && res <= eps * un;
    flags[F_EARLY] = exit ? 1 : 0;
    if (exit) {  // U = U_1: no Algorithm 2, no final loop
      flags[F_KSTOP] = 1;
      flags[F_KCONV] = 1;
      flags[F_M] = 0;
      if (use_handle) cudaGraphSetConditional(h, 0u);
    }
    flags[F_EARLYCNT] = 0;
  }
}

void launch_early_check(Ctx &c, const double *G, const double *U, int64_t nt, int64_t ny, int64_t nx,
                        const double *rxl, const double *rxd, const double *rxu, const double *ryl,
                        const double *ryd, const double *ryu, int64_t nym, double eps, double *part, double *scal,
                        int *flags, int use_handle, cudaGraphConditionalHandle h) {
  const int nb = (int)(ny * nx);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((nt * nb + 255) / 256, 4 * (int64_t)sm_count()));
  c.launch("early_check", (double)nt * nb * 16.0, [&] {
    if (ryl)
      pdl_launch(c.pdl, k_early_check<true>, dim3(grid), dim3(256), 0, c.stream, G, U, nt, nb, (int)nx, rxl, rxd, rxu,
                 ryl, ryd, ryu, (int)ny, (int)nym, eps, part, scal, flags, use_handle, h);
    else
      pdl_launch(c.pdl, k_early_check<false>, dim3(grid), dim3(256), 0, c.stream, G, U, nt, nb, (int)nx, rxl, rxd, rxu,
                 ryl, ryd, ryu, (int)ny, (int)nym, eps, part, scal, flags, use_handle, h);
  });
}

// ---- persistent Algorithm-2 step ---------------------------------------------------

// z[j] = sum_k Re(omega_k H[k][j]) (eq. 13's z) over the whole grid: tiles of cw = 512 / rg
// adjacent columns, rg row groups per tile (thread (tx, ty) sums rows ty, ty + rg, ...
// with kZB loads in flight), the groups' partials added pairwise in a fixed order.  The
// weights are rounded once into shared memory (om, nf entries).  With h0 the zero
// frequency comes from the FP64 lane, added in FP64.
constexpr int kZB = 16;
template <typename T>
__device__ void step_zsum(int nf, int n, const cpx<T> *__restrict__ H, int64_t ldh,
                          const double2 *__restrict__ omega, double *z, const double *__restrict__ h0, int rg,
                          cpx<T> *om, T *sm) {
  for (int k = threadIdx.x; k < nf; k += blockDim.x) om[k] = mk<T>((T)omega[k].x, (T)omega[k].y);
  __syncthreads();
  const int cw = (int)blockDim.x / rg;
  const int tx = threadIdx.x % cw, ty = threadIdx.x / cw;
  const int kfirst = h0 ? 1 : 0;
  const int ntile = (n + cw - 1) / cw;
  for (int tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const int j = tile * cw + tx;
    T acc = T(0), acc2 = T(0);
    if (j < n) {
      for (int k0 = ty; k0 < nf; k0 += kZB * rg) {
        cpx<T> hv[kZB];
#pragma unroll
        for (int u = 0; u < kZB; ++u) {
          const int k = k0 + u * rg;
          hv[u] = (k < nf && k >= kfirst) ? H[(int64_t)k * ldh + j] : mk<T>(T(0), T(0));
        }
#pragma unroll
        for (int u = 0; u < kZB; u += 2) {
          const int k = k0 + u * rg, k2 = k + rg;
          if (k < nf) acc += om[k].x * hv[u].x - om[k].y * hv[u].y;
          if (k2 < nf) acc2 += om[k2].x * hv[u + 1].x - om[k2].y * hv[u + 1].y;
        }
      }
    }
    sm[threadIdx.x] = acc + acc2;
    for (int w = rg >> 1; w >= 1; w >>= 1) {
      __syncthreads();
      if (ty < w) sm[threadIdx.x] += sm[threadIdx.x + w * cw];
    }
    __syncthreads();
    if (ty == 0 && j < n) z[j] = h0 ? (double)sm[tx] + omega[0].x * h0[j] : (double)sm[tx];
    __syncthreads();  // sm is rewritten by the next tile
  }
}

// One Algorithm-2 step after its shifted solves (see StepArgs).  The vector phases (eq.
// 13, Arnoldi) run in the first a.nv CTAs, which hold E entries per thread in registers
// (VMODE kSingle: nv = 1, no grid barrier; kPersist: bounded barriers among the nv CTAs
// inside each reduction); the other CTAs leave once z is written.
template <typename T, int VMODE, int E>
__global__ void __launch_bounds__(kBlasSingle, 1) k_step_tail(StepArgs<T> a) {
  BarCtx &bc = bar_ctx();
  int *flags = a.flags;
  if (threadIdx.x == 0) {
    bc.flags = flags;
    bc.limit = a.bar_polls;
    bc.expect = (int)gridDim.x + a.bar_extra;
    bc.use_handle = a.use_handle;
    bc.h = a.h;
    bc.failed = 0;
    bc.nv = a.nv;
  }
  __syncthreads();
  // after a timeout the loop only winds down (a CTA of the failed launch may have set the
  // conditional to run once more before another CTA's timeout set it to stop)
  if (flags[F_TIMEOUT]) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      flags[F_KSTOP] = 1;
      if (a.use_handle) cudaGraphSetConditional(a.h, 0u);
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ T zsm[kBlasSingle];
  bool ok = true;
  if (!flags[F_FROZEN]) {  // a frozen step (q > 1) forms no eq. (12) system and no z
    const int m = flags[F_M] + 1;
    const int nwall = (int)blockDim.x >> 5;
    const int nwk = m == 1 ? nwall : max(1, min(nwall, (int)(a.smem / k5a_warp_bytes(m))));
    capacitance_terms_body(blockIdx.x, gridDim.x, nwk, m, a.nf, a.maxit, a.tau, a.T, a.shift, a.wg, a.gpart, a.nblk,
                           a.msys_part, a.srow, a.scal, flags, 0, 0, smraw, 1, a.sinv);
    if (last_cta_done(flags + F_CAPCNT)) {
      capacitance_solve_cta(a.nf, m, gridDim.x, a.msys_part, a.srow, a.omega, a.y, a.scal, smraw);
      if (threadIdx.x == 0) flags[F_CAPCNT] = 0;
    }
    ok = bounded_grid_sync();  // omega
    if (ok && !flags[F_NOH])   // no z after a breakdown (eq. 13 gives 0)
      step_zsum<T>(a.nf, a.n, a.H, a.ldh, a.omega, a.z, a.h0, a.zrg, reinterpret_cast<cpx<T> *>(smraw), zsm);
    if (ok) ok = bounded_grid_sync((int)blockIdx.x < a.nv);  // z
  }
  if (threadIdx.x == 0) bc.expect = a.nv + a.bar_extra;  // the vector phases' barriers
  if (ok && (int)blockIdx.x < a.nv) {
    project_body<VMODE, E>(a.n, a.V, a.z, a.tau, a.part, a.ld, a.scal, flags, a.kc, a.use_handle, a.h);
    __syncthreads();  // the decision (thread 0 of CTA 0) is read by the whole CTA
    ok = !bc.failed;
    if (VMODE == kPersist && ok) ok = bounded_grid_sync();  // ... and by every vector CTA
    if (ok && !*(volatile int *)(flags + F_KSTOP)) {
      arnoldi_body<VMODE, E>(a.n, a.klo, a.kdiag, a.kup, a.V, a.Vf, a.w, a.T, a.maxit, a.part, a.ld, a.scal, flags,
                             a.q, a.maxit);
      ok = !bc.failed;
    }
  }
  if (!ok && threadIdx.x == 0) {  // the last word on the loop: stop
    flags[F_KSTOP] = 1;
    if (a.use_handle) cudaGraphSetConditional(a.h, 0u);
  }
}

// ---- launchers -------------------------------------------------------------------

// One CTA (plain launch) when the vector is short, else a cooperative launch through
// cudaLaunchKernelEx (capturable into a CUDA graph).
// Cluster variant: one CTA per SM (the dynamic shared memory request keeps a second
// CTA off the SM), kBlasCluster threads each.
constexpr int kClusterSpreadSmem = 120 * 1024;

// Largest cluster size <= want (halving, down to 4: with 128 threads per CTA and at most
// 16 register-held entries per thread, 4 CTAs cover the 8192 entries one CTA would
// take) the device can co-schedule for the cluster variant of the vector kernels; 0 if
// none.
int krylov_cluster_size(int want) {
  const void *fn = (const void *)k_arnoldi_coop<kCluster, 1>;
  cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  allow_dyn_smem((const void *)fn);
  for (int cl = want; cl >= 4; cl >>= 1) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(kBlasCluster);
    cfg.dynamicSmemBytes = kClusterSpreadSmem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) == cudaSuccess && n > 0) return cl;
    cudaGetLastError();
  }
  return 0;
}

// Cooperative grids: entries per thread held in registers (0 = stream from memory when the
// grid's registers cannot hold the vector).
static int coop_elems(int n, int grid) {
  const int64_t threads = (int64_t)grid * kBlas;
  return (int64_t)n > threads * kEMax ? 0 : reg_elems(n, (int)threads);
}
#define PD_COOP_E(E, KERNEL) ((E) == 0 ? (const void *)KERNEL<kCoop, 0> : PD_BY_E(E, KERNEL, kCoop))

#define PD_BY_E(E, KERNEL, MODE)                                                              \
  ((E) <= 1 ? (const void *)KERNEL<MODE, 1>                                                  \
            : (E) == 2 ? (const void *)KERNEL<MODE, 2>                                       \
                       : (E) == 4 ? (const void *)KERNEL<MODE, 4>                            \
                                  : (E) == 8 ? (const void *)KERNEL<MODE, 8> : (const void *)KERNEL<MODE, 16>)

static void coop_launch(Ctx &c, const char *fam, double bytes, const void *fn_single, const void *fn_coop,
                        const void *fn_cluster, int grid, int cluster, void **args) {
  if (grid <= 1 && cluster > 1) {
    cudaFuncSetAttribute(fn_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    allow_dyn_smem((const void *)fn_cluster);
    c.launch(fam, bytes, [&] {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)cluster);
      cfg.blockDim = dim3(kBlasCluster);
      cfg.dynamicSmemBytes = kClusterSpreadSmem;
      cfg.stream = c.stream;
      cudaLaunchAttribute attr[2];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = (unsigned)cluster;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[1].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = c.pdl ? 2 : 1;
      cudaLaunchKernelExC(&cfg, fn_cluster, args);
    });
    return;
  }
  if (grid <= 1) {
    c.launch(fam, bytes, [&] {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(1);
      cfg.blockDim = dim3(kBlasSingle);
      cfg.stream = c.stream;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[0].val.programmaticStreamSerializationAllowed = 1;
      cfg.attrs = attr;
      cfg.numAttrs = c.pdl ? 1 : 0;
      cudaLaunchKernelExC(&cfg, fn_single, args);
    });
    return;
  }
  const void *fn = fn_coop;
  c.launch(fam, bytes, [&] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlas);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelExC(&cfg, fn, args);
  });
}

void launch_vec_norm_init(Ctx &c, KrylovBufs &k, const double *b, int use_handle, cudaGraphConditionalHandle h) {
  const int ld = k.maxit + 2;
  int n = k.n;
  double *part = k.part, *V = k.V, *scal = k.scal;
  float *Vf = k.Vf;
  int *flags = k.flags;
  double *T = k.T;
  int nT = (k.maxit + 1) * k.maxit;
  void *args[] = {(void *)&b, &n, &part, (void *)&ld, &V, &Vf, &scal, &flags, &use_handle, &h, &T, &nT};
  coop_launch(c, "krylov_init", (double)k.n * 16, PD_BY_E(reg_elems(k.n, kBlasSingle), k_init_v0_coop, kSingle),
              PD_COOP_E(coop_elems(k.n, k.grid), k_init_v0_coop),
              PD_BY_E(reg_elems(k.n, k.cluster * kBlasCluster), k_init_v0_coop, kCluster),
              k.grid, k.cluster, args);
}

// Partial buffers: k.part holds three (grid, maxit+2) panels.
void launch_arnoldi(Ctx &c, KrylovBufs &k) {
  const int ld = k.maxit + 2;
  int n = k.n, ldT = k.maxit;
  const double *klo = k.klo, *kdiag = k.kdiag, *kup = k.kup;
  double *V = k.V, *w = k.w, *T = k.T, *part = k.part, *scal = k.scal;
  float *Vf = k.Vf;
  int *flags = k.flags;
  int q = k.q, maxit = k.maxit;
  void *args[] = {&n, (void *)&klo, (void *)&kdiag, (void *)&kup, &V, &Vf, &w, &T, &ldT, &part, (void *)&ld,
                  &scal, &flags, &q, &maxit};
  coop_launch(c, "krylov_arnoldi", (double)k.n * 8.0 * 8, PD_BY_E(reg_elems(k.n, kBlasSingle), k_arnoldi_coop, kSingle),
              PD_COOP_E(coop_elems(k.n, k.grid), k_arnoldi_coop),
              PD_BY_E(reg_elems(k.n, k.cluster * kBlasCluster), k_arnoldi_coop, kCluster),
              k.grid, k.cluster, args);
}

void launch_capacitance(Ctx &c, KrylovBufs &k, int nf, double tau, const double2 *shift, const double2 *wg,
                        const double2 *gpart, int nblk, double *msys_part, int k5_grid, double2 *srow,
                        double2 *omega, double *y, int members, int bpm, double2 *sinv) {
  const size_t smem = k5a_warp_bytes(k.maxit) * kK5Warps;  // sized for the largest m
  allow_dyn_smem((const void *)k_capacitance_terms);
  c.launch("capacitance", (double)nf * nblk * 16, [&] {
    pdl_launch(c.pdl, k_capacitance_terms, dim3(k5_grid, members ? members : 1), dim3(kK5Warps * 32), smem,
               c.stream, nf, k.maxit, tau, (const double *)k.T, shift, wg, gpart, nblk, msys_part, srow,
               members ? k.mscal : k.scal, members ? k.mflags : k.flags, omega, y, members, bpm, sinv);
  });
}

// ||(I - V_m V_m^T) z|| with two CGS passes (z is overwritten by the projection).
void launch_project_resnorm(Ctx &c, KrylovBufs &k, const double *z, double tau, const KrylovCtl &kc0, int use_handle,
                            cudaGraphConditionalHandle h) {
  const int ld = k.maxit + 2;
  int n = k.n;
  const double *V = k.V;
  double *zz = const_cast<double *>(z);
  double *part = k.part, *scal = k.scal;
  int *flags = k.flags;
  KrylovCtl kc = kc0;
  void *args[] = {&n, (void *)&V, &zz, &tau, &part, (void *)&ld, &scal, &flags, &kc, &use_handle, &h};
  coop_launch(c, "krylov_project", (double)k.n * 8.0 * 6, PD_BY_E(reg_elems(k.n, kBlasSingle), k_project_coop, kSingle),
              PD_COOP_E(coop_elems(k.n, k.grid), k_project_coop),
              PD_BY_E(reg_elems(k.n, k.cluster * kBlasCluster), k_project_coop, kCluster),
              k.grid, k.cluster, args);
}

// Dynamic shared memory of the persistent step: the capacitance phase's warp slices (up to
// four sized for the largest m, within 150 KB; more warps join while m is small), its m x m
// solve, and the z weights.
size_t step_tail_smem(int maxit, int nf, int elem_bytes) {
  const size_t solve = (size_t)(2 * maxit * maxit + maxit) * sizeof(cpx<double>) + (size_t)(maxit + 1) * 8;
  const size_t wb = k5a_warp_bytes(maxit);
  const size_t terms = wb * std::max<size_t>(1, std::min<size_t>(kK5Warps, (150 * 1024) / wb));
  const size_t om = (size_t)nf * 2 * elem_bytes;
  return (std::max(std::max(solve, terms), om) + 15) & ~(size_t)15;
}

// nv = 1: the vector phases in one CTA without grid barriers (E = 1: n_bar <= 512)
template <typename T>
static const void *step_tail_fn(int nv, int E) {
  if (nv <= 1) return (const void *)k_step_tail<T, kSingle, 1>;
  return E <= 1 ? (const void *)k_step_tail<T, kPersist, 1>
       : E == 2 ? (const void *)k_step_tail<T, kPersist, 2>
                : (const void *)k_step_tail<T, kPersist, 4>;
}

static const void *step_tail_pick(int nv, int E, int elem_bytes) {
  return elem_bytes == 8 ? step_tail_fn<double>(nv, E) : step_tail_fn<float>(nv, E);
}

int step_tail_max_grid(int nv, int E, int elem_bytes, size_t smem) {
  const void *fn = step_tail_pick(nv, E, elem_bytes);
  if ((int64_t)smem > (int64_t)allow_dyn_smem(fn)) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBlasSingle, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sm_count();
}

template <typename T>
void launch_step_tail(Ctx &c, const StepArgs<T> &a0, int grid, int E) {
  const void *fn = step_tail_pick(a0.nv, E, (int)sizeof(T));
  allow_dyn_smem((const void *)fn);
  StepArgs<T> a = a0;
  void *args[] = {&a};
  // algorithmic bytes: the stored h_k read once by the z sum
  c.launch("krylov_step", (double)a.nf * a.n * sizeof(cpx<T>), [&] {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kBlasSingle);
    cfg.dynamicSmemBytes = a.smem;
    cfg.stream = c.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelExC(&cfg, fn, args);
  });
}
template void launch_step_tail<float>(Ctx &, const StepArgs<float> &, int, int);
template void launch_step_tail<double>(Ctx &, const StepArgs<double> &, int, int);

void launch_xm(Ctx &c, KrylovBufs &k, const double *y, double *x, float *xf) {
  c.launch("krylov_xm", (double)k.n * 8.0 * 2,
           [&] { pdl_launch(c.pdl, k_xm, dim3(k.grid), dim3(kBlas), 0, c.stream, k.n, (const int *)k.flags, (const double *)k.V,
                                y, x, xf); });
}

template <typename T>
void launch_final_comb(Ctx &c, int nf, int64_t n, int64_t lds, double tau, double aroot, const double2 *shift,
                       const double *Tm, const double *y, const double *V, const T *Vb, const double *scal,
                       int *flags, const double2 *sinv, int maxm, const cpx<T> *L, const cpx<T> *H, cpx<T> *S,
                       double *x) {
  const dim3 grid((unsigned)(nf + 1), (unsigned)std::min<int64_t>((n + kCombCols - 1) / kCombCols, 65535));
  const int mm = std::min(maxm, kCombMaxM);
  // algorithmic bytes: L and h_k read, S written (when the final loop is formed here)
  c.launch("final_comb", (double)nf * n * 3.0 * sizeof(cpx<T>), [&] {
    pdl_launch(c.pdl, k_final_comb<T>, grid, dim3(256), 0, c.stream, nf, n, lds, tau, aroot, shift, Tm, y, V, Vb,
               scal, flags, sinv, mm, L, H, S, x);
  });
}
template void launch_final_comb<float>(Ctx &, int, int64_t, int64_t, double, double, const double2 *,
                                       const double *, const double *, const double *, const float *,
                                       const double *, int *, const double2 *, int, const cpx<float> *,
                                       const cpx<float> *, cpx<float> *, double *);
template void launch_final_comb<double>(Ctx &, int, int64_t, int64_t, double, double, const double2 *,
                                        const double *, const double *, const double *, const double *,
                                        const double *, int *, const double2 *, int, const cpx<double> *,
                                        const cpx<double> *, cpx<double> *, double *);

void launch_sumsq(Ctx &c, const double *part, int nparts, double *dst) {
  c.launch("krylov_sumsq", 0.0, [&] { pdl_launch(c.pdl, k_sumsq_final, dim3(1), dim3(32), 0, c.stream, part, nparts, dst); });
}

}  // namespace pd
