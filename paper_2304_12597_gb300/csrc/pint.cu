// Parallel-in-time loop of Algorithms 1 and 2: for every frequency k of the half
// spectrum, solve the shifted system ((1 - pi_k) I + tau K) y_k = r_k (Sec. 2,
// the block-diagonal P), with K tridiagonal (in 2D: block-decoupled tridiagonal
// after the DST along y).  The ~l/2 systems are independent; pi_{l-k} =
// conj(pi_k) makes the other half the complex conjugate.
//
// One team of P threads solves one tridiagonal block of `blen` rows:
//  1. the right-hand side is staged in shared memory with coalesced loads;
//  2. each thread eliminates its chunk of M rows so that every interior row
//     depends only on the chunk's first and last unknowns (partitioned Thomas);
//  3. the 2P first/last rows form a tridiagonal interface system, solved by
//     parallel cyclic reduction (PCR) in shared memory;
//  4. each thread back-substitutes its interior rows.
// Elimination is without pivoting: (1 - pi_k) has nonnegative real part and
// tau K is positive real for the operators in scope, so every pivot stays away
// from zero (the same argument as for Thomas on these matrices).
//
// Fused epilogues (per frequency k, in FP64):
//  - acc += Re(omega_k y_k): b = sum_i gamma_i L_i (eq. 7) with omega_k = w_k gamma_k,
//    and z = sum_i gamma_i h_i (e_m^T S_i y_m) (eq. 13) with omega_k = w_k gamma_k c_k,
//    w_k = 1 for k = 0, l/2 and 2 otherwise (the conjugate half);
//  - dots g_k = V_m^T h_k needed by eq. (12);
//  - optional store of y_k (the final loop of Algorithm 1).
// A team handles one block and a contiguous range of k, so its accumulators stay
// on chip; the per-team partial rows are reduced in a fixed order afterwards.
#include <algorithm>

#include "pd_internal.h"
#include "pd_krylov.cuh"

namespace pd {

template <typename T, int M>
struct TeamSmem {
  // staged coefficients tau*K (lo, diag, up), padded like the right-hand side
  __host__ __device__ static size_t stage_bytes(int P, int stage) {
    return stage ? (((size_t)3 * P * (M + 1) * sizeof(T) + 15) & ~(size_t)15) : 0;
  }
  // exchange rows of P: the eliminating loop double-buffers its PCR (8) unless its team
  // is one warp; the factored loop needs one buffer (5)
  __host__ __device__ static int xrows(int P, bool fact) { return (fact || P < 64) ? 5 : 8; }
  // fact: the factored loop
  static size_t bytes(int P, int mdots, int stage, bool fact = false) {
    size_t b = stage_bytes(P, stage);
    b += (size_t)P * (M + 1) * sizeof(cpx<T>);   // rhs / dd, padded one slot per chunk
    b += (size_t)P * xrows(P, fact) * sizeof(cpx<T>);  // condensed rows a, c, d, 1/b
    b += ((size_t)P * M * sizeof(T) + 15) & ~(size_t)15;  // per-team accumulators (compute type)
    b += (size_t)(P / 32) * std::max(mdots, 1) * sizeof(double2);  // dot reductions
    return (b + 15) & ~(size_t)15;
  }
};

// Precomputed factors of one frequency's shifted system (they depend on k and K only,
// not on the right-hand side): per block and team thread t, the complex values below,
// slot s of thread t at ((k nblk + blk) NS + s) P + t, so a warp reads 256 contiguous
// bytes per slot.  Chunk rows i = 1..M-1 and PCR levels l = 0..L-1 (P = 2^L):
//   rd_i   pivot reciprocals of the chunk elimination          slots 0 .. M-2
//   ccf_i  forward cc_i (i <= M-3), for the backward sweep       M-1 .. 2M-5
//   C0     the interface row's coupling to xe_t                   2M-4
//   aa_i, cc_i after the backward sweep (back substitution)     2M-3 .. 4M-6
//   k1_l, k2_l  PCR multipliers (zero past the team's ends)     4M-5 + 2l, +1
//   1/B    of the reduced interface row                           4M-5 + 2L
template <int M>
__host__ __device__ constexpr int fs_rd(int i) { return i - 1; }
template <int M>
__host__ __device__ constexpr int fs_ccf(int i) { return M - 1 + i - 1; }
template <int M>
__host__ __device__ constexpr int fs_c0() { return 2 * M - 4; }
template <int M>
__host__ __device__ constexpr int fs_aa(int i) { return 2 * M - 3 + i - 1; }
template <int M>
__host__ __device__ constexpr int fs_cc(int i) { return 3 * M - 4 + i - 1; }
template <int M>
__host__ __device__ constexpr int fs_k1(int l) { return 4 * M - 5 + 2 * l; }
template <int M>
__host__ __device__ constexpr int fs_binv(int L) { return 4 * M - 5 + 2 * L; }
__host__ __device__ inline int ilog2_pow2(int P) {
  int L = 0;
  while ((1 << L) < P) ++L;
  return L;
}
// slots per (k, block, thread)
__host__ __device__ inline int fac_slots(int M, int P) { return 4 * M - 4 + 2 * ilog2_pow2(P); }

size_t pint_factor_elems(const PintGeom &g) {
  return (size_t)g.nf * g.nblk * fac_slots(g.M, g.P) * g.P;
}
size_t pint_k0_factor_elems(const PintGeom &g) { return (size_t)g.nblk * fac_slots(g.M, g.P) * g.P; }

template <typename T>
__device__ __forceinline__ void coef(const PintArgs<T> &a, const T *cs, int cs_stride, int64_t j, int ps, bool valid,
                                     cpx<T> s, T &lo, cpx<T> &d, T &up) {
  if (valid) {
    if (cs) {  // staged in shared memory at padded index ps
      lo = cs[ps];
      d = mk<T>(s.x + cs[cs_stride + ps], s.y);
      up = cs[2 * cs_stride + ps];
    } else {
      lo = a.tlo[j];
      up = a.tup[j];
      d = mk<T>(s.x + a.tdiag[j], s.y);
    }
  } else {
    lo = T(0);
    up = T(0);
    d = mk<T>(T(1), T(0));
  }
}

// Zero-frequency lane of the binary32 path (PintArgs::k0_fp64): the team's block of
// (s_0 I + tau K) y = r in FP64, with the real shift s_0 = 1 - pi_0 = 1 - alpha^{1/l} and
// real data (the zero frequency of real time series is real).  Same partitioned Thomas +
// PCR as the complex solve below, in real FP64 arithmetic, reusing the team's shared
// memory: a double takes the bytes of a cpx<float>.  Its factors depend on K only, so a
// factor pass (fac0_out) stores them once per operator in the slot layout of the complex
// factors (fs_*), and every loop (fac0_in) applies them to its right-hand side: about six
// FP64 operations per row and no division, so the lane stays off the kernel's critical
// path on GB300's slow FP64 pipe.  The right-hand side: the spectrum row R[0] (its real
// part) minus xm_scale x_m with x_m = V_m y_m in FP64 (final loop), or v_{m+1} of the FP64
// basis (dots pass).  Epilogues in FP64: acc0 = omega_0 y (b of eq. 7), h0 = y and the dots
// g_0 = V_m^T y (eq. 12), and the binary32 store of y into Y[0].
template <int M>
__device__ void pint_k0_lane(const PintGeom &g, const PintArgs<float> &a, int P, int t, int tic, int64_t off,
                             int blen, int blk, cpx<float> *dd_f, cpx<float> *px_f, double2 *red) {
  double *dd = reinterpret_cast<double *>(dd_f);
  double *pa = reinterpret_cast<double *>(px_f), *pc = pa + P, *pd = pc + P, *pib = pd + P;
  const double s0 = a.shift[0].x;
  const int NS = fac_slots(M, P);
  double *Fo = a.fac0_out ? a.fac0_out + (int64_t)blk * NS * P + t : nullptr;
  const double *Fi = a.fac0_in ? a.fac0_in + (int64_t)blk * NS * P + t : nullptr;
  // 1. stage the right-hand side (element e at dd[e + e/M])
  const double *vrhs = nullptr;
  int mdots = 0;
  if (a.mcount) {
    const int m = *a.mcount + 1;
    vrhs = a.Vd + (int64_t)m * a.ldv + off;
    mdots = a.want_dots ? m : 0;
  } else if (a.V) {
    mdots = a.mdots;
  }
  if (!a.Vd) mdots = 0;
  const int mx = a.xm_count ? *a.xm_count : 0;
  const double *xy = a.xm_count ? a.xm_y + (int64_t)(blk / (a.xm_bpm > 1 ? a.xm_bpm : 1)) * a.xm_ldy : nullptr;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int e = t + i * P;
    double v = 0.0;
    if (e < blen) {
      if (a.R) {
        v = (double)a.R[off + e].x;
        if (xy) {
          double xm = 0.0;
          for (int q = 0; q < mx; ++q) xm += xy[q] * a.Vd[(int64_t)q * a.ldv + off + e];
          v -= a.xm_scale * xm;
        } else if (a.rvec) {
          v -= (double)a.rvec[off + e];
        }
      } else if (vrhs) {
        v = vrhs[e];
      } else if (a.rvec) {
        v = (double)a.rvec[off + e];
      }
    }
    dd[e + e / M] = v;
  }
  team_sync(P, tic);
  double *my = dd + (size_t)t * (M + 1);
  const int e0 = t * M;
  auto lo_of = [&](int i) { return e0 + i < blen ? a.tlo_d[off + e0 + i] : 0.0; };
  auto up_of = [&](int i) { return e0 + i < blen ? a.tup_d[off + e0 + i] : 0.0; };
  auto d_of = [&](int i) { return e0 + i < blen ? s0 + a.tdiag_d[off + e0 + i] : 1.0; };
  double r[M];
#pragma unroll
  for (int i = 0; i < M; ++i) r[i] = my[i];
  const double lo0 = lo_of(0), up0 = up_of(0);
  double xf, xl, D1, A1, C1;
  double aa[M], cc[M];
  if (Fi) {
    // 2-4 with the stored factors: the same elimination, PCR and back substitution applied
    // to the right-hand side only
    r[1] *= Fi[fs_rd<M>(1) * P];
#pragma unroll
    for (int i = 2; i < M; ++i) r[i] = (r[i] - lo_of(i) * r[i - 1]) * Fi[fs_rd<M>(i) * P];
#pragma unroll
    for (int i = M - 3; i >= 1; --i) r[i] -= Fi[fs_ccf<M>(i) * P] * r[i + 1];
    const double D0 = r[0] - up0 * r[1];
    D1 = r[M - 1];
    pd[t] = D1;
    team_sync(P, tic);
    const double pD1 = t > 0 ? pd[t - 1] : 0.0;
    double D = D0 - lo0 * pD1 - Fi[fs_c0<M>() * P] * D1;
    team_sync(P, tic);
    int l = 0;
    for (int sig = 1; sig < P; sig <<= 1, ++l) {
      pd[t] = D;
      team_sync(P, tic);
      double nD = D;
      if (t - sig >= 0) nD -= Fi[fs_k1<M>(l) * P] * pd[t - sig];
      if (t + sig < P) nD -= Fi[(fs_k1<M>(l) + 1) * P] * pd[t + sig];
      team_sync(P, tic);
      D = nD;
    }
    xf = D * Fi[fs_binv<M>(l) * P];
    pd[t] = xf;
    team_sync(P, tic);
    const double xnext = t + 1 < P ? pd[t + 1] : 0.0;
    xl = D1 - Fi[fs_aa<M>(M - 1) * P] * xf - Fi[fs_cc<M>(M - 1) * P] * xnext;
    my[0] = xf;
#pragma unroll
    for (int i = 1; i < M - 1; ++i) my[i] = r[i] - Fi[fs_aa<M>(i) * P] * xf - Fi[fs_cc<M>(i) * P] * xl;
    my[M - 1] = xl;
  } else {
    // 2. chunk elimination: row i becomes x_i + aa_i x_0 + cc_i x_{M-1} = r_i (factors
    // stored when Fo is set)
    const double d0 = d_of(0);
    {
      const double rb = 1.0 / d_of(1);
      aa[1] = lo_of(1) * rb;
      cc[1] = up_of(1) * rb;
      r[1] *= rb;
      if (Fo) {
        Fo[fs_rd<M>(1) * P] = rb;
        if (1 <= M - 3) Fo[fs_ccf<M>(1) * P] = cc[1];
      }
    }
#pragma unroll
    for (int i = 2; i < M; ++i) {
      const double lo = lo_of(i);
      const double rd = 1.0 / (d_of(i) - lo * cc[i - 1]);
      aa[i] = -lo * aa[i - 1] * rd;
      cc[i] = up_of(i) * rd;
      r[i] = (r[i] - lo * r[i - 1]) * rd;
      if (Fo) {
        Fo[fs_rd<M>(i) * P] = rd;
        if (i <= M - 3) Fo[fs_ccf<M>(i) * P] = cc[i];
      }
    }
#pragma unroll
    for (int i = M - 3; i >= 1; --i) {
      aa[i] -= cc[i] * aa[i + 1];
      r[i] -= cc[i] * r[i + 1];
      cc[i] = -cc[i] * cc[i + 1];
    }
    const double A0 = lo0, B0 = d0 - up0 * aa[1], C0 = -up0 * cc[1], D0 = r[0] - up0 * r[1];
    A1 = aa[M - 1];
    C1 = cc[M - 1];
    D1 = r[M - 1];
    if (Fo) {
      Fo[fs_c0<M>() * P] = C0;
#pragma unroll
      for (int i = 1; i < M; ++i) {
        Fo[fs_aa<M>(i) * P] = aa[i];
        Fo[fs_cc<M>(i) * P] = cc[i];
      }
    }
    // 3a. eliminate the chunks' last unknowns: P interface rows in the first unknowns
    pa[t] = A1;
    pc[t] = C1;
    pd[t] = D1;
    team_sync(P, tic);
    double A, B, C, D;
    {
      const double pA1 = t > 0 ? pa[t - 1] : 0.0, pC1 = t > 0 ? pc[t - 1] : 0.0, pD1 = t > 0 ? pd[t - 1] : 0.0;
      A = -A0 * pA1;
      B = B0 - A0 * pC1 - C0 * A1;
      C = -C0 * C1;
      D = D0 - A0 * pD1 - C0 * D1;
    }
    team_sync(P, tic);
    // 3b. PCR on the interface rows (one buffer, two barriers per level)
    int l = 0;
    for (int sig = 1; sig < P; sig <<= 1, ++l) {
      pa[t] = A;
      pc[t] = C;
      pd[t] = D;
      pib[t] = 1.0 / B;
      team_sync(P, tic);
      double nA = 0.0, nB = B, nC = 0.0, nD = D, k1 = 0.0, k2 = 0.0;
      if (t - sig >= 0) {
        k1 = A * pib[t - sig];
        nA = -k1 * pa[t - sig];
        nB -= k1 * pc[t - sig];
        nD -= k1 * pd[t - sig];
      }
      if (t + sig < P) {
        k2 = C * pib[t + sig];
        nC = -k2 * pc[t + sig];
        nB -= k2 * pa[t + sig];
        nD -= k2 * pd[t + sig];
      }
      if (Fo) {
        Fo[fs_k1<M>(l) * P] = k1;
        Fo[(fs_k1<M>(l) + 1) * P] = k2;
      }
      team_sync(P, tic);
      A = nA;
      B = nB;
      C = nC;
      D = nD;
    }
    const double rB = 1.0 / B;
    if (Fo) Fo[fs_binv<M>(l) * P] = rB;
    xf = D * rB;
    pd[t] = xf;
    team_sync(P, tic);
    const double xnext = t + 1 < P ? pd[t + 1] : 0.0;
    xl = D1 - A1 * xf - C1 * xnext;
    // 4. back substitution
    my[0] = xf;
#pragma unroll
    for (int i = 1; i < M - 1; ++i) my[i] = r[i] - aa[i] * xf - cc[i] * xl;
    my[M - 1] = xl;
  }
  team_sync(P, tic);
  // 5. epilogues, coalesced
  const double om = a.omega ? a.omega[0].x : 0.0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const int e = t + i * P;
    if (e < blen) {
      const double y = dd[e + e / M];
      if (a.omega && a.acc0) a.acc0[off + e] = om * y;
      if (a.h0) a.h0[off + e] = y;
      if (a.Y) a.Y[off + e] = mk<float>((float)y, 0.0f);
    }
  }
  if (mdots > 0) {
    const int nw = P >> 5, w = t >> 5, l = t & 31;
    for (int q = 0; q < mdots; ++q) {
      const double *vq = a.Vd + (int64_t)q * a.ldv + off;
      double sq = 0.0;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const int e = t + i * P;
        if (e < blen) sq += vq[e] * dd[e + e / M];
      }
      sq = warp_sum(sq);
      if (l == 0) red[w * mdots + q] = make_double2(sq, 0.0);
    }
    team_sync(P, tic);
    for (int q = t; q < mdots; q += P) {
      double sx = 0.0;
      for (int i = 0; i < nw; ++i) sx += red[i * mdots + q].x;
      a.gpart[((int64_t)0 * g.nblk + blk) * mdots + q] = make_double2(sx, 0.0);
    }
  }
  team_sync(P, tic);
}

// MAXT: the launch's thread count is at most MAXT (256 leaves room for 255
// registers per thread, which the FP64 variants use without spilling).
// FACT: solve with a.fac_in (a separate instantiation, so that its register budget is
// its own).
template <typename T, int M, int MAXT, bool FACT>
__global__ void __launch_bounds__(MAXT) k_pint(PintGeom g, PintArgs<T> a, size_t team_bytes) {
  grid_dep_wait();
  if (a.skip_flag && *a.skip_flag) return;
  if (a.skip_flag2 && *a.skip_flag2) return;
  const int P = g.P;
  const int tic = threadIdx.x / P;
  const int t = threadIdx.x - tic * P;
  const int team = blockIdx.x * g.teams_per_cta + tic;
  const bool active = team < g.nblk * g.R;  // idle teams stay for the CTA-level sum
  const int blk = active ? team / g.R : 0;
  const int rr = team - blk * g.R;
  int k0 = active ? (int)((int64_t)rr * g.nf / g.R) : 0;
  int k1 = active ? (int)((int64_t)(rr + 1) * g.nf / g.R) : 0;
  if (active && a.k0_fp64 && g.R >= 2 && g.nf >= 2) {
    // the zero-frequency lane (FP64) is a team's whole share; the other teams split
    // k = 1..nf-1
    k0 = rr == 0 ? 0 : 1 + (int)((int64_t)(rr - 1) * (g.nf - 1) / (g.R - 1));
    k1 = rr == 0 ? 1 : 1 + (int)((int64_t)rr * (g.nf - 1) / (g.R - 1));
  }
  if (a.fac0_out) k1 = (k0 == 0 && k1 > 0) ? 1 : k0;  // the lane's factor pass: frequency 0 only
  const int blen = g.blen;
  const int64_t off = (int64_t)blk * blen;
  const int N = P;  // condensed interface rows
  const cpx<T> *fin = FACT ? a.fac_in : nullptr;  // precomputed factors (right-hand side only)
  cpx<T> *fout = a.fac_out;      // store the factors (the right-hand side is zero)
  const int NS = fac_slots(M, P);
  // elements per batch of back-to-back loads (fewer in FP64, where registers are scarcer)
  constexpr int SB = sizeof(T) == 8 ? (M < 4 ? M : 4) : M;

  extern __shared__ __align__(16) unsigned char smraw[];
  unsigned char *base = smraw + (size_t)tic * team_bytes;
  T *cs = g.stage ? reinterpret_cast<T *>(base) : nullptr;
  const int cs_stride = P * (M + 1);
  cpx<T> *dd = reinterpret_cast<cpx<T> *>(base + TeamSmem<T, M>::stage_bytes(P, g.stage));
  cpx<T> *pa = dd + (size_t)P * (M + 1);
  cpx<T> *pb = pa + N;
  cpx<T> *pc = pb + N;
  cpx<T> *pd = pc + N;
  cpx<T> *pib = pd + N;
  // second PCR buffer (a, c, d, 1/b): levels alternate buffers, one barrier per level
  cpx<T> *qa = pb, *qc = pib + N, *qd = qc + N, *qib = qd + N;
  T *acc = reinterpret_cast<T *>(pa + (size_t)N * TeamSmem<T, M>::xrows(P, FACT));
  double2 *red = reinterpret_cast<double2 *>(reinterpret_cast<unsigned char *>(acc) +
                                             (((size_t)P * M * sizeof(T) + 15) & ~(size_t)15));

  // right-hand-side vector and number of dots: fixed, or from the device step count
  const T *rvec = a.rvec;
  int mdots = a.V ? a.mdots : 0;
  if (a.mcount) {
    const int m = *a.mcount + 1;  // v_m of the step in progress
    rvec = a.V + (int64_t)m * a.ldv;
    mdots = a.want_dots ? m : 0;
  }
  const bool do_acc = a.omega != nullptr;
  if (do_acc) {
#pragma unroll
    for (int i = 0; i < M; ++i) acc[i * P + t] = T(0);
  }
  cpx<T> *my = dd + (size_t)t * (M + 1);
  const int e0 = t * M;
  const int ps0 = t * (M + 1);  // padded index of this thread's first row
  if (cs && k0 < k1) {
    // tau K does not depend on k: stage the team's block once (read after the first
    // team barrier of the k loop)
#pragma unroll
    for (int i0 = 0; i0 < M; i0 += SB) {
      T lo[SB], di[SB], up[SB];
#pragma unroll
      for (int i = 0; i < SB; ++i) {
        const int e = t + (i0 + i) * P;
        const bool in = e < blen;
        lo[i] = in ? a.tlo[off + e] : T(0);
        di[i] = in ? a.tdiag[off + e] : T(0);
        up[i] = in ? a.tup[off + e] : T(0);
      }
#pragma unroll
      for (int i = 0; i < SB; ++i) {
        const int e = t + (i0 + i) * P;
        const int pe = e + e / M;
        cs[pe] = lo[i];
        cs[cs_stride + pe] = di[i];
        cs[2 * cs_stride + pe] = up[i];
      }
    }
  }

  // Thread t owns elements e = t + i P (i < M) of the block in every load loop
  // below; each loop issues all its global loads before using them, so a thread
  // waits for one memory latency per loop rather than one per element.

  // x_m = V_m y_m for the team's rows (final loop of Algorithm 1; Algorithm 3 weights
  // it by alpha^{1/l}), kept in the accumulator region, which this pass does not
  // otherwise use
  T *xs = nullptr;
  if (a.xm_count && active) {
    xs = acc;
    const int m = *a.xm_count;
    // per-member y_m in batched plans (a member owns xm_bpm consecutive blocks)
    const double *xy = a.xm_y + (int64_t)(blk / (a.xm_bpm > 1 ? a.xm_bpm : 1)) * a.xm_ldy;
    T v[M];
#pragma unroll
    for (int i = 0; i < M; ++i) v[i] = T(0);
    for (int q = 0; q < m; ++q) {
      const T yq = (T)xy[q];
      const T *vq = a.V + (int64_t)q * a.ldv + off;
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (t + i * P < blen) v[i] += yq * vq[t + i * P];
    }
    const T xsc = (T)a.xm_scale;
#pragma unroll
    for (int i = 0; i < M; ++i) xs[t + i * P] = xsc * v[i];
    if (rr == 0 && a.xm_out) {
      double vd[M];
#pragma unroll
      for (int i = 0; i < M; ++i) vd[i] = 0.0;
      for (int q = 0; q < m; ++q) {
        const double yq = xy[q];
        const double *vq = a.xm_Vd + (int64_t)q * a.ldv + off;
#pragma unroll
        for (int i = 0; i < M; ++i)
          if (t + i * P < blen) vd[i] += yq * vq[t + i * P];
      }
#pragma unroll
      for (int i = 0; i < M; ++i)
        if (t + i * P < blen) a.xm_out[off + t + i * P] = vd[i];
    }
  }

  for (int k = k0; k < k1; ++k) {
    if constexpr (sizeof(T) == 4) {
      if (k == 0 && a.k0_fp64) {
        pint_k0_lane<M>(g, a, P, t, tic, off, blen, blk, dd, pa, red);
        continue;
      }
    }
    // the shift in the compute type (binary32 plans keep a converted copy: no FP64-pipe
    // conversion per frequency on GB300)
    cpx<T> s;
    if (a.shift_t) {
      s = a.shift_t[k];
    } else {
      const double2 sk = a.shift[k];
      s = mk<T>((T)sk.x, (T)sk.y);
    }
    const cpx<T> *Rk = a.R ? a.R + (int64_t)k * a.ldr + off : nullptr;  // this block's row of R
    const T *rv = rvec ? rvec + off : nullptr;
    // 1. stage the right-hand side (element e at dd[e + e/M])
#pragma unroll
    for (int i0 = 0; i0 < M; i0 += SB) {
      cpx<T> v[SB];
      T sub[SB];
#pragma unroll
      for (int i = 0; i < SB; ++i) {
        const int e = t + (i0 + i) * P;
        v[i] = mk<T>(T(0), T(0));
        sub[i] = T(0);
        if (e < blen) {
          if (Rk) {
            v[i] = Rk[e];
            if (xs)
              sub[i] = xs[e];
            else if (rv)
              sub[i] = rv[e];
          } else if (rv) {
            v[i].x = rv[e];
          }
        }
      }
#pragma unroll
      for (int i = 0; i < SB; ++i) {
        const int e = t + (i0 + i) * P;
        v[i].x -= sub[i];
        dd[e + e / M] = v[i];
      }
    }
    team_sync(P, tic);

    if constexpr (FACT) {
      // 2-4 with the frequency's factors precomputed (fac_slot layout): the same
      // elimination, PCR and back substitution applied to the right-hand side only
      const cpx<T> *F = fin + ((int64_t)k * g.nblk + blk) * ((int64_t)NS * P) + t;
      T lo0, up0;
      cpx<T> d0;
      coef(a, cs, cs_stride, off + e0, ps0, e0 < blen, s, lo0, d0, up0);
      cpx<T> r[M];
#pragma unroll
      for (int i = 0; i < M; ++i) r[i] = my[i];
      r[1] = mul(r[1], F[fs_rd<M>(1) * P]);
#pragma unroll
      for (int i = 2; i < M; ++i) {
        T lo, up;
        cpx<T> d;
        coef(a, cs, cs_stride, off + e0 + i, ps0 + i, e0 + i < blen, s, lo, d, up);
        r[i] = mul(fnms_r(r[i], lo, r[i - 1]), F[fs_rd<M>(i) * P]);
      }
#pragma unroll
      for (int i = M - 3; i >= 1; --i) r[i] = fnms(r[i], F[fs_ccf<M>(i) * P], r[i + 1]);
      const cpx<T> D0 = fnms_r(r[0], up0, r[1]);
      const cpx<T> D1 = r[M - 1];
      pd[t] = D1;
      team_sync(P, tic);
      const cpx<T> pD1 = t > 0 ? pd[t - 1] : mk<T>(T(0), T(0));
      cpx<T> D = fnms(fnms_r(D0, lo0, pD1), F[fs_c0<M>() * P], D1);
      // PCR on the right-hand side, double-buffered in pa / pb (one barrier per level)
      int l = 0;
      for (int sig = 1; sig < P; sig <<= 1, ++l) {
        cpx<T> *bw = (l & 1) ? pb : pa;
        bw[t] = D;
        team_sync(P, tic);
        cpx<T> nD = D;
        if (t - sig >= 0) nD = fnms(nD, F[fs_k1<M>(l) * P], bw[t - sig]);
        if (t + sig < P) nD = fnms(nD, F[(fs_k1<M>(l) + 1) * P], bw[t + sig]);
        D = nD;
      }
      const cpx<T> xf = mul(D, F[fs_binv<M>(l) * P]);
      pd[t] = xf;
      team_sync(P, tic);
      const cpx<T> xnext = t + 1 < P ? pd[t + 1] : mk<T>(T(0), T(0));
      const cpx<T> xl = fnms(fnms(D1, F[fs_aa<M>(M - 1) * P], xf), F[fs_cc<M>(M - 1) * P], xnext);
      my[0] = xf;
#pragma unroll
      for (int i = 1; i < M - 1; ++i) my[i] = fnms(fnms(r[i], F[fs_aa<M>(i) * P], xf), F[fs_cc<M>(i) * P], xl);
      my[M - 1] = xl;
    } else {
    // 2. chunk elimination: row i of the chunk becomes x_i + aa_i x_0 + cc_i x_{M-1} = dd_i
    cpx<T> aa[M], cc[M];
    // with fout: this frequency's factors are stored (RHS-independent; see fac_slot)
    cpx<T> *F = fout ? fout + ((int64_t)k * g.nblk + blk) * ((int64_t)NS * P) + t : nullptr;
    T lo0, up0;
    cpx<T> d0;
    coef(a, cs, cs_stride, off + e0, ps0, e0 < blen, s, lo0, d0, up0);
    const cpx<T> r0 = my[0];
    {
      T lo, up;
      cpx<T> d;
      coef(a, cs, cs_stride, off + e0 + 1, ps0 + 1, e0 + 1 < blen, s, lo, d, up);
      const cpx<T> rb = recip(d);
      aa[1] = scal(lo, rb);
      cc[1] = scal(up, rb);
      my[1] = mul(my[1], rb);
      if (F) {
        F[fs_rd<M>(1) * P] = rb;
        if (1 <= M - 3) F[fs_ccf<M>(1) * P] = cc[1];
      }
    }
#pragma unroll
    for (int i = 2; i < M; ++i) {
      T lo, up;
      cpx<T> d;
      coef(a, cs, cs_stride, off + e0 + i, ps0 + i, e0 + i < blen, s, lo, d, up);
      const cpx<T> rd = recip(fnms_r(d, lo, cc[i - 1]));
      aa[i] = scal(-lo, mul(aa[i - 1], rd));
      cc[i] = scal(up, rd);
      my[i] = mul(fnms_r(my[i], lo, my[i - 1]), rd);
      if (F) {
        F[fs_rd<M>(i) * P] = rd;
        if (i <= M - 3) F[fs_ccf<M>(i) * P] = cc[i];
      }
    }
#pragma unroll
    for (int i = M - 3; i >= 1; --i) {
      aa[i] = fnms(aa[i], cc[i], aa[i + 1]);
      my[i] = fnms(my[i], cc[i], my[i + 1]);
      const cpx<T> c2 = mul(cc[i], cc[i + 1]);
      cc[i] = mk<T>(-c2.x, -c2.y);
    }
    // interface rows: first row of the chunk (unknown xs_t) couples xe_{t-1}, xs_t, xe_t;
    // last row (unknown xe_t, unit diagonal) couples xs_t, xe_t, xs_{t+1}
    const cpx<T> A0 = mk<T>(lo0, T(0));
    const cpx<T> B0 = fnms_r(d0, up0, aa[1]);
    const cpx<T> C0 = scal(-up0, cc[1]);
    const cpx<T> D0 = fnms_r(r0, up0, my[1]);
    const cpx<T> A1 = aa[M - 1];
    const cpx<T> C1 = cc[M - 1];
    if (F) {
      F[fs_c0<M>() * P] = C0;
#pragma unroll
      for (int i = 1; i < M; ++i) {
        F[fs_aa<M>(i) * P] = aa[i];
        F[fs_cc<M>(i) * P] = cc[i];
      }
    }
    const cpx<T> D1 = my[M - 1];

    // 3a. eliminate every xe with the last rows: P rows in the xs alone, one per thread
    pa[t] = A1;
    pc[t] = C1;
    pd[t] = D1;
    team_sync(P, tic);
    cpx<T> A, B, C, D;
    {
      const cpx<T> z = mk<T>(T(0), T(0));
      const cpx<T> pA1 = t > 0 ? pa[t - 1] : z, pC1 = t > 0 ? pc[t - 1] : z, pD1 = t > 0 ? pd[t - 1] : z;
      // xe_{t-1} = pD1 - pA1 xs_{t-1} - pC1 xs_t ;  xe_t = D1 - A1 xs_t - C1 xs_{t+1}
      A = mul(A0, pA1);
      A = mk<T>(-A.x, -A.y);
      B = fnms(fnms(B0, A0, pC1), C0, A1);
      C = mul(C0, C1);
      C = mk<T>(-C.x, -C.y);
      D = fnms(fnms(D0, A0, pD1), C0, D1);
    }
    // one-warp teams synchronise with __syncwarp: they keep one buffer and two barriers
    const bool dbl = P >= 64;
    if (!dbl) team_sync(P, tic);

    // 3b. PCR on the P condensed rows.  Level l writes buffer q when l is even and p
    // when odd (level 0 must not overwrite the 3a exchange in p while a thread still
    // reads it); a buffer is rewritten two levels later, after every thread has passed
    // the barrier between, so one barrier per level suffices
    int lvl = 0;
    for (int sig = 1; sig < P; sig <<= 1, ++lvl) {
      const bool odd = !dbl || (lvl & 1);
      cpx<T> *ba = odd ? pa : qa, *bc = odd ? pc : qc, *bd = odd ? pd : qd, *bi = odd ? pib : qib;
      ba[t] = A; bc[t] = C; bd[t] = D; bi[t] = recip(B);
      team_sync(P, tic);
      cpx<T> nA = mk<T>(T(0), T(0)), nB = B, nC = mk<T>(T(0), T(0)), nD = D;
      const int lo = t - sig, hi = t + sig;
      cpx<T> k1 = mk<T>(T(0), T(0)), k2 = mk<T>(T(0), T(0));
      if (lo >= 0) {
        k1 = mul(A, bi[lo]);
        nA = fnms(nA, k1, ba[lo]);
        nB = fnms(nB, k1, bc[lo]);
        nD = fnms(nD, k1, bd[lo]);
      }
      if (hi < P) {
        k2 = mul(C, bi[hi]);
        nC = fnms(nC, k2, bc[hi]);
        nB = fnms(nB, k2, ba[hi]);
        nD = fnms(nD, k2, bd[hi]);
      }
      if (F) {
        F[fs_k1<M>(lvl) * P] = k1;
        F[(fs_k1<M>(lvl) + 1) * P] = k2;
      }
      if (!dbl) team_sync(P, tic);
      A = nA; B = nB; C = nC; D = nD;
    }
    const cpx<T> rB = recip(B);
    if (F) F[fs_binv<M>(lvl) * P] = rB;
    const cpx<T> xf = mul(D, rB);
    // 3c. recover xe_t from the last row and xs_{t+1}, through the buffer the last PCR
    // level did not use
    cpx<T> *x3 = (dbl && ((lvl - 1) & 1)) ? qd : pd;
    x3[t] = xf;
    team_sync(P, tic);
    const cpx<T> xnext = t + 1 < P ? x3[t + 1] : mk<T>(T(0), T(0));
    const cpx<T> xl = fnms(fnms(D1, A1, xf), C1, xnext);

    // 4. back substitution of the interior rows
    my[0] = xf;
#pragma unroll
    for (int i = 1; i < M - 1; ++i) my[i] = fnms(fnms(my[i], aa[i], xf), cc[i], xl);
    my[M - 1] = xl;
    }
    if (do_acc) {
      T ox, oy;
      if (a.omega_t) {
        ox = a.omega_t[k].x;
        oy = a.omega_t[k].y;
      } else {
        const double2 omd = a.omega[k];
        ox = (T)omd.x;
        oy = (T)omd.y;
      }
#pragma unroll
      for (int i = 0; i < M; ++i) acc[i * P + t] += ox * my[i].x - oy * my[i].y;
    }
    team_sync(P, tic);

    // 5. store
    if (a.Y) {
      cpx<T> *Yk = a.Y + (int64_t)k * a.ldy + off;
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const int e = t + i * P;
        if (e < blen) Yk[e] = dd[e + e / M];
      }
    }
    // 6. dots with the Krylov basis: y_k in registers, four basis vectors per pass, and
    // their eight partial sums (re, im) reduced over the warp together by a reduce-scatter
    // (9 shuffles instead of 40); warp sums in the compute type (binary32 in the mixed
    // path, where h_k itself is binary32), the per-warp partials added in FP64
    if (mdots > 0) {
      const int nw = P >> 5, w = t >> 5, l = t & 31;
      cpx<T> yv[M];
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const int e = t + i * P;
        yv[i] = dd[e + e / M];  // zero beyond blen
      }
      const bool b4 = l & 16, b3 = l & 8, b2 = l & 4;
      for (int q0 = 0; q0 < mdots; q0 += 4) {
        T s8[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) s8[j] = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (q0 + j < mdots) {
            const T *vq = a.V + (int64_t)(q0 + j) * a.ldv + off;
            T vv[M];
#pragma unroll
            for (int i = 0; i < M; ++i) vv[i] = (t + i * P < blen) ? vq[t + i * P] : T(0);
#pragma unroll
            for (int i = 0; i < M; ++i) {
              s8[2 * j] += vv[i] * yv[i].x;
              s8[2 * j + 1] += vv[i] * yv[i].y;
            }
          }
        }
        // lane l ends with value (b4, b3, b2) of the eight, summed over the warp
        T r4[4], r2[2];
#pragma unroll
        for (int i = 0; i < 4; ++i) r4[i] = (b4 ? s8[i + 4] : s8[i]) + shfl_xor(b4 ? s8[i] : s8[i + 4], 16);
#pragma unroll
        for (int i = 0; i < 2; ++i) r2[i] = (b3 ? r4[i + 2] : r4[i]) + shfl_xor(b3 ? r4[i] : r4[i + 2], 8);
        T r1 = (b2 ? r2[1] : r2[0]) + shfl_xor(b2 ? r2[0] : r2[1], 4);
        r1 += shfl_xor(r1, 2);
        r1 += shfl_xor(r1, 1);
        const int vi = (b4 ? 4 : 0) | (b3 ? 2 : 0) | (b2 ? 1 : 0);
        if ((l & 3) == 0 && q0 + (vi >> 1) < mdots)
          reinterpret_cast<double *>(&red[w * mdots + q0 + (vi >> 1)])[vi & 1] = (double)r1;
      }
      team_sync(P, tic);
      for (int q = t; q < mdots; q += P) {
        double sx = 0.0, sy = 0.0;
        for (int i = 0; i < nw; ++i) {
          sx += red[i * mdots + q].x;
          sy += red[i * mdots + q].y;
        }
        a.gpart[((int64_t)k * g.nblk + blk) * mdots + q] = make_double2(sx, sy);
      }
    }
    team_sync(P, tic);
  }
  if (do_acc) {
    if (g.cta_sum) {
      // nblk == 1: every team of the CTA owns the same rows, so the CTA adds its
      // teams' accumulators (fixed order) and writes one partial row
      __syncthreads();
      if (tic == 0) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const int e = e0 + i;
          double sum = 0.0;
          for (int j = 0; j < g.teams_per_cta; ++j)
            sum += (double)reinterpret_cast<const T *>(reinterpret_cast<const unsigned char *>(acc) +
                                                       (size_t)j * team_bytes)[i * P + t];
          if (e < blen) a.acc_part[(int64_t)blockIdx.x * blen + e] = sum;
        }
      }
    } else if (active) {
#pragma unroll
      for (int i = 0; i < M; ++i) {
        const int e = e0 + i;
        if (e < blen) a.acc_part[(int64_t)team * blen + e] = (double)acc[i * P + t];
      }
    }
  }
}

// Column sums out[j] = sum_r X[r][j] in a fixed order.  A CTA of CW x RG = 512 threads
// owns CW adjacent columns and RG row groups; group y sums rows y, y + RG, ... with
// kColB loads in flight, then the groups' partials are added in a fixed two-level order,
// so the result does not depend on scheduling.  Many rows: 8 columns (one 64-byte
// segment) x 64 groups; few rows (<= 256): 32 columns x 16 groups, so that each thread
// still has several rows and the grid is not thousands of tiny CTAs.
constexpr int kColB = 8;

template <typename V, int CW, int RG>
__device__ __forceinline__ V colsum_finish(V v, V (*sm)[CW + 1], int tx, int ty) {
  constexpr int G = RG < 8 ? RG : 8;  // second-level groups
  sm[ty][tx] = v;
  __syncthreads();
  V t = V(0);
  if (ty < G) {
#pragma unroll
    for (int i = 0; i < RG / G; ++i) t += sm[ty * (RG / G) + i][tx];
  }
  __syncthreads();
  if (ty < G) sm[ty][tx] = t;
  __syncthreads();
  t = V(0);
  if (ty == 0) {
#pragma unroll
    for (int i = 0; i < G; ++i) t += sm[i][tx];
  }
  return t;  // valid for ty == 0
}

// out[j] = sum_r part[(blk*R + r)*blen + e], j = blk*blen + e (the per-team partial
// rows of b or z).  One-dimensional CTAs of CW * RG threads: column tx, group ty.
// With tail.enabled the last CTA to finish then starts Algorithm 2 on out (beta, v_1),
// for vectors one CTA handles.
template <int CW, int RG>
__global__ void __launch_bounds__(CW * RG) k_acc_reduce(int nblk, int blen, int R, const double *__restrict__ part,
                                                        double *__restrict__ out, const int *skip_flag,
                                                        InitTail tail, const double *__restrict__ extra) {
  grid_dep_wait();
  if (skip_flag && *skip_flag && !tail.enabled) return;
  __shared__ double sm[RG][CW + 1];
  const int tx = threadIdx.x % CW, ty = threadIdx.x / CW;
  const int64_t n = (skip_flag && *skip_flag) ? 0 : (int64_t)nblk * blen;
  const int64_t j = (int64_t)blockIdx.x * CW + tx;
  double acc[kColB];
#pragma unroll
  for (int u = 0; u < kColB; ++u) acc[u] = 0.0;
  if (j < n) {
    const int blk = (int)(j / blen);
    const int e = (int)(j - (int64_t)blk * blen);
    const double *base = part + (int64_t)blk * R * blen + e;  // R = partial rows per block
    for (int r0 = ty; r0 < R; r0 += RG * kColB) {
      double v[kColB];
#pragma unroll
      for (int u = 0; u < kColB; ++u) {
        const int r = r0 + u * RG;
        v[u] = r < R ? base[(int64_t)r * blen] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kColB; ++u) acc[u] += v[u];
    }
  }
  double tot = 0.0;
#pragma unroll
  for (int u = 0; u < kColB; ++u) tot += acc[u];
  tot = colsum_finish<double, CW, RG>(tot, sm, tx, ty);
  if (ty == 0 && j < n) out[j] = extra ? tot + extra[j] : tot;
  if (tail.enabled && last_cta_done(tail.counter)) {
    init_v0_body<kTail>(out, tail.n, tail.part, tail.ld, tail.V, tail.Vf, tail.scal, tail.flags, tail.use_handle,
                        tail.h, tail.T, tail.nT);
    if (threadIdx.x == 0) *tail.counter = 0;
  }
}

// z[j] = sum_k Re(omega_k H[k][j]) over the stored h_k (eq. 13's z), j < n.  In
// binary32 the weights are rounded once into shared memory (nf * 8 bytes).  With
// tail.enabled the last CTA to finish then projects z and takes the decision of the
// Algorithm-2 step (eq. 13), for vectors one CTA handles.
template <typename T, int CW, int RG>
__global__ void __launch_bounds__(CW * RG) k_zsum(int nf, int64_t n, const cpx<T> *__restrict__ H, int64_t ldh,
                                                  const double2 *__restrict__ omega, double *__restrict__ z,
                                                  const int *skip_flag, ProjTail tail, int mlen,
                                                  const double *__restrict__ h0) {
  grid_dep_wait();
  const bool skip = skip_flag && *skip_flag;  // breakdown: no z (eq. 13 gives 0); the tail still decides
  // z only feeds the eq. (13) estimate, so the column sums stay in the compute type (FP64
  // adds would bound this kernel on GB300's FP64 pipe); the zero-frequency lane's FP64
  // term (h0) is added in FP64
  __shared__ T sm[RG][CW + 1];
  extern __shared__ __align__(16) unsigned char om_raw[];
  cpx<T> *om = reinterpret_cast<cpx<T> *>(om_raw);
  const int tx = threadIdx.x % CW, ty = threadIdx.x / CW;
  if (!skip) {
    // batched plans with one Algorithm 2 per member (mlen rows each): column j takes
    // the weights of its member; those of the CTA's first member are staged
    const int mem0 = mlen ? (int)((int64_t)blockIdx.x * CW / mlen) : 0;
    const double2 *om0 = omega + (int64_t)mem0 * nf;
    const int64_t j = (int64_t)blockIdx.x * CW + tx;
    const int memj = (mlen && j < n) ? (int)(j / mlen) : mem0;
    const bool own = j < n && memj == mem0;
    // the first batch of h_k loads is issued before the weights are staged, so the two
    // memory round trips overlap
    // with h0 the zero frequency comes from the FP64 lane (added below), not from row 0
    const int kfirst = h0 ? 1 : 0;
    cpx<T> h[kColB];
#pragma unroll
    for (int u = 0; u < kColB; ++u) {
      const int k = ty + u * RG;
      h[u] = (own && k < nf && k >= kfirst) ? H[(int64_t)k * ldh + j] : mk<T>(T(0), T(0));
    }
    for (int k = threadIdx.x; k < nf; k += CW * RG) om[k] = mk<T>((T)om0[k].x, (T)om0[k].y);
    __syncthreads();
    T acc[kColB];
#pragma unroll
    for (int u = 0; u < kColB; ++u) acc[u] = T(0);
    if (j < n && !own) {  // a later member in this CTA: its weights from memory
      const double2 *omj = omega + (int64_t)memj * nf;
      for (int k = ty < kfirst ? ty + RG : ty; k < nf; k += RG) {
        const cpx<T> hk = H[(int64_t)k * ldh + j];
        acc[0] += (T)omj[k].x * hk.x - (T)omj[k].y * hk.y;
      }
    } else if (own) {
      for (int k0 = ty;;) {
#pragma unroll
        for (int u = 0; u < kColB; ++u) {
          const int k = k0 + u * RG;
          if (k < nf) acc[u] += om[k].x * h[u].x - om[k].y * h[u].y;
        }
        k0 += RG * kColB;
        if (k0 >= nf) break;
#pragma unroll
        for (int u = 0; u < kColB; ++u) {
          const int k = k0 + u * RG;
          h[u] = (k < nf && k >= kfirst) ? H[(int64_t)k * ldh + j] : mk<T>(T(0), T(0));
        }
      }
    }
    T tot = T(0);
#pragma unroll
    for (int u = 0; u < kColB; ++u) tot += acc[u];
    tot = colsum_finish<T, CW, RG>(tot, sm, tx, ty);
    if (ty == 0 && j < n) z[j] = h0 ? (double)tot + omega[(int64_t)memj * nf].x * h0[j] : (double)tot;
  }
  if (tail.enabled && last_cta_done(tail.counter)) {
    project_body<kTail>(tail.n, tail.V, z, tail.tau, tail.part, tail.ld, tail.scal, tail.flags, tail.kc,
                        tail.use_handle, tail.h);
    if (threadIdx.x == 0) *tail.counter = 0;
  }
}

template <typename T>
void launch_zsum(Ctx &c, int nf, int64_t n, const cpx<T> *H, int64_t ldh, const double2 *omega, double *z,
                 const int *skip_flag, const ProjTail *tailp, int mlen, const double *h0) {
  const size_t smem = (size_t)nf * sizeof(cpx<T>);
  ProjTail tail{};
  if (tailp) tail = *tailp;
  c.launch("zsum", (double)nf * n * sizeof(cpx<T>) + n * 8.0, [&] {
    if (nf <= 256) {
      const int grid = (int)((n + 31) / 32);
      pdl_launch(c.pdl, k_zsum<T, 32, 16>, dim3(grid), dim3(512), smem, c.stream, nf, n, H, ldh, omega, z,
                 skip_flag, tail, mlen, h0);
    } else {
      const int grid = (int)((n + 7) / 8);
      if (smem > 48 * 1024)
        allow_dyn_smem((const void *)k_zsum<T, 8, 64>);
      pdl_launch(c.pdl, k_zsum<T, 8, 64>, dim3(grid), dim3(512), smem, c.stream, nf, n, H, ldh, omega, z,
                 skip_flag, tail, mlen, h0);
    }
  });
}
template void launch_zsum<double>(Ctx &, int, int64_t, const cpx<double> *, int64_t, const double2 *, double *,
                                  const int *, const ProjTail *, int, const double *);
template void launch_zsum<float>(Ctx &, int, int64_t, const cpx<float> *, int64_t, const double2 *, double *,
                                 const int *, const ProjTail *, int, const double *);

static int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

void set_acc_rows(PintGeom &g) {
  g.cta_sum = (g.nblk == 1 && g.teams_per_cta > 1) ? 1 : 0;
  g.acc_rows = g.cta_sum ? (g.R + g.teams_per_cta - 1) / g.teams_per_cta : g.R;
}

PintGeom pint_geometry(int nf, int nblk, int blen, int target_teams, int elem_bytes, int m_req, int teams_req,
                       bool fact) {
  PintGeom g;
  g.nf = nf;
  g.nblk = nblk;
  g.blen = blen;
  // rows per thread: 8 balances the serial chunk elimination against the PCR depth
  // (16 rows, binary32 only, is available on request)
  g.M = blen <= 128 ? 4 : 8;
  if (m_req) g.M = m_req;
  g.P = std::max(32, next_pow2((blen + g.M - 1) / g.M));
  const int max_threads = g.M >= 16 ? 256 : 512;  // the kernel's launch bounds
  g.teams_per_cta = std::max(1, 256 / g.P);
  int R = (target_teams + nblk - 1) / nblk;
  g.R = std::max(1, std::min(R, nf));
  // fewer teams per CTA while the grid would not cover every SM
  const int nteams = nblk * g.R;
  while (g.teams_per_cta > 1 && (nteams + g.teams_per_cta - 1) / g.teams_per_cta < sm_count()) g.teams_per_cta >>= 1;
  if (teams_req) g.teams_per_cta = std::max(1, std::min(teams_req, max_threads / g.P));
  // stage tau K in shared memory when the CTA stays within ~160 KB
  const size_t esz = elem_bytes == 16 ? 8 : 4;  // real type of the compute precision
  const size_t rest = (size_t)g.P * (g.M + 1) * 2 * esz + (size_t)g.P * ((fact || g.P < 64) ? 5 : 8) * 2 * esz +
                      (size_t)g.P * g.M * esz +
                      (size_t)(g.P / 32) * 33 * 16;
  const size_t stage = (size_t)3 * g.P * (g.M + 1) * esz;
  g.stage = (rest + stage) * g.teams_per_cta <= 160 * 1024 ? 1 : 0;
  set_acc_rows(g);
  return g;
}

template <typename T, int M>
static void launch_pint_m(Ctx &c, const PintGeom &g, const PintArgs<T> &a) {
  const size_t tb =
      TeamSmem<T, M>::bytes(g.P, a.mcount ? (a.want_dots ? a.mdots_max : 0) : a.mdots, g.stage, a.fac_in != nullptr);
  const size_t smem = tb * g.teams_per_cta;
  const int nteams = g.nblk * g.R;
  const int grid = (nteams + g.teams_per_cta - 1) / g.teams_per_cta;
  const int threads = g.P * g.teams_per_cta;
  auto kern = a.fac_in ? (threads <= 256 ? k_pint<T, M, 256, true> : k_pint<T, M, (M >= 16 ? 256 : 512), true>)
                       : (threads <= 256 ? k_pint<T, M, 256, false> : k_pint<T, M, (M >= 16 ? 256 : 512), false>);
  allow_dyn_smem((const void *)kern);
  // algorithmic bytes: spectrum rows read/written as requested, plus the vector rhs
  double bytes = 0.0;
  const double per = (double)g.nf * g.nblk * g.blen;
  if (a.R) bytes += per * sizeof(cpx<T>);
  if (a.Y) bytes += per * sizeof(cpx<T>);
  const bool dots = a.mcount ? a.want_dots != 0 : a.mdots > 0;
  // the b pass may also store L (Y set): it is named by its accumulation
  const char *fam = sizeof(T) == 8 ? (dots ? "pint_dots_f64" : (a.omega ? "pint_acc_f64" : "pint_store_f64"))
                                   : (dots ? "pint_dots_f32" : (a.omega ? "pint_acc_f32" : "pint_store_f32"));
  if (a.fac_out) {
    fam = sizeof(T) == 8 ? "pint_factor_f64" : "pint_factor_f32";
    bytes = (double)pint_factor_elems(g) * sizeof(cpx<T>);
  } else if (a.fac_in) {
    bytes += (double)pint_factor_elems(g) * sizeof(cpx<T>);
  }
  c.launch(fam, bytes, [&] { pdl_launch(c.pdl, kern, dim3(grid), dim3(threads), smem, c.stream, g, a, tb); });
}

template <typename T>
void launch_pint(Ctx &c, const PintGeom &g, const PintArgs<T> &a) {
  if (g.M == 4) {
    launch_pint_m<T, 4>(c, g, a);
  } else if (g.M == 16) {
    if constexpr (sizeof(T) == 4) launch_pint_m<T, 16>(c, g, a);
  } else {
    launch_pint_m<T, 8>(c, g, a);
  }
}

void launch_acc_reduce(Ctx &c, const PintGeom &g, const double *acc_part, double *out, const int *skip_flag,
                       const InitTail *tailp, const double *extra) {
  const int64_t n = (int64_t)g.nblk * g.blen;
  InitTail tail{};
  if (tailp) tail = *tailp;
  c.launch("acc_reduce", (double)n * g.acc_rows * 8.0 + n * 8.0, [&] {
    if (g.acc_rows <= 32)  // few partial rows (2D, batches): 128 columns x 4 row groups
      pdl_launch(c.pdl, k_acc_reduce<128, 4>, dim3((int)((n + 127) / 128)), dim3(512), 0, c.stream, g.nblk, g.blen,
                 g.acc_rows, acc_part, out, skip_flag, tail, extra);
    else if (g.acc_rows <= 256)
      pdl_launch(c.pdl, k_acc_reduce<32, 16>, dim3((int)((n + 31) / 32)), dim3(512), 0, c.stream, g.nblk, g.blen,
                 g.acc_rows, acc_part, out, skip_flag, tail, extra);
    else
      pdl_launch(c.pdl, k_acc_reduce<8, 64>, dim3((int)((n + 7) / 8)), dim3(512), 0, c.stream, g.nblk, g.blen,
                 g.acc_rows, acc_part, out, skip_flag, tail, extra);
  });
}

// r[i] = the binary32 reciprocal of the mixed-precision shifted solves (rcp_nr), for the
// verification entry point paradiag_recip_f32.
__global__ void k_recip_f32(const float *__restrict__ x, float *__restrict__ r, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = rcp_nr(x[i]);
}

void launch_recip_f32(cudaStream_t s, const float *x, float *r, int64_t n) {
  const int64_t grid = (n + 255) / 256;
  if (grid > 0) k_recip_f32<<<(unsigned)grid, 256, 0, s>>>(x, r, n);
}

template void launch_pint<double>(Ctx &, const PintGeom &, const PintArgs<double> &);
template void launch_pint<float>(Ctx &, const PintGeom &, const PintArgs<float> &);

}  // namespace pd
