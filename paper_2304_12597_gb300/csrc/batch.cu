// Per-problem scaling for batched plans: `batch` independent problems share one
// plan as a block-diagonal problem (slot b = columns [b*nxm, (b+1)*nxm) of every
// time row).  The Krylov and refinement stopping rules measure the whole stack, so
// every problem is first scaled to unit Frobenius norm (up to a factor of two) and
// scaled back after the solve.  The scale factors are powers of two: the scaling is
// exact and costs integer work on the exponent field, not FP64 multiplies.
#include <algorithm>

#include "pd_internal.h"

namespace pd {

// part[b * nc + c] = sum over time rows t = c, c + nc, ... of slot b's squares.
__global__ void __launch_bounds__(256) k_batch_sumsq(const double *__restrict__ X, int64_t nt, int64_t ld, int nxm,
                                                     int nc, double *__restrict__ part) {
  grid_dep_wait();
  const int c = blockIdx.x, b = blockIdx.y;
  double s = 0.0;
  for (int64_t t = c; t < nt; t += nc) {
    const double *row = X + t * ld + (int64_t)b * nxm;
    for (int i = threadIdx.x; i < nxm; i += blockDim.x) s = fma(row[i], row[i], s);
  }
  __shared__ double red[8];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    part[(int64_t)b * nc + c] = t;
  }
}

// ex[b] = -round(log2 ||slot b||_F): slot b is multiplied by 2^ex[b] before the solve
// and its solution by 2^-ex[b] after it (0 for an all-zero or non-finite slot).
// zero[b] = 1 for an all-zero slot: its solution is exactly zero, whatever rounding-level
// values the paired real DFTs leave in its columns, and it takes no part in the
// refinement decision.
__global__ void k_batch_exponents(int batch, int nc, const double *__restrict__ part, int *__restrict__ ex,
                                  int *__restrict__ zero) {
  grid_dep_wait();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double s = 0.0;
  for (int c = 0; c < nc; ++c) s += part[(int64_t)b * nc + c];
  int e = 0;
  if (s > 0.0 && isfinite(s)) {
    int e2;
    frexp(s, &e2);  // s = f 2^e2, f in [0.5, 1): ||x|| ~ 2^(e2/2)
    e = -(e2 / 2);
  }
  ex[b] = e;
  zero[b] = s == 0.0 ? 1 : 0;
}

// x * 2^k exactly: an exponent-field add for normal x whose result stays normal
// (zero stays zero); other cases (subnormal, overflow, Inf/NaN) take ldexp.
__device__ __forceinline__ double pow2_scale(double x, int k) {
  const long long bits = __double_as_longlong(x);
  if ((bits & 0x7fffffffffffffffLL) == 0) return x;
  const int e = (int)((bits >> 52) & 0x7ff);
  if (e > 0 && e < 0x7ff && e + k > 0 && e + k < 0x7ff) return __longlong_as_double(bits + ((long long)k << 52));
  return ldexp(x, k);
}

// Y = X * 2^(sign * ex[slot]) over the (nt, ld) array, one time row per blockIdx.y;
// Y may alias X.  With nxb != NULL, columns past problem b's n_x, and every column of an
// all-zero problem (zero[b]), are set to zero (they are decoupled from the problem, but
// the paired real-to-complex DFT leaves rounding-level values there).
__global__ void __launch_bounds__(256) k_batch_scale(const double *X, double *Y, int ld, int nxm,
                                                     const int *__restrict__ ex, int sign,
                                                     const int *__restrict__ nxb, const int *__restrict__ zero) {
  grid_dep_wait();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ld) return;
  const int b = j / nxm;
  const int64_t i = (int64_t)blockIdx.y * ld + j;
  Y[i] = (nxb && (j - b * nxm >= nxb[b] || zero[b])) ? 0.0 : pow2_scale(X[i], sign * ex[b]);
}

void launch_batch_normalize(Ctx &c, const double *G, double *Gs, int64_t nt, int batch, int nxm, int nc,
                            double *part, int *ex, int *zero) {
  const int64_t ld = (int64_t)batch * nxm;
  c.launch("batch_scale", (double)nt * ld * 8.0, [&] {
    pdl_launch(c.pdl, k_batch_sumsq, dim3(nc, batch), dim3(256), 0, c.stream, G, nt, ld, nxm, nc, part);
  });
  c.launch("batch_scale", 0.0, [&] { pdl_launch(c.pdl, k_batch_exponents, dim3((batch + 127) / 128), dim3(128), 0, c.stream, batch, nc, part, ex,
                                                        zero); });
  const dim3 grid((unsigned)((ld + 255) / 256), (unsigned)nt);
  c.launch("batch_scale", (double)nt * ld * 16.0,
           [&] { pdl_launch(c.pdl, k_batch_scale, grid, dim3(256), 0, c.stream, G, Gs, (int)ld, nxm, (const int *)ex, 1,
                                  (const int *)nullptr, (const int *)nullptr); });
}

// A problem joining a running batch (join[b]): its U slot starts at zero and its refinement
// state restarts; so does every unused slot (zero[b]: an all-zero right-hand side, whose U
// may hold anything); the other slots' U goes back into the solve's units, U * 2^ex[b]
// (exact).
__global__ void __launch_bounds__(256) k_member_join(double *U, int ld, int nxm, int batch, const int *__restrict__ ex,
                                                     const int *__restrict__ join, const int *__restrict__ zero,
                                                     int *msw, double *prev, double *ref2, int *mex, int *mconv) {
  grid_dep_wait();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.y == 0 && j < batch && (join[j] || zero[j])) {  // (an unused slot's mex may be stale)
    msw[j] = 0;
    prev[j] = 0.0;
    ref2[j] = 0.0;
    mex[j] = 0;
    mconv[j] = 0;
  }
  if (j >= ld) return;
  const int b = j / nxm;
  const int64_t i = (int64_t)blockIdx.y * ld + j;
  U[i] = (join[b] || zero[b]) ? 0.0 : pow2_scale(U[i], ex[b]);
}

void launch_member_join(Ctx &c, double *U, int64_t nt, int batch, int nxm, const int *ex, const int *join,
                        const int *zero, int *msw, double *prev, double *ref2, int *mex, int *mconv) {
  const int64_t ld = (int64_t)batch * nxm;
  const dim3 grid((unsigned)((std::max<int64_t>(ld, batch) + 255) / 256), (unsigned)nt);
  c.launch("batch_scale", (double)nt * ld * 16.0, [&] {
    pdl_launch(c.pdl, k_member_join, grid, dim3(256), 0, c.stream, U, (int)ld, nxm, batch, ex, join, zero, msw, prev,
               ref2, mex, mconv);
  });
}

void launch_batch_unscale(Ctx &c, double *U, int64_t nt, int batch, int nxm, const int *ex, const int *nxb,
                          const int *zero) {
  const int64_t ld = (int64_t)batch * nxm;
  const dim3 grid((unsigned)((ld + 255) / 256), (unsigned)nt);
  c.launch("batch_scale", (double)nt * ld * 16.0,
           [&] { pdl_launch(c.pdl, k_batch_scale, grid, dim3(256), 0, c.stream, (const double *)U, U, (int)ld, nxm, ex, -1,
                                  nxb, zero); });
}

// out[t][j] = in[t][j] * s[j] (in place allowed): the diagonal mass matrix's symmetric
// scaling of G (s = M^{-1/2}) and of U (s = M^{-1/2}, from w = M^{1/2} u).
__global__ void k_col_scale(const double *in, double *out, int nb, const double *__restrict__ s) {
  grid_dep_wait();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int64_t o = (int64_t)blockIdx.y * nb + j;
  out[o] = in[o] * s[j];
}

void launch_col_scale(Ctx &c, const double *in, double *out, int64_t nt, int64_t nb, const double *s) {
  const dim3 grid((unsigned)((nb + 255) / 256), (unsigned)nt);
  c.launch("mass_scale", (double)nt * nb * 16.0,
           [&] { pdl_launch(c.pdl, k_col_scale, grid, dim3(256), 0, c.stream, in, out, (int)nb, s); });
}

}  // namespace pd
