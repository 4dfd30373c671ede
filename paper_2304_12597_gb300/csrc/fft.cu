// Time-axis DFTs of the all-at-once block (eq. 5: U F^T and Y F^{-T}) and the
// orthonormal DST-I along y that diagonalises T_y of the 2D operator (Sec. 6.1).
//
// Each CTA owns a tile of TX adjacent spatial columns and all n time points, so
// every global load/store touches TX contiguous elements of an n_bar-contiguous
// row.  Two real columns are packed into one complex series (z = a + i b), the
// series are transformed in shared memory by an in-place radix-4 (with a final
// radix-2) decimation-in-time Cooley-Tukey FFT from bit-reversed input, and the
// two real spectra are separated on the way out:
//   A[k] = (Z[k] + conj Z[-k]) / 2,   B[k] = (Z[k] - conj Z[-k]) / (2i).
// Twiddles omega_n^k = exp(-2 pi i k / n), k < n/2, come from a table computed
// on the host in FP64 (rounded to FP32 for the mixed path).
#include <algorithm>

#include "pd_control.cuh"

namespace pd {

// Global loads a thread issues back to back before it uses any of them.
constexpr int kLoadBatch = 8;
// Output elements per thread in flight in the stores that read U first (mode 1): half the
// load batch keeps those epilogues from setting the kernels' register count.
constexpr int kEpiBatch = 4;
// Threads per CTA of the forward time DFTs: 512 once a tile holds >= 4096 values (n TX),
// so each thread issues one batch of loads and takes one butterfly per pass; else 256.
// (The inverse DFT keeps 256: its FP64 update needs more than the 64 registers a thread
// may hold with two 512-thread CTAs per SM.)
constexpr int kFftMaxThreads = 512;
static int fft_threads(int n, int tx) { return (int64_t)n * tx >= 4096 ? 512 : 256; }

// Series of length n sit n + 1 complex values apart in shared memory: the columns of a
// tile (two per series) then fall into different banks when a warp writes one time row
// (or reads one frequency) of every series, instead of all series mapping to one bank.
__host__ __device__ inline int series_stride(int n) { return n + 1; }

// In-place DIT FFT of `nseries` series of length n = 2^logn stored back to back
// in shared memory, input in bit-reversed order, output in natural order.
// All threads of the CTA take part; the caller synchronises before the call.
template <typename T>
__device__ void fft_smem(cpx<T> *buf, int n, int logn, int nseries, const cpx<T> *__restrict__ tw) {
  const int sst = series_stride(n);
  int s = 0;
  if (logn >= 2) {  // first radix-4 pass: every twiddle is 1 (j = 0), no multiplications
    const int lq = logn - 2;
    const int total = nseries << lq;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int ser = idx >> lq;
      const int base = (idx & ((1 << lq) - 1)) << 2;
      cpx<T> *p = buf + (size_t)ser * sst + base;
      const cpx<T> x0 = p[0], x1 = p[1], x2 = p[2], x3 = p[3];
      const cpx<T> a0 = add(x0, x1), a1 = sub(x0, x1), a2 = add(x2, x3), a3 = sub(x2, x3);
      const cpx<T> mu = mk<T>(a3.y, -a3.x);  // -i * a3
      p[0] = add(a0, a2);
      p[2] = sub(a0, a2);
      p[1] = add(a1, mu);
      p[3] = sub(a1, mu);
    }
    __syncthreads();
    s = 2;
  }
  while (s + 1 < logn) {  // radix-4 pass = DIT stages with half-spans h and 2h
    const int h = 1 << s;
    const int lq = logn - 2;
    const int total = nseries << lq;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int ser = idx >> lq;
      const int q = idx & ((1 << lq) - 1);
      const int j = q & (h - 1);
      const int base = ((q >> s) << (s + 2)) + j;
      cpx<T> *p = buf + (size_t)ser * sst;
      const cpx<T> w1 = tw[j << (logn - s - 1)];
      const cpx<T> w2 = tw[j << (logn - s - 2)];
      cpx<T> x0 = p[base], x1 = p[base + h], x2 = p[base + 2 * h], x3 = p[base + 3 * h];
      cpx<T> t1 = mul(w1, x1), t3 = mul(w1, x3);
      cpx<T> a0 = add(x0, t1), a1 = sub(x0, t1), a2 = add(x2, t3), a3 = sub(x2, t3);
      cpx<T> t2 = mul(w2, a2);
      cpx<T> u = mul(w2, a3);
      cpx<T> mu = mk<T>(u.y, -u.x);  // omega_{4h}^{j+h} a3 = -i * (omega_{4h}^j a3)
      p[base] = add(a0, t2);
      p[base + 2 * h] = sub(a0, t2);
      p[base + h] = add(a1, mu);
      p[base + 3 * h] = sub(a1, mu);
    }
    __syncthreads();
    s += 2;
  }
  if (s < logn) {  // last radix-2 stage, half-span h = n/2
    const int h = 1 << s;
    const int lh = logn - 1;
    const int total = nseries << lh;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int ser = idx >> lh;
      const int b = idx & ((1 << lh) - 1);
      const int j = b & (h - 1);
      const int i0 = ((b >> s) << (s + 1)) + j;
      cpx<T> *p = buf + (size_t)ser * sst;
      const cpx<T> w = tw[j << (logn - s - 1)];
      cpx<T> x0 = p[i0], x1 = p[i0 + h];
      cpx<T> t = mul(w, x1);
      p[i0] = add(x0, t);
      p[i0 + h] = sub(x0, t);
    }
    __syncthreads();
  }
}

// Separate the packed spectra and store the half spectrum of the tile's columns.
template <typename T, int TX>
__device__ void r2c_store(const cpx<T> *buf, int n, int logn, int64_t x0, int64_t ncols, cpx<T> *__restrict__ S,
                          int64_t lds) {
  const int nf = (n >> 1) + 1;
  const int tot2 = nf * TX;
  for (int idx = threadIdx.x; idx < tot2; idx += blockDim.x) {
    const int k = idx / TX;
    const int c = idx - k * TX;
    const int64_t col = x0 + c;
    if (col >= ncols) continue;
    const cpx<T> *z = buf + (size_t)(c >> 1) * series_stride(n);
    const cpx<T> zk = z[k], zm = z[(n - k) & (n - 1)];
    cpx<T> r;
    if ((c & 1) == 0) {
      r = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
    } else {
      r = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
    }
    S[(int64_t)k * lds + col] = r;
  }
}

// Sum of squares of the transformed data (per thread: ss), reduced over the launch: each
// CTA stores its partial, and the last CTA to finish (no CTA waits for another) adds the
// partials in a fixed order and stores the square root into *rn.dst.
__device__ void rhs_norm_finish(float ss, const RhsNorm &rn) {
  __shared__ double red[32];
  __shared__ int last;
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  ss = warp_sum(ss);  // binary32 within a warp (a reference scale; FP64 adds cost GB300's FP64 pipe)
  if (l == 0) red[w] = (double)ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += red[i];
    rn.part[blockIdx.x] = t;
    __threadfence();
    last = atomicAdd(rn.counter, 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double t = 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += __ldcg(rn.part + i);
  t = warp_sum(t);
  __syncthreads();  // red is reused
  if (l == 0) red[w] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int i = 0; i < nw; ++i) s2 += red[i];
    *rn.dst = sqrt(s2);
    *rn.counter = 0;
  }
}

// ---- Radix-16 first stage in registers (series of n >= 16 points) -------------------
// With bit-reversed input, the first four DIT stages (half-spans 1..8) act within blocks of
// 16 consecutive positions: block g holds the times r + i n/16, r = bitrev_{L-4}(g) (i =
// 0..15, bit-reversed), and after those stages their natural-order 16-point DFT.  A thread
// therefore loads a block's 16 time samples straight from global memory, transforms them
// in registers (dft16) and writes the block to shared memory; fft_smem16 runs the
// remaining stages.  In shared memory a series keeps one pad slot after every 16 values
// (element i at pz(i) = i + i/16) and series are series_stride16(n) = 2 (mod 16) complex
// values apart, so that the block writes (lanes over column pairs and blocks), the
// butterflies of the later stages and the column-wise reads of the output are free of
// bank conflicts.
__host__ __device__ inline int pz(int i) { return i + (i >> 4); }
__host__ __device__ inline int series_stride16(int n) {
  const int s0 = n + n / 16;
  return s0 + (((2 - s0) % 16) + 16) % 16;
}

// X[k] = sum_i x[i] w^{ik}, w = exp(-2 pi i / 16), in place, natural order in and out:
// radix-4 over i = 4 i1 + i2 (i1 first), twiddles w^{i2 k1}, radix-4 over i2.
template <typename T>
__device__ __forceinline__ void radix4_fwd(cpx<T> &a0, cpx<T> &a1, cpx<T> &a2, cpx<T> &a3) {
  const cpx<T> t0 = add(a0, a2), t1 = sub(a0, a2), t2 = add(a1, a3), t3 = sub(a1, a3);
  const cpx<T> mt3 = mk<T>(t3.y, -t3.x);  // -i t3
  a0 = add(t0, t2);
  a2 = sub(t0, t2);
  a1 = add(t1, mt3);
  a3 = sub(t1, mt3);
}
template <typename T>
__device__ __forceinline__ cpx<T> w16(int m) {  // w^m for the products m of i2, k1 < 4
  constexpr double c = 0.92387953251128675613;  // cos(pi/8)
  constexpr double s = 0.38268343236508977173;  // sin(pi/8)
  constexpr double r = 0.70710678118654752440;  // cos(pi/4)
  switch (m) {
    case 1: return mk<T>((T)c, (T)-s);
    case 2: return mk<T>((T)r, (T)-r);
    case 3: return mk<T>((T)s, (T)-c);
    case 4: return mk<T>(T(0), T(-1));
    case 6: return mk<T>((T)-r, (T)-r);
    case 9: return mk<T>((T)-c, (T)s);
    default: return mk<T>(T(1), T(0));
  }
}
template <typename T>
__device__ __forceinline__ void dft16(cpx<T> (&x)[16]) {
#pragma unroll
  for (int i2 = 0; i2 < 4; ++i2) radix4_fwd(x[i2], x[4 + i2], x[8 + i2], x[12 + i2]);  // x[4 k1 + i2]
#pragma unroll
  for (int k1 = 1; k1 < 4; ++k1)
#pragma unroll
    for (int i2 = 1; i2 < 4; ++i2) x[4 * k1 + i2] = mul(w16<T>(i2 * k1), x[4 * k1 + i2]);
  cpx<T> y[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    cpx<T> b0 = x[4 * k1], b1 = x[4 * k1 + 1], b2 = x[4 * k1 + 2], b3 = x[4 * k1 + 3];
    radix4_fwd(b0, b1, b2, b3);
    y[k1] = b0;
    y[k1 + 4] = b1;
    y[k1 + 8] = b2;
    y[k1 + 12] = b3;
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = y[k];
}

// The DIT stages of half-span 16 and up (the radix-16 first stage done), on series held
// with pz padding, series S apart.  Same butterflies and twiddles as fft_smem.
template <typename T>
__device__ void fft_smem16(cpx<T> *buf, int n, int logn, int nseries, int S, const cpx<T> *__restrict__ tw) {
  int s = 4;
  const int lq = logn - 2;
  while (s + 1 < logn) {  // radix-4 pass = DIT stages with half-spans h and 2h
    const int h = 1 << s;
    const int total = nseries << lq;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int ser = idx >> lq;
      const int q = idx & ((1 << lq) - 1);
      const int j = q & (h - 1);
      const int base = ((q >> s) << (s + 2)) + j;
      cpx<T> *p = buf + (size_t)ser * S;
      const cpx<T> w1 = tw[j << (logn - s - 1)];
      const cpx<T> w2 = tw[j << (logn - s - 2)];
      const int i0 = pz(base), i1 = pz(base + h), i2 = pz(base + 2 * h), i3 = pz(base + 3 * h);
      cpx<T> x0 = p[i0], x1 = p[i1], x2 = p[i2], x3 = p[i3];
      cpx<T> t1 = mul(w1, x1), t3 = mul(w1, x3);
      cpx<T> a0 = add(x0, t1), a1 = sub(x0, t1), a2 = add(x2, t3), a3 = sub(x2, t3);
      cpx<T> t2 = mul(w2, a2);
      cpx<T> u = mul(w2, a3);
      cpx<T> mu = mk<T>(u.y, -u.x);  // omega_{4h}^{j+h} a3 = -i * (omega_{4h}^j a3)
      p[i0] = add(a0, t2);
      p[i2] = sub(a0, t2);
      p[i1] = add(a1, mu);
      p[i3] = sub(a1, mu);
    }
    __syncthreads();
    s += 2;
  }
  if (s < logn) {  // last radix-2 stage, half-span h = n/2
    const int h = 1 << s;
    const int lh = logn - 1;
    const int total = nseries << lh;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
      const int ser = idx >> lh;
      const int b = idx & ((1 << lh) - 1);
      const int j = b & (h - 1);
      const int i0 = ((b >> s) << (s + 1)) + j;
      cpx<T> *p = buf + (size_t)ser * S;
      const cpx<T> w = tw[j << (logn - s - 1)];
      const int a = pz(i0), c = pz(i0 + h);
      cpx<T> x0 = p[a], x1 = p[c];
      cpx<T> t = mul(w, x1);
      p[a] = add(x0, t);
      p[c] = sub(x0, t);
    }
    __syncthreads();
  }
}

// r2c_store on the padded layout
template <typename T, int TX>
__device__ void r2c_store16(const cpx<T> *buf, int n, int64_t x0, int64_t ncols, cpx<T> *__restrict__ S, int64_t lds,
                            int SS) {
  const int nf = (n >> 1) + 1;
  const int tot2 = nf * TX;
  for (int idx = threadIdx.x; idx < tot2; idx += blockDim.x) {
    const int k = idx / TX;
    const int c = idx - k * TX;
    const int64_t col = x0 + c;
    if (col >= ncols) continue;
    const cpx<T> *z = buf + (size_t)(c >> 1) * SS;
    const cpx<T> zk = z[pz(k)], zm = z[pz((n - k) & (n - 1))];
    cpx<T> r;
    if ((c & 1) == 0) {
      r = mk<T>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
    } else {
      r = mk<T>(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
    }
    S[(int64_t)k * lds + col] = r;
  }
}

// Forward DFT of TX columns per CTA (n >= 16): each thread takes a (column pair, block)
// item: loads the block's 16 time samples of both columns (packed z = a + i b), dft16,
// writes the block; then the later stages and the separated half spectra.
template <typename T, typename Tin, int TX>
__global__ void __launch_bounds__(sizeof(T) == 8 ? 256 : 512)
    k_fft_r2c16(const Tin *__restrict__ X, int64_t ldx, int64_t ncols, int n, int logn, const cpx<T> *__restrict__ tw,
                cpx<T> *__restrict__ S, int64_t lds, const T *__restrict__ rs, RhsNorm rn) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T> *buf = reinterpret_cast<cpx<T> *>(smraw);
  constexpr int NP = TX / 2;
  const int64_t x0 = (int64_t)blockIdx.x * TX;
  const int SS = series_stride16(n), nb = n >> 4, lb = logn - 4;
  T ss = T(0);
  for (int it = threadIdx.x; it < NP * nb; it += blockDim.x) {
    const int p = it % NP, g = it / NP;
    const int r = bitrev(g, lb);
    const int64_t ca = x0 + 2 * p, cb = ca + 1;
    const bool va = ca < ncols, vb = cb < ncols;
    cpx<T> z[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int64_t j = r + i * nb;
      const Tin *row = X + j * ldx;
      z[i] = mk<T>(va ? cvt<T>(row[ca]) : T(0), vb ? cvt<T>(row[cb]) : T(0));
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      ss += z[i].x * z[i].x + z[i].y * z[i].y;
      if (rs) z[i] = scal(rs[r + i * nb], z[i]);
    }
    dft16(z);
    cpx<T> *blk = buf + (size_t)p * SS + 17 * g;  // pz(16 g + k) = 17 g + k
#pragma unroll
    for (int k = 0; k < 16; ++k) blk[k] = z[k];
  }
  __syncthreads();
  fft_smem16<T>(buf, n, logn, NP, SS, tw);
  r2c_store16<T, TX>(buf, n, x0, ncols, S, lds, SS);
  if (rn.part) rhs_norm_finish((float)ss, rn);
}

template <typename T, typename Tin, int TX>
__global__ void __launch_bounds__(kFftMaxThreads) k_fft_r2c(const Tin *__restrict__ X, int64_t ldx, int64_t ncols,
                                                 int n, int logn, const cpx<T> *__restrict__ tw,
                                                 cpx<T> *__restrict__ S, int64_t lds, const T *__restrict__ rs,
                                                 RhsNorm rn) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T> *buf = reinterpret_cast<cpx<T> *>(smraw);
  const int64_t x0 = (int64_t)blockIdx.x * TX;
  const int total = n * TX;
  T ss = T(0);  // squares of the loaded values (rn)
  // kLoadBatch loads in flight per thread before any is used
  for (int i0 = threadIdx.x; i0 < total; i0 += kLoadBatch * blockDim.x) {
    T v[kLoadBatch];
#pragma unroll
    // element idx = (slot s, column c): time row j = bitrev(s), so that consecutive threads
    // store to consecutive shared-memory slots (distinct banks)
    for (int u = 0; u < kLoadBatch; ++u) {
      const int idx = i0 + u * (int)blockDim.x;
      const int sl = idx / TX;
      const int j = idx < total ? bitrev(sl, logn) : 0;
      const int64_t col = x0 + (idx - sl * TX);
      v[u] = (idx < total && col < ncols) ? cvt<T>(X[(int64_t)j * ldx + col]) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kLoadBatch; ++u) {
      const int idx = i0 + u * (int)blockDim.x;
      if (idx < total) {
        const int sl = idx / TX;
        const int c = idx - sl * TX;
        T *slot = reinterpret_cast<T *>(&buf[(size_t)(c >> 1) * series_stride(n) + sl]);
        slot[c & 1] = rs ? v[u] * rs[bitrev(sl, logn)] : v[u];
        ss += v[u] * v[u];
      }
    }
  }
  __syncthreads();
  fft_smem<T>(buf, n, logn, TX >> 1, tw);
  r2c_store<T, TX>(buf, n, logn, x0, ncols, S, lds);
  if (rn.part) rhs_norm_finish((float)ss, rn);
}

// Same transform of the 1D FP64 residual r = G_t + u_{t-1} - (I + tau K) u_t, formed
// while the tile is loaded (rx = (tau lo, 1 + tau diag, tau up)); neighbour columns
// outside the tile come from L1/L2.
template <typename T, int TX>
__global__ void __launch_bounds__(kFftMaxThreads, 2) k_fft_r2c_res(const double *__restrict__ G, const double *__restrict__ U,
                                                     int64_t ncols, int n, int logn, const double *__restrict__ rxl,
                                                     const double *__restrict__ rxd,
                                                     const double *__restrict__ rxu,
                                                     const cpx<T> *__restrict__ tw, cpx<T> *__restrict__ S,
                                                     int64_t lds, const T *__restrict__ rs,
                                                     const int *__restrict__ mex, int mnx, RhsNorm rn) {
  grid_dep_wait();
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T> *buf = reinterpret_cast<cpx<T> *>(smraw);
  const int64_t x0 = (int64_t)blockIdx.x * TX;
  const int total = n * TX;
  // blockDim.x is a multiple of TX, so every element a thread loads lies in one
  // column: its residual coefficients are loaded once
  const int c = (int)threadIdx.x % TX;
  const int64_t col = x0 + c;
  const bool live = col < ncols;
  const double cl = (live && col > 0) ? rxl[col] : 0.0;
  const double cd = live ? rxd[col] : 0.0;
  const double cu = (live && col + 1 < ncols) ? rxu[col] : 0.0;
  const int64_t ol = col > 0 ? -1 : 0, ou = col + 1 < ncols ? 1 : 0;  // in-range neighbour offsets
  // batched plans: problem (col / mnx) scaled by 2^mex[problem] (exact)
  const T msc = (mex && live) ? (T)ldexp(1.0, mex[col / mnx]) : T(1);
  T *col_buf = reinterpret_cast<T *>(buf + (size_t)(c >> 1) * series_stride(n)) + (c & 1);
  constexpr int kB = kLoadBatch / 2;  // five FP64 loads per element
  T ss = T(0);  // squares of the residual (rn)
  // the threads of a warp take consecutive bit-reversed slots s (time row j = bitrev(s)), so
  // their shared-memory stores hit distinct banks; each row is its own sector either way
  for (int s0 = (int)threadIdx.x / TX; s0 < n; s0 += kB * ((int)blockDim.x / TX)) {
    double g[kB], um[kB], ul[kB], uc[kB], ur[kB];
#pragma unroll
    for (int q = 0; q < kB; ++q) {
      const int sq = s0 + q * ((int)blockDim.x / TX);
      const int j = sq < n ? bitrev(sq, logn) : n;
      const bool in = live && j < n;
      const double *u = U + (int64_t)j * ncols + col;
      g[q] = in ? G[(int64_t)j * ncols + col] : 0.0;
      uc[q] = in ? u[0] : 0.0;
      ul[q] = in ? u[ol] : 0.0;
      ur[q] = in ? u[ou] : 0.0;
      um[q] = (in && j > 0) ? u[-ncols] : 0.0;
    }
#pragma unroll
    for (int q = 0; q < kB; ++q) {
      const int sq = s0 + q * ((int)blockDim.x / TX);
      if (sq < n) {
        const int j = bitrev(sq, logn);
        // four FP64 operations per element (GB300 runs FP64 at ~1/64 of the FP32 rate)
        const double res = fma(-cu, ur[q], fma(-cl, ul[q], fma(-cd, uc[q], g[q] + um[q])));
        const T r = cvt<T>(res) * msc;
        col_buf[2 * sq] = rs ? r * rs[j] : r;
        ss += r * r;
      }
    }
  }
  __syncthreads();
  fft_smem<T>(buf, n, logn, TX >> 1, tw);
  r2c_store<T, TX>(buf, n, logn, x0, ncols, S, lds);
  if (rn.part) rhs_norm_finish((float)ss, rn);
}

// Inverse: Z[k] = A[k] + i B[k] over the full spectrum (A[n-k] = conj A[k]);
// z = IDFT(Z) = conj(DFT(conj Z)) / n; column 2p = Re z, column 2p+1 = Im z.
template <typename T, int TX, bool R16>
__global__ void __launch_bounds__(256) k_fft_c2r(const cpx<T> *__restrict__ S, int64_t lds, int64_t ncols,
                                                 int n, int logn, const cpx<T> *__restrict__ tw,
                                                 void *__restrict__ out, int64_t ldo, int mode,
                                                 double *__restrict__ norm_part, StepFinish fin,
                                                 const T *__restrict__ rsi, double *__restrict__ colsum,
                                                 const int *__restrict__ mex, int mnx, const int *skip) {
  grid_dep_wait();
  if (skip && *skip) return;  // U already holds the result (Algorithm 3's U_1 exit)
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T> *buf = reinterpret_cast<cpx<T> *>(smraw);
  const int64_t x0 = (int64_t)blockIdx.x * TX;
  const int np = TX >> 1;
  const int half = n >> 1;
  if constexpr (R16) {  // radix-16 first stage in registers (see k_fft_r2c16)
    const int SS = series_stride16(n), nb = n >> 4, lb = logn - 4;
    for (int it = threadIdx.x; it < np * nb; it += blockDim.x) {
      const int p = it % np, g = it / np;
      const int r = bitrev(g, lb);
      const int64_t ca = x0 + 2 * p, cb = ca + 1;
      cpx<T> z[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int idx = r + i * nb;
        const int kk = idx <= half ? idx : n - idx;
        const cpx<T> A = ca < ncols ? S[(int64_t)kk * lds + ca] : mk<T>(T(0), T(0));
        const cpx<T> B = cb < ncols ? S[(int64_t)kk * lds + cb] : mk<T>(T(0), T(0));
        // conj(A + i B) at kk <= n/2; the conjugate half at n - kk
        z[i] = idx <= half ? mk<T>(A.x - B.y, -(A.y + B.x)) : mk<T>(A.x + B.y, A.y - B.x);
      }
      dft16(z);
      cpx<T> *blk = buf + (size_t)p * SS + 17 * g;
#pragma unroll
      for (int k = 0; k < 16; ++k) blk[k] = z[k];
    }
    __syncthreads();
    fft_smem16<T>(buf, n, logn, np, SS, tw);
  } else {
    // each stored row kk <= n/2 is loaded once and fills both Z[kk] and Z[n - kk]
    const int total = (half + 1) * np;
    for (int i0 = threadIdx.x; i0 < total; i0 += kLoadBatch * blockDim.x) {
      cpx<T> A[kLoadBatch], B[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = i0 + u * (int)blockDim.x;
        const int kk = idx / np;
        const int p = idx - kk * np;
        const int64_t ca = x0 + 2 * p, cb = ca + 1;
        A[u] = mk<T>(T(0), T(0));
        B[u] = mk<T>(T(0), T(0));
        if (idx < total && ca < ncols) A[u] = S[(int64_t)kk * lds + ca];
        if (idx < total && cb < ncols) B[u] = S[(int64_t)kk * lds + cb];
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = i0 + u * (int)blockDim.x;
        if (idx < total) {
          const int kk = idx / np;
          const int p = idx - kk * np;
          cpx<T> *ser = buf + (size_t)p * series_stride(n);
          // conj(A + i B) = (A.x - B.y) - i (A.y + B.x); at n - kk the conjugate half
          // gives (A.x + B.y) + i (A.y - B.x)
          ser[bitrev(kk, logn)] = mk<T>(A[u].x - B[u].y, -(A[u].y + B[u].x));
          if (kk > 0 && kk < half) ser[bitrev(n - kk, logn)] = mk<T>(A[u].x + B[u].y, A[u].y - B[u].x);
        }
      }
    }
    __syncthreads();
    fft_smem<T>(buf, n, logn, np, tw);
  }
  T inv_n = T(1) / T(n);
  if (mex) {  // batched plans: undo the problem's 2^mex scaling (every element a thread
              // writes lies in column x0 + threadIdx.x % TX)
    const int64_t c0 = x0 + (int64_t)(threadIdx.x % TX);
    if (c0 < ncols) inv_n = (T)ldexp((double)inv_n, -mex[c0 / mnx]);
  }
  float ss = 0.0f;  // a few dozen squares per thread; the stop rule needs a few digits
  const int tot2 = n * TX;
  for (int i0 = threadIdx.x; i0 < tot2; i0 += kEpiBatch * blockDim.x) {
    double old[kEpiBatch];  // U before the update (mode 1)
#pragma unroll
    for (int u = 0; u < kEpiBatch; ++u) {
      const int idx = i0 + u * (int)blockDim.x;
      const int j = idx / TX;
      const int64_t col = x0 + (idx - j * TX);
      old[u] = (mode == 1 && idx < tot2 && col < ncols) ? reinterpret_cast<const double *>(out)[(int64_t)j * ldo + col]
                                                         : 0.0;
    }
#pragma unroll
    for (int u = 0; u < kEpiBatch; ++u) {
      const int idx = i0 + u * (int)blockDim.x;
      const int j = idx / TX;
      const int c = idx - j * TX;
      const int64_t col = x0 + c;
      if (idx >= tot2 || col >= ncols) continue;
      const cpx<T> r = R16 ? buf[(size_t)(c >> 1) * series_stride16(n) + pz(j)]
                           : buf[(size_t)(c >> 1) * series_stride(n) + j];
      const T sc = rsi ? inv_n * rsi[j] : inv_n;
      const T v = ((c & 1) == 0) ? r.x * sc : -r.y * sc;
      const int64_t o = (int64_t)j * ldo + col;
      if (mode == 0) {
        reinterpret_cast<double *>(out)[o] = cvt<double>(v);
      } else if (mode == 1) {
        reinterpret_cast<double *>(out)[o] = old[u] + cvt<double>(v);
      } else {
        reinterpret_cast<float *>(out)[o] = (float)v;
      }
      const float vf = (float)v;
      ss = fmaf(vf, vf, ss);
    }
  }
  if (colsum) {
    // per-column sums of squares: blockDim.x is a multiple of TX, so every element a
    // thread wrote lies in column threadIdx.x % TX
    __shared__ double cred[256];
    cred[threadIdx.x] = (double)ss;
    __syncthreads();
    if ((int)threadIdx.x < TX) {
      double t = 0.0;
      for (int i = threadIdx.x; i < (int)blockDim.x; i += TX) t += cred[i];
      if (x0 + threadIdx.x < ncols) colsum[x0 + threadIdx.x] = t;
    }
  }
  if (norm_part) {
    const double sd = warp_sum((double)ss);
    __shared__ double red[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = sd;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
      norm_part[blockIdx.x] = t;
    }
    if (fin.enabled) {
      // the last CTA to finish (no CTA waits) sums the squares and decides
      __shared__ int last;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) last = atomicAdd(fin.counter, 1) == (int)gridDim.x - 1;
      __syncthreads();
      if (last) {
        __threadfence();
        // every thread loads its share at once (the partials sit in L2, possibly on the
        // other die: one round trip instead of one per partial), then a fixed-order sum
        double t = 0.0;
#pragma unroll 4
        for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += norm_part[i];
        t = warp_sum(t);
        if (l == 0) red[w] = t;
        __syncthreads();
        if (threadIdx.x == 0) {
          t = 0.0;
          for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
          fin.scal[S_D2] = t;
          *fin.counter = 0;
          refine_decide(fin.scal, fin.flags, fin.rc, fin.use_handle, fin.h);
        }
      }
    }
  }
}

// The FP64 all-at-once residual as the DST's input (ResIn.G != null): element (row y, column
// col) of slab s (time t = s / batch, problem b = s % batch) is
// r = G_t + u_{t-1} - [(I + tau T_x) u_t + tau T_y u_t] at row b nym + y of the stacked grid
// (ny = batch nym rows, x-coefficients of problem b), times 2^mex[b] for batches: five
// FMAs in FP64 per element after G_t + u_{t-1} (the diagonal 1 + tau (d_x + d_y) comes
// precombined per grid point in rdd), formed while the DST loads its tile.
struct ResIn {
  const double *G, *U;
  const double *rxl, *rdd, *rxu, *ryl, *ryu;
  int ny, nym, batch;
  const int *mex;
};

// Orthonormal DST-I along y via a length N = 2(ny+1) complex FFT of the odd
// extension, two x-columns packed per series (a + i b):
//   DST_l(a) = -Im Z[l] / 2,  DST_l(b) = Re Z[l] / 2,  scaled by sqrt(2/(ny+1)).
// RES: the input is the residual of ResIn, staged once per element in shared memory
// (TX columns x ny rows of T after the series), so that its FP64 work is done once.
// Binary32 variants: 48 registers, five 256-thread CTAs per SM (the load-latency-bound
// transforms measured 5 % faster than at four, despite a few dozen bytes of spills).
template <typename Tin, typename Tout, typename T, int TX, bool R16, bool RES>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 1) k_dst_y(const Tin *__restrict__ X, Tout *__restrict__ Y, int64_t ny,
                                               int64_t nx, int N, int logN,
                                               const cpx<T> *__restrict__ tw, T scale, int mode, const int *skip,
                                               ResIn rin, size_t res_off) {
  grid_dep_wait();
  if (skip && *skip) return;  // U already holds the result (Algorithm 3's U_1 exit)
  extern __shared__ __align__(16) unsigned char smraw[];
  cpx<T> *buf = reinterpret_cast<cpx<T> *>(smraw);
  const int ntile = (int)((nx + TX - 1) / TX);
  const int64_t t = blockIdx.x / ntile;
  const int64_t x0 = (int64_t)(blockIdx.x % ntile) * TX;
  const Tin *Xt = X + t * ny * nx;
  Tout *Yt = Y + t * ny * nx;
  const int np = TX >> 1;
  const int total = (int)ny * TX;
  T *rt = reinterpret_cast<T *>(smraw + res_off);  // RES: the residual tile, [y][c]
  if constexpr (RES) {
    const int64_t tt = t / rin.batch;                // time step
    const int b = (int)(t - tt * rin.batch);         // problem
    const int64_t nb = (int64_t)rin.ny * nx;         // unknowns per time row
    const double msc = rin.mex ? ldexp(1.0, rin.mex[b]) : 1.0;
    for (int i0 = threadIdx.x; i0 < total; i0 += kLoadBatch * blockDim.x) {
      double rv[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = i0 + u * (int)blockDim.x;
        const int y = idx / TX;
        const int c = idx - y * TX;
        const int64_t col = x0 + c;
        double r = 0.0;
        if (idx < total && col < nx) {
          const int iy = b * rin.nym + y;
          const int64_t j = (int64_t)iy * nx + col;
          const int64_t cx = (int64_t)b * nx + col;  // x-coefficients of problem b
          const double *u = rin.U + tt * nb;
          r = rin.G[tt * nb + j];
          if (tt > 0) r += u[j - nb];
          r = fma(-rin.rdd[j], u[j], r);
          if (col > 0) r = fma(-rin.rxl[cx], u[j - 1], r);
          if (col + 1 < nx) r = fma(-rin.rxu[cx], u[j + 1], r);
          if (iy > 0) r = fma(-rin.ryl[iy], u[j - nx], r);
          if (iy + 1 < rin.ny) r = fma(-rin.ryu[iy], u[j + nx], r);
        }
        rv[u] = r;
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = i0 + u * (int)blockDim.x;
        if (idx < total) rt[idx] = cvt<T>(rin.mex ? rv[u] * msc : rv[u]);
      }
    }
    __syncthreads();
  }
  // element (y, col) of the tile's input
  auto in_at = [&](int y, int64_t col) -> T {
    if constexpr (RES)
      return rt[y * TX + (int)(col - x0)];
    else
      return cvt<T>(Xt[(int64_t)y * nx + col]);
  };
  if constexpr (R16) {  // radix-16 first stage in registers (see k_fft_r2c16)
    const int SS = series_stride16(N), nb = N >> 4, lb = logN - 4, half = N >> 1;
    for (int it = threadIdx.x; it < np * nb; it += blockDim.x) {
      const int p = it % np, g = it / np;
      const int r = bitrev(g, lb);
      const int64_t ca = x0 + 2 * p, cb = ca + 1;
      cpx<T> z[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        // odd extension of length N = 2 (ny + 1): 0 at 0 and N/2, x_{idx-1} below N/2,
        // -x_{N-idx-1} above
        const int idx = r + i * nb;
        const bool zero = idx == 0 || idx == half;
        const int y = idx < half ? idx - 1 : N - idx - 1;
        const T sg = idx < half ? T(1) : T(-1);
        const int yy = zero ? 0 : y;
        z[i] = mk<T>((!zero && ca < nx) ? sg * in_at(yy, ca) : T(0), (!zero && cb < nx) ? sg * in_at(yy, cb) : T(0));
      }
      dft16(z);
      cpx<T> *blk = buf + (size_t)p * SS + 17 * g;
#pragma unroll
      for (int k = 0; k < 16; ++k) blk[k] = z[k];
    }
    __syncthreads();
    fft_smem16<T>(buf, N, logN, np, SS, tw);
  } else {
    // the odd extension: entries 0 and ny + 1 = N/2 are zero (bit-reversed slots 0 and 1),
    // the scatter below writes the rest
    for (int idx = threadIdx.x; idx < 2 * np; idx += blockDim.x)
      buf[(size_t)(idx >> 1) * series_stride(N) + bitrev((idx & 1) ? (N >> 1) : 0, logN)] = mk<T>(T(0), T(0));
    for (int i0 = threadIdx.x; i0 < total; i0 += kLoadBatch * blockDim.x) {
      T v[kLoadBatch];
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = i0 + u * (int)blockDim.x;
        const int y = idx / TX;
        const int64_t col = x0 + (idx - y * TX);
        v[u] = (idx < total && col < nx) ? in_at(y, col) : T(0);
      }
#pragma unroll
      for (int u = 0; u < kLoadBatch; ++u) {
        const int idx = i0 + u * (int)blockDim.x;
        if (idx >= total) continue;
        const int y = idx / TX;
        const int c = idx - y * TX;
        cpx<T> *ser = buf + (size_t)(c >> 1) * series_stride(N);
        T *pos = reinterpret_cast<T *>(&ser[bitrev(y + 1, logN)]);
        T *neg = reinterpret_cast<T *>(&ser[bitrev(N - (y + 1), logN)]);
        pos[c & 1] = v[u];
        neg[c & 1] = -v[u];
      }
    }
    __syncthreads();
    fft_smem<T>(buf, N, logN, np, tw);
  }
  for (int i0 = threadIdx.x; i0 < total; i0 += kEpiBatch * blockDim.x) {
    Tout old[kEpiBatch];  // Y before the update (mode 1)
#pragma unroll
    for (int u = 0; u < kEpiBatch; ++u) {
      const int idx = i0 + u * (int)blockDim.x;
      const int l = idx / TX;
      const int64_t col = x0 + (idx - l * TX);
      old[u] = (mode != 0 && idx < total && col < nx) ? Yt[(int64_t)l * nx + col] : Tout(0);
    }
#pragma unroll
    for (int u = 0; u < kEpiBatch; ++u) {
      const int idx = i0 + u * (int)blockDim.x;
      const int l = idx / TX;  // output index l = 0..ny-1  <->  mode l+1
      const int c = idx - l * TX;
      const int64_t col = x0 + c;
      if (idx >= total || col >= nx) continue;
      const cpx<T> z = R16 ? buf[(size_t)(c >> 1) * series_stride16(N) + pz(l + 1)]
                           : buf[(size_t)(c >> 1) * series_stride(N) + l + 1];
      const T v = ((c & 1) == 0) ? (T(-0.5) * scale) * z.y : (T(0.5) * scale) * z.x;
      const int64_t o = (int64_t)l * nx + col;
      if (mode == 0) {
        Yt[o] = cvt<Tout>(v);
      } else {
        Yt[o] = old[u] + cvt<Tout>(v);
      }
    }
  }
}

static int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// Columns per CTA: as many as fit ~96 KB of series (two CTAs per SM), capped,
// then narrowed (down to 4 columns = one 32-byte sector of doubles per row) until
// the grid covers every SM four times.
// The radix-16 first stage serves the binary32 transforms of n >= 16 points; the FP64 ones
// (bound by GB300's FP64 pipe, where the register stage lowered occupancy) keep the
// in-place radix-4 passes.
// Ctx::fft_radix (pd_desc.tune_fft_radix) overrides the choice.
template <typename T>
static bool use_r16(const Ctx &c, int n) {
  if (n < 16 || c.fft_radix == 4) return false;
  return c.fft_radix == 16 || sizeof(T) == 4;
}
// Series stride of a tile in shared memory: the radix-16 layout or n + 1.
template <typename T>
static int fft_sst(const Ctx &c, int n) {
  return use_r16<T>(c, n) ? series_stride16(n) : series_stride(n);
}
// Threads of a radix-16 launch: one (column pair, block) item each, within [64, maxt].
static int fft16_threads(int items, int maxt) { return std::max(64, std::min(maxt, (items + 31) / 32 * 32)); }

template <typename T>
static int pick_tx(const Ctx &c, int n, int cap, int64_t ncols, int req = 0) {
  const size_t budget = 96 * 1024;
  const size_t sst = (size_t)fft_sst<T>(c, n);
  if (req) {  // the caller's choice, within the shared-memory budget of one CTA
    int tx = std::min(req, cap);
    while (tx > 2 && (size_t)(tx / 2) * sst * sizeof(cpx<T>) > 2 * budget) tx >>= 1;
    return tx;
  }
  int tx = cap;
  while (tx > 2 && (size_t)(tx / 2) * sst * sizeof(cpx<T>) > budget) tx >>= 1;
  while (tx > 4 && (ncols + tx - 1) / tx < 4 * (int64_t)sm_count()) tx >>= 1;
  return tx;
}

// Instantiate the body for the tile width chosen at run time (kTX is a constant).
#define PD_TX_DISPATCH(TX, ...)                        \
  switch (TX) {                                        \
    case 2: { constexpr int kTX = 2; __VA_ARGS__; } break;  \
    case 4: { constexpr int kTX = 4; __VA_ARGS__; } break;  \
    case 8: { constexpr int kTX = 8; __VA_ARGS__; } break;  \
    default: { constexpr int kTX = 16; __VA_ARGS__; } break; \
  }

template <typename T, typename Tin>
void launch_fft_r2c(Ctx &c, const Tin *X, int64_t ldx, int64_t ncols, int n, const cpx<T> *tw,
                    cpx<T> *S, int64_t lds, const T *rs, const RhsNorm *rnp) {
  const RhsNorm rn = rnp ? *rnp : RhsNorm{nullptr, nullptr, nullptr};
  const int logn = ilog2(n);
  const int TX = pick_tx<T>(c, n, sizeof(T) == 8 ? 8 : 16, ncols, c.fft_cols);
  const size_t smem = (size_t)(TX / 2) * fft_sst<T>(c, n) * sizeof(cpx<T>);
  const int grid = (int)((ncols + TX - 1) / TX);
  const double bytes = (double)n * ncols * sizeof(Tin) + (double)(n / 2 + 1) * ncols * sizeof(cpx<T>);
  c.launch(sizeof(T) == 8 ? "fft_r2c_f64" : "fft_r2c_f32", bytes, [&] {
    PD_TX_DISPATCH(TX, {
      if (use_r16<T>(c, n)) {
        const int thr = fft16_threads((kTX / 2) * (n / 16), 512);
        if (smem > 48 * 1024)
          allow_dyn_smem((const void *)k_fft_r2c16<T, Tin, kTX>);
        pdl_launch(c.pdl, k_fft_r2c16<T, Tin, kTX>, dim3(grid), dim3(thr), smem, c.stream, X, ldx, ncols, n, logn, tw,
                   S, lds, rs, rn);
      } else {
        if (smem > 48 * 1024)
          allow_dyn_smem((const void *)k_fft_r2c<T, Tin, kTX>);
        pdl_launch(c.pdl, k_fft_r2c<T, Tin, kTX>, dim3(grid), dim3(fft_threads(n, kTX)), smem, c.stream, X, ldx, ncols,
                   n, logn, tw, S, lds, rs, rn);
      }
    })
  });
}

template <typename T>
void launch_fft_r2c_residual(Ctx &c, const double *G, const double *U, int64_t ncols, int n, const double *rxl,
                             const double *rxd, const double *rxu, const cpx<T> *tw, cpx<T> *S, int64_t lds,
                             const T *rs, const int *mex, int mnx, const RhsNorm *rnp) {
  const RhsNorm rn = rnp ? *rnp : RhsNorm{nullptr, nullptr, nullptr};
  const int logn = ilog2(n);
  const int TX = pick_tx<T>(c, n, sizeof(T) == 8 ? 8 : 16, ncols, c.fft_cols);
  const size_t smem = (size_t)(TX / 2) * series_stride(n) * sizeof(cpx<T>);
  const int grid = (int)((ncols + TX - 1) / TX);
  const double bytes = (double)n * ncols * 16.0 + (double)(n / 2 + 1) * ncols * sizeof(cpx<T>);
  c.launch(sizeof(T) == 8 ? "fft_r2c_res_f64" : "fft_r2c_res_f32", bytes, [&] {
    PD_TX_DISPATCH(TX, {
      if (smem > 48 * 1024)
        allow_dyn_smem((const void *)k_fft_r2c_res<T, kTX>);
      pdl_launch(c.pdl, k_fft_r2c_res<T, kTX>, dim3(grid), dim3(fft_threads(n, kTX)), smem, c.stream, G, U, ncols, n,
                 logn, rxl, rxd, rxu, tw, S, lds, rs, mex, mnx, rn);
    })
  });
}

template <typename T>
void launch_fft_c2r(Ctx &c, const cpx<T> *S, int64_t lds, int64_t ncols, int n, const cpx<T> *tw,
                    void *out, int64_t ldo, int mode, double *norm_part, int *nparts, const StepFinish *finp,
                    const T *rsi, double *colsum, const int *mex, int mnx, const int *skip) {
  StepFinish fin{};
  if (finp && norm_part) fin = *finp;
  const int logn = ilog2(n);
  const int TX = pick_tx<T>(c, n, sizeof(T) == 8 ? 8 : 16, ncols, c.fft_cols);
  const size_t smem = (size_t)(TX / 2) * fft_sst<T>(c, n) * sizeof(cpx<T>);
  const int grid = (int)((ncols + TX - 1) / TX);
  if (nparts) *nparts = grid;
  const double obytes = (mode == 2) ? 4.0 : (mode == 1 ? 16.0 : 8.0);
  const double bytes = (double)(n / 2 + 1) * ncols * sizeof(cpx<T>) + (double)n * ncols * obytes;
  c.launch(sizeof(T) == 8 ? "fft_c2r_f64" : "fft_c2r_f32", bytes, [&] {
    PD_TX_DISPATCH(TX, {
      if (use_r16<T>(c, n)) {
        const int thr = fft16_threads((kTX / 2) * (n / 16), 256);
        if (smem > 48 * 1024)
          allow_dyn_smem((const void *)k_fft_c2r<T, kTX, true>);
        pdl_launch(c.pdl, k_fft_c2r<T, kTX, true>, dim3(grid), dim3(thr), smem, c.stream, S, lds, ncols, n, logn, tw, out,
                   ldo, mode, norm_part, fin, rsi, colsum, mex, mnx, skip);
      } else {
        if (smem > 48 * 1024)
          allow_dyn_smem((const void *)k_fft_c2r<T, kTX, false>);
        pdl_launch(c.pdl, k_fft_c2r<T, kTX, false>, dim3(grid), dim3(256), smem, c.stream, S, lds, ncols, n, logn, tw,
                   out, ldo, mode, norm_part, fin, rsi, colsum, mex, mnx, skip);
      }
    })
  });
}

template <typename Tin, typename Tout, typename T, bool RES>
static void dst_launch(Ctx &c, const Tin *X, Tout *Y, int64_t nslab, int64_t ny, int64_t nx, const cpx<T> *tw,
                       int mode, const int *skip, const ResIn &rin, const char *fam, double bytes) {
  const int N = (int)(2 * (ny + 1));
  const int logN = ilog2(N);
  const int TX = pick_tx<T>(c, N, sizeof(T) == 8 ? 8 : 16, nslab * nx);
  const size_t ser = (size_t)(TX / 2) * fft_sst<T>(c, N) * sizeof(cpx<T>);
  const size_t res_off = (ser + 15) & ~(size_t)15;
  const size_t smem = RES ? res_off + (size_t)ny * TX * sizeof(T) : ser;
  const int ntile = (int)((nx + TX - 1) / TX);
  const int64_t grid = nslab * ntile;
  const T scale = (T)sqrt(2.0 / (double)(ny + 1));
  c.launch(fam, bytes, [&] {
    PD_TX_DISPATCH(TX, {
      if (use_r16<T>(c, N)) {
        if (smem > 48 * 1024)
          allow_dyn_smem((const void *)k_dst_y<Tin, Tout, T, kTX, true, RES>);
        pdl_launch(c.pdl, k_dst_y<Tin, Tout, T, kTX, true, RES>, dim3((unsigned)grid), dim3(256), smem, c.stream, X, Y,
                   ny, nx, N, logN, tw, scale, mode, skip, rin, res_off);
      } else {
        if (smem > 48 * 1024)
          allow_dyn_smem((const void *)k_dst_y<Tin, Tout, T, kTX, false, RES>);
        pdl_launch(c.pdl, k_dst_y<Tin, Tout, T, kTX, false, RES>, dim3((unsigned)grid), dim3(256), smem, c.stream, X,
                   Y, ny, nx, N, logN, tw, scale, mode, skip, rin, res_off);
      }
    })
  });
}

template <typename Tin, typename Tout, typename T>
void launch_dst_y(Ctx &c, const Tin *X, Tout *Y, int64_t nt, int64_t ny, int64_t nx, const cpx<T> *tw,
                  int mode, const int *skip) {
  const double bytes = (double)nt * ny * nx * (sizeof(Tin) + sizeof(Tout) * (mode ? 2 : 1));
  dst_launch<Tin, Tout, T, false>(c, X, Y, nt, ny, nx, tw, mode, skip, ResIn{}, sizeof(T) == 8 ? "dst_y_f64" : "dst_y_f32",
                                  bytes);
}

template <typename T>
void launch_dst_y_residual(Ctx &c, const double *G, const double *U, T *Y, int64_t nt, int batch, int64_t nym,
                           int64_t nx, const double *rxl, const double *rdd, const double *rxu, const double *ryl,
                           const double *ryu, const int *mex, const cpx<T> *tw) {
  ResIn rin{G, U, rxl, rdd, rxu, ryl, ryu, (int)(nym * batch), (int)nym, batch, mex};
  // G and U read once (neighbours from the caches), the binary32 / FP64 transform written
  const double bytes = (double)nt * batch * nym * nx * (16.0 + sizeof(T));
  dst_launch<double, T, T, true>(c, (const double *)nullptr, Y, nt * batch, nym, nx, tw, 0, nullptr, rin,
                                 sizeof(T) == 8 ? "dst_y_res_f64" : "dst_y_res_f32", bytes);
}

template void launch_fft_r2c<double, double>(Ctx &, const double *, int64_t, int64_t, int, const cpx<double> *,
                                             cpx<double> *, int64_t, const double *, const RhsNorm *);
template void launch_fft_r2c<float, double>(Ctx &, const double *, int64_t, int64_t, int, const cpx<float> *,
                                            cpx<float> *, int64_t, const float *, const RhsNorm *);
template void launch_fft_r2c<float, float>(Ctx &, const float *, int64_t, int64_t, int, const cpx<float> *,
                                           cpx<float> *, int64_t, const float *, const RhsNorm *);
template void launch_fft_c2r<double>(Ctx &, const cpx<double> *, int64_t, int64_t, int, const cpx<double> *,
                                     void *, int64_t, int, double *, int *, const StepFinish *, const double *,
                                     double *, const int *, int, const int *);
template void launch_fft_c2r<float>(Ctx &, const cpx<float> *, int64_t, int64_t, int, const cpx<float> *,
                                    void *, int64_t, int, double *, int *, const StepFinish *, const float *,
                                    double *, const int *, int, const int *);
template void launch_fft_r2c_residual<double>(Ctx &, const double *, const double *, int64_t, int, const double *,
                                              const double *, const double *, const cpx<double> *, cpx<double> *,
                                              int64_t, const double *, const int *, int, const RhsNorm *);
template void launch_fft_r2c_residual<float>(Ctx &, const double *, const double *, int64_t, int, const double *,
                                             const double *, const double *, const cpx<float> *, cpx<float> *,
                                             int64_t, const float *, const int *, int, const RhsNorm *);
template void launch_dst_y<double, double, double>(Ctx &, const double *, double *, int64_t, int64_t, int64_t,
                                                   const cpx<double> *, int, const int *);
template void launch_dst_y<double, float, float>(Ctx &, const double *, float *, int64_t, int64_t, int64_t,
                                                 const cpx<float> *, int, const int *);
template void launch_dst_y<float, float, float>(Ctx &, const float *, float *, int64_t, int64_t, int64_t,
                                                const cpx<float> *, int, const int *);
template void launch_dst_y<float, double, float>(Ctx &, const float *, double *, int64_t, int64_t, int64_t,
                                                 const cpx<float> *, int, const int *);
template void launch_dst_y_residual<float>(Ctx &, const double *, const double *, float *, int64_t, int, int64_t,
                                           int64_t, const double *, const double *, const double *, const double *,
                                           const double *, const int *, const cpx<float> *);
template void launch_dst_y_residual<double>(Ctx &, const double *, const double *, double *, int64_t, int, int64_t,
                                            int64_t, const double *, const double *, const double *, const double *,
                                            const double *, const int *, const cpx<double> *);

}  // namespace pd
