// Shared device helpers for the ParaDiag kernels (complex arithmetic, team
// barriers, warp reductions).  Internal header; not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pd {

// Interleaved complex number of real type T (layout-compatible with float2 /
// double2 and with numpy complex64 / complex128).
template <typename T>
struct alignas(2 * sizeof(T)) cpx {
  T x, y;
};

template <typename T>
__host__ __device__ __forceinline__ cpx<T> mk(T a, T b) {
  cpx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cpx<T> add(cpx<T> a, cpx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> sub(cpx<T> a, cpx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cpx<T> mul(cpx<T> a, cpx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cpx<T> scal(T s, cpx<T> a) { return mk<T>(s * a.x, s * a.y); }
template <typename T>
__device__ __forceinline__ cpx<T> conjg(cpx<T> a) { return mk<T>(a.x, -a.y); }
// a - b * c
template <typename T>
__device__ __forceinline__ cpx<T> fnms(cpx<T> a, cpx<T> b, cpx<T> c) {
  return mk<T>(a.x - b.x * c.x + b.y * c.y, a.y - b.x * c.y - b.y * c.x);
}
// a - s * c with real s
template <typename T>
__device__ __forceinline__ cpx<T> fnms_r(cpx<T> a, T s, cpx<T> c) { return mk<T>(a.x - s * c.x, a.y - s * c.y); }
// 1 / a  =  conj(a) / |a|^2.  The operands met here are bounded away from zero and
// from overflow (|a| between ~1e-3 and ~1e8), so no Smith-style scaling is needed.
// binary32: the hardware approximation (rcp.approx.ftz, at most 1 ulp from 1/v) refined
// by one Newton-Raphson step, r + r (1 - v r).  The step roughly squares the relative
// error of the approximation and adds the rounding of two fused operations, so the
// result is within 1 ulp of 1/v but NOT always correctly rounded; .ftz flushes
// subnormal operands and results to zero, which normal-range operands never produce.
// paradiag_recip_f32 exposes this function so that a test can bound its error against
// the correctly rounded reciprocal.  binary64: __drcp_rn, correctly rounded.
__device__ __forceinline__ float rcp_nr(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return fmaf(r, fmaf(-v, r, 1.0f), r);
}
__device__ __forceinline__ double rcp_nr(double v) { return __drcp_rn(v); }
template <typename T>
__device__ __forceinline__ cpx<T> recip(cpx<T> a) {
  const T d = rcp_nr(a.x * a.x + a.y * a.y);  // 1 / |a|^2 (within 1 ulp in binary32)
  return mk<T>(a.x * d, -a.y * d);
}
template <typename T>
__device__ __forceinline__ T abs2(cpx<T> a) { return a.x * a.x + a.y * a.y; }

template <typename T>
__device__ __forceinline__ T shfl_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Barrier over a team of P threads (P a multiple of 32) inside a CTA that holds
// blockDim.x / P teams.  Team 0..(teams-1) use named barriers 1..teams.
__device__ __forceinline__ void team_sync(int P, int team_in_cta) {
  if (P == 32) {
    __syncwarp();
  } else if (P == (int)blockDim.x) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(1 + team_in_cta), "r"(P) : "memory");
  }
}

// binary64 -> binary32 by integer operations on the bit pattern: GB300 issues FP64
// instructions, conversions included, at a small fraction of its FP32 and integer rates, and
// the binary32 path converts every FP64 element it loads (in the kernels that also run FP64
// arithmetic, such as the residual, this frees the FP64 pipe; measured 8% on the 2D residual
// DST).  The significand is truncated (error below one binary32 ulp, where round-to-nearest
// gives half an ulp); magnitudes below binary32's normal range become zero, above it
// infinity; NaN stays NaN.  binary32 -> binary64 keeps the hardware conversion, which
// measured faster than its integer form.
__device__ __forceinline__ float f64_to_f32_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  const int ef = e - 896;  // binary32 biased exponent: e - 1023 + 127
  unsigned r;
  if (ef >= 255) {
    r = sign | 0x7f800000u | ((e == 0x7ff && ((hi & 0xfffffu) | lo)) ? 0x00400000u : 0u);
  } else if (ef <= 0) {
    r = sign;
  } else {
    r = sign | ((unsigned)ef << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  }
  return __uint_as_float(r);
}
// cvt<To>(x): x in type To, binary64 -> binary32 through the integer conversion above.
template <typename To, typename From>
__device__ __forceinline__ To cvt(From x) {
  if constexpr (sizeof(To) == 4 && sizeof(From) == 8)
    return f64_to_f32_bits(x);
  else
    return (To)x;
}

// Programmatic dependent launch: every kernel of this library opens with this wait,
// so a kernel scheduled early (while its predecessor in the stream drains) reads
// nothing before the predecessor has completed; without such a launch it returns at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ int bitrev(int j, int logn) {
  return logn == 0 ? 0 : (int)(__brev((unsigned)j) >> (32 - logn));
}

}  // namespace pd
