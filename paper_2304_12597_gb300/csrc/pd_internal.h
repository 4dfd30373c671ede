// Internal host-side interfaces shared by the .cu files of the library:
// launch context with per-kernel CUDA-event tracing, and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "pd_common.cuh"

namespace pd {

// Launch context: the stream every kernel is ordered on, a launch counter, and
// optional per-launch timing with CUDA events recorded on that same stream.
struct Ctx {
  cudaStream_t stream = nullptr;
  bool timing = false;
  int64_t launches = 0;
  cudaError_t err = cudaSuccess;
  const char *err_where = "";

  struct Family {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0;
    double bytes = 0.0;
  };
  struct Pending {
    int fam;
    cudaEvent_t a, b;
    double bytes;
  };
  std::vector<Family> fams;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> free_events;

  int family(const char *name);
  cudaEvent_t event();
  // Launch through f(); records events around it when timing is on.
  void launch(const char *fam, double bytes, const std::function<void()> &f);
  // Resolve recorded events (call after the stream has been synchronised).
  void collect();
  void release();
};

int sm_count();
size_t smem_optin();
// Sets the thread-local message returned by paradiag_last_error().
void set_last_error(const char *msg);

// ---- time FFT / DST (fft.cu) ----------------------------------------------------
// Forward DFT along time of real (n, ncols) rows -> half spectrum (n/2+1, ncols).
template <typename T, typename Tin>
void launch_fft_r2c(Ctx &c, const Tin *X, int64_t ldx, int64_t ncols, int n, const cpx<T> *tw,
                    cpx<T> *S, int64_t lds);
// Inverse DFT along time of a half spectrum; mode 0: store double, 1: add into
// double, 2: store float.  norm_part (may be null) receives per-CTA sums of the
// squared output values; *nparts = number of CTAs.
template <typename T>
void launch_fft_c2r(Ctx &c, const cpx<T> *S, int64_t lds, int64_t ncols, int n, const cpx<T> *tw,
                    void *out, int64_t ldo, int mode, double *norm_part, int *nparts);
// Orthonormal DST-I along the middle axis of (nt, ny, nx); ny + 1 a power of two.
// mode 0: store, 1: add into (double output only).
template <typename Tin, typename Tout, typename T>
void launch_dst_y(Ctx &c, const Tin *X, Tout *Y, int64_t nt, int64_t ny, int64_t nx,
                  const cpx<T> *tw, int mode);

// ---- shifted tridiagonal solves (pint.cu) ------------------------------------------
struct PintGeom {
  int nf;        // frequencies k = 0..nf-1 (half spectrum)
  int nblk;      // independent tridiagonal blocks per frequency
  int blen;      // rows per block
  int P;         // threads per team (power of two, >= 32)
  int R;         // k-range splits: teams = nblk * R
  int teams_per_cta;
  int M;         // rows per thread (template value)
};
PintGeom pint_geometry(int nf, int nblk, int blen, int target_teams, int elem_bytes);

template <typename T>
struct PintArgs {
  const double2 *shift;    // s_k = 1 - pi_k, length nf
  const T *tlo, *tdiag, *tup;  // tau * K (block-decoupled), length nblk*blen
  const cpx<T> *R;         // spectrum right-hand sides (nf, ldr) or null
  int64_t ldr;
  const T *rvec;           // real vector: the right-hand side when R is null,
                           // subtracted from every R[k] otherwise (may be null)
  cpx<T> *Y;               // solution store (nf, ldy) or null
  int64_t ldy;
  const double2 *omega;    // accumulation weights: acc += Re(omega_k y_k) (summed in T per
                           // team, over that team's few frequencies), or null
  double *acc_part;        // (teams, blen) partial sums when omega != null
  const T *V;              // Krylov basis rows in the compute type (ldv stride) for dots, or null
  int64_t ldv;
  int mdots;               // number of basis vectors dotted with y_k
  double2 *gpart;          // (nf, nblk, mdots) dot products y_k . V[q]
  const int *skip_flag;    // if non-null and *skip_flag != 0 the kernel does nothing
};
template <typename T>
void launch_pint(Ctx &c, const PintGeom &g, const PintArgs<T> &a);
// out[j] = sum_r acc_part[(blk*R + r)*blen + e], j = blk*blen + e
void launch_acc_reduce(Ctx &c, const PintGeom &g, const double *acc_part, double *out,
                       const int *skip_flag);

// ---- Krylov / small systems / residual (krylov.cu) -----------------------------------
struct KrylovBufs {
  int n;              // vector length n_bar
  int maxit;
  const double *klo, *kdiag, *kup;  // K (block-decoupled tridiagonal), unscaled
  double *V;          // (maxit+1, n)
  float *Vf;          // binary32 copy of V for the mixed-precision shifted solves, or null
  double *T;          // (maxit+1, maxit) upper Hessenberg, row-major T[q*maxit + c]
  double *w;          // work vector (n)
  double *part;       // per-CTA partials (grid, maxit+2)
  int grid;           // CTAs of the BLAS-1 kernels
  double *scal;       // scalar block (see krylov.cu)
  int *flags;         // flag block (see krylov.cu)
};
void launch_vec_norm_init(Ctx &c, KrylovBufs &k, const double *b);
void launch_arnoldi(Ctx &c, KrylovBufs &k, int m);
void launch_capacitance(Ctx &c, KrylovBufs &k, int m, int nf, double tau, const double2 *shift,
                        const double2 *wg, const double2 *gpart, int nblk, double *msys_part,
                        int k5_grid, double2 *srow, double2 *omega, double *y);
void launch_project_resnorm(Ctx &c, KrylovBufs &k, int m, const double *z, double tau);
void launch_xm(Ctx &c, KrylovBufs &k, int m, const double *y, double *x, float *xf);
void launch_sumsq(Ctx &c, const double *part, int nparts, double *dst);
// FP64 all-at-once residual R = G - [(I + tau K) U - U Sigma_1^T], stored as Tout
// (float for the mixed path, double for the FP64 path).  1D: K tridiagonal
// (lo, diag, up) of length nx; 2D adds T_y along the middle axis.
template <typename Tout>
void launch_residual(Ctx &c, const double *G, const double *U, Tout *R, int64_t nt, int64_t ny, int64_t nx,
                     double tau, const double *xlo, const double *xdiag, const double *xup, const double *ylo,
                     const double *ydiag, const double *yup, double *norm_part, int *nparts);

}  // namespace pd
