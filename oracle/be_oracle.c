/*
 * FP64 CPU oracle for the all-at-once backward-Euler system (eq. 2):
 *
 *     (M + tau K) U - M U Sigma_1^T = G,   U = [u_1, ..., u_l],
 *
 * written out as its plain definition: sequential time stepping
 *     (M + tau K) u_j = M u_{j-1} + G_j,  j = 1..l,  u_0 := 0
 * (column j of U Sigma_1^T is u_{j-1}; G_1 already holds u_0 + tau f_1).
 * M = I in the paper; a diagonal M is accepted here (NULL means I).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or table with the CUDA path.
 *
 * Layout: G and U are row-major (l, n) float64, row j = time step j+1.
 * All routines use plain Gaussian elimination without pivoting; every
 * operator used with them makes M + tau K (and the shifted complex matrices)
 * diagonally dominant or positive real, where elimination without pivoting
 * cannot break down.  Return value: 0 on success, 1 on a zero pivot,
 * 2 on a bad argument.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Sequential backward Euler, tridiagonal K (1D).  Thomas algorithm: the LU
 * factors of M + tau K are formed once and reused for all l steps. */
int or_be_tridiag(int64_t n, int64_t nt, double tau, const double *lo, const double *diag,
                  const double *up, const double *mdiag, const double *G, double *U) {
  if (n < 1 || nt < 1 || tau <= 0.0) return 2;
  double *piv = (double *)malloc(sizeof(double) * n);   /* U-factor diagonal */
  double *mul = (double *)malloc(sizeof(double) * n);   /* L-factor multipliers */
  double *y = (double *)malloc(sizeof(double) * n);
  if (!piv || !mul || !y) { free(piv); free(mul); free(y); return 2; }
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    double m = mdiag ? mdiag[i] : 1.0;
    double b = m + tau * diag[i];
    if (i > 0) {
      mul[i] = tau * lo[i] / piv[i - 1];
      b -= mul[i] * tau * up[i - 1];
    } else {
      mul[i] = 0.0;
    }
    if (b == 0.0) { rc = 1; goto done; }
    piv[i] = b;
  }
  for (int64_t j = 0; j < nt; ++j) {
    const double *g = G + j * n;
    const double *uprev = (j > 0) ? U + (j - 1) * n : NULL;
    double *u = U + j * n;
    /* right-hand side M u_{j-1} + G_j, then forward elimination */
    for (int64_t i = 0; i < n; ++i) {
      double r = g[i];
      if (uprev) r += (mdiag ? mdiag[i] : 1.0) * uprev[i];
      y[i] = (i > 0) ? r - mul[i] * y[i - 1] : r;
    }
    /* back substitution */
    u[n - 1] = y[n - 1] / piv[n - 1];
    for (int64_t i = n - 2; i >= 0; --i) u[i] = (y[i] - tau * up[i] * u[i + 1]) / piv[i];
  }
done:
  free(piv); free(mul); free(y);
  return rc;
}

/* Sequential backward Euler, banded K (used for the 2D 5-point operator).
 * Kband is row-major (n, kl+ku+1): Kband[i*(kl+ku+1) + (j - i + kl)] = K[i][j]
 * for max(0, i-kl) <= j <= min(n-1, i+ku).  M + tau K is factored once by banded
 * LU without pivoting (fill stays inside the band), then each step is one
 * banded forward and back substitution. */
int or_be_banded(int64_t n, int64_t kl, int64_t ku, double tau, const double *Kband,
                 const double *mdiag, int64_t nt, const double *G, double *U) {
  if (n < 1 || nt < 1 || kl < 0 || ku < 0 || tau <= 0.0) return 2;
  const int64_t w = kl + ku + 1;
  double *A = (double *)malloc(sizeof(double) * n * w);
  double *y = (double *)malloc(sizeof(double) * n);
  if (!A || !y) { free(A); free(y); return 2; }
  int rc = 0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t c = 0; c < w; ++c) A[i * w + c] = tau * Kband[i * w + c];
  for (int64_t i = 0; i < n; ++i) A[i * w + kl] += mdiag ? mdiag[i] : 1.0;
  /* A[i][j] lives at A[i*w + (j - i + kl)] */
  for (int64_t k = 0; k < n; ++k) {
    double p = A[k * w + kl];
    if (p == 0.0) { rc = 1; goto done; }
    int64_t imax = (k + kl < n - 1) ? k + kl : n - 1;
    int64_t jmax = (k + ku < n - 1) ? k + ku : n - 1;
    for (int64_t i = k + 1; i <= imax; ++i) {
      double l = A[i * w + (k - i + kl)] / p;
      A[i * w + (k - i + kl)] = l; /* store the multiplier in place of the eliminated entry */
      if (l == 0.0) continue;
      for (int64_t j = k + 1; j <= jmax; ++j) A[i * w + (j - i + kl)] -= l * A[k * w + (j - k + kl)];
    }
  }
  for (int64_t s = 0; s < nt; ++s) {
    const double *g = G + s * n;
    const double *uprev = (s > 0) ? U + (s - 1) * n : NULL;
    double *u = U + s * n;
    for (int64_t i = 0; i < n; ++i) {
      double r = g[i];
      if (uprev) r += (mdiag ? mdiag[i] : 1.0) * uprev[i];
      int64_t j0 = (i - kl > 0) ? i - kl : 0;
      for (int64_t j = j0; j < i; ++j) r -= A[i * w + (j - i + kl)] * y[j];
      y[i] = r;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double r = y[i];
      int64_t j1 = (i + ku < n - 1) ? i + ku : n - 1;
      for (int64_t j = i + 1; j <= j1; ++j) r -= A[i * w + (j - i + kl)] * u[j];
      u[i] = r / A[i * w + kl];
    }
  }
done:
  free(A); free(y);
  return rc;
}

/* One complex tridiagonal solve  (s I + tau K) x = r  for a complex shift s,
 * K tridiagonal real (lo, diag, up).  This is the shifted system
 * ((1 - pi_i) I + tau K) of Sec. 2 with s = 1 - pi_i.  Interleaved complex
 * arrays (re, im).  Thomas algorithm without pivoting. */
int or_shifted_tridiag_solve(int64_t n, double s_re, double s_im, double tau, const double *lo,
                             const double *diag, const double *up, const double *r, double *x) {
  if (n < 1) return 2;
  double complex s = s_re + I * s_im;
  double complex *cp = (double complex *)malloc(sizeof(double complex) * n);
  double complex *dp = (double complex *)malloc(sizeof(double complex) * n);
  if (!cp || !dp) { free(cp); free(dp); return 2; }
  int rc = 0;
  for (int64_t i = 0; i < n; ++i) {
    double complex b = s + tau * diag[i];
    double complex rhs = r[2 * i] + I * r[2 * i + 1];
    if (i > 0) {
      double a = tau * lo[i];
      b -= a * cp[i - 1];
      rhs -= a * dp[i - 1];
    }
    if (b == 0.0) { rc = 1; goto done; }
    cp[i] = (i < n - 1) ? tau * up[i] / b : 0.0;
    dp[i] = rhs / b;
  }
  {
    double complex xi = dp[n - 1];
    x[2 * (n - 1)] = creal(xi);
    x[2 * (n - 1) + 1] = cimag(xi);
    for (int64_t i = n - 2; i >= 0; --i) {
      xi = dp[i] - cp[i] * xi;
      x[2 * i] = creal(xi);
      x[2 * i + 1] = cimag(xi);
    }
  }
done:
  free(cp); free(dp);
  return rc;
}
