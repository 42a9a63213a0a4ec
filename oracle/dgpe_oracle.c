/*
 * dgpe_oracle.c -- plain, slow, FP64 CPU oracle for the split-step
 * Crank-Nicolson step of the dipolar Gross-Pitaevskii equation
 * (arXiv:1601.04640: "Solution method"; the substeps are the functions named
 * in "Summary of revisions": calcpsidd2, calcnu, calclux/calcluy/calcluz,
 * calcnorm, calcmuen, calcrms).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  The product path never links or loads it,
 * and it shares no code with the CUDA path.
 *
 * Everything here follows the definitions directly:
 *   - the DFT is the textbook sum, evaluated by a recursive mixed-radix
 *     Cooley-Tukey split (primes 2, 3, 5) and, for checking, by the O(N^2) sum;
 *   - the dipolar potential is the convolution theorem written out;
 *   - each Crank-Nicolson substep builds the right-hand side B psi and solves
 *     the tridiagonal system A psi+ = B psi with the Thomas algorithm;
 *   - observables are rectangle-rule sums.
 * Lines are independent, so the outer loops run under OpenMP; every sum is
 * evaluated in a fixed order (per-plane partials summed serially), so the
 * result does not depend on the number of threads.
 *
 * Readings of points the paper leaves open (each one is listed with its
 * reason in the design notes):
 *   - substep order: Phi_d from the step-start density, then the exponential,
 *     then CN along x, y, z, then (imaginary time) renormalisation;
 *   - CN coefficients: tau = dt / (4 h^2); kappa = i (real time) or 1
 *     (imaginary time); A = I + kappa tau T, B = I - kappa tau T with
 *     T = tridiag(-1, 2, -1) (the 3-point stencil of -1/2 d^2/dx^2 times
 *     dt/2);
 *   - Dirichlet ghosts psi_{-1} = psi_N = 0;
 *   - k_j = 2 pi j / (N h) for j <= N/2, else 2 pi (j - N) / (N h); U(0) = 0;
 *   - time of step n is t_n = n dt;
 *   - mu and E divided by the norm (per particle).
 */
#include "dgpe_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

int or_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ DFT */

/* O(N^2) textbook sum: X[k] = sum_j x[j] exp(sign 2 pi i j k / N). */
void or_dft(const double complex *x, double complex *X, int n, int sign) {
  for (int k = 0; k < n; ++k) {
    double complex s = 0.0;
    for (int j = 0; j < n; ++j) {
      long t = ((long)j * (long)k) % n;
      double a = sign * 2.0 * M_PI * (double)t / (double)n;
      s += x[j] * (cos(a) + I * sin(a));
    }
    X[k] = s;
  }
}

static int smallest_factor(int n) {
  if (n % 2 == 0) return 2;
  if (n % 3 == 0) return 3;
  if (n % 5 == 0) return 5;
  return n; /* prime other than 2, 3, 5: handled by the direct sum */
}

/* Root table w[t] = exp(sign 2 pi i t / n), t = 0..n-1. */
static double complex *root_table(int n, int sign) {
  double complex *w = (double complex *)malloc(sizeof(double complex) * n);
  for (int t = 0; t < n; ++t) {
    double a = sign * 2.0 * M_PI * (double)t / (double)n;
    w[t] = cos(a) + I * sin(a);
  }
  return w;
}

/*
 * Decimation in time: with p the smallest prime factor of n and m = n / p,
 *   X[k + m q] = sum_{r<p} w_n^{r (k + m q)} Y_r[k],   Y_r = DFT_m(x[r + p j]).
 * w0 is the root table of the top-level length n0; w_n^t = w0[t * (n0/n)].
 */
static void fft_rec(const double complex *x, long xs, double complex *X, int n,
                    const double complex *w0, int n0, double complex *tmp) {
  if (n == 1) {
    X[0] = x[0];
    return;
  }
  int p = smallest_factor(n);
  if (p == n && n > 5) {
    /* direct sum for an unsupported prime (not used by the solver) */
    for (int k = 0; k < n; ++k) {
      double complex s = 0.0;
      for (int j = 0; j < n; ++j)
        s += x[j * xs] * w0[(long)((long)j * k % n) * (n0 / n)];
      X[k] = s;
    }
    return;
  }
  int m = n / p;
  /* sub-transforms of the p decimated sequences, stored in X[r*m .. r*m+m) */
  for (int r = 0; r < p; ++r)
    fft_rec(x + r * xs, xs * p, X + (long)r * m, m, w0, n0, tmp + n);
  for (int k = 0; k < n; ++k) tmp[k] = X[k];
  long step = n0 / n;
  for (int q = 0; q < p; ++q) {
    for (int k = 0; k < m; ++k) {
      long kk = k + (long)m * q;
      double complex s = 0.0;
      for (int r = 0; r < p; ++r) {
        long t = ((long)r * kk) % n;
        s += w0[t * step] * tmp[(long)r * m + k];
      }
      X[kk] = s;
    }
  }
}

int or_fft(double complex *x, int n, int sign) {
  if (n <= 0) return -1;
  double complex *w = root_table(n, sign);
  double complex *X = (double complex *)malloc(sizeof(double complex) * n);
  /* scratch for every recursion level: sum of n / p^k < 2n */
  double complex *tmp = (double complex *)malloc(sizeof(double complex) * 2 * n + 16);
  fft_rec(x, 1, X, n, w, n, tmp);
  memcpy(x, X, sizeof(double complex) * n);
  free(tmp);
  free(X);
  free(w);
  return 0;
}

/* Transform along every axis of a row-major array (dims[0] slowest). */
int or_fftn(double complex *a, const int *dims, int ndim, int sign) {
  long total = 1;
  for (int d = 0; d < ndim; ++d) total *= dims[d];
  for (int ax = 0; ax < ndim; ++ax) {
    int n = dims[ax];
    long stride = 1;
    for (int d = ax + 1; d < ndim; ++d) stride *= dims[d];
    long nlines = total / n;
    double complex *w = root_table(n, sign);
#pragma omp parallel
    {
      double complex *line = (double complex *)malloc(sizeof(double complex) * n);
      double complex *X = (double complex *)malloc(sizeof(double complex) * n);
      double complex *tmp = (double complex *)malloc(sizeof(double complex) * 2 * n + 16);
#pragma omp for schedule(static)
      for (long L = 0; L < nlines; ++L) {
        long outer = L / stride, inner = L % stride;
        long base = outer * stride * n + inner;
        for (int i = 0; i < n; ++i) line[i] = a[base + (long)i * stride];
        fft_rec(line, 1, X, n, w, n, tmp);
        for (int i = 0; i < n; ++i) a[base + (long)i * stride] = X[i];
      }
      free(tmp);
      free(X);
      free(line);
    }
    free(w);
  }
  return 0;
}

/* ---------------------------------------------------------- grid helpers */

static long nsites(const or_params *p) {
  return (long)p->n[0] * p->n[1] * (p->dim == 3 ? p->n[2] : 1);
}

static double coord(const or_params *p, int axis, int i) {
  return ((double)i - (double)(p->n[axis] / 2)) * p->h[axis];
}

static double kval(int j, int n, double h) {
  int jj = (j <= n / 2) ? j : j - n;
  return 2.0 * M_PI * (double)jj / ((double)n * h);
}

static double cell(const or_params *p) {
  double c = p->h[0] * p->h[1];
  if (p->dim == 3) c *= p->h[2];
  return c;
}

/* ------------------------------------------------------- dipolar kernels */

/* U(k) = (4 pi / 3) (3 kz^2 / k^2 - 1), dipoles along z; U(0) = 0. */
void or_kernel_3d(double *U, const int n[3], const double h[3]) {
  for (int z = 0; z < n[2]; ++z)
    for (int y = 0; y < n[1]; ++y)
      for (int x = 0; x < n[0]; ++x) {
        double kx = kval(x, n[0], h[0]), ky = kval(y, n[1], h[1]), kz = kval(z, n[2], h[2]);
        double k2 = kx * kx + ky * ky + kz * kz;
        long idx = ((long)z * n[1] + y) * n[0] + x;
        U[idx] = (k2 == 0.0) ? 0.0 : (4.0 * M_PI / 3.0) * (3.0 * kz * kz / k2 - 1.0);
      }
}

/* Scaled complementary error function erfcx(u) = exp(u^2) erfc(u), u >= 0.
 * Direct form below u = 25; asymptotic series (Abramowitz-Stegun 7.1.23)
 * above, where the direct form underflows. */
static double erfcx_pos(double u) {
  if (u < 25.0) return exp(u * u) * erfc(u);
  double u2 = u * u, term = 1.0, sum = 1.0;
  for (int m = 1; m < 8; ++m) {
    term *= -(2.0 * m - 1.0) / (2.0 * u2);
    sum += term;
  }
  return sum / (u * sqrt(M_PI));
}

double or_erfcx(double u) { return erfcx_pos(u); }

/* Quasi-2D XY kernel: the 3D kernel averaged over the z-profile
 * |phi(z)|^2 = exp(-z^2/d^2) / (sqrt(pi) d):
 *   U2(k) = (4 pi/3) / (sqrt(2 pi) d) * [2 - 3 sqrt(pi/2) q erfcx(q / sqrt 2)],
 * q = k d.  U2(0) = (8 pi / 3) / (sqrt(2 pi) d) is kept (finite). */
double or_q2d_value(double krho, double d) {
  double q = krho * d;
  double pref = (4.0 * M_PI / 3.0) / (sqrt(2.0 * M_PI) * d);
  return pref * (2.0 - 3.0 * sqrt(M_PI / 2.0) * q * erfcx_pos(q / sqrt(2.0)));
}

void or_kernel_q2d(double *U, const int n[3], const double h[3], double d) {
  for (int y = 0; y < n[1]; ++y)
    for (int x = 0; x < n[0]; ++x) {
      double kx = kval(x, n[0], h[0]), ky = kval(y, n[1], h[1]);
      U[(long)y * n[0] + x] = or_q2d_value(sqrt(kx * kx + ky * ky), d);
    }
}

/* Quasi-2D XZ kernel: the grid is the (x, z) plane, the dipoles point along
 * z (in the plane) and the density has the transverse profile
 * |phi(y)|^2 = exp(-y^2/d^2) / (sqrt(pi) d).  Averaging the 3D kernel over y
 * (the profile's pair weight exp(-ky^2 d^2 / 2) in k_y, as for the XY kernel),
 *   U(kx, kz) = int dky/(2 pi) (4 pi/3) (3 kz^2/(kx^2 + ky^2 + kz^2) - 1) exp(-ky^2 d^2/2),
 * and with int dky exp(-a ky^2)/(k^2 + ky^2) = (pi/k) erfcx(sqrt(a) k):
 *   U(kx, kz) = (4 pi/3)/(sqrt(2 pi) d) [3 sqrt(pi/2) (kz^2 d / krho) erfcx(krho d/sqrt 2) - 1],
 * krho^2 = kx^2 + kz^2.  Limits: U -> (4 pi/3)(3 kz^2/krho^2 - 1) for
 * krho d >> 1 (in-plane dipoles), U(kx, 0) = U(0) = -(4 pi/3)/(sqrt(2 pi) d). */
double or_q2dxz_value(double kx, double kz, double d) {
  double pref = (4.0 * M_PI / 3.0) / (sqrt(2.0 * M_PI) * d);
  double krho = sqrt(kx * kx + kz * kz);
  if (krho == 0.0) return -pref;
  double q = krho * d;
  return pref * (3.0 * sqrt(M_PI / 2.0) * (kz * kz * d / krho) * erfcx_pos(q / sqrt(2.0)) - 1.0);
}

void or_kernel_q2dxz(double *U, const int n[3], const double h[3], double d) {
  for (int z = 0; z < n[1]; ++z)
    for (int x = 0; x < n[0]; ++x) {
      double kx = kval(x, n[0], h[0]), kz = kval(z, n[1], h[1]);
      U[(long)z * n[0] + x] = or_q2dxz_value(kx, kz, d);
    }
}

/* Phi = Re IDFT[ U DFT(n) ] / N_total   (convolution theorem). */
int or_dipolar_potential(const or_params *p, const double *dens, double *phi) {
  long N = nsites(p);
  if (p->kernel == OR_KERNEL_NONE) {
    for (long i = 0; i < N; ++i) phi[i] = 0.0;
    return 0;
  }
  double *U = (double *)malloc(sizeof(double) * N);
  if (p->kernel == OR_KERNEL_DIPOLAR_3D) {
    if (p->dim != 3) { free(U); return -1; }
    or_kernel_3d(U, p->n, p->h);
  } else if (p->kernel == OR_KERNEL_QUASI2D_XZ) {
    if (p->dim != 2) { free(U); return -1; }
    or_kernel_q2dxz(U, p->n, p->h, p->qd);
  } else {
    if (p->dim != 2) { free(U); return -1; }
    or_kernel_q2d(U, p->n, p->h, p->qd);
  }
  double complex *a = (double complex *)malloc(sizeof(double complex) * N);
  for (long i = 0; i < N; ++i) a[i] = dens[i];
  int dims[3];
  int nd = p->dim;
  if (nd == 3) { dims[0] = p->n[2]; dims[1] = p->n[1]; dims[2] = p->n[0]; }
  else { dims[0] = p->n[1]; dims[1] = p->n[0]; }
  or_fftn(a, dims, nd, -1);
  for (long i = 0; i < N; ++i) a[i] *= U[i];
  or_fftn(a, dims, nd, +1);
  for (long i = 0; i < N; ++i) phi[i] = creal(a[i]) / (double)N;
  free(a);
  free(U);
  return 0;
}

/* ------------------------------------------------------------ potential */

void or_trap(const or_params *p, double *V0) {
  int nz = (p->dim == 3) ? p->n[2] : 1;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < p->n[1]; ++y)
      for (int x = 0; x < p->n[0]; ++x) {
        double X = coord(p, 0, x), Y = coord(p, 1, y);
        double v = p->nu[0] * p->nu[0] * X * X + p->nu[1] * p->nu[1] * Y * Y;
        if (p->dim == 3) {
          double Z = coord(p, 2, z);
          v += p->nu[2] * p->nu[2] * Z * Z;
        }
        V0[((long)z * p->n[1] + y) * p->n[0] + x] = 0.5 * v;
      }
}

double or_trap_scale(const or_params *p, double t) {
  double s = 1.0;
  for (int m = 1; m <= p->M; ++m) s += p->cm[m - 1] * sin((double)m * t);
  return s;
}

/* ------------------------------------------------------------- substeps */

/* psi <- exp(-kappa f dt (s(t) V0 + g n + g_dd Phi)) psi, n = |psi|^2 at
 * entry: the exponential substep over the fraction f of a time step with the
 * trap evaluated at time t. */
int or_nonlinear_frac(const or_params *p, double complex *psi, double t, double f) {
  long N = nsites(p);
  double *dens = (double *)malloc(sizeof(double) * N);
  double *phi = (double *)malloc(sizeof(double) * N);
  double *V0 = (double *)malloc(sizeof(double) * N);
  for (long i = 0; i < N; ++i) dens[i] = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
  int rc = or_dipolar_potential(p, dens, phi);
  if (rc) { free(dens); free(phi); free(V0); return rc; }
  or_trap(p, V0);
  double s = or_trap_scale(p, t);
  double fdt = f * p->dt;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < N; ++i) {
    double th = fdt * (s * V0[i] + p->g * dens[i] + p->gdd * phi[i]);
    if (p->imag)
      psi[i] *= exp(-th);
    else
      psi[i] *= cos(th) - I * sin(th);
  }
  free(dens);
  free(phi);
  free(V0);
  return 0;
}

/* The exponential substep of step `step` (a full dt at t = step dt). */
int or_nonlinear(const or_params *p, double complex *psi, long step) {
  return or_nonlinear_frac(p, psi, (double)step * p->dt, 1.0);
}

/* Thomas algorithm for a_i x_{i-1} + b_i x_i + c_i x_{i+1} = d_i. */
void or_thomas(const double complex *a, const double complex *b,
               const double complex *c, const double complex *d,
               double complex *x, int n) {
  double complex *cp = (double complex *)malloc(sizeof(double complex) * n);
  double complex *dp = (double complex *)malloc(sizeof(double complex) * n);
  cp[0] = c[0] / b[0];
  dp[0] = d[0] / b[0];
  for (int i = 1; i < n; ++i) {
    double complex den = b[i] - a[i] * cp[i - 1];
    cp[i] = c[i] / den;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
  }
  x[n - 1] = dp[n - 1];
  for (int i = n - 2; i >= 0; --i) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
}

/* One Crank-Nicolson substep along `axis` (0 = x, 1 = y, 2 = z):
 * A psi+ = B psi on every line, A = I + kappa tau T, B = I - kappa tau T. */
static void cn_axis_sign(const or_params *p, double complex *psi, int axis, int adjoint) {
  int n = p->n[axis];
  double tau = p->dt / (4.0 * p->h[axis] * p->h[axis]);
  double complex kt = p->imag ? tau : I * tau;
  /* Adjoint (real time): C^dagger = B^dagger A^{-dagger}.  Conjugating
   * kappa tau turns the right-hand side into A psi and the solved matrix into
   * B, which is exactly B^{-1} A = C^dagger (A and B commute). */
  if (adjoint) kt = conj(kt);
  long sx = 1, sy = p->n[0], sz = (long)p->n[0] * p->n[1];
  long stride = (axis == 0) ? sx : (axis == 1) ? sy : sz;
  int nz = (p->dim == 3) ? p->n[2] : 1;
  int na = (axis == 0) ? p->n[1] : p->n[0];
  int nb = (axis == 2) ? p->n[1] : nz;
  long total = (long)na * nb;
#pragma omp parallel
  {
    double complex *al = (double complex *)malloc(sizeof(double complex) * n);
    double complex *bl = (double complex *)malloc(sizeof(double complex) * n);
    double complex *cl = (double complex *)malloc(sizeof(double complex) * n);
    double complex *d = (double complex *)malloc(sizeof(double complex) * n);
    double complex *x = (double complex *)malloc(sizeof(double complex) * n);
    for (int i = 0; i < n; ++i) {
      al[i] = -kt;
      bl[i] = 1.0 + 2.0 * kt;
      cl[i] = -kt;
    }
#pragma omp for schedule(static)
    for (long L = 0; L < total; ++L) {
      int ia = (int)(L % na), ib = (int)(L / na);
      long base;
      if (axis == 0) base = ib * sz + ia * sy;      /* line over x at (y = ia, z = ib) */
      else if (axis == 1) base = ib * sz + ia * sx; /* line over y at (x = ia, z = ib) */
      else base = ib * sy + ia * sx;                /* line over z at (x = ia, y = ib) */
      for (int i = 0; i < n; ++i) {
        double complex lo = (i > 0) ? psi[base + (i - 1) * stride] : 0.0;
        double complex hi = (i < n - 1) ? psi[base + (i + 1) * stride] : 0.0;
        d[i] = (1.0 - 2.0 * kt) * psi[base + i * stride] + kt * (lo + hi);
      }
      or_thomas(al, bl, cl, d, x, n);
      for (int i = 0; i < n; ++i) psi[base + i * stride] = x[i];
    }
    free(al); free(bl); free(cl); free(d); free(x);
  }
}

void or_cn_axis(const or_params *p, double complex *psi, int axis) {
  cn_axis_sign(p, psi, axis, 0);
}

/* The adjoint C_a^dagger of the Crank-Nicolson substep along `axis`. */
void or_cn_axis_adjoint(const or_params *p, double complex *psi, int axis) {
  cn_axis_sign(p, psi, axis, 1);
}

/* psi <- psi / sqrt(h^d sum |psi|^2) */
void or_normalize(const or_params *p, double complex *psi) {
  long N = nsites(p);
  int rows = (p->dim == 3) ? p->n[2] : 1;
  long per = N / rows;
  double *part = (double *)malloc(sizeof(double) * rows);
#pragma omp parallel for schedule(static)
  for (int r = 0; r < rows; ++r) {
    double s = 0.0;
    for (long i = 0; i < per; ++i) {
      double complex v = psi[(long)r * per + i];
      s += creal(v) * creal(v) + cimag(v) * cimag(v);
    }
    part[r] = s;
  }
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += part[r];
  free(part);
  double f = 1.0 / sqrt(cell(p) * s);
  for (long i = 0; i < N; ++i) psi[i] *= f;
}

int or_step(const or_params *p, double complex *psi, long step) {
  int rc = or_nonlinear(p, psi, step);
  if (rc) return rc;
  or_cn_axis(p, psi, 0);
  or_cn_axis(p, psi, 1);
  if (p->dim == 3) or_cn_axis(p, psi, 2);
  if (p->imag) or_normalize(p, psi);
  return 0;
}

/* Second-order (Strang) splitting of step `step`, real time:
 *   psi <- E(dt/2, t_{k+1}) C_z C_y C_x E(dt/2, t_k) psi,  t_k = step dt,
 * where E(f dt, t) is the exponential substep with the density of its own
 * input, so the closing half uses the density after the Crank-Nicolson
 * substeps.  (The paper uses first-order splitting; this symmetric variant is
 * second order in dt.)  Returns -3 in imaginary time. */
int or_step_strang(const or_params *p, double complex *psi, long step) {
  if (p->imag) return -3;
  int rc = or_nonlinear_frac(p, psi, (double)step * p->dt, 0.5);
  if (rc) return rc;
  or_cn_axis(p, psi, 0);
  or_cn_axis(p, psi, 1);
  if (p->dim == 3) or_cn_axis(p, psi, 2);
  return or_nonlinear_frac(p, psi, (double)(step + 1) * p->dt, 0.5);
}

int or_run_strang(const or_params *p, double complex *psi, long step0, long nsteps) {
  for (long s = 0; s < nsteps; ++s) {
    int rc = or_step_strang(p, psi, step0 + s);
    if (rc) return rc;
  }
  return 0;
}

int or_run(const or_params *p, double complex *psi, long step0, long nsteps) {
  for (long s = 0; s < nsteps; ++s) {
    int rc = or_step(p, psi, step0 + s);
    if (rc) return rc;
  }
  return 0;
}

/* ---------------------------------------------------------- observables */

/* Per-particle observables of the current psi (time t = step * dt).
 * Kinetic term: 1/2 sum_a sum_{i=-1}^{N-1} |psi_{i+1} - psi_i|^2 / h_a^2 with
 * ghost zeros, which equals <psi, H_a psi> for the 3-point stencil. */
int or_observables(const or_params *p, const double complex *psi, long step, or_obs *o) {
  long N = nsites(p);
  int nx = p->n[0], ny = p->n[1], nz = (p->dim == 3) ? p->n[2] : 1;
  double *dens = (double *)malloc(sizeof(double) * N);
  double *phi = (double *)malloc(sizeof(double) * N);
  double *V0 = (double *)malloc(sizeof(double) * N);
  for (long i = 0; i < N; ++i) dens[i] = creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
  int rc = or_dipolar_potential(p, dens, phi);
  if (rc) { free(dens); free(phi); free(V0); return rc; }
  or_trap(p, V0);
  double s = or_trap_scale(p, (double)step * p->dt);
  enum { S_N, S_X2, S_Y2, S_Z2, S_V, S_N2, S_PHI, S_KX, S_KY, S_KZ, S_COUNT };
  double *part = (double *)calloc((size_t)nz * S_COUNT, sizeof(double));
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z) {
    double acc[S_COUNT] = {0};
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        long i = ((long)z * ny + y) * nx + x;
        double n = dens[i];
        double X = coord(p, 0, x), Y = coord(p, 1, y), Z = (p->dim == 3) ? coord(p, 2, z) : 0.0;
        acc[S_N] += n;
        acc[S_X2] += X * X * n;
        acc[S_Y2] += Y * Y * n;
        acc[S_Z2] += Z * Z * n;
        acc[S_V] += s * V0[i] * n;
        acc[S_N2] += n * n;
        acc[S_PHI] += phi[i] * n;
        /* forward differences psi_{i+1} - psi_i, including the pair
         * (ghost at -1, first point) */
        double complex cur = psi[i];
        double complex nxp = (x + 1 < nx) ? psi[i + 1] : 0.0;
        double complex nyp = (y + 1 < ny) ? psi[i + nx] : 0.0;
        acc[S_KX] += cabs(nxp - cur) * cabs(nxp - cur);
        acc[S_KY] += cabs(nyp - cur) * cabs(nyp - cur);
        if (x == 0) acc[S_KX] += cabs(cur) * cabs(cur);
        if (y == 0) acc[S_KY] += cabs(cur) * cabs(cur);
        if (p->dim == 3) {
          double complex nzp = (z + 1 < nz) ? psi[i + (long)nx * ny] : 0.0;
          acc[S_KZ] += cabs(nzp - cur) * cabs(nzp - cur);
          if (z == 0) acc[S_KZ] += cabs(cur) * cabs(cur);
        }
      }
    for (int k = 0; k < S_COUNT; ++k) part[(long)z * S_COUNT + k] = acc[k];
  }
  double tot[S_COUNT] = {0};
  for (int z = 0; z < nz; ++z)
    for (int k = 0; k < S_COUNT; ++k) tot[k] += part[(long)z * S_COUNT + k];
  free(part);
  free(dens);
  free(phi);
  free(V0);
  double w = cell(p);
  double norm = w * tot[S_N];
  double kin = 0.5 * w * (tot[S_KX] / (p->h[0] * p->h[0]) + tot[S_KY] / (p->h[1] * p->h[1]));
  if (p->dim == 3) kin += 0.5 * w * tot[S_KZ] / (p->h[2] * p->h[2]);
  double pot = w * tot[S_V];
  double con = w * tot[S_N2];
  double dip = w * tot[S_PHI];
  o->norm = norm;
  o->kin = kin / norm;
  o->pot = pot / norm;
  o->contact = p->g * con / norm;
  o->dipolar = p->gdd * dip / norm;
  o->mu = (kin + pot + p->g * con + p->gdd * dip) / norm;
  o->energy = (kin + pot + 0.5 * p->g * con + 0.5 * p->gdd * dip) / norm;
  o->rms[0] = sqrt(tot[S_X2] / tot[S_N]);
  o->rms[1] = sqrt(tot[S_Y2] / tot[S_N]);
  o->rms[2] = sqrt(tot[S_Z2] / tot[S_N]);
  o->rms_r = sqrt((tot[S_X2] + tot[S_Y2] + tot[S_Z2]) / tot[S_N]);
  return 0;
}

/* ------------------------------------------------------------- adjoint */

/*
 * Reverse mode through one real-time step psi' = C e^{-i theta} psi,
 * theta = dt (s_n V0 + g n + g_dd K*n), n = |psi|^2, C = C_z C_y C_x.
 * Convention: G = 2 dL/dpsi* (so dL = Re sum conj(G) dpsi).
 * On entry G holds G' for psi'; on exit it holds G for psi.
 *   G_phi = C^dagger G' = C_x^dagger C_y^dagger C_z^dagger G',
 *     C_a^dagger = B_a^dagger A_a^{-dagger}: right-hand side A_a G (because
 *     B_a^dagger = A_a in real time), then solve with B_a (= A_a^dagger);
 *   sig = Im(conj(G_phi) phi),   phi = e^{-i theta} psi;
 *   G = e^{+i theta} G_phi + 2 dt (g sig + g_dd K*sig) psi;
 *   dL/dg   += dt sum sig n;
 *   dL/dc_m += dt sin(m t_n) sum sig V0.
 */
int or_step_adjoint(const or_params *p, const double complex *psi_in,
                    double complex *G, long step, double *dL_dg, double *dL_dc) {
  if (p->imag) return -1;
  long N = nsites(p);
  double *dens = (double *)malloc(sizeof(double) * N);
  double *phi = (double *)malloc(sizeof(double) * N);
  double *V0 = (double *)malloc(sizeof(double) * N);
  double *th = (double *)malloc(sizeof(double) * N);
  double *sig = (double *)malloc(sizeof(double) * N);
  double *ksig = (double *)malloc(sizeof(double) * N);
  for (long i = 0; i < N; ++i)
    dens[i] = creal(psi_in[i]) * creal(psi_in[i]) + cimag(psi_in[i]) * cimag(psi_in[i]);
  int rc = or_dipolar_potential(p, dens, phi);
  if (rc) goto done;
  or_trap(p, V0);
  double t = (double)step * p->dt;
  double s = or_trap_scale(p, t);
  for (long i = 0; i < N; ++i) th[i] = p->dt * (s * V0[i] + p->g * dens[i] + p->gdd * phi[i]);
  /* G_phi = C^dagger G' : z, then y, then x (reverse of the forward order) */
  if (p->dim == 3) cn_axis_sign(p, G, 2, 1);
  cn_axis_sign(p, G, 1, 1);
  cn_axis_sign(p, G, 0, 1);
  for (long i = 0; i < N; ++i) {
    double complex ph = psi_in[i] * (cos(th[i]) - I * sin(th[i]));
    sig[i] = cimag(conj(G[i]) * ph);
  }
  rc = or_dipolar_potential(p, sig, ksig);
  if (rc) goto done;
  {
    double sg = 0.0, sv = 0.0;
    for (long i = 0; i < N; ++i) {
      sg += sig[i] * dens[i];
      sv += sig[i] * V0[i];
    }
    if (dL_dg) *dL_dg += p->dt * sg;
    if (dL_dc)
      for (int m = 1; m <= p->M; ++m) dL_dc[m - 1] += p->dt * sin((double)m * t) * sv;
  }
  for (long i = 0; i < N; ++i) {
    double complex e = cos(th[i]) + I * sin(th[i]);
    G[i] = e * G[i] + 2.0 * p->dt * (p->g * sig[i] + p->gdd * ksig[i]) * psi_in[i];
  }
done:
  free(dens); free(phi); free(V0); free(th); free(sig); free(ksig);
  return rc;
}
