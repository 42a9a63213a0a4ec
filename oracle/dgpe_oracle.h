/*
 * dgpe_oracle.h -- plain FP64 CPU oracle for one split-step Crank-Nicolson
 * time step of the dipolar Gross-Pitaevskii equation (arXiv:1601.04640,
 * "Solution method"; the function list in "Summary of revisions").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this library; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm use it.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * Arrays are row-major with x fastest: psi[z][y][x] (3D) or psi[y][x] (2D),
 * complex values as C99 double complex (interleaved re, im).
 *
 * Equation (dimensionless trap units):
 *   i dpsi/dt = [ -1/2 lap + V + g |psi|^2 + g_dd Phi_d ] psi,
 *   V = s(t) * 1/2 sum_a nu_a^2 x_a^2,  s(t) = 1 + sum_m c_m sin(m t),
 *   Phi_d = IDFT[ U(k) DFT(|psi|^2) ]  (unnormalised forward, 1/N inverse).
 * Grid: x_i = (i - N/2) h, i = 0..N-1; Dirichlet boundaries for the kinetic
 * operator (ghost values psi_{-1} = psi_N = 0); periodic box for the FFT.
 */
#ifndef DGPE_ORACLE_H
#define DGPE_ORACLE_H

#include <complex.h>

#define OR_KERNEL_NONE 0
#define OR_KERNEL_DIPOLAR_3D 1
#define OR_KERNEL_QUASI2D_XY 2
#define OR_KERNEL_QUASI2D_XZ 3  /* 2D grid in the (x, z) plane, dipoles along z in-plane */
#define OR_MAXM 16

typedef struct {
  int dim;          /* 2 (XY or XZ plane, by kernel) or 3 */
  int n[3];         /* nx, ny, nz (nz = 1 in 2D) */
  double h[3];      /* grid spacings */
  double nu[3];     /* trap frequencies: V0 = 1/2 sum nu_a^2 x_a^2 */
  double g, gdd;    /* contact and dipolar strengths */
  double dt;        /* time step */
  int imag;         /* 1 = imaginary time (renormalised each step), 0 = real */
  int kernel;       /* OR_KERNEL_* */
  double qd;        /* quasi-2D width d of the transverse profile (z for XY, y for XZ) */
  int M;            /* number of trap-modulation coefficients c_1..c_M */
  double cm[OR_MAXM];
} or_params;

typedef struct {
  double norm, mu, energy, rms[3], rms_r;
  double kin, pot, contact, dipolar; /* the four energy integrals, per particle */
} or_obs;

/* 1-D transforms (sign = -1 forward, +1 inverse, both unnormalised). */
int or_fft(double complex *x, int n, int sign);
void or_dft(const double complex *x, double complex *X, int n, int sign);
/* In-place transform of a row-major array along every axis. dims[0] slowest. */
int or_fftn(double complex *a, const int *dims, int ndim, int sign);

/* Kernel tables on the full (nz, ny, nx) grid; U(0) = 0. */
void or_kernel_3d(double *U, const int n[3], const double h[3]);
void or_kernel_q2d(double *U, const int n[3], const double h[3], double d);
double or_q2d_value(double krho, double d);
/* erfcx(u) = exp(u^2) erfc(u) for u >= 0, as the quasi-2D kernels use it. */
double or_erfcx(double u);
/* Quasi-2D XZ kernel on the (nz, nx) grid (n[1], h[1] hold the z axis). */
void or_kernel_q2dxz(double *U, const int n[3], const double h[3], double d);
double or_q2dxz_value(double kx, double kz, double d);

/* Phi_d for a real density on the grid of p. */
int or_dipolar_potential(const or_params *p, const double *dens, double *phi);

/* Trap potential V0 (unmodulated) on the grid; s(t) multiplier. */
void or_trap(const or_params *p, double *V0);
double or_trap_scale(const or_params *p, double t);

/* Substeps. */
int or_nonlinear(const or_params *p, double complex *psi, long step);
int or_nonlinear_frac(const or_params *p, double complex *psi, double t, double f);
void or_thomas(const double complex *a, const double complex *b,
               const double complex *c, const double complex *d,
               double complex *x, int n);
void or_cn_axis(const or_params *p, double complex *psi, int axis);
void or_cn_axis_adjoint(const or_params *p, double complex *psi, int axis);
void or_normalize(const or_params *p, double complex *psi);
int or_step(const or_params *p, double complex *psi, long step);
int or_run(const or_params *p, double complex *psi, long step0, long nsteps);
/* second-order (Strang) splitting, real time only (-3 in imaginary time) */
int or_step_strang(const or_params *p, double complex *psi, long step);
int or_run_strang(const or_params *p, double complex *psi, long step0, long nsteps);
int or_observables(const or_params *p, const double complex *psi, long step,
                   or_obs *o);

/* Adjoint of one real-time step and of a run (reverse mode, Wirtinger
 * convention G = 2 dL/dpsi*).  See the implementation for the formulas. */
int or_step_adjoint(const or_params *p, const double complex *psi_in,
                    double complex *G, long step, double *dL_dg,
                    double *dL_dc);

int or_threads(void);
void or_set_threads(int n);

#endif
