/*
 * dgpe.h -- C ABI of the GB300-native split-step Crank-Nicolson solver for the
 * dipolar Gross-Pitaevskii equation (arXiv:1601.04640: "Nature of problem",
 * "Solution method").
 *
 * Equation solved (dimensionless trap units, "Nature of problem"):
 *   i dpsi/dt = [ -1/2 lap + V + g |psi|^2 + g_dd Phi_d ] psi
 *   V = s(t) * 1/2 (nu_x^2 x^2 + nu_y^2 y^2 [+ nu_z^2 z^2]),
 *   s(t) = 1 + sum_{m=1..M} c_m sin(m t)        (s = 1 unless set),
 *   Phi_d = IDFT[ U(k) DFT(|psi|^2) ] / N,  U(k) = (4 pi/3)(3 kz^2/k^2 - 1),
 *   U(0) = 0 (3D); quasi-2D XY: U(k) averaged over a Gaussian z-profile of
 *   width d ("Solution method": Fourier transform + convolution theorem).
 * One time step ("Solution method", the functions of "Summary of revisions"):
 *   1. Phi_d from the step-start density (calcpsidd2);
 *   2. psi <- exp(-kappa dt (V + g|psi|^2 + g_dd Phi_d)) psi, kappa = i in real
 *      time, 1 in imaginary time (calcnu);
 *   3. Crank-Nicolson along x, y (, z): (I + kappa tau T) psi+ =
 *      (I - kappa tau T) psi on every grid line, tau = dt/(4 h^2),
 *      T = tridiag(-1, 2, -1), Dirichlet ghosts psi_{-1} = psi_N = 0
 *      (calclux, calcluy, calcluz);
 *   4. imaginary time only: psi <- psi / sqrt(h^d sum |psi|^2) (calcnorm).
 * Grid: x_i = (i - N/2) h; psi is row-major with x fastest: [z][y][x] (3D),
 * [y][x] (2D XY).  Interleaved complex (re, im).
 *
 * Conventions of every call:
 *   - return DGPE_OK (0) or a negative DGPE_E* code; nothing aborts or traps;
 *     dgpe_last_error() gives the text of the last failure of a handle;
 *   - the library owns every device buffer it allocates; the caller owns the
 *     CUDA stream passed to dgpe_create (NULL = the legacy default stream) and
 *     every host or device buffer it passes in;
 *   - work is enqueued on the handle's stream; calls that return data to the
 *     host (get_psi, observables, sync) synchronise that stream, and errors of
 *     earlier asynchronous work surface there as DGPE_ECUDA.
 */
#ifndef DGPE_H
#define DGPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DGPE_OK 0
#define DGPE_EINVAL (-1)        /* bad argument or parameter */
#define DGPE_EUNSUPPORTED (-2)  /* valid but not supported: a grid length
                                   outside the supported set, or a flag that
                                   the mode or form does not take */
#define DGPE_ENOMEM (-3)        /* device allocation failed */
#define DGPE_ECUDA (-4)         /* a CUDA call failed */
#define DGPE_ENONFINITE (-5)    /* NaN or Inf found in the state */
#define DGPE_ETIMEOUT (-6)      /* a bounded device-side wait ran out: a kernel
                                   gave up waiting for its own asynchronous
                                   copies (or, in the batched form, for another
                                   block's pass) and returned; the state is then
                                   incomplete.  Reported by dgpe_observables
                                   and dgpe_sync (dgpe_batch_step for the
                                   batched form) */

/* dgpe_params.mode */
#define DGPE_IMAG 0             /* imaginary time: stationary states */
#define DGPE_REAL 1             /* real time: dynamics */
/* dgpe_params.precision */
#define DGPE_FP64 0             /* every substep in FP64 */
#define DGPE_FP32_BULK 1        /* FFT, exponential and Thomas arithmetic and
                                   the state in FP32; norm/mu/energy reductions
                                   (the step's norm above 16-site FP32 partial
                                   sums), renormalisation and all tables built
                                   in FP64 */
/* dgpe_params.kernel */
#define DGPE_KERNEL_NONE 0
#define DGPE_KERNEL_DIPOLAR_3D 1
#define DGPE_KERNEL_QUASI2D_XY 2  /* 2D XY plane, dipoles along z (normal to the plane) */
#define DGPE_KERNEL_QUASI2D_XZ 3  /* 2D XZ plane, dipoles along z (in the plane):
                                     U(kx, kz) = (4pi/3)/(sqrt(2pi) d) [3 sqrt(pi/2)
                                     (kz^2 d/krho) erfcx(krho d/sqrt2) - 1], the 3D
                                     kernel averaged over the y-profile
                                     exp(-y^2/d^2)/(sqrt(pi) d) */
/* dgpe_params.plane (2D only).  For XZ the second axis is z: n[1], h[1] and
   nu[1] describe z, and psi is stored [z][x]. */
#define DGPE_PLANE_XY 0
#define DGPE_PLANE_XZ 1
/* dgpe_params.flags */
#define DGPE_FLAG_NO_GRAPH 1u   /* launch the passes directly instead of
                                   replaying a captured CUDA graph */
#define DGPE_FLAG_CN_SERIAL 2u  /* FP64 form: solve every CN line serially,
                                   one thread per line (the default once the
                                   grid has >= 8192 lines per axis); the FP32
                                   form returns DGPE_EUNSUPPORTED */
#define DGPE_FLAG_CN_CHUNKED 4u /* FP64 form: always use the chunk-parallel
                                   CN solve (exclusive with CN_SERIAL) */
#define DGPE_FLAG_STRANG 8u     /* real time: second-order (Strang) splitting,
                                   one step = E(dt/2, t_{k+1}) C_z C_y C_x
                                   E(dt/2, t_k), the closing half with the
                                   density after the CN substeps (the paper's
                                   step is first order: E(dt, t_k) then CN).
                                   dgpe_step(h, n) runs it as n first-order
                                   steps between an exponential substep over
                                   -dt/2 and one over +dt/2 (|psi| is unchanged
                                   by the exponential in real time).  Imaginary
                                   time, the reverse step and the batched form
                                   return DGPE_EUNSUPPORTED. */
#define DGPE_FLAG_REAL_PSI 16u  /* imaginary time: hold psi as a real field
                                   (nx reals per row; half the bytes of the
                                   complex state).  Imaginary-time evolution
                                   with a real potential keeps a real state
                                   real, so the step is the complex step on
                                   the real part.  dgpe_set_psi keeps the real
                                   part of its input; dgpe_get_psi returns
                                   (psi, 0).  Uses the chunk-parallel CN solve
                                   (CN_SERIAL returns DGPE_EUNSUPPORTED), as do
                                   real time (at create and in dgpe_set_mode)
                                   and the batched form. */

#define DGPE_FLAG_P1_ONESHOT 32u /* FP32 bulk: run the two x-line passes
                                   (density + R2C; C2R, exponential, CN_x) as
                                   one CTA per tile instead of the default
                                   persistent CTAs fed by bulk asynchronous
                                   copies, and the strided transforms as
                                   register-fed tiles instead of persistent
                                   CTAs fed by tensor-map copies (same
                                   arithmetic, except that the 3D z-pass
                                   then reads U(k) from its FP32 table
                                   instead of evaluating it in FP32) */

#define DGPE_FLAG_BATCH_CLASSES 64u /* batched form (set on any problem): step
                                   the batch as per-size-class batched kernels
                                   (4 per class) in one captured graph whose
                                   class branches run concurrently, instead of
                                   the persistent work-list kernel (same
                                   arithmetic; no bounded waits) */

typedef struct dgpe_params {
  int dim;          /* 2 or 3 */
  int plane;        /* DGPE_PLANE_* (2D) */
  int n[3];         /* nx, ny, nz (nz ignored in 2D); each 2^k, 3 2^k or
                       5 2^k between 32 and 512 (e.g. 64, 96, 160, 384);
                       any other length (240 = 16 15 included) returns
                       DGPE_EUNSUPPORTED */
  double h[3];      /* spacings hx, hy, hz > 0 */
  double nu[3];     /* trap frequencies nu_x, nu_y, nu_z >= 0 */
  double g;         /* contact strength */
  double gdd;       /* dipolar strength */
  double dt;        /* time step > 0 */
  int mode;         /* DGPE_IMAG or DGPE_REAL */
  int precision;    /* DGPE_FP64 or DGPE_FP32_BULK */
  int kernel;       /* DGPE_KERNEL_* (DIPOLAR_3D needs dim 3, QUASI2D_XY dim 2
                       and the XY plane, QUASI2D_XZ dim 2 and the XZ plane) */
  double qd;        /* quasi-2D width d > 0 of the transverse profile (z for
                       QUASI2D_XY, y for QUASI2D_XZ) */
  unsigned flags;   /* DGPE_FLAG_* */
} dgpe_params;

typedef struct dgpe_obs {
  double norm;      /* h^d sum |psi|^2 */
  double mu;        /* chemical potential, per particle (divided by norm) */
  double energy;    /* energy per particle (divided by norm) */
  double rms[3];    /* sqrt(<x^2>), sqrt(<y^2>), sqrt(<z^2>) (0 for z in 2D) */
  double rms_r;     /* sqrt(<r^2>) */
  double t;         /* time of the state: steps taken * dt */
  double kin;       /* kinetic energy per particle: 1/2 sum_a sum |psi_{i+1} -
                       psi_i|^2 / h_a^2 over forward differences, ghosts 0 */
  double pot;       /* trap energy per particle */
  double contact;   /* g sum |psi|^4 h^d / norm */
  double dipolar;   /* g_dd sum Phi_d |psi|^2 h^d / norm */
} dgpe_obs;

typedef struct dgpe_solver *dgpe_t;

/* Create a solver for one condensate.  Validates p, allocates psi (zero), the
 * half spectrum and the tables, builds U(k)/N, the Thomas tables and the FFT
 * roots in FP64, and captures one step into a CUDA graph.  cuda_stream is a
 * cudaStream_t (or NULL).  On failure *out is NULL. */
int dgpe_create(const dgpe_params *p, void *cuda_stream, dgpe_t *out);

/* Release every resource of h; NULL is a no-op. */
void dgpe_destroy(dgpe_t h);

/* Copy the state in/out as host FP64 interleaved complex, n_sites =
 * nx*ny(*nz) complex values.  set_psi starts the time at t = 0 unless
 * dgpe_set_time is called after it.  get_psi synchronises. */
int dgpe_set_psi(dgpe_t h, const double *psi, size_t n_sites);
int dgpe_get_psi(dgpe_t h, double *psi, size_t n_sites);

/* Device-pointer variants: psi is a device buffer of n_sites complex values,
 * complex128 when fp64 != 0, else complex64.  Asynchronous on the stream. */
int dgpe_set_psi_device(dgpe_t h, const void *psi, size_t n_sites, int fp64);
int dgpe_get_psi_device(dgpe_t h, void *psi, size_t n_sites, int fp64);

/* Advance n >= 0 steps (graph replays; with DGPE_FLAG_STRANG, an exponential
 * pass over -dt/2 before them and one over +dt/2 after them).  Asynchronous. */
int dgpe_step(dgpe_t h, int n);

/* norm, mu, energy, rms sizes of the current state in FP64 (calcmuen,
 * calcrms, calcnorm).  Synchronises.  DGPE_ENONFINITE if the state holds a
 * NaN or an Inf. */
int dgpe_observables(dgpe_t h, dgpe_obs *o);

/* Phi_d of the current density, written to a host FP64 array of n_sites
 * reals (calcpsidd2).  Synchronises. */
int dgpe_dipolar_potential(dgpe_t h, double *phi, size_t n_sites);

/* Change the contact strength (a quench), the mode (imaginary <-> real) or the
 * trap modulation V(t) = V0 (1 + sum_{m=1..M} c_m sin(m t)), M <= 16. */
int dgpe_set_g(dgpe_t h, double g);
int dgpe_set_mode(dgpe_t h, int mode);
int dgpe_set_trap_modulation(dgpe_t h, const double *c, int M);

/* Step counter n of the next step (its time is t_n = n dt). */
int dgpe_set_time(dgpe_t h, long long step);
int dgpe_get_time(dgpe_t h, long long *step);

/* Wait for all work of h; report asynchronous errors. */
int dgpe_sync(dgpe_t h);

/* Number of kernel launches one dgpe_step(1) makes. */
int dgpe_launches_per_step(dgpe_t h);

/* Profiling: run n steps with the passes launched one by one on the stream
 * and a CUDA event recorded between consecutive passes; pass_ms[i] receives
 * the mean duration (ms) of pass i over the n steps.  Returns the number of
 * passes of one step (<= cap) or a negative status.  Synchronises. */
int dgpe_profile_steps(dgpe_t h, int n, double *pass_ms, int cap);

/* Kernel name of pass i of one step, and its algorithmic HBM traffic per
 * launch in bytes (each array element the pass must read or write, once). */
const char *dgpe_pass_name(dgpe_t h, int i);
double dgpe_pass_bytes(dgpe_t h, int i);

/* Floating-point operations of pass i per launch, an FMA counting 2: the
 * operation count of the pass's algorithm (FFT codelets and twiddles, pair
 * packing of the real transforms, the exponential substep with sin and
 * cos - 1 by Taylor series (expm1 counted as one operation), the Thomas
 * recurrences).  0 for an index out of range or a NULL handle. */
double dgpe_pass_flops(dgpe_t h, int i);

/* Kernels this handle has launched since it was created (each replay of the
 * step graph counts the step's kernels; observables, copies in and out and
 * the adjoint calls count theirs).  0 for a NULL handle. */
long long dgpe_kernel_launches(dgpe_t h);

/* Reverse mode of one real-time step (the adjoint form: Wirtinger
 * convention G = 2 dL/dpsi*).  psi_in: device state at the start of step
 * `step` (complex128 for DGPE_FP64, complex64 for DGPE_FP32_BULK); G: device
 * buffer of the same type holding G' = 2 dL/dpsi'* for the state after the
 * step, overwritten with G for psi_in.  Applies C^dagger (Thomas with
 * conjugated coefficients along z, y, x), the adjoint of the exponential and
 * one extra dipolar convolution:
 *   sig = Im(conj(G_phi) e^{-i theta} psi_in),
 *   G = e^{i theta} G_phi + 2 dt (g sig + g_dd Phi_d[sig]) psi_in,
 * and adds dt sum sig |psi_in|^2 to *dL_dg and dt sin(m t) sum sig V0 to
 * dL_dc[m-1] for the current trap modulation (FP64 reductions).  Synchronises.
 * DGPE_EUNSUPPORTED in imaginary-time mode.  (Differentiation of the step;
 * the paper computes no gradients.) */
int dgpe_step_adjoint(dgpe_t h, const void *psi_in, void *G, long long step,
                      double *dL_dg, double *dL_dc);

/* Fidelity F = |<target|psi(T)>|^2 (inner product h^d sum conj(a) b) after
 * nsteps real-time steps from psi0 (host FP64 interleaved complex, both), and
 * its gradient with respect to g and the trap-modulation coefficients c_1..c_M
 * of dgpe_set_trap_modulation, by a reverse sweep over checkpoints taken every
 * `every` steps (the states of one segment are recomputed while it is
 * reversed).  Leaves psi at the last recomputed state.  Synchronises. */
int dgpe_fidelity_gradient(dgpe_t h, const double *psi0, const double *target, int nsteps,
                           int every, double *F, double *dF_dg, double *dF_dc);

/* ---- Batched form: many independent 2D XY condensates stepped together ----
 * (the paper's imag2dXY / real2dXY programs, one problem each; here a
 * parameter sweep).  ps[0..count-1]: dim 2, plane XY, square grids
 * (nx == ny, any supported length), precision DGPE_FP32_BULK, kernel
 * QUASI2D_XY, imaginary or real time each.  dgpe_batch_step(b, n) is one
 * launch of a persistent kernel that advances every problem n steps: its
 * CTAs take (problem, pass, tile) items from a device work list in ticket
 * order, each item waiting until its problem's earlier passes are complete
 * (per-problem counters; every wait is bounded and a wait that runs out makes
 * the next dgpe_batch_sync / get_psi / observables return DGPE_ETIMEOUT);
 * 64 x 64 problems stay in one CTA's shared memory for all n steps.  At create
 * time an autotuner times the orders of the FFT radices for each size and
 * mode.  States start at zero; problem i is addressed by its index. */
typedef struct dgpe_batch *dgpe_batch_t;
int dgpe_batch_create(const dgpe_params *ps, int count, void *cuda_stream, dgpe_batch_t *out);
void dgpe_batch_destroy(dgpe_batch_t b);
int dgpe_batch_set_psi(dgpe_batch_t b, int i, const double *psi, size_t n_sites);
int dgpe_batch_get_psi(dgpe_batch_t b, int i, double *psi, size_t n_sites);   /* synchronises */
int dgpe_batch_step(dgpe_batch_t b, int n);                                    /* one launch, n steps; asynchronous */
/* Wait for the batch's work; DGPE_ETIMEOUT if a bounded wait ran out. */
int dgpe_batch_sync(dgpe_batch_t b);
/* Test hooks of the bounded waits: hold problem i (-1: none) so that its
 * tiles never count as complete -- every wait on it runs out and the step
 * returns early with DGPE_ETIMEOUT at the next sync; and the number of polls
 * (about 64 ns apart) after which a wait gives up (default 4194304). */
int dgpe_batch_hold_problem(dgpe_batch_t b, int i);
int dgpe_batch_set_wait_limit(dgpe_batch_t b, long long polls);
int dgpe_batch_observables(dgpe_batch_t b, int i, dgpe_obs *o);                /* synchronises */
/* number of classes, total sites, algorithmic HBM bytes of one step */
int dgpe_batch_info(dgpe_batch_t b, int *classes, long long *sites, double *bytes_per_step);
int dgpe_batch_launches_per_step(dgpe_batch_t b);  /* kernel launches per dgpe_batch_step call: 1 */
const char *dgpe_batch_last_error(dgpe_batch_t b);

/* Phi_d of |psi|^2 for a caller's state, computed without allocating any
 * device memory (the paper has no counterpart: this serves callers that must
 * not call cudaMalloc while they run -- work recorded into another
 * framework's stream capture, fixed device-memory budgets or caching
 * allocators that must own every allocation, real-time loops that cannot
 * afford an allocation's latency or failure).
 *   psi: device buffer of n_sites complex values, complex128 when fp64 != 0,
 *        else complex64, layout [z][y][x] / [y][x];
 *   phi: device buffer of n_sites reals (double when fp64 != 0, else float);
 *   dim, n, h, kernel, qd: as in dgpe_params (kernel DIPOLAR_3D with dim 3 or
 *        QUASI2D_XY with dim 2; QUASI2D_XZ returns DGPE_EUNSUPPORTED); each
 *        n a power of two in [32, 512] and at most 262144 sites in total,
 *        else DGPE_EUNSUPPORTED;
 *   cuda_stream: cudaStream_t (NULL = legacy default stream); asynchronous.
 * All scratch (half spectrum, U(k)/N, FFT roots) lives in one 4 MiB static
 * device array that every GPU loading this library keeps until exit.  The
 * first call on a device looks up that array's address (with the device
 * current), so make it before any stream capture.  Every call reuses the same
 * array and re-initialises what it reads first; calls that overlap on the GPU
 * (other streams, other threads) race on it.  No allocation of any kind.
 * The array's address is looked up once per device and kept: do not call
 * this entry point again after cudaDeviceReset in the same process.
 * Devices 0..63 only.
 * Errors: DGPE_EINVAL / DGPE_EUNSUPPORTED / DGPE_ECUDA, text in
 * dgpe_noalloc_last_error(). */
int dgpe_dipolar_potential_noalloc(const void *psi, void *phi, int fp64, int dim,
                                   const int n[3], const double h[3], int kernel,
                                   double qd, void *cuda_stream);
const char *dgpe_noalloc_last_error(void);

/* Text of the last error of h (or of the last failed dgpe_create when h is
 * NULL).  Valid until the next call on the same handle. */
const char *dgpe_last_error(dgpe_t h);

#ifdef __cplusplus
}
#endif

#endif /* DGPE_H */
