// dgpe_kernels.cuh -- the passes of one split-step Crank-Nicolson step of the
// dipolar GP equation (arXiv:1601.04640, "Solution method"; the GPU functions
// calcpsidd2, calcnu, calclux/calcluy/calcluz and calcnorm of "Summary of
// revisions"), as fused tile kernels for sm_103a.  Included by the FP64 and
// FP32-bulk instantiation units.
//
// Layout: psi [z][y][x] complex (x fastest); half spectrum [z][y][kx] with
// kx = 0..nx/2 and row pitch px; U table with the spectrum's layout.
// One 3D step = 7 passes:
//   P4 density + R2C_x   P5 FFT_y   P6 FFT_z . U . IFFT_z   P7 IFFT_y
//   P1 C2R_x + exponential + CN_x   P2 CN_y   P3 CN_z (+ norm, step counter)
// A 2D step = P4, P6 along y, P1, P2 (CN_y is the final pass).
#pragma once

#include <cuda.h>  // CUtensorMap (the type of a TMA descriptor parameter)

#include "dgpe_device.cuh"

// Kernels have internal linkage (unnamed namespace): every translation unit
// that launches a kernel registers and configures its own copy, so a kernel
// attribute set in one unit always applies to the copy that unit launches.
namespace dgpe {
namespace {

// FP64 parameter block read by every pass (so quenches and modulation need no
// graph re-capture).  Index constants:
enum {
  PRM_SC = 0,    // lazy normalisation: the true psi is sc * stored psi
  PRM_DT = 1,
  PRM_G = 2,
  PRM_GDD = 3,
  PRM_CELL = 4,  // h^d
  PRM_M = 5,     // number of trap-modulation coefficients
  PRM_CM = 6,    // c_1 .. c_16
  PRM_NONFINITE = 22,  // set to 1 by the norm finaliser when the norm is not finite
  PRM_TIMEOUT = 23,    // set to 1 by a kernel whose bounded device-side wait ran out
  PRM_COUNT = 24
};

template <typename R> struct XArgs {  // x-line passes
  cx<R> *psi;
  cx<R> *spec;
  R *phi_out;
  const R *dens_in;  // P4 with SRC = 1: transform this real field instead of |psi|^2
  const double *prm;
  const long long *step;
  const cx<R> *tw;
  const rt4<R> *twf, *twi;  // FMA-form roots of the axis (power-of-two lengths; forward, inverse)
  const R *vx, *vy, *vz;
  const void *cntab;
  FftPlan pl;
  int nx, ny, nrows, px, LP;
  int pitchz, pitch, TPL, C;
  int imag, has_dip;
  int cnd;  // chunk-scan reach of the CN_x solve (0: all lanes)
  double tau;
  double dtf;  // fraction of dt taken by the exponential substep (1: a full step)
};

template <typename R> struct SArgs {  // strided FFT passes over the spectrum
  cx<R> *spec;
  const R *U;
  double *partial;
  const cx<R> *tw;
  const rt4<R> *twf, *twi;  // FMA-form roots of the axis (power-of-two lengths; forward, inverse)
  FftPlan pl;
  long long estride, ostride;
  int n, ncols, W, nxh;
  // 3D dipolar kernel from the wavenumbers (FP32 tensor-map z-pass):
  // dq_x, dq_y, dq_z (2 pi / (n h) per axis), (4 pi / 3) / N_sites; ny
  float uq[4];
  int uny;
};

template <typename R> struct CArgs {  // strided CN passes
  cx<R> *psi;
  const void *cntab;
  double *prm;
  double *partial;
  unsigned *counter;
  long long *step;
  long long estride, ostride;
  int n, ncols, W, TPL, C, pitch;
  int final_pass, norm;
  int cnd;  // chunk-scan reach of the CN solve (0: all lanes)
  double tau;
};

template <typename R> struct OArgs {  // observables over sites
  const cx<R> *psi;
  const double *prm;
  double *partial;
  int nx, ny, nz, dim, rows_per_block;
  double hx, hy, hz, nux, nuy, nuz;
};

template <typename Coef> __device__ __forceinline__ Coef make_kt(double tau);
template <> __device__ __forceinline__ double make_kt<double>(double tau) { return tau; }
template <> __device__ __forceinline__ float make_kt<float>(double tau) { return (float)tau; }
template <> __device__ __forceinline__ double2 make_kt<double2>(double tau) { return make_double2(0.0, tau); }
template <> __device__ __forceinline__ float2 make_kt<float2>(double tau) { return make_float2(0.0f, (float)tau); }

// sin x and cos x - 1.  For |x| <= 1/8 their Taylor series about 0,
//   sin x     = x - x^3/3! + x^5/5! - ...,
//   cos x - 1 = -x^2/2! + x^4/4! - x^6/6! + ...,
// truncated where the first omitted term (the series alternate with
// decreasing terms, so it bounds the remainder) is below half an ulp relative:
// through x^9 / x^10 in FP64 (omitted terms 2.3e-17 and 3.9e-18 relative at
// |x| = 1/8), through x^5 / x^6 in FP32 (7.6e-10, 1.9e-10).  cos x - 1 is
// formed directly, so it keeps full relative precision for small x.  Larger
// arguments use the half-angle identities cos x - 1 = -2 sin^2(x/2) and
// sin x = 2 sin(x/2) cos(x/2) with the library sincos.
template <typename R> __device__ __forceinline__ void sin_cosm1(R x, R *sn, R *cm1) {
  if (fabs(x) <= (R)0.125) {  // compared in R: an FP64 compare per site is FP64-pipe work in the FP32 form
    const R x2 = x * x;
    R ps, pc;
    if (sizeof(R) == 8) {
      ps = (R)(1.0 / 362880.0);
      ps = ps * x2 + (R)(-1.0 / 5040.0);
      ps = ps * x2 + (R)(1.0 / 120.0);
      ps = ps * x2 + (R)(-1.0 / 6.0);
      pc = (R)(-1.0 / 3628800.0);
      pc = pc * x2 + (R)(1.0 / 40320.0);
      pc = pc * x2 + (R)(-1.0 / 720.0);
      pc = pc * x2 + (R)(1.0 / 24.0);
      pc = pc * x2 + (R)(-0.5);
    } else {
      ps = (R)(1.0 / 120.0);
      ps = ps * x2 + (R)(-1.0 / 6.0);
      pc = (R)(-1.0 / 720.0);
      pc = pc * x2 + (R)(1.0 / 24.0);
      pc = pc * x2 + (R)(-0.5);
    }
    *sn = x + (x * x2) * ps;
    *cm1 = x2 * pc;
  } else {
    R s, c;
    fsincos(x * (R)0.5, &s, &c);
    *cm1 = (R)-2 * s * s;
    *sn = (R)2 * s * c;
  }
}

// psi <- psi exp(-kappa theta) in increment form (psi + psi (e - 1)) so that
// rounding of the factor scales with theta, not with psi.
template <typename R> __device__ __forceinline__ cx<R> nonlinear_factor(cx<R> v, R th, int imag) {
  if (imag) {
    R f = fexpm1(-th);
    return mk<R>(v.x + v.x * f, v.y + v.y * f);
  }
  R sn, cm1;
  sin_cosm1<R>(th, &sn, &cm1);
  // v (cm1 - i sn)
  return mk<R>(v.x + (v.x * cm1 + v.y * sn), v.y + (v.y * cm1 - v.x * sn));
}

// s(t) dt with s(t) = 1 + sum_m c_m sin(m t), t = step * dt (FP64, one thread)
__device__ __forceinline__ double trap_dts(const double *prm, long long step) {
  const double dt = prm[PRM_DT];
  const int M = (int)prm[PRM_M];
  const double t = (double)step * dt;
  double s = 1.0;
  for (int m = 1; m <= M; ++m) s += prm[PRM_CM + m - 1] * sin((double)m * t);
  return s * dt;
}

// ------------------------------------------------------------------ P4
// elements per 128 bytes: the pad period of line-major tiles
template <typename R> struct Pad { static constexpr int W = 128 / (int)sizeof(cx<R>); };

// Every pass is launched with at most DGPE_MAXT threads per block and held to
// 2 resident blocks per SM worth of registers (128 per thread), except these
// FP32 kernels, whose register budgets (65536 / (256 x blocks)) were picked by
// timing the 256^3 step: strided transforms 4 blocks (64 registers; 3 blocks
// made FFT_z.U.IFFT_z 11 % slower), C2R/exponential/CN_x 3 blocks (2: 7 %
// slower, 4: 13 % slower), pipelined CN 2 blocks (3: 14 % slower).
#define DGPE_MAXT 256
#ifndef DGPE_MAXT_FFT
#define DGPE_MAXT_FFT 256  // strided transforms
#endif
#ifndef DGPE_W_FFT_F32
#define DGPE_W_FFT_F32 16  // FP32 strided transforms: columns per tile
#endif
#define DGPE_MINB(R) 2
// The density/R2C and strided transform passes read their twiddles from a
// shared copy made once per block (1) or from global memory through L1 (0):
// the copy relieves the L1TEX pipe, the FP64 transforms' top stall (1-3 %).
#ifndef DGPE_TW_SMEM
#define DGPE_TW_SMEM 1
#endif
#ifndef DGPE_MINB_FFT_F32
#define DGPE_MINB_FFT_F32 4
#endif
// FP64: 3 blocks for EPT <= 8 (85 registers, no spills; 3-6 % faster than 2),
// 2 for the 3 2^k and 5 2^k variants (EPT 12, 20), which spill at 3
#ifndef DGPE_MINB_FFT_F64
#define DGPE_MINB_FFT_F64 3
#endif
#define DGPE_MINB_FFT(R, EPT) (sizeof(R) == 4 ? DGPE_MINB_FFT_F32 : ((EPT) <= 8 ? DGPE_MINB_FFT_F64 : 2))
#ifndef DGPE_MINB_P1_F32
#define DGPE_MINB_P1_F32 3
#endif
#ifndef DGPE_MINB_CN_F32
#define DGPE_MINB_CN_F32 2
#endif
#define DGPE_MINB_P1(R) (sizeof(R) == 4 ? DGPE_MINB_P1_F32 : 2)
#ifndef DGPE_MINB_P4_F64
#define DGPE_MINB_P4_F64 2
#endif
#define DGPE_MINB_P4(R) (sizeof(R) == 4 ? 2 : DGPE_MINB_P4_F64)
#define DGPE_MINB_CN(R) (sizeof(R) == 4 ? DGPE_MINB_CN_F32 : 2)

// Copy the n twiddles of an axis into shared memory (all threads take part;
// the caller's next barrier publishes them).
template <typename R>
__device__ __forceinline__ const cx<R> *stage_twiddles(cx<R> *dst, const cx<R> *__restrict__ tw, int n) {
  if (!DGPE_TW_SMEM) return tw;
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = tw[i];
  __syncthreads();
  return dst;
}

// Copy the n FMA-form roots of an axis into shared memory (all threads; the
// barrier publishes them).  At most 512 roots.
template <typename T> __device__ __forceinline__ const T *stage_roots(T *dst, const T *__restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
  return dst;
}

// Batched kernels: the block's problem arguments, copied once into shared
// memory (a by-value copy of a struct whose members are passed on by
// reference lands in local memory, one local load per field access).
template <typename T> __device__ __forceinline__ const T &block_args(const T *__restrict__ args, T &dst) {
  if (threadIdx.x == 0) dst = args[blockIdx.z];
  __syncthreads();
  return dst;
}

// Shared scratch of a pass body: the bytes a body would otherwise declare as
// static __shared__ arrays.  A body called with SCR = 0 takes its own size;
// a kernel that runs several bodies passes one common size to all of them, so
// they use the same allocation (function-scope __shared__ storage is one
// object per template instantiation and kernel).
template <int BYTES> __device__ __forceinline__ unsigned char *shared_scratch() {
  __shared__ __align__(32) unsigned char buf[BYTES];
  return buf;
}
__host__ __device__ constexpr int scr_align(int b) { return (b + 31) & ~31; }

// SRC 0: the density sc^2 |psi|^2;  SRC 1: the real field A.dens_in;
// SRC 2: sc^2 psi^2 of a real state (A.psi holds nx reals per row).
// FMA: twiddled stages in FMA form (tile_fft), roots from A.twf.
// NC > 0 (FP32, nx = NC, the default tile of 2 LP rows and DGPE_MAXT
// threads): the line length, tile and plan are compile-time constants and
// the transform is tile_fft_ct.
template <typename R, int EPT, int SRC, bool POW2, bool FMA = false, int SCR = 0, int NC = 0>
__device__ __forceinline__ void dens_r2c_x_body(const XArgs<R> &A, int bx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *zt = reinterpret_cast<cx<R> *>(smraw);
  constexpr int PW = Pad<R>::W;
  // CN chunk of the length's variant (2^k: 16, 3 2^k: 12, 5 2^k: 10) sets the
  // tile: LP = (DGPE_MAXT / 2) / (n / CL) lines
  constexpr int CLX = (NC % 3 == 0) ? 12 : (NC % 5 == 0) ? 10 : 16;
  constexpr int LPC = NC ? (DGPE_MAXT / 2) / (NC / CLX) : 0, SLC = NC ? NC + NC / PW + 1 : 0;
  const int n = NC ? NC : A.nx, SL = NC ? SLC : A.pitchz, nrows = A.nrows, LP = NC ? LPC : A.LP;
  const int px = NC ? NC / 2 + 2 : A.px;
  const int p0 = bx * LP;
  const R sc = (R)A.prm[PRM_SC];
  const R sc2 = sc * sc;
  const cx<R> *__restrict__ psi = A.psi;
  auto load = [&](int l, int a) -> cx<R> {
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    R d0 = 0, d1 = 0;
    if (SRC == 1) {
      if (r0 < nrows) d0 = A.dens_in[(size_t)r0 * n + a];
      if (r1 < nrows) d1 = A.dens_in[(size_t)r1 * n + a];
    } else if (SRC == 2) {
      const R *__restrict__ pr = reinterpret_cast<const R *>(psi);
      if (r0 < nrows) { const R v = pr[(size_t)r0 * n + a]; d0 = sc2 * (v * v); }
      if (r1 < nrows) { const R v = pr[(size_t)r1 * n + a]; d1 = sc2 * (v * v); }
    } else {
      if (r0 < nrows) { cx<R> v = psi[(size_t)r0 * n + a]; d0 = sc2 * (v.x * v.x + v.y * v.y); }
      if (r1 < nrows) { cx<R> v = psi[(size_t)r1 * n + a]; d1 = sc2 * (v.x * v.x + v.y * v.y); }
    }
    return mk<R>(d0, d1);
  };
  auto store = [&](int l, int a, cx<R> v) { zt[sidx<PW>(l, a, SL, 1)] = v; };
  constexpr int NTW = (DGPE_TW_SMEM && !FMA) ? 512 : 1, NRT = FMA ? 512 : 1;
  constexpr int OFF_RT = scr_align(sizeof(cx<R>) * NTW), NEED = OFF_RT + sizeof(rt4<R>) * NRT;
  static_assert(SCR == 0 || NEED <= SCR, "shared scratch too small");
  unsigned char *scr = shared_scratch<SCR ? SCR : NEED>();
  cx<R> *s_tw = reinterpret_cast<cx<R> *>(scr);
  rt4<R> *s_rt = reinterpret_cast<rt4<R> *>(scr + OFF_RT);
  const cx<R> *tw = FMA ? A.tw : stage_twiddles<R>(s_tw, A.tw, n);
  const rt4<R> *rt = FMA ? stage_roots(s_rt, A.twf, n) : nullptr;
  if constexpr (NC > 0) tile_fft_ct<R, NC, EPT, false, PW, SLC, LPC, DGPE_MAXT>(zt, tw, load, store);
  else tile_fft<R, EPT, false, false, PW, POW2, FMA>(zt, SL, 1, A.LP, A.pl, tw, load, store, rt);
  // two real lines were packed as Z = n0 + i n1: X0 = (Z_k + conj Z_{n-k}) / 2,
  // X1 = (Z_k - conj Z_{n-k}) / (2i), k = 0..n/2
  const int nh = n / 2 + 1;
  for (int idx = threadIdx.x; idx < LP * nh; idx += blockDim.x) {
    const int l = idx / nh, k = idx - l * nh;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    if (r0 >= nrows) continue;
    const cx<R> Zk = zt[sidx<PW>(l, k, SL, 1)], Zm = zt[sidx<PW>(l, (k == 0 ? 0 : n - k), SL, 1)];
    const cx<R> X0 = mk<R>((R)0.5 * (Zk.x + Zm.x), (R)0.5 * (Zk.y - Zm.y));
    const cx<R> X1 = mk<R>((R)0.5 * (Zk.y + Zm.y), (R)0.5 * (Zm.x - Zk.x));
    A.spec[(size_t)r0 * px + k] = X0;
    if (r1 < nrows) A.spec[(size_t)r1 * px + k] = X1;
  }
}
template <typename R, int EPT, int SRC = 0, bool POW2 = true, bool FMA = false>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB_P4(R)) k_dens_r2c_x(const __grid_constant__ XArgs<R> A) {
  dens_r2c_x_body<R, EPT, SRC, POW2, FMA>(A, blockIdx.x);
}
// batched: one problem per blockIdx.z
template <typename R, int EPT, bool POW2>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB_P4(R)) k_dens_r2c_x_batch(const XArgs<R> *__restrict__ args) {
  __shared__ XArgs<R> sA;
  const XArgs<R> &A = block_args(args, sA);
  if (blockIdx.x * A.LP * 2 >= (unsigned)A.nrows) return;
  dens_r2c_x_body<R, EPT, 0, POW2>(A, blockIdx.x);
}

// ------------------------------------------------------------------ P1
// MODE 0: full substep (C2R_x, exponential, CN_x).  MODE 1: write Phi_d only.
// MODE 2: CN_x alone (the reverse step applies it to the adjoint field).
// MODE 3: C2R_x and the exponential, no CN (a separate CN_x pass follows).
// MODE 4: MODE 0 for a real state in imaginary time (A.psi holds nx reals per
//   row).  Rows 2l and 2l + 1 of the CTA share tile line l as its real and
//   imaginary parts: the exponential scales each part by its own row's
//   factor, and one Crank-Nicolson solve with the real coefficients of
//   imaginary time advances both rows.
// NC > 0 (FP32, nx = NC, the default tile, DGPE_MAXT threads): compile-time
// lengths and tile, the C2R transform by tile_fft_ct.
template <typename R, typename Coef, int EPT, int CL, int MODE, bool POW2, bool FMA = false, int SCR = 0, int NC = 0>
__device__ __forceinline__ void c2r_x_exp_cnx_body(const XArgs<R> &A, int bx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int PW = Pad<R>::W;
  constexpr int LPC = NC ? (DGPE_MAXT / 2) / (NC / CL) : 0, PC = NC ? NC + NC / CL + 1 : 0;
  constexpr int PZC = NC ? NC + NC / PW + 1 : 0;
  const int LP = NC ? LPC : A.LP;
  cx<R> *pt = reinterpret_cast<cx<R> *>(smraw);          // psi tile: 2 LP lines, pitch P
  cx<R> *zt = pt + 2 * LP * (NC ? PC : A.pitch);         // Z tile: LP lines, pitch pitchz
  constexpr bool TAB = (sizeof(R) == 8);
  // shared scratch: s_k[4] (dt s(t) f, g dt f, g_dd dt f, sc; thread 0, from
  // FP64), s_vyz[DGPE_MAXT] (V_y + V_z of the CTA's rows, 2 LP <= DGPE_MAXT),
  // s_dvx (FP64 real time: dt s(t) V_x), s_tab (FP32: padded shared copy of
  // the four CN tables; FP64 reads them from global memory: its FP64 pipe,
  // not the table loads, is the limit), s_rt (FMA-form roots)
  constexpr int NDVX = TAB ? 512 : 1, NTAB = TAB ? 1 : 4 * (512 + 512 / CL + 1);
  constexpr int NRT = (FMA && MODE != 2) ? 512 : 1;
  constexpr int OFF_VYZ = scr_align(sizeof(R) * 4), OFF_DVX = OFF_VYZ + scr_align(sizeof(R) * DGPE_MAXT);
  constexpr int OFF_TAB = OFF_DVX + scr_align(sizeof(R) * NDVX), OFF_RT = OFF_TAB + scr_align(sizeof(Coef) * NTAB);
  constexpr int NEED = OFF_RT + sizeof(rt4<R>) * NRT;
  static_assert(SCR == 0 || NEED <= SCR, "shared scratch too small");
  unsigned char *scr = shared_scratch<SCR ? SCR : NEED>();
  R *const s_k = reinterpret_cast<R *>(scr);
  R *const s_vyz = reinterpret_cast<R *>(scr + OFF_VYZ);
  R *const s_dvx = reinterpret_cast<R *>(scr + OFF_DVX);
  Coef *const s_tab = reinterpret_cast<Coef *>(scr + OFF_TAB);
  if (!TAB && MODE != 1 && MODE != 3) stage_cn_tables<Coef, CL>(s_tab, reinterpret_cast<const Coef *>(A.cntab), NC ? NC : A.nx);
  constexpr bool RS = (MODE == 4);  // real state
  R *const ptr = reinterpret_cast<R *>(pt);
  // tile element of row L, column a: (line, component) for a real state
  const int n = NC ? NC : A.nx, nh = n / 2, nrows = A.nrows, P = NC ? PC : A.pitch;
  const int px = NC ? NC / 2 + 2 : A.px;
  auto rs_at = [&](int L, int a) -> R & { return ptr[2 * ((L >> 1) * P + a + a / CL) + (L & 1)]; };
  const int ln = POW2 ? ilog2(n) : 0;
  const int p0 = bx * LP;
  const int T = blockDim.x, t = threadIdx.x;
  auto row_of = [&](int idx) { return POW2 ? (idx >> ln) : (idx / n); };
  auto col_of = [&](int idx) { return POW2 ? (idx & (n - 1)) : (idx % n); };
  // the trap tables are read only by the modes that apply the exponential
  // (MODE 1 and 2 callers may leave vx, vy, vz NULL)
  if constexpr (MODE != 1 && MODE != 2) {
    if (t < 2 * LP) {
      const int row = 2 * p0 + t;
      s_vyz[t] = (row < nrows) ? A.vy[row % A.ny] + A.vz[row / A.ny] : (R)0;
    }
  }
  // x twiddles: read from global memory here (a shared copy measured slower
  // for this pass; the FP32 block's shared memory is sized for 3 blocks/SM);
  // the FMA-form roots (FP64) from a shared copy
  const cx<R> *s_twp = A.tw;
  rt4<R> *const s_rt = reinterpret_cast<rt4<R> *>(scr + OFF_RT);
  const rt4<R> *rt = nullptr;
  if constexpr (FMA && MODE != 2) rt = stage_roots(s_rt, A.twi, n);
  if constexpr (RS) {
    const R *__restrict__ pr = reinterpret_cast<const R *>(A.psi);
    R buf[CL];
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int idx = t + i * T;
      const int row = 2 * p0 + row_of(idx);
      buf[i] = (row < nrows) ? pr[(size_t)row * n + col_of(idx)] : (R)0;
    }
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int idx = t + i * T;
      rs_at(row_of(idx), col_of(idx)) = buf[i];
    }
  } else if (MODE != 1) {
    // the CTA's rows 2 p0 .. 2 p0 + 2 LP - 1 are one contiguous block of psi:
    // every load of the tile is issued before any is used (2 LP n = CL T)
    cx<R> buf[CL];
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int idx = t + i * T;
      const int L = row_of(idx), a = col_of(idx);
      const int row = 2 * p0 + L;
      buf[i] = (row < nrows) ? A.psi[(size_t)row * n + a] : czero<cx<R>>();
    }
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int idx = t + i * T;
      const int L = row_of(idx), a = col_of(idx);
      pt[L * P + a + a / CL] = buf[i];
    }
  }
  if (t == 0) {
    s_k[0] = (MODE != 1 && MODE != 2) ? (R)(trap_dts(A.prm, *A.step) * A.dtf) : (R)0;
    s_k[1] = (R)(A.prm[PRM_DT] * A.dtf * A.prm[PRM_G]);
    s_k[2] = (R)(A.prm[PRM_DT] * A.dtf * A.prm[PRM_GDD]);
    s_k[3] = (R)A.prm[PRM_SC];
  }
  __syncthreads();
  const R dts = s_k[0], gdt = s_k[1], gdddt = s_k[2], sc = s_k[3];
  const int imag = A.imag;
  constexpr bool DIRECT = (sizeof(R) == 8);  // FP64: the direct (scaled) phase factor in real time
  if (DIRECT && !imag && MODE != 1 && MODE != 2) {
    // dt s(t) V with the scale of V_y + V_z applied in place (each CTA owns its rows)
    for (int a = t; a < n; a += T) s_dvx[a] = dts * A.vx[a];
    if (t < 2 * LP) s_vyz[t] *= dts;
    __syncthreads();
  }
  // exponential substep on the tile element (L, a) in place.  FP64 real
  // time multiplies the stored value by sc e^{-i theta} directly (the scale
  // folded into the factor); FP32 forms the scaled value and updates it in
  // increment form.
  const R gdt_sc2 = gdt * sc * sc;
  auto apply_e = [&](int L, int a, R phi) {
    if constexpr (RS) {
      R &u = rs_at(L, a);
      const R v = u * sc;
      const R th = dts * (A.vx[a] + s_vyz[L]) + gdt * (v * v) + gdddt * phi;
      const R f = fexpm1(-th);
      u = v + v * f;
      return;
    }
    const int ia = L * P + a + a / CL;
    if (DIRECT && !imag) {
      const cx<R> u = pt[ia];
      const R th = gdt_sc2 * (u.x * u.x + u.y * u.y) + (gdddt * phi + (s_dvx[a] + s_vyz[L]));
      R sn, cm1;
      sin_cosm1<R>(th, &sn, &cm1);
      const R fr = sc + sc * cm1, fi = -sc * sn;  // sc (cos th - i sin th)
      pt[ia] = mk<R>(u.x * fr - u.y * fi, u.x * fi + u.y * fr);
      return;
    }
    const R V = A.vx[a] + s_vyz[L];
    cx<R> v = cscale(pt[ia], sc);
    const R dens = v.x * v.x + v.y * v.y;
    const R th = dts * V + gdt * dens + gdddt * phi;
    pt[ia] = nonlinear_factor<R>(v, th, imag);
  };
  if (MODE == 2) {
    __syncthreads();
  } else if (A.has_dip) {
    auto load = [&](int l, int a) -> cx<R> {
      const int r0 = 2 * (p0 + l), r1 = r0 + 1;
      const int k = (a <= nh) ? a : n - a;
      cx<R> X0 = czero<cx<R>>(), X1 = czero<cx<R>>();
      if (r0 < nrows) X0 = A.spec[(size_t)r0 * px + k];
      if (r1 < nrows) X1 = A.spec[(size_t)r1 * px + k];
      if (a == 0 || a == nh) { X0.y = 0; X1.y = 0; }  // real-to-real ends of a real line
      if (a > nh) { X0.y = -X0.y; X1.y = -X1.y; }    // Hermitian extension
      return mk<R>(X0.x - X1.y, X0.y + X1.x);        // Z = X0 + i X1
    };
    auto store = [&](int l, int a, cx<R> v) {
      const int r0 = 2 * (p0 + l), r1 = r0 + 1;
      if (MODE == 1) {
        if (r0 < nrows) A.phi_out[(size_t)r0 * n + a] = v.x;
        if (r1 < nrows) A.phi_out[(size_t)r1 * n + a] = v.y;
        return;
      }
      apply_e(2 * l, a, v.x);
      apply_e(2 * l + 1, a, v.y);
    };
    if constexpr (NC > 0) tile_fft_ct<R, NC, EPT, true, PW, PZC, LPC, DGPE_MAXT>(zt, s_twp, load, store);
    else tile_fft<R, EPT, true, false, PW, POW2, FMA>(zt, A.pitchz, 1, A.LP, A.pl, s_twp, load, store, rt);
  } else if (MODE == 0 || MODE == 3 || MODE == 4) {
    for (int idx = t; idx < 2 * LP * n; idx += T) apply_e(row_of(idx), col_of(idx), (R)0);
    __syncthreads();
  }
  if (MODE == 1) return;
  if (MODE == 3) {
    __syncthreads();
    for (int idx = t; idx < 2 * LP * n; idx += T) {
      const int L = row_of(idx), a = col_of(idx);
      const int row = 2 * p0 + L;
      if (row < nrows) A.psi[(size_t)row * n + a] = pt[L * P + a + a / CL];
    }
    return;
  }
  // Crank-Nicolson along x: TPL lanes per line (a real state: LP lines, each
  // a pair of rows; the other half of the threads idles)
  const int TPLr = NC ? NC / CL : A.TPL;
  const int l = t / TPLr, q = t - l * TPLr;
  const bool active = RS ? (l < LP && 2 * (p0 + l) < nrows) : (2 * p0 + l) < nrows;
  if constexpr (TAB) cn_line<R, Coef, CL>(pt + l * P, n, TPLr, q, make_kt<Coef>(A.tau),
                                      reinterpret_cast<const Coef *>(A.cntab), active);
  else cn_line_st<R, Coef, CL>(pt + l * P, n, TPLr, q, make_kt<Coef>(A.tau), s_tab, active, A.cnd);
  __syncthreads();
  if constexpr (RS) {
    R *__restrict__ pr = reinterpret_cast<R *>(A.psi);
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int idx = t + i * T;
      const int L = row_of(idx), a = col_of(idx);
      const int row = 2 * p0 + L;
      if (row < nrows) pr[(size_t)row * n + a] = rs_at(L, a);
    }
    return;
  }
#pragma unroll
  for (int i = 0; i < CL; ++i) {
    const int idx = t + i * T;
    const int L = row_of(idx), a = col_of(idx);
    const int row = 2 * p0 + L;
    if (row < nrows) A.psi[(size_t)row * n + a] = pt[L * P + a + a / CL];
  }
}
template <typename R, typename Coef, int EPT, int CL, int MODE, bool POW2 = true, bool FMA = false>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB_P1(R)) k_c2r_x_exp_cnx(const __grid_constant__ XArgs<R> A) {
  c2r_x_exp_cnx_body<R, Coef, EPT, CL, MODE, POW2, FMA>(A, blockIdx.x);
}
template <typename R, typename Coef, int EPT, int CL, bool POW2>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB_P1(R)) k_c2r_x_exp_cnx_batch(const XArgs<R> *__restrict__ args) {
  __shared__ XArgs<R> sA;
  const XArgs<R> &A = block_args(args, sA);
  c2r_x_exp_cnx_body<R, Coef, EPT, CL, 0, POW2>(A, blockIdx.x);
}

#ifndef DGPE_WAIT_LIMIT
#define DGPE_WAIT_LIMIT (1 << 22)  // polls of a bounded mbarrier wait
#endif

// ----------------------------------------------- P4, FP32 pipelined form
// The density + R2C pass of the FP32 bulk (complex state, power-of-two nx) as
// a persistent pipeline: a tile's 2 LP rows of psi are one contiguous block,
// brought into one of two staging buffers by a bulk copy on that buffer's
// mbarrier, two tiles ahead of the transform.  The density is formed as the
// first Stockham stage reads the staged rows; the separated half spectra are
// stored from the Z tile.  Shared memory (dynamic): 2 psi stages [2 LP][nx],
// Z tile [LP][pitchz].
template <int EPT, int N>
__global__ void __launch_bounds__(DGPE_MAXT, 2) k_p4_pipe(const __grid_constant__ XArgs<float> A, int ntiles,
                                                         double *timeout_flag) {
  typedef float R;
  typedef float2 Cx;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int PW = Pad<R>::W;
  constexpr int T = DGPE_MAXT, TPL = N / 16, LP = (DGPE_MAXT / 2) / TPL, ROWS = 2 * LP;
  constexpr int SL = N + N / PW + 1, PX = N / 2 + 2, LN = ct_log2(N), NH = N / 2 + 1;
  const int nrows = A.nrows;
  const int t = threadIdx.x;
  Cx *const stg0 = reinterpret_cast<Cx *>(smraw);  // stage k at stg0 + k ROWS N
  Cx *const zt = reinterpret_cast<Cx *>(smraw) + 2 * ROWS * N;
  __shared__ unsigned long long bar[2];
  __shared__ R s_sc2;
  __shared__ __align__(16) Cx s_tw[N];
  auto issue = [&](int tile, int k) {  // thread 0
    const int r0 = tile * ROWS;
    const int nr = (nrows - r0 < ROWS) ? nrows - r0 : ROWS;
    const unsigned bp = (unsigned)(sizeof(Cx) * (size_t)nr * N);
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[k], bp);
    bulk_g2s(stg0 + k * ROWS * N, A.psi + (size_t)r0 * N, bp, &bar[k]);
  };
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    const R sc = (R)A.prm[PRM_SC];
    s_sc2 = sc * sc;
  }
  __syncthreads();
  if (t == 0) {
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
  }
  for (int i = t; i < N; i += T) s_tw[i] = A.tw[i];
  __syncthreads();
  const R sc2 = s_sc2;
  unsigned ph = 0u;  // bit k: the phase parity stage k waits for next
  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, k ^= 1) {
    const int r0 = tile * ROWS;
    const bool ok = mbar_wait_bounded(&bar[k], (ph >> k) & 1u, DGPE_WAIT_LIMIT);
    ph ^= 1u << k;
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        // the copy into the other stage, if one was issued, lands (bounded wait) before the block exits
        if (tile + (int)gridDim.x < ntiles) mbar_wait_bounded(&bar[k ^ 1], (ph >> (k ^ 1)) & 1u, DGPE_WAIT_LIMIT);
        *timeout_flag = 1.0;
      }
      return;
    }
    const Cx *__restrict__ sp = stg0 + k * ROWS * N;
    const bool full = (r0 + ROWS <= nrows);
    auto load = [&](int l, int a) -> cx<R> {
      R d0 = 0, d1 = 0;
      if (full || r0 + 2 * l < nrows) { const Cx v = sp[((2 * l) << LN) + a]; d0 = sc2 * (v.x * v.x + v.y * v.y); }
      if (full || r0 + 2 * l + 1 < nrows) { const Cx v = sp[((2 * l + 1) << LN) + a]; d1 = sc2 * (v.x * v.x + v.y * v.y); }
      return mk<R>(d0, d1);
    };
    auto store = [&](int l, int a, cx<R> v) { zt[l * SL + a + a / PW] = v; };
    tile_fft_ct<R, N, EPT, false, PW, SL, LP, T>(zt, s_tw, load, store);
    // this stage is consumed: refill it two tiles ahead
    const int next2 = tile + 2 * gridDim.x;
    if (t == 0 && next2 < ntiles) issue(next2, k);
    // two real lines were packed as Z = n0 + i n1
    for (int idx = t; idx < LP * NH; idx += T) {
      const int l = idx / NH, kk = idx - l * NH;
      const int ra = r0 + 2 * l, rb = ra + 1;
      if (ra >= nrows) continue;
      const int km = (kk == 0 ? 0 : N - kk);
      const cx<R> Zk = zt[l * SL + kk + kk / PW], Zm = zt[l * SL + km + km / PW];
      A.spec[(size_t)ra * PX + kk] = mk<R>((R)0.5 * (Zk.x + Zm.x), (R)0.5 * (Zk.y - Zm.y));
      if (rb < nrows) A.spec[(size_t)rb * PX + kk] = mk<R>((R)0.5 * (Zk.y + Zm.y), (R)0.5 * (Zm.x - Zk.x));
    }
  }
  __syncthreads();
  if (t == 0) { mbar_inval(&bar[0]); mbar_inval(&bar[1]); }
}

// ----------------------------------------------- P1, FP32 pipelined form
// The x-line pass of the FP32 bulk (complex state, power-of-two nx) as a
// persistent pipeline.  A tile is the 2 LP consecutive rows of psi and of the
// half spectrum that the one-shot kernel above gives a CTA; both are
// contiguous blocks, so one thread brings them into shared memory with two
// bulk copies that complete on an mbarrier (no per-element load
// instructions), and the next tile's copies are issued as soon as the
// current tile's C2R transform and exponential have consumed the staged data,
// so they overlap its Crank-Nicolson solve and store.  The Z tile of the C2R
// transform reuses the spectrum's staging buffer (every Stockham stage reads
// all of its inputs before a barrier and writes after it).  The tables (CN
// m, alpha, P, Q; the trap potentials) are staged once per CTA.  Shared
// memory (dynamic): psi stage [2 LP][nx], spectrum stage / Z tile,
// padded psi tile [2 LP][pitch], CN tables, V_x, V_y, V_z.
struct P1Smem {
  size_t sp, sz, pt, tab, vx, vy, vz, total;  // byte offsets
};
__host__ __device__ inline size_t p1_align16(size_t b) { return (b + 15) & ~(size_t)15; }
template <typename Coef>
__host__ __device__ inline P1Smem p1_smem_layout(int nx, int ny, int nz, int LP, int px, int pitchz, int pitch, int CL) {
  P1Smem L;
  const int rows = 2 * LP;
  const size_t zel = (size_t)((rows * px > LP * pitchz) ? rows * px : LP * pitchz);
  L.sp = 0;
  L.sz = p1_align16(L.sp + sizeof(float2) * (size_t)rows * nx);
  L.pt = p1_align16(L.sz + sizeof(float2) * zel);
  L.tab = p1_align16(L.pt + sizeof(float2) * (size_t)rows * pitch);
  L.vx = p1_align16(L.tab + sizeof(Coef) * 4 * (size_t)(nx + nx / CL + 1));
  L.vy = p1_align16(L.vx + sizeof(float) * (size_t)nx);
  L.vz = p1_align16(L.vy + sizeof(float) * (size_t)ny);
  L.total = p1_align16(L.vz + sizeof(float) * (size_t)nz);
  return L;
}
template <typename Coef, int EPT, int CL, int N>
__global__ void __launch_bounds__(DGPE_MAXT, 2) k_p1_pipe(const __grid_constant__ XArgs<float> A, int ntiles, int nz,
                                                         double *timeout_flag) {
  typedef float R;
  typedef float2 Cx;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int PW = Pad<R>::W;
  constexpr int T = DGPE_MAXT, TPL = N / CL, LP = (DGPE_MAXT / 2) / TPL, ROWS = 2 * LP;
  constexpr int P = N + N / CL + 1, PZ = N + N / PW + 1, PX = N / 2 + 2, LN = ct_log2(N), NHALF = N / 2;
  static_assert(ROWS * N == CL * T, "a tile holds CL elements per thread");
  const int nrows = A.nrows, ny = A.ny;
  const int t = threadIdx.x;
  const P1Smem Ly = p1_smem_layout<Coef>(N, ny, nz, LP, PX, PZ, P, CL);
  Cx *const sp = reinterpret_cast<Cx *>(smraw + Ly.sp);
  Cx *const sz = reinterpret_cast<Cx *>(smraw + Ly.sz);
  Cx *const pt = reinterpret_cast<Cx *>(smraw + Ly.pt);
  Coef *const tab = reinterpret_cast<Coef *>(smraw + Ly.tab);
  R *const svx = reinterpret_cast<R *>(smraw + Ly.vx);
  R *const svy = reinterpret_cast<R *>(smraw + Ly.vy);
  R *const svz = reinterpret_cast<R *>(smraw + Ly.vz);
  __shared__ unsigned long long bar;
  __shared__ R s_vyz[ROWS];  // V_y + V_z of the tile's rows
  __shared__ R s_k[4];
  __shared__ __align__(16) Cx s_tw[N];
  const bool dip = A.has_dip != 0;
  auto issue = [&](int tile) {  // thread 0
    const int r0 = tile * ROWS;
    const int nr = (nrows - r0 < ROWS) ? nrows - r0 : ROWS;
    const unsigned bp = (unsigned)(sizeof(Cx) * (size_t)nr * N);
    const unsigned bs = dip ? (unsigned)(sizeof(Cx) * (size_t)nr * PX) : 0u;
    fence_proxy_async_smem();
    mbar_expect_tx(&bar, bp + bs);
    bulk_g2s(sp, A.psi + (size_t)r0 * N, bp, &bar);
    if (dip) bulk_g2s(sz, A.spec + (size_t)r0 * PX, bs, &bar);
  };
  if (t == 0) {
    mbar_init(&bar, 1);
    s_k[0] = (R)(trap_dts(A.prm, *A.step) * A.dtf);
    s_k[1] = (R)(A.prm[PRM_DT] * A.dtf * A.prm[PRM_G]);
    s_k[2] = (R)(A.prm[PRM_DT] * A.dtf * A.prm[PRM_GDD]);
    s_k[3] = (R)A.prm[PRM_SC];
  }
  __syncthreads();
  if (t == 0 && (int)blockIdx.x < ntiles) issue(blockIdx.x);
  stage_cn_tables<Coef, CL>(tab, reinterpret_cast<const Coef *>(A.cntab), N);
  for (int i = t; i < N; i += T) { svx[i] = A.vx[i]; s_tw[i] = A.tw[i]; }
  for (int i = t; i < ny; i += T) svy[i] = A.vy[i];
  for (int i = t; i < nz; i += T) svz[i] = A.vz[i];
  __syncthreads();
  const R dts = s_k[0], gdt = s_k[1], gdddt = s_k[2], sc = s_k[3];
  const int imag = A.imag;
  constexpr bool RT = sizeof(Coef) == sizeof(Cx);
  unsigned phase = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, phase ^= 1u) {
    const int r0 = tile * ROWS;
    const bool full = (r0 + ROWS <= nrows);
    // every thread polls the barrier; the block then agrees on the outcome
    const bool ok = mbar_wait_bounded(&bar, phase, DGPE_WAIT_LIMIT);
    if (t < ROWS) {
      const int row = r0 + t;
      s_vyz[t] = (row < nrows) ? svy[row % ny] + svz[row / ny] : (R)0;
    }
    if (__syncthreads_or(!ok)) {
      if (t == 0) *timeout_flag = 1.0;
      return;
    }
    // exponential substep: staged psi (dense) -> padded tile
    auto apply_e = [&](int L, int a, R phi) {
      // real time (complex CN coefficients): the lazy norm scale is 1 (only
      // imaginary-time norm passes change it; a mode switch folds it into psi)
      const cx<R> v = RT ? sp[(L << LN) + a] : cscale(sp[(L << LN) + a], sc);
      const R dens = v.x * v.x + v.y * v.y;
      const R th = dts * (svx[a] + s_vyz[L]) + gdt * dens + gdddt * phi;
      pt[L * P + a + a / CL] = nonlinear_factor<R>(v, th, imag);
    };
    if (dip) {
      auto load = [&](int l, int a) -> cx<R> {
        const int k = (a <= NHALF) ? a : N - a;
        cx<R> X0 = czero<cx<R>>(), X1 = czero<cx<R>>();
        if (full || r0 + 2 * l < nrows) X0 = sz[(2 * l) * PX + k];
        if (full || r0 + 2 * l + 1 < nrows) X1 = sz[(2 * l + 1) * PX + k];
        if (a == 0 || a == NHALF) { X0.y = 0; X1.y = 0; }  // real-to-real ends of a real line
        if (a > NHALF) { X0.y = -X0.y; X1.y = -X1.y; }    // Hermitian extension
        return mk<R>(X0.x - X1.y, X0.y + X1.x);           // Z = X0 + i X1
      };
      auto store = [&](int l, int a, cx<R> v) {
        apply_e(2 * l, a, v.x);
        apply_e(2 * l + 1, a, v.y);
      };
      tile_fft_ct<R, N, EPT, true, PW, PZ, LP, T>(sz, s_tw, load, store);
    } else {
#pragma unroll 4
      for (int i = 0; i < CL; ++i) {
        const int idx = t + i * T;
        apply_e(idx >> LN, idx & (N - 1), (R)0);
      }
      __syncthreads();
    }
    // the staged blocks are consumed: fetch the next tile behind the solve
    const int next = tile + gridDim.x;
    if (t == 0 && next < ntiles) issue(next);
    // Crank-Nicolson along x: TPL lanes per line
    const int l = t / TPL, q = t - l * TPL;
    cn_line_st<R, Coef, CL>(pt + l * P, N, TPL, q, make_kt<Coef>(A.tau), tab, full || (r0 + l) < nrows,
                            A.cnd);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int idx = t + i * T;
      const int L = idx >> LN, a = idx & (N - 1);
      if (full || r0 + L < nrows) A.psi[(size_t)(r0 + L) * N + a] = pt[L * P + a + a / CL];
    }
  }
  __syncthreads();
  if (t == 0) mbar_inval(&bar);
}

// ------------------------------------------------- P5 / P6 / P7 (strided)
// MODE 0 forward, 1 inverse, 2 forward . U . inverse, 3 forward and
// accumulate sum_k w_k U_k |F_k|^2 (FP64) for the dipolar energy.
// NC > 0 (FP32, line length NC, tile width WC, WC NC / EPT threads):
// compile-time lengths, the transforms by tile_fft_ct_cols.
template <typename R, int EPT, int MODE, bool POW2, bool FMA = false, int SCR = 0, int NC = 0, int WC = 0>
__device__ __forceinline__ void fft_strided_body(const SArgs<R> &A, int bx, int by, int gx) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);  // [a][W]
  // FMA-form roots: forward (modes 0, 2, 3) and inverse (modes 1, 2)
  constexpr bool NF = FMA && MODE != 1, NI = FMA && (MODE == 1 || MODE == 2);
  // shared scratch: red[32], twiddles, forward and inverse FMA-form roots
  constexpr int NTW = (DGPE_TW_SMEM && !FMA) ? 512 : 1;
  constexpr int OFF_TW = scr_align(sizeof(double) * 32), OFF_RF = OFF_TW + scr_align(sizeof(cx<R>) * NTW);
  constexpr int OFF_RI = OFF_RF + scr_align(sizeof(rt4<R>) * (NF ? 512 : 1));
  constexpr int NEED = OFF_RI + sizeof(rt4<R>) * (NI ? 512 : 1);
  static_assert(SCR == 0 || NEED <= SCR, "shared scratch too small");
  unsigned char *scr = shared_scratch<SCR ? SCR : NEED>();
  double *const red = reinterpret_cast<double *>(scr);
  cx<R> *const s_tw = reinterpret_cast<cx<R> *>(scr + OFF_TW);
  rt4<R> *const s_rf = reinterpret_cast<rt4<R> *>(scr + OFF_RF);
  rt4<R> *const s_ri = reinterpret_cast<rt4<R> *>(scr + OFF_RI);
  const cx<R> *tw = FMA ? A.tw : stage_twiddles<R>(s_tw, A.tw, NC ? NC : A.n);
  const rt4<R> *rf = nullptr, *ri = nullptr;
  if constexpr (NF) rf = stage_roots(s_rf, A.twf, A.n);
  if constexpr (NI) ri = stage_roots(s_ri, A.twi, A.n);
  const int W = NC ? WC : A.W;
  const int c0 = bx * W;
  const size_t base = (size_t)by * A.ostride + c0;
  const long long es = A.estride;
  cx<R> *__restrict__ spec = A.spec;
  auto gload = [&](int l, int a) -> cx<R> {
    return (c0 + l < A.ncols) ? spec[base + a * es + l] : czero<cx<R>>();
  };
  auto gstore = [&](int l, int a, cx<R> v) {
    if (c0 + l < A.ncols) spec[base + a * es + l] = v;
  };
  if constexpr (NC > 0 && MODE == 2) {
    constexpr int TC = WC * NC / EPT;
    auto mstore = [&](int l, int a, cx<R> v) {
      const R u = (c0 + l < A.ncols) ? A.U[base + a * es + l] : (R)0;
      sm[a * WC + l] = cscale(v, u);
    };
    tile_fft_ct_cols<R, NC, EPT, false, WC, TC>(sm, tw, gload, mstore);
    auto sload = [&](int l, int a) -> cx<R> { return sm[a * WC + l]; };
    tile_fft_ct_cols<R, NC, EPT, true, WC, TC>(sm, tw, sload, gstore);
  } else if (MODE == 0) {
    tile_fft<R, EPT, false, true, 0, POW2, FMA>(sm, 1, W, W, A.pl, tw, gload, gstore, rf);
  } else if (MODE == 1) {
    tile_fft<R, EPT, true, true, 0, POW2, FMA>(sm, 1, W, W, A.pl, tw, gload, gstore, ri);
  } else if (MODE == 2) {
    auto mstore = [&](int l, int a, cx<R> v) {
      const R u = (c0 + l < A.ncols) ? A.U[base + a * es + l] : (R)0;
      sm[a * W + l] = cscale(v, u);
    };
    tile_fft<R, EPT, false, true, 0, POW2, FMA>(sm, 1, W, W, A.pl, tw, gload, mstore, rf);
    auto sload = [&](int l, int a) -> cx<R> { return sm[a * W + l]; };
    tile_fft<R, EPT, true, true, 0, POW2, FMA>(sm, 1, W, W, A.pl, tw, sload, gstore, ri);
  } else {
    double acc = 0.0;
    auto astore = [&](int l, int a, cx<R> v) {
      const int kx = c0 + l;
      if (kx < A.ncols) {
        const double w = (kx == 0 || kx == A.nxh) ? 1.0 : 2.0;
        acc += w * (double)A.U[base + a * es + l] * ((double)v.x * v.x + (double)v.y * v.y);
      }
    };
    tile_fft<R, EPT, false, true, 0, POW2, FMA>(sm, 1, W, W, A.pl, tw, gload, astore, rf);
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) A.partial[(size_t)by * gx + bx] = s;
  }
}
template <typename R, int EPT, int MODE, bool POW2 = true, bool FMA = false>
__global__ void __launch_bounds__(DGPE_MAXT_FFT, DGPE_MINB_FFT(R, EPT)) k_fft_strided(const __grid_constant__ SArgs<R> A) {
  fft_strided_body<R, EPT, MODE, POW2, FMA>(A, blockIdx.x, blockIdx.y, gridDim.x);
}
template <typename R, int EPT, int MODE, bool POW2>
__global__ void __launch_bounds__(DGPE_MAXT_FFT, DGPE_MINB_FFT(R, EPT)) k_fft_strided_batch(const SArgs<R> *__restrict__ args) {
  __shared__ SArgs<R> sA;
  const SArgs<R> &A = block_args(args, sA);
  fft_strided_body<R, EPT, MODE, POW2>(A, blockIdx.x, blockIdx.y, gridDim.x);
}

// FP32 strided transforms (MODE 0 forward, 1 inverse, 2 forward . U .
// inverse) with the line length N and tile width W as compile-time constants
// (power-of-two lengths): the same arithmetic as fft_strided_body, with every
// index folded (tile_fft_ct_cols).  Twiddles from a shared copy.
template <int EPT, int MODE, int N, int W>
__global__ void __launch_bounds__(DGPE_MAXT_FFT, DGPE_MINB_FFT_F32) k_fft_strided_ct(const __grid_constant__ SArgs<float> A) {
  typedef float R;
  typedef float2 Cx;
  constexpr int T = W * N / EPT;
  extern __shared__ __align__(16) unsigned char smraw[];
  Cx *sm = reinterpret_cast<Cx *>(smraw);  // [a][W]
  __shared__ __align__(16) Cx s_tw[N];
  for (int i = threadIdx.x; i < N; i += T) s_tw[i] = A.tw[i];
  __syncthreads();
  const int c0 = blockIdx.x * W;
  const size_t base = (size_t)blockIdx.y * A.ostride + c0;
  const long long es = A.estride;
  const bool fullw = c0 + W <= A.ncols;
  Cx *__restrict__ spec = A.spec;
  auto gload = [&](int l, int a) -> Cx {
    return (fullw || c0 + l < A.ncols) ? spec[base + a * es + l] : czero<Cx>();
  };
  auto gstore = [&](int l, int a, Cx v) {
    if (fullw || c0 + l < A.ncols) spec[base + a * es + l] = v;
  };
  if constexpr (MODE == 0) {
    tile_fft_ct_cols<R, N, EPT, false, W, T>(sm, s_tw, gload, gstore);
  } else if constexpr (MODE == 1) {
    tile_fft_ct_cols<R, N, EPT, true, W, T>(sm, s_tw, gload, gstore);
  } else {
    auto mstore = [&](int l, int a, Cx v) {
      const R u = (fullw || c0 + l < A.ncols) ? A.U[base + a * es + l] : (R)0;
      sm[a * W + l] = cscale(v, u);
    };
    tile_fft_ct_cols<R, N, EPT, false, W, T>(sm, s_tw, gload, mstore);
    auto sload = [&](int l, int a) -> Cx { return sm[a * W + l]; };
    tile_fft_ct_cols<R, N, EPT, true, W, T>(sm, s_tw, sload, gstore);
  }
}

// FP32 strided transforms with TMA tiles (power-of-two lengths): persistent
// CTAs walk the tiles; one thread loads a tile of W spectrum columns x N
// rows into shared memory with tensor-map copies (the dense box layout
// [row][column] is the transform's column-tile layout), two tiles ahead in
// two buffers, and writes the transformed tile back with tensor-map stores,
// so no thread issues a global load or store of the spectrum.  AXIS 1: the
// lines run along y (coordinates kx, y = row, z = outer index); AXIS 2: along
// z (kx, y = outer index, z = row).  Boxes are at most 256 rows (N = 512 takes
// two).  Columns beyond the spectrum's width load as zeros and are not
// stored.  Waits are bounded as in the x-line pipelines.
#ifndef DGPE_TMA_MINB
#define DGPE_TMA_MINB 3  // resident blocks per SM the tensor-map transforms are compiled for
#endif
// The 3D z-pass (MODE 2, AXIS 2) evaluates U(k) = (4 pi / 3)(3 k_z^2 / k^2 - 1)
// / N_sites in FP32 from the wavenumbers (U(0) = 0) instead of reading the
// table: four bytes less per spectrum element and no global load inside the
// transform pair.
template <int EPT, int MODE, int N, int W, int AXIS>
__global__ void __launch_bounds__(DGPE_MAXT_FFT, DGPE_TMA_MINB)
    k_fft_tma(const __grid_constant__ CUtensorMap tm, const __grid_constant__ SArgs<float> A, int ncb, int ntiles,
              double *timeout_flag) {
  typedef float R;
  typedef float2 Cx;
  constexpr int T = W * N / EPT, TILE = W * N;
  constexpr int NBOX = (N + 255) / 256, BOXR = N / NBOX;
  extern __shared__ __align__(16) unsigned char smraw[];
  // tiles 128-byte aligned inside the dynamic allocation (it has 128 spare bytes)
  Cx *const buf0 = reinterpret_cast<Cx *>(smraw + ((128 - (smem_u32(smraw) & 127)) & 127));
  __shared__ unsigned long long bar[2];
  __shared__ __align__(16) Cx s_tw[N];
  const int t = threadIdx.x;
  auto issue = [&](int tile, int k) {  // thread 0
    const int c0 = (tile % ncb) * W, o = tile / ncb;
    Cx *dst = buf0 + k * TILE;
    fence_proxy_async_smem();
    mbar_expect_tx(&bar[k], (unsigned)(sizeof(Cx) * TILE));
#pragma unroll
    for (int b = 0; b < NBOX; ++b) {
      if (AXIS == 1) tma_load_3d(dst + b * BOXR * W, &tm, c0, b * BOXR, o, &bar[k]);
      else tma_load_3d(dst + b * BOXR * W, &tm, c0, o, b * BOXR, &bar[k]);
    }
  };
  if (t == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
  }
  __syncthreads();
  if (t == 0) {
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
    if ((int)(blockIdx.x + gridDim.x) < ntiles) issue(blockIdx.x + gridDim.x, 1);
  }
  for (int i = t; i < N; i += T) s_tw[i] = A.tw[i];
  __syncthreads();
  unsigned ph = 0u;  // bit k: the phase parity buffer k waits for next
  int k = 0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, k ^= 1) {
    const bool ok = mbar_wait_bounded(&bar[k], (ph >> k) & 1u, DGPE_WAIT_LIMIT);
    ph ^= 1u << k;
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        bulk_wait_all();
        if (tile + (int)gridDim.x < ntiles) mbar_wait_bounded(&bar[k ^ 1], (ph >> (k ^ 1)) & 1u, DGPE_WAIT_LIMIT);
        *timeout_flag = 1.0;
      }
      return;
    }
    Cx *const sm = buf0 + k * TILE;
    const int c0 = (tile % ncb) * W, o = tile / ncb;
    auto sload = [&](int l, int a) -> Cx { return sm[a * W + l]; };
    auto sstore = [&](int l, int a, Cx v) { sm[a * W + l] = v; };
    if constexpr (MODE == 0) {
      tile_fft_ct_cols<R, N, EPT, false, W, T>(sm, s_tw, sload, sstore);
    } else if constexpr (MODE == 1) {
      tile_fft_ct_cols<R, N, EPT, true, W, T>(sm, s_tw, sload, sstore);
    } else if constexpr (AXIS == 2) {
      // tile: kx = c0 + l, ky = o, kz = row a
      const int jy = (o <= A.uny / 2) ? o : o - A.uny;
      const R qy = (R)jy * A.uq[1];
      const R qy2 = qy * qy, dqx = A.uq[0], dqz = A.uq[2], pref = A.uq[3];
      auto mstore = [&](int l, int a, Cx v) {
        const R qx = (R)(c0 + l) * dqx, qz = (R)((a <= N / 2) ? a : a - N) * dqz;
        const R qz2 = qz * qz, k2 = fmaf(qx, qx, qy2) + qz2;
        const R u = (k2 > (R)0) ? pref * ((R)3 * qz2 / k2 - (R)1) : (R)0;
        sm[a * W + l] = cscale(v, u);
      };
      tile_fft_ct_cols<R, N, EPT, false, W, T>(sm, s_tw, sload, mstore);
      tile_fft_ct_cols<R, N, EPT, true, W, T>(sm, s_tw, sload, sstore);
    } else {
      const size_t base = (size_t)o * A.ostride + c0;
      const long long es = A.estride;
      auto mstore = [&](int l, int a, Cx v) {
        const R u = (c0 + l < A.ncols) ? A.U[base + a * es + l] : (R)0;
        sm[a * W + l] = cscale(v, u);
      };
      tile_fft_ct_cols<R, N, EPT, false, W, T>(sm, s_tw, sload, mstore);
      tile_fft_ct_cols<R, N, EPT, true, W, T>(sm, s_tw, sload, sstore);
    }
    // the transformed tile goes back by tensor-map stores
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
#pragma unroll
      for (int b = 0; b < NBOX; ++b) {
        if (AXIS == 1) tma_store_3d(&tm, c0, b * BOXR, o, sm + b * BOXR * W);
        else tma_store_3d(&tm, c0, o, b * BOXR, sm + b * BOXR * W);
      }
      bulk_commit();
      const int next2 = tile + 2 * gridDim.x;
      if (next2 < ntiles) {
        bulk_wait_read_all();  // the store has read this buffer before it is refilled
        issue(next2, k);
      }
    }
  }
  if (t == 0) bulk_wait_all();
  __syncthreads();
  if (t == 0) { mbar_inval(&bar[0]); mbar_inval(&bar[1]); }
}

// ------------------------------------------------------- P2 / P3 (strided)
// NORM false: a pass without the norm (no |x|^2 code at all); true: the
// runtime flag A.norm decides.
// NC > 0 (line length NC, power-of-two tile width WC): compile-time lengths.
template <typename R, typename Coef, int CL, bool NORM = true, int SCR = 0, int NC = 0, int WC = 0>
__device__ __forceinline__ void cn_strided_body(const CArgs<R> &A, int bx, int by, int gx, int gy) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *tile = reinterpret_cast<cx<R> *>(smraw);  // [W][pitch]
  constexpr bool TAB = (sizeof(R) == 8);
  // shared scratch: red[32], am_last, s_tab (FP32: padded copy of the tables)
  constexpr int OFF_LAST = scr_align(sizeof(double) * 32), OFF_TAB = OFF_LAST + 32;
  constexpr int NEED = OFF_TAB + sizeof(Coef) * (TAB ? 1 : 4 * (512 + 512 / CL + 1));
  static_assert(SCR == 0 || NEED <= SCR, "shared scratch too small");
  unsigned char *scr = shared_scratch<SCR ? SCR : NEED>();
  double *const red = reinterpret_cast<double *>(scr);
  int &am_last = *reinterpret_cast<int *>(scr + OFF_LAST);
  Coef *const s_tab = reinterpret_cast<Coef *>(scr + OFF_TAB);
  const int W = NC ? WC : A.W, n = NC ? NC : A.n, P = NC ? NC + NC / CL + 1 : A.pitch;
  const int lW = NC ? ct_log2(WC) : ilog2(W);
  const int TPL = NC ? NC / CL : A.TPL;
  const int c0 = bx * W;
  const size_t base = (size_t)by * A.ostride + c0;
  const long long es = A.estride;
  // thread t owns column t % W and rows t / W + i TPL, i < CL (blockDim =
  // W TPL, n = CL TPL): all CL loads are in flight before the first
  // shared-memory store
  const int lc = threadIdx.x & (W - 1), r0 = threadIdx.x >> lW;
  {
    const bool ok = c0 + lc < A.ncols;
    cx<R> buf[CL];
#pragma unroll
    for (int i = 0; i < CL; ++i) buf[i] = ok ? A.psi[base + (size_t)(r0 + i * TPL) * es + lc] : czero<cx<R>>();
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int a = r0 + i * TPL;
      tile[lc * P + a + a / CL] = buf[i];
    }
  }
  __syncthreads();
  if (!TAB) {
    stage_cn_tables<Coef, CL>(s_tab, reinterpret_cast<const Coef *>(A.cntab), n);
    __syncthreads();
  }
  const int l = threadIdx.x / TPL, q = threadIdx.x - l * TPL;
  if constexpr (TAB) cn_line<R, Coef, CL>(tile + l * P, n, TPL, q, make_kt<Coef>(A.tau),
                                      reinterpret_cast<const Coef *>(A.cntab), c0 + l < A.ncols);
  else cn_line_st<R, Coef, CL>(tile + l * P, n, TPL, q, make_kt<Coef>(A.tau), s_tab, c0 + l < A.ncols, A.cnd);
  __syncthreads();
  double acc = 0.0;
  if (c0 + lc < A.ncols) {
    R ts = (R)0;  // the thread's CL sites in R, then FP64 above the tile
#pragma unroll
    for (int i = 0; i < CL; ++i) {
      const int a = r0 + i * TPL;
      const cx<R> v = tile[lc * P + a + a / CL];
      A.psi[base + (size_t)a * es + lc] = v;
      if (NORM && A.norm) ts += v.x * v.x + v.y * v.y;
    }
    acc = (double)ts;
  }
  if (!A.final_pass) return;
  // Last pass of the step: norm partials (imaginary time) and, in the last
  // block to finish, the deterministic FP64 total, the new scale and the
  // step counter.
  const unsigned nblk = (unsigned)(gx * gy);
  const unsigned bid = (unsigned)(by * gx + bx);
  if (A.norm) {
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) A.partial[bid] = s;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(A.counter, 1u);
    am_last = (ticket == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (A.norm) {
    double s = 0.0;
    for (unsigned i = threadIdx.x; i < nblk; i += blockDim.x) s += __ldcg(A.partial + i);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
      const double norm = A.prm[PRM_CELL] * s;
      if (norm > 0.0 && isfinite(norm)) A.prm[PRM_SC] = 1.0 / sqrt(norm);
      else A.prm[PRM_NONFINITE] = 1.0;
    }
  }
  if (threadIdx.x == 0) {
    *A.step += 1;
    *A.counter = 0u;
  }
}
template <typename R, typename Coef, int CL, bool NORM = true>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB(R)) k_cn_strided(const __grid_constant__ CArgs<R> A) {
  cn_strided_body<R, Coef, CL, NORM>(A, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}
template <typename R, typename Coef, int CL, bool NORM = true>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB(R)) k_cn_strided_batch(const CArgs<R> *__restrict__ args) {
  __shared__ CArgs<R> sA;
  const CArgs<R> &A = block_args(args, sA);
  cn_strided_body<R, Coef, CL, NORM>(A, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y);
}

// Persistent, double-buffered CN pass: each CTA walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ...; the copies of the next tile into
// the other shared buffer are in flight while the current tile is solved.
// Tile id -> (column block id % nx_blocks, outer index id / nx_blocks).
template <typename R, typename Coef, int CL, bool NORM = true>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB_CN(R)) k_cn_strided_pipe(const __grid_constant__ CArgs<R> A, int ncb, int ntiles) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  __shared__ int am_last;
  const int W = A.W, n = A.n, P = A.pitch;
  const int lW = ilog2(W);
  cx<R> *buf[2] = {reinterpret_cast<cx<R> *>(smraw), reinterpret_cast<cx<R> *>(smraw) + W * P};
  const long long es = A.estride;
  const int lc = threadIdx.x & (W - 1), r0 = threadIdx.x >> lW;
  auto fetch = [&](int tile, cx<R> *tb) {
    const int cb = tile % ncb, o = tile / ncb;
    const int c0 = cb * W;
    if (c0 + lc < A.ncols) {
      const cx<R> *src = A.psi + (size_t)o * A.ostride + c0 + lc;
#pragma unroll
      for (int i = 0; i < CL; ++i) {
        const int a = r0 + i * A.TPL;
        cp_async_elem(tb + lc * P + a + a / CL, src + (size_t)a * es);
      }
    }
    cp_async_commit();
  };
  constexpr bool TAB = (sizeof(R) == 8);
  __shared__ __align__(16) Coef s_tab[TAB ? 1 : 4 * (512 + 512 / CL + 1)];
  if (!TAB) stage_cn_tables<Coef, CL>(s_tab, reinterpret_cast<const Coef *>(A.cntab), n);  // visible after the loop's first barrier
  double acc = 0.0;
  int k = 0;
  if ((int)blockIdx.x < ntiles) fetch(blockIdx.x, buf[0]);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, k ^= 1) {
    const int next = tile + gridDim.x;
    if (next < ntiles) fetch(next, buf[k ^ 1]);
    else cp_async_commit();  // keep one group per iteration
    cp_async_wait<1>();      // this tile's copies are done (the next may be in flight)
    __syncthreads();
    const int cb = tile % ncb, o = tile / ncb;
    const int c0 = cb * W;
    cx<R> *tb = buf[k];
    const int l = threadIdx.x / A.TPL, q = threadIdx.x - l * A.TPL;
    if constexpr (TAB) cn_line<R, Coef, CL>(tb + l * P, n, A.TPL, q, make_kt<Coef>(A.tau),
                                        reinterpret_cast<const Coef *>(A.cntab), c0 + l < A.ncols);
    else cn_line_st<R, Coef, CL>(tb + l * P, n, A.TPL, q, make_kt<Coef>(A.tau), s_tab, c0 + l < A.ncols,
                                 A.cnd);
    __syncthreads();
    if (c0 + lc < A.ncols) {
      cx<R> *dst = A.psi + (size_t)o * A.ostride + c0 + lc;
      // |x|^2 of the thread's CL sites summed in R (FP32: an FP64 sum per
      // site held the FP32 final pass at the FP64 pipe's rate, 0.21 against
      // 0.08 ms at 256^3), then accumulated in FP64 across tiles and blocks
      R ts = (R)0;
#pragma unroll
      for (int i = 0; i < CL; ++i) {
        const int a = r0 + i * A.TPL;
        const cx<R> v = tb[lc * P + a + a / CL];
        dst[(size_t)a * es] = v;
        if (NORM && A.norm) ts += v.x * v.x + v.y * v.y;
      }
      if (NORM && A.norm) acc += (double)ts;
    }
    __syncthreads();  // the buffer is refilled two iterations later
  }
  cp_async_wait<0>();
  if (!A.final_pass) return;
  const unsigned nblk = gridDim.x;
  if (NORM && A.norm) {
    double sblk = block_sum(acc, red);
    if (threadIdx.x == 0) A.partial[blockIdx.x] = sblk;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(A.counter, 1u);
    am_last = (ticket == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (NORM && A.norm) {
    double sum = 0.0;
    for (unsigned i = threadIdx.x; i < nblk; i += blockDim.x) sum += __ldcg(A.partial + i);
    sum = block_sum(sum, red);
    if (threadIdx.x == 0) {
      const double norm = A.prm[PRM_CELL] * sum;
      if (norm > 0.0 && isfinite(norm)) A.prm[PRM_SC] = 1.0 / sqrt(norm);
      else A.prm[PRM_NONFINITE] = 1.0;
    }
  }
  if (threadIdx.x == 0) {
    *A.step += 1;
    *A.counter = 0u;
  }
}

// The same pass with the line length N and tile width W as compile-time
// constants (FP32, power-of-two lengths): every index folds.
template <typename R, typename Coef, int CL, bool NORM, int N, int W>
__global__ void __launch_bounds__(DGPE_MAXT, DGPE_MINB_CN(R)) k_cn_pipe_ct(const __grid_constant__ CArgs<R> A, int ncb, int ntiles) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  __shared__ int am_last;
  constexpr int n = N, TPL = N / CL, P = N + N / CL + 1, lW = ct_log2(W);
  static_assert(W * TPL <= DGPE_MAXT, "block size");
  cx<R> *const buf0 = reinterpret_cast<cx<R> *>(smraw);  // buffer k at buf0 + k W P
  const long long es = A.estride;
  const int lc = threadIdx.x & (W - 1), r0 = threadIdx.x >> lW;
  auto fetch = [&](int tile, cx<R> *tb) {
    const int cb = tile % ncb, o = tile / ncb;
    const int c0 = cb * W;
    if (c0 + lc < A.ncols) {
      const cx<R> *src = A.psi + (size_t)o * A.ostride + c0 + lc;
#pragma unroll
      for (int i = 0; i < CL; ++i) {
        const int a = r0 + i * TPL;
        cp_async_elem(tb + lc * P + a + a / CL, src + (size_t)a * es);
      }
    }
    cp_async_commit();
  };
  constexpr bool TAB = (sizeof(R) == 8);
  __shared__ __align__(16) Coef s_tab[TAB ? 1 : 4 * P];
  if (!TAB) stage_cn_tables<Coef, CL>(s_tab, reinterpret_cast<const Coef *>(A.cntab), n);  // visible after the loop's first barrier
  double acc = 0.0;
  int k = 0;
  if ((int)blockIdx.x < ntiles) fetch(blockIdx.x, buf0);
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, k ^= 1) {
    const int next = tile + gridDim.x;
    if (next < ntiles) fetch(next, buf0 + (k ^ 1) * W * P);
    else cp_async_commit();  // keep one group per iteration
    cp_async_wait<1>();      // this tile's copies are done (the next may be in flight)
    __syncthreads();
    const int cb = tile % ncb, o = tile / ncb;
    const int c0 = cb * W;
    cx<R> *tb = buf0 + k * W * P;
    const int l = threadIdx.x / TPL, q = threadIdx.x - l * TPL;
    if constexpr (TAB) cn_line<R, Coef, CL>(tb + l * P, n, TPL, q, make_kt<Coef>(A.tau),
                                        reinterpret_cast<const Coef *>(A.cntab), c0 + l < A.ncols);
    else cn_line_st<R, Coef, CL>(tb + l * P, n, TPL, q, make_kt<Coef>(A.tau), s_tab, c0 + l < A.ncols, A.cnd);
    __syncthreads();
    if (c0 + lc < A.ncols) {
      cx<R> *dst = A.psi + (size_t)o * A.ostride + c0 + lc;
      // |x|^2 of the thread's CL sites summed in R (FP32: an FP64 sum per
      // site held the FP32 final pass at the FP64 pipe's rate, 0.21 against
      // 0.08 ms at 256^3), then accumulated in FP64 across tiles and blocks
      R ts = (R)0;
#pragma unroll
      for (int i = 0; i < CL; ++i) {
        const int a = r0 + i * TPL;
        const cx<R> v = tb[lc * P + a + a / CL];
        dst[(size_t)a * es] = v;
        if (NORM && A.norm) ts += v.x * v.x + v.y * v.y;
      }
      if (NORM && A.norm) acc += (double)ts;
    }
    __syncthreads();  // the buffer is refilled two iterations later
  }
  cp_async_wait<0>();
  if (!A.final_pass) return;
  const unsigned nblk = gridDim.x;
  if (NORM && A.norm) {
    double sblk = block_sum(acc, red);
    if (threadIdx.x == 0) A.partial[blockIdx.x] = sblk;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(A.counter, 1u);
    am_last = (ticket == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (NORM && A.norm) {
    double sum = 0.0;
    for (unsigned i = threadIdx.x; i < nblk; i += blockDim.x) sum += __ldcg(A.partial + i);
    sum = block_sum(sum, red);
    if (threadIdx.x == 0) {
      const double norm = A.prm[PRM_CELL] * sum;
      if (norm > 0.0 && isfinite(norm)) A.prm[PRM_SC] = 1.0 / sqrt(norm);
      else A.prm[PRM_NONFINITE] = 1.0;
    }
  }
  if (threadIdx.x == 0) {
    *A.step += 1;
    *A.counter = 0u;
  }
}

// ------------------------------------------ line-serial Crank-Nicolson
// One thread per grid line, streaming the line through registers: the Thomas
// elimination of the CN system A x = B psi of Sec. 2 (A = I + kt T, Dirichlet
// ghosts), with the right-hand side formed on the fly,
//   d_a  = psi_a + kt (psi_{a-1} - 2 psi_a + psi_{a+1}),
// and run from both ends of the line at once.  A has constant coefficients
// and is persymmetric, so eliminating upwards from the last row has the same
// pivots m_j = 1 / (1 + 2 kt - kt^2 m_{j-1}) counted from the end:
//   top    (a = j = 0 .. k-1):      d'_a = m_j (d_a + kt d'_{a-1}),
//   bottom (b = n-1-j, j < k-1):    e'_b = m_j (d_b + kt e'_{b+1}),
//   middle row k = n/2:             x_k = mu (d_k + kt (d'_{k-1} + e'_{k+1})),
//                                   mu = 1 / (1 + 2 kt - kt (alpha_{k-1} + alpha_{k-2})),
//   back substitution outwards:     x_a = d'_a + alpha_j x_{a+1},  x_b = e'_b + alpha_j x_{b-1},
// alpha_j = kt m_j.  The two halves are independent recurrences, which
// doubles the arithmetic each thread has in flight (the FP64 pipe's latency,
// not its throughput, limits a one-chain sweep at these occupancies), at the
// operation count of the plain sweep: about half that of the chunk-parallel
// solve.  d' and e' are written over psi and read back by the same thread.
// Neighbouring threads own neighbouring lines, so a y or z sweep reads and
// writes one coalesced segment per warp and step; an x sweep walks rows (each
// row's 128-byte line stays in L1 for the next steps).  Loads run LS_K sites
// ahead of the stores, from registers.  tab holds m (n values), alpha (n),
// two chunk tables (2n, unused here) and mu.
struct LArgs {
  void *psi;
  const void *tab;
  double *prm;
  double *partial;
  unsigned *counter;
  long long *step;
  long long es;  // element stride along a line
  long long cs;  // stride between neighbouring lines
  long long os;  // stride of the outer index (blockIdx.y)
  int n, ncols, final_pass, norm;
  double tau;
};
#define DGPE_LS_K 4
#ifndef DGPE_LINES_T
#define DGPE_LINES_T 64  // threads (lines) per block: 65536 lines make ~7 blocks per SM, an even single wave
#endif

__device__ __forceinline__ double fma_r(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
// Products with kt = tau (imaginary time, real Coef) or kt = i tau (real
// time), written as FMAs:  fma: kt v + w;  rhs: (1 - 2 kt) c + kt s, the
// Crank-Nicolson right-hand side B psi at a site with value c and neighbour
// sum s;  cfma: a v + w for a table coefficient a.
template <typename R, typename Coef> struct KtMul;
template <typename R> struct KtMul<R, R> {
  static __device__ __forceinline__ cx<R> fma(R tau, cx<R> v, cx<R> w) {
    return mk<R>(fma_r(tau, v.x, w.x), fma_r(tau, v.y, w.y));
  }
  static __device__ __forceinline__ cx<R> rhs(R tau, R one_m2tau, cx<R> c, cx<R> s) {
    return mk<R>(fma_r(tau, s.x, one_m2tau * c.x), fma_r(tau, s.y, one_m2tau * c.y));
  }
  static __device__ __forceinline__ cx<R> cfma(R a, cx<R> v, cx<R> w) {
    return mk<R>(fma_r(a, v.x, w.x), fma_r(a, v.y, w.y));
  }
};
template <typename R> struct KtMul<R, cx<R>> {
  static __device__ __forceinline__ cx<R> fma(R tau, cx<R> v, cx<R> w) {
    return mk<R>(fma_r(-tau, v.y, w.x), fma_r(tau, v.x, w.y));
  }
  // c + i tau (s - 2 c); t2 = 2 tau
  static __device__ __forceinline__ cx<R> rhs(R tau, R t2, cx<R> c, cx<R> s) {
    return mk<R>(fma_r(-tau, s.y, fma_r(t2, c.y, c.x)), fma_r(tau, s.x, fma_r(-t2, c.x, c.y)));
  }
  static __device__ __forceinline__ cx<R> cfma(cx<R> a, cx<R> v, cx<R> w) {
    return mk<R>(fma_r(a.x, v.x, fma_r(-a.y, v.y, w.x)), fma_r(a.x, v.y, fma_r(a.y, v.x, w.y)));
  }
};

// NORM: accumulate the FP64 norm (the final pass of an imaginary-time step);
// a template flag so that the real-time passes carry no norm arithmetic.
template <typename R, typename Coef, bool NORM>
__global__ void __launch_bounds__(128) k_cn_lines(const __grid_constant__ LArgs A) {
  __shared__ double red[32];
  __shared__ int am_last;
  typedef cx<R> Cx;
  typedef KtMul<R, Coef> KT;
  constexpr int K = DGPE_LS_K;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = A.n, k = n / 2;
  const long long es = A.es;
  // second constant of KT::rhs: 1 - 2 tau (real kt) or 2 tau (imaginary kt)
  const R tau = (R)A.tau;
  const R one_m2tau = (sizeof(Coef) == sizeof(R)) ? (R)(1.0 - 2.0 * A.tau) : (R)(2.0 * A.tau);
  const Coef *tm = reinterpret_cast<const Coef *>(A.tab), *ta = tm + n;
  double acc = 0.0;
  if (c < A.ncols) {
    Cx *p = reinterpret_cast<Cx *>(A.psi) + (size_t)blockIdx.y * A.os + (size_t)c * A.cs;
    auto ld = [&](int a) { return p[(size_t)a * es]; };
    auto nrm = [&](Cx v) {
      if constexpr (NORM) acc += (double)v.x * v.x + (double)v.y * v.y;
    };
    // forward elimination from both ends; for step j:
    //   top row j, bt[i] = psi_{j+1};  bottom row n-1-j, bb[i] = psi_{n-2-j}
    Cx bt[K], bb[K], nt[K], nb[K];
    Cx prt = czero<Cx>(), cut = ld(0), dpt = czero<Cx>();
    Cx prb = czero<Cx>(), cub = ld(n - 1), dpb = czero<Cx>();
#pragma unroll
    for (int i = 0; i < K; ++i) {
      bt[i] = (1 + i <= k) ? ld(1 + i) : czero<Cx>();
      bb[i] = (n - 2 - i >= k) ? ld(n - 2 - i) : czero<Cx>();
    }
    for (int j0 = 0; j0 < k; j0 += K) {
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int jt = j0 + K + 1 + i, jb = n - 2 - (j0 + K + i);
        nt[i] = (jt <= k) ? ld(jt) : czero<Cx>();
        nb[i] = (jb >= k) ? ld(jb) : czero<Cx>();
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int j = j0 + i;
        if (j < k) {
          const Coef mj = __ldg(tm + j);
          {
            const Cx nxt = bt[i];
            const Cx d = KT::rhs(tau, one_m2tau, cut, prt + nxt);
            dpt = coef_mul(mj, KT::fma(tau, dpt, d));
            p[(size_t)j * es] = dpt;
            prt = cut;
            cut = nxt;
          }
          if (j < k - 1) {
            const Cx nxt = bb[i];
            const Cx d = KT::rhs(tau, one_m2tau, cub, prb + nxt);
            dpb = coef_mul(mj, KT::fma(tau, dpb, d));
            p[(size_t)(n - 1 - j) * es] = dpb;
            prb = cub;
            cub = nxt;
          }
        }
      }
#pragma unroll
      for (int i = 0; i < K; ++i) { bt[i] = nt[i]; bb[i] = nb[i]; }
    }
    // middle row: cut = psi_k, prt = psi_{k-1}, prb = psi_{k+1}
    const Cx dk = KT::rhs(tau, one_m2tau, cut, prt + prb);
    const Cx xk = coef_mul(__ldg(tm + 4 * n), KT::fma(tau, dpt + dpb, dk));
    p[(size_t)k * es] = xk;
    nrm(xk);
    // back substitution outwards; for step j (from k-1 down):
    //   top row j, bt[i] = d'_j;  bottom row n-1-j (j <= k-2), bb[i] = e'_{n-1-j}
    Cx xt = xk, xb = xk;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const int j = k - 1 - i;
      bt[i] = (j >= 0) ? ld(j) : czero<Cx>();
      bb[i] = (j >= 0 && j <= k - 2) ? ld(n - 1 - j) : czero<Cx>();
    }
    for (int j0 = k - 1; j0 >= 0; j0 -= K) {
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int j = j0 - K - i;
        nt[i] = (j >= 0) ? ld(j) : czero<Cx>();
        nb[i] = (j >= 0 && j <= k - 2) ? ld(n - 1 - j) : czero<Cx>();
      }
#pragma unroll
      for (int i = 0; i < K; ++i) {
        const int j = j0 - i;
        if (j >= 0) {
          const Coef aj = __ldg(ta + j);
          xt = KT::cfma(aj, xt, bt[i]);
          p[(size_t)j * es] = xt;
          nrm(xt);
          if (j <= k - 2) {
            xb = KT::cfma(aj, xb, bb[i]);
            p[(size_t)(n - 1 - j) * es] = xb;
            nrm(xb);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < K; ++i) { bt[i] = nt[i]; bb[i] = nb[i]; }
    }
  }
  if (!A.final_pass) return;
  const int t = threadIdx.x, T = blockDim.x;
  const unsigned nblk = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
  if (NORM) {
    const double sblk = block_sum(acc, red);
    if (t == 0) A.partial[bid] = sblk;
  }
  if (t == 0) {
    __threadfence();
    const unsigned ticket = atomicAdd(A.counter, 1u);
    am_last = (ticket == nblk - 1);
  }
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  if (NORM) {
    double sum = 0.0;
    for (unsigned i = t; i < nblk; i += T) sum += __ldcg(A.partial + i);
    sum = block_sum(sum, red);
    if (t == 0) {
      const double norm = A.prm[PRM_CELL] * sum;
      if (norm > 0.0 && isfinite(norm)) A.prm[PRM_SC] = 1.0 / sqrt(norm);
      else A.prm[PRM_NONFINITE] = 1.0;
    }
  }
  if (t == 0) {
    *A.step += 1;
    *A.counter = 0u;
  }
}

// ------------------------------------------------------------ observables
// Per-block FP64 partial sums over whole x-rows:
//  0 n  1 x^2 n  2 y^2 n  3 z^2 n  4 V0 n  5 n^2  6 Kx  7 Ky  8 Kz  9 non-finite
enum { OBS_N, OBS_X2, OBS_Y2, OBS_Z2, OBS_V, OBS_N2, OBS_KX, OBS_KY, OBS_KZ, OBS_BAD, OBS_COUNT };

template <typename R>
__global__ void k_obs_sites(const __grid_constant__ OArgs<R> A) {
  __shared__ double red[32];
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const size_t N = (size_t)nx * ny * nz;
  const double sc = A.prm[PRM_SC];
  double acc[OBS_COUNT];
#pragma unroll
  for (int k = 0; k < OBS_COUNT; ++k) acc[k] = 0.0;
  const int nxh = nx / 2, nyh = ny / 2, nzh = nz / 2;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const size_t r = i / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const cx<R> v0 = A.psi[i];
    const cx<R> wx = (x + 1 < nx) ? A.psi[i + 1] : czero<cx<R>>();
    const cx<R> wy = (y + 1 < ny) ? A.psi[i + nx] : czero<cx<R>>();
    const cx<R> wz = (A.dim == 3 && z + 1 < nz) ? A.psi[i + (size_t)nx * ny] : czero<cx<R>>();
    const double vr = sc * (double)v0.x, vi = sc * (double)v0.y;
    const double nn = vr * vr + vi * vi;
    if (!isfinite(nn)) { acc[OBS_BAD] += 1.0; continue; }
    const double X = (double)(x - nxh) * A.hx, Y = (double)(y - nyh) * A.hy;
    const double Z = (A.dim == 3) ? (double)(z - nzh) * A.hz : 0.0;
    acc[OBS_N] += nn;
    acc[OBS_X2] += X * X * nn;
    acc[OBS_Y2] += Y * Y * nn;
    acc[OBS_Z2] += Z * Z * nn;
    acc[OBS_V] += 0.5 * (A.nux * A.nux * X * X + A.nuy * A.nuy * Y * Y + A.nuz * A.nuz * Z * Z) * nn;
    acc[OBS_N2] += nn * nn;
    // forward differences with zero ghosts; the (ghost, first) pair adds |psi_0|^2
    double dr = sc * (double)wx.x - vr, di = sc * (double)wx.y - vi;
    acc[OBS_KX] += dr * dr + di * di + (x == 0 ? nn : 0.0);
    dr = sc * (double)wy.x - vr; di = sc * (double)wy.y - vi;
    acc[OBS_KY] += dr * dr + di * di + (y == 0 ? nn : 0.0);
    if (A.dim == 3) {
      dr = sc * (double)wz.x - vr; di = sc * (double)wz.y - vi;
      acc[OBS_KZ] += dr * dr + di * di + (z == 0 ? nn : 0.0);
    }
  }
#pragma unroll
  for (int k = 0; k < OBS_COUNT; ++k) {
    const double s = block_sum(acc[k], red);
    if (threadIdx.x == 0) A.partial[(size_t)blockIdx.x * OBS_COUNT + k] = s;
  }
}

// Second stage: fixed-order totals of the site partials and the spectral
// partials (one block).
static __global__ void k_obs_final(const double *site_partial, int nsite_blocks,
                            const double *dip_partial, int ndip, double *out) {
  __shared__ double red[32];
  for (int k = 0; k < OBS_COUNT; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nsite_blocks; i += blockDim.x) s += site_partial[(size_t)i * OBS_COUNT + k];
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[k] = s;
    __syncthreads();
  }
  double s = 0.0;
  for (int i = threadIdx.x; i < ndip; i += blockDim.x) s += dip_partial[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[OBS_COUNT] = s;
}

// ------------------------------------------------------------- adjoint
// Reverse step of one real-time step psi' = C e^{-i theta} psi (G = 2 dL/dpsi*):
//   sig = Im(conj(G_phi) phi), phi = e^{-i theta} psi_in, G_phi = C^dagger G';
//   G = e^{+i theta} G_phi + 2 dt (g sig + g_dd K*sig) psi_in;
//   dL/dg += dt sum sig n,  dL/dc_m += dt sin(m t) sum sig V0.
template <typename R> struct AArgs {
  const cx<R> *psi_in;
  cx<R> *G;
  const R *phi, *sig, *ksig;
  R *sig_out;
  const R *vx, *vy, *vz;
  double *partial;  // [block][2]: sum sig n, sum sig V0
  int nx, ny, dim;
  size_t n;
  double dts, gdt, gdddt, two_dt_g, two_dt_gdd;
};

template <typename R> __device__ __forceinline__ R adj_theta(const AArgs<R> &A, size_t i, cx<R> v, R *dens, R *v0) {
  const int x = (int)(i % A.nx);
  const size_t r = i / A.nx;
  const int y = (int)(r % A.ny), z = (int)(r / A.ny);
  *dens = v.x * v.x + v.y * v.y;
  *v0 = A.vx[x] + A.vy[y] + A.vz[z];
  return (R)A.dts * *v0 + (R)A.gdt * *dens + (R)A.gdddt * A.phi[i];
}

template <typename R>
__global__ void k_adj_sigma(const __grid_constant__ AArgs<R> A) {
  __shared__ double red[32];
  double sn = 0.0, sv = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < A.n; i += (size_t)gridDim.x * blockDim.x) {
    const cx<R> v = A.psi_in[i];
    R dens, v0;
    const R th = adj_theta(A, i, v, &dens, &v0);
    R s, c;
    fsincos(th, &s, &c);
    const cx<R> ph = mk<R>(v.x * c + v.y * s, v.y * c - v.x * s);  // e^{-i th} psi
    const cx<R> g = A.G[i];
    const R sig = g.x * ph.y - g.y * ph.x;  // Im(conj(g) ph)
    A.sig_out[i] = sig;
    sn += (double)sig * dens;
    sv += (double)sig * v0;
  }
  sn = block_sum(sn, red);
  if (threadIdx.x == 0) A.partial[2 * blockIdx.x] = sn;
  sv = block_sum(sv, red);
  if (threadIdx.x == 0) A.partial[2 * blockIdx.x + 1] = sv;
}

template <typename R>
__global__ void k_adj_update(const __grid_constant__ AArgs<R> A) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < A.n; i += (size_t)gridDim.x * blockDim.x) {
    const cx<R> v = A.psi_in[i];
    R dens, v0;
    const R th = adj_theta(A, i, v, &dens, &v0);
    R s, c;
    fsincos(th, &s, &c);
    const cx<R> g = A.G[i];
    const R f = (R)A.two_dt_g * A.sig[i] + (R)A.two_dt_gdd * A.ksig[i];
    // e^{+i th} G_phi + f psi_in
    A.G[i] = mk<R>(g.x * c - g.y * s + f * v.x, g.y * c + g.x * s + f * v.y);
  }
}

// Fixed-order totals of the per-block partials, accumulated in FP64:
// acc[0] += dt S_n,  acc[1 + m - 1] += dt sin(m t) S_V.
static __global__ void k_adj_accumulate(const double *partial, int nblk, double *acc, double dt, double t, int M) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) { a += partial[2 * i]; b += partial[2 * i + 1]; }
  a = block_sum(a, red);
  b = block_sum(b, red);
  if (threadIdx.x == 0) {
    acc[0] += dt * a;
    for (int m = 1; m <= M; ++m) acc[m] += dt * sin((double)m * t) * b;
  }
}

// partial[block] = sum conj(a) b (complex, FP64)
template <typename R>
__global__ void k_cdot(const cx<R> *a, const cx<R> *b, size_t n, double *partial) {
  __shared__ double red[32];
  double re = 0.0, im = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cx<R> u = a[i], v = b[i];
    re += (double)u.x * v.x + (double)u.y * v.y;
    im += (double)u.x * v.y - (double)u.y * v.x;
  }
  re = block_sum(re, red);
  if (threadIdx.x == 0) partial[2 * blockIdx.x] = re;
  im = block_sum(im, red);
  if (threadIdx.x == 0) partial[2 * blockIdx.x + 1] = im;
}

// out = (cr + i ci) * in
template <typename R>
__global__ void k_cscale(cx<R> *out, const cx<R> *in, double cr, double ci, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const cx<R> v = in[i];
    out[i] = mk<R>((R)(cr * v.x - ci * v.y), (R)(cr * v.y + ci * v.x));
  }
}

// --------------------------------------------------------- state transfer
// dst (stored precision) <- src (complex128 or complex64), and back with the
// lazy scale folded in.
template <typename R, typename S>
__global__ void k_import(cx<R> *dst, const S *src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    S v = src[i];
    dst[i] = mk<R>((R)v.x, (R)v.y);
  }
}
template <typename R, typename S>
__global__ void k_export(S *dst, const cx<R> *src, const double *prm, size_t n) {
  const double sc = prm[PRM_SC];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    cx<R> v = src[i];
    S o;
    o.x = (decltype(o.x))(sc * (double)v.x);
    o.y = (decltype(o.y))(sc * (double)v.y);
    dst[i] = o;
  }
}
// real state (imaginary time): import the real part; export (sc psi, 0)
template <typename R, typename S>
__global__ void k_import_real(R *dst, const S *src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = (R)src[i].x;
}
template <typename R, typename S>
__global__ void k_export_real(S *dst, const R *src, const double *prm, size_t n) {
  const double sc = prm[PRM_SC];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    S o;
    o.x = (decltype(o.x))(sc * (double)src[i]);
    o.y = (decltype(o.y))0;
    dst[i] = o;
  }
}
// real state -> complex (v, 0), unscaled (the observables' input)
template <typename R>
__global__ void k_widen_real(cx<R> *dst, const R *src, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = mk<R>(src[i], (R)0);
}
template <typename R>
__global__ void k_fold_scale(cx<R> *psi, double *prm, size_t n) {
  const R sc = (R)prm[PRM_SC];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    psi[i] = cscale(psi[i], sc);
}

}  // namespace
}  // namespace dgpe
