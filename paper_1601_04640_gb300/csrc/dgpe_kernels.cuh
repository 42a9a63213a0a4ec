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

#include "dgpe_device.cuh"

namespace dgpe {

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
  PRM_COUNT = 24
};

template <typename R> struct XArgs {  // x-line passes
  cx<R> *psi;
  cx<R> *spec;
  R *phi_out;
  const double *prm;
  const long long *step;
  const cx<R> *tw;
  const R *vx, *vy, *vz;
  const void *cntab;
  FftPlan pl;
  int nx, ny, nrows, px, LP;
  int pitchz, pitch, TPL, C;
  int imag, has_dip;
  double tau;
};

template <typename R> struct SArgs {  // strided FFT passes over the spectrum
  cx<R> *spec;
  const R *U;
  double *partial;
  const cx<R> *tw;
  FftPlan pl;
  long long estride, ostride;
  int n, ncols, W, nxh;
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

// psi <- psi exp(-kappa theta) in increment form (psi + psi (e - 1)) so that
// rounding of the factor scales with theta, not with psi.
template <typename R> __device__ __forceinline__ cx<R> nonlinear_factor(cx<R> v, R th, int imag) {
  if (imag) {
    R f = fexpm1(-th);
    return mk<R>(v.x + v.x * f, v.y + v.y * f);
  }
  R s, c;
  fsincos(th * (R)0.5, &s, &c);
  const R cm1 = (R)-2 * s * s;   // cos th - 1
  const R sn = (R)2 * s * c;     // sin th
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
template <typename R, int EPT>
__global__ void k_dens_r2c_x(XArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *zt = reinterpret_cast<cx<R> *>(smraw);
  const int n = A.nx, SL = A.pitchz, nrows = A.nrows;
  const int p0 = blockIdx.x * A.LP;
  const R sc = (R)A.prm[PRM_SC];
  const R sc2 = sc * sc;
  const cx<R> *__restrict__ psi = A.psi;
  auto load = [&](int l, int a) -> cx<R> {
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    R d0 = 0, d1 = 0;
    if (r0 < nrows) { cx<R> v = psi[(size_t)r0 * n + a]; d0 = sc2 * (v.x * v.x + v.y * v.y); }
    if (r1 < nrows) { cx<R> v = psi[(size_t)r1 * n + a]; d1 = sc2 * (v.x * v.x + v.y * v.y); }
    return mk<R>(d0, d1);
  };
  auto store = [&](int l, int a, cx<R> v) { zt[l * SL + a] = v; };
  tile_fft<R, EPT, false, false>(zt, SL, 1, A.LP, A.pl, A.tw, load, store);
  // two real lines were packed as Z = n0 + i n1: X0 = (Z_k + conj Z_{n-k}) / 2,
  // X1 = (Z_k - conj Z_{n-k}) / (2i), k = 0..n/2
  const int nh = n / 2 + 1;
  for (int idx = threadIdx.x; idx < A.LP * nh; idx += blockDim.x) {
    const int l = idx / nh, k = idx - l * nh;
    const int r0 = 2 * (p0 + l), r1 = r0 + 1;
    if (r0 >= nrows) continue;
    const cx<R> Zk = zt[l * SL + k], Zm = zt[l * SL + (k == 0 ? 0 : n - k)];
    const cx<R> X0 = mk<R>((R)0.5 * (Zk.x + Zm.x), (R)0.5 * (Zk.y - Zm.y));
    const cx<R> X1 = mk<R>((R)0.5 * (Zk.y + Zm.y), (R)0.5 * (Zm.x - Zk.x));
    A.spec[(size_t)r0 * A.px + k] = X0;
    if (r1 < nrows) A.spec[(size_t)r1 * A.px + k] = X1;
  }
}

// ------------------------------------------------------------------ P1
// MODE 0: full substep (C2R_x, exponential, CN_x).  MODE 1: write Phi_d only.
template <typename R, typename Coef, int EPT, int CMAX, int MODE>
__global__ void k_c2r_x_exp_cnx(XArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *pt = reinterpret_cast<cx<R> *>(smraw);  // psi tile, 2 LP lines
  cx<R> *zt = pt;  // the Z tile aliases it until the last FFT stage's barrier
  __shared__ double s_dts;
  if (threadIdx.x == 0) s_dts = trap_dts(A.prm, *A.step);
  __syncthreads();
  const int n = A.nx, nh = n / 2, nrows = A.nrows, P = A.pitch, C = A.C;
  const int p0 = blockIdx.x * A.LP;
  const R dts = (R)s_dts;
  const R gdt = (R)(A.prm[PRM_DT] * A.prm[PRM_G]);
  const R gdddt = (R)(A.prm[PRM_DT] * A.prm[PRM_GDD]);
  const R sc = (R)A.prm[PRM_SC];
  const int imag = A.imag;
  const cx<R> *__restrict__ psi = A.psi;
  auto apply_e = [&](int row, int a, R phi) -> cx<R> {
    cx<R> v = psi[(size_t)row * n + a];
    v = cscale(v, sc);
    const R dens = v.x * v.x + v.y * v.y;
    const int y = row % A.ny, z = row / A.ny;
    const R V = A.vx[a] + A.vy[y] + A.vz[z];
    const R th = dts * V + gdt * dens + gdddt * phi;
    return nonlinear_factor<R>(v, th, imag);
  };
  if (A.has_dip) {
    auto load = [&](int l, int a) -> cx<R> {
      const int r0 = 2 * (p0 + l), r1 = r0 + 1;
      const int k = (a <= nh) ? a : n - a;
      cx<R> X0 = czero<cx<R>>(), X1 = czero<cx<R>>();
      if (r0 < nrows) X0 = A.spec[(size_t)r0 * A.px + k];
      if (r1 < nrows) X1 = A.spec[(size_t)r1 * A.px + k];
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
      const int ia = a + a / C;
      pt[(2 * l) * P + ia] = (r0 < nrows) ? apply_e(r0, a, v.x) : czero<cx<R>>();
      pt[(2 * l + 1) * P + ia] = (r1 < nrows) ? apply_e(r1, a, v.y) : czero<cx<R>>();
    };
    tile_fft<R, EPT, true, false>(zt, A.pitchz, 1, A.LP, A.pl, A.tw, load, store);
  } else {
    for (int idx = threadIdx.x; idx < 2 * A.LP * n; idx += blockDim.x) {
      const int L = idx / n, a = idx - L * n;
      const int row = 2 * p0 + L;
      pt[L * P + a + a / C] = (row < nrows) ? apply_e(row, a, (R)0) : czero<cx<R>>();
    }
    __syncthreads();
  }
  if (MODE == 1) return;
  // Crank-Nicolson along x: TPL lanes per line
  const int l = threadIdx.x / A.TPL, q = threadIdx.x - l * A.TPL;
  const bool active = (2 * p0 + l) < nrows;
  cn_line<R, Coef, CMAX>(pt + l * P, n, C, A.TPL, q, make_kt<Coef>(A.tau),
                         reinterpret_cast<const Coef *>(A.cntab), active);
  __syncthreads();
  for (int idx = threadIdx.x; idx < 2 * A.LP * n; idx += blockDim.x) {
    const int L = idx / n, a = idx - L * n;
    const int row = 2 * p0 + L;
    if (row < nrows) A.psi[(size_t)row * n + a] = pt[L * P + a + a / C];
  }
}

// ------------------------------------------------- P5 / P6 / P7 (strided)
// MODE 0 forward, 1 inverse, 2 forward . U . inverse, 3 forward and
// accumulate sum_k w_k U_k |F_k|^2 (FP64) for the dipolar energy.
template <typename R, int EPT, int MODE>
__global__ void k_fft_strided(SArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *sm = reinterpret_cast<cx<R> *>(smraw);  // [a][W]
  __shared__ double red[32];
  const int W = A.W;
  const int c0 = blockIdx.x * W;
  const size_t base = (size_t)blockIdx.y * A.ostride + c0;
  const long long es = A.estride;
  cx<R> *__restrict__ spec = A.spec;
  auto gload = [&](int l, int a) -> cx<R> {
    return (c0 + l < A.ncols) ? spec[base + a * es + l] : czero<cx<R>>();
  };
  auto gstore = [&](int l, int a, cx<R> v) {
    if (c0 + l < A.ncols) spec[base + a * es + l] = v;
  };
  if (MODE == 0) {
    tile_fft<R, EPT, false, true>(sm, 1, W, W, A.pl, A.tw, gload, gstore);
  } else if (MODE == 1) {
    tile_fft<R, EPT, true, true>(sm, 1, W, W, A.pl, A.tw, gload, gstore);
  } else if (MODE == 2) {
    auto mstore = [&](int l, int a, cx<R> v) {
      const R u = (c0 + l < A.ncols) ? A.U[base + a * es + l] : (R)0;
      sm[a * W + l] = cscale(v, u);
    };
    tile_fft<R, EPT, false, true>(sm, 1, W, W, A.pl, A.tw, gload, mstore);
    auto sload = [&](int l, int a) -> cx<R> { return sm[a * W + l]; };
    tile_fft<R, EPT, true, true>(sm, 1, W, W, A.pl, A.tw, sload, gstore);
  } else {
    double acc = 0.0;
    auto astore = [&](int l, int a, cx<R> v) {
      const int kx = c0 + l;
      if (kx < A.ncols) {
        const double w = (kx == 0 || kx == A.nxh) ? 1.0 : 2.0;
        acc += w * (double)A.U[base + a * es + l] * ((double)v.x * v.x + (double)v.y * v.y);
      }
    };
    tile_fft<R, EPT, false, true>(sm, 1, W, W, A.pl, A.tw, gload, astore);
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) A.partial[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// ------------------------------------------------------- P2 / P3 (strided)
template <typename R, typename Coef, int CMAX>
__global__ void k_cn_strided(CArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smraw[];
  cx<R> *tile = reinterpret_cast<cx<R> *>(smraw);  // [W][pitch]
  __shared__ double red[32];
  __shared__ int am_last;
  const int W = A.W, n = A.n, C = A.C, P = A.pitch;
  const int c0 = blockIdx.x * W;
  const size_t base = (size_t)blockIdx.y * A.ostride + c0;
  const long long es = A.estride;
  for (int idx = threadIdx.x; idx < n * W; idx += blockDim.x) {
    const int a = idx / W, l = idx - a * W;
    tile[l * P + a + a / C] = (c0 + l < A.ncols) ? A.psi[base + a * es + l] : czero<cx<R>>();
  }
  __syncthreads();
  const int l = threadIdx.x / A.TPL, q = threadIdx.x - l * A.TPL;
  cn_line<R, Coef, CMAX>(tile + l * P, n, C, A.TPL, q, make_kt<Coef>(A.tau),
                         reinterpret_cast<const Coef *>(A.cntab), c0 + l < A.ncols);
  __syncthreads();
  double acc = 0.0;
  for (int idx = threadIdx.x; idx < n * W; idx += blockDim.x) {
    const int a = idx / W, l2 = idx - a * W;
    if (c0 + l2 < A.ncols) {
      const cx<R> v = tile[l2 * P + a + a / C];
      A.psi[base + a * es + l2] = v;
      if (A.norm) acc += (double)v.x * v.x + (double)v.y * v.y;
    }
  }
  if (!A.final_pass) return;
  // Last pass of the step: norm partials (imaginary time) and, in the last
  // block to finish, the deterministic FP64 total, the new scale and the
  // step counter.
  const unsigned nblk = gridDim.x * gridDim.y;
  const unsigned bid = blockIdx.y * gridDim.x + blockIdx.x;
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

// ------------------------------------------------------------ observables
// Per-block FP64 partial sums over whole x-rows:
//  0 n  1 x^2 n  2 y^2 n  3 z^2 n  4 V0 n  5 n^2  6 Kx  7 Ky  8 Kz  9 non-finite
enum { OBS_N, OBS_X2, OBS_Y2, OBS_Z2, OBS_V, OBS_N2, OBS_KX, OBS_KY, OBS_KZ, OBS_BAD, OBS_COUNT };

template <typename R>
__global__ void k_obs_sites(OArgs<R> A) {
  __shared__ double red[32];
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int nrows = ny * nz;
  const double sc = A.prm[PRM_SC];
  double acc[OBS_COUNT];
#pragma unroll
  for (int k = 0; k < OBS_COUNT; ++k) acc[k] = 0.0;
  const int r_begin = blockIdx.x * A.rows_per_block;
  const int r_end = min(nrows, r_begin + A.rows_per_block);
  const int nxh = nx / 2, nyh = ny / 2, nzh = nz / 2;
  for (int r = r_begin; r < r_end; ++r) {
    const int y = r % ny, z = r / ny;
    const double Y = (double)(y - nyh) * A.hy, Z = (A.dim == 3) ? (double)(z - nzh) * A.hz : 0.0;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      const size_t i = (size_t)r * nx + x;
      const cx<R> v0 = A.psi[i];
      const double vr = sc * (double)v0.x, vi = sc * (double)v0.y;
      const double nn = vr * vr + vi * vi;
      if (!isfinite(nn)) { acc[OBS_BAD] += 1.0; continue; }
      const double X = (double)(x - nxh) * A.hx;
      acc[OBS_N] += nn;
      acc[OBS_X2] += X * X * nn;
      acc[OBS_Y2] += Y * Y * nn;
      acc[OBS_Z2] += Z * Z * nn;
      acc[OBS_V] += 0.5 * (A.nux * A.nux * X * X + A.nuy * A.nuy * Y * Y + A.nuz * A.nuz * Z * Z) * nn;
      acc[OBS_N2] += nn * nn;
      double dr, di;
      // forward differences with zero ghosts; the (ghost, first) pair adds |psi_0|^2
      if (x + 1 < nx) { const cx<R> w = A.psi[i + 1]; dr = sc * (double)w.x - vr; di = sc * (double)w.y - vi; }
      else { dr = -vr; di = -vi; }
      acc[OBS_KX] += dr * dr + di * di + (x == 0 ? nn : 0.0);
      if (y + 1 < ny) { const cx<R> w = A.psi[i + nx]; dr = sc * (double)w.x - vr; di = sc * (double)w.y - vi; }
      else { dr = -vr; di = -vi; }
      acc[OBS_KY] += dr * dr + di * di + (y == 0 ? nn : 0.0);
      if (A.dim == 3) {
        if (z + 1 < nz) { const cx<R> w = A.psi[i + (size_t)nx * ny]; dr = sc * (double)w.x - vr; di = sc * (double)w.y - vi; }
        else { dr = -vr; di = -vi; }
        acc[OBS_KZ] += dr * dr + di * di + (z == 0 ? nn : 0.0);
      }
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
template <typename R>
__global__ void k_fold_scale(cx<R> *psi, double *prm, size_t n) {
  const R sc = (R)prm[PRM_SC];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    psi[i] = cscale(psi[i], sc);
}

}  // namespace dgpe
