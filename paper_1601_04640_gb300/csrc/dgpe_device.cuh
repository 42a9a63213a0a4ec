// dgpe_device.cuh -- device building blocks of the GB300 split-step solver:
// complex arithmetic, small DFT codelets, a shared-memory Stockham FFT over a
// tile of lines, the chunk-parallel Thomas solve of one Crank-Nicolson
// substep, and deterministic FP64 block reductions.
//
// The method ("Solution method" of arXiv:1601.04640): the dipolar potential is
// a convolution evaluated with FFTs; the kinetic substeps are Crank-Nicolson
// tridiagonal solves along x, y, z ("Summary of revisions": calclux, calcluy,
// calcluz).  Everything here is written for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dgpe {

// ------------------------------------------------------------ complex type
template <typename R> struct V2;
template <> struct V2<double> { using T = double2; };
template <> struct V2<float> { using T = float2; };
template <typename R> using cx = typename V2<R>::T;
template <typename R> struct V4;
template <> struct V4<double> { using T = double4; };
template <> struct V4<float> { using T = float4; };
template <typename R> using rt4 = typename V4<R>::T;  // an FMA-form root (t, fx, fy, swap)

template <typename R> __device__ __forceinline__ cx<R> mk(R x, R y) {
  cx<R> c; c.x = x; c.y = y; return c;
}
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __device__ __forceinline__ C cmulconj(C a, C b) {  // a * conj(b)
  C c; c.x = a.x * b.x + a.y * b.y; c.y = a.y * b.x - a.x * b.y; return c;
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) {
  C c; c.x = a.x * s; c.y = a.y * s; return c;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C> __device__ __forceinline__ C czero() { C c; c.x = 0; c.y = 0; return c; }

// Thomas coefficients are real in imaginary time and complex in real time.
__device__ __forceinline__ double2 coef_mul(double s, double2 v) { return make_double2(s * v.x, s * v.y); }
__device__ __forceinline__ float2 coef_mul(float s, float2 v) { return make_float2(s * v.x, s * v.y); }
__device__ __forceinline__ double2 coef_mul(double2 s, double2 v) { return cmul(s, v); }
__device__ __forceinline__ float2 coef_mul(float2 s, float2 v) { return cmul(s, v); }
__device__ __forceinline__ double coef_prod(double a, double b) { return a * b; }
__device__ __forceinline__ float coef_prod(float a, float b) { return a * b; }
__device__ __forceinline__ double2 coef_prod(double2 a, double2 b) { return cmul(a, b); }
__device__ __forceinline__ float2 coef_prod(float2 a, float2 b) { return cmul(a, b); }
template <typename T> __device__ __forceinline__ T coef_zero();
template <> __device__ __forceinline__ double coef_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ float coef_zero<float>() { return 0.0f; }
template <> __device__ __forceinline__ double2 coef_zero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 coef_zero<float2>() { return make_float2(0.0f, 0.0f); }
__device__ __forceinline__ double coef_scale(double c, double s) { return c * s; }
__device__ __forceinline__ float coef_scale(float c, float s) { return c * s; }
__device__ __forceinline__ double2 coef_scale(double2 c, double s) { return make_double2(c.x * s, c.y * s); }
__device__ __forceinline__ float2 coef_scale(float2 c, float s) { return make_float2(c.x * s, c.y * s); }

// warp shuffles within segments of `w` lanes
__device__ __forceinline__ double shfl_up(double v, int d, int w) { return __shfl_up_sync(0xffffffffu, v, d, w); }
__device__ __forceinline__ float shfl_up(float v, int d, int w) { return __shfl_up_sync(0xffffffffu, v, d, w); }
__device__ __forceinline__ double shfl_down(double v, int d, int w) { return __shfl_down_sync(0xffffffffu, v, d, w); }
__device__ __forceinline__ float shfl_down(float v, int d, int w) { return __shfl_down_sync(0xffffffffu, v, d, w); }
__device__ __forceinline__ double2 shfl_up(double2 v, int d, int w) { v.x = shfl_up(v.x, d, w); v.y = shfl_up(v.y, d, w); return v; }
__device__ __forceinline__ float2 shfl_up(float2 v, int d, int w) { v.x = shfl_up(v.x, d, w); v.y = shfl_up(v.y, d, w); return v; }
__device__ __forceinline__ double2 shfl_down(double2 v, int d, int w) { v.x = shfl_down(v.x, d, w); v.y = shfl_down(v.y, d, w); return v; }
__device__ __forceinline__ float2 shfl_down(float2 v, int d, int w) { v.x = shfl_down(v.x, d, w); v.y = shfl_down(v.y, d, w); return v; }

__device__ __forceinline__ void fsincos(double a, double *s, double *c) { sincos(a, s, c); }
__device__ __forceinline__ void fsincos(float a, float *s, float *c) { sincosf(a, s, c); }
__device__ __forceinline__ double fexpm1(double a) { return expm1(a); }
__device__ __forceinline__ float fexpm1(float a) { return expm1f(a); }

// ------------------------------------------------------------ DFT codelets
// Forward transforms use w_N = exp(-2 pi i / N), inverse exp(+2 pi i / N),
// both unnormalised.  The constants are cos / sin of multiples of 2 pi / N.
#define DGPE_SQRT1_2 0.70710678118654752440
#define DGPE_COS_PI8 0.92387953251128675613
#define DGPE_SIN_PI8 0.38268343236508977173
#define DGPE_SIN_2PI3 0.86602540378443864676
#define DGPE_C1_5 0.30901699437494742410    /* cos(2 pi / 5) */
#define DGPE_C2_5 (-0.80901699437494742410) /* cos(4 pi / 5) */
#define DGPE_S1_5 0.95105651629515357212    /* sin(2 pi / 5) */
#define DGPE_S2_5 0.58778525229247312917    /* sin(4 pi / 5) */

// multiply by w_4 = -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C rot4(C a) {
  C c;
  if (INV) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; }
  return c;
}
// multiply by w_16^k (k in 0..9); w_16^2 = w_8, w_16^4 = w_4
template <bool INV, typename C> __device__ __forceinline__ C rot16(C a, int k) {
  typedef decltype(a.x) R;
  if (k == 0) return a;
  if (k == 4) return rot4<INV>(a);
  R c, s;  // forward angle -2 pi k / 16: w = c + i s
  switch (k) {
    case 1: c = (R)DGPE_COS_PI8; s = -(R)DGPE_SIN_PI8; break;
    case 2: c = (R)DGPE_SQRT1_2; s = -(R)DGPE_SQRT1_2; break;
    case 3: c = (R)DGPE_SIN_PI8; s = -(R)DGPE_COS_PI8; break;
    case 6: c = -(R)DGPE_SQRT1_2; s = -(R)DGPE_SQRT1_2; break;
    default: c = -(R)DGPE_COS_PI8; s = (R)DGPE_SIN_PI8; break;  // k = 9
  }
  if (INV) s = -s;
  C r; r.x = a.x * c - a.y * s; r.y = a.x * s + a.y * c; return r;
}

template <bool INV, typename C> __device__ __forceinline__ void dft2(C *v) {
  C t = v[0]; v[0] = t + v[1]; v[1] = t - v[1];
}
template <bool INV, typename C> __device__ __forceinline__ void dft4s(C &a0, C &a1, C &a2, C &a3) {
  C t0 = a0 + a2, t1 = a0 - a2, t2 = a1 + a3, t3 = rot4<INV>(a1 - a3);
  a0 = t0 + t2; a2 = t0 - t2; a1 = t1 + t3; a3 = t1 - t3;
}
template <bool INV, typename C> __device__ __forceinline__ void dft4(C *v) { dft4s<INV>(v[0], v[1], v[2], v[3]); }
template <bool INV, typename C> __device__ __forceinline__ void dft8(C *v) {
  // even/odd split: X[k] = E[k] + w8^k O[k], X[k+4] = E[k] - w8^k O[k]
  C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4s<INV>(e0, e1, e2, e3);
  dft4s<INV>(o0, o1, o2, o3);
  o1 = rot16<INV>(o1, 2);
  o2 = rot4<INV>(o2);
  o3 = rot16<INV>(o3, 6);
  v[0] = e0 + o0; v[4] = e0 - o0;
  v[1] = e1 + o1; v[5] = e1 - o1;
  v[2] = e2 + o2; v[6] = e2 - o2;
  v[3] = e3 + o3; v[7] = e3 - o3;
}
template <bool INV, typename C> __device__ __forceinline__ void dft16(C *v) {
  // A_r[k] = DFT4_m(x[4m + r]);  X[k + 4s] = sum_r w4^{rs} (w16^{rk} A_r[k])
#pragma unroll
  for (int r = 0; r < 4; ++r) dft4s<INV>(v[r], v[r + 4], v[r + 8], v[r + 12]);
  // now v[r + 4k] = A_r[k]
#pragma unroll
  for (int k = 1; k < 4; ++k)
#pragma unroll
    for (int r = 1; r < 4; ++r) v[r + 4 * k] = rot16<INV>(v[r + 4 * k], r * k);
#pragma unroll
  for (int k = 0; k < 4; ++k) dft4s<INV>(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
  // v[s + 4k] = X[k + 4s]: transpose the 4x4 block into natural order
  C t[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int s = 0; s < 4; ++s) v[k + 4 * s] = t[s + 4 * k];
}
template <bool INV, typename C> __device__ __forceinline__ void dft3(C *v) {
  typedef decltype(v[0].x) R;
  const R s3 = INV ? (R)DGPE_SIN_2PI3 : -(R)DGPE_SIN_2PI3;
  C t = v[1] + v[2], u = v[1] - v[2];
  C a; a.x = v[0].x - (R)0.5 * t.x; a.y = v[0].y - (R)0.5 * t.y;
  C b; b.x = -s3 * u.y; b.y = s3 * u.x;  // i s3 u
  v[0] = v[0] + t;
  v[1] = a + b;
  v[2] = a - b;
}
template <bool INV, typename C> __device__ __forceinline__ void dft5(C *v) {
  typedef decltype(v[0].x) R;
  const R c1 = (R)DGPE_C1_5, c2 = (R)DGPE_C2_5;
  const R s1 = INV ? (R)DGPE_S1_5 : -(R)DGPE_S1_5;
  const R s2 = INV ? (R)DGPE_S2_5 : -(R)DGPE_S2_5;
  C t1 = v[1] + v[4], t2 = v[2] + v[3], u1 = v[1] - v[4], u2 = v[2] - v[3];
  C a1, a2, b1, b2;
  a1.x = v[0].x + c1 * t1.x + c2 * t2.x; a1.y = v[0].y + c1 * t1.y + c2 * t2.y;
  a2.x = v[0].x + c2 * t1.x + c1 * t2.x; a2.y = v[0].y + c2 * t1.y + c1 * t2.y;
  // b1 = i (s1 u1 + s2 u2), b2 = i (s2 u1 - s1 u2)   (signs folded into s1, s2)
  R p1x = s1 * u1.x + s2 * u2.x, p1y = s1 * u1.y + s2 * u2.y;
  R p2x = s2 * u1.x - s1 * u2.x, p2y = s2 * u1.y - s1 * u2.y;
  b1.x = -p1y; b1.y = p1x;
  b2.x = -p2y; b2.y = p2x;
  v[0] = v[0] + t1 + t2;
  v[1] = a1 + b1; v[4] = a1 - b1;
  v[2] = a2 + b2; v[3] = a2 - b2;
}
template <int RAD, bool INV, typename C> __device__ __forceinline__ void dft(C *v) {
  if constexpr (RAD == 2) dft2<INV>(v);
  else if constexpr (RAD == 3) dft3<INV>(v);
  else if constexpr (RAD == 4) dft4<INV>(v);
  else if constexpr (RAD == 5) dft5<INV>(v);
  else if constexpr (RAD == 8) dft8<INV>(v);
  else if constexpr (RAD == 16) dft16<INV>(v);
}

// ------------------------------------ FMA form of a twiddled radix-2^L DFT
// Y_q = sum_r u_r w^r W_R^{rq} (the inputs of a Stockham stage times their
// twiddles w^r, then the radix-R DFT) as L layers of radix-2 butterflies:
// splitting r into even and odd halves gives Y_q = E_q + (w W_R^q) O_q and
// Y_{q+R/2} = E_q - (w W_R^q) O_q, where E and O are the same problem of size
// R/2 with twiddle w^2.  Bottom-up with the leaves in bit-reversed order, the
// size-S combine uses the roots w^{R/S} W_S^q, q < S/2 (n-th root index
// (R/S) rho + q n/S for w = root rho).  Each root c + i s is tabulated as
// (t, fx, fy, sw): for |c| >= |s|, t = s/c and (fx, fy) = (c, c); otherwise
// the root is i (s - i c), t = -c/s, (fx, fy) = (-s, s) and sw = 1.  Then
// w b = (fx p.x, fy p.y) with v = (b.x - t b.y, b.y + t b.x) and p = v or v
// swapped, and a butterfly a +- w b is six FMAs (two for v, four for the
// outputs) with |t| <= 1, instead of a complex product and four additions.
// This is the rotation-by-ratio device of S. Goedecker's FFT algorithms for
// machines with fused multiply-add.  The swap is an integer select.
__device__ __forceinline__ void bfly_fma(double2 &a, double2 &b, const double4 P) {
  const double vx = fma(-P.x, b.y, b.x), vy = fma(P.x, b.x, b.y);
  const bool sw = __double_as_longlong(P.w) != 0;
  const double px = sw ? vy : vx, py = sw ? vx : vy;
  const double ax = a.x, ay = a.y;
  a = make_double2(fma(P.y, px, ax), fma(P.z, py, ay));
  b = make_double2(fma(-P.y, px, ax), fma(-P.z, py, ay));
}
__device__ __forceinline__ void bfly_fma(float2 &a, float2 &b, const float4 P) {
  const float vx = fmaf(-P.x, b.y, b.x), vy = fmaf(P.x, b.x, b.y);
  const bool sw = __float_as_int(P.w) != 0;
  const float px = sw ? vy : vx, py = sw ? vx : vy;
  const float ax = a.x, ay = a.y;
  a = make_float2(fmaf(P.y, px, ax), fmaf(P.z, py, ay));
  b = make_float2(fmaf(-P.y, px, ax), fmaf(-P.z, py, ay));
}
template <int R> struct BitRev {
  static constexpr int of(int r) {
    int o = 0;
    for (int m = R >> 1, b = 1; m > 0; m >>= 1, b <<= 1)
      if (r & b) o |= m;
    return o;
  }
};
// u: the stage's R inputs in natural order, replaced by Y_0..Y_{R-1};
// rho: the root index of w; n: line length; T: the tabulated roots (n of them)
template <int RAD, typename R>
__device__ __forceinline__ void tw_dft_fma(cx<R> *u, int rho, int n, const rt4<R> *__restrict__ T) {
  cx<R> x[RAD];
#pragma unroll
  for (int r = 0; r < RAD; ++r) x[BitRev<RAD>::of(r)] = u[r];
#pragma unroll
  for (int S = 2; S <= RAD; S <<= 1) {
    const int half = S / 2, ns = n / S;
    const int base = (RAD / S) * rho;
#pragma unroll
    for (int q = 0; q < half; ++q) {
      const rt4<R> P = T[(base + q * ns) & (n - 1)];
#pragma unroll
      for (int g = 0; g < RAD; g += S) bfly_fma(x[g + q], x[g + q + half], P);
    }
  }
#pragma unroll
  for (int r = 0; r < RAD; ++r) u[r] = x[r];
}

// ------------------------------------------------- Stockham FFT over a tile
// Radix sequence of one line length (forward order; the inverse runs it
// reversed so that its first stage reads what the forward's last wrote).
// Every length and radix product here is a power of two, so index arithmetic
// uses shifts and masks.
struct FftPlan {
  int n;
  int ns;
  int rad[10];
};

template <int V> struct Log2 { static constexpr int value = 1 + Log2<V / 2>::value; };
template <> struct Log2<1> { static constexpr int value = 0; };
__device__ __forceinline__ int ilog2(int v) { return 31 - __clz(v); }

// Shared-memory index of element a of line l.  Line-major tiles (SA = 1) pad
// one element after every PADW elements (PADW elements = 128 bytes), which
// makes every Stockham read and write pattern conflict-free; column tiles
// (SL = 1) need no pad.
template <int PADW> __device__ __forceinline__ int sidx(int l, int a, int SL, int SA) {
  if (PADW > 0) return l * SL + a + (a / PADW);
  return l * SL + a * SA;
}

// Index arithmetic of one Stockham stage.  POW2: n, nlines and Ns are powers
// of two and the stage uses shifts and masks; otherwise divisions.
struct StageIdx {
  int n, nbl, nlines, Ns, ln, lnbl, lnl, lNs, lr;
};

// One Stockham stage with radix RAD over `nlines` lines of length n held in
// shared memory.  Butterfly j of a line reads elements j + r n/RAD, twiddles
// them by w_{Ns RAD}^{(j mod Ns) r}, applies the RAD-point DFT and writes
// element (j / Ns) Ns RAD + (j mod Ns) + r Ns.  The first stage reads through
// `load` instead of shared memory and the last writes through `store` (its
// outputs are in natural order).  Each thread owns EPT / RAD butterflies, so
// all of its values stay in registers across the barrier that separates the
// reads from the writes (in-place update).
template <typename R, int EPT, int RAD, bool INV, bool LINE_FAST, int PADW, bool POW2, bool FMA, class Load,
          class Store>
__device__ __forceinline__ void fft_stage(cx<R> *sm, int SL, int SA, const StageIdx &I, bool first,
                                          bool last, const cx<R> *__restrict__ tw,
                                          const rt4<R> *__restrict__ tf, Load &load, Store &store) {
  static_assert(EPT % RAD == 0, "radix must divide the elements per thread");
  constexpr int NB = EPT / RAD;
  const int T = blockDim.x, t = threadIdx.x;
  const int nbl = I.nbl, nlines = I.nlines, Ns = I.Ns;
  const int B = nbl * nlines;
  const int tstride = I.n / (Ns * RAD);  // twiddle stride n / (Ns RAD)
  auto line_of = [&](int b) {
    if (POW2) return LINE_FAST ? (b & (nlines - 1)) : (b >> I.lnbl);
    return LINE_FAST ? (b % nlines) : (b / nbl);
  };
  auto bfly_of = [&](int b) {
    if (POW2) return LINE_FAST ? (b >> I.lnl) : (b & (nbl - 1));
    return LINE_FAST ? (b / nlines) : (b % nbl);
  };
  cx<R> v[EPT];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = t + i * T;
    const bool ok = b < B;
    const int l = line_of(b), j = bfly_of(b);
    cx<R> *u = v + i * RAD;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int a = j + r * nbl;
      if (!ok) u[r] = czero<cx<R>>();
      else if (first) u[r] = load(l, a);
      else u[r] = sm[sidx<PADW>(l, a, SL, SA)];
    }
    if (!first) {
      const int k = POW2 ? (j & (Ns - 1)) : (j % Ns);
      if constexpr (FMA && (RAD & (RAD - 1)) == 0) {
        tw_dft_fma<RAD, R>(u, k * tstride, I.n, tf);
      } else {
#pragma unroll
        for (int r = 1; r < RAD; ++r) {
          cx<R> w = tw[k * r * tstride];
          u[r] = INV ? cmulconj(u[r], w) : cmul(u[r], w);
        }
        dft<RAD, INV>(u);
      }
    } else {
      dft<RAD, INV>(u);
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = t + i * T;
    if (b < B) {
      const int l = line_of(b), j = bfly_of(b);
      const int base = POW2 ? (((j >> I.lNs) << (I.lNs + I.lr)) + (j & (Ns - 1)))
                            : ((j / Ns) * Ns * RAD + (j % Ns));
      cx<R> *u = v + i * RAD;
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int a = base + r * Ns;
        if (last) store(l, a, u[r]);
        else sm[sidx<PADW>(l, a, SL, SA)] = u[r];
      }
    }
  }
  __syncthreads();
}

// Full transform of every line of the tile.  tw[t] = exp(-2 pi i t / n).
// FMA (power-of-two lengths): the twiddled stages use tw_dft_fma with
// the tabulated roots tf (exp(-2 pi i t/n) forward, exp(+2 pi i t/n) inverse).
template <typename R, int EPT, bool INV, bool LINE_FAST, int PADW, bool POW2 = true, bool FMA = false,
          class Load, class Store>
__device__ __forceinline__ void tile_fft(cx<R> *sm, int SL, int SA, int nlines, const FftPlan &pl,
                         const cx<R> *__restrict__ tw, Load load, Store store,
                         const rt4<R> *__restrict__ tf = nullptr) {
  StageIdx I;
  I.n = pl.n;
  I.nlines = nlines;
  I.Ns = 1;
  I.ln = POW2 ? ilog2(pl.n) : 0;
  I.lnl = (POW2 && LINE_FAST) ? ilog2(nlines) : 0;
  I.lNs = 0;
  for (int s = 0; s < pl.ns; ++s) {
    const int rad = INV ? pl.rad[pl.ns - 1 - s] : pl.rad[s];
    const bool first = (s == 0), last = (s == pl.ns - 1);
    I.nbl = pl.n / rad;
    I.lr = (rad == 2) ? 1 : (rad == 4) ? 2 : (rad == 8) ? 3 : (rad == 16) ? 4 : 0;
    I.lnbl = I.ln - I.lr;
    switch (rad) {
      case 2: if constexpr (EPT % 2 == 0) fft_stage<R, EPT, 2, INV, LINE_FAST, PADW, POW2, FMA>(sm, SL, SA, I, first, last, tw, tf, load, store); break;
      case 3: if constexpr (EPT % 3 == 0 && !POW2) fft_stage<R, EPT, 3, INV, LINE_FAST, PADW, POW2, FMA>(sm, SL, SA, I, first, last, tw, tf, load, store); break;
      case 4: if constexpr (EPT % 4 == 0) fft_stage<R, EPT, 4, INV, LINE_FAST, PADW, POW2, FMA>(sm, SL, SA, I, first, last, tw, tf, load, store); break;
      case 5: if constexpr (EPT % 5 == 0 && !POW2) fft_stage<R, EPT, 5, INV, LINE_FAST, PADW, POW2, FMA>(sm, SL, SA, I, first, last, tw, tf, load, store); break;
      case 8: if constexpr (EPT % 8 == 0) fft_stage<R, EPT, 8, INV, LINE_FAST, PADW, POW2, FMA>(sm, SL, SA, I, first, last, tw, tf, load, store); break;
      case 16: if constexpr (EPT % 16 == 0) fft_stage<R, EPT, 16, INV, LINE_FAST, PADW, POW2, FMA>(sm, SL, SA, I, first, last, tw, tf, load, store); break;
      default: break;
    }
    I.Ns *= rad;
    I.lNs += I.lr;
  }
}

// ------------------------------- compile-time Stockham FFT over a line tile
// The same transform as tile_fft for a line-major tile (line l, element a at
// l SL + a + a / PADW) when the line length N, the number of lines NL, the
// block size T and the radix sequence are compile-time constants: every
// index (line, butterfly, twiddle, shared-memory address) folds to shifts,
// masks and immediate offsets, and only the stages the length needs are
// compiled.  Radices: the first of 16, 8, 5, 4, 3, 2 dividing both EPT and
// what is left of N, in order (the runtime plans' sequence; the inverse runs
// it reversed).
constexpr int ct_radix(int n, int ept, int s) {
  // candidates in the order of the runtime plans: 16, 8, 5, 4, 3, 2
  int m = n;
  for (int k = 0; k < 16; ++k) {
    int r = 0;
    if (ept % 16 == 0 && m % 16 == 0) r = 16;
    else if (ept % 8 == 0 && m % 8 == 0) r = 8;
    else if (ept % 5 == 0 && m % 5 == 0) r = 5;
    else if (ept % 4 == 0 && m % 4 == 0) r = 4;
    else if (ept % 3 == 0 && m % 3 == 0) r = 3;
    else if (m % 2 == 0) r = 2;
    if (r == 0) return 0;
    if (k == s) return r;
    m /= r;
  }
  return 0;
}
constexpr int ct_nstages(int n, int ept) {
  int s = 0, m = n;
  while (m > 1) { m /= ct_radix(n, ept, s); ++s; }
  return s;
}
constexpr int ct_log2(int v) { return v <= 1 ? 0 : 1 + ct_log2(v / 2); }

// LINE_FAST: consecutive threads take consecutive lines (column tiles, element
// a of line l at l + a SA); otherwise consecutive butterflies of one line
// (line-major tiles, l SL + a + a / PADW).
template <int PADW, int SL, int SA>
__device__ __forceinline__ int ct_sidx(int l, int a) {
  if constexpr (PADW > 0) return l * SL + a + a / PADW;
  else return l * SL + a * SA;
}
template <typename R, int N, int EPT, int RAD, int NS, bool INV, int PADW, int SL, int NL, int T, bool FIRST,
          bool LAST, bool LINE_FAST, int SA, class Load, class Store>
__device__ __forceinline__ void fft_stage_ct(cx<R> *sm, const cx<R> *__restrict__ tw, Load &load, Store &store) {
  static_assert(EPT % RAD == 0, "radix must divide the elements per thread");
  constexpr int NB = EPT / RAD;
  constexpr int NBL = N / RAD;
  constexpr int B = NBL * NL;
  constexpr int TSTR = N / (NS * RAD);
  // divisions by constants: shifts and masks for powers of two, multiplies
  // by reciprocals otherwise (3 2^k and 5 2^k lengths)
  const int t = threadIdx.x;
  cx<R> v[EPT];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = t + i * T;
    const bool ok = (B == T * NB) || b < B;  // every butterfly slot of the block is real
    const unsigned ub = (unsigned)b;
    const int l = (int)(LINE_FAST ? (ub % NL) : (ub / NBL));
    const int j = (int)(LINE_FAST ? (ub / NL) : (ub % NBL));
    cx<R> *u = v + i * RAD;
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      const int a = j + r * NBL;
      if (!ok) u[r] = czero<cx<R>>();
      else if (FIRST) u[r] = load(l, a);
      else u[r] = sm[ct_sidx<PADW, SL, SA>(l, a)];
    }
    if constexpr (!FIRST) {
      const int k = (int)((unsigned)j % NS);
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const cx<R> w = tw[k * r * TSTR];
        u[r] = INV ? cmulconj(u[r], w) : cmul(u[r], w);
      }
    }
    dft<RAD, INV>(u);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    const int b = t + i * T;
    if ((B == T * NB) || b < B) {
      const unsigned ub = (unsigned)b;
      const int l = (int)(LINE_FAST ? (ub % NL) : (ub / NBL));
      const unsigned uj = LINE_FAST ? (ub / NL) : (ub % NBL);
      const int base = (int)((uj / NS) * NS * RAD + (uj % NS));
      cx<R> *u = v + i * RAD;
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        const int a = base + r * NS;
        if (LAST) store(l, a, u[r]);
        else sm[ct_sidx<PADW, SL, SA>(l, a)] = u[r];
      }
    }
  }
  __syncthreads();
}
template <typename R, int N, int EPT, bool INV, int PADW, int SL, int NL, int T, bool LINE_FAST, int SA, int S,
          int NSACC, class Load, class Store>
__device__ __forceinline__ void tile_fft_ct_from(cx<R> *sm, const cx<R> *__restrict__ tw, Load &load, Store &store) {
  constexpr int NST = ct_nstages(N, EPT);
  if constexpr (S < NST) {
    constexpr int RAD = INV ? ct_radix(N, EPT, NST - 1 - S) : ct_radix(N, EPT, S);
    fft_stage_ct<R, N, EPT, RAD, NSACC, INV, PADW, SL, NL, T, S == 0, S == NST - 1, LINE_FAST, SA>(sm, tw, load,
                                                                                                  store);
    tile_fft_ct_from<R, N, EPT, INV, PADW, SL, NL, T, LINE_FAST, SA, S + 1, NSACC * RAD>(sm, tw, load, store);
  }
}
// Full transform of the NL lines of a line-major tile; tw[t] = exp(-2 pi i t / N).
template <typename R, int N, int EPT, bool INV, int PADW, int SL, int NL, int T, class Load, class Store>
__device__ __forceinline__ void tile_fft_ct(cx<R> *sm, const cx<R> *__restrict__ tw, Load load, Store store) {
  tile_fft_ct_from<R, N, EPT, INV, PADW, SL, NL, T, false, 1, 0, 1>(sm, tw, load, store);
}
// ... of a column tile of NL lines (element a of line l at a NL + l).
template <typename R, int N, int EPT, bool INV, int NL, int T, class Load, class Store>
__device__ __forceinline__ void tile_fft_ct_cols(cx<R> *sm, const cx<R> *__restrict__ tw, Load load, Store store) {
  tile_fft_ct_from<R, N, EPT, INV, 0, 1, NL, T, true, NL, 0, 1>(sm, tw, load, store);
}

// ------------------------------------------- Crank-Nicolson (Thomas) solve
// One CN substep along a line of n points, in increment form:
//   x = psi + w,  A w = r,  r = -2 kt (2 psi_a - psi_{a-1} - psi_{a+1}),
// A = I + kt T (kt = kappa tau), which equals A x = B psi with B = I - kt T.
// LU of A: m_0 = 1/(1+2kt), m_a = 1/(1+2kt - kt^2 m_{a-1}), alpha_a = kt m_a;
//   forward  y_a = alpha_a y_{a-1} + m_a r_a,
//   backward w_a = y_a + alpha_a w_{a+1}.
// Both first-order recurrences are split into TPL chunks of CL points (one
// per lane of a TPL-wide lane segment); chunk-local passes with zero inflow,
// a Kogge-Stone scan of the chunk maps (P, Y) over the lanes, and a fix-up
// with the in-chunk products P_a = prod_{b=a0..a} alpha_b and
// Q_a = prod_{b=a..a0+CL-1} alpha_b.  This form (FP64) reads the tables m,
// alpha, P, Q (n each, in that order) from global memory.  The line lives in
// shared memory at line[a + a / CL] (one pad per chunk keeps the lanes'
// accesses on distinct banks).
template <typename R, typename Coef, int CL>
__device__ __forceinline__ void cn_line(cx<R> *line, int n, int TPL, int q, Coef kt,
                                        const Coef *__restrict__ tab, bool active) {
  typedef cx<R> Cx;
  const Coef *tm = tab, *ta = tab + n, *tp = tab + 2 * n, *tq = tab + 3 * n;
  const int a0 = q * CL;
  Cx y[CL];
  Cx acc = czero<Cx>();
  Cx prev = (active && a0 > 0) ? line[(a0 - 1) + (a0 - 1) / CL] : czero<Cx>();
  Cx cur = active ? line[a0 + a0 / CL] : czero<Cx>();
  const Coef m2kt = coef_scale(kt, (R)(-2));
#pragma unroll
  for (int i = 0; i < CL; ++i) {
    const int a = a0 + i;
    Cx nxt = (active && a + 1 < n) ? line[(a + 1) + (a + 1) / CL] : czero<Cx>();
    Cx lap = cur + cur - prev - nxt;
    Cx r = coef_mul(m2kt, lap);
    const Coef ma = active ? tm[a] : coef_zero<Coef>();
    const Coef al = active ? ta[a] : coef_zero<Coef>();
    acc = coef_mul(al, acc) + coef_mul(ma, r);
    y[i] = acc;
    prev = cur;
    cur = nxt;
  }
  // inclusive scan over the chunks (lane segment of width TPL)
  Coef P = active ? tp[a0 + CL - 1] : coef_zero<Coef>();
  Cx Y = acc;
  for (int d = 1; d < TPL; d <<= 1) {
    Coef Pn = shfl_up(P, d, TPL);
    Cx Yn = shfl_up(Y, d, TPL);
    if (q >= d) { Y = Y + coef_mul(P, Yn); P = coef_prod(P, Pn); }
  }
  Cx yin = shfl_up(Y, 1, TPL);
  if (q == 0) yin = czero<Cx>();
#pragma unroll
  for (int i = 0; i < CL; ++i) {
    const Coef f = active ? tp[a0 + i] : coef_zero<Coef>();
    y[i] = y[i] + coef_mul(f, yin);
  }
  // chunk-local backward recurrence
  acc = czero<Cx>();
#pragma unroll
  for (int i = CL - 1; i >= 0; --i) {
    const Coef al = active ? ta[a0 + i] : coef_zero<Coef>();
    acc = y[i] + coef_mul(al, acc);
    y[i] = acc;
  }
  Coef Q = active ? tq[a0] : coef_zero<Coef>();
  Cx W = acc;
  for (int d = 1; d < TPL; d <<= 1) {
    Coef Qn = shfl_down(Q, d, TPL);
    Cx Wn = shfl_down(W, d, TPL);
    if (q + d < TPL) { W = W + coef_mul(Q, Wn); Q = coef_prod(Q, Qn); }
  }
  Cx win = shfl_down(W, 1, TPL);
  if (q == TPL - 1) win = czero<Cx>();
  if (active) {
#pragma unroll
    for (int i = CL - 1; i >= 0; --i) {
      const int a = a0 + i;
      Cx w = y[i] + coef_mul(tq[a], win);
      const int ia = a + a / CL;
      line[ia] = line[ia] + w;
    }
  }
}

// The same solve with the four tables m, alpha, P, Q read from a padded
// shared copy (table k at tab + k TS, TS = n + n/CL + 1, coefficient a at
// a + a/CL; see stage_cn_tables), for the FP32 bulk.  Every access is a
// constant offset from the chunk's base (element a0 + i of the chunk sits at
// base + i, a0 + CL at base + CL + 1, a0 - 1 at base - 2), the recurrences are
// written as FMAs, and kt enters only through products with the real
// (imaginary time) or purely imaginary (real time, make_kt gives (0, tau))
// number kt, two multiplies each.
__device__ __forceinline__ float2 kt_times(float kt, float2 v) { return make_float2(kt * v.x, kt * v.y); }
__device__ __forceinline__ float2 kt_times(float2 kt, float2 v) { return make_float2(-kt.y * v.y, kt.y * v.x); }
__device__ __forceinline__ double2 kt_times(double kt, double2 v) { return make_double2(kt * v.x, kt * v.y); }
__device__ __forceinline__ double2 kt_times(double2 kt, double2 v) { return make_double2(-kt.y * v.y, kt.y * v.x); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
// a v + w for a real or complex coefficient a
__device__ __forceinline__ float2 coef_fma(float a, float2 v, float2 w) {
  return make_float2(fmaf(a, v.x, w.x), fmaf(a, v.y, w.y));
}
__device__ __forceinline__ float2 coef_fma(float2 a, float2 v, float2 w) {
  return make_float2(fmaf(a.x, v.x, fmaf(-a.y, v.y, w.x)), fmaf(a.x, v.y, fmaf(a.y, v.x, w.y)));
}
__device__ __forceinline__ double2 coef_fma(double a, double2 v, double2 w) {
  return make_double2(fma(a, v.x, w.x), fma(a, v.y, w.y));
}
__device__ __forceinline__ double2 coef_fma(double2 a, double2 v, double2 w) {
  return make_double2(fma(a.x, v.x, fma(-a.y, v.y, w.x)), fma(a.x, v.y, fma(a.y, v.x, w.y)));
}
//
// dlim > 0 limits the Kogge-Stone scans to the rounds d < dlim: the inflow of
// a chunk then gathers the dlim chunks before it exactly and drops the rest,
// whose weights are products of at least dlim whole-chunk products P_chunk.
// The host picks dlim from rho = max |P_chunk| so that the dropped part,
// at most rho^dlim / (1 - rho) of the largest chunk value, is below 2^-32
// of it (kt = dt / (4 h^2) small: rho is tiny and a chunk needs only its
// neighbour's value); dlim <= 0 runs all rounds.
template <typename R, typename Coef, int CL>
__device__ __forceinline__ void cn_line_st(cx<R> *line, int n, int TPL, int q, Coef kt,
                                           const Coef *__restrict__ tab, bool active, int dlim = 0) {
  typedef cx<R> Cx;
  const int TS = n + n / CL + 1;
  const int DL = (dlim > 0 && dlim < TPL) ? dlim : TPL;
  const int a0 = q * CL;
  Cx *lp = line + a0 + q;                 // padded address of element a0
  const Coef *tm = tab + a0 + q, *ta = tm + TS, *tp = ta + TS, *tq = tp + TS;
  const Coef m2kt = coef_scale(kt, (R)(-2));
  Cx y[CL];
  Cx acc = czero<Cx>();
  Cx prev = (active && a0 > 0) ? lp[-2] : czero<Cx>();
  Cx cur = active ? lp[0] : czero<Cx>();
#pragma unroll
  for (int i = 0; i < CL; ++i) {
    const int off = (i + 1 < CL) ? i + 1 : CL + 1;
    const Cx nxt = (active && a0 + i + 1 < n) ? lp[off] : czero<Cx>();
    // r = -2 kt (2 cur - prev - nxt)
    const Cx s = prev + nxt;
    const Cx r = kt_times(m2kt, mk<R>(fma_t((R)2, cur.x, -s.x), fma_t((R)2, cur.y, -s.y)));
    const Coef ma = active ? tm[i] : coef_zero<Coef>();
    const Coef al = active ? ta[i] : coef_zero<Coef>();
    acc = coef_fma(al, acc, coef_mul(ma, r));
    y[i] = acc;
    prev = cur;
    cur = nxt;
  }
  Coef P = active ? tp[CL - 1] : coef_zero<Coef>();
  Cx Y = acc;
  for (int d = 1; d < DL; d <<= 1) {
    Coef Pn = shfl_up(P, d, TPL);
    Cx Yn = shfl_up(Y, d, TPL);
    if (q >= d) { Y = coef_fma(P, Yn, Y); P = coef_prod(P, Pn); }
  }
  Cx yin = shfl_up(Y, 1, TPL);
  if (q == 0) yin = czero<Cx>();
#pragma unroll
  for (int i = 0; i < CL; ++i) y[i] = coef_fma(active ? tp[i] : coef_zero<Coef>(), yin, y[i]);
  acc = czero<Cx>();
#pragma unroll
  for (int i = CL - 1; i >= 0; --i) {
    acc = coef_fma(active ? ta[i] : coef_zero<Coef>(), acc, y[i]);
    y[i] = acc;
  }
  Coef Q = active ? tq[0] : coef_zero<Coef>();
  Cx W = acc;
  for (int d = 1; d < DL; d <<= 1) {
    Coef Qn = shfl_down(Q, d, TPL);
    Cx Wn = shfl_down(W, d, TPL);
    if (q + d < TPL) { W = coef_fma(Q, Wn, W); Q = coef_prod(Q, Qn); }
  }
  Cx win = shfl_down(W, 1, TPL);
  if (q == TPL - 1) win = czero<Cx>();
  if (active) {
#pragma unroll
    for (int i = 0; i < CL; ++i) lp[i] = lp[i] + coef_fma(tq[i], win, y[i]);
  }
}

// Copy the four CN tables of an axis (m, alpha, P, Q; n each, in that order)
// into shared memory in the padded layout cn_line_st reads.  All threads take
// part; the caller synchronises before use.
template <typename Coef, int CL>
__device__ __forceinline__ void stage_cn_tables(Coef *dst, const Coef *__restrict__ tab, int n) {
  const int TS = n + n / CL + 1;
  for (int i = threadIdx.x; i < 4 * n; i += blockDim.x) {
    const int k = i / n, a = i - k * n;
    dst[k * TS + a + a / CL] = tab[i];
  }
}

// ------------------------------------------------ asynchronous tile copies
// cp.async global -> shared copies (issued by every thread for its own
// elements, completed per commit group) let a persistent CTA fetch its next
// tile while it computes the current one.
__device__ __forceinline__ void cp_async_elem(float2 *smem, const float2 *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double2 *smem, const double2 *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------- bulk asynchronous copies (mbarrier)
// One thread moves a contiguous block of global memory into shared memory
// with cp.async.bulk; the copy signals an mbarrier with the bytes it wrote,
// and the consumers wait for the barrier's phase.  Addresses and sizes are
// multiples of 16 bytes.  Before a buffer that generic loads or stores used
// is refilled, the issuing thread orders those accesses before the copy
// with fence.proxy.async (after a block barrier).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long *bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete, giving up after
// `limit` polls (each poll may suspend the thread for a short,
// hardware-defined time).  Returns false on give-up.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// ------------------------------------------ tensor-map copies (TMA tiles)
// A 3D box of a tensor described by a CUtensorMap (passed as a
// __grid_constant__ kernel parameter; `tmap` is its generic address) moved
// between global and shared memory by the TMA unit.  Loads complete on an
// mbarrier with the box's byte count (out-of-range elements are filled with
// zeros); stores clip to the tensor's bounds, are committed as a bulk group,
// and the issuing thread waits for the group to have read its shared memory
// before that memory is reused.  Coordinates are in elements, innermost
// first; the innermost one times the element size is a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_3d(void *dst, const void *tmap, int c0, int c1, int c2,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_3d(const void *tmap, int c0, int c1, int c2, const void *src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];\n" ::"l"(tmap),
               "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(src))
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }

// --------------------------------------------------- FP64 block reductions
// Deterministic for a fixed block size: warp tree, then warp totals in order.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
// Returns the block total in thread 0 (other threads: unspecified).
__device__ __forceinline__ double block_sum(double v, double *red /* >= 32 */) {
  const int t = threadIdx.x, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if ((t & 31) == 0) red[t >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (t == 0)
    for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

}  // namespace dgpe
