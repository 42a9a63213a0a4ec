// dgpe_batch.cu -- many independent 2D XY condensates (a parameter sweep over
// grid size, trap anisotropy, g and g_dd, in imaginary and real time) stepped
// together by one persistent kernel (k_batch_run) per dgpe_batch_step call:
// CTAs walk a device work list of (problem, pass, tile) items -- density +
// R2C_x, FFT_y . U . IFFT_y, C2R_x + exponential + CN_x, CN_y + norm -- with
// per-problem counters of completed tiles ordering the passes of a problem,
// and the 64 x 64 problems held in one CTA's shared memory for all the steps
// of the call.  Problems of equal size and mode form a class; at create time
// an autotuner times the orders of the FFT radices of each class.  FP32-bulk.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <map>
#include <string>
#include <vector>

#include "dgpe.h"
#include "dgpe_engine.cuh"

namespace dgpe {
namespace {

typedef EngineT<float> Eng;
typedef cx<float> Cx;

struct Cls {
  int n = 0, imag = 0, var = VAR_P2;
  std::vector<int> members;
  XArgs<float> *dX = nullptr;
  SArgs<float> *dS = nullptr;
  CArgs<float> *dC = nullptr;
  int LP = 0, xT = 0, xgrid = 0, sW = 0, sT = 0, cW = 0, cT = 0;
  size_t xs = 0, x4s = 0, ss = 0, cs = 0;
  dim3 sgrid, cgrid;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;  // join of the class's branch in the step graph
};

// ------------------------------------------------ persistent batched step
// One launch advances every problem of the batch by `nsteps` steps.  CTAs
// take work items in ticket order (one atomic counter):
//   * first, one item per resident problem (n = 64): its CTA keeps the state,
//     the half spectrum and the work tiles in shared memory for all nsteps
//     steps (k_batch_run's resident64 path) and touches HBM only to load and
//     store the state once;
//   * then, for every step, a list of (problem, pass, tile range) items for the
//     other problems, pass-major (density/R2C_x, FFT_y.U.IFFT_y,
//     C2R_x/exp/CN_x, CN_y + norm), largest problems first within a pass.  An
//     item of pass L of step s may start once its problem's completed-tile
//     counter reaches s * (tiles per step) + (tiles of passes < L): every item
//     it waits for has a smaller ticket, so it has been taken by a running CTA
//     and the wait ends.
// Waits are bounded: a CTA that has polled `wait_limit` times (or sees that
// another CTA gave up) skips its item, raises the timeout flag and goes on, so
// the kernel always finishes; the host reports DGPE_ETIMEOUT.  The last CTA to
// leave resets the counters for the next launch.
struct BProb {
  XArgs<float> X;
  SArgs<float> S;
  CArgs<float> C;
  int var, imag, resident, n;
  int tiles[4];  // per pass of one step
  int per_step;  // tiles of one step
  int pad[3];
};
// work-list state in device memory (unsigned words): the ticket counter, CTAs
// that have left, the abort and timeout flags, the held problem + 1 (0: none),
// the problem count, then one completed-tile counter per problem
enum { BS_TICKET = 0, BS_EXIT = 1, BS_ABORT = 2, BS_TIMEOUT = 3, BS_HOLD = 4, BS_NPROB = 5, BS_DONE = 8 };
constexpr int kBatchScr = 20 << 10;  // shared scratch common to all pass bodies (bytes)
constexpr int kRes = 64;              // side of the shared-memory-resident problems

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Shared-memory layout of a resident 64 x 64 problem (bytes)
struct ResLayout {
  static constexpr int N = kRes, CL = 16, TPL = N / CL, P = N + N / CL + 1, PZ = N + N / 16 + 1;
  static constexpr int PSI = 0, SPEC = PSI + N * P * 8, ZT = SPEC + N * N * 8, TABX = ZT + (N / 2) * PZ * 8;
  static constexpr int TABY = TABX + 4 * P * 8, VX = TABY + 2 * N * 8, VY = VX + N * 4, TW = VY + N * 4;
  static constexpr int TOTAL = TW + N * 8;
};

// All nsteps steps of one 64 x 64 problem in one CTA, its data in shared
// memory: the same substeps and arithmetic as the tile passes (R2C along x of
// row pairs, FFT_y.U.IFFT_y of the half-spectrum columns, C2R + exponential +
// chunk-parallel CN_x of the rows), with CN_y solved serially per column (one
// thread per column; the forward sweep keeps its intermediate values in the
// spectrum buffer, which is free by then) and, in imaginary time, the state
// renormalised at the end of each step (FP64 norm).  The state leaves the CTA
// normalised, so the lazy scale is reset to 1.
template <typename Coef>
__device__ __forceinline__ void resident64_run(const BProb &B, int nsteps) {
  typedef float R;
  typedef float2 Cx;
  typedef ResLayout L;
  constexpr int N = L::N, P = L::P, PZ = L::PZ, T = DGPE_MAXT, CL = L::CL, TPL = L::TPL, PW = 16;
  extern __shared__ __align__(16) unsigned char smraw[];
  Cx *const ps = reinterpret_cast<Cx *>(smraw + L::PSI);
  Cx *const sp = reinterpret_cast<Cx *>(smraw + L::SPEC);
  Cx *const zt = reinterpret_cast<Cx *>(smraw + L::ZT);
  Coef *const tabx = reinterpret_cast<Coef *>(smraw + L::TABX);
  Coef *const taby = reinterpret_cast<Coef *>(smraw + L::TABY);
  R *const svx = reinterpret_cast<R *>(smraw + L::VX);
  R *const svy = reinterpret_cast<R *>(smraw + L::VY);
  Cx *const stw = reinterpret_cast<Cx *>(smraw + L::TW);
  __shared__ double s_red[32];
  __shared__ R s_c[4];  // dt s(t), g dt, g_dd dt, 1/sqrt(norm)
  const XArgs<float> &X = B.X;
  const int t = threadIdx.x;
  const int imag = B.imag;
  const double sc0 = X.prm[PRM_SC];
  for (int i = t; i < N * N; i += T) {
    const int y = i >> 6, x = i & (N - 1);
    ps[y * P + x + x / CL] = cscale(X.psi[i], (R)sc0);
  }
  stage_cn_tables<Coef, CL>(tabx, reinterpret_cast<const Coef *>(X.cntab), N);
  for (int i = t; i < 2 * N; i += T) taby[i] = reinterpret_cast<const Coef *>(B.C.cntab)[i];
  for (int i = t; i < N; i += T) { svx[i] = X.vx[i]; svy[i] = X.vy[i]; stw[i] = X.tw[i]; }
  const Coef ktx = make_kt<Coef>(X.tau), kty = make_kt<Coef>(B.C.tau);
  const R *__restrict__ Ug = B.S.U;
  const int px = X.px;
  __syncthreads();
  for (int st = 0; st < nsteps; ++st) {
    if (t == 0) {
      const double dt = X.prm[PRM_DT];
      s_c[0] = (R)trap_dts(X.prm, *X.step);
      s_c[1] = (R)(dt * X.prm[PRM_G]);
      s_c[2] = (R)(dt * X.prm[PRM_GDD]);
    }
    // density of row pairs -> R2C along x -> half spectrum sp[y][kx], kx <= N/2
    {
      auto load = [&](int l, int a) -> Cx {
        const Cx u = ps[(2 * l) * P + a + a / CL], v = ps[(2 * l + 1) * P + a + a / CL];
        return mk<R>(u.x * u.x + u.y * u.y, v.x * v.x + v.y * v.y);
      };
      auto store = [&](int l, int a, Cx v) { zt[l * PZ + a + a / PW] = v; };
      tile_fft_ct<R, N, 8, false, PW, PZ, N / 2, T>(zt, stw, load, store);
      for (int idx = t; idx < (N / 2) * (N / 2 + 1); idx += T) {
        const int l = idx / (N / 2 + 1), k = idx - l * (N / 2 + 1);
        const int km = (k == 0) ? 0 : N - k;
        const Cx Zk = zt[l * PZ + k + k / PW], Zm = zt[l * PZ + km + km / PW];
        sp[(2 * l) * N + k] = mk<R>((R)0.5 * (Zk.x + Zm.x), (R)0.5 * (Zk.y - Zm.y));
        sp[(2 * l + 1) * N + k] = mk<R>((R)0.5 * (Zk.y + Zm.y), (R)0.5 * (Zm.x - Zk.x));
      }
      __syncthreads();
    }
    // FFT_y . U/N . IFFT_y on the half-spectrum columns (column l at sp[a N + l])
    {
      auto load = [&](int l, int a) -> Cx { return (l <= N / 2) ? sp[a * N + l] : czero<Cx>(); };
      auto mstore = [&](int l, int a, Cx v) {
        sp[a * N + l] = (l <= N / 2) ? cscale(v, Ug[(size_t)a * px + l]) : czero<Cx>();
      };
      tile_fft_ct_cols<R, N, 16, false, N, T>(sp, stw, load, mstore);
      auto sload = [&](int l, int a) -> Cx { return sp[a * N + l]; };
      auto sstore = [&](int l, int a, Cx v) { sp[a * N + l] = v; };
      tile_fft_ct_cols<R, N, 16, true, N, T>(sp, stw, sload, sstore);
    }
    const R dts = s_c[0], gdt = s_c[1], gdddt = s_c[2];
    // C2R along x of row pairs + exponential substep on the rows in place
    {
      auto load = [&](int l, int a) -> Cx {
        const int k = (a <= N / 2) ? a : N - a;
        Cx X0 = sp[(2 * l) * N + k], X1 = sp[(2 * l + 1) * N + k];
        if (a == 0 || a == N / 2) { X0.y = 0; X1.y = 0; }
        if (a > N / 2) { X0.y = -X0.y; X1.y = -X1.y; }
        return mk<R>(X0.x - X1.y, X0.y + X1.x);
      };
      auto apply_e = [&](int row, int a, R phi) {
        const int ia = row * P + a + a / CL;
        const Cx v = ps[ia];
        const R th = dts * (svx[a] + svy[row]) + gdt * (v.x * v.x + v.y * v.y) + gdddt * phi;
        ps[ia] = nonlinear_factor<R>(v, th, imag);
      };
      auto store = [&](int l, int a, Cx v) {
        apply_e(2 * l, a, v.x);
        apply_e(2 * l + 1, a, v.y);
      };
      tile_fft_ct<R, N, 8, true, PW, PZ, N / 2, T>(zt, stw, load, store);
    }
    // Crank-Nicolson along x: TPL lanes per row
    {
      const int l = t / TPL, q = t - l * TPL;
      cn_line_st<R, Coef, CL>(ps + l * P, N, TPL, q, ktx, tabx, true, X.cnd);
      __syncthreads();
    }
    // Crank-Nicolson along y, one thread per column, increment form:
    //   r_a = -2 kt (2 psi_a - psi_{a-1} - psi_{a+1}),
    //   y_a = alpha_a y_{a-1} + m_a r_a,  w_a = y_a + alpha_a w_{a+1},  psi_a += w_a
    if (t < N) {
      const int xo = t + t / CL;
      const Coef m2kt = coef_scale(kty, (R)(-2));
      Cx prev = czero<Cx>(), cur = ps[xo], acc = czero<Cx>();
      for (int a = 0; a < N; ++a) {
        const Cx nxt = (a + 1 < N) ? ps[(a + 1) * P + xo] : czero<Cx>();
        const Cx s2 = prev + nxt;
        const Cx r = kt_times(m2kt, mk<R>(fma_t((R)2, cur.x, -s2.x), fma_t((R)2, cur.y, -s2.y)));
        acc = coef_fma(taby[N + a], acc, coef_mul(taby[a], r));
        sp[a * N + t] = acc;
        prev = cur;
        cur = nxt;
      }
      Cx w = czero<Cx>();
      for (int a = N - 1; a >= 0; --a) {
        w = coef_fma(taby[N + a], w, sp[a * N + t]);
        ps[a * P + xo] = ps[a * P + xo] + w;
      }
    }
    __syncthreads();
    if (imag) {
      R ts = 0;
      for (int i = t; i < N * N; i += T) {
        const int y = i >> 6, x = i & (N - 1);
        const Cx v = ps[y * P + x + x / CL];
        ts += v.x * v.x + v.y * v.y;
      }
      const double sum = block_sum((double)ts, s_red);
      if (t == 0) {
        const double norm = X.prm[PRM_CELL] * sum;
        if (norm > 0.0 && isfinite(norm)) s_c[3] = (R)(1.0 / sqrt(norm));
        else { s_c[3] = (R)1; const_cast<double *>(X.prm)[PRM_NONFINITE] = 1.0; }
      }
      __syncthreads();
      const R f = s_c[3];
      for (int i = t; i < N * N; i += T) {
        const int y = i >> 6, x = i & (N - 1);
        const int ia = y * P + x + x / CL;
        ps[ia] = cscale(ps[ia], f);
      }
    }
    if (t == 0) *const_cast<long long *>(X.step) += 1;
    __syncthreads();
  }
  for (int i = t; i < N * N; i += T) {
    const int y = i >> 6, x = i & (N - 1);
    X.psi[i] = ps[y * P + x + x / CL];
  }
  if (t == 0) const_cast<double *>(X.prm)[PRM_SC] = 1.0;
}

// One tile of one pass, one body per function: each is compiled (and its
// registers allocated) on its own, so the large switch of the persistent
// kernel does not make the bodies spill.  N > 0: power-of-two side N with
// compile-time lengths (the default tile shapes of the persistent step).
template <int EX, int EPS, int CL, bool P2, int N, int LEVEL, typename Coef>
__device__ __noinline__ void batch_body(const BProb &B, int tile) {
  constexpr int WS = N ? DGPE_MAXT * EPS / N : 0, WCN = N ? DGPE_MAXT / (N / CL) : 0;
  constexpr bool IMAG = std::is_same<Coef, float>::value;
  if constexpr (LEVEL == 0) dens_r2c_x_body<float, EX, 0, P2, false, kBatchScr, N>(B.X, tile);
  else if constexpr (LEVEL == 1) fft_strided_body<float, EPS, 2, P2, false, kBatchScr, N, WS>(B.S, tile, 0, B.tiles[1]);
  else if constexpr (LEVEL == 2) c2r_x_exp_cnx_body<float, Coef, EX, CL, 0, P2, false, kBatchScr, N>(B.X, tile);
  else cn_strided_body<float, Coef, CL, IMAG, kBatchScr, N, WCN>(B.C, tile, 0, B.tiles[3], 1);
}
template <int EX, int EPS, int CL, bool P2, int N>
__device__ __forceinline__ void batch_pass(const BProb &B, int level, int tile) {
  switch (level) {
    case 0: batch_body<EX, EPS, CL, P2, N, 0, float>(B, tile); break;
    case 1: batch_body<EX, EPS, CL, P2, N, 1, float>(B, tile); break;
    case 2:
      if (B.imag) batch_body<EX, EPS, CL, P2, N, 2, float>(B, tile);
      else batch_body<EX, EPS, CL, P2, N, 2, float2>(B, tile);
      break;
    default:
      if (B.imag) batch_body<EX, EPS, CL, P2, N, 3, float>(B, tile);
      else batch_body<EX, EPS, CL, P2, N, 3, float2>(B, tile);
  }
}
template <typename Coef>
__device__ __noinline__ void batch_resident(const BProb &B, int nsteps) {
  resident64_run<Coef>(B, nsteps);
}

__global__ void __launch_bounds__(DGPE_MAXT, 2)
    k_batch_run(const BProb *__restrict__ probs, const int4 *__restrict__ items, const int *__restrict__ counts,
                int L, const int *__restrict__ res, int nres, int nsteps, unsigned *sync, long long wait_limit) {
  __shared__ BProb sP;
  __shared__ int s_it[5];  // problem (-1: no work left), pass, first tile, run it, tile count
  int have = -1;           // problem whose arguments sP holds
  unsigned *const done = sync + BS_DONE;
  const long long total = (long long)nres + (long long)nsteps * L;
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned k = atomicAdd(sync + BS_TICKET, 1u);
      int p = -1, level = 0, tile = 0, go = 1, cnt = 1;
      unsigned need = 0;
      if ((long long)k < total) {
        if ((long long)k < nres) {
          p = res[k];
          level = 4;
        } else {
          const long long kk = (long long)k - nres;
          const int stp = (int)(kk / L);
          const int4 it = items[kk % L];
          p = it.x;
          level = it.y;
          tile = it.z;
          cnt = counts[kk % L];
          need = (unsigned)stp * (unsigned)probs[p].per_step + (unsigned)it.w;
        }
        // a problem held by the host never completes a tile (test hook)
        const unsigned hold = ld_acquire_u32(sync + BS_HOLD);
        const unsigned have_extra = (hold != 0u && (int)(hold - 1u) == p) ? 1u : 0u;
        if (need > 0 || have_extra) {
          long long polls = 0;
          while (ld_acquire_u32(done + p) < need + have_extra) {
            if (ld_acquire_u32(sync + BS_ABORT) != 0u || ++polls > wait_limit) {
              go = 0;
              atomicExch(sync + BS_ABORT, 1u);
              atomicExch(sync + BS_TIMEOUT, 1u);
              break;
            }
            __nanosleep(64);
          }
        }
        __threadfence();
      }
      s_it[0] = p; s_it[1] = level; s_it[2] = tile; s_it[3] = go; s_it[4] = cnt;
    }
    __syncthreads();
    const int p = s_it[0], level = s_it[1], tile0 = s_it[2], go = s_it[3], cnt = s_it[4];
    if (p < 0) break;
    if (go) {
      if (p != have) {
        const int *src = reinterpret_cast<const int *>(probs + p);
        int *dst = reinterpret_cast<int *>(&sP);
        for (int i = threadIdx.x; i < (int)(sizeof(BProb) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
        have = p;
        __syncthreads();
      }
      const BProb &B = sP;
      for (int tile = tile0; tile < tile0 + cnt; ++tile) {
      if (level == 4) {
        if (B.imag) batch_resident<float>(B, nsteps);
        else batch_resident<float2>(B, nsteps);
      } else if (B.var == VAR_P2 && B.n == 128) {
        batch_pass<8, 16, 16, true, 128>(B, level, tile);
      } else if (B.var == VAR_P2 && B.n == 256) {
        batch_pass<8, 16, 16, true, 256>(B, level, tile);
      } else if (B.var == VAR_P2 && B.n == 512) {
        batch_pass<8, 16, 16, true, 512>(B, level, tile);
      } else if (B.var == VAR_P2) {
        batch_pass<8, 16, 16, true, 0>(B, level, tile);
      } else if (B.var == VAR_3 && B.n == 96) {
        batch_pass<12, 12, 12, false, 96>(B, level, tile);
      } else if (B.var == VAR_3 && B.n == 384) {
        batch_pass<12, 12, 12, false, 384>(B, level, tile);
      } else if (B.var == VAR_3) {
        batch_pass<12, 12, 12, false, 0>(B, level, tile);
      } else if (B.var == VAR_5 && B.n == 160) {
        batch_pass<20, 20, 10, false, 160>(B, level, tile);
      } else {
        batch_pass<20, 20, 10, false, 0>(B, level, tile);
      }
      __syncthreads();
      }
      if (threadIdx.x == 0 && level != 4) {
        __threadfence();
        atomicAdd(done + p, (unsigned)cnt);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(sync + BS_EXIT, 1u) == gridDim.x - 1) {
      // every CTA has left: reset the counters for the next launch
      const int np = (int)sync[BS_NPROB];
      for (int q = 0; q < np; ++q) done[q] = 0u;
      sync[BS_TICKET] = 0u;
      sync[BS_EXIT] = 0u;
      sync[BS_ABORT] = 0u;
      __threadfence();
    }
  }
}

}  // namespace
}  // namespace dgpe

using namespace dgpe;

struct dgpe_batch {
  std::vector<Eng *> eng;
  std::vector<Cls> cls;
  cudaStream_t stream = nullptr, cap = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long sites = 0;
  double bytes = 0;
  std::string err;
  // persistent step (k_batch_run): problems, one step's work list, resident
  // problems, work-list state, launch shape, bound of every device wait
  BProb *dprobs = nullptr;
  int4 *ditems = nullptr;
  int *dcounts = nullptr;  // tiles of each item
  int *dres = nullptr;
  unsigned *dsync = nullptr;
  int L = 0, nres = 0, grid = 0;
  size_t smem = 0;
  long long wait_limit = 1ll << 22;
  bool classes = false;  // DGPE_FLAG_BATCH_CLASSES: per-class batched kernels in one graph
  ~dgpe_batch() {
    if (dprobs) cudaFree(dprobs);
    if (ditems) cudaFree(ditems);
    if (dcounts) cudaFree(dcounts);
    if (dres) cudaFree(dres);
    if (dsync) cudaFree(dsync);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto &c : cls) {
      if (c.dX) cudaFree(c.dX);
      if (c.dS) cudaFree(c.dS);
      if (c.dC) cudaFree(c.dC);
      if (c.st) cudaStreamDestroy(c.st);
      if (c.done) cudaEventDestroy(c.done);
    }
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    for (Eng *e : eng) delete e;
  }
};

namespace {

#define BCK(call)                                                                \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) { b->err = std::string(#call) + ": " + cudaGetErrorString(e_); return DGPE_ECUDA; } \
  } while (0)

// Raise the kernel's opt-in shared-memory limit to the device maximum (the
// limit belongs to the kernel, shared by every class that launches it).
template <typename K> cudaError_t attr(K k, size_t bytes) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k);
  if (e != cudaSuccess) return e;
  const size_t room = (size_t)optin - fa.sharedSizeBytes;
  if (bytes > room) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  return e;
}

// Fill the class's argument arrays for tile schedule (LP, sW, cW) and upload.
int configure(dgpe_batch *b, Cls &c, int LP, int sW, int cW) {
  Eng *e0 = b->eng[c.members[0]];
  const int n = c.n, TPL = e0->x_TPL, cl = e0->x_C;
  c.LP = LP;
  c.xT = 2 * LP * TPL;
  c.xgrid = ((e0->nrows + 1) / 2 + LP - 1) / LP;
  c.xs = sizeof(Cx) * (size_t)(LP * e0->x_pitchz + 2 * LP * e0->x_pitch);
  c.x4s = sizeof(Cx) * (size_t)(LP * e0->x_pitchz);
  const int es = variant_ept_s(c.var, Eng::EPT_S);
  c.sW = sW;
  c.sT = sW * n / es;
  c.sgrid = dim3((e0->ncol_spec + sW - 1) / sW, 1, (unsigned)c.members.size());
  c.ss = sizeof(Cx) * (size_t)n * sW;
  const int ctpl = n / cl;
  c.cW = cW;
  c.cT = cW * ctpl;
  c.cgrid = dim3((n + cW - 1) / cW, 1, (unsigned)c.members.size());
  c.cs = sizeof(Cx) * (size_t)cW * (n + n / cl + 1);
  std::vector<XArgs<float>> X;
  std::vector<SArgs<float>> S;
  std::vector<CArgs<float>> Cn;
  for (int i : c.members) {
    Eng *e = b->eng[i];
    XArgs<float> a = e->xargs();
    a.LP = LP;
    X.push_back(a);
    SArgs<float> s = e->sargs(e->fy);
    s.W = sW;
    S.push_back(s);
    CArgs<float> q{};
    const auto &cc = e->cn[1];
    q.psi = e->psi; q.cntab = e->cntab[1]; q.prm = e->prm; q.partial = e->partial; q.counter = e->counter;
    q.step = e->dstep; q.estride = cc.es; q.ostride = cc.os; q.n = cc.n; q.ncols = cc.ncols; q.W = cW;
    q.TPL = cc.TPL; q.C = cc.C; q.pitch = cc.pitch; q.final_pass = 1; q.norm = c.imag; q.tau = e->tau[1];
    q.cnd = e->cn_dlim[1];
    Cn.push_back(q);
  }
  BCK(cudaMemcpy(c.dX, X.data(), sizeof(XArgs<float>) * X.size(), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(c.dS, S.data(), sizeof(SArgs<float>) * S.size(), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(c.dC, Cn.data(), sizeof(CArgs<float>) * Cn.size(), cudaMemcpyHostToDevice));
  return DGPE_OK;
}

int launch_class(dgpe_batch *b, Cls &c, cudaStream_t s) {
  const unsigned cnt = (unsigned)c.members.size();
  const dim3 xg(c.xgrid, 1, cnt);
  int rc = with_xvar(c.var, [&](auto CLc, auto EXc, auto P2c) -> int {
    constexpr int CL = decltype(CLc)::value, EX = decltype(EXc)::value;
    constexpr bool P2 = decltype(P2c)::value;
    k_dens_r2c_x_batch<float, EX, P2><<<xg, c.xT, c.x4s, s>>>(c.dX);
    if (cudaPeekAtLastError() != cudaSuccess) return 1;
    with_svar<Eng::EPT_S>(c.var, [&](auto EPc, auto SP2c) -> int {
      constexpr int EP = decltype(EPc)::value;
      constexpr bool SP2 = decltype(SP2c)::value;
      k_fft_strided_batch<float, EP, 2, SP2><<<c.sgrid, c.sT, c.ss, s>>>(c.dS);
      return 0;
    });
    if (cudaPeekAtLastError() != cudaSuccess) return 2;
    if (c.imag) {
      k_c2r_x_exp_cnx_batch<float, float, EX, CL, P2><<<xg, c.xT, c.xs, s>>>(c.dX);
      if (cudaPeekAtLastError() != cudaSuccess) return 3;
      k_cn_strided_batch<float, float, CL><<<c.cgrid, c.cT, c.cs, s>>>(c.dC);
    } else {
      k_c2r_x_exp_cnx_batch<float, Cx, EX, CL, P2><<<xg, c.xT, c.xs, s>>>(c.dX);
      if (cudaPeekAtLastError() != cudaSuccess) return 3;
      k_cn_strided_batch<float, Cx, CL, false><<<c.cgrid, c.cT, c.cs, s>>>(c.dC);  // real time: no norm
    }
    if (cudaPeekAtLastError() != cudaSuccess) return 4;
    return 0;
  });
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    static const char *names[] = {"", "density/R2C", "FFT_y.U.IFFT_y", "C2R/exp/CN_x", "CN_y"};
    b->err = std::string("batched launch (n = ") + std::to_string(c.n) + ", " + names[rc > 0 && rc < 5 ? rc : 0] +
             "): " + cudaGetErrorString(e);
    return DGPE_ECUDA;
  }
  return DGPE_OK;
}

int set_attrs(dgpe_batch *b, const Cls &c) {
  cudaError_t e = cudaSuccess;
  with_xvar(c.var, [&](auto CLc, auto EXc, auto P2c) -> int {
    constexpr int CL = decltype(CLc)::value, EX = decltype(EXc)::value;
    constexpr bool P2 = decltype(P2c)::value;
    const size_t xs = std::max<size_t>(c.xs, 1);
    if (e == cudaSuccess) e = attr(k_dens_r2c_x_batch<float, EX, P2>, std::max<size_t>(c.x4s, 1));
    if (e == cudaSuccess) e = attr(k_c2r_x_exp_cnx_batch<float, float, EX, CL, P2>, xs);
    if (e == cudaSuccess) e = attr(k_c2r_x_exp_cnx_batch<float, Cx, EX, CL, P2>, xs);
    if (e == cudaSuccess) e = attr(k_cn_strided_batch<float, float, CL>, c.cs);
    if (e == cudaSuccess) e = attr(k_cn_strided_batch<float, Cx, CL, false>, c.cs);
    with_svar<Eng::EPT_S>(c.var, [&](auto EPc, auto SP2c) -> int {
      constexpr int EP = decltype(EPc)::value;
      constexpr bool SP2 = decltype(SP2c)::value;
      if (e == cudaSuccess) e = attr(k_fft_strided_batch<float, EP, 2, SP2>, c.ss);
      return 0;
    });
    return 0;
  });
  if (e != cudaSuccess) { b->err = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e); return DGPE_ECUDA; }
  return DGPE_OK;
}

// Tile shapes of the persistent step: every pass runs with DGPE_MAXT threads
// (x passes: LP = 128 / TPL; strided transform: W = DGPE_MAXT EPT / n columns;
// CN_y: W = DGPE_MAXT / TPL columns).
void persistent_shapes(const Cls &c, Eng *e0, int &LP, int &sW, int &cW) {
  LP = e0->x_LP;
  sW = DGPE_MAXT * variant_ept_s(c.var, Eng::EPT_S) / c.n;
  cW = DGPE_MAXT / (c.n / e0->cn[1].C);
}

// The distinct orders of a plan's radices (at most `cap`, the plan's own
// order first).
std::vector<FftPlan> radix_orders(const FftPlan &pl, size_t cap) {
  std::vector<int> r(pl.rad, pl.rad + pl.ns);
  std::sort(r.begin(), r.end());
  std::vector<FftPlan> out{pl};
  do {
    FftPlan q = pl;
    for (int k = 0; k < pl.ns; ++k) q.rad[k] = r[k];
    bool dup = false;
    for (auto &o : out) dup |= std::equal(o.rad, o.rad + o.ns, q.rad);
    if (!dup) out.push_back(q);
  } while (out.size() < cap && std::next_permutation(r.begin(), r.end()));
  return out;
}

// Autotuner: for each class time the candidate orders of the FFT radices
// (x transform and y transform, the Stockham stages in every order of the
// plan's radices) at the persistent step's tile shapes, on the class's own
// problems, and keep the fastest pair.  The timed steps advance the states,
// which the caller resets afterwards (create runs before any set_psi).
int autotune(dgpe_batch *b, Cls &c) {
  Eng *e0 = b->eng[c.members[0]];
  int LP, sW, cW;
  persistent_shapes(c, e0, LP, sW, cW);
  const std::vector<FftPlan> xs = radix_orders(e0->plx, 4), ys = radix_orders(e0->ply, 4);
  cudaEvent_t a, z;
  BCK(cudaEventCreate(&a));
  BCK(cudaEventCreate(&z));
  float best = 1e30f;
  FftPlan bx = e0->plx, by = e0->ply;
  for (const FftPlan &px : xs)
    for (const FftPlan &py : ys) {
      for (int i : c.members) { b->eng[i]->plx = px; b->eng[i]->ply = py; b->eng[i]->fy.pl = py; }
      int rc;
      if ((rc = configure(b, c, LP, sW, cW))) return rc;
      if ((rc = set_attrs(b, c))) return rc;
      if ((rc = launch_class(b, c, c.st))) return rc;  // warm-up
      BCK(cudaEventRecord(a, c.st));
      for (int r = 0; r < 3; ++r)
        if ((rc = launch_class(b, c, c.st))) return rc;
      BCK(cudaEventRecord(z, c.st));
      BCK(cudaEventSynchronize(z));
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, a, z));
      if (ms < best) { best = ms; bx = px; by = py; }
    }
  BCK(cudaEventDestroy(a));
  BCK(cudaEventDestroy(z));
  for (int i : c.members) { b->eng[i]->plx = bx; b->eng[i]->ply = by; b->eng[i]->fy.pl = by; }
  int rc;
  if ((rc = configure(b, c, LP, sW, cW))) return rc;
  return set_attrs(b, c);
}

// The persistent step's data: one BProb per problem (its pass arguments at
// the persistent tile shapes and tuned plans), one step's work list
// (pass-major, largest problems first within a pass), the resident problems,
// the launch shape and the work-list state.
int build_persistent(dgpe_batch *b) {
  const int np = (int)b->eng.size();
  std::vector<BProb> P(np);
  std::vector<int> res;
  size_t smem = (size_t)ResLayout::TOTAL;
  for (const Cls &c : b->cls) {
    Eng *e0 = b->eng[c.members[0]];
    int LP, sW, cW;
    persistent_shapes(c, e0, LP, sW, cW);
    for (int i : c.members) {
      Eng *e = b->eng[i];
      BProb &q = P[i];
      memset(&q, 0, sizeof(q));
      q.X = e->xargs();
      q.X.LP = LP;
      q.S = e->sargs(e->fy);
      q.S.W = sW;
      q.C.psi = e->psi; q.C.cntab = e->cntab[1]; q.C.prm = e->prm; q.C.partial = e->partial;
      q.C.counter = e->counter; q.C.step = e->dstep; q.C.estride = e->cn[1].es; q.C.ostride = e->cn[1].os;
      q.C.n = e->cn[1].n; q.C.ncols = e->cn[1].ncols; q.C.W = cW; q.C.TPL = e->cn[1].TPL; q.C.C = e->cn[1].C;
      q.C.pitch = e->cn[1].pitch; q.C.final_pass = 1; q.C.norm = c.imag; q.C.tau = e->tau[1];
      q.C.cnd = e->cn_dlim[1];
      q.var = c.var;
      q.imag = c.imag;
      q.n = c.n;
      q.resident = (c.n == kRes && c.var == VAR_P2) ? 1 : 0;
      q.tiles[0] = ((e->nrows + 1) / 2 + LP - 1) / LP;
      q.tiles[1] = (e->ncol_spec + sW - 1) / sW;
      q.tiles[2] = q.tiles[0];
      q.tiles[3] = (c.n + cW - 1) / cW;
      q.per_step = q.tiles[0] + q.tiles[1] + q.tiles[2] + q.tiles[3];
      if (q.resident) res.push_back(i);
      const size_t xs = sizeof(Cx) * (size_t)(LP * e->x_pitchz + 2 * LP * e->x_pitch);
      const size_t ss = sizeof(Cx) * (size_t)c.n * sW;
      const size_t cs = sizeof(Cx) * (size_t)cW * e->cn[1].pitch;
      if (!q.resident) smem = std::max(smem, std::max(xs, std::max(ss, cs)));
    }
  }
  // one step's items, pass-major, largest problems first within a pass
  std::vector<int> order;
  for (int i = 0; i < np; ++i)
    if (!P[i].resident) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return P[x].n > P[y].n; });
  // Items are ranges of consecutive tiles of one pass: about eight items per
  // CTA and step in all (fewer tickets, argument copies and waits), a
  // problem's pass never split below one tile per item.
  int dev0 = 0, nsm0 = 0;
  BCK(cudaGetDevice(&dev0));
  BCK(cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev0));
  long long total_tiles = 0;
  for (int i : order) total_tiles += P[i].per_step;
  const int chunk = (int)std::max<long long>(1, total_tiles / (8LL * 2 * nsm0));
  std::vector<int4> items;
  std::vector<int> counts;
  for (int lev = 0; lev < 4; ++lev)
    for (int i : order) {
      int before = 0;
      for (int l = 0; l < lev; ++l) before += P[i].tiles[l];
      const int nt = P[i].tiles[lev];
      const int nitems = (nt + chunk - 1) / chunk;
      for (int k = 0; k < nitems; ++k) {
        const int t0 = (int)((long long)nt * k / nitems), t1 = (int)((long long)nt * (k + 1) / nitems);
        items.push_back(make_int4(i, lev, t0, before));
        counts.push_back(t1 - t0);
      }
    }
  b->L = (int)items.size();
  b->nres = (int)res.size();
  b->smem = smem;
  BCK(cudaMalloc(&b->dprobs, sizeof(BProb) * np));
  BCK(cudaMemcpy(b->dprobs, P.data(), sizeof(BProb) * np, cudaMemcpyHostToDevice));
  BCK(cudaMalloc(&b->ditems, sizeof(int4) * std::max<size_t>(1, items.size())));
  if (!items.empty()) BCK(cudaMemcpy(b->ditems, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
  BCK(cudaMalloc(&b->dcounts, sizeof(int) * std::max<size_t>(1, counts.size())));
  if (!counts.empty()) BCK(cudaMemcpy(b->dcounts, counts.data(), sizeof(int) * counts.size(), cudaMemcpyHostToDevice));
  BCK(cudaMalloc(&b->dres, sizeof(int) * std::max<size_t>(1, res.size())));
  if (!res.empty()) BCK(cudaMemcpy(b->dres, res.data(), sizeof(int) * res.size(), cudaMemcpyHostToDevice));
  std::vector<unsigned> st(BS_DONE + np, 0u);
  st[BS_NPROB] = (unsigned)np;
  BCK(cudaMalloc(&b->dsync, sizeof(unsigned) * st.size()));
  BCK(cudaMemcpy(b->dsync, st.data(), sizeof(unsigned) * st.size(), cudaMemcpyHostToDevice));
  BCK(cudaFuncSetAttribute(k_batch_run, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int dev = 0, nsm = 0, occ = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_run, DGPE_MAXT, b->smem));
  if (occ < 1) { b->err = "the persistent batched step does not fit on a multiprocessor"; return DGPE_EUNSUPPORTED; }
  b->grid = nsm * occ;
  return DGPE_OK;
}

// DGPE_ETIMEOUT if a bounded wait of the persistent step ran out since the
// last check (the flag is cleared).  Synchronises.
int check_timeout(dgpe_batch *b) {
  if (!b->dsync) {
    BCK(cudaStreamSynchronize(b->stream));
    return DGPE_OK;
  }
  unsigned f = 0;
  BCK(cudaMemcpyAsync(&f, b->dsync + BS_TIMEOUT, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  if (f) {
    const unsigned zero = 0;
    BCK(cudaMemcpy(b->dsync + BS_TIMEOUT, &zero, sizeof(unsigned), cudaMemcpyHostToDevice));
    b->err = "a bounded device-side wait of the batched step ran out (the states are incomplete)";
    return DGPE_ETIMEOUT;
  }
  return DGPE_OK;
}

// The per-class form (DGPE_FLAG_BATCH_CLASSES): one step of every class as one
// graph; the capture stream forks into one branch per class (the class's own
// stream), the branches join back before the capture ends, so the classes'
// batched kernels run concurrently.  Kept for comparison with the persistent
// step (same arithmetic; 4 launches per class and step).
int capture(dgpe_batch *b) {
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
  int rc = DGPE_OK;
  if (cudaEventRecord(b->fork, b->cap) != cudaSuccess) rc = DGPE_ECUDA;
  for (auto &c : b->cls) {
    if (rc) break;
    if (cudaStreamWaitEvent(c.st, b->fork, 0) != cudaSuccess) { rc = DGPE_ECUDA; break; }
    if ((rc = launch_class(b, c, c.st))) break;
    if (cudaEventRecord(c.done, c.st) != cudaSuccess || cudaStreamWaitEvent(b->cap, c.done, 0) != cudaSuccess)
      rc = DGPE_ECUDA;
  }
  if (rc == DGPE_ECUDA) b->err = std::string("graph fork/join: ") + cudaGetErrorString(cudaGetLastError());
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) { b->err = std::string("capture: ") + cudaGetErrorString(e); return DGPE_ECUDA; }
  b->graph = g;
  BCK(cudaGraphInstantiate(&b->exec, g, 0));
  return DGPE_OK;
}

thread_local std::string g_batch_err;

}  // namespace

extern "C" int dgpe_batch_create(const dgpe_params *ps, int count, void *cuda_stream, dgpe_batch_t *out) {
  if (!out || !ps || count < 1) { g_batch_err = "bad arguments"; return DGPE_EINVAL; }
  *out = nullptr;
  dgpe_batch *b = new dgpe_batch();
  b->stream = (cudaStream_t)cuda_stream;
  cudaGetLastError();  // start from a clean error state
  std::map<std::pair<int, int>, int> index;
  for (int i = 0; i < count; ++i) {
    dgpe_params p = ps[i];
    if (p.flags & DGPE_FLAG_BATCH_CLASSES) b->classes = true;
    p.flags &= ~DGPE_FLAG_BATCH_CLASSES;
    if (p.dim != 2 || p.plane != DGPE_PLANE_XY || p.precision != DGPE_FP32_BULK || p.n[0] != p.n[1] ||
        (p.kernel != DGPE_KERNEL_QUASI2D_XY && p.kernel != DGPE_KERNEL_NONE)) {
      g_batch_err = "batch problems must be square 2D XY FP32-bulk grids";
      delete b;
      return DGPE_EUNSUPPORTED;
    }
    if (p.flags & (DGPE_FLAG_STRANG | DGPE_FLAG_REAL_PSI)) {
      g_batch_err = "batch problems use first-order splitting and a complex state";
      delete b;
      return DGPE_EUNSUPPORTED;
    }
    p.flags |= DGPE_FLAG_NO_GRAPH;
    if (p.n[0] < 32 || p.n[0] > 512 || !(p.h[0] > 0.0) || !(p.h[1] > 0.0) || !(p.dt > 0.0) ||
        (p.mode != DGPE_IMAG && p.mode != DGPE_REAL) || !(p.qd > 0.0)) {
      g_batch_err = std::string("problem ") + std::to_string(i) + ": invalid parameters";
      delete b;
      return DGPE_EINVAL;
    }
    b->eng.push_back(nullptr);
    Eng *e = new Eng();
    int rc = e->init(p, (cudaStream_t)cuda_stream);
    if (rc == DGPE_OK) {
      cudaError_t le = cudaGetLastError();
      if (le != cudaSuccess) { rc = DGPE_ECUDA; e->err = std::string("engine set-up: ") + cudaGetErrorString(le); }
    }
    if (rc) { g_batch_err = std::string("problem ") + std::to_string(i) + ": " + e->err; delete e; delete b; return rc; }
    if (!e->has_dip) {
      g_batch_err = "batch problems need the quasi-2D kernel";
      delete e;
      delete b;
      return DGPE_EUNSUPPORTED;
    }
    b->eng.back() = e;
    b->sites += (long long)e->nsites;
    for (int k = 0; k < e->launches_per_step(); ++k) b->bytes += e->pass_bytes(k);
    auto key = std::make_pair(p.n[0], p.mode == DGPE_IMAG ? 1 : 0);
    if (!index.count(key)) {
      index[key] = (int)b->cls.size();
      Cls c;
      c.n = p.n[0];
      c.imag = key.second;
      c.var = e->var[0];
      b->cls.push_back(c);
    }
    b->cls[index[key]].members.push_back(i);
  }
  auto fail = [&](int rc) { g_batch_err = b->err; delete b; return rc; };
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) { b->err = "stream"; return fail(DGPE_ECUDA); }
  for (auto &c : b->cls) {
    const size_t m = c.members.size();
    if (cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&c.dX, sizeof(XArgs<float>) * m) != cudaSuccess ||
        cudaMalloc(&c.dS, sizeof(SArgs<float>) * m) != cudaSuccess ||
        cudaMalloc(&c.dC, sizeof(CArgs<float>) * m) != cudaSuccess) {
      b->err = "allocation of the batch argument arrays failed";
      return fail(DGPE_ENOMEM);
    }
    int rc = autotune(b, c);
    if (rc) return fail(rc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { b->err = std::string("autotune (n = ") + std::to_string(c.n) + "): " + cudaGetErrorString(e); return fail(DGPE_ECUDA); }
  }
  {
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { b->err = std::string("after autotuning: ") + cudaGetErrorString(e); return fail(DGPE_ECUDA); }
  }
  // reset every problem (the autotuner stepped the zero states) and time
  for (Eng *e : b->eng) {
    int rc = e->set_time(0, b->stream);
    if (rc) { b->err = e->err; return fail(rc); }
  }
  int rc = b->classes ? capture(b) : build_persistent(b);
  if (rc) return fail(rc);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { b->err = std::string("after set-up: ") + cudaGetErrorString(e); return fail(DGPE_ECUDA); }
  }
  *out = b;
  return DGPE_OK;
}

extern "C" void dgpe_batch_destroy(dgpe_batch_t b) {
  if (!b) return;
  cudaDeviceSynchronize();
  delete b;
}

extern "C" int dgpe_batch_set_psi(dgpe_batch_t b, int i, const double *psi, size_t n_sites) {
  if (!b || i < 0 || i >= (int)b->eng.size() || !psi) return DGPE_EINVAL;
  if (n_sites != b->eng[i]->nsites) { b->err = "n_sites does not match"; return DGPE_EINVAL; }
  int rc = b->eng[i]->set_psi_host(psi, b->stream);
  if (rc) b->err = b->eng[i]->err;
  return rc;
}

extern "C" int dgpe_batch_get_psi(dgpe_batch_t b, int i, double *psi, size_t n_sites) {
  if (!b || i < 0 || i >= (int)b->eng.size() || !psi) return DGPE_EINVAL;
  if (n_sites != b->eng[i]->nsites) { b->err = "n_sites does not match"; return DGPE_EINVAL; }
  if (int tr = check_timeout(b)) return tr;
  int rc = b->eng[i]->get_psi_host(psi, b->stream);
  if (rc) b->err = b->eng[i]->err;
  return rc;
}

extern "C" int dgpe_batch_step(dgpe_batch_t b, int n) {
  if (!b || n < 0) return DGPE_EINVAL;
  if (n == 0) return DGPE_OK;
  if (b->classes) {
    for (int k = 0; k < n; ++k) {
      cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
      if (e != cudaSuccess) { b->err = std::string("graph launch: ") + cudaGetErrorString(e); return DGPE_ECUDA; }
    }
    return DGPE_OK;
  }
  k_batch_run<<<b->grid, DGPE_MAXT, b->smem, b->stream>>>(b->dprobs, b->ditems, b->dcounts, b->L, b->dres, b->nres, n,
                                                         b->dsync, b->wait_limit);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) { b->err = std::string("batched step launch: ") + cudaGetErrorString(e); return DGPE_ECUDA; }
  return DGPE_OK;
}

extern "C" int dgpe_batch_sync(dgpe_batch_t b) {
  if (!b) return DGPE_EINVAL;
  return check_timeout(b);
}

extern "C" int dgpe_batch_hold_problem(dgpe_batch_t b, int i) {
  if (!b || i < -1 || i >= (int)b->eng.size()) return DGPE_EINVAL;
  if (!b->dsync) { b->err = "no bounded waits in the per-class form"; return DGPE_EUNSUPPORTED; }
  const unsigned v = (unsigned)(i + 1);
  cudaError_t e = cudaMemcpyAsync(b->dsync + BS_HOLD, &v, sizeof(unsigned), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) { b->err = std::string("hold: ") + cudaGetErrorString(e); return DGPE_ECUDA; }
  return DGPE_OK;
}

extern "C" int dgpe_batch_set_wait_limit(dgpe_batch_t b, long long polls) {
  if (!b || polls < 1) return DGPE_EINVAL;
  b->wait_limit = polls;
  return DGPE_OK;
}

extern "C" int dgpe_batch_observables(dgpe_batch_t b, int i, dgpe_obs *o) {
  if (!b || i < 0 || i >= (int)b->eng.size() || !o) return DGPE_EINVAL;
  if (int tr = check_timeout(b)) return tr;
  int rc = b->eng[i]->observables(o, b->stream);
  if (rc) b->err = b->eng[i]->err;
  return rc;
}

extern "C" int dgpe_batch_info(dgpe_batch_t b, int *classes, long long *sites, double *bytes_per_step) {
  if (!b) return DGPE_EINVAL;
  if (classes) *classes = (int)b->cls.size();
  if (sites) *sites = b->sites;
  if (bytes_per_step) *bytes_per_step = b->bytes;
  return DGPE_OK;
}

// one launch of the persistent step per dgpe_batch_step call, whatever n
extern "C" int dgpe_batch_launches_per_step(dgpe_batch_t b) {
  return b ? (b->classes ? 4 * (int)b->cls.size() : 1) : 0;
}

extern "C" const char *dgpe_batch_last_error(dgpe_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }
