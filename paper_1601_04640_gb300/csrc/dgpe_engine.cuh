// dgpe_engine.cuh -- host runtime of one solver: FP64 precompute of the
// tables (dipolar kernel U(k)/N, Crank-Nicolson LU and scan tables, FFT
// roots, trap potential), pass configuration, launch sequence and CUDA-graph
// capture.  Instantiated for double (FP64 form) and float (FP32-bulk form).
#pragma once

#include <algorithm>
#include <cmath>
#include <complex>
#include <type_traits>
#include <cstring>
#include <string>
#include <vector>

#include "dgpe.h"
#include "dgpe_kernels.cuh"

namespace dgpe {

typedef std::complex<double> zd;

// Engine interface used by the C ABI.
struct Engine {
  virtual ~Engine() {}
  virtual int init(const dgpe_params &p, cudaStream_t user) = 0;
  virtual int set_psi_device(const void *src, int fp64, cudaStream_t s) = 0;
  virtual int get_psi_device(void *dst, int fp64, cudaStream_t s) = 0;
  virtual int set_psi_host(const double *src, cudaStream_t s) = 0;
  virtual int get_psi_host(double *dst, cudaStream_t s) = 0;
  virtual int step(int n, cudaStream_t s) = 0;
  virtual int observables(dgpe_obs *o, cudaStream_t s) = 0;
  virtual int dipolar_potential(double *phi_host, cudaStream_t s) = 0;
  virtual int set_g(double g, cudaStream_t s) = 0;
  virtual int set_mode(int mode, cudaStream_t s) = 0;
  virtual int set_modulation(const double *c, int M, cudaStream_t s) = 0;
  virtual int set_time(long long step, cudaStream_t s) = 0;
  virtual int get_time(long long *step, cudaStream_t s) = 0;
  virtual int launches_per_step() const = 0;
  virtual int profile_steps(int n, double *pass_ms, int cap, cudaStream_t s) = 0;
  virtual int step_adjoint(const void *psi_in, void *G, long long step, double *dg, double *dc,
                           cudaStream_t s) = 0;
  virtual int fidelity_gradient(const double *psi0, const double *target, int nsteps, int every,
                                double *F, double *dFdg, double *dFdc, cudaStream_t s) = 0;
  virtual const char *pass_name(int i) const = 0;
  virtual double pass_bytes(int i) const = 0;
  virtual double pass_flops(int i) const = 0;
  virtual long long kernel_launches() const = 0;
  virtual size_t sites() const = 0;
  // DGPE_ETIMEOUT if a kernel's bounded wait ran out since the last set_psi
  virtual int wait_status(cudaStream_t s) = 0;
  std::string err;
};

Engine *make_engine_f64();
Engine *make_engine_f32();

// Everything below has internal linkage: each translation unit gets its own
// solver template and kernels (see dgpe_kernels.cuh).
namespace {

// ----------------------------------------------------------- host helpers
// Radix sequence for length n whose radices divide ept (largest first).
inline bool make_plan(int n, int ept, FftPlan &pl) {
  static const int cand[6] = {16, 8, 5, 4, 3, 2};
  pl.n = n;
  pl.ns = 0;
  int m = n;
  for (int ci = 0; ci < 6; ++ci) {
    const int R = cand[ci];
    while (m % R == 0 && ept % R == 0) {
      if (pl.ns >= 10) return false;
      pl.rad[pl.ns++] = R;
      m /= R;
    }
  }
  return m == 1 && pl.ns > 0;
}

// Kernel variant of one axis length n: CN chunk length CL (n / CL lanes per
// line, a power of two <= 32), elements per thread of the x-line and strided
// FFTs, and whether n is a power of two (shift/mask index arithmetic).
//   powers of two: CL 16, EPT_X 8, EPT_S 8 (FP64) / 16 (FP32)
//   3 * 2^k:       CL 12, EPT_X 12, EPT_S 12  (radices 4, 3, 2)
//   5 * 2^k:       CL 10, EPT_X 20, EPT_S 20  (radices 5, 4, 2)
//   (VAR_P2S: CL 8 for short power-of-two lines; measured slower, unused)
enum { VAR_P2 = 0, VAR_3 = 1, VAR_5 = 2, VAR_P2S = 3, VAR_NONE = -1 };
inline bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
inline int axis_variant(int n) {
  if (is_pow2(n) && n >= 32 && n <= 512) return VAR_P2;
  if (n % 3 == 0 && is_pow2(n / 3) && n / 12 >= 1 && n / 12 <= 32 && n % 12 == 0) return VAR_3;
  if (n % 5 == 0 && is_pow2(n / 5) && n % 10 == 0 && n / 10 <= 32) return VAR_5;
  return VAR_NONE;
}
inline int variant_cl(int v) { return v == VAR_P2 ? 16 : v == VAR_P2S ? 8 : v == VAR_3 ? 12 : 10; }

// Call f(CL, EPT_X, POW2) with compile-time constants for variant v.
template <class F> int with_xvar(int v, F &&f) {
  switch (v) {
    case VAR_P2: return f(std::integral_constant<int, 16>{}, std::integral_constant<int, 8>{}, std::true_type{});
    case VAR_P2S: return f(std::integral_constant<int, 8>{}, std::integral_constant<int, 8>{}, std::true_type{});
    case VAR_3: return f(std::integral_constant<int, 12>{}, std::integral_constant<int, 12>{}, std::false_type{});
    default: return f(std::integral_constant<int, 10>{}, std::integral_constant<int, 20>{}, std::false_type{});
  }
}
// Call f(EPT_S, POW2) for the strided FFT of variant v (pow2 EPT_S given).
template <int EPTP2, class F> int with_svar(int v, F &&f) {
  switch (v) {
    case VAR_P2:
    case VAR_P2S: return f(std::integral_constant<int, EPTP2>{}, std::true_type{});
    case VAR_3: return f(std::integral_constant<int, 12>{}, std::false_type{});
    default: return f(std::integral_constant<int, 20>{}, std::false_type{});
  }
}
// Call f(CL) for the CN chunk of variant v.
template <class F> int with_cl(int v, F &&f) {
  switch (v) {
    case VAR_P2: return f(std::integral_constant<int, 16>{});
    case VAR_P2S: return f(std::integral_constant<int, 8>{});
    case VAR_3: return f(std::integral_constant<int, 12>{});
    default: return f(std::integral_constant<int, 10>{});
  }
}
inline int variant_ept_x(int v) { return (v == VAR_P2 || v == VAR_P2S) ? 8 : v == VAR_3 ? 12 : 20; }
inline int variant_ept_s(int v, int p2) { return (v == VAR_P2 || v == VAR_P2S) ? p2 : v == VAR_3 ? 12 : 20; }

// erfcx(u) = exp(u^2) erfc(u) for u >= 0; continued asymptotic series where
// erfc underflows.
inline double host_erfcx(double u) {
  if (u < 25.0) return std::exp(u * u) * std::erfc(u);
  const double u2 = u * u;
  double term = 1.0, sum = 1.0;
  for (int m = 1; m < 8; ++m) {
    term *= -(2.0 * m - 1.0) / (2.0 * u2);
    sum += term;
  }
  return sum / (u * std::sqrt(M_PI));
}

inline double wavenumber(int j, int n, double h) {
  const int jj = (j <= n / 2) ? j : j - n;
  return 2.0 * M_PI * (double)jj / ((double)n * h);
}

#define DGPE_LCK(name)                                                       \
  do {                                                                       \
    cudaError_t e_ = cudaGetLastError();                                     \
    if (e_ != cudaSuccess) {                                                 \
      err = std::string("launch of ") + (name) + ": " + cudaGetErrorString(e_); \
      return DGPE_ECUDA;                                                     \
    }                                                                        \
  } while (0)

#define DGPE_CK(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      err = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      return (e_ == cudaErrorMemoryAllocation) ? DGPE_ENOMEM : DGPE_ECUDA;   \
    }                                                                        \
  } while (0)

#ifndef DGPE_EPT_S_F64
#define DGPE_EPT_S_F64 8  // FP64 strided transforms: elements per thread (power-of-two lengths)
#endif
#ifndef DGPE_FFT_FMA_F32
#define DGPE_FFT_FMA_F32 0  // FP32 density and strided transforms in FMA form too (measured 3 % slower)
#endif
// cuTensorMapEncodeTiled from the driver, found once through the runtime's
// entry-point query (no link-time dependency on the driver library).
typedef CUresult (*TensorMapEncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                           const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                           CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                           CUtensorMapFloatOOBfill);
inline TensorMapEncodeTiledFn tensor_map_encoder() {
  static TensorMapEncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<TensorMapEncodeTiledFn>(p);
  }();
  return fn;
}

// Call f(N) with N = n as a compile-time constant for the power-of-two line
// lengths of the length-specialised kernels (0 when n is not one of them).
template <class F> int with_pow2_len(int n, F &&f) {
  switch (n) {
    case 32: return f(std::integral_constant<int, 32>{});
    case 64: return f(std::integral_constant<int, 64>{});
    case 128: return f(std::integral_constant<int, 128>{});
    case 256: return f(std::integral_constant<int, 256>{});
    case 512: return f(std::integral_constant<int, 512>{});
    default: return f(std::integral_constant<int, 0>{});
  }
}

template <typename R> struct EngineT : Engine {
  typedef cx<R> Cx;
  static constexpr int EPT_S = sizeof(R) == 8 ? DGPE_EPT_S_F64 : 16;  // strided FFTs, power-of-two lengths
  int var[3] = {VAR_P2, VAR_P2, VAR_P2};           // kernel variant per axis
  static constexpr int PW = 128 / (int)sizeof(Cx); // pad period of line-major tiles
  static constexpr int W = 128 / (int)sizeof(Cx);  // columns per strided tile (128 B)

  dgpe_params p{};
  int dim = 3, nx = 0, ny = 0, nz = 1, nrows = 0, px = 0, ncol_spec = 0;
  size_t nsites = 0, nspec = 0;
  bool has_dip = false;
  int imag = 1;

  Cx *psi = nullptr, *spec = nullptr;
  R *U = nullptr, *phi_tmp = nullptr;
  Cx *tw[3] = {nullptr, nullptr, nullptr};
  // FMA-form roots per axis (forward and inverse): (t, fx, fy, swap), built in FP64
  rt4<R> *twf[3] = {nullptr, nullptr, nullptr}, *twi[3] = {nullptr, nullptr, nullptr};
  R *vt[3] = {nullptr, nullptr, nullptr};
  void *cntab[3] = {nullptr, nullptr, nullptr};
  double *prm = nullptr, *partial = nullptr, *obs_part = nullptr, *dip_part = nullptr, *obs_out = nullptr;
  double2 *stage = nullptr;  // FP64 staging buffer for host transfers (lazy)
  // reverse-mode buffers (allocated on first use)
  Cx *adjG = nullptr, *adjT = nullptr;
  R *adj_phi = nullptr, *adj_sig = nullptr, *adj_ksig = nullptr;
  double *adj_part = nullptr, *adj_acc = nullptr;
  void *cntab_adj[3] = {nullptr, nullptr, nullptr};
  std::vector<Cx *> ckpts, states;
  double host_cm[16] = {0};
  int host_M = 0;
  long long *dstep = nullptr;
  unsigned *counter = nullptr;
  FftPlan plx{}, ply{}, plz{}, plx_s{};
  double tau[3] = {0, 0, 0};
  // chunk-scan reach of the FP32 chunk-parallel CN solve per axis (cn_line_st)
  int cn_dlim[3] = {0, 0, 0};

  // pass configurations
  int x_LP = 0, x_T = 0, x_TPL = 0, x_C = 0, x_pitchz = 0, x_pitch = 0, x_grid = 0;
  size_t x_smem = 0, x4_smem = 0;  // the C2R/exp/CN pass; the density pass (Z tile only)
  // FP32 bulk, complex state, power-of-two nx: the pipelined x-line pass
  // (k_p1_pipe, persistent CTAs fed by bulk copies); grid and shared memory
  bool p1_pipe = false;
  int p1_grid[2] = {0, 0};  // real, complex CN coefficients
  size_t p1_smem[2] = {0, 0};
  // ... and the pipelined density / R2C pass (k_p4_pipe)
  bool p4_pipe = false;
  int p4_grid = 0;
  size_t p4_smem = 0;
  // ... and the TMA-tiled strided transforms (k_fft_tma): tensor maps of the
  // half spectrum for lines along y and along z
  bool tma_fft = false;
  CUtensorMap tm_y{}, tm_z{};
  struct CnCfg {
    int n, ncols, W, TPL, C, pitch, T;
    long long es, os;
    dim3 grid;
    size_t smem;   // one tile
    int pgrid[2];  // persistent grid of the double-buffered kernel (real, complex coefficients)
  };
  int nsm = 1;
  CnCfg cn[3];   // index = axis (0 unused: x is fused into P1)
  // line-serial CN (one thread per line, k_cn_lines), used by the FP64 form on
  // grids with enough lines to fill the GPU; x is then a pass of its own
  struct LnCfg { int n, ncols, T; long long es, cs, os; dim3 grid; };
  LnCfg ln[3];
  bool cn_serial = false;
  // kernels this solver has launched (a graph replay counts its kernels;
  // launches recorded into a capture are not counted)
  long long nlaunch = 0;
  bool capturing = false;
  void launched(int k) { if (!capturing) nlaunch += k; }
  long long kernel_launches() const override { return nlaunch; }
  struct FtCfg { int n, T, W; long long es, os; dim3 grid; size_t smem; FftPlan pl; int axis; };
  FtCfg fy{}, fz{};
  int obs_rows = 1, obs_blocks = 0, ndip = 0;

  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool use_graph = true;
  bool strang = false;  // second-order splitting (real time)
  // real state (imaginary time): psi holds nx reals per row, viewed by the
  // strided CN passes as nx/2 complex columns (pairs of real lines)
  bool rpsi = false;
  Cx *ocx = nullptr;  // complex copy of a real state for the observables

  ~EngineT() override {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    void *bufs[] = {psi, spec, U, phi_tmp, tw[0], tw[1], tw[2], vt[0], vt[1], vt[2],
                    cntab[0], cntab[1], cntab[2], prm, partial, obs_part, dip_part, obs_out,
                    dstep, counter, stage, adjG, adjT, adj_phi, adj_sig, adj_ksig, adj_part,
                    adj_acc, cntab_adj[0], cntab_adj[1], cntab_adj[2], twf[0], twf[1], twf[2],
                    twi[0], twi[1], twi[2], ocx};
    for (void *b : bufs)
      if (b) cudaFree(b);
    for (Cx *b : ckpts) cudaFree(b);
    for (Cx *b : states) cudaFree(b);
  }

  size_t sites() const override { return nsites; }
  // complex elements of the state buffer (a real state packs two sites in one)
  size_t psi_elems() const { return rpsi ? nsites / 2 : nsites; }
  int row_cx() const { return rpsi ? nx / 2 : nx; }  // complex elements per x row

  int launches_per_step() const override {
    int k = 1 + (dim == 3 ? 2 : 1) + (cn_serial ? 1 : 0);  // P1, CN passes
    if (has_dip) k += (dim == 3 ? 4 : 2);
    return k;
  }

  template <typename T> int dalloc(T **ptr, size_t count) {
    DGPE_CK(cudaMalloc((void **)ptr, sizeof(T) * (count ? count : 1)));
    return DGPE_OK;
  }
  template <typename T> int upload(T *dst, const std::vector<T> &src) {
    DGPE_CK(cudaMemcpy(dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice));
    return DGPE_OK;
  }

  // ---------------------------------------------------------------- init
  int init(const dgpe_params &pin, cudaStream_t user) override {
    p = pin;
    dim = p.dim;
    nx = p.n[0];
    ny = p.n[1];
    nz = (dim == 3) ? p.n[2] : 1;
    nrows = ny * nz;
    nsites = (size_t)nx * ny * nz;
    imag = (p.mode == DGPE_IMAG);
    has_dip = (p.kernel != DGPE_KERNEL_NONE);
    rpsi = (p.flags & DGPE_FLAG_REAL_PSI) != 0;
    if (rpsi && !imag) { err = "a real state is an imaginary-time option"; return DGPE_EUNSUPPORTED; }
    px = nx / 2 + 1;
    if (sizeof(Cx) == 8) px = (px + 1) & ~1;  // 16-byte rows for FP32 complex
    ncol_spec = nx / 2 + 1;
    nspec = (size_t)px * nrows;

    // kernel variants and FFT plans
    const int nsz[3] = {nx, ny, nz};
    for (int a = 0; a < dim; ++a) {
      var[a] = axis_variant(nsz[a]);
      if (var[a] == VAR_NONE) {
        err = "grid length not supported (powers of two, 3*2^k or 5*2^k, 32..512)";
        return DGPE_EUNSUPPORTED;
      }
    }
    if (!make_plan(nx, variant_ept_x(var[0]), plx) || !make_plan(ny, variant_ept_s(var[1], EPT_S), ply) ||
        (dim == 3 && !make_plan(nz, variant_ept_s(var[2], EPT_S), plz))) {
      err = "grid size not supported by the FFT plans";
      return DGPE_EUNSUPPORTED;
    }
    int rc;
    if ((rc = dalloc(&psi, psi_elems()))) return rc;
    DGPE_CK(cudaMemset(psi, 0, sizeof(Cx) * psi_elems()));
    if (has_dip && (rc = dalloc(&spec, nspec))) return rc;
    if ((rc = dalloc(&prm, PRM_COUNT))) return rc;
    if ((rc = dalloc(&dstep, 1))) return rc;
    if ((rc = dalloc(&counter, 1))) return rc;
    DGPE_CK(cudaMemset(dstep, 0, sizeof(long long)));
    DGPE_CK(cudaMemset(counter, 0, sizeof(unsigned)));
    std::vector<double> hp(PRM_COUNT, 0.0);
    hp[PRM_SC] = 1.0;
    hp[PRM_DT] = p.dt;
    hp[PRM_G] = p.g;
    hp[PRM_GDD] = p.gdd;
    hp[PRM_CELL] = p.h[0] * p.h[1] * (dim == 3 ? p.h[2] : 1.0);
    if ((rc = upload(prm, hp))) return rc;

    // twiddles and potential tables
    const int ns[3] = {nx, ny, nz};
    for (int a = 0; a < dim; ++a) {
      std::vector<Cx> w(ns[a]);
      for (int t = 0; t < ns[a]; ++t) {
        const double ang = -2.0 * M_PI * (double)t / (double)ns[a];
        w[t].x = (R)std::cos(ang);
        w[t].y = (R)std::sin(ang);
      }
      if ((rc = dalloc(&tw[a], ns[a]))) return rc;
      if ((rc = upload(tw[a], w))) return rc;
      {
        // root c + i s of exp(-+2 pi i t/n): |c| >= |s| -> (s/c, c, c, 0);
        // else the root is i (s - i c) -> (-c/s, -s, s, 1)
        for (int dir = 0; dir < 2; ++dir) {
          std::vector<rt4<R>> f(ns[a]);
          for (int t = 0; t < ns[a]; ++t) {
            const double ang = (dir ? 2.0 : -2.0) * M_PI * (double)t / (double)ns[a];
            const double c = std::cos(ang), sn = std::sin(ang);
            const bool sw = !(std::fabs(c) >= std::fabs(sn));
            f[t].x = (R)(sw ? -c / sn : sn / c);
            f[t].y = (R)(sw ? -sn : c);
            f[t].z = (R)(sw ? sn : c);
            f[t].w = (R)(sw ? 1.0 : 0.0);
          }
          rt4<R> **dst = dir ? &twi[a] : &twf[a];
          if ((rc = dalloc(dst, ns[a]))) return rc;
          if ((rc = upload(*dst, f))) return rc;
        }
      }
    }
    for (int a = 0; a < 3; ++a) {
      const int n = (a < dim) ? ns[a] : 1;
      std::vector<R> v(n, (R)0);
      if (a < dim)
        for (int i = 0; i < n; ++i) {
          const double x = ((double)i - (double)(n / 2)) * p.h[a];
          v[i] = (R)(0.5 * p.nu[a] * p.nu[a] * x * x);
        }
      if ((rc = dalloc(&vt[a], n))) return rc;
      if ((rc = upload(vt[a], v))) return rc;
    }
    if (has_dip && (rc = build_kernel_table())) return rc;

    // configurations
    x_C = variant_cl(var[0]);
    if (nx % x_C) { err = "nx is not a multiple of the CN chunk"; return DGPE_EUNSUPPORTED; }
    x_TPL = nx / x_C;
    if (x_TPL > 32) { err = "nx > 512 not supported"; return DGPE_EUNSUPPORTED; }
    x_LP = std::max(1, (sizeof(R) == 8 ? 64 : DGPE_MAXT / 2) / x_TPL);
    x_T = 2 * x_LP * x_TPL;
    x_pitchz = nx + nx / PW + 1;
    x_pitch = nx + nx / x_C + 1;
    x_smem = sizeof(Cx) * (size_t)(x_LP * x_pitchz + 2 * x_LP * x_pitch);
    x4_smem = sizeof(Cx) * (size_t)(x_LP * x_pitchz);
    {
      const int npairs = (nrows + 1) / 2;
      x_grid = (npairs + x_LP - 1) / x_LP;
    }
    if ((rc = make_cn_cfg(1))) return rc;
    if (dim == 3 && (rc = make_cn_cfg(2))) return rc;
    if ((rc = choose_cn_form())) return rc;
    if ((rc = build_cn_tables())) return rc;
    fy.axis = 1;
    fz.axis = 2;
    if (has_dip) {
      // y transform over the spectrum
      // tile width W columns (128 B rows), narrowed (by powers of two) so
      // blocks stay <= DGPE_MAXT threads
      auto wfor = [&](int n, int ept) {
        int w = (sizeof(R) == 4) ? DGPE_W_FFT_F32 : W;
        while (w > 1 && w * n / ept > DGPE_MAXT_FFT) w >>= 1;
        return w;
      };
      const int ey = variant_ept_s(var[1], EPT_S);
      fy.n = ny; fy.W = wfor(ny, ey); fy.T = fy.W * ny / ey; fy.es = px; fy.os = (long long)ny * px;
      fy.grid = dim3((ncol_spec + fy.W - 1) / fy.W, nz); fy.smem = sizeof(Cx) * (size_t)ny * fy.W; fy.pl = ply;
      if (dim == 3) {
        const int ez = variant_ept_s(var[2], EPT_S);
        fz.n = nz; fz.W = wfor(nz, ez); fz.T = fz.W * nz / ez; fz.es = (long long)ny * px; fz.os = px;
        fz.grid = dim3((ncol_spec + fz.W - 1) / fz.W, ny); fz.smem = sizeof(Cx) * (size_t)nz * fz.W; fz.pl = plz;
      }
      if (fy.T > DGPE_MAXT_FFT || fz.T > DGPE_MAXT_FFT) { err = "strided FFT block too large"; return DGPE_EUNSUPPORTED; }
    }
    // scratch: norm partials, observable partials
    obs_blocks = (int)std::min<size_t>(152 * 8, (nsites + 255) / 256);
    const FtCfg &last = (dim == 3) ? fz : fy;
    ndip = has_dip ? (int)(last.grid.x * last.grid.y) : 0;
    const CnCfg &fin = cn[dim == 3 ? 2 : 1];
    const LnCfg &lfin = ln[dim == 3 ? 2 : 1];
    // norm partials of the final pass (twice its default grid: a batch may run
    // the pass with half-width tiles)
    if ((rc = dalloc(&partial, std::max(2 * (size_t)fin.grid.x * fin.grid.y,
                                        cn_serial ? (size_t)lfin.grid.x * lfin.grid.y : (size_t)0)))) return rc;
    if ((rc = dalloc(&obs_part, (size_t)obs_blocks * OBS_COUNT))) return rc;
    if ((rc = dalloc(&dip_part, (size_t)std::max(ndip, 1)))) return rc;
    if ((rc = dalloc(&obs_out, OBS_COUNT + 1))) return rc;
    if ((rc = set_smem_attrs())) return rc;
    DGPE_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    use_graph = !(p.flags & DGPE_FLAG_NO_GRAPH);
    strang = (p.flags & DGPE_FLAG_STRANG) != 0;
    if (use_graph && (rc = capture())) return rc;
    (void)user;
    return DGPE_OK;
  }

  // The FP64 form solves each line serially once there are enough lines for
  // one warp per SM sub-partition at least (it is FP64-pipe-bound, and the
  // serial solve does half the arithmetic); flags force either form.
  int choose_cn_form() {
    const size_t lines_min = nsites / (size_t)std::max(nx, std::max(ny, nz));
    if ((p.flags & DGPE_FLAG_CN_SERIAL) && (p.flags & DGPE_FLAG_CN_CHUNKED)) {
      err = "DGPE_FLAG_CN_SERIAL and DGPE_FLAG_CN_CHUNKED are exclusive";
      return DGPE_EINVAL;
    }
    if (sizeof(R) == 4 || rpsi) {
      if (p.flags & DGPE_FLAG_CN_SERIAL) {
        err = rpsi ? "a real state uses the chunk-parallel CN solve" : "the line-serial CN solve is an FP64-form option";
        return DGPE_EUNSUPPORTED;
      }
      cn_serial = false;
    } else if (p.flags & DGPE_FLAG_CN_SERIAL) cn_serial = true;
    else if (p.flags & DGPE_FLAG_CN_CHUNKED) cn_serial = false;
    else cn_serial = lines_min >= 8192;
    const int ns[3] = {nx, ny, nz};
    for (int a = 0; a < dim; ++a) {
      LnCfg &L = ln[a];
      L.n = ns[a];
      if (a == 0) { L.ncols = (int)nrows; L.es = 1; L.cs = nx; L.os = 0; }
      else if (a == 1) { L.ncols = nx; L.es = nx; L.cs = 1; L.os = (long long)nx * ny; }
      else { L.ncols = nx; L.es = (long long)nx * ny; L.cs = 1; L.os = nx; }
      L.T = std::min(DGPE_LINES_T, (L.ncols + 31) / 32 * 32);
      const unsigned outer = (a == 0) ? 1u : (a == 1 ? (unsigned)nz : (unsigned)ny);
      L.grid = dim3((unsigned)((L.ncols + L.T - 1) / L.T), outer);
    }
    return DGPE_OK;
  }
  int make_cn_cfg(int axis) {
    CnCfg &c = cn[axis];
    const int n = (axis == 1) ? ny : nz;
    c.n = n;
    const int xw = row_cx();
    c.ncols = xw;
    const int cl = variant_cl(var[axis]);
    const int tpl = n / cl;
    if (tpl < 1 || tpl > 32 || n % cl || !is_pow2(tpl)) { err = "line length not supported by the CN chunking"; return DGPE_EUNSUPPORTED; }
    c.TPL = tpl;
    c.C = cl;
    c.W = std::min(W, DGPE_MAXT / tpl);  // blocks of at most DGPE_MAXT threads
    c.pitch = n + n / c.C + 1;
    c.T = c.W * tpl;
    if (axis == 1) { c.es = xw; c.os = (long long)xw * ny; c.grid = dim3((xw + c.W - 1) / c.W, nz); }
    else { c.es = (long long)xw * ny; c.os = xw; c.grid = dim3((xw + c.W - 1) / c.W, ny); }
    c.smem = sizeof(Cx) * (size_t)c.W * c.pitch;
    return DGPE_OK;
  }

  // U(k)/N on the half spectrum [z][y][kx], FP64 then rounded to R.
  int build_kernel_table() {
    std::vector<R> hu(nspec, (R)0);
    const double N = (double)nsites;
    for (int kz = 0; kz < nz; ++kz)
      for (int ky = 0; ky < ny; ++ky)
        for (int kx = 0; kx < ncol_spec; ++kx) {
          const double qx = wavenumber(kx, nx, p.h[0]), qy = wavenumber(ky, ny, p.h[1]);
          double u;
          if (dim == 3) {
            const double qz = wavenumber(kz, nz, p.h[2]);
            const double k2 = qx * qx + qy * qy + qz * qz;
            u = (k2 == 0.0) ? 0.0 : (4.0 * M_PI / 3.0) * (3.0 * qz * qz / k2 - 1.0);
          } else if (p.kernel == DGPE_KERNEL_QUASI2D_XZ) {
            // (x, z) plane (the second axis is z), dipoles along z in the
            // plane, Gaussian y-profile exp(-y^2/d^2)/(sqrt(pi) d):
            // U2 = (4pi/3)/(sqrt(2pi) d) [3 sqrt(pi/2) (kz^2 d/krho) erfcx(krho d/sqrt2) - 1]
            const double d = p.qd, qz = qy, krho = std::sqrt(qx * qx + qz * qz);
            const double pref = (4.0 * M_PI / 3.0) / (std::sqrt(2.0 * M_PI) * d);
            u = (krho == 0.0) ? -pref
                              : pref * (3.0 * std::sqrt(M_PI / 2.0) * (qz * qz * d / krho) *
                                            host_erfcx(krho * d / std::sqrt(2.0)) - 1.0);
          } else {
            // dipoles along z, Gaussian z-profile exp(-z^2/d^2)/(sqrt(pi) d):
            // U2 = (4pi/3)/(sqrt(2pi) d) [2 - 3 sqrt(pi/2) q erfcx(q/sqrt2)], q = k d
            const double d = p.qd, q = std::sqrt(qx * qx + qy * qy) * d;
            u = (4.0 * M_PI / 3.0) / (std::sqrt(2.0 * M_PI) * d) *
                (2.0 - 3.0 * std::sqrt(M_PI / 2.0) * q * host_erfcx(q / std::sqrt(2.0)));
          }
          hu[((size_t)kz * ny + ky) * px + kx] = (R)(u / N);
        }
    int rc;
    if ((rc = dalloc(&U, nspec))) return rc;
    return upload(U, hu);
  }

  // Crank-Nicolson LU and chunk-scan tables for axis a: m, alpha, P, Q (n
  // each), then the middle-row pivot mu of the two-ended elimination.
  int build_cn_tables() {
    const int ns[3] = {nx, ny, nz};
    const int Cs[3] = {x_C, cn[1].C, dim == 3 ? cn[2].C : 1};
    for (int a = 0; a < dim; ++a) {
      const int n = ns[a], C = Cs[a];
      tau[a] = p.dt / (4.0 * p.h[a] * p.h[a]);
      const zd kt = imag ? zd(tau[a], 0.0) : zd(0.0, tau[a]);
      std::vector<zd> m(n), al(n), P(n), Q(n);
      const zd b = 1.0 + 2.0 * kt;
      m[0] = 1.0 / b;
      for (int i = 1; i < n; ++i) m[i] = 1.0 / (b - kt * kt * m[i - 1]);
      for (int i = 0; i < n; ++i) al[i] = kt * m[i];
      // reciprocal pivot of the middle row k = n/2 when the line is
      // eliminated from both ends at once (the matrix is persymmetric, so the
      // bottom-up elimination has the same m and alpha, indexed from the end):
      //   mu = 1 / (1 + 2kt - kt (alpha_{k-1} + alpha_{n-2-k}))
      const int kmid = n / 2;
      const zd mu = 1.0 / (b - kt * (al[kmid - 1] + al[n - 2 - kmid]));
      double rho = 0.0;  // largest whole-chunk product |alpha_a0 ... alpha_a0+C-1|
      for (int c0 = 0; c0 < n; c0 += C) {
        zd pr = 1.0;
        for (int i = c0; i < c0 + C; ++i) { pr *= al[i]; P[i] = pr; }
        pr = 1.0;
        for (int i = c0 + C - 1; i >= c0; --i) { pr *= al[i]; Q[i] = pr; }
        rho = std::max(rho, std::abs(P[c0 + C - 1]));
      }
      // scan rounds d < dl reach dl chunks back; what they drop is at most
      // rho^dl / (1 - rho) of the largest chunk value: keep it below 2^-32
      int dl = 1;
      if (rho >= 0.5) {
        dl = 0;  // all rounds
      } else {
        double e = rho;
        while (dl < 64 && e / (1.0 - rho) > 0x1p-32) { e *= e; dl <<= 1; }
        if (dl >= 64) dl = 0;
      }
      cn_dlim[a] = dl;
      if (!cntab[a]) {
        int rc = dalloc((Cx **)&cntab[a], 4 * (size_t)n + 1);
        if (rc) return rc;
      }
      if (!imag) {
        // conjugated tables for the reverse step (C^dagger = B^dagger A^-dagger)
        if (!cntab_adj[a]) {
          int rc = dalloc((Cx **)&cntab_adj[a], 4 * (size_t)n + 1);
          if (rc) return rc;
        }
        std::vector<Cx> t(4 * (size_t)n + 1);
        auto put = [&](size_t i, zd v) { t[i].x = (R)v.real(); t[i].y = (R)(-v.imag()); };
        for (int i = 0; i < n; ++i) {
          put(i, m[i]); put(n + i, al[i]); put(2 * n + i, P[i]); put(3 * n + i, Q[i]);
        }
        put(4 * (size_t)n, mu);
        DGPE_CK(cudaMemcpy(cntab_adj[a], t.data(), sizeof(Cx) * t.size(), cudaMemcpyHostToDevice));
      }
      if (imag) {
        std::vector<R> t(4 * (size_t)n + 1);
        for (int i = 0; i < n; ++i) {
          t[i] = (R)m[i].real(); t[n + i] = (R)al[i].real();
          t[2 * n + i] = (R)P[i].real(); t[3 * n + i] = (R)Q[i].real();
        }
        t[4 * (size_t)n] = (R)mu.real();
        DGPE_CK(cudaMemcpy(cntab[a], t.data(), sizeof(R) * t.size(), cudaMemcpyHostToDevice));
      } else {
        std::vector<Cx> t(4 * (size_t)n + 1);
        auto put = [&](size_t i, zd v) { t[i].x = (R)v.real(); t[i].y = (R)v.imag(); };
        for (int i = 0; i < n; ++i) {
          put(i, m[i]); put(n + i, al[i]); put(2 * n + i, P[i]); put(3 * n + i, Q[i]);
        }
        put(4 * (size_t)n, mu);
        DGPE_CK(cudaMemcpy(cntab[a], t.data(), sizeof(Cx) * t.size(), cudaMemcpyHostToDevice));
      }
    }
    return DGPE_OK;
  }

  // The opt-in dynamic shared-memory limit is a property of the kernel, shared
  // by every solver that launches it, so it is raised to the device maximum
  // (never set to one solver's size, which could be below another's).
  template <typename K> int smem_attr(K kernel, size_t bytes) {
    int dev = 0, optin = 0;
    DGPE_CK(cudaGetDevice(&dev));
    DGPE_CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    DGPE_CK(cudaFuncGetAttributes(&fa, kernel));
    const size_t room = (size_t)optin - fa.sharedSizeBytes;
    if (bytes > room) { err = "tile needs more shared memory than the device offers"; return DGPE_EUNSUPPORTED; }
    DGPE_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)room));
    DGPE_CK(cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    return DGPE_OK;
  }
  int set_smem_attrs() {
    {
      int dev = 0;
      DGPE_CK(cudaGetDevice(&dev));
      DGPE_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    }
    int rc = with_xvar(var[0], [&](auto CLc, auto EXc, auto P2c) -> int {
      constexpr int CL = decltype(CLc)::value, EX = decltype(EXc)::value;
      constexpr bool P2 = decltype(P2c)::value;
      constexpr bool FM = P2 && (sizeof(R) == 8 || DGPE_FFT_FMA_F32);  // FMA-form twiddled stages
      constexpr bool FM1 = P2 && sizeof(R) == 8;  // the C2R pass: FP64 only
      int r;
      if ((r = smem_attr(k_dens_r2c_x<R, EX, 0, P2, FM>, x4_smem))) return r;
      if ((r = smem_attr(k_dens_r2c_x<R, EX, 1, P2, FM>, x4_smem))) return r;
      if ((r = smem_attr(k_dens_r2c_x<R, EX, 2, P2, FM>, x4_smem))) return r;
      if ((r = smem_attr(k_c2r_x_exp_cnx<R, R, EX, CL, 4, P2, FM1>, x_smem))) return r;
      if ((r = smem_attr(k_c2r_x_exp_cnx<R, R, EX, CL, 0, P2, FM1>, x_smem))) return r;
      if ((r = smem_attr(k_c2r_x_exp_cnx<R, Cx, EX, CL, 0, P2, FM1>, x_smem))) return r;
      if ((r = smem_attr(k_c2r_x_exp_cnx<R, R, EX, CL, 1, P2, FM1>, x_smem))) return r;
      if ((r = smem_attr(k_c2r_x_exp_cnx<R, Cx, EX, CL, 2, P2, FM1>, x_smem))) return r;
      if ((r = smem_attr(k_c2r_x_exp_cnx<R, R, EX, CL, 3, P2, FM1>, x_smem))) return r;
      if constexpr (sizeof(R) == 4 && P2) {
        p1_pipe = !rpsi && !(p.flags & DGPE_FLAG_P1_ONESHOT);
        if (p1_pipe) {
          // as many persistent CTAs as fit, at most one per tile
          p1_smem[0] = p1_smem_layout<R>(nx, ny, nz, x_LP, px, x_pitchz, x_pitch, CL).total;
          p1_smem[1] = p1_smem_layout<Cx>(nx, ny, nz, x_LP, px, x_pitchz, x_pitch, CL).total;
          r = with_pow2_len(nx, [&](auto Nc) -> int {
            constexpr int N = decltype(Nc)::value;
            if constexpr (N == 0 || CL != 16) {
              p1_pipe = false;
              return DGPE_OK;
            } else {
              int q;
              if ((q = smem_attr(k_p1_pipe<R, EX, CL, N>, p1_smem[0]))) return q;
              if ((q = smem_attr(k_p1_pipe<Cx, EX, CL, N>, p1_smem[1]))) return q;
              int occ0 = 0, occ1 = 0;
              DGPE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k_p1_pipe<R, EX, CL, N>, x_T, p1_smem[0]));
              DGPE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k_p1_pipe<Cx, EX, CL, N>, x_T, p1_smem[1]));
              if (occ0 < 1 || occ1 < 1) p1_pipe = false;
              p1_grid[0] = std::max(1, std::min(x_grid, nsm * occ0));
              p1_grid[1] = std::max(1, std::min(x_grid, nsm * occ1));
              return DGPE_OK;
            }
          });
          if (r) return r;
        }
        p4_pipe = !rpsi && !(p.flags & DGPE_FLAG_P1_ONESHOT);
        if (p4_pipe) {
          p4_smem = sizeof(Cx) * (2 * (size_t)2 * x_LP * nx + (size_t)x_LP * x_pitchz);
          r = with_pow2_len(nx, [&](auto Nc) -> int {
            constexpr int N = decltype(Nc)::value;
            if constexpr (N == 0 || CL != 16) {
              p4_pipe = false;
              return DGPE_OK;
            } else {
              int q;
              if ((q = smem_attr(k_p4_pipe<EX, N>, p4_smem))) return q;
              int occ = 0;
              DGPE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_p4_pipe<EX, N>, x_T, p4_smem));
              if (occ < 1) p4_pipe = false;
              p4_grid = std::max(1, std::min(x_grid, nsm * occ));
              return DGPE_OK;
            }
          });
          if (r) return r;
        }
      }
      return DGPE_OK;
    });
    if (rc) return rc;
    for (int a = 1; a < dim; ++a) {
      const size_t fs = (a == 1) ? fy.smem : fz.smem;
      rc = with_svar<EPT_S>(var[a], [&](auto EPc, auto P2c) -> int {
        constexpr int EP = decltype(EPc)::value;
        constexpr bool P2 = decltype(P2c)::value;
      constexpr bool FM = P2 && (sizeof(R) == 8 || DGPE_FFT_FMA_F32);  // FMA-form twiddled stages
      constexpr bool FM1 = P2 && sizeof(R) == 8;  // the C2R pass: FP64 only
        int r;
        if ((r = smem_attr(k_fft_strided<R, EP, 0, P2, FM>, fs))) return r;
        if ((r = smem_attr(k_fft_strided<R, EP, 1, P2, FM>, fs))) return r;
        if ((r = smem_attr(k_fft_strided<R, EP, 2, P2, FM>, fs))) return r;
        if ((r = smem_attr(k_fft_strided<R, EP, 3, P2, FM>, fs))) return r;
        return DGPE_OK;
      });
      if (rc) return rc;
      rc = with_cl(var[a], [&](auto CLc) -> int {
        constexpr int CL = decltype(CLc)::value;
        int r;
        const size_t one = cn[a].smem, two = 2 * cn[a].smem;
        if ((r = smem_attr(k_cn_strided<R, R, CL>, one))) return r;
        if ((r = smem_attr(k_cn_strided<R, Cx, CL>, one))) return r;
        if ((r = smem_attr(k_cn_strided_pipe<R, R, CL>, two))) return r;
        if ((r = smem_attr(k_cn_strided_pipe<R, Cx, CL>, two))) return r;
        if ((r = smem_attr(k_cn_strided_pipe<R, R, CL, false>, two))) return r;
        if ((r = smem_attr(k_cn_strided_pipe<R, Cx, CL, false>, two))) return r;
        if constexpr (sizeof(R) == 4 && CL == 16) {
          r = with_pow2_len(cn[a].n, [&](auto Nc) -> int {
            constexpr int N = decltype(Nc)::value;
            if constexpr (N != 0) {
              int q;
              if constexpr (16 * (N / 16) <= DGPE_MAXT) {
                if ((q = smem_attr(k_cn_pipe_ct<R, R, 16, true, N, 16>, two))) return q;
                if ((q = smem_attr(k_cn_pipe_ct<R, R, 16, false, N, 16>, two))) return q;
                if ((q = smem_attr(k_cn_pipe_ct<R, Cx, 16, false, N, 16>, two))) return q;
              }
              if constexpr (8 * (N / 16) <= DGPE_MAXT) {
                if ((q = smem_attr(k_cn_pipe_ct<R, R, 16, true, N, 8>, two))) return q;
                if ((q = smem_attr(k_cn_pipe_ct<R, R, 16, false, N, 8>, two))) return q;
                if ((q = smem_attr(k_cn_pipe_ct<R, Cx, 16, false, N, 8>, two))) return q;
              }
            }
            return DGPE_OK;
          });
          if (r) return r;
        }
        // persistent grid: as many CTAs as fit on the device, at most one per
        // tile, each double-buffered (the next tile is prefetched)
        const int ntiles = (int)(cn[a].grid.x * cn[a].grid.y);
        int occ = 0;
        DGPE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cn_strided_pipe<R, R, CL>, cn[a].T, two));
        cn[a].pgrid[0] = std::max(1, std::min(ntiles, nsm * std::max(occ, 1)));
        DGPE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cn_strided_pipe<R, Cx, CL, false>, cn[a].T, two));
        cn[a].pgrid[1] = std::max(1, std::min(ntiles, nsm * std::max(occ, 1)));
        return DGPE_OK;
      });
      if (rc) return rc;
    }
    return setup_tma();
  }

  // ------------------------------------------------------------- launches
  XArgs<R> xargs() const {
    XArgs<R> A{};
    A.psi = psi; A.spec = spec; A.phi_out = phi_tmp; A.prm = prm; A.step = dstep;
    A.tw = tw[0]; A.twf = twf[0]; A.twi = twi[0]; A.vx = vt[0]; A.vy = vt[1]; A.vz = vt[2]; A.cntab = cntab[0];
    A.pl = plx; A.nx = nx; A.ny = ny; A.nrows = nrows; A.px = px; A.LP = x_LP;
    A.pitchz = x_pitchz; A.pitch = x_pitch; A.TPL = x_TPL; A.C = x_C;
    A.imag = imag; A.has_dip = has_dip ? 1 : 0; A.tau = tau[0]; A.dtf = 1.0;
    A.cnd = cn_dlim[0];
    return A;
  }
  SArgs<R> sargs(const FtCfg &f) const {
    SArgs<R> A{};
    A.spec = spec; A.U = U; A.partial = dip_part; A.tw = tw[f.axis]; A.pl = f.pl;
    A.twf = twf[f.axis]; A.twi = twi[f.axis];
    A.estride = f.es; A.ostride = f.os; A.n = f.n; A.ncols = ncol_spec; A.W = f.W; A.nxh = nx / 2;
    if (dim == 3) {
      A.uq[0] = (float)(2.0 * M_PI / (nx * p.h[0]));
      A.uq[1] = (float)(2.0 * M_PI / (ny * p.h[1]));
      A.uq[2] = (float)(2.0 * M_PI / (nz * p.h[2]));
      A.uq[3] = (float)((4.0 * M_PI / 3.0) / (double)nsites);
    }
    A.uny = ny;
    return A;
  }
  // FP32, power-of-two length, modes 0-2: the length-specialised transform
  bool launch_fft_ct(const FtCfg &f, int mode, const SArgs<R> &A, cudaStream_t s) {
    if constexpr (sizeof(R) != 4) {
      return false;
    } else {
      if (mode > 2 || var[f.axis] != VAR_P2 || !(f.W == 16 || f.W == 8 || f.W == 4)) return false;
      return with_pow2_len(f.n, [&](auto Nc) -> int {
        constexpr int N = decltype(Nc)::value;
        if constexpr (N == 0) {
          return 0;
        } else {
          auto go = [&](auto Wc) {
            constexpr int WW = decltype(Wc)::value;
            if constexpr (WW * N / EPT_S <= DGPE_MAXT_FFT) {
              if (mode == 0) k_fft_strided_ct<EPT_S, 0, N, WW><<<f.grid, f.T, f.smem, s>>>(A);
              else if (mode == 1) k_fft_strided_ct<EPT_S, 1, N, WW><<<f.grid, f.T, f.smem, s>>>(A);
              else k_fft_strided_ct<EPT_S, 2, N, WW><<<f.grid, f.T, f.smem, s>>>(A);
              return 1;
            } else {
              return 0;
            }
          };
          if (f.W == 16) return go(std::integral_constant<int, 16>{});
          if (f.W == 8) return go(std::integral_constant<int, 8>{});
          return go(std::integral_constant<int, 4>{});
        }
      }) != 0;
    }
  }
  // FP32, power-of-two lengths: tensor maps of the half spectrum (kx, y, z;
  // kx valid columns, rows of px elements) for the TMA-tiled transforms.
  // Not fatal when unavailable: the length-specialised kernels run instead.
  int tma_grid[2] = {0, 0};
  template <int AX, int N, int WW> int tma_attrs(int &grid) {
    const size_t sm = 2 * sizeof(Cx) * (size_t)WW * N + 128;
    int r;
    if constexpr (AX == 1) {  // lines along y: FFT_y, IFFT_y (3D) and FFT_y.U.IFFT_y (2D)
      if ((r = smem_attr(k_fft_tma<EPT_S, 0, N, WW, AX>, sm))) return r;
      if ((r = smem_attr(k_fft_tma<EPT_S, 1, N, WW, AX>, sm))) return r;
    }
    if ((r = smem_attr(k_fft_tma<EPT_S, 2, N, WW, AX>, sm))) return r;
    int occ = 0;
    DGPE_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fft_tma<EPT_S, 2, N, WW, AX>, WW * N / EPT_S, sm));
    grid = nsm * occ;
    return DGPE_OK;
  }
  template <int AX> int tma_axis(const FtCfg &f, int &grid) {
    return with_pow2_len(f.n, [&](auto Nc) -> int {
      constexpr int N = decltype(Nc)::value;
      if constexpr (N == 0) {
        return DGPE_EUNSUPPORTED;
      } else {
        if (f.W == 16) {
          if constexpr (16 * N / EPT_S <= DGPE_MAXT_FFT) return this->template tma_attrs<AX, N, 16>(grid);
        } else if (f.W == 8) {
          if constexpr (8 * N / EPT_S <= DGPE_MAXT_FFT) return this->template tma_attrs<AX, N, 8>(grid);
        }
        return DGPE_EUNSUPPORTED;
      }
    });
  }
  int setup_tma() {
    if constexpr (sizeof(R) != 4) {
      return DGPE_OK;
    } else {
      tma_fft = false;
      if (!has_dip || (p.flags & DGPE_FLAG_P1_ONESHOT)) return DGPE_OK;
      if (var[1] != VAR_P2 || (dim == 3 && var[2] != VAR_P2)) return DGPE_OK;
      TensorMapEncodeTiledFn enc = tensor_map_encoder();
      if (!enc) return DGPE_OK;
      const cuuint64_t dims[3] = {(cuuint64_t)ncol_spec, (cuuint64_t)ny, (cuuint64_t)nz};
      const cuuint64_t strides[2] = {(cuuint64_t)px * sizeof(Cx), (cuuint64_t)ny * px * sizeof(Cx)};
      const cuuint32_t es[3] = {1, 1, 1};
      auto rows = [](int n) { return (cuuint32_t)(n / ((n + 255) / 256)); };
      const cuuint32_t by[3] = {(cuuint32_t)fy.W, rows(ny), 1};
      if (enc(&tm_y, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, spec, dims, strides, by, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return DGPE_OK;
      if (dim == 3) {
        const cuuint32_t bz[3] = {(cuuint32_t)fz.W, 1, rows(nz)};
        if (enc(&tm_z, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, spec, dims, strides, bz, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
          return DGPE_OK;
      }
      int r = this->template tma_axis<1>(fy, tma_grid[0]);
      if (r == DGPE_EUNSUPPORTED) return DGPE_OK;
      if (r) return r;
      if (dim == 3) {
        r = this->template tma_axis<2>(fz, tma_grid[1]);
        if (r == DGPE_EUNSUPPORTED) return DGPE_OK;
        if (r) return r;
      }
      tma_fft = tma_grid[0] > 0 && (dim == 2 || tma_grid[1] > 0);
      return DGPE_OK;
    }
  }
  bool launch_fft_tma(const FtCfg &f, int mode, const SArgs<R> &A, cudaStream_t s) {
    if constexpr (sizeof(R) != 4) {
      return false;
    } else {
      if (!tma_fft || mode > 2) return false;
      const int ncb = (int)f.grid.x, ntiles = (int)(f.grid.x * f.grid.y);
      return with_pow2_len(f.n, [&](auto Nc) -> int {
        constexpr int N = decltype(Nc)::value;
        if constexpr (N == 0) {
          return 0;
        } else {
          auto go = [&](auto Wc) -> int {
            constexpr int WW = decltype(Wc)::value;
            if constexpr (WW * N / EPT_S <= DGPE_MAXT_FFT) {
              const size_t sm = 2 * sizeof(Cx) * (size_t)WW * N + 128;
              const int T = WW * N / EPT_S;
              double *tf = prm + PRM_TIMEOUT;
              if (f.axis == 1) {
                const int g = std::max(1, std::min(ntiles, tma_grid[0]));
                if (mode == 0) k_fft_tma<EPT_S, 0, N, WW, 1><<<g, T, sm, s>>>(tm_y, A, ncb, ntiles, tf);
                else if (mode == 1) k_fft_tma<EPT_S, 1, N, WW, 1><<<g, T, sm, s>>>(tm_y, A, ncb, ntiles, tf);
                else k_fft_tma<EPT_S, 2, N, WW, 1><<<g, T, sm, s>>>(tm_y, A, ncb, ntiles, tf);
              } else {
                const int g = std::max(1, std::min(ntiles, tma_grid[1]));
                if (mode != 2) return 0;
                k_fft_tma<EPT_S, 2, N, WW, 2><<<g, T, sm, s>>>(tm_z, A, ncb, ntiles, tf);
              }
              return 1;
            } else {
              return 0;
            }
          };
          if (f.W == 16) return go(std::integral_constant<int, 16>{});
          if (f.W == 8) return go(std::integral_constant<int, 8>{});
          return 0;
        }
      }) != 0;
    }
  }
  int launch_fft(const FtCfg &f, int mode, cudaStream_t s) {
    SArgs<R> A = sargs(f);
    if (launch_fft_tma(f, mode, A, s) || launch_fft_ct(f, mode, A, s)) {
      launched(1);
      DGPE_LCK(__func__);
      return DGPE_OK;
    }
    with_svar<EPT_S>(var[f.axis], [&](auto EPc, auto P2c) -> int {
      constexpr int EP = decltype(EPc)::value;
      constexpr bool P2 = decltype(P2c)::value;
      constexpr bool FM = P2 && (sizeof(R) == 8 || DGPE_FFT_FMA_F32);  // FMA-form twiddled stages
      constexpr bool FM1 = P2 && sizeof(R) == 8;  // the C2R pass: FP64 only
      switch (mode) {
        case 0: k_fft_strided<R, EP, 0, P2, FM><<<f.grid, f.T, f.smem, s>>>(A); break;
        case 1: k_fft_strided<R, EP, 1, P2, FM><<<f.grid, f.T, f.smem, s>>>(A); break;
        case 2: k_fft_strided<R, EP, 2, P2, FM><<<f.grid, f.T, f.smem, s>>>(A); break;
        default: k_fft_strided<R, EP, 3, P2, FM><<<f.grid, f.T, f.smem, s>>>(A); break;
      }
      return DGPE_OK;
    });
    launched(1);
    DGPE_LCK(__func__);
    return DGPE_OK;
  }
  // FP32, power-of-two length, tile width 16 or 8: the length-specialised
  // CN pass (same grid, block and shared memory as k_cn_strided_pipe)
  bool launch_cn_ct(const CnCfg &c, int axis, const CArgs<R> &A, int ncb, int ntiles, cudaStream_t s) {
    if constexpr (sizeof(R) != 4) {
      return false;
    } else {
      if (var[axis] != VAR_P2 || !(c.W == 16 || c.W == 8)) return false;
      return with_pow2_len(c.n, [&](auto Nc) -> int {
        constexpr int N = decltype(Nc)::value;
        if constexpr (N == 0) {
          return 0;
        } else {
          auto go = [&](auto Wc) {
            constexpr int WW = decltype(Wc)::value;
            if constexpr (WW * (N / 16) <= DGPE_MAXT) {
              if (imag && A.norm) k_cn_pipe_ct<R, R, 16, true, N, WW><<<c.pgrid[0], c.T, 2 * c.smem, s>>>(A, ncb, ntiles);
              else if (imag) k_cn_pipe_ct<R, R, 16, false, N, WW><<<c.pgrid[0], c.T, 2 * c.smem, s>>>(A, ncb, ntiles);
              else k_cn_pipe_ct<R, Cx, 16, false, N, WW><<<c.pgrid[1], c.T, 2 * c.smem, s>>>(A, ncb, ntiles);
              return 1;
            } else {
              return 0;
            }
          };
          return (c.W == 16) ? go(std::integral_constant<int, 16>{}) : go(std::integral_constant<int, 8>{});
        }
      }) != 0;
    }
  }
  int launch_cn(int axis, bool final_pass, cudaStream_t s, Cx *buf = nullptr, bool adjoint = false) {
    if (cn_serial) return launch_lines(axis, final_pass, s, buf, adjoint);
    const CnCfg &c = cn[axis];
    CArgs<R> A{};
    A.psi = buf ? buf : psi; A.cntab = adjoint ? cntab_adj[axis] : cntab[axis];
    A.prm = prm; A.partial = partial; A.counter = counter;
    A.step = dstep; A.estride = c.es; A.ostride = c.os; A.n = c.n; A.ncols = c.ncols; A.W = c.W;
    A.TPL = c.TPL; A.C = c.C; A.pitch = c.pitch; A.final_pass = final_pass ? 1 : 0;
    A.norm = (final_pass && imag) ? 1 : 0; A.tau = adjoint ? -tau[axis] : tau[axis];
    A.cnd = cn_dlim[axis];
    const int ncb = (int)c.grid.x, ntiles = (int)(c.grid.x * c.grid.y);
    if (launch_cn_ct(c, axis, A, ncb, ntiles, s)) {
      launched(1);
      DGPE_LCK(__func__);
      return DGPE_OK;
    }
    with_cl(var[axis], [&](auto CLc) -> int {
      constexpr int CL = decltype(CLc)::value;
      // the norm's code only in the pass that takes the norm
      if (imag && A.norm) k_cn_strided_pipe<R, R, CL, true><<<c.pgrid[0], c.T, 2 * c.smem, s>>>(A, ncb, ntiles);
      else if (imag) k_cn_strided_pipe<R, R, CL, false><<<c.pgrid[0], c.T, 2 * c.smem, s>>>(A, ncb, ntiles);
      else k_cn_strided_pipe<R, Cx, CL, false><<<c.pgrid[1], c.T, 2 * c.smem, s>>>(A, ncb, ntiles);
      return DGPE_OK;
    });
    launched(1);
    DGPE_LCK(__func__);
    return DGPE_OK;
  }
  int launch_lines(int axis, bool final_pass, cudaStream_t s, Cx *buf, bool adjoint) {
    const LnCfg &L = ln[axis];
    LArgs A{};
    A.psi = buf ? buf : psi; A.tab = adjoint ? cntab_adj[axis] : cntab[axis];
    A.prm = prm; A.partial = partial; A.counter = counter; A.step = dstep;
    A.es = L.es; A.cs = L.cs; A.os = L.os; A.n = L.n; A.ncols = L.ncols;
    A.final_pass = final_pass ? 1 : 0; A.norm = (final_pass && imag) ? 1 : 0;
    A.tau = adjoint ? -tau[axis] : tau[axis];
    if (imag && A.norm) k_cn_lines<R, R, true><<<L.grid, L.T, 0, s>>>(A);
    else if (imag) k_cn_lines<R, R, false><<<L.grid, L.T, 0, s>>>(A);
    else k_cn_lines<R, Cx, false><<<L.grid, L.T, 0, s>>>(A);
    launched(1);
    DGPE_LCK(__func__);
    return DGPE_OK;
  }
  // density (of `src`, or the real field `dens_in`) -> half spectrum along x
  int launch_forward_spectrum(cudaStream_t s, const Cx *src = nullptr, const R *dens_in = nullptr) {
    XArgs<R> A = xargs();
    if (src) A.psi = const_cast<Cx *>(src);
    if (dens_in) A.dens_in = dens_in;
    with_xvar(var[0], [&](auto CLc, auto EXc, auto P2c) -> int {
      constexpr int EX = decltype(EXc)::value;
      constexpr bool P2 = decltype(P2c)::value;
      constexpr bool FM = P2 && (sizeof(R) == 8 || DGPE_FFT_FMA_F32);  // FMA-form twiddled stages
      constexpr bool FM1 = P2 && sizeof(R) == 8;  // the C2R pass: FP64 only
      if (dens_in) k_dens_r2c_x<R, EX, 1, P2, FM><<<x_grid, x_T, x4_smem, s>>>(A);
      else if (rpsi && !src) k_dens_r2c_x<R, EX, 2, P2, FM><<<x_grid, x_T, x4_smem, s>>>(A);
      else if (p4_pipe) {
        if constexpr (sizeof(R) == 4 && P2 && decltype(CLc)::value == 16) {
          with_pow2_len(nx, [&](auto Nc) -> int {
            constexpr int N = decltype(Nc)::value;
            if constexpr (N != 0) k_p4_pipe<EX, N><<<p4_grid, x_T, p4_smem, s>>>(A, x_grid, prm + PRM_TIMEOUT);
            return 0;
          });
        }
      } else k_dens_r2c_x<R, EX, 0, P2, FM><<<x_grid, x_T, x4_smem, s>>>(A);
      return DGPE_OK;
    });
    launched(1);
    DGPE_LCK(__func__);
    return DGPE_OK;
  }
  // mode 0: step pass on psi; 1: Phi_d into phi_out; 2: CN_x (conjugated) on
  // buf; 3: step pass without CN_x (the line-serial CN_x pass follows), its
  // exponential over the fraction dtf of dt
  int launch_p1(int mode, cudaStream_t s, Cx *buf = nullptr, R *phi_out = nullptr, double dtf = 1.0) {
    if (mode == 2 && cn_serial) return launch_lines(0, false, s, buf, true);
    XArgs<R> A = xargs();
    A.dtf = dtf;
    if (buf) A.psi = buf;
    if (phi_out) A.phi_out = phi_out;
    if (mode == 2) {
      A.cntab = cntab_adj[0];
      A.tau = -tau[0];
      A.cnd = cn_dlim[0];
    }
    with_xvar(var[0], [&](auto CLc, auto EXc, auto P2c) -> int {
      constexpr int CL = decltype(CLc)::value, EX = decltype(EXc)::value;
      constexpr bool P2 = decltype(P2c)::value;
      constexpr bool FM = P2 && (sizeof(R) == 8 || DGPE_FFT_FMA_F32);  // FMA-form twiddled stages
      constexpr bool FM1 = P2 && sizeof(R) == 8;  // the C2R pass: FP64 only
      if (mode == 0 && rpsi) {
        k_c2r_x_exp_cnx<R, R, EX, CL, 4, P2, FM1><<<x_grid, x_T, x_smem, s>>>(A);
      } else if (mode == 0 && p1_pipe) {
        if constexpr (sizeof(R) == 4 && P2 && CL == 16) {
          with_pow2_len(nx, [&](auto Nc) -> int {
            constexpr int N = decltype(Nc)::value;
            if constexpr (N != 0) {
              if (imag) k_p1_pipe<R, EX, CL, N><<<p1_grid[0], x_T, p1_smem[0], s>>>(A, x_grid, nz, prm + PRM_TIMEOUT);
              else k_p1_pipe<Cx, EX, CL, N><<<p1_grid[1], x_T, p1_smem[1], s>>>(A, x_grid, nz, prm + PRM_TIMEOUT);
            }
            return 0;
          });
        }
      } else if (mode == 0) {
        if (imag) k_c2r_x_exp_cnx<R, R, EX, CL, 0, P2, FM1><<<x_grid, x_T, x_smem, s>>>(A);
        else k_c2r_x_exp_cnx<R, Cx, EX, CL, 0, P2, FM1><<<x_grid, x_T, x_smem, s>>>(A);
      } else if (mode == 3) {
        k_c2r_x_exp_cnx<R, R, EX, CL, 3, P2, FM1><<<x_grid, x_T, x_smem, s>>>(A);
      } else if (mode == 1) {
        k_c2r_x_exp_cnx<R, R, EX, CL, 1, P2, FM1><<<x_grid, x_T, x_smem, s>>>(A);
      } else {
        k_c2r_x_exp_cnx<R, Cx, EX, CL, 2, P2, FM1><<<x_grid, x_T, x_smem, s>>>(A);
      }
      return DGPE_OK;
    });
    launched(1);
    DGPE_LCK(__func__);
    return DGPE_OK;
  }
  // Phi_d chain up to (not including) the C2R along x.
  int launch_dipolar_chain(cudaStream_t s, const Cx *src = nullptr, const R *dens_in = nullptr) {
    int rc;
    if ((rc = launch_forward_spectrum(s, src, dens_in))) return rc;
    if (dim == 3) {
      if ((rc = launch_fft(fy, 0, s))) return rc;
      if ((rc = launch_fft(fz, 2, s))) return rc;
      if ((rc = launch_fft(fy, 1, s))) return rc;
    } else {
      if ((rc = launch_fft(fy, 2, s))) return rc;
    }
    return DGPE_OK;
  }
  // The passes of one step, in order (id, name, algorithmic HBM bytes).
  enum { PS_DENS_R2C, PS_FFT_Y, PS_FFT_Z_U, PS_IFFT_Y, PS_FFT_Y_U, PS_P1, PS_CN_Y, PS_CN_Z, PS_P1_NOCN, PS_CN_X };
  std::vector<int> pass_ids() const {
    std::vector<int> v;
    if (has_dip) {
      v.push_back(PS_DENS_R2C);
      if (dim == 3) { v.push_back(PS_FFT_Y); v.push_back(PS_FFT_Z_U); v.push_back(PS_IFFT_Y); }
      else v.push_back(PS_FFT_Y_U);
    }
    if (cn_serial) { v.push_back(PS_P1_NOCN); v.push_back(PS_CN_X); }
    else v.push_back(PS_P1);
    v.push_back(PS_CN_Y);
    if (dim == 3) v.push_back(PS_CN_Z);
    return v;
  }
  int launch_pass(int id, cudaStream_t s) {
    switch (id) {
      case PS_DENS_R2C: return launch_forward_spectrum(s);
      case PS_FFT_Y: return launch_fft(fy, 0, s);
      case PS_FFT_Z_U: return launch_fft(fz, 2, s);
      case PS_IFFT_Y: return launch_fft(fy, 1, s);
      case PS_FFT_Y_U: return launch_fft(fy, 2, s);
      case PS_P1: return launch_p1(0, s);
      case PS_P1_NOCN: return launch_p1(3, s);
      case PS_CN_X: return launch_cn(0, false, s);
      case PS_CN_Y: return launch_cn(1, dim == 2, s);
      default: return launch_cn(2, true, s);
    }
  }
  int launch_step(cudaStream_t s) {
    for (int id : pass_ids()) {
      int rc = launch_pass(id, s);
      if (rc) return rc;
    }
    return DGPE_OK;
  }
  // Exponential substep alone over f dt at the current time (Phi_d of the
  // current density first): the ends of a run of Strang steps.  In real time
  // the substep leaves |psi| unchanged, so n Strang steps
  //   E(dt/2, t_{k+1}) C E(dt/2, t_k)
  // telescope into E(-dt/2, t_0) [C E(dt, t_k)]_{k=0..n-1} E(dt/2, t_n): the n
  // first-order steps with one half-step pass before and after them.
  int launch_exp_only(double f, cudaStream_t s) {
    int rc;
    if (has_dip && (rc = launch_dipolar_chain(s))) return rc;
    return launch_p1(3, s, nullptr, nullptr, f);
  }
  const char *pass_name(int i) const override {
    static const char *names[] = {"dens_r2c_x", "fft_y", "fft_z_u_ifft_z", "ifft_y",
                                  "fft_y_u_ifft_y", "c2r_x_exp_cn_x", "cn_y", "cn_z", "c2r_x_exp", "cn_x"};
    std::vector<int> v = pass_ids();
    return (i >= 0 && i < (int)v.size()) ? names[v[i]] : "";
  }
  double pass_bytes(int i) const override {
    std::vector<int> v = pass_ids();
    if (i < 0 || i >= (int)v.size()) return 0.0;
    const double S = (double)sizeof(Cx), N = (double)nsites;
    const double SP = rpsi ? (double)sizeof(R) : S;  // bytes of psi per site
    const double sp = (double)ncol_spec * nrows, ub = sp * sizeof(R);
    switch (v[i]) {
      case PS_DENS_R2C: return N * SP + sp * S;
      case PS_FFT_Y: case PS_IFFT_Y: return 2.0 * sp * S;
      // the FP32 3D tensor-map z-pass evaluates U(k) instead of reading it
      case PS_FFT_Z_U: return 2.0 * sp * S + ((tma_fft && dim == 3) ? 0.0 : ub);
      case PS_FFT_Y_U: return 2.0 * sp * S + ub;
      case PS_P1: case PS_P1_NOCN: return (has_dip ? sp * S : 0.0) + 2.0 * N * SP;
      default: return 2.0 * N * SP;
    }
  }
  // Floating-point operations of pass i per launch (an FMA counts 2), from
  // the arithmetic each algorithm specifies: Stockham FFT stages (codelet
  // operation counts plus (r - 1) twiddle products per radix-r butterfly
  // after the first stage), the pair packing/unpacking of the real
  // transforms, the exponential substep, and the Thomas recurrences.
  static double codelet_flops(int r) {
    switch (r) {
      case 2: return 4;     // one complex sum and difference
      case 3: return 16;
      case 4: return 16;    // 8 complex additions
      case 5: return 48;
      case 8: return 60;    // two radix-4 (32) + two w8 rotations (12) + 8 additions (16)
      case 16: return 176;  // eight radix-4 (128) + eight inner twiddle rotations (48)
      default: return 0;
    }
  }
  static double fft_line_flops(const FftPlan &pl) {
    double f = 0.0;
    for (int s = 0; s < pl.ns; ++s) {
      const double nb = (double)pl.n / pl.rad[s];
      f += nb * codelet_flops(pl.rad[s]);
      if (s > 0) f += nb * (pl.rad[s] - 1) * 6.0;
    }
    return f;
  }
  // exponential substep per site.  FP32 and imaginary time: V (1), scaled
  // psi (2), density (3), theta (5 with the dipolar term, else 3), the factor
  // (real time: sin and cos - 1 by Taylor series, 11 in FP32; imaginary time:
  // expm1 counted as 1) and its increment-form update (8 real / 4 imaginary).
  // FP64 real time: theta from |psi|^2 and the dt-scaled potentials (8 with
  // the dipolar term, else 6), sin and cos - 1 (19), the scaled factor (3)
  // and one complex product (6).
  double exp_flops_per_site() const {
    if (sizeof(R) == 8 && !imag) return (has_dip ? 8.0 : 6.0) + 19.0 + 3.0 + 6.0;
    const double th = has_dip ? 5.0 : 3.0;
    if (rpsi) return 1 + 1 + 1 + th + 1 + 2;  // real state: V, scale, square, theta, expm1, update
    if (imag) return 1 + 2 + 3 + th + 1 + 4;
    return 1 + 2 + 3 + th + 11.0 + 8;
  }
  // Thomas solve per site: line-serial (forward right-hand side, forward
  // elimination, back substitution) or chunk-parallel (chunk passes, the two
  // lane scans amortised over the chunk, fix-ups)
  double cn_flops_per_site(int axis) const {
    if (cn_serial) return imag ? 16.0 : 28.0;
    // a real state: one complex solve with real coefficients advances two sites
    if (rpsi) return 0.5 * cn_flops_chunked(axis);
    return cn_flops_chunked(axis);
  }
  double cn_flops_chunked(int axis) const {
    const int cl = (axis == 0) ? x_C : cn[axis].C;
    const int tpl = (axis == 0) ? x_TPL : cn[axis].TPL;
    const double lg = std::log2((double)std::max(tpl, 1));
    if (imag) return 28.0 + 2.0 * 5.0 * lg / cl;
    return 52.0 + 2.0 * 14.0 * lg / cl;
  }
  double pass_flops(int i) const override {
    std::vector<int> v = pass_ids();
    if (i < 0 || i >= (int)v.size()) return 0.0;
    const double N = (double)nsites, pairs = (double)((nrows + 1) / 2);
    const double norm = (imag ? 4.0 : 0.0);  // FP64 |x|^2 accumulation of the final pass
    switch (v[i]) {
      case PS_DENS_R2C: return (rpsi ? 2.0 : 4.0) * N + pairs * fft_line_flops(plx) + pairs * (nx / 2 + 1) * 8.0;
      case PS_FFT_Y: case PS_IFFT_Y: return (double)ncol_spec * nz * fft_line_flops(ply);
      case PS_FFT_Z_U: return (double)ncol_spec * ny * (2.0 * fft_line_flops(plz) + 2.0 * nz);
      case PS_FFT_Y_U: return (double)ncol_spec * (2.0 * fft_line_flops(ply) + 2.0 * ny);
      case PS_P1: case PS_P1_NOCN: {
        double f = (has_dip ? pairs * fft_line_flops(plx) : 0.0) + N * exp_flops_per_site();
        if (v[i] == PS_P1) f += N * cn_flops_per_site(0);
        return f;
      }
      case PS_CN_X: return N * cn_flops_per_site(0);
      case PS_CN_Y: return N * (cn_flops_per_site(1) + (dim == 2 ? norm : 0.0));
      default: return N * (cn_flops_per_site(2) + norm);
    }
  }
  int profile_steps(int n, double *pass_ms, int cap, cudaStream_t s) override {
    std::vector<int> v = pass_ids();
    const int np = (int)v.size();
    if (cap < np) { err = "pass_ms too small"; return DGPE_EINVAL; }
    std::vector<cudaEvent_t> ev(np + 1);
    for (auto &e : ev) DGPE_CK(cudaEventCreate(&e));
    std::vector<double> acc(np, 0.0);
    int rc = DGPE_OK;
    for (int k = 0; k < n && rc == DGPE_OK; ++k) {
      for (int i = 0; i < np && rc == DGPE_OK; ++i) {
        cudaEventRecord(ev[i], s);
        rc = launch_pass(v[i], s);
      }
      cudaEventRecord(ev[np], s);
      if (cudaEventSynchronize(ev[np]) != cudaSuccess) { err = "event sync failed"; rc = DGPE_ECUDA; }
      for (int i = 0; i < np && rc == DGPE_OK; ++i) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
        acc[i] += ms;
      }
    }
    for (auto &e : ev) cudaEventDestroy(e);
    if (rc) return rc;
    for (int i = 0; i < np; ++i) pass_ms[i] = n > 0 ? acc[i] / n : 0.0;
    return np;
  }
  int capture() {
    if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
    if (graph) { cudaGraphDestroy(graph); graph = nullptr; }
    DGPE_CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    capturing = true;
    int rc = launch_step(cap);
    capturing = false;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) { err = std::string("graph capture: ") + cudaGetErrorString(e); return DGPE_ECUDA; }
    graph = g;
    DGPE_CK(cudaGraphInstantiate(&gexec, graph, 0));
    return DGPE_OK;
  }

  // ------------------------------------------------------------ API calls
  int step(int n, cudaStream_t s) override {
    int rc;
    if (strang && n > 0 && (rc = launch_exp_only(-0.5, s))) return rc;
    for (int i = 0; i < n; ++i) {
      if (use_graph) {
        DGPE_CK(cudaGraphLaunch(gexec, s));
        nlaunch += launches_per_step();
      }
      else {
        if ((rc = launch_step(s))) return rc;
      }
    }
    if (strang && n > 0 && (rc = launch_exp_only(0.5, s))) return rc;
    return DGPE_OK;
  }
  int reset_scale(cudaStream_t s) {
    const double one = 1.0, zero = 0.0;
    DGPE_CK(cudaMemcpyAsync(prm + PRM_SC, &one, sizeof(double), cudaMemcpyHostToDevice, s));
    DGPE_CK(cudaMemcpyAsync(prm + PRM_NONFINITE, &zero, sizeof(double), cudaMemcpyHostToDevice, s));
    DGPE_CK(cudaMemcpyAsync(prm + PRM_TIMEOUT, &zero, sizeof(double), cudaMemcpyHostToDevice, s));
    DGPE_CK(cudaStreamSynchronize(s));
    return DGPE_OK;
  }
  int wait_status(cudaStream_t s) override {
    double f = 0.0;
    DGPE_CK(cudaMemcpyAsync(&f, prm + PRM_TIMEOUT, sizeof(double), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaStreamSynchronize(s));
    if (f != 0.0) {
      err = "a bounded device-side wait ran out (the step's results are incomplete)";
      return DGPE_ETIMEOUT;
    }
    return DGPE_OK;
  }
  int set_psi_host(const double *src, cudaStream_t s) override {
    if (!stage) { int rc = dalloc(&stage, nsites); if (rc) return rc; }
    DGPE_CK(cudaMemcpyAsync(stage, src, sizeof(double2) * nsites, cudaMemcpyHostToDevice, s));
    return set_psi_device(stage, 1, s);
  }
  int get_psi_host(double *dst, cudaStream_t s) override {
    if (!stage) { int rc = dalloc(&stage, nsites); if (rc) return rc; }
    int rc = get_psi_device(stage, 1, s);
    if (rc) return rc;
    DGPE_CK(cudaMemcpyAsync(dst, stage, sizeof(double2) * nsites, cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaStreamSynchronize(s));
    return DGPE_OK;
  }
  int set_psi_device(const void *src, int fp64, cudaStream_t s) override {
    const int blocks = 152 * 8;
    if (rpsi && fp64) k_import_real<R, double2><<<blocks, 256, 0, s>>>((R *)psi, (const double2 *)src, nsites);
    else if (rpsi) k_import_real<R, float2><<<blocks, 256, 0, s>>>((R *)psi, (const float2 *)src, nsites);
    else if (fp64) k_import<R, double2><<<blocks, 256, 0, s>>>(psi, (const double2 *)src, nsites);
    else k_import<R, float2><<<blocks, 256, 0, s>>>(psi, (const float2 *)src, nsites);
    launched(1);
    DGPE_LCK(__func__);
    int rc = reset_scale(s);
    if (rc) return rc;
    return set_time(0, s);
  }
  int get_psi_device(void *dst, int fp64, cudaStream_t s) override {
    const int blocks = 152 * 8;
    if (rpsi && fp64) k_export_real<R, double2><<<blocks, 256, 0, s>>>((double2 *)dst, (const R *)psi, prm, nsites);
    else if (rpsi) k_export_real<R, float2><<<blocks, 256, 0, s>>>((float2 *)dst, (const R *)psi, prm, nsites);
    else if (fp64) k_export<R, double2><<<blocks, 256, 0, s>>>((double2 *)dst, psi, prm, nsites);
    else k_export<R, float2><<<blocks, 256, 0, s>>>((float2 *)dst, psi, prm, nsites);
    launched(1);
    DGPE_LCK(__func__);
    return DGPE_OK;
  }
  int observables(dgpe_obs *o, cudaStream_t s) override {
    int rc;
    DGPE_LCK("(pending before observables)");
    // a real state is widened to (psi, 0) first; the sums below then run
    // unchanged on the complex copy
    const Cx *obs_psi = psi;
    if (rpsi) {
      if (!ocx && (rc = dalloc(&ocx, nsites))) return rc;
      k_widen_real<R><<<152 * 8, 256, 0, s>>>(ocx, (const R *)psi, nsites);
      launched(1);
      DGPE_LCK("widen");
      obs_psi = ocx;
    }
    if (has_dip) {
      if ((rc = launch_forward_spectrum(s, obs_psi))) return rc;
      DGPE_LCK("density/R2C");
      if (dim == 3) {
        if ((rc = launch_fft(fy, 0, s))) return rc;
        if ((rc = launch_fft(fz, 3, s))) return rc;
      } else {
        if ((rc = launch_fft(fy, 3, s))) return rc;
      }
      DGPE_LCK("spectral energy sum");
    }
    OArgs<R> A{};
    A.psi = obs_psi; A.prm = prm; A.partial = obs_part; A.nx = nx; A.ny = ny; A.nz = nz; A.dim = dim;
    A.rows_per_block = 0; A.hx = p.h[0]; A.hy = p.h[1]; A.hz = (dim == 3) ? p.h[2] : 0.0;
    A.nux = p.nu[0]; A.nuy = p.nu[1]; A.nuz = (dim == 3) ? p.nu[2] : 0.0;
    k_obs_sites<R><<<obs_blocks, 256, 0, s>>>(A);
    launched(1);
    DGPE_LCK("site sums");
    k_obs_final<<<1, 256, 0, s>>>(obs_part, obs_blocks, dip_part, ndip, obs_out);
    launched(1);
    DGPE_LCK("final sums");
    double h[OBS_COUNT + 1];
    double hp[PRM_COUNT];
    long long st = 0;
    DGPE_CK(cudaMemcpyAsync(h, obs_out, sizeof(h), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaMemcpyAsync(hp, prm, sizeof(hp), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaMemcpyAsync(&st, dstep, sizeof(st), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaStreamSynchronize(s));
    if (hp[PRM_TIMEOUT] != 0.0) {
      err = "a bounded device-side wait ran out (the step's results are incomplete)";
      return DGPE_ETIMEOUT;
    }
    if (h[OBS_BAD] > 0.0 || hp[PRM_NONFINITE] != 0.0) {
      err = "state holds NaN or Inf";
      return DGPE_ENONFINITE;
    }
    const double cell = hp[PRM_CELL];
    const double t = (double)st * p.dt;
    double sm = 1.0;
    for (int m = 1; m <= (int)hp[PRM_M]; ++m) sm += hp[PRM_CM + m - 1] * std::sin((double)m * t);
    const double norm = cell * h[OBS_N];
    double kin = 0.5 * cell * (h[OBS_KX] / (p.h[0] * p.h[0]) + h[OBS_KY] / (p.h[1] * p.h[1]));
    if (dim == 3) kin += 0.5 * cell * h[OBS_KZ] / (p.h[2] * p.h[2]);
    const double pot = sm * cell * h[OBS_V];
    const double con = hp[PRM_G] * cell * h[OBS_N2];
    const double dip = has_dip ? hp[PRM_GDD] * cell * h[OBS_COUNT] : 0.0;
    o->norm = norm;
    o->kin = kin / norm;
    o->pot = pot / norm;
    o->contact = con / norm;
    o->dipolar = dip / norm;
    o->mu = (kin + pot + con + dip) / norm;
    o->energy = (kin + pot + 0.5 * con + 0.5 * dip) / norm;
    o->rms[0] = std::sqrt(h[OBS_X2] / h[OBS_N]);
    o->rms[1] = std::sqrt(h[OBS_Y2] / h[OBS_N]);
    o->rms[2] = (dim == 3) ? std::sqrt(h[OBS_Z2] / h[OBS_N]) : 0.0;
    o->rms_r = std::sqrt((h[OBS_X2] + h[OBS_Y2] + h[OBS_Z2]) / h[OBS_N]);
    o->t = t;
    if (!std::isfinite(o->mu) || !std::isfinite(norm)) { err = "non-finite observables"; return DGPE_ENONFINITE; }
    return DGPE_OK;
  }
  int dipolar_potential(double *phi_host, cudaStream_t s) override {
    std::vector<R> tmp(nsites, (R)0);
    if (has_dip) {
      if (!phi_tmp) { int rc = dalloc(&phi_tmp, nsites); if (rc) return rc; }
      int rc;
      if ((rc = launch_dipolar_chain(s))) return rc;
      if ((rc = launch_p1(1, s))) return rc;
      DGPE_CK(cudaMemcpyAsync(tmp.data(), phi_tmp, sizeof(R) * nsites, cudaMemcpyDeviceToHost, s));
      DGPE_CK(cudaStreamSynchronize(s));
    }
    for (size_t i = 0; i < nsites; ++i) phi_host[i] = (double)tmp[i];
    return DGPE_OK;
  }
  int set_g(double g, cudaStream_t s) override {
    p.g = g;
    DGPE_CK(cudaMemcpyAsync(prm + PRM_G, &p.g, sizeof(double), cudaMemcpyHostToDevice, s));
    DGPE_CK(cudaStreamSynchronize(s));
    return DGPE_OK;
  }
  int set_mode(int mode, cudaStream_t s) override {
    if (mode != DGPE_IMAG && mode != DGPE_REAL) { err = "bad mode"; return DGPE_EINVAL; }
    if (strang && mode == DGPE_IMAG) { err = "Strang splitting is defined for real time"; return DGPE_EUNSUPPORTED; }
    if (rpsi && mode == DGPE_REAL) { err = "a real state is an imaginary-time option"; return DGPE_EUNSUPPORTED; }
    // fold the lazy scale into psi, then rebuild the CN tables and the graph
    k_fold_scale<R><<<152 * 8, 256, 0, s>>>(psi, prm, psi_elems());
    launched(1);
    DGPE_LCK(__func__);
    int rc = reset_scale(s);
    if (rc) return rc;
    p.mode = mode;
    imag = (mode == DGPE_IMAG);
    if ((rc = build_cn_tables())) return rc;
    if (use_graph && (rc = capture())) return rc;
    return DGPE_OK;
  }
  int set_modulation(const double *c, int M, cudaStream_t s) override {
    if (M < 0 || M > 16 || (M > 0 && !c)) { err = "M must be 0..16"; return DGPE_EINVAL; }
    double h[17] = {0};
    h[0] = (double)M;
    for (int i = 0; i < M; ++i) h[1 + i] = c[i];
    host_M = M;
    for (int i = 0; i < 16; ++i) host_cm[i] = (i < M) ? c[i] : 0.0;
    DGPE_CK(cudaMemcpyAsync(prm + PRM_M, h, sizeof(h), cudaMemcpyHostToDevice, s));
    DGPE_CK(cudaStreamSynchronize(s));
    return DGPE_OK;
  }
  // ---------------------------------------------------------- reverse mode
  int adj_alloc() {
    int rc;
    if (!adjG && (rc = dalloc(&adjG, nsites))) return rc;
    if (!adjT && (rc = dalloc(&adjT, nsites))) return rc;
    if (!adj_phi && (rc = dalloc(&adj_phi, nsites))) return rc;
    if (!adj_sig && (rc = dalloc(&adj_sig, nsites))) return rc;
    if (!adj_ksig && (rc = dalloc(&adj_ksig, nsites))) return rc;
    if (!adj_part && (rc = dalloc(&adj_part, 2 * 152 * 8))) return rc;
    if (!adj_acc && (rc = dalloc(&adj_acc, 17))) return rc;
    return DGPE_OK;
  }
  // One reverse step on device buffers; contributions added to adj_acc.
  int adjoint_on_device(const Cx *pin, Cx *G, long long st, cudaStream_t s) {
    int rc;
    // G_phi = C_x^dagger C_y^dagger C_z^dagger G'
    if (dim == 3 && (rc = launch_cn(2, false, s, G, true))) return rc;
    if ((rc = launch_cn(1, false, s, G, true))) return rc;
    if ((rc = launch_p1(2, s, G))) return rc;
    // Phi_d of the step-start state
    if (has_dip) {
      if ((rc = launch_dipolar_chain(s, pin))) return rc;
      if ((rc = launch_p1(1, s, nullptr, adj_phi))) return rc;
    } else {
      DGPE_CK(cudaMemsetAsync(adj_phi, 0, sizeof(R) * nsites, s));
    }
    const double t = (double)st * p.dt;
    double sm = 1.0;
    for (int m = 1; m <= host_M; ++m) sm += host_cm[m - 1] * std::sin((double)m * t);
    AArgs<R> A{};
    A.psi_in = pin; A.G = G; A.phi = adj_phi; A.sig = adj_sig; A.ksig = adj_ksig; A.sig_out = adj_sig;
    A.vx = vt[0]; A.vy = vt[1]; A.vz = vt[2]; A.partial = adj_part; A.nx = nx; A.ny = ny; A.dim = dim;
    A.n = nsites; A.dts = p.dt * sm; A.gdt = p.dt * p.g; A.gdddt = p.dt * p.gdd;
    A.two_dt_g = 2.0 * p.dt * p.g; A.two_dt_gdd = 2.0 * p.dt * p.gdd;
    const int nblk = 152 * 8;
    k_adj_sigma<R><<<nblk, 256, 0, s>>>(A);
    k_adj_accumulate<<<1, 256, 0, s>>>(adj_part, nblk, adj_acc, p.dt, t, host_M);
    launched(2);
    DGPE_LCK(__func__);
    if (has_dip) {
      if ((rc = launch_dipolar_chain(s, nullptr, adj_sig))) return rc;
      if ((rc = launch_p1(1, s, nullptr, adj_ksig))) return rc;
    } else {
      DGPE_CK(cudaMemsetAsync(adj_ksig, 0, sizeof(R) * nsites, s));
    }
    k_adj_update<R><<<nblk, 256, 0, s>>>(A);
    launched(1);
    DGPE_LCK(__func__);
    return DGPE_OK;
  }
  int step_adjoint(const void *psi_in, void *G, long long st, double *dg, double *dc,
                   cudaStream_t s) override {
    if (imag) { err = "the reverse step is defined for real time"; return DGPE_EUNSUPPORTED; }
    if (strang) { err = "the reverse step is defined for first-order splitting"; return DGPE_EUNSUPPORTED; }
    int rc = adj_alloc();
    if (rc) return rc;
    DGPE_CK(cudaMemsetAsync(adj_acc, 0, 17 * sizeof(double), s));
    if ((rc = adjoint_on_device((const Cx *)psi_in, (Cx *)G, st, s))) return rc;
    double acc[17];
    DGPE_CK(cudaMemcpyAsync(acc, adj_acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaStreamSynchronize(s));
    if (dg) *dg += acc[0];
    if (dc) for (int m = 0; m < host_M; ++m) dc[m] += acc[1 + m];
    return DGPE_OK;
  }
  // F = |<target|psi(T)>|^2 (h^d inner product) after nsteps steps from psi0,
  // and dF/dg, dF/dc_m by the reverse sweep with checkpoints every `every`
  // steps (states of one segment recomputed and kept while it is reversed).
  int fidelity_gradient(const double *psi0, const double *target, int nsteps, int every,
                        double *F, double *dFdg, double *dFdc, cudaStream_t s) override {
    if (imag) { err = "the reverse step is defined for real time"; return DGPE_EUNSUPPORTED; }
    if (strang) { err = "the reverse step is defined for first-order splitting"; return DGPE_EUNSUPPORTED; }
    if (nsteps < 1 || every < 1) { err = "nsteps and every must be >= 1"; return DGPE_EINVAL; }
    int rc = adj_alloc();
    if (rc) return rc;
    const int nseg = (nsteps + every - 1) / every;
    while ((int)ckpts.size() < nseg) { Cx *b = nullptr; if ((rc = dalloc(&b, nsites))) return rc; ckpts.push_back(b); }
    while ((int)states.size() < every) { Cx *b = nullptr; if ((rc = dalloc(&b, nsites))) return rc; states.push_back(b); }
    // target into adjT (stored precision)
    if ((rc = set_psi_host(target, s))) return rc;
    DGPE_CK(cudaMemcpyAsync(adjT, psi, sizeof(Cx) * nsites, cudaMemcpyDeviceToDevice, s));
    if ((rc = set_psi_host(psi0, s))) return rc;
    // forward with checkpoints
    for (int j = 0; j < nseg; ++j) {
      DGPE_CK(cudaMemcpyAsync(ckpts[j], psi, sizeof(Cx) * nsites, cudaMemcpyDeviceToDevice, s));
      const int len = std::min(every, nsteps - j * every);
      if ((rc = step(len, s))) return rc;
    }
    // c = h^d sum conj(target) psi_T, F = |c|^2, G_T = 2 h^d c target
    const int nblk = 152 * 8;
    k_cdot<R><<<nblk, 256, 0, s>>>(adjT, psi, nsites, adj_part);
    launched(1);
    DGPE_LCK(__func__);
    std::vector<double> part(2 * nblk);
    DGPE_CK(cudaMemcpyAsync(part.data(), adj_part, sizeof(double) * part.size(), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaStreamSynchronize(s));
    double cr = 0.0, ci = 0.0;
    for (int i = 0; i < nblk; ++i) { cr += part[2 * i]; ci += part[2 * i + 1]; }
    const double cell = p.h[0] * p.h[1] * (dim == 3 ? p.h[2] : 1.0);
    cr *= cell; ci *= cell;
    *F = cr * cr + ci * ci;
    k_cscale<R><<<nblk, 256, 0, s>>>(adjG, adjT, 2.0 * cell * cr, 2.0 * cell * ci, nsites);
    launched(1);
    DGPE_CK(cudaMemsetAsync(adj_acc, 0, 17 * sizeof(double), s));
    // reverse sweep
    for (int j = nseg - 1; j >= 0; --j) {
      const int len = std::min(every, nsteps - j * every);
      DGPE_CK(cudaMemcpyAsync(psi, ckpts[j], sizeof(Cx) * nsites, cudaMemcpyDeviceToDevice, s));
      long long st0 = (long long)j * every;
      DGPE_CK(cudaMemcpyAsync(dstep, &st0, sizeof(st0), cudaMemcpyHostToDevice, s));
      for (int i = 0; i < len; ++i) {
        DGPE_CK(cudaMemcpyAsync(states[i], psi, sizeof(Cx) * nsites, cudaMemcpyDeviceToDevice, s));
        if (i + 1 < len && (rc = step(1, s))) return rc;
      }
      for (int i = len - 1; i >= 0; --i)
        if ((rc = adjoint_on_device(states[i], adjG, st0 + i, s))) return rc;
    }
    double acc[17];
    DGPE_CK(cudaMemcpyAsync(acc, adj_acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaStreamSynchronize(s));
    *dFdg = acc[0];
    if (dFdc) for (int m = 0; m < host_M; ++m) dFdc[m] = acc[1 + m];
    return DGPE_OK;
  }

  int set_time(long long st, cudaStream_t s) override {
    DGPE_CK(cudaMemcpyAsync(dstep, &st, sizeof(st), cudaMemcpyHostToDevice, s));
    DGPE_CK(cudaStreamSynchronize(s));
    return DGPE_OK;
  }
  int get_time(long long *st, cudaStream_t s) override {
    DGPE_CK(cudaMemcpyAsync(st, dstep, sizeof(*st), cudaMemcpyDeviceToHost, s));
    DGPE_CK(cudaStreamSynchronize(s));
    return DGPE_OK;
  }
};

}  // namespace
}  // namespace dgpe
