// dgpe_noalloc.cu -- dgpe_dipolar_potential_noalloc: the dipolar-potential
// chain (density + R2C along x, transforms along y / z with the kernel
// multiply, C2R along x) on caller-owned device buffers, with every piece of
// scratch (half spectrum, U(k)/N table, FFT roots, parameter block) placed in
// one file-scope device array instead of memory from cudaMalloc.
//
// Who needs it: code that may not allocate device memory while it runs --
// work recorded into a stream capture by a host framework that owns every
// allocation, callers running under a fixed device-memory budget or a caching
// allocator that must see all allocations, and real-time loops where an
// allocation's latency and possible failure are not acceptable.
//
// The array below stays resident on every GPU that loads this library until
// the process exits.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "dgpe.h"
#include "dgpe_kernels.cuh"

namespace dgpe {
namespace {

constexpr size_t kScratchBytes = size_t(4) << 20;     // 4 MiB per device
constexpr size_t kMaxSites = size_t(1) << 18;         // largest grid accepted
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices];      // device address of g_scratch, per device
bool g_ready[kMaxDevices];
thread_local char g_err[256];  // fixed buffer: no allocation on error paths either

void set_err(const char *msg, const char *detail = nullptr) {
  if (detail) snprintf(g_err, sizeof(g_err), "%s: %s", msg, detail);
  else snprintf(g_err, sizeof(g_err), "%s", msg);
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Roots w[t] = exp(-2 pi i t / n) per axis, U(k)/N on the half spectrum
// [z][y][kx] (pitch px), and the parameter block (sc = 1, everything else 0).
template <typename R>
__global__ void k_noalloc_tables(cx<R> *tw0, cx<R> *tw1, cx<R> *tw2, R *U, double *prm,
                                 long long *step, int dim, int nx, int ny, int nz, int px,
                                 double hx, double hy, double hz, int kernel, double qd) {
  const size_t gid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t gs = (size_t)gridDim.x * blockDim.x;
  const int ns[3] = {nx, ny, nz};
  cx<R> *tw[3] = {tw0, tw1, tw2};
  for (int a = 0; a < dim; ++a)
    for (size_t t = gid; t < (size_t)ns[a]; t += gs) {
      double s, c;
      sincospi(-2.0 * (double)t / (double)ns[a], &s, &c);
      tw[a][t] = mk<R>((R)c, (R)s);
    }
  const int nxh = nx / 2 + 1;
  const size_t nspec = (size_t)nxh * ny * nz;
  const double N = (double)nx * ny * nz;
  const double twopi = 6.283185307179586476925286766559;
  for (size_t i = gid; i < nspec; i += gs) {
    const int kx = (int)(i % nxh);
    const size_t r = i / nxh;
    const int ky = (int)(r % ny), kz = (int)(r / ny);
    const double qx = twopi * (double)(kx <= nx / 2 ? kx : kx - nx) / (nx * hx);
    const double qy = twopi * (double)(ky <= ny / 2 ? ky : ky - ny) / (ny * hy);
    double u = 0.0;
    if (kernel == DGPE_KERNEL_DIPOLAR_3D) {
      const double qz = twopi * (double)(kz <= nz / 2 ? kz : kz - nz) / (nz * hz);
      const double k2 = qx * qx + qy * qy + qz * qz;
      u = (k2 == 0.0) ? 0.0 : (4.0 * M_PI / 3.0) * (3.0 * qz * qz / k2 - 1.0);
    } else if (kernel == DGPE_KERNEL_QUASI2D_XY) {
      const double q = sqrt(qx * qx + qy * qy) * qd, v = q / sqrt(2.0);
      double ex;
      if (v < 25.0) {
        ex = exp(v * v) * erfc(v);
      } else {  // asymptotic series of exp(v^2) erfc(v)
        double term = 1.0, sum = 1.0;
        for (int m = 1; m < 8; ++m) { term *= -(2.0 * m - 1.0) / (2.0 * v * v); sum += term; }
        ex = sum / (v * sqrt(M_PI));
      }
      u = (4.0 * M_PI / 3.0) / (sqrt(2.0 * M_PI) * qd) * (2.0 - 3.0 * sqrt(M_PI / 2.0) * q * ex);
    }
    U[r * px + kx] = (R)(u / N);
  }
  if (gid < PRM_COUNT) prm[gid] = (gid == PRM_SC) ? 1.0 : 0.0;
  if (gid == 0) *step = 0;
}

bool pow2_in_range(int n) { return n >= 32 && n <= 512 && (n & (n - 1)) == 0; }

bool make_plan_pow2(int n, int ept, FftPlan &pl) {
  pl.n = n;
  pl.ns = 0;
  int m = n;
  for (int R : {16, 8, 4, 2})
    while (m % R == 0 && ept % R == 0) { pl.rad[pl.ns++] = R; m /= R; }
  return m == 1;
}

template <typename K> cudaError_t smem_attr(K kernel, size_t bytes) {
  cudaError_t e = cudaSuccess;
  if (bytes > 48 * 1024) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return e;
}

template <typename R>
int run(const void *psi, void *phi, int dim, const int *n, const double *h, int kernel, double qd,
        cudaStream_t s, unsigned char *base) {
  typedef cx<R> Cx;
  constexpr int EPT_X = 8, EPT_S = sizeof(R) == 8 ? 8 : 16, CL = 16;
  constexpr int W = 128 / (int)sizeof(Cx), PW = 128 / (int)sizeof(Cx);
  const int nx = n[0], ny = n[1], nz = (dim == 3) ? n[2] : 1;
  const int nrows = ny * nz;
  int px = nx / 2 + 1;
  if (sizeof(Cx) == 8) px = (px + 1) & ~1;
  const int ncols = nx / 2 + 1;
  const size_t nspec = (size_t)px * nrows;
  // carve the scratch array
  size_t off = 0;
  Cx *spec = (Cx *)(base + off); off = align256(off + nspec * sizeof(Cx));
  R *U = (R *)(base + off); off = align256(off + nspec * sizeof(R));
  Cx *tw[3];
  for (int a = 0; a < 3; ++a) { tw[a] = (Cx *)(base + off); off = align256(off + 512 * sizeof(Cx)); }
  double *prm = (double *)(base + off); off = align256(off + PRM_COUNT * sizeof(double));
  long long *step = (long long *)(base + off); off = align256(off + sizeof(long long));
  if (off > kScratchBytes) { set_err("grid too large for the static scratch array"); return DGPE_EUNSUPPORTED; }

  FftPlan plx, ply, plz;
  if (!make_plan_pow2(nx, EPT_X, plx) || !make_plan_pow2(ny, EPT_S, ply) ||
      (dim == 3 && !make_plan_pow2(nz, EPT_S, plz))) {
    set_err("unsupported grid size");
    return DGPE_EUNSUPPORTED;
  }
  // x-line configuration (same rules as the solver's)
  const int TPL = nx / CL;
  const int LP = std::max(1, (sizeof(R) == 8 ? 64 : DGPE_MAXT / 2) / TPL);
  const int T = 2 * LP * TPL;
  const int pitchz = nx + nx / PW + 1, pitch = nx + nx / CL + 1;
  const size_t xsm = sizeof(Cx) * (size_t)(LP * pitchz + 2 * LP * pitch);
  const int xgrid = ((nrows + 1) / 2 + LP - 1) / LP;

  cudaError_t e;
  if ((e = smem_attr(k_dens_r2c_x<R, EPT_X>, xsm)) != cudaSuccess ||
      (e = smem_attr(k_c2r_x_exp_cnx<R, R, EPT_X, CL, 1>, xsm)) != cudaSuccess) {
    set_err("cudaFuncSetAttribute", cudaGetErrorString(e));
    return DGPE_ECUDA;
  }
  k_noalloc_tables<R><<<64, 256, 0, s>>>(tw[0], tw[1], tw[2], U, prm, step, dim, nx, ny, nz, px,
                                          h[0], h[1], dim == 3 ? h[2] : 1.0, kernel, qd);
  XArgs<R> X{};
  X.psi = (Cx *)psi; X.spec = spec; X.phi_out = (R *)phi; X.prm = prm; X.step = step;
  X.tw = tw[0]; X.pl = plx; X.nx = nx; X.ny = ny; X.nrows = nrows; X.px = px; X.LP = LP;
  X.pitchz = pitchz; X.pitch = pitch; X.TPL = TPL; X.C = CL; X.has_dip = 1;
  k_dens_r2c_x<R, EPT_X><<<xgrid, T, xsm, s>>>(X);
  auto strided = [&](int mode, int nn, long long es, long long os, int outer, const FftPlan &pl, const Cx *t) {
    const int w = std::max(1, std::min(W, DGPE_MAXT * EPT_S / nn));
    SArgs<R> A{};
    A.spec = spec; A.U = U; A.tw = t; A.pl = pl; A.estride = es; A.ostride = os; A.n = nn;
    A.ncols = ncols; A.W = w; A.nxh = nx / 2;
    dim3 grid((ncols + w - 1) / w, outer);
    const int TT = w * nn / EPT_S;
    const size_t sm = sizeof(Cx) * (size_t)nn * w;
    if (mode == 0) k_fft_strided<R, EPT_S, 0><<<grid, TT, sm, s>>>(A);
    else if (mode == 1) k_fft_strided<R, EPT_S, 1><<<grid, TT, sm, s>>>(A);
    else k_fft_strided<R, EPT_S, 2><<<grid, TT, sm, s>>>(A);
  };
  if (dim == 3) {
    strided(0, ny, px, (long long)ny * px, nz, ply, tw[1]);
    strided(2, nz, (long long)ny * px, px, ny, plz, tw[2]);
    strided(1, ny, px, (long long)ny * px, nz, ply, tw[1]);
  } else {
    strided(2, ny, px, (long long)ny * px, 1, ply, tw[1]);
  }
  k_c2r_x_exp_cnx<R, R, EPT_X, CL, 1><<<xgrid, T, xsm, s>>>(X);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    set_err("launch", cudaGetErrorString(e));
    return DGPE_ECUDA;
  }
  return DGPE_OK;
}

}  // namespace
}  // namespace dgpe

// Phi_d of |psi|^2 for a caller's state, without allocating device memory.
extern "C" int dgpe_dipolar_potential_noalloc(const void *psi, void *phi, int fp64, int dim,
                                              const int n[3], const double h[3], int kernel,
                                              double qd, void *cuda_stream) {
  using namespace dgpe;
  if (!psi || !phi || !n || !h) { set_err("NULL argument"); return DGPE_EINVAL; }
  if (dim != 2 && dim != 3) { set_err("dim must be 2 or 3"); return DGPE_EINVAL; }
  if (kernel == DGPE_KERNEL_QUASI2D_XZ) {
    set_err("the quasi-2D XZ kernel is not supported by this entry point");
    return DGPE_EUNSUPPORTED;
  }
  if ((kernel == DGPE_KERNEL_DIPOLAR_3D && dim != 3) ||
      (kernel == DGPE_KERNEL_QUASI2D_XY && (dim != 2 || !(qd > 0.0))) ||
      (kernel != DGPE_KERNEL_DIPOLAR_3D && kernel != DGPE_KERNEL_QUASI2D_XY)) {
    set_err("kernel does not match the dimension");
    return DGPE_EINVAL;
  }
  size_t sites = 1;
  for (int a = 0; a < dim; ++a) {
    if (!pow2_in_range(n[a])) { set_err("each n must be a power of two in [32, 512]"); return DGPE_EUNSUPPORTED; }
    if (!(h[a] > 0.0) || !std::isfinite(h[a])) { set_err("spacing must be > 0"); return DGPE_EINVAL; }
    sites *= (size_t)n[a];
  }
  if (sites > kMaxSites) {
    set_err("grid has more than 262144 sites, the limit of the static scratch array");
    return DGPE_EUNSUPPORTED;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_err("cudaGetDevice", cudaGetErrorString(e));
    return DGPE_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    set_err("device index above 63: this entry point serves devices 0..63");
    return DGPE_EUNSUPPORTED;
  }
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ready[dev]) {
      // first call on this device: look up where the array lives
      e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_scratch);
      if (e != cudaSuccess) {
        set_err("cudaGetSymbolAddress", cudaGetErrorString(e));
        return DGPE_ECUDA;
      }
      g_ready[dev] = true;
    }
    base = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  return fp64 ? run<double>(psi, phi, dim, n, h, kernel, qd, s, (unsigned char *)base)
              : run<float>(psi, phi, dim, n, h, kernel, qd, s, (unsigned char *)base);
}

extern "C" const char *dgpe_noalloc_last_error(void) { return dgpe::g_err; }
