// dgpe_plain.cu -- the comparison step: the same split step built the way the
// paper's programs build it ("Summary of revisions": a series of grid-stride
// kernels, cuFFT real-to-complex / complex-to-real transforms for the dipolar
// term, and Crank-Nicolson recursions with one thread per grid line and the
// forward-sweep values kept in a temporary array).  Timed only, beside the
// fused path in libdgpe.so; never used by it.
#include <cufft.h>

#include <cmath>
#include <complex>
#include <string>
#include <vector>

#include "dgpe.h"
#include "dgpe_plain.h"

namespace {

template <typename R> struct V2;
template <> struct V2<double> { using T = double2; };
template <> struct V2<float> { using T = float2; };

thread_local std::string g_err;

template <typename R>
__global__ void k_pl_density(const typename V2<R>::T *psi, R *dens, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    auto v = psi[i];
    dens[i] = v.x * v.x + v.y * v.y;
  }
}

template <typename R>
__global__ void k_pl_mul(typename V2<R>::T *spec, const R *U, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    auto v = spec[i];
    const R u = U[i];
    v.x *= u;
    v.y *= u;
    spec[i] = v;
  }
}

// psi <- psi exp(-kappa dt (V + g n + g_dd Phi))
template <typename R>
__global__ void k_pl_nonlin(typename V2<R>::T *psi, const R *phi, int nx, int ny, int nz, R hx, R hy, R hz,
                            R nx2, R ny2, R nz2, R dt, R g, R gdd, int imag, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx);
    const size_t r = i / nx;
    const int y = (int)(r % ny), z = (int)(r / ny);
    const R X = (R)(x - nx / 2) * hx, Y = (R)(y - ny / 2) * hy, Z = (R)(z - nz / 2) * hz;
    const R V = (R)0.5 * (nx2 * X * X + ny2 * Y * Y + nz2 * Z * Z);
    auto v = psi[i];
    const R th = dt * (V + g * (v.x * v.x + v.y * v.y) + gdd * phi[i]);
    if (imag) {
      const R f = exp(-th);
      v.x *= f;
      v.y *= f;
    } else {
      R s, c;
      sincos(th, &s, &c);
      const R a = v.x * c + v.y * s, b = v.y * c - v.x * s;
      v.x = a;
      v.y = b;
    }
    psi[i] = v;
  }
}

// One thread per line: B psi on the fly, forward sweep into tmp, back
// substitution into psi.  tab: m_a (1 / pivot) and c'_a, complex, FP64-built.
template <typename R>
__global__ void k_pl_cn(typename V2<R>::T *psi, typename V2<R>::T *tmp, const typename V2<R>::T *tab, int n,
                        long long nlines, int axis, int nx, int ny, R kre, R kim) {
  typedef typename V2<R>::T C;
  const long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (L >= nlines) return;
  size_t base, stride;
  if (axis == 0) { base = (size_t)L * nx; stride = 1; }
  else if (axis == 1) { const long long x = L % nx, z = L / nx; base = (size_t)z * nx * ny + x; stride = nx; }
  else { base = (size_t)L; stride = (size_t)nx * ny; }
  const C *tm = tab, *tc = tab + n;
  // B = I - kt T: diag 1 - 2 kt, off +kt;  lower of A: a = -kt
  C prev = {0, 0}, cur = psi[base], dprev = {0, 0};
  for (int i = 0; i < n; ++i) {
    C nxt = (i + 1 < n) ? psi[base + (size_t)(i + 1) * stride] : C{0, 0};
    const R sr = prev.x + nxt.x, si = prev.y + nxt.y;
    // d = (1 - 2 kt) cur + kt (prev + next)
    C d;
    d.x = cur.x - 2 * (kre * cur.x - kim * cur.y) + (kre * sr - kim * si);
    d.y = cur.y - 2 * (kre * cur.y + kim * cur.x) + (kre * si + kim * sr);
    // d' = (d - a d'_{i-1}) m_i, a = -kt
    const R ax = kre * dprev.x - kim * dprev.y, ay = kre * dprev.y + kim * dprev.x;
    const R ux = d.x + ax, uy = d.y + ay;
    const C m = tm[i];
    C dp;
    dp.x = ux * m.x - uy * m.y;
    dp.y = ux * m.y + uy * m.x;
    tmp[base + (size_t)i * stride] = dp;
    dprev = dp;
    prev = cur;
    cur = nxt;
  }
  C xn = {0, 0};
  for (int i = n - 1; i >= 0; --i) {
    const C dp = tmp[base + (size_t)i * stride];
    const C c = tc[i];
    C x;
    x.x = dp.x - (c.x * xn.x - c.y * xn.y);
    x.y = dp.y - (c.x * xn.y + c.y * xn.x);
    psi[base + (size_t)i * stride] = x;
    xn = x;
  }
}

struct PlainBase {
  virtual ~PlainBase() {}
  virtual int init(const dgpe_params &p, cudaStream_t s) = 0;
  virtual int set_psi(const double *h) = 0;
  virtual int get_psi(double *h) = 0;
  virtual int step(int n) = 0;
};

#define PCK(call)                                                                    \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) { g_err = std::string(#call) + ": " + cudaGetErrorString(e_); return DGPE_ECUDA; } \
  } while (0)
#define FCK(call)                                                                    \
  do {                                                                               \
    cufftResult r_ = (call);                                                         \
    if (r_ != CUFFT_SUCCESS) { g_err = std::string(#call) + " failed: " + std::to_string((int)r_); return DGPE_ECUDA; } \
  } while (0)

template <typename R> struct Plain : PlainBase {
  typedef typename V2<R>::T C;
  dgpe_params p{};
  cudaStream_t s = nullptr;
  int nx = 0, ny = 0, nz = 1, dim = 3;
  size_t N = 0, NS = 0;
  C *psi = nullptr, *spec = nullptr, *tmp = nullptr, *tab[3] = {nullptr, nullptr, nullptr};
  R *dens = nullptr, *U = nullptr;
  cufftHandle fwd = 0, inv = 0;
  bool plans = false;
  double kt_im[3] = {0, 0, 0}, kt_re[3] = {0, 0, 0};

  ~Plain() override {
    if (plans) { cufftDestroy(fwd); cufftDestroy(inv); }
    void *b[] = {psi, spec, tmp, tab[0], tab[1], tab[2], dens, U};
    for (void *x : b) if (x) cudaFree(x);
  }
  int init(const dgpe_params &pin, cudaStream_t st) override {
    p = pin;
    s = st;
    dim = p.dim;
    nx = p.n[0]; ny = p.n[1]; nz = (dim == 3) ? p.n[2] : 1;
    N = (size_t)nx * ny * nz;
    NS = (size_t)(nx / 2 + 1) * ny * nz;
    PCK(cudaMalloc(&psi, N * sizeof(C)));
    PCK(cudaMalloc(&tmp, N * sizeof(C)));
    PCK(cudaMalloc(&spec, NS * sizeof(C)));
    PCK(cudaMalloc(&dens, N * sizeof(R)));
    PCK(cudaMalloc(&U, NS * sizeof(R)));
    const bool f64 = sizeof(R) == 8;
    if (dim == 3) {
      FCK(cufftPlan3d(&fwd, nz, ny, nx, f64 ? CUFFT_D2Z : CUFFT_R2C));
      FCK(cufftPlan3d(&inv, nz, ny, nx, f64 ? CUFFT_Z2D : CUFFT_C2R));
    } else {
      FCK(cufftPlan2d(&fwd, ny, nx, f64 ? CUFFT_D2Z : CUFFT_R2C));
      FCK(cufftPlan2d(&inv, ny, nx, f64 ? CUFFT_Z2D : CUFFT_C2R));
    }
    plans = true;
    FCK(cufftSetStream(fwd, s));
    FCK(cufftSetStream(inv, s));
    // U(k)/N on cuFFT's half spectrum [z][y][kx]
    std::vector<R> hu(NS);
    const int nxh = nx / 2 + 1;
    auto kv = [](int j, int n, double h) { int jj = (j <= n / 2) ? j : j - n; return 2.0 * M_PI * jj / (n * h); };
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nxh; ++x) {
          const double qx = kv(x, nx, p.h[0]), qy = kv(y, ny, p.h[1]);
          double u = 0.0;
          if (p.kernel == DGPE_KERNEL_DIPOLAR_3D) {
            const double qz = kv(z, nz, p.h[2]), k2 = qx * qx + qy * qy + qz * qz;
            u = (k2 == 0.0) ? 0.0 : (4.0 * M_PI / 3.0) * (3.0 * qz * qz / k2 - 1.0);
          } else if (p.kernel == DGPE_KERNEL_QUASI2D_XY) {
            const double q = std::sqrt(qx * qx + qy * qy) * p.qd, v = q / std::sqrt(2.0);
            const double ex = (v < 25.0) ? std::exp(v * v) * std::erfc(v) : 1.0 / (v * std::sqrt(M_PI));
            u = (4.0 * M_PI / 3.0) / (std::sqrt(2.0 * M_PI) * p.qd) * (2.0 - 3.0 * std::sqrt(M_PI / 2.0) * q * ex);
          }
          hu[((size_t)z * ny + y) * nxh + x] = (R)(u / (double)N);
        }
    PCK(cudaMemcpy(U, hu.data(), NS * sizeof(R), cudaMemcpyHostToDevice));
    const int ns[3] = {nx, ny, nz};
    for (int a = 0; a < dim; ++a) {
      const double tau = p.dt / (4.0 * p.h[a] * p.h[a]);
      const std::complex<double> kt = (p.mode == DGPE_IMAG) ? std::complex<double>(tau, 0) : std::complex<double>(0, tau);
      kt_re[a] = kt.real();
      kt_im[a] = kt.imag();
      const int n = ns[a];
      std::vector<C> t(2 * (size_t)n);
      const std::complex<double> b = 1.0 + 2.0 * kt, al = -kt;
      std::complex<double> cp = 0.0;
      for (int i = 0; i < n; ++i) {
        const std::complex<double> den = b - al * cp;  // pivot
        const std::complex<double> m = 1.0 / den;
        cp = al * m;  // c'_i = (upper) / pivot, upper = -kt
        t[i].x = (R)m.real(); t[i].y = (R)m.imag();
        t[n + i].x = (R)cp.real(); t[n + i].y = (R)cp.imag();
      }
      PCK(cudaMalloc(&tab[a], 2 * (size_t)n * sizeof(C)));
      PCK(cudaMemcpy(tab[a], t.data(), 2 * (size_t)n * sizeof(C), cudaMemcpyHostToDevice));
    }
    return DGPE_OK;
  }
  int set_psi(const double *h) override {
    std::vector<C> t(N);
    for (size_t i = 0; i < N; ++i) { t[i].x = (R)h[2 * i]; t[i].y = (R)h[2 * i + 1]; }
    PCK(cudaMemcpy(psi, t.data(), N * sizeof(C), cudaMemcpyHostToDevice));
    return DGPE_OK;
  }
  int get_psi(double *h) override {
    std::vector<C> t(N);
    PCK(cudaStreamSynchronize(s));
    PCK(cudaMemcpy(t.data(), psi, N * sizeof(C), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < N; ++i) { h[2 * i] = t[i].x; h[2 * i + 1] = t[i].y; }
    return DGPE_OK;
  }
  int exec_fwd() {
    if (sizeof(R) == 8) FCK(cufftExecD2Z(fwd, (cufftDoubleReal *)dens, (cufftDoubleComplex *)spec));
    else FCK(cufftExecR2C(fwd, (cufftReal *)dens, (cufftComplex *)spec));
    return DGPE_OK;
  }
  int exec_inv() {
    if (sizeof(R) == 8) FCK(cufftExecZ2D(inv, (cufftDoubleComplex *)spec, (cufftDoubleReal *)dens));
    else FCK(cufftExecC2R(inv, (cufftComplex *)spec, (cufftReal *)dens));
    return DGPE_OK;
  }
  int step(int nsteps) override {
    const int G = 152 * 8, T = 256;
    const int ns[3] = {nx, ny, nz};
    for (int k = 0; k < nsteps; ++k) {
      int rc;
      if (p.kernel != DGPE_KERNEL_NONE) {
        k_pl_density<R><<<G, T, 0, s>>>(psi, dens, N);
        if ((rc = exec_fwd())) return rc;
        k_pl_mul<R><<<G, T, 0, s>>>(spec, U, NS);
        if ((rc = exec_inv())) return rc;
      } else {
        PCK(cudaMemsetAsync(dens, 0, N * sizeof(R), s));
      }
      k_pl_nonlin<R><<<G, T, 0, s>>>(psi, dens, nx, ny, nz, (R)p.h[0], (R)p.h[1], (R)(dim == 3 ? p.h[2] : 1.0),
                                     (R)(p.nu[0] * p.nu[0]), (R)(p.nu[1] * p.nu[1]),
                                     (R)(dim == 3 ? p.nu[2] * p.nu[2] : 0.0), (R)p.dt, (R)p.g, (R)p.gdd,
                                     p.mode == DGPE_IMAG, N);
      for (int a = 0; a < dim; ++a) {
        const long long nl = (long long)(N / ns[a]);
        k_pl_cn<R><<<(unsigned)((nl + 127) / 128), 128, 0, s>>>(psi, tmp, tab[a], ns[a], nl, a, nx, ny,
                                                                (R)kt_re[a], (R)kt_im[a]);
      }
      PCK(cudaGetLastError());
    }
    return DGPE_OK;
  }
};

}  // namespace

struct dgpe_plain_solver {
  PlainBase *impl = nullptr;
};

extern "C" int dgpe_plain_create(const dgpe_params *p, void *stream, dgpe_plain_t *out) {
  if (!p || !out) { g_err = "NULL argument"; return DGPE_EINVAL; }
  *out = nullptr;
  if (p->mode == DGPE_IMAG) { g_err = "the comparison step is real time only"; return DGPE_EUNSUPPORTED; }
  dgpe_plain_solver *h = new dgpe_plain_solver();
  if (p->precision == DGPE_FP64) h->impl = new Plain<double>();
  else h->impl = new Plain<float>();
  int rc = h->impl->init(*p, (cudaStream_t)stream);
  if (rc) { delete h->impl; delete h; return rc; }
  *out = h;
  return DGPE_OK;
}

extern "C" void dgpe_plain_destroy(dgpe_plain_t h) {
  if (!h) return;
  cudaDeviceSynchronize();
  delete h->impl;
  delete h;
}

extern "C" int dgpe_plain_set_psi(dgpe_plain_t h, const double *psi) { return h ? h->impl->set_psi(psi) : DGPE_EINVAL; }
extern "C" int dgpe_plain_get_psi(dgpe_plain_t h, double *psi) { return h ? h->impl->get_psi(psi) : DGPE_EINVAL; }
extern "C" int dgpe_plain_step(dgpe_plain_t h, int n) { return h ? h->impl->step(n) : DGPE_EINVAL; }
extern "C" const char *dgpe_plain_last_error(void) { return g_err.c_str(); }
