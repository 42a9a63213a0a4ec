// dgpe_batch.cu -- many independent 2D XY condensates (a parameter sweep over
// grid size, trap anisotropy, g and g_dd, in imaginary and real time) stepped
// together: problems are grouped into classes of equal grid size and mode;
// each class runs the four 2D passes (density + R2C_x, FFT_y . U . IFFT_y,
// C2R_x + exponential + CN_x, CN_y + norm) as batched kernels with one problem
// per blockIdx.z; every class's tile schedule is picked by timing candidates
// at create time; the whole step of all classes is one CUDA graph whose
// branches (one per class) run concurrently.  FP32-bulk form.
#include <algorithm>
#include <cstdio>
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
  ~dgpe_batch() {
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

// Autotuner: for each class time the candidate tile schedules (x-tile lines
// per CTA LP and LP/2; strided tile widths W and W/2) on the class's own
// problems and keep the fastest.  The timed steps advance the states, which
// are restored afterwards by the caller (create runs before any set_psi).
int autotune(dgpe_batch *b, Cls &c) {
  Eng *e0 = b->eng[c.members[0]];
  const int LP0 = e0->x_LP, sW0 = e0->fy.W, cW0 = e0->cn[1].W;
  struct Cand { int LP, sW, cW; };
  std::vector<Cand> cands;
  for (int lp : {LP0, std::max(1, LP0 / 2)})
    for (int sw : {sW0, std::max(1, sW0 / 2)})
      for (int cw : {cW0, std::max(1, cW0 / 2)}) {
        bool dup = false;
        for (auto &q : cands) dup |= (q.LP == lp && q.sW == sw && q.cW == cw);
        if (!dup) cands.push_back({lp, sw, cw});
      }
  cudaEvent_t a, z;
  BCK(cudaEventCreate(&a));
  BCK(cudaEventCreate(&z));
  float best = 1e30f;
  Cand pick = cands[0];
  for (const Cand &q : cands) {
    int rc;
    if ((rc = configure(b, c, q.LP, q.sW, q.cW))) return rc;
    if ((rc = set_attrs(b, c))) return rc;
    if ((rc = launch_class(b, c, c.st))) return rc;  // warm-up
    BCK(cudaEventRecord(a, c.st));
    for (int r = 0; r < 3; ++r)
      if ((rc = launch_class(b, c, c.st))) return rc;
    BCK(cudaEventRecord(z, c.st));
    BCK(cudaEventSynchronize(z));
    float ms = 0.f;
    BCK(cudaEventElapsedTime(&ms, a, z));
    if (ms < best) { best = ms; pick = q; }
  }
  BCK(cudaEventDestroy(a));
  BCK(cudaEventDestroy(z));
  int rc;
  if ((rc = configure(b, c, pick.LP, pick.sW, pick.cW))) return rc;
  return set_attrs(b, c);
}

// One step of every class as one graph: the capture stream forks into one
// branch per class (the class's own stream), the branches join back before
// the capture ends, so the classes' kernels are free to run concurrently.
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
  int rc = capture(b);
  if (rc) return fail(rc);
  {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) { b->err = std::string("after capture: ") + cudaGetErrorString(e); return fail(DGPE_ECUDA); }
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
  int rc = b->eng[i]->get_psi_host(psi, b->stream);
  if (rc) b->err = b->eng[i]->err;
  return rc;
}

extern "C" int dgpe_batch_step(dgpe_batch_t b, int n) {
  if (!b || n < 0) return DGPE_EINVAL;
  for (int k = 0; k < n; ++k) {
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) { b->err = std::string("graph launch: ") + cudaGetErrorString(e); return DGPE_ECUDA; }
  }
  return DGPE_OK;
}

extern "C" int dgpe_batch_observables(dgpe_batch_t b, int i, dgpe_obs *o) {
  if (!b || i < 0 || i >= (int)b->eng.size() || !o) return DGPE_EINVAL;
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

extern "C" int dgpe_batch_launches_per_step(dgpe_batch_t b) { return b ? 4 * (int)b->cls.size() : 0; }

extern "C" const char *dgpe_batch_last_error(dgpe_batch_t b) { return b ? b->err.c_str() : g_batch_err.c_str(); }
