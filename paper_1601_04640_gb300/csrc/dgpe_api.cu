// dgpe_api.cu -- the extern "C" boundary (declared in include/dgpe.h).
// Validates arguments, owns the handle, dispatches to the FP64 or the
// FP32-bulk engine, and turns every failure into a status code plus text.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "dgpe.h"
#include "dgpe_engine.cuh"

struct dgpe_solver {
  dgpe::Engine *eng = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
};

static thread_local std::string g_create_err;

static int fail(dgpe_t h, int code, const std::string &msg) {
  if (h) h->err = msg;
  else g_create_err = msg;
  return code;
}

static int from_engine(dgpe_t h, int rc) {
  if (rc != DGPE_OK) h->err = h->eng->err;
  return rc;
}

static bool good_len(int n) {
  if (n < 32 || n > 512 || (n & 1)) return false;
  int m = n;
  for (int f : {2, 3, 5})
    while (m % f == 0) m /= f;
  return m == 1;
}

extern "C" int dgpe_create(const dgpe_params *p, void *cuda_stream, dgpe_t *out) {
  if (!out) return fail(nullptr, DGPE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!p) return fail(nullptr, DGPE_EINVAL, "params is NULL");
  if (p->dim != 2 && p->dim != 3) return fail(nullptr, DGPE_EINVAL, "dim must be 2 or 3");
  if (p->dim == 2 && p->plane != DGPE_PLANE_XY && p->plane != DGPE_PLANE_XZ)
    return fail(nullptr, DGPE_EINVAL, "bad plane");
  for (int a = 0; a < p->dim; ++a) {
    if (!(p->h[a] > 0.0) || !std::isfinite(p->h[a])) return fail(nullptr, DGPE_EINVAL, "spacing must be > 0");
    if (!(p->nu[a] >= 0.0) || !std::isfinite(p->nu[a])) return fail(nullptr, DGPE_EINVAL, "trap frequency must be >= 0");
    if (!good_len(p->n[a]))
      return fail(nullptr, DGPE_EUNSUPPORTED, "each n must be an even 2^a 3^b 5^c in [32, 512]");
  }
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return fail(nullptr, DGPE_EINVAL, "dt must be > 0");
  if (!std::isfinite(p->g) || !std::isfinite(p->gdd)) return fail(nullptr, DGPE_EINVAL, "g, g_dd must be finite");
  if (p->mode != DGPE_IMAG && p->mode != DGPE_REAL) return fail(nullptr, DGPE_EINVAL, "bad mode");
  if (p->precision != DGPE_FP64 && p->precision != DGPE_FP32_BULK) return fail(nullptr, DGPE_EINVAL, "bad precision");
  if (p->kernel == DGPE_KERNEL_DIPOLAR_3D && p->dim != 3)
    return fail(nullptr, DGPE_EINVAL, "the 3D dipolar kernel needs dim 3");
  if (p->kernel == DGPE_KERNEL_QUASI2D_XY && (p->dim != 2 || p->plane != DGPE_PLANE_XY || !(p->qd > 0.0)))
    return fail(nullptr, DGPE_EINVAL, "the quasi-2D XY kernel needs dim 2, the XY plane and qd > 0");
  if (p->kernel == DGPE_KERNEL_QUASI2D_XZ && (p->dim != 2 || p->plane != DGPE_PLANE_XZ || !(p->qd > 0.0)))
    return fail(nullptr, DGPE_EINVAL, "the quasi-2D XZ kernel needs dim 2, the XZ plane and qd > 0");
  if (p->kernel < 0 || p->kernel > 3) return fail(nullptr, DGPE_EINVAL, "bad kernel");
  if ((p->flags & DGPE_FLAG_STRANG) && p->mode != DGPE_REAL)
    return fail(nullptr, DGPE_EUNSUPPORTED, "Strang splitting is defined for real time");
  if ((p->flags & DGPE_FLAG_REAL_PSI) && p->mode != DGPE_IMAG)
    return fail(nullptr, DGPE_EUNSUPPORTED, "a real state is an imaginary-time option");
  if ((p->flags & DGPE_FLAG_REAL_PSI) && (p->flags & DGPE_FLAG_CN_SERIAL))
    return fail(nullptr, DGPE_EUNSUPPORTED, "a real state uses the chunk-parallel CN solve");
  dgpe_solver *h = new (std::nothrow) dgpe_solver();
  if (!h) return fail(nullptr, DGPE_ENOMEM, "host allocation failed");
  h->stream = (cudaStream_t)cuda_stream;
  h->eng = (p->precision == DGPE_FP64) ? dgpe::make_engine_f64() : dgpe::make_engine_f32();
  int rc = h->eng->init(*p, h->stream);
  if (rc != DGPE_OK) {
    g_create_err = h->eng->err;
    delete h->eng;
    delete h;
    return rc;
  }
  *out = h;
  return DGPE_OK;
}

extern "C" void dgpe_destroy(dgpe_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  delete h->eng;
  delete h;
}

#define CHECK_H(h) \
  if (!(h)) return fail(nullptr, DGPE_EINVAL, "handle is NULL")

extern "C" int dgpe_set_psi(dgpe_t h, const double *psi, size_t n_sites) {
  CHECK_H(h);
  if (!psi) return fail(h, DGPE_EINVAL, "psi is NULL");
  if (n_sites != h->eng->sites()) return fail(h, DGPE_EINVAL, "n_sites does not match the grid");
  return from_engine(h, h->eng->set_psi_host(psi, h->stream));
}

extern "C" int dgpe_get_psi(dgpe_t h, double *psi, size_t n_sites) {
  CHECK_H(h);
  if (!psi) return fail(h, DGPE_EINVAL, "psi is NULL");
  if (n_sites != h->eng->sites()) return fail(h, DGPE_EINVAL, "n_sites does not match the grid");
  return from_engine(h, h->eng->get_psi_host(psi, h->stream));
}

extern "C" int dgpe_set_psi_device(dgpe_t h, const void *psi, size_t n_sites, int fp64) {
  CHECK_H(h);
  if (!psi) return fail(h, DGPE_EINVAL, "psi is NULL");
  if (n_sites != h->eng->sites()) return fail(h, DGPE_EINVAL, "n_sites does not match the grid");
  return from_engine(h, h->eng->set_psi_device(psi, fp64, h->stream));
}

extern "C" int dgpe_get_psi_device(dgpe_t h, void *psi, size_t n_sites, int fp64) {
  CHECK_H(h);
  if (!psi) return fail(h, DGPE_EINVAL, "psi is NULL");
  if (n_sites != h->eng->sites()) return fail(h, DGPE_EINVAL, "n_sites does not match the grid");
  return from_engine(h, h->eng->get_psi_device(psi, fp64, h->stream));
}

extern "C" int dgpe_step(dgpe_t h, int n) {
  CHECK_H(h);
  if (n < 0) return fail(h, DGPE_EINVAL, "n must be >= 0");
  return from_engine(h, h->eng->step(n, h->stream));
}

extern "C" int dgpe_observables(dgpe_t h, dgpe_obs *o) {
  CHECK_H(h);
  if (!o) return fail(h, DGPE_EINVAL, "obs is NULL");
  return from_engine(h, h->eng->observables(o, h->stream));
}

extern "C" int dgpe_dipolar_potential(dgpe_t h, double *phi, size_t n_sites) {
  CHECK_H(h);
  if (!phi) return fail(h, DGPE_EINVAL, "phi is NULL");
  if (n_sites != h->eng->sites()) return fail(h, DGPE_EINVAL, "n_sites does not match the grid");
  return from_engine(h, h->eng->dipolar_potential(phi, h->stream));
}

extern "C" int dgpe_set_g(dgpe_t h, double g) {
  CHECK_H(h);
  if (!std::isfinite(g)) return fail(h, DGPE_EINVAL, "g must be finite");
  return from_engine(h, h->eng->set_g(g, h->stream));
}

extern "C" int dgpe_set_mode(dgpe_t h, int mode) {
  CHECK_H(h);
  return from_engine(h, h->eng->set_mode(mode, h->stream));
}

extern "C" int dgpe_set_trap_modulation(dgpe_t h, const double *c, int M) {
  CHECK_H(h);
  return from_engine(h, h->eng->set_modulation(c, M, h->stream));
}

extern "C" int dgpe_set_time(dgpe_t h, long long step) {
  CHECK_H(h);
  if (step < 0) return fail(h, DGPE_EINVAL, "step must be >= 0");
  return from_engine(h, h->eng->set_time(step, h->stream));
}

extern "C" int dgpe_get_time(dgpe_t h, long long *step) {
  CHECK_H(h);
  if (!step) return fail(h, DGPE_EINVAL, "step is NULL");
  return from_engine(h, h->eng->get_time(step, h->stream));
}

extern "C" int dgpe_sync(dgpe_t h) {
  CHECK_H(h);
  cudaError_t e = h->stream ? cudaStreamSynchronize(h->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(h, DGPE_ECUDA, std::string("sync: ") + cudaGetErrorString(e));
  return from_engine(h, h->eng->wait_status(h->stream));
}

extern "C" int dgpe_launches_per_step(dgpe_t h) {
  if (!h) return fail(nullptr, DGPE_EINVAL, "handle is NULL");
  return h->eng->launches_per_step();
}

extern "C" const char *dgpe_last_error(dgpe_t h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

extern "C" int dgpe_profile_steps(dgpe_t h, int n, double *pass_ms, int cap) {
  CHECK_H(h);
  if (n < 0 || !pass_ms) return fail(h, DGPE_EINVAL, "bad arguments");
  int rc = h->eng->profile_steps(n, pass_ms, cap, h->stream);
  if (rc < 0) h->err = h->eng->err;
  return rc;
}

extern "C" const char *dgpe_pass_name(dgpe_t h, int i) { return h ? h->eng->pass_name(i) : ""; }

extern "C" double dgpe_pass_bytes(dgpe_t h, int i) { return h ? h->eng->pass_bytes(i) : 0.0; }
extern "C" double dgpe_pass_flops(dgpe_t h, int i) { return h ? h->eng->pass_flops(i) : 0.0; }
extern "C" long long dgpe_kernel_launches(dgpe_t h) { return h ? h->eng->kernel_launches() : 0; }

extern "C" int dgpe_step_adjoint(dgpe_t h, const void *psi_in, void *G, long long step, double *dL_dg,
                                 double *dL_dc) {
  CHECK_H(h);
  if (!psi_in || !G || step < 0) return fail(h, DGPE_EINVAL, "bad arguments");
  return from_engine(h, h->eng->step_adjoint(psi_in, G, step, dL_dg, dL_dc, h->stream));
}

extern "C" int dgpe_fidelity_gradient(dgpe_t h, const double *psi0, const double *target, int nsteps,
                                      int every, double *F, double *dF_dg, double *dF_dc) {
  CHECK_H(h);
  if (!psi0 || !target || !F || !dF_dg) return fail(h, DGPE_EINVAL, "NULL argument");
  return from_engine(h, h->eng->fidelity_gradient(psi0, target, nsteps, every, F, dF_dg, dF_dc, h->stream));
}
