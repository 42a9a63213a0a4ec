"""Thin ctypes binding of the C ABI in include/dgpe.h (libdgpe.so).

Argument marshalling only: every step of the solver runs in the CUDA kernels
of libdgpe.so.  There is no CPU fallback; if the library has not been built
(``paper_1601_04640_gb300.build.build()``) the first call raises.

Function names match the C entry points (``dgpe_create``, ``dgpe_step``, ...).
``Solver`` is a small convenience wrapper over them.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgpe.so")

DGPE_OK = 0
DGPE_EINVAL = -1
DGPE_EUNSUPPORTED = -2
DGPE_ENOMEM = -3
DGPE_ECUDA = -4
DGPE_ENONFINITE = -5
DGPE_ETIMEOUT = -6

DGPE_IMAG = 0
DGPE_REAL = 1
DGPE_FP64 = 0
DGPE_FP32_BULK = 1
DGPE_KERNEL_NONE = 0
DGPE_KERNEL_DIPOLAR_3D = 1
DGPE_KERNEL_QUASI2D_XY = 2
DGPE_KERNEL_QUASI2D_XZ = 3
DGPE_PLANE_XY = 0
DGPE_PLANE_XZ = 1
DGPE_FLAG_NO_GRAPH = 1
DGPE_FLAG_CN_SERIAL = 2
DGPE_FLAG_CN_CHUNKED = 4
DGPE_FLAG_STRANG = 8
DGPE_FLAG_REAL_PSI = 16
DGPE_FLAG_P1_ONESHOT = 32
DGPE_FLAG_BATCH_CLASSES = 64

EXPORTS = [
    "dgpe_create", "dgpe_destroy", "dgpe_set_psi", "dgpe_get_psi", "dgpe_set_psi_device",
    "dgpe_get_psi_device", "dgpe_step", "dgpe_observables", "dgpe_dipolar_potential",
    "dgpe_set_g", "dgpe_set_mode", "dgpe_set_trap_modulation", "dgpe_set_time",
    "dgpe_get_time", "dgpe_sync", "dgpe_launches_per_step", "dgpe_last_error",
    "dgpe_profile_steps", "dgpe_pass_name", "dgpe_pass_bytes", "dgpe_pass_flops", "dgpe_kernel_launches",
    "dgpe_dipolar_potential_noalloc", "dgpe_noalloc_last_error",
    "dgpe_step_adjoint", "dgpe_fidelity_gradient",
    "dgpe_batch_create", "dgpe_batch_destroy", "dgpe_batch_set_psi", "dgpe_batch_get_psi",
    "dgpe_batch_step", "dgpe_batch_observables", "dgpe_batch_info", "dgpe_batch_launches_per_step",
    "dgpe_batch_last_error", "dgpe_batch_sync", "dgpe_batch_hold_problem", "dgpe_batch_set_wait_limit",
]


class dgpe_params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("plane", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3),
        ("nu", C.c_double * 3), ("g", C.c_double), ("gdd", C.c_double), ("dt", C.c_double),
        ("mode", C.c_int), ("precision", C.c_int), ("kernel", C.c_int), ("qd", C.c_double),
        ("flags", C.c_uint),
    ]


class dgpe_obs(C.Structure):
    _fields_ = [
        ("norm", C.c_double), ("mu", C.c_double), ("energy", C.c_double),
        ("rms", C.c_double * 3), ("rms_r", C.c_double), ("t", C.c_double),
        ("kin", C.c_double), ("pot", C.c_double), ("contact", C.c_double),
        ("dipolar", C.c_double),
    ]


class DgpeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("dgpe error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load libdgpe.so; raise if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("libdgpe.so not built: run paper_1601_04640_gb300.build.build()")
        lib = C.CDLL(path)
        H = C.c_void_p
        P = C.POINTER(dgpe_params)
        lib.dgpe_create.argtypes = [P, C.c_void_p, C.POINTER(H)]
        lib.dgpe_destroy.argtypes = [H]
        lib.dgpe_destroy.restype = None
        for f in ("dgpe_set_psi", "dgpe_get_psi", "dgpe_dipolar_potential"):
            getattr(lib, f).argtypes = [H, C.c_void_p, C.c_size_t]
        lib.dgpe_set_psi_device.argtypes = [H, C.c_void_p, C.c_size_t, C.c_int]
        lib.dgpe_get_psi_device.argtypes = [H, C.c_void_p, C.c_size_t, C.c_int]
        lib.dgpe_step.argtypes = [H, C.c_int]
        lib.dgpe_observables.argtypes = [H, C.POINTER(dgpe_obs)]
        lib.dgpe_set_g.argtypes = [H, C.c_double]
        lib.dgpe_set_mode.argtypes = [H, C.c_int]
        lib.dgpe_set_trap_modulation.argtypes = [H, C.POINTER(C.c_double), C.c_int]
        lib.dgpe_set_time.argtypes = [H, C.c_longlong]
        lib.dgpe_get_time.argtypes = [H, C.POINTER(C.c_longlong)]
        lib.dgpe_sync.argtypes = [H]
        lib.dgpe_launches_per_step.argtypes = [H]
        lib.dgpe_last_error.argtypes = [H]
        lib.dgpe_last_error.restype = C.c_char_p
        lib.dgpe_profile_steps.argtypes = [H, C.c_int, C.POINTER(C.c_double), C.c_int]
        lib.dgpe_pass_name.argtypes = [H, C.c_int]
        lib.dgpe_pass_name.restype = C.c_char_p
        lib.dgpe_pass_bytes.argtypes = [H, C.c_int]
        lib.dgpe_pass_bytes.restype = C.c_double
        lib.dgpe_pass_flops.argtypes = [H, C.c_int]
        lib.dgpe_pass_flops.restype = C.c_double
        lib.dgpe_kernel_launches.argtypes = [H]
        lib.dgpe_kernel_launches.restype = C.c_longlong
        lib.dgpe_dipolar_potential_noalloc.argtypes = [
            C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double),
            C.c_int, C.c_double, C.c_void_p]
        lib.dgpe_noalloc_last_error.argtypes = []
        lib.dgpe_noalloc_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _check(rc, h=None):
    if rc != DGPE_OK:
        msg = load().dgpe_last_error(h)
        raise DgpeError(rc, msg.decode() if msg else "")
    return rc


def make_params(dim, n, h, nu, g=0.0, gdd=0.0, dt=1e-3, imag=False, fp64=True,
                kernel=None, qd=0.5, graph=True, cn=None, plane=None, split="lie", real_psi=False,
                flags=0):
    """cn: None (automatic), "serial" or "chunked" (FP64 Crank-Nicolson form).
    split: "lie" (the paper's first-order step) or "strang" (second order,
    real time).  real_psi: hold the state as a real field (imaginary time).
    plane (2D): "xy" or "xz"; default XZ for the XZ kernel, else XY.  For XZ the
    second axis is z: n, h, nu = (nx, nz), (hx, hz), (nu_x, nu_z)."""
    p = dgpe_params()
    p.dim = dim
    if plane is None:
        plane = "xz" if kernel == DGPE_KERNEL_QUASI2D_XZ else "xy"
    p.plane = {"xy": DGPE_PLANE_XY, "xz": DGPE_PLANE_XZ}[plane]
    nn = list(n) + [1] * (3 - len(n))
    hh = list(h) + [1.0] * (3 - len(h))
    vv = list(nu) + [0.0] * (3 - len(nu))
    for i in range(3):
        p.n[i] = int(nn[i]); p.h[i] = float(hh[i]); p.nu[i] = float(vv[i])
    p.g = float(g); p.gdd = float(gdd); p.dt = float(dt)
    p.mode = DGPE_IMAG if imag else DGPE_REAL
    p.precision = DGPE_FP64 if fp64 else DGPE_FP32_BULK
    if kernel is None:
        kernel = DGPE_KERNEL_DIPOLAR_3D if dim == 3 else DGPE_KERNEL_QUASI2D_XY
    p.kernel = kernel
    p.qd = float(qd)
    p.flags = 0 if graph else DGPE_FLAG_NO_GRAPH
    if cn == "serial":
        p.flags |= DGPE_FLAG_CN_SERIAL
    elif cn == "chunked":
        p.flags |= DGPE_FLAG_CN_CHUNKED
    elif cn is not None:
        raise ValueError("cn must be None, 'serial' or 'chunked'")
    if split == "strang":
        p.flags |= DGPE_FLAG_STRANG
    elif split != "lie":
        raise ValueError("split must be 'lie' or 'strang'")
    if real_psi:
        p.flags |= DGPE_FLAG_REAL_PSI
    p.flags |= int(flags)
    return p


# ------------------------------------------------------- C-ABI-named calls
def dgpe_create(params: dgpe_params, stream: int = 0):
    h = C.c_void_p()
    _check(load().dgpe_create(C.byref(params), C.c_void_p(stream), C.byref(h)))
    return h


def dgpe_destroy(h):
    load().dgpe_destroy(h)


def dgpe_set_psi(h, psi: np.ndarray):
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    _check(load().dgpe_set_psi(h, a.ctypes.data, a.size), h)


def dgpe_get_psi(h, shape):
    out = np.empty(shape, dtype=np.complex128)
    _check(load().dgpe_get_psi(h, out.ctypes.data, out.size), h)
    return out


def dgpe_set_psi_device(h, ptr: int, n_sites: int, fp64: bool):
    _check(load().dgpe_set_psi_device(h, C.c_void_p(ptr), n_sites, 1 if fp64 else 0), h)


def dgpe_get_psi_device(h, ptr: int, n_sites: int, fp64: bool):
    _check(load().dgpe_get_psi_device(h, C.c_void_p(ptr), n_sites, 1 if fp64 else 0), h)


def dgpe_step(h, n: int = 1):
    _check(load().dgpe_step(h, int(n)), h)


def dgpe_observables(h):
    o = dgpe_obs()
    _check(load().dgpe_observables(h, C.byref(o)), h)
    return {
        "norm": o.norm, "mu": o.mu, "energy": o.energy, "rms": (o.rms[0], o.rms[1], o.rms[2]),
        "rms_r": o.rms_r, "t": o.t, "kin": o.kin, "pot": o.pot, "contact": o.contact,
        "dipolar": o.dipolar,
    }


def dgpe_dipolar_potential(h, shape):
    out = np.empty(shape, dtype=np.float64)
    _check(load().dgpe_dipolar_potential(h, out.ctypes.data, out.size), h)
    return out


def dgpe_set_g(h, g: float):
    _check(load().dgpe_set_g(h, float(g)), h)


def dgpe_set_mode(h, imag: bool):
    _check(load().dgpe_set_mode(h, DGPE_IMAG if imag else DGPE_REAL), h)


def dgpe_set_trap_modulation(h, c):
    arr = (C.c_double * max(1, len(c)))(*[float(v) for v in c])
    _check(load().dgpe_set_trap_modulation(h, arr, len(c)), h)


def dgpe_set_time(h, step: int):
    _check(load().dgpe_set_time(h, int(step)), h)


def dgpe_get_time(h):
    v = C.c_longlong()
    _check(load().dgpe_get_time(h, C.byref(v)), h)
    return v.value


def dgpe_sync(h):
    _check(load().dgpe_sync(h), h)


def dgpe_launches_per_step(h):
    return load().dgpe_launches_per_step(h)


def dgpe_kernel_launches(h):
    return load().dgpe_kernel_launches(h)


def dgpe_profile_steps(h, n):
    """[(pass name, mean ms per launch, algorithmic bytes per launch,
    floating-point operations per launch)]."""
    buf = (C.c_double * 16)()
    rc = load().dgpe_profile_steps(h, int(n), buf, 16)
    if rc < 0:
        _check(rc, h)
    lib = load()
    return [(lib.dgpe_pass_name(h, i).decode(), buf[i], lib.dgpe_pass_bytes(h, i), lib.dgpe_pass_flops(h, i))
            for i in range(rc)]


def dgpe_dipolar_potential_noalloc(psi_ptr: int, phi_ptr: int, fp64: bool, dim: int, n, h,
                                   kernel=None, qd=0.5, stream: int = 0):
    """Phi_d of |psi|^2 from device buffers, with no device allocation (the
    scratch is a static device array inside libdgpe.so; see include/dgpe.h)."""
    if kernel is None:
        kernel = DGPE_KERNEL_DIPOLAR_3D if dim == 3 else DGPE_KERNEL_QUASI2D_XY
    nn = (C.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    hh = (C.c_double * 3)(*(list(h) + [1.0] * (3 - len(h))))
    rc = load().dgpe_dipolar_potential_noalloc(C.c_void_p(psi_ptr), C.c_void_p(phi_ptr),
                                               1 if fp64 else 0, dim, nn, hh, kernel, float(qd),
                                               C.c_void_p(stream))
    if rc != DGPE_OK:
        raise DgpeError(rc, load().dgpe_noalloc_last_error().decode())


class Solver:
    """One condensate on the GPU: create, set/get psi, step, observe."""

    def __init__(self, dim, n, h, nu, g=0.0, gdd=0.0, dt=1e-3, imag=False, fp64=True,
                 kernel=None, qd=0.5, graph=True, stream: int = 0, cn=None, split="lie",
                 real_psi=False, flags=0):
        self.dim = dim
        self.n = tuple(n)
        self.shape = (n[2], n[1], n[0]) if dim == 3 else (n[1], n[0])
        self.params = make_params(dim, n, h, nu, g, gdd, dt, imag, fp64, kernel, qd, graph, cn,
                                  split=split, real_psi=real_psi, flags=flags)
        self.h = dgpe_create(self.params, stream)

    def close(self):
        if self.h:
            dgpe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_psi(self, psi):
        dgpe_set_psi(self.h, psi)

    def get_psi(self):
        return dgpe_get_psi(self.h, self.shape)

    def step(self, n=1):
        dgpe_step(self.h, n)

    def observables(self):
        return dgpe_observables(self.h)

    def dipolar_potential(self):
        return dgpe_dipolar_potential(self.h, self.shape)

    def set_g(self, g):
        dgpe_set_g(self.h, g)

    def set_mode(self, imag):
        dgpe_set_mode(self.h, imag)

    def set_trap_modulation(self, c):
        dgpe_set_trap_modulation(self.h, c)

    def set_time(self, step):
        dgpe_set_time(self.h, step)

    def time(self):
        return dgpe_get_time(self.h)

    def sync(self):
        dgpe_sync(self.h)


# ------------------------------------------------------------- reverse mode
def _bind_adjoint():
    lib = load()
    if not getattr(lib, "_adj_bound", False):
        lib.dgpe_step_adjoint.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong,
                                          C.POINTER(C.c_double), C.POINTER(C.c_double)]
        lib.dgpe_fidelity_gradient.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                               C.POINTER(C.c_double), C.POINTER(C.c_double),
                                               C.POINTER(C.c_double)]
        lib._adj_bound = True
    return lib


def dgpe_step_adjoint(h, psi_in_ptr: int, G_ptr: int, step: int, M: int = 0):
    """Pull G back through one real-time step (device buffers); returns the
    step's (dL/dg, [dL/dc_m]) contributions."""
    lib = _bind_adjoint()
    dg = C.c_double(0.0)
    dc = (C.c_double * 16)()
    _check(lib.dgpe_step_adjoint(h, C.c_void_p(psi_in_ptr), C.c_void_p(G_ptr), int(step),
                                 C.byref(dg), dc), h)
    return dg.value, [dc[i] for i in range(M)]


def dgpe_fidelity_gradient(h, psi0, target, nsteps: int, every: int, M: int = 0):
    """(F, dF/dg, [dF/dc_m]) for F = |<target|psi(T)>|^2 after nsteps steps."""
    lib = _bind_adjoint()
    a = np.ascontiguousarray(psi0, dtype=np.complex128)
    b = np.ascontiguousarray(target, dtype=np.complex128)
    F = C.c_double(0.0)
    dg = C.c_double(0.0)
    dc = (C.c_double * 16)()
    _check(lib.dgpe_fidelity_gradient(h, a.ctypes.data, b.ctypes.data, int(nsteps), int(every),
                                      C.byref(F), C.byref(dg), dc), h)
    return F.value, dg.value, [dc[i] for i in range(M)]


# ------------------------------------------------------------- batched form
class Batch:
    """Many independent 2D XY problems (FP32-bulk) stepped by one graph launch.

    problems: list of dicts with keys n (nx, ny), h, nu, g, gdd, dt, imag, qd.
    classes: step with per-size-class batched kernels in one graph (the
    comparison form) instead of the persistent work-list kernel."""

    def __init__(self, problems, stream: int = 0, classes: bool = False):
        lib = load()
        if not getattr(lib, "_batch_bound", False):
            lib.dgpe_batch_create.argtypes = [C.POINTER(dgpe_params), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
            lib.dgpe_batch_destroy.argtypes = [C.c_void_p]
            lib.dgpe_batch_destroy.restype = None
            lib.dgpe_batch_set_psi.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]
            lib.dgpe_batch_get_psi.argtypes = [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]
            lib.dgpe_batch_step.argtypes = [C.c_void_p, C.c_int]
            lib.dgpe_batch_observables.argtypes = [C.c_void_p, C.c_int, C.POINTER(dgpe_obs)]
            lib.dgpe_batch_info.argtypes = [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                            C.POINTER(C.c_double)]
            lib.dgpe_batch_launches_per_step.argtypes = [C.c_void_p]
            lib.dgpe_batch_last_error.argtypes = [C.c_void_p]
            lib.dgpe_batch_last_error.restype = C.c_char_p
            lib.dgpe_batch_sync.argtypes = [C.c_void_p]
            lib.dgpe_batch_hold_problem.argtypes = [C.c_void_p, C.c_int]
            lib.dgpe_batch_set_wait_limit.argtypes = [C.c_void_p, C.c_longlong]
            lib._batch_bound = True
        self.lib = lib
        arr = (dgpe_params * len(problems))()
        self.shapes = []
        for i, q in enumerate(problems):
            arr[i] = make_params(2, q["n"], q["h"], q["nu"], q["g"], q["gdd"], q["dt"], q["imag"], False,
                                 DGPE_KERNEL_QUASI2D_XY, q.get("qd", 0.5), split=q.get("split", "lie"),
                                 real_psi=q.get("real_psi", False),
                                 flags=DGPE_FLAG_BATCH_CLASSES if classes else 0)
            self.shapes.append((q["n"][1], q["n"][0]))
        self.h = C.c_void_p()
        rc = lib.dgpe_batch_create(arr, len(problems), C.c_void_p(stream), C.byref(self.h))
        if rc:
            raise DgpeError(rc, lib.dgpe_batch_last_error(None).decode())

    def _chk(self, rc):
        if rc:
            raise DgpeError(rc, self.lib.dgpe_batch_last_error(self.h).decode())

    def set_psi(self, i, psi):
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        self._chk(self.lib.dgpe_batch_set_psi(self.h, i, a.ctypes.data, a.size))

    def get_psi(self, i):
        out = np.empty(self.shapes[i], dtype=np.complex128)
        self._chk(self.lib.dgpe_batch_get_psi(self.h, i, out.ctypes.data, out.size))
        return out

    def step(self, n=1):
        self._chk(self.lib.dgpe_batch_step(self.h, int(n)))

    def sync(self):
        self._chk(self.lib.dgpe_batch_sync(self.h))

    def hold_problem(self, i):
        """Test hook: problem i's tiles never complete (-1 releases)."""
        self._chk(self.lib.dgpe_batch_hold_problem(self.h, int(i)))

    def set_wait_limit(self, polls):
        self._chk(self.lib.dgpe_batch_set_wait_limit(self.h, int(polls)))

    def observables(self, i):
        o = dgpe_obs()
        self._chk(self.lib.dgpe_batch_observables(self.h, i, C.byref(o)))
        return {"norm": o.norm, "mu": o.mu, "energy": o.energy, "rms": (o.rms[0], o.rms[1], o.rms[2])}

    def info(self):
        c, s, b = C.c_int(), C.c_longlong(), C.c_double()
        self._chk(self.lib.dgpe_batch_info(self.h, C.byref(c), C.byref(s), C.byref(b)))
        return {"classes": c.value, "sites": s.value, "bytes_per_step": b.value,
                "launches_per_step": self.lib.dgpe_batch_launches_per_step(self.h)}

    def close(self):
        if self.h:
            self.lib.dgpe_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
