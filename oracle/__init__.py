"""FP64 CPU oracle for the split-step Crank-Nicolson dipolar GP step.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA path (``paper_1601_04640_gb300``) and never
imports it.  The arithmetic lives in ``dgpe_oracle.c``; this module only
marshals numpy arrays through ctypes.

Arrays: complex128 psi of shape (nz, ny, nx) in 3D or (ny, nx) in 2D,
x fastest.
"""
import ctypes as C
import os
from dataclasses import dataclass, field
from typing import Sequence

import numpy as np

from . import build as _build

KERNELS = {"none": 0, "dipolar3d": 1, "quasi2d": 2, "quasi2d_xz": 3}
MAXM = 16


class _Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("n", C.c_int * 3), ("h", C.c_double * 3),
        ("nu", C.c_double * 3), ("g", C.c_double), ("gdd", C.c_double),
        ("dt", C.c_double), ("imag", C.c_int), ("kernel", C.c_int),
        ("qd", C.c_double), ("M", C.c_int), ("cm", C.c_double * MAXM),
    ]


class _Obs(C.Structure):
    _fields_ = [
        ("norm", C.c_double), ("mu", C.c_double), ("energy", C.c_double),
        ("rms", C.c_double * 3), ("rms_r", C.c_double), ("kin", C.c_double),
        ("pot", C.c_double), ("contact", C.c_double), ("dipolar", C.c_double),
    ]


@dataclass
class Params:
    """Physical and numerical parameters (dimensionless trap units)."""
    dim: int
    n: Sequence[int]            # (nx, ny, nz); nz ignored in 2D
    h: Sequence[float]
    nu: Sequence[float]
    g: float = 0.0
    gdd: float = 0.0
    dt: float = 1e-3
    imag: bool = False
    kernel: str = "dipolar3d"
    qd: float = 0.5
    cm: Sequence[float] = field(default_factory=list)

    def shape(self):
        nx, ny = self.n[0], self.n[1]
        return (self.n[2], ny, nx) if self.dim == 3 else (ny, nx)

    def _c(self):
        p = _Params()
        p.dim = self.dim
        n = list(self.n) + [1] * (3 - len(self.n))
        h = list(self.h) + [1.0] * (3 - len(self.h))
        nu = list(self.nu) + [0.0] * (3 - len(self.nu))
        if self.dim == 2:
            n[2] = 1
        for i in range(3):
            p.n[i] = int(n[i]); p.h[i] = float(h[i]); p.nu[i] = float(nu[i])
        p.g = float(self.g); p.gdd = float(self.gdd); p.dt = float(self.dt)
        p.imag = 1 if self.imag else 0
        p.kernel = KERNELS[self.kernel]
        p.qd = float(self.qd)
        if len(self.cm) > MAXM:
            raise ValueError("at most %d trap-modulation coefficients" % MAXM)
        p.M = len(self.cm)
        for i, c in enumerate(self.cm):
            p.cm[i] = float(c)
        return p


_lib = None


def load():
    global _lib
    if _lib is None:
        lib = C.CDLL(_build.build())
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        cp = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
        P = C.POINTER(_Params)
        lib.or_fft.argtypes = [cp, C.c_int, C.c_int]
        lib.or_dft.argtypes = [cp, cp, C.c_int, C.c_int]
        lib.or_fftn.argtypes = [cp, C.POINTER(C.c_int), C.c_int, C.c_int]
        lib.or_kernel_3d.argtypes = [dp, C.POINTER(C.c_int), C.POINTER(C.c_double)]
        lib.or_kernel_q2d.argtypes = [dp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_double]
        lib.or_q2d_value.argtypes = [C.c_double, C.c_double]
        lib.or_q2d_value.restype = C.c_double
        lib.or_erfcx.argtypes = [C.c_double]
        lib.or_erfcx.restype = C.c_double
        lib.or_kernel_q2dxz.argtypes = [dp, C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_double]
        lib.or_q2dxz_value.argtypes = [C.c_double, C.c_double, C.c_double]
        lib.or_q2dxz_value.restype = C.c_double
        lib.or_dipolar_potential.argtypes = [P, dp, dp]
        lib.or_trap.argtypes = [P, dp]
        lib.or_trap_scale.argtypes = [P, C.c_double]
        lib.or_trap_scale.restype = C.c_double
        lib.or_nonlinear.argtypes = [P, cp, C.c_long]
        lib.or_nonlinear_frac.argtypes = [P, cp, C.c_double, C.c_double]
        lib.or_thomas.argtypes = [cp, cp, cp, cp, cp, C.c_int]
        lib.or_cn_axis.argtypes = [P, cp, C.c_int]
        lib.or_cn_axis_adjoint.argtypes = [P, cp, C.c_int]
        lib.or_normalize.argtypes = [P, cp]
        lib.or_step.argtypes = [P, cp, C.c_long]
        lib.or_run.argtypes = [P, cp, C.c_long, C.c_long]
        lib.or_step_strang.argtypes = [P, cp, C.c_long]
        lib.or_run_strang.argtypes = [P, cp, C.c_long, C.c_long]
        lib.or_observables.argtypes = [P, cp, C.c_long, C.POINTER(_Obs)]
        lib.or_step_adjoint.argtypes = [P, cp, cp, C.c_long, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double)]
        lib.or_threads.restype = C.c_int
        lib.or_set_threads.argtypes = [C.c_int]
        _lib = lib
    return _lib


def threads() -> int:
    return load().or_threads()


def set_threads(n: int) -> None:
    load().or_set_threads(int(n))


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128).copy()


def fft(x, sign=-1):
    x = _c128(x)
    if load().or_fft(x, x.size, sign):
        raise ValueError("bad length")
    return x


def dft(x, sign=-1):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    X = np.empty_like(x)
    load().or_dft(x, X, x.size, sign)
    return X


def fftn(a, sign=-1):
    a = _c128(a)
    dims = (C.c_int * a.ndim)(*a.shape)
    load().or_fftn(a, dims, a.ndim, sign)
    return a


def kernel_3d(n, h):
    U = np.empty((n[2], n[1], n[0]), dtype=np.float64)
    load().or_kernel_3d(U, (C.c_int * 3)(*n), (C.c_double * 3)(*h))
    return U


def kernel_q2d(n, h, d):
    U = np.empty((n[1], n[0]), dtype=np.float64)
    nn = list(n) + [1] * (3 - len(n))
    hh = list(h) + [1.0] * (3 - len(h))
    load().or_kernel_q2d(U, (C.c_int * 3)(*nn), (C.c_double * 3)(*hh), float(d))
    return U


def q2d_value(k, d):
    return load().or_q2d_value(float(k), float(d))


def erfcx(u):
    """exp(u^2) erfc(u), u >= 0, as the quasi-2D kernels evaluate it."""
    return load().or_erfcx(float(u))


def kernel_q2dxz(n, h, d):
    """Quasi-2D XZ kernel on the (nz, nx) grid: n = (nx, nz), h = (hx, hz)."""
    U = np.empty((n[1], n[0]), dtype=np.float64)
    nn = list(n) + [1] * (3 - len(n))
    hh = list(h) + [1.0] * (3 - len(h))
    load().or_kernel_q2dxz(U, (C.c_int * 3)(*nn), (C.c_double * 3)(*hh), float(d))
    return U


def q2dxz_value(kx, kz, d):
    return load().or_q2dxz_value(float(kx), float(kz), float(d))


def dipolar_potential(p: Params, dens):
    dens = np.ascontiguousarray(dens, dtype=np.float64)
    phi = np.empty_like(dens)
    if load().or_dipolar_potential(C.byref(p._c()), dens, phi):
        raise ValueError("kernel does not match dimension")
    return phi


def trap(p: Params):
    V = np.empty(p.shape(), dtype=np.float64)
    load().or_trap(C.byref(p._c()), V)
    return V


def trap_scale(p: Params, t: float) -> float:
    return load().or_trap_scale(C.byref(p._c()), float(t))


def nonlinear(p: Params, psi, step=0):
    psi = _c128(psi)
    if load().or_nonlinear(C.byref(p._c()), psi, int(step)):
        raise ValueError("nonlinear substep failed")
    return psi


def thomas(a, b, c, d):
    a, b, c, d = (_c128(v) for v in (a, b, c, d))
    x = np.empty_like(d)
    load().or_thomas(a, b, c, d, x, d.size)
    return x


def cn_axis(p: Params, psi, axis):
    psi = _c128(psi)
    load().or_cn_axis(C.byref(p._c()), psi, int(axis))
    return psi


def cn_axis_adjoint(p: Params, psi, axis):
    """C_a^dagger psi (the conjugate transpose of the CN substep along axis)."""
    psi = _c128(psi)
    load().or_cn_axis_adjoint(C.byref(p._c()), psi, int(axis))
    return psi


def normalize(p: Params, psi):
    psi = _c128(psi)
    load().or_normalize(C.byref(p._c()), psi)
    return psi


def nonlinear_frac(p: Params, psi, t, f):
    """Exponential substep over f dt with the trap at time t."""
    psi = _c128(psi)
    if load().or_nonlinear_frac(C.byref(p._c()), psi, float(t), float(f)):
        raise ValueError("nonlinear substep failed")
    return psi


SPLITS = ("lie", "strang")


def step(p: Params, psi, step0=0, nsteps=1, split="lie"):
    """Advance nsteps steps starting at step index step0; returns a new array.

    split "lie": the paper's first-order splitting (exponential, then CN along
    x, y, z); "strang": half exponential, CN, half exponential (real time)."""
    psi = _c128(psi)
    if psi.shape != p.shape():
        raise ValueError("psi shape %s != %s" % (psi.shape, p.shape()))
    if split not in SPLITS:
        raise ValueError("split must be one of %s" % (SPLITS,))
    run = load().or_run if split == "lie" else load().or_run_strang
    if run(C.byref(p._c()), psi, int(step0), int(nsteps)):
        raise ValueError("step failed")
    return psi


def observables(p: Params, psi, step=0):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    o = _Obs()
    if load().or_observables(C.byref(p._c()), psi, int(step), C.byref(o)):
        raise ValueError("observables failed")
    return {
        "norm": o.norm, "mu": o.mu, "energy": o.energy,
        "rms": (o.rms[0], o.rms[1], o.rms[2]), "rms_r": o.rms_r,
        "kin": o.kin, "pot": o.pot, "contact": o.contact, "dipolar": o.dipolar,
    }


def step_adjoint(p: Params, psi_in, G, step):
    """Pull G' (= 2 dL/dpsi'*) back through step `step` taken from psi_in.

    Returns (G, dL/dg contribution, dL/dc contributions)."""
    psi_in = np.ascontiguousarray(psi_in, dtype=np.complex128)
    G = _c128(G)
    dg = C.c_double(0.0)
    dc = (C.c_double * MAXM)()
    if load().or_step_adjoint(C.byref(p._c()), psi_in, G, int(step), C.byref(dg), dc):
        raise ValueError("adjoint is defined for real time only")
    return G, dg.value, np.array([dc[i] for i in range(len(p.cm))])
