"""ctypes binding of the comparison step (include/dgpe_plain.h,
libdgpe_plain.so): the paper's kernel + cuFFT design, timed beside the fused
path.  Argument marshalling only."""
import ctypes as C
import os

import numpy as np

from .dgpe import DgpeError, dgpe_params, make_params

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgpe_plain.so")
_lib = None


def load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdgpe_plain.so not built: run paper_1601_04640_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        lib.dgpe_plain_create.argtypes = [C.POINTER(dgpe_params), C.c_void_p, C.POINTER(C.c_void_p)]
        lib.dgpe_plain_destroy.argtypes = [C.c_void_p]
        lib.dgpe_plain_destroy.restype = None
        lib.dgpe_plain_set_psi.argtypes = [C.c_void_p, C.c_void_p]
        lib.dgpe_plain_get_psi.argtypes = [C.c_void_p, C.c_void_p]
        lib.dgpe_plain_step.argtypes = [C.c_void_p, C.c_int]
        lib.dgpe_plain_last_error.restype = C.c_char_p
        _lib = lib
    return _lib


def _check(rc):
    if rc != 0:
        raise DgpeError(rc, load().dgpe_plain_last_error().decode())


class PlainSolver:
    def __init__(self, dim, n, h, nu, g=0.0, gdd=0.0, dt=1e-3, fp64=True, kernel=None, qd=0.5,
                 stream: int = 0):
        self.shape = (n[2], n[1], n[0]) if dim == 3 else (n[1], n[0])
        self.params = make_params(dim, n, h, nu, g, gdd, dt, False, fp64, kernel, qd)
        self.h = C.c_void_p()
        _check(load().dgpe_plain_create(C.byref(self.params), C.c_void_p(stream), C.byref(self.h)))

    def set_psi(self, psi):
        a = np.ascontiguousarray(psi, dtype=np.complex128)
        _check(load().dgpe_plain_set_psi(self.h, a.ctypes.data))

    def get_psi(self):
        out = np.empty(self.shape, dtype=np.complex128)
        _check(load().dgpe_plain_get_psi(self.h, out.ctypes.data))
        return out

    def step(self, n=1):
        _check(load().dgpe_plain_step(self.h, int(n)))

    def close(self):
        if self.h:
            load().dgpe_plain_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
