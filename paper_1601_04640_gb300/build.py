"""Build the CUDA library libdgpe.so (sm_103a) in-tree.

nvcc compiles the translation units in parallel and links one shared library
next to this file.  Used by ``__graft_entry__.build()``; the Python binding
loads the result and fails loudly when it is missing.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdgpe.so")
PLAIN_LIB = os.path.join(HERE, "libdgpe_plain.so")
PLAIN_SRC = os.path.join(CSRC, "plain", "dgpe_plain.cu")
UNITS = ["dgpe_api.cu", "dgpe_f64.cu", "dgpe_f32.cu", "dgpe_noalloc.cu", "dgpe_batch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", CSRC, "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(lib, deps):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in deps)


def build_plain(force: bool = False) -> str:
    """The cuFFT-based comparison step (timed beside the fused path only)."""
    deps = [PLAIN_SRC, os.path.join(ROOT, "include", "dgpe_plain.h"), os.path.join(ROOT, "include", "dgpe.h")]
    if not force and not _stale(PLAIN_LIB, deps):
        return PLAIN_LIB
    tmp = PLAIN_LIB + ".tmp"
    cmd = [_nvcc(), *ARCH, *FLAGS, "-shared", "-cudart", "static", PLAIN_SRC, "-o", tmp, "-lcufft"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for the comparison step:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, PLAIN_LIB)
    return PLAIN_LIB


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    srcs = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh"))]
    srcs.append(os.path.join(ROOT, "include", "dgpe.h"))
    if not force and not _stale(LIB, srcs):
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()

    def compile_unit(u):
        obj = os.path.join(OUT, u.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, u), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (u, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(UNITS) + 1) as ex:
        plain = ex.submit(build_plain, force)
        objs = list(ex.map(compile_unit, UNITS))
        plain.result()
    tmp = LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv,
                extra=["-Xptxas", "-v"] if "-v" in sys.argv else []))
