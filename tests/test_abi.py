"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/dgpe.h declares; the oracle library is separate from it."""
import ctypes
import os
import re

import pytest

from paper_1601_04640_gb300 import build as gbuild
from paper_1601_04640_gb300 import dgpe

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header="dgpe.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    return set(re.findall(r"^\s*(?:const\s+)?(?:\w+\s+)*?\w+\s*\*?\s*(dgpe_\w+)\s*\(", src, re.M))


def test_every_header_is_checked():
    assert sorted(f for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")) == [
        "dgpe.h", "dgpe_plain.h"]


def test_comparison_library_exports(lib):
    plain = ctypes.CDLL(gbuild.PLAIN_LIB)
    names = _declared("dgpe_plain.h")
    assert "dgpe_plain_step" in names
    for n in sorted(names):
        assert hasattr(plain, n), n


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return ctypes.CDLL(gbuild.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "dgpe_create" in names and "dgpe_step" in names and "dgpe_observables" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    assert set(dgpe.EXPORTS) <= names


def test_binding_loads(lib):
    assert dgpe.load() is not None


def test_struct_layouts_match_header():
    src = open(os.path.join(ROOT, "include", "dgpe.h")).read()
    body = re.search(r"typedef struct dgpe_params \{(.*?)\} dgpe_params;", src, re.S).group(1)
    fields = re.findall(r"^\s*\w[\w\s]*?\s(\w+)(?:\[\d\])?;", body, re.M)
    assert fields == [f[0] for f in dgpe.dgpe_params._fields_]
    body = re.search(r"typedef struct dgpe_obs \{(.*?)\} dgpe_obs;", src, re.S).group(1)
    fields = re.findall(r"^\s*double\s+(\w+)(?:\[\d\])?;", body, re.M)
    assert fields == [f[0] for f in dgpe.dgpe_obs._fields_]


def test_argument_errors_without_device(lib):
    """Host-side validation fails before any CUDA call."""
    p = dgpe.make_params(3, (32, 32, 32), (0.25,) * 3, (1, 1, 2), dt=-1.0)
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.dgpe_create(p)
    assert e.value.code == dgpe.DGPE_EINVAL
    p = dgpe.make_params(3, (33, 32, 32), (0.25,) * 3, (1, 1, 2))
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.dgpe_create(p)
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    # the quasi-2D kernels must match the plane; an unknown plane is an error
    for kernel, plane in ((dgpe.DGPE_KERNEL_QUASI2D_XY, dgpe.DGPE_PLANE_XZ),
                          (dgpe.DGPE_KERNEL_QUASI2D_XZ, dgpe.DGPE_PLANE_XY), (dgpe.DGPE_KERNEL_NONE, 7)):
        p = dgpe.make_params(2, (32, 32), (0.25,) * 2, (1, 1), kernel=kernel)
        p.plane = plane
        with pytest.raises(dgpe.DgpeError) as e:
            dgpe.dgpe_create(p)
        assert e.value.code == dgpe.DGPE_EINVAL
    p = dgpe.make_params(2, (32, 32), (0.25,) * 2, (1, 1), kernel=dgpe.DGPE_KERNEL_DIPOLAR_3D)
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.dgpe_create(p)
    assert e.value.code == dgpe.DGPE_EINVAL
    # second-order splitting is a real-time option
    p = dgpe.make_params(3, (32, 32, 32), (0.25,) * 3, (1, 1, 2), imag=True, split="strang")
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.dgpe_create(p)
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    # a real state is an imaginary-time option on the chunk-parallel CN solve
    for kw in (dict(imag=False), dict(imag=True, cn="serial")):
        p = dgpe.make_params(3, (32, 32, 32), (0.25,) * 3, (1, 1, 2), real_psi=True, **kw)
        with pytest.raises(dgpe.DgpeError) as e:
            dgpe.dgpe_create(p)
        assert e.value.code == dgpe.DGPE_EUNSUPPORTED


def test_product_path_does_not_reference_the_oracle():
    pkg = os.path.join(ROOT, "paper_1601_04640_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "dgpe_oracle" not in txt, f
