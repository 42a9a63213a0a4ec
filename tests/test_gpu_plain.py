"""The cuFFT-based comparison step (libdgpe_plain.so, the paper's kernel +
cuFFT design) against the oracle: it is only timed, but it must compute the
same step."""
import numpy as np
import pytest

import oracle
from paper_1601_04640_gb300 import build as gbuild
from paper_1601_04640_gb300 import synth
from paper_1601_04640_gb300.plain import PlainSolver

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp64,tol", [(True, 1e-10), (False, 1e-5)])
@pytest.mark.parametrize("dim", [2, 3])
def test_plain_step_matches_oracle(fp64, tol, dim):
    gbuild.build()
    if dim == 3:
        n, h, nu = (32, 64, 32), (0.25, 0.2, 0.25), (1.0, 1.2, 2.0)
        kernel = "dipolar3d"
    else:
        n, h, nu = (64, 32), (0.2, 0.3), (1.0, 1.5)
        kernel = "quasi2d"
    op = oracle.Params(dim=dim, n=n, h=h, nu=nu, g=60, gdd=25, dt=1e-3, imag=False, kernel=kernel)
    psi0 = synth.gaussian_state(n, h, nu, 0.01, 77)
    ref = oracle.step(op, psi0, 0, 5)
    with PlainSolver(dim, n, h, nu, 60, 25, 1e-3, fp64) as s:
        s.set_psi(psi0)
        s.step(5)
        psi = s.get_psi()
    e = float(np.linalg.norm(psi - ref) / np.linalg.norm(ref))
    print("plain rel L2", e)
    assert e < tol
