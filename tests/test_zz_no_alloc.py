"""The no-allocation dipolar-potential entry point against dgpe_dipolar_potential.

dgpe_dipolar_potential_noalloc serves callers that may not allocate device
memory while they run (work recorded into a host framework's stream capture,
fixed memory budgets, real-time loops): its scratch is a static device array.
This file is collected last on purpose.  It calls the entry point through the
C ABI twice in a row with different states (the second call reuses the scratch
the first one left behind) and compares each result with the allocating
solver's Phi_d within the tolerances of the other parity tests."""
import numpy as np
import pytest

from paper_1601_04640_gb300 import build as gbuild
from paper_1601_04640_gb300 import dgpe, synth

pytestmark = pytest.mark.gpu

CASES = [
    (3, (32, 32, 64), (0.25, 0.25, 0.2), (1.0, 1.2, 2.0)),
    (2, (64, 128), (0.2, 0.15), (1.0, 1.5)),
]


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_noalloc_matches_solver(fp64, case):
    torch = pytest.importorskip("torch")
    gbuild.build()
    dim, n, h, nu = CASES[case]
    shape = tuple(reversed(n))
    tol = 1e-12 if fp64 else 2e-6
    ctype = torch.complex128 if fp64 else torch.complex64
    rtype = torch.float64 if fp64 else torch.float32
    for call, seed in enumerate((11, 12)):
        psi = synth.gaussian_state(n, h, [0.8 + 0.1 * seed % 3 for _ in nu], 0.05, seed)
        with dgpe.Solver(dim, n, h, nu, 10.0, 5.0, 1e-3, False, fp64) as s:
            s.set_psi(psi)
            ref = s.dipolar_potential()
        psi_dev = torch.from_numpy(psi).to("cuda").to(ctype).contiguous()
        phi_dev = torch.full(shape, float("nan"), dtype=rtype, device="cuda")
        stream = torch.cuda.current_stream().cuda_stream
        dgpe.dgpe_dipolar_potential_noalloc(psi_dev.data_ptr(), phi_dev.data_ptr(), fp64, dim, n, h,
                                            stream=stream)
        torch.cuda.synchronize()
        out = phi_dev.double().cpu().numpy()
        err = np.max(np.abs(out - ref)) / np.max(np.abs(ref))
        print("call", call, "rel max err", err)
        assert err < tol


def test_noalloc_rejects_oversize_grid():
    torch = pytest.importorskip("torch")
    gbuild.build()
    psi = torch.zeros((64, 128, 128), dtype=torch.complex128, device="cuda")
    phi = torch.zeros((64, 128, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.dgpe_dipolar_potential_noalloc(psi.data_ptr(), phi.data_ptr(), True, 3, (128, 128, 64),
                                            (0.1, 0.1, 0.1))
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    assert "262144" in str(e.value)
