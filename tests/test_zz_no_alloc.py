"""The no-allocation dipolar-potential entry point against dgpe_dipolar_potential
and against the FP64 oracle.

dgpe_dipolar_potential_noalloc serves callers that may not allocate device
memory while they run (work recorded into a host framework's stream capture,
fixed memory budgets, real-time loops): its scratch is a static device array.
This file is collected last on purpose.  It calls the entry point through the
C ABI twice in a row with different states (the second call reuses the scratch
the first one left behind) and compares each result with the allocating
solver's Phi_d and with the oracle's, within the tolerances of the other
parity tests.  The cases include the limits the 4 MiB scratch is carved for:
the widest x-line (512 x 512 in 2D), exactly 262144 sites in 3D (64^3) and the
largest spectrum in rows (32 x 32 x 256)."""
import numpy as np
import pytest

import oracle
from paper_1601_04640_gb300 import build as gbuild
from paper_1601_04640_gb300 import dgpe, synth

pytestmark = pytest.mark.gpu

CASES = [
    (3, (32, 32, 64), (0.25, 0.25, 0.2), (1.0, 1.2, 2.0)),
    (2, (64, 128), (0.2, 0.15), (1.0, 1.5)),
    (2, (512, 512), (0.05, 0.05), (1.0, 1.2)),
    (3, (64, 64, 64), (0.2, 0.2, 0.2), (1.0, 1.0, 0.5)),
    (3, (32, 32, 256), (0.3, 0.3, 0.06), (1.0, 1.1, 0.7)),
]


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_noalloc_matches_solver_and_oracle(fp64, case):
    torch = pytest.importorskip("torch")
    gbuild.build()
    dim, n, h, nu = CASES[case]
    shape = tuple(reversed(n))
    tol_solver = 1e-12 if fp64 else 2e-6
    tol_oracle = 1e-12 if fp64 else 1e-5
    ctype = torch.complex128 if fp64 else torch.complex64
    rtype = torch.float64 if fp64 else torch.float32
    op = oracle.Params(dim=dim, n=n, h=h, nu=nu, kernel="dipolar3d" if dim == 3 else "quasi2d", qd=0.5)
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
        # the oracle sees the state the GPU form holds (FP32: psi rounded once)
        psi_in = psi_dev.cpu().numpy().astype(np.complex128)
        orc = oracle.dipolar_potential(op, np.abs(psi_in) ** 2)
        eo = np.max(np.abs(out - orc)) / np.max(np.abs(orc))
        print("call", call, "rel max err vs solver", err, "vs oracle", eo)
        assert err < tol_solver
        assert eo < tol_oracle


def test_noalloc_rejects_oversize_grid_and_xz():
    torch = pytest.importorskip("torch")
    gbuild.build()
    psi = torch.zeros((64, 128, 128), dtype=torch.complex128, device="cuda")
    phi = torch.zeros((64, 128, 128), dtype=torch.float64, device="cuda")
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.dgpe_dipolar_potential_noalloc(psi.data_ptr(), phi.data_ptr(), True, 3, (128, 128, 64),
                                            (0.1, 0.1, 0.1))
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    assert "262144" in str(e.value)
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.dgpe_dipolar_potential_noalloc(psi.data_ptr(), phi.data_ptr(), True, 2, (64, 64),
                                            (0.1, 0.1), kernel=dgpe.DGPE_KERNEL_QUASI2D_XZ)
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    assert "XZ" in str(e.value)
