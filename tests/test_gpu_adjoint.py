"""The GPU reverse-mode step against the oracle's adjoint and against central
finite differences of the GPU forward; the torch.autograd.Function wrapper."""
import copy

import numpy as np
import pytest

import oracle
from paper_1601_04640_gb300 import build as gbuild
from paper_1601_04640_gb300 import dgpe, synth

pytestmark = pytest.mark.gpu

N, H, NU = (32, 32, 32), (0.3, 0.3, 0.3), (1.0, 1.0, 0.5)
G0, GDD, DT = 80.0, 30.0, 5e-3


def _states():
    cm = list(synth.trap_modulation(160104640, 8, 0.05))
    psi0 = synth.gaussian_state(N, H, (1.0, 1.0, 0.5), 0.02, 21)
    target = synth.gaussian_state(N, H, (1.1, 0.9, 0.5), 0.02, 22)
    return cm, psi0, target


@pytest.mark.parametrize("cn", [None, "serial"])
def test_step_adjoint_matches_oracle(cn):
    torch = pytest.importorskip("torch")
    gbuild.build()
    cm, psi0, target = _states()
    op = oracle.Params(dim=3, n=N, h=H, nu=NU, g=G0, gdd=GDD, dt=DT, imag=False, kernel="dipolar3d", cm=cm)
    rng = np.random.default_rng(5)
    Gp = rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape)
    step = 7
    ref_G, ref_dg, ref_dc = oracle.step_adjoint(op, psi0, Gp, step)
    with dgpe.Solver(3, N, H, NU, G0, GDD, DT, False, True, cn=cn) as s:
        s.set_trap_modulation(cm)
        pin = torch.from_numpy(psi0).cuda()
        G = torch.from_numpy(Gp).cuda()
        dg, dc = dgpe.dgpe_step_adjoint(s.h, pin.data_ptr(), G.data_ptr(), step, len(cm))
        out = G.cpu().numpy()
    e = np.linalg.norm(out - ref_G) / np.linalg.norm(ref_G)
    print("adjoint G rel", e, "dg", dg, ref_dg)
    assert e < 1e-12
    assert abs(dg - ref_dg) <= 1e-10 * abs(ref_dg)
    assert np.max(np.abs(np.array(dc) - ref_dc)) <= 1e-10 * np.max(np.abs(ref_dc))


def _fid(s, psi0, target, K):
    s.set_psi(psi0)
    s.step(K)
    psi = s.get_psi()
    c = np.prod(H) * np.vdot(target, psi)
    return abs(c) ** 2


@pytest.mark.parametrize("every", [4, 32])
def test_fidelity_gradient_vs_oracle_and_fd(every):
    gbuild.build()
    cm, psi0, target = _states()
    K = 24
    op = oracle.Params(dim=3, n=N, h=H, nu=NU, g=G0, gdd=GDD, dt=DT, imag=False, kernel="dipolar3d", cm=cm)
    # oracle adjoint over the same run
    w = np.prod(H)
    states = [psi0]
    for k in range(K):
        states.append(oracle.step(op, states[-1], k, 1))
    c = w * np.vdot(target, states[-1])
    Gr = 2 * w * c * target
    rdg, rdc = 0.0, np.zeros(len(cm))
    for k in reversed(range(K)):
        Gr, a, b = oracle.step_adjoint(op, states[k], Gr, k)
        rdg += a
        rdc += b
    with dgpe.Solver(3, N, H, NU, G0, GDD, DT, False, True) as s:
        s.set_trap_modulation(cm)
        F, dg, dc = dgpe.dgpe_fidelity_gradient(s.h, psi0, target, K, every, len(cm))
        assert abs(F - abs(c) ** 2) <= 1e-12 * abs(c) ** 2
        assert abs(dg - rdg) <= 1e-10 * abs(rdg)
        assert np.max(np.abs(np.array(dc) - rdc)) <= 1e-10 * np.max(np.abs(rdc))
        # central finite differences of the GPU forward (FP64 form)
        eps = 1e-4
        s.set_g(G0 + eps); fp = _fid(s, psi0, target, K)
        s.set_g(G0 - eps); fm = _fid(s, psi0, target, K)
        s.set_g(G0)
        fd = (fp - fm) / (2 * eps)
        print("dF/dg adjoint", dg, "fd", fd)
        assert abs(dg - fd) <= 1e-6 * abs(fd)
        for m in (0, 3, 7):
            cp = list(cm); cp[m] += eps
            cq = list(cm); cq[m] -= eps
            s.set_trap_modulation(cp); fp = _fid(s, psi0, target, K)
            s.set_trap_modulation(cq); fm = _fid(s, psi0, target, K)
            fd = (fp - fm) / (2 * eps)
            assert abs(dc[m] - fd) <= 1e-6 * abs(fd) + 1e-12


def test_fp32_bulk_gradient_close_to_fp64():
    gbuild.build()
    cm, psi0, target = _states()
    out = []
    for fp64 in (True, False):
        with dgpe.Solver(3, N, H, NU, G0, GDD, DT, False, fp64) as s:
            s.set_trap_modulation(cm)
            out.append(dgpe.dgpe_fidelity_gradient(s.h, psi0, target, 64, 8, len(cm)))
    (F64, g64, c64), (F32, g32, c32) = out
    print("F", F64, F32, "dg", g64, g32)
    assert abs(F32 - F64) <= 1e-5 * abs(F64)
    assert abs(g32 - g64) <= 1e-3 * abs(g64)
    assert np.max(np.abs(np.array(c32) - c64)) <= 1e-3 * np.max(np.abs(c64))


def test_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_1601_04640_gb300.autograd import fidelity
    gbuild.build()
    cm, psi0, target = _states()
    with dgpe.Solver(3, N, H, NU, G0, GDD, DT, False, True) as s:
        g = torch.tensor(G0, dtype=torch.float64, requires_grad=True)
        c = torch.tensor(cm, dtype=torch.float64, requires_grad=True)
        F = fidelity(g, c, s, psi0, target, 16, 4)
        (2.0 * F).backward()
        _, dg, dc = dgpe.dgpe_fidelity_gradient(s.h, psi0, target, 16, 4, len(cm))
    assert abs(g.grad.item() - 2.0 * dg) <= 1e-12 * abs(dg)
    assert np.allclose(c.grad.numpy(), 2.0 * np.array(dc), rtol=1e-12, atol=0)


def test_adjoint_config_full_length_fd():
    """The adjoint workload at its own size and length: 128^3, h = 0.15, cigar
    trap, g = 200, g_dd = 60, dt = 1e-3, V(t) = V0 (1 + sum_m c_m sin(m t)) with
    the seeded c_1..c_8, 1000 steps, checkpoints every 32 steps.  FP64 form:
    the reverse sweep's dF/dg and dF/dc_m against central finite differences
    of the GPU forward at the benchmark spec's bound (1e-6 relative); the FP32-bulk
    gradient against the FP64 one."""
    gbuild.build()
    n, h, nu = (128, 128, 128), (0.15,) * 3, (1.0, 1.0, 0.5)
    g0, gdd, dt, K, every = 200.0, 60.0, 1e-3, 1000, 32
    cm = list(synth.trap_modulation(160104640, 8, 0.05))
    psi0 = synth.gaussian_state(n, h, (1.0, 1.0, 0.5), 0.01, 1)
    target = synth.gaussian_state(n, h, (1.1, 0.9, 0.5), 0.01, 2)
    w = np.prod(h)

    def fid(s):
        s.set_psi(psi0)
        s.step(K)
        return abs(w * np.vdot(target, s.get_psi())) ** 2

    with dgpe.Solver(3, n, h, nu, g0, gdd, dt, False, True) as s:
        s.set_trap_modulation(cm)
        F, dg, dc = dgpe.dgpe_fidelity_gradient(s.h, psi0, target, K, every, len(cm))
        s.set_trap_modulation(cm)
        assert abs(fid(s) - F) <= 1e-12 * F
        eps = 1e-3
        s.set_g(g0 + eps); fp = fid(s)
        s.set_g(g0 - eps); fm = fid(s)
        s.set_g(g0)
        fd = (fp - fm) / (2 * eps)
        print("F", F, "dF/dg adjoint", dg, "fd", fd, "rel", abs(dg - fd) / abs(fd))
        assert abs(dg - fd) <= 1e-6 * abs(fd)
        eps = 1e-4
        for m in (0, 1, 4, 7):
            cp = list(cm); cp[m] += eps
            cq = list(cm); cq[m] -= eps
            s.set_trap_modulation(cp); fp = fid(s)
            s.set_trap_modulation(cq); fm = fid(s)
            fd = (fp - fm) / (2 * eps)
            print("dF/dc_%d adjoint" % (m + 1), dc[m], "fd", fd, "rel", abs(dc[m] - fd) / abs(fd))
            assert abs(dc[m] - fd) <= 1e-6 * abs(fd) + 1e-12 * F
    with dgpe.Solver(3, n, h, nu, g0, gdd, dt, False, False) as s:
        s.set_trap_modulation(cm)
        F32, g32, c32 = dgpe.dgpe_fidelity_gradient(s.h, psi0, target, K, every, len(cm))
    print("FP32 bulk: F", F32, "dF/dg", g32)
    assert abs(F32 - F) <= 1e-5 * F
    assert abs(g32 - dg) <= 1e-3 * abs(dg)
    assert np.max(np.abs(np.array(c32) - dc)) <= 1e-3 * np.max(np.abs(dc))
