"""Pins for the oracle's reverse-mode step: central finite differences of the
fidelity |<psi_t|psi(T)>|^2 with respect to g, the trap coefficients c_m and
the initial state."""
import numpy as np

import oracle
from paper_1601_04640_gb300 import synth


def _setup():
    n, h = (10, 10, 12), (0.5, 0.5, 0.5)
    cm = list(synth.trap_modulation(160104640, 4, 0.05))
    p = oracle.Params(dim=3, n=n, h=h, nu=(1, 1, 0.5), g=40.0, gdd=15.0, dt=2e-2,
                      imag=False, kernel="dipolar3d", cm=cm)
    psi0 = synth.gaussian_state(n, h, (1, 1, 0.5), 0.02, 11)
    target = synth.gaussian_state(n, h, (1.1, 0.9, 0.5), 0.02, 12)
    return p, psi0, target, 12


def _loss(p, psi0, target, K):
    w = p.h[0] * p.h[1] * p.h[2]
    psi = oracle.step(p, psi0, 0, K)
    c = w * np.vdot(target, psi)
    return abs(c) ** 2, psi, c


def _adjoint(p, psi0, target, K):
    w = p.h[0] * p.h[1] * p.h[2]
    states = [psi0]
    for s in range(K):
        states.append(oracle.step(p, states[-1], s, 1))
    c = w * np.vdot(target, states[-1])
    G = 2 * w * c * target            # 2 dL/dpsi*
    dg, dc = 0.0, np.zeros(len(p.cm))
    for s in reversed(range(K)):
        G, g1, c1 = oracle.step_adjoint(p, states[s], G, s)
        dg += g1
        dc += c1
    return G, dg, dc


def test_adjoint_vs_finite_differences():
    p, psi0, target, K = _setup()
    G, dg, dc = _adjoint(p, psi0, target, K)
    eps = 1e-5
    import copy
    pp, pm = copy.deepcopy(p), copy.deepcopy(p)
    pp.g += eps
    pm.g -= eps
    fd = (_loss(pp, psi0, target, K)[0] - _loss(pm, psi0, target, K)[0]) / (2 * eps)
    assert abs(dg - fd) < 1e-6 * abs(fd)
    for m in range(len(p.cm)):
        pp, pm = copy.deepcopy(p), copy.deepcopy(p)
        pp.cm = list(p.cm); pm.cm = list(p.cm)
        pp.cm[m] += eps
        pm.cm[m] -= eps
        fd = (_loss(pp, psi0, target, K)[0] - _loss(pm, psi0, target, K)[0]) / (2 * eps)
        assert abs(dc[m] - fd) < 1e-6 * abs(fd) + 1e-12
    rng = np.random.default_rng(3)
    d = rng.standard_normal(psi0.shape) + 1j * rng.standard_normal(psi0.shape)
    fd = (_loss(p, psi0 + eps * d, target, K)[0] - _loss(p, psi0 - eps * d, target, K)[0]) / (2 * eps)
    assert abs(np.real(np.vdot(G, d)) - fd) < 1e-6 * abs(fd)
