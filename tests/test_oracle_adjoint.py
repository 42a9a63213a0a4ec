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


# ---- dot-product tests: the reverse step against tangents written from the
# forward step's own definition, exact to rounding

def _rand(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_cn_substep_adjoint_dot_product():
    """<C_a u, v> = <u, C_a^dagger v> on every axis; in real time C^dagger = C^{-1}."""
    p = oracle.Params(dim=3, n=(10, 12, 14), h=(0.3, 0.35, 0.4), nu=(1, 1, 1), dt=0.03,
                      imag=False, kernel="none")
    u, v = _rand(p.shape(), 1), _rand(p.shape(), 2)
    for a in range(3):
        lhs = np.vdot(oracle.cn_axis(p, u, a), v)
        rhs = np.vdot(u, oracle.cn_axis_adjoint(p, v, a))
        assert abs(lhs - rhs) < 1e-13 * abs(lhs)
        back = oracle.cn_axis_adjoint(p, oracle.cn_axis(p, u, a), a)
        assert np.max(np.abs(back - u)) < 1e-13 * np.max(np.abs(u))


def _tangent(p, psi, d, step, dg=0.0, dc=None):
    """J d of one real-time step at psi: the exponential substep's tangent
    e^{-i theta} (d - i dtheta psi), dtheta = dt (g dn + g_dd K*dn + n dg +
    sum_m sin(m t) V0 dc_m), dn = 2 Re(conj(psi) d), then the (linear) CN
    substeps."""
    n = np.abs(psi) ** 2
    V0 = oracle.trap(p)
    t = step * p.dt
    th = p.dt * (oracle.trap_scale(p, t) * V0 + p.g * n + p.gdd * oracle.dipolar_potential(p, n))
    dn = 2.0 * np.real(np.conj(psi) * d)
    dth = p.dt * (p.g * dn + p.gdd * oracle.dipolar_potential(p, dn) + n * dg)
    if dc is not None:
        dth = dth + p.dt * V0 * sum(c * np.sin((m + 1) * t) for m, c in enumerate(dc))
    out = np.exp(-1j * th) * (d - 1j * dth * psi)
    for a in range(p.dim):
        out = oracle.cn_axis(p, out, a)
    return out


def test_step_adjoint_dot_product_linear():
    """g = g_dd = 0: the step is complex-linear and its reverse is its adjoint."""
    p = oracle.Params(dim=2, n=(24, 20), h=(0.3, 0.35), nu=(1.0, 1.3), dt=0.02, imag=False,
                      kernel="quasi2d", cm=[0.3, -0.1])
    u, v = _rand(p.shape(), 3), _rand(p.shape(), 4)
    step = 5
    lhs = np.vdot(v, oracle.step(p, u, step, 1))
    G, _, _ = oracle.step_adjoint(p, u, v, step)
    rhs = np.vdot(G, u)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_step_adjoint_dot_product_nonlinear():
    """Re<v, J d> = Re<G, d> with G the reverse step of v (Wirtinger G = 2 dL/dpsi*
    for L = Re<v, psi'>), and dL/dg, dL/dc_m against the tangents in g and c_m."""
    cm = [0.2, -0.1, 0.05]
    p = oracle.Params(dim=3, n=(12, 10, 16), h=(0.4, 0.45, 0.35), nu=(1.0, 1.2, 0.8), g=40.0, gdd=15.0,
                      dt=0.02, imag=False, kernel="dipolar3d", cm=cm)
    psi = synth.gaussian_state(p.n, p.h, p.nu, 0.05, 17)
    v, d = _rand(p.shape(), 5), _rand(p.shape(), 6)
    step = 7
    G, dLg, dLc = oracle.step_adjoint(p, psi, v, step)
    lhs = np.real(np.vdot(v, _tangent(p, psi, d, step)))
    assert abs(lhs - np.real(np.vdot(G, d))) < 1e-12 * np.linalg.norm(v) * np.linalg.norm(d)
    tg = np.real(np.vdot(v, _tangent(p, psi, np.zeros_like(psi), step, dg=1.0)))
    assert abs(dLg - tg) < 1e-12 * abs(tg)
    for m in range(len(cm)):
        e = np.zeros(len(cm))
        e[m] = 1.0
        tc = np.real(np.vdot(v, _tangent(p, psi, np.zeros_like(psi), step, dc=e)))
        assert abs(dLc[m] - tc) < 1e-12 * max(abs(tc), 1e-30)
