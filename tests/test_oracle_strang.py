"""Pins for the oracle's second-order (Strang) splitting,
psi <- E(dt/2, t_{k+1}) C_z C_y C_x E(dt/2, t_k) psi (real time):

* the observed order of convergence in dt is 2 with interaction, dipolar
  term and a time-dependent trap (the paper's first-order splitting shows
  order 1 on the same case, and two plausible mistakes planted in a
  composition of the oracle's substeps fall back to order 1);
* the step is time-reversible: S(-dt) S(dt) = I to rounding (first-order
  splitting is not);
* with g = g_dd = 0 it equals the product of dense matrices
  diag(e^{-i dt s(t_{k+1}) V / 2}) A^{-1} B diag(e^{-i dt s(t_k) V / 2}) per axis
  (numpy.linalg.solve on the Crank-Nicolson matrices).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1601_04640_gb300 import synth

N = 32
H = 0.25


def _params(dt, **kw):
    d = dict(dim=2, n=(N, N), h=(H, H), nu=(1.0, 1.3), g=20.0, gdd=10.0, dt=dt, imag=False,
             kernel="quasi2d", qd=0.5, cm=[1.0, 0.0, 0.0, 0.8])
    d.update(kw)
    return oracle.Params(**d)


def _psi0(seed=1):
    x = synth.axis(N, H)
    rng = np.random.default_rng(seed)
    psi = np.exp(-(1.2 * x[None, :] ** 2 + 0.8 * x[:, None] ** 2) / 2).astype(complex)
    psi *= 1 + 0.05 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N)))
    psi *= np.exp(0.3j * x[None, :])
    return psi / math.sqrt(np.sum(np.abs(psi) ** 2) * H * H)


T_END = 0.16


def _errors(run, ks=(16, 32, 64)):
    psi0 = _psi0()
    ref = oracle.step(_params(T_END / 1024), psi0, 0, 1024, split="strang")
    return [np.linalg.norm(run(k, psi0) - ref) / np.linalg.norm(ref) for k in ks]


def _ratios(e):
    return [e[i] / e[i + 1] for i in range(len(e) - 1)]


def test_strang_second_order():
    e = _errors(lambda k, psi: oracle.step(_params(T_END / k), psi, 0, k, split="strang"))
    for r in _ratios(e):
        assert 3.6 < r < 4.4, (e, _ratios(e))


def test_lie_first_order_on_the_same_case():
    e = _errors(lambda k, psi: oracle.step(_params(T_END / k), psi, 0, k, split="lie"))
    assert _ratios(e)[-1] < 2.5, (e, _ratios(e))


def _cn(p, psi):
    for a in range(p.dim):
        psi = oracle.cn_axis(p, psi, a)
    return psi


def _frozen_density_strang(k, psi):
    """Planted mistake: the closing half reuses the step-start density."""
    p = _params(T_END / k)
    for s in range(k):
        dens = np.abs(psi) ** 2
        phi = oracle.dipolar_potential(p, dens)
        v = oracle.trap(p)
        th0 = 0.5 * p.dt * (oracle.trap_scale(p, s * p.dt) * v + p.g * dens + p.gdd * phi)
        th1 = 0.5 * p.dt * (oracle.trap_scale(p, (s + 1) * p.dt) * v + p.g * dens + p.gdd * phi)
        psi = np.exp(-1j * th1) * _cn(p, np.exp(-1j * th0) * psi)
    return psi


def _step_start_time_strang(k, psi):
    """Planted mistake: both halves take the trap at the step-start time."""
    p = _params(T_END / k)
    for s in range(k):
        psi = oracle.nonlinear_frac(p, psi, s * p.dt, 0.5)
        psi = _cn(p, psi)
        psi = oracle.nonlinear_frac(p, psi, s * p.dt, 0.5)
    return psi


@pytest.mark.parametrize("run", [_frozen_density_strang, _step_start_time_strang])
def test_planted_mistakes_lose_second_order(run):
    e = _errors(run)
    assert _ratios(e)[-1] < 2.6, (e, _ratios(e))


def test_composition_matches_the_oracle_step():
    """The literal composition of the oracle's own substeps (used above for the
    planted mistakes) is the oracle's Strang step."""
    p = _params(0.01)
    psi = _psi0()
    k = 5
    ref = oracle.step(p, psi, k, 1, split="strang")
    alt = oracle.nonlinear_frac(p, _cn(p, oracle.nonlinear_frac(p, psi, k * p.dt, 0.5)),
                                (k + 1) * p.dt, 0.5)
    assert np.max(np.abs(ref - alt)) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_strang_time_reversible(dim):
    if dim == 2:
        p, m = _params(0.01, cm=[]), _params(-0.01, cm=[])
        psi = _psi0()
    else:
        kw = dict(dim=3, n=(16, 12, 10), h=(0.4, 0.45, 0.5), nu=(1.0, 1.2, 1.5), g=15.0, gdd=8.0,
                  imag=False, kernel="dipolar3d")
        p, m = oracle.Params(dt=0.01, **kw), oracle.Params(dt=-0.01, **kw)
        rng = np.random.default_rng(3)
        psi = rng.standard_normal(p.shape()) + 1j * rng.standard_normal(p.shape())
    back = oracle.step(m, oracle.step(p, psi, 0, 1, split="strang"), 0, 1, split="strang")
    assert np.linalg.norm(back - psi) / np.linalg.norm(psi) < 1e-13
    lie = oracle.step(m, oracle.step(p, psi, 0, 1), 0, 1)
    assert np.linalg.norm(lie - psi) / np.linalg.norm(psi) > 1e-5


def _cn_matrix(n, tau):
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A = np.eye(n) + 1j * tau * T
    B = np.eye(n) - 1j * tau * T
    return np.linalg.solve(A, B)


def test_strang_noninteracting_dense():
    nx, ny, hx, hy, dt, k = 12, 10, 0.35, 0.3, 0.05, 3
    cm = [0.4, 0.1]
    p = oracle.Params(dim=2, n=(nx, ny), h=(hx, hy), nu=(1.0, 1.7), g=0.0, gdd=0.0, dt=dt,
                      imag=False, kernel="none", cm=cm)
    rng = np.random.default_rng(11)
    psi = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    x, y = synth.axis(nx, hx), synth.axis(ny, hy)
    V = 0.5 * ((1.0 * x[None, :]) ** 2 + (1.7 * y[:, None]) ** 2)

    def s(t):
        return 1 + sum(c * math.sin((m + 1) * t) for m, c in enumerate(cm))

    Cx = _cn_matrix(nx, dt / (4 * hx * hx))
    Cy = _cn_matrix(ny, dt / (4 * hy * hy))
    ref = np.exp(-0.5j * dt * s(k * dt) * V) * psi
    ref = Cy @ (ref @ Cx.T)
    ref = np.exp(-0.5j * dt * s((k + 1) * dt) * V) * ref
    out = oracle.step(p, psi, k, 1, split="strang")
    assert np.max(np.abs(out - ref)) < 1e-13 * np.max(np.abs(ref))


def test_strang_imaginary_time_refused():
    p = _params(0.01, imag=True)
    with pytest.raises(ValueError):
        oracle.step(p, _psi0(), 0, 1, split="strang")
