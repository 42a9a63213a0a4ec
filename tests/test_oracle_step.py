"""Pins for the oracle's full step and observables: closed forms of the
exponential substep, exact real-time norm conservation, the exact discrete
noninteracting ground state (dense power iteration on the 1-D factors),
mu = (nu_x + nu_y + nu_z)/2 in the continuum limit, Gaussian observables and
an independent k-space quadrature of the dipolar energy."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from paper_1601_04640_gb300 import synth

RNG = np.random.default_rng(2016)


def _grid(n, h):
    x = [synth.axis(n[a], h[a]) for a in range(len(n))]
    return np.meshgrid(*reversed(x), indexing="ij")


def _V(p):
    G = _grid(tuple(p.n[:p.dim]), tuple(p.h[:p.dim]))
    coords = list(reversed(G))       # X, Y[, Z]
    return 0.5 * sum((p.nu[a] * coords[a]) ** 2 for a in range(p.dim))


@pytest.mark.parametrize("imag", [False, True])
def test_exp_substep_closed_form(imag):
    cm = [0.03, -0.02, 0.01]
    p = oracle.Params(dim=3, n=(8, 10, 12), h=(0.3, 0.3, 0.25), nu=(1, 1.5, 2), g=0, gdd=0,
                      dt=0.01, imag=imag, kernel="dipolar3d", cm=cm)
    psi = RNG.standard_normal(p.shape()) + 1j * RNG.standard_normal(p.shape())
    step = 7
    t = step * p.dt
    s = 1 + sum(c * math.sin((m + 1) * t) for m, c in enumerate(cm))
    th = p.dt * s * _V(p)
    ref = psi * (np.exp(-th) if imag else np.exp(-1j * th))
    assert np.max(np.abs(oracle.nonlinear(p, psi, step) - ref)) < 1e-14


def test_exp_substep_real_time_keeps_modulus():
    p = oracle.Params(dim=3, n=(12, 12, 12), h=(0.3,) * 3, nu=(1, 1, 1), g=30, gdd=20,
                      dt=0.01, imag=False, kernel="dipolar3d")
    psi = synth.gaussian_state((12, 12, 12), (0.3,) * 3, (1, 1, 1), 0.05, 3)
    out = oracle.nonlinear(p, psi, 0)
    assert np.max(np.abs(np.abs(out) - np.abs(psi))) < 1e-15


@pytest.mark.parametrize("dim", [2, 3])
def test_real_time_norm_conserved(dim):
    if dim == 3:
        p = oracle.Params(dim=3, n=(16, 16, 16), h=(0.4,) * 3, nu=(1, 1, 0.5), g=150, gdd=60,
                          dt=5e-3, imag=False, kernel="dipolar3d")
        psi = synth.gaussian_state((16, 16, 16), (0.4,) * 3, (1, 1, 0.5), 0.01, 5)
    else:
        p = oracle.Params(dim=2, n=(32, 24), h=(0.3, 0.3), nu=(1, 1.5), g=50, gdd=30,
                          dt=5e-3, imag=False, kernel="quasi2d", qd=0.5)
        psi = synth.gaussian_state((32, 24), (0.3, 0.3), (1, 1.5), 0.01, 5)
    n0 = oracle.observables(p, psi)["norm"]
    out = oracle.step(p, psi, 0, 200)
    assert abs(oracle.observables(p, out)["norm"] / n0 - 1) < 1e-12
    # and over the 2000 steps of the real-time workload (rounding only: measured 6e-13 to 7e-13)
    out = oracle.step(p, out, 200, 1800)
    assert abs(oracle.observables(p, out)["norm"] / n0 - 1) < 2e-12


def _dominant(n, h, nu, dt):
    """Dominant eigenvector of (A^-1 B) diag(exp(-dt nu^2 x^2 / 2)) (dense)."""
    x = synth.axis(n, h)
    tau = dt / (4 * h * h)
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    A = np.eye(n) + tau * T
    B = np.eye(n) - tau * T
    M = np.linalg.solve(A, B) @ np.diag(np.exp(-dt * 0.5 * nu * nu * x * x))
    w, v = np.linalg.eig(M)
    u = np.real(v[:, np.argmax(np.abs(w))])
    return u * np.sign(u[n // 2])


def test_noninteracting_ground_state_exact_discrete():
    """g = g_dd = 0: the step is the tensor product of the 1-D maps
    (A_a^-1 B_a) exp(-dt V_a); normalised power iteration converges to the
    product of their dominant eigenvectors."""
    n, h, nu, dt = (16, 14, 12), (0.5, 0.5, 0.5), (1.0, 1.5, 2.0), 0.05
    p = oracle.Params(dim=3, n=n, h=h, nu=nu, g=0, gdd=0, dt=dt, imag=True, kernel="dipolar3d")
    psi = synth.gaussian_state(n, h, (1, 1, 1), 0.0)
    out = oracle.step(p, psi, 0, 600)
    ux, uy, uz = (_dominant(n[a], h[a], nu[a], dt) for a in range(3))
    ref = uz[:, None, None] * uy[None, :, None] * ux[None, None, :]
    ref /= math.sqrt(np.sum(ref ** 2) * h[0] * h[1] * h[2])
    assert np.max(np.abs(out - ref)) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_noninteracting_mu_continuum(dim):
    """mu -> (nu_x + nu_y [+ nu_z]) / 2 as h, dt -> 0 (harmonic ground state)."""
    if dim == 3:
        n, h, nu = (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)
    else:
        n, h, nu = (48, 40), (0.2, 0.2), (1.0, 1.5)
    p = oracle.Params(dim=dim, n=n, h=h, nu=nu, g=0, gdd=0, dt=0.005, imag=True,
                      kernel="dipolar3d" if dim == 3 else "quasi2d")
    psi = synth.gaussian_state(n, h, nu, 0.0)
    out = oracle.step(p, psi, 0, 1500)
    o = oracle.observables(p, out)
    # O(h^2) from the 3-point kinetic stencil dominates at these spacings
    assert abs(o["mu"] - sum(nu) / 2) < 2e-2
    assert abs(o["energy"] - sum(nu) / 2) < 2e-2
    assert abs(o["norm"] - 1) < 1e-12
    for a in range(dim):
        assert abs(o["rms"][a] - 1 / math.sqrt(2 * nu[a])) < 1e-2


def test_noninteracting_mu_second_order_in_h():
    """Halving h (with dt/4) cuts |mu - (nu_x + nu_y)/2| by about 4 (2D)."""
    errs = []
    for h, n, dt, steps in ((0.4, 24, 0.02, 800), (0.2, 48, 0.005, 3200)):
        nu = (1.0, 1.5)
        p = oracle.Params(dim=2, n=(n, n), h=(h, h), nu=nu, g=0, gdd=0, dt=dt, imag=True,
                          kernel="quasi2d")
        out = oracle.step(p, synth.gaussian_state((n, n), (h, h), nu, 0.0), 0, steps)
        errs.append(abs(oracle.observables(p, out)["mu"] - 1.25))
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_gaussian_observables():
    n, h, nu = (48, 48, 48), (0.2,) * 3, (1.0, 1.0, 1.0)
    g = 7.0
    p = oracle.Params(dim=3, n=n, h=h, nu=nu, g=g, gdd=0, dt=0.01, kernel="dipolar3d")
    psi = synth.gaussian_state(n, h, nu, 0.0)          # pi^-3/4 exp(-r^2/2)
    o = oracle.observables(p, psi)
    assert abs(o["norm"] - 1) < 1e-10
    assert abs(o["pot"] - 0.75) < 1e-8
    assert abs(o["contact"] - g * (2 * math.pi) ** -1.5) < 1e-8
    assert all(abs(r - 1 / math.sqrt(2)) < 1e-8 for r in o["rms"])
    assert abs(o["rms_r"] - math.sqrt(1.5)) < 1e-8
    assert abs(o["kin"] - 0.75) < 0.75 * h[0] ** 2    # forward differences: O(h^2)


def test_kinetic_summation_by_parts():
    """The forward-difference kinetic sum equals <psi, H psi> with the
    3-point second difference and zero ghosts (independent formula)."""
    n, h = (10, 12, 9), (0.3, 0.35, 0.4)
    p = oracle.Params(dim=3, n=n, h=h, nu=(0, 0, 0), g=0, gdd=0, kernel="none")
    psi = RNG.standard_normal(p.shape()) + 1j * RNG.standard_normal(p.shape())
    o = oracle.observables(p, psi)
    pad = np.pad(psi, 1)
    lap = np.zeros_like(psi)
    for ax, hh in ((2, h[0]), (1, h[1]), (0, h[2])):
        sl_p = [slice(1, -1)] * 3
        sl_m = [slice(1, -1)] * 3
        sl_p[ax] = slice(2, None)
        sl_m[ax] = slice(0, -2)
        lap += (pad[tuple(sl_p)] - 2 * psi + pad[tuple(sl_m)]) / hh ** 2
    w = h[0] * h[1] * h[2]
    K = np.real(np.sum(np.conj(psi) * (-0.5 * lap))) * w
    assert abs(o["kin"] * o["norm"] - K) < 1e-10 * abs(K)


@pytest.mark.parametrize("sr,sz,sign", [(1.0, 0.6, 1), (0.6, 1.0, -1)])
def test_dipolar_energy_anisotropic_gaussian(sr, sz, sign):
    """sum n Phi for n = exp(-rho^2/sr^2 - z^2/sz^2)/(pi^1.5 sr^2 sz) vs
    (4 pi/3) int d^3k/(2pi)^3 (3 cos^2 a - 1) exp(-k^2 c(a)/2),
    c(a) = sr^2 sin^2 a + sz^2 cos^2 a, by 1-D quadrature over a."""
    f = lambda a: math.sin(a) * (3 * math.cos(a) ** 2 - 1) * math.sqrt(math.pi) / (
        4 * ((sr ** 2 * math.sin(a) ** 2 + sz ** 2 * math.cos(a) ** 2) / 2) ** 1.5)
    val, _ = integrate.quad(f, 0, math.pi, epsabs=1e-14, epsrel=1e-13)
    ref = (4 * math.pi / 3) / (4 * math.pi ** 2) * val
    n, h = (64, 64, 64), (0.25,) * 3
    p = oracle.Params(dim=3, n=n, h=h, nu=(0, 0, 0), g=0, gdd=1.0, kernel="dipolar3d")
    # psi^2 = n  ->  psi = exp(-rho^2/(2 sr^2) - z^2/(2 sz^2)) / (pi^0.75 sr sz^0.5)
    psi = synth.gaussian_state(n, h, (1 / sr ** 2, 1 / sr ** 2, 1 / sz ** 2), 0.0)
    o = oracle.observables(p, psi)
    assert np.sign(ref) == sign     # oblate (flattened along the dipoles) > 0
    assert abs(o["dipolar"] - ref) < 2e-3 * abs(ref)


@pytest.mark.parametrize("dim", [2, 3])
def test_imaginary_time_keeps_a_real_state_real(dim):
    """Imaginary-time evolution with a real potential maps real states to real
    states: every substep (the real factor e^{-dt(...)}, Crank-Nicolson with
    real coefficients, the renormalisation) is real.  The oracle's complex step
    on a real input keeps the imaginary part exactly zero over many steps; a
    real-time step does not."""
    if dim == 3:
        n, h, nu, kernel = (16, 12, 20), (0.3, 0.35, 0.25), (1.0, 1.2, 0.8), "dipolar3d"
    else:
        n, h, nu, kernel = (24, 20), (0.25, 0.3), (1.0, 1.4), "quasi2d"
    psi = RNG.standard_normal(tuple(reversed(n))) + 0.0j
    p = oracle.Params(dim=dim, n=n, h=h, nu=nu, g=40.0, gdd=15.0, dt=2e-3, imag=True, kernel=kernel,
                      cm=[0.2])
    out = oracle.step(p, psi, 0, 25)
    assert np.max(np.abs(out.imag)) == 0.0
    assert np.max(np.abs(out.real)) > 0.0
    p.imag = False
    assert np.max(np.abs(oracle.step(p, psi, 0, 1).imag)) > 1e-6


def test_divergence_golden_first_checkpoint_reproduces():
    """tests/golden/divergence_64.json came from the oracle: its first
    checkpoint (100 steps, 2^-24 noise after every step) is re-derived here."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "divergence_64.json")
    with open(path) as f:
        gold = json.load(f)
    assert gold["checkpoints"][0] == 100
    n, h, nu = (64, 64, 64), (0.2,) * 3, (1.0, 1.0, 0.5)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=150, gdd=60, dt=5e-4, imag=False, kernel="dipolar3d")
    psi0 = synth.gaussian_state(n, h, (0.8, 0.8, 0.4), 0.01, 9)
    base = oracle.step(op, psi0, 0, 100)
    psi, eps = psi0, gold["fp32_rounding"]["eps"]
    for s in range(100):
        psi = oracle.step(op, psi, s, 1)
        xi, _ = synth.normal_pairs(77 + s, psi.size)
        psi = psi * (1.0 + eps * xi.reshape(psi.shape))
    d = float(np.linalg.norm(psi - base) / np.linalg.norm(base))
    assert abs(d / gold["fp32_rounding"]["every_step"][0] - 1) < 1e-6
