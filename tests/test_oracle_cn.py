"""Pins for the oracle's Thomas solver and Crank-Nicolson substeps: dense LU,
exact Dirichlet sine modes, unitarity, commutation."""
import numpy as np
import pytest

import oracle

RNG = np.random.default_rng(4640)


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 255])
def test_thomas_vs_dense(n):
    a = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    c = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    b = 3.0 + np.abs(a) + np.abs(c) + 1j * RNG.standard_normal(n)
    d = RNG.standard_normal(n) + 1j * RNG.standard_normal(n)
    A = np.diag(b) + np.diag(a[1:], -1) + np.diag(c[:-1], 1)
    x = oracle.thomas(a, b, c, d)
    ref = np.linalg.solve(A, d)
    assert np.max(np.abs(x - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))
    assert np.max(np.abs(A @ x - d)) <= 1e-13 * np.max(np.abs(d)) * 4


def _params(imag, n=(10, 12, 14), h=(0.3, 0.25, 0.2), dt=0.01, dim=3):
    return oracle.Params(dim=dim, n=n, h=h, nu=(1, 1, 1), g=0, gdd=0, dt=dt,
                         imag=imag, kernel="none")


@pytest.mark.parametrize("imag", [False, True])
@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("mode", [1, 2, 5])
def test_cn_dirichlet_sine_mode(imag, axis, mode):
    """v_j(i) = sin(pi j (i+1)/(N+1)) is an eigenvector of T = tridiag(-1,2,-1)
    with eigenvalue mu_j = 4 sin^2(pi j / (2(N+1))); CN multiplies it by
    (1 - kappa tau mu) / (1 + kappa tau mu)."""
    p = _params(imag)
    N = p.n[axis]
    i = np.arange(N)
    v = np.sin(np.pi * mode * (i + 1) / (N + 1))
    oshape = list(p.shape())
    oshape[2 - axis] = 1          # the other factor is constant along the axis
    other = RNG.standard_normal(oshape) + 1j * RNG.standard_normal(oshape)
    shape = [1, 1, 1]
    shape[2 - axis] = N
    psi = np.ascontiguousarray(np.broadcast_to(other * v.reshape(shape), p.shape()))
    tau = p.dt / (4 * p.h[axis] ** 2)
    kt = tau if imag else 1j * tau
    mu = 4 * np.sin(np.pi * mode / (2 * (N + 1))) ** 2
    factor = (1 - kt * mu) / (1 + kt * mu)
    out = oracle.cn_axis(p, psi, axis)
    assert np.max(np.abs(out - factor * psi)) < 1e-13


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_cn_real_time_unitary(axis):
    p = _params(False, dt=0.05)
    psi = RNG.standard_normal(p.shape()) + 1j * RNG.standard_normal(p.shape())
    out = oracle.cn_axis(p, psi, axis)
    # per-line norm is preserved: sum over the axis of |psi|^2
    ax = 2 - axis
    assert np.max(np.abs(np.sum(np.abs(out) ** 2, axis=ax) - np.sum(np.abs(psi) ** 2, axis=ax))) < 1e-12


def test_cn_axes_commute():
    p = _params(False, dt=0.05)
    psi = RNG.standard_normal(p.shape()) + 1j * RNG.standard_normal(p.shape())
    a = oracle.cn_axis(p, oracle.cn_axis(p, psi, 0), 2)
    b = oracle.cn_axis(p, oracle.cn_axis(p, psi, 2), 0)
    assert np.max(np.abs(a - b)) < 1e-13


def test_cn_2d_axes():
    p = _params(False, n=(12, 9), h=(0.2, 0.3), dim=2)
    psi = RNG.standard_normal(p.shape()) + 1j * RNG.standard_normal(p.shape())
    out = oracle.cn_axis(p, psi, 1)
    assert np.allclose(np.sum(np.abs(out) ** 2, axis=0), np.sum(np.abs(psi) ** 2, axis=0), atol=1e-12)
