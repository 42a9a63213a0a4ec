"""Pins for the oracle's dipolar potential (convolution theorem with
U(k) = (4 pi/3)(3 kz^2/k^2 - 1), U(0) = 0) and the quasi-2D XY kernel:
exact single Fourier modes, a continuum closed form for a Gaussian density,
a brute-force direct-space sum, and quadrature of the 3D kernel."""
import math

import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_1601_04640_gb300 import synth


def _grid(n, h):
    x = [synth.axis(n[a], h[a]) for a in range(len(n))]
    return np.meshgrid(*reversed(x), indexing="ij")  # Z, Y, X (3D) or Y, X


def _p3(n, h):
    return oracle.Params(dim=3, n=n, h=h, nu=(1, 1, 1), kernel="dipolar3d")


@pytest.mark.parametrize("axis,m,factor", [
    (2, 1, 8 * math.pi / 3),      # k along z: U = (4pi/3)(3 - 1)
    (2, 3, 8 * math.pi / 3),
    (0, 2, -4 * math.pi / 3),     # k along x: U = (4pi/3)(0 - 1)
    (1, 5, -4 * math.pi / 3),
])
def test_single_mode(axis, m, factor):
    n, h = (16, 12, 20), (0.3, 0.4, 0.25)
    Z, Y, X = _grid(n, h)
    c = (X, Y, Z)[axis]
    k = 2 * math.pi * m / (n[axis] * h[axis])
    eps = 0.1
    dens = 1.0 + eps * np.cos(k * c)
    phi = oracle.dipolar_potential(_p3(n, h), dens)
    assert np.max(np.abs(phi - factor * eps * np.cos(k * c))) < 1e-12


def test_diagonal_mode_and_constant():
    n, h = (16, 16, 16), (0.25, 0.25, 0.25)
    Z, Y, X = _grid(n, h)
    k = 2 * math.pi * 2 / (n[0] * h[0])
    dens = 2.0 + 0.3 * np.cos(k * X + k * Z)      # 3 cos^2 = 3/2
    phi = oracle.dipolar_potential(_p3(n, h), dens)
    assert np.max(np.abs(phi - 0.3 * (2 * math.pi / 3) * np.cos(k * X + k * Z))) < 1e-12
    phi0 = oracle.dipolar_potential(_p3(n, h), np.full(Z.shape, 3.7))
    assert np.max(np.abs(phi0)) < 1e-13


def _gaussian_phi(X, Y, Z, sigma):
    """Continuum Phi for n = (2 pi s^2)^(-3/2) exp(-r^2/(2 s^2)):
    (1 - 3 cos^2)/r^3 = -d_z^2 (1/r) - (4 pi/3) delta, so
    Phi = -d_z^2 phiN - (4 pi/3) n with phiN = erf(r/a)/r, a = sqrt(2) s."""
    a = math.sqrt(2.0) * sigma
    r = np.sqrt(X * X + Y * Y + Z * Z)
    n = (2 * math.pi * sigma ** 2) ** -1.5 * np.exp(-r * r / (2 * sigma ** 2))
    c0 = 2.0 / (a * math.sqrt(math.pi))
    small = r < 0.05 * a
    rs = np.where(small, 1.0, r)
    E = special.erf(rs / a)
    E1 = c0 * np.exp(-rs * rs / (a * a))
    E2 = -(2 * rs / (a * a)) * E1
    d1 = E1 / rs - E / rs ** 2                    # phiN'
    d2 = E2 / rs - 2 * E1 / rs ** 2 + 2 * E / rs ** 3   # phiN''
    d1_over_r = d1 / rs
    # series phiN = c0 (1 - r^2/(3a^2) + r^4/(10 a^4)) near the origin
    c2, c4 = -c0 / (3 * a * a), c0 / (10 * a ** 4)
    d1_over_r = np.where(small, 2 * c2 + 4 * c4 * r * r, d1_over_r)
    d2 = np.where(small, 2 * c2 + 12 * c4 * r * r, d2)
    cz2 = np.where(r > 0, Z * Z / np.where(r > 0, r * r, 1.0), 1.0 / 3.0)
    dzz = d2 * cz2 + d1_over_r * (1.0 - cz2)
    return -dzz - (4 * math.pi / 3) * n, n


def test_gaussian_closed_form():
    """Anisotropic spacing (hz != hx) pins the k-grid scaling and the axis.
    The remaining difference is the periodic-image field, which falls as
    (sigma/L)^3: check the level and the cubic rate between two boxes."""
    sigma = 0.6
    errs = []
    for L in (8.0, 12.0):
        n = (int(L / 0.25), int(L / 0.25), int(L / 0.2))
        h = (0.25, 0.25, 0.2)
        Z, Y, X = _grid(n, h)
        ref, dens = _gaussian_phi(X, Y, Z, sigma)
        phi = oracle.dipolar_potential(_p3(n, h), dens)
        errs.append(np.max(np.abs((phi - phi.mean()) - (ref - ref.mean()))) / np.max(np.abs(ref)))
    assert errs[1] < 0.02
    assert 2.8 < errs[0] / errs[1] < 4.0      # (12/8)^3 = 3.375


def _brute(n, h, dens):
    """Direct sum h^3 sum_{j != i} (1 - 3 cos^2 theta_ij)/r_ij^3 n_j over the
    minimum-image box (the on-site cell integrates to zero by cubic symmetry)."""
    Z, Y, X = _grid((n, n, n), (h, h, h))
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    nn = dens.ravel()
    L = n * h
    out = np.empty(len(pts))
    for i in range(len(pts)):
        d = pts - pts[i]
        d -= L * np.round(d / L)
        r2 = (d * d).sum(1)
        r2[i] = 1.0
        u = (1.0 - 3.0 * d[:, 2] ** 2 / r2) / r2 ** 1.5
        u[i] = 0.0
        out[i] = h ** 3 * np.dot(u, nn)
    return out.reshape(dens.shape)


def test_brute_force_direct_sum_converges():
    """FFT route vs brute-force real-space sum on tiny grids: the discrepancy
    comes from periodic images and falls as the box grows (h fixed)."""
    errs = []
    for n in (16, 24):
        h = 0.5
        Z, Y, X = _grid((n, n, n), (h, h, h))
        dens = np.exp(-(X ** 2 + Y ** 2 + (Z / 1.3) ** 2) / (2 * 0.81))
        f = oracle.dipolar_potential(_p3((n, n, n), (h, h, h)), dens)
        b = _brute(n, h, dens)
        f -= f.mean()
        b -= b.mean()
        errs.append(np.max(np.abs(f - b)) / np.max(np.abs(f)))
    assert errs[1] < errs[0]
    assert errs[1] < 0.06


def test_cubic_symmetry_zero_energy():
    """On a cubic grid a density symmetric under axis permutations has
    sum n Phi = 0 (the angular average of 3 cos^2 - 1 vanishes)."""
    n, h = (16, 16, 16), (0.4, 0.4, 0.4)
    Z, Y, X = _grid(n, h)
    dens = np.exp(-(X ** 2 + Y ** 2 + Z ** 2)) + 0.3 * np.exp(-((X * Y) ** 2 + (Y * Z) ** 2 + (X * Z) ** 2))
    phi = oracle.dipolar_potential(_p3(n, h), dens)
    assert abs(np.sum(phi * dens)) < 1e-12 * np.sum(np.abs(phi * dens))


# k d / sqrt(2) reaches the asymptotic erfcx branch (u >= 25) from k = 40 at
# d = 1 and k = 80 at d = 0.5 (the corner of a 128^2 grid at h = 0.05 has
# k = 88.9)
@pytest.mark.parametrize("k", [0.0, 0.3, 1.0, 2.5, 7.0, 20.0, 40.0, 60.0, 80.0, 120.0])
@pytest.mark.parametrize("d", [0.5, 1.0])
def test_quasi2d_kernel_vs_quadrature(k, d):
    """U2(k) = int dkz/(2pi) (4pi/3)(3 kz^2/(k^2 + kz^2) - 1) exp(-kz^2 d^2/2)."""
    f = lambda kz: (4 * math.pi / 3) * (3 * kz * kz / (k * k + kz * kz) - 1) * math.exp(-kz * kz * d * d / 2) / (2 * math.pi) if (k > 0 or kz != 0) else -(4 * math.pi / 3) / (2 * math.pi)
    val, _ = integrate.quad(f, -np.inf, np.inf, epsabs=1e-13, epsrel=1e-12, limit=400)
    assert abs(oracle.q2d_value(k, d) - val) < 1e-10 * max(1.0, abs(val))


def test_quasi2d_single_mode():
    n, h, d = (24, 20), (0.2, 0.3), 0.5
    Y, X = _grid(n, h)
    kx = 2 * math.pi * 3 / (n[0] * h[0])
    p = oracle.Params(dim=2, n=n, h=h, nu=(1, 1), kernel="quasi2d", qd=d)
    dens = 1.0 + 0.2 * np.cos(kx * X)
    phi = oracle.dipolar_potential(p, dens)
    U0 = oracle.q2d_value(0.0, d)
    ref = U0 * 1.0 + 0.2 * oracle.q2d_value(kx, d) * np.cos(kx * X)
    assert np.max(np.abs(phi - ref)) < 1e-12


@pytest.mark.parametrize("kx,kz", [(0.0, 0.4), (0.7, 0.0), (1.0, 1.0), (0.3, 2.5), (5.0, 3.0), (12.0, 20.0),
                                   (60.0, 60.0), (0.0, 90.0), (20.0, 80.0), (62.8, 31.4)])
@pytest.mark.parametrize("d", [0.5, 1.0])
def test_quasi2d_xz_kernel_vs_quadrature(kx, kz, d):
    """XZ plane, dipoles along z in the plane, transverse profile in y:
    U(kx, kz) = int dky/(2pi) (4pi/3)(3 kz^2/(kx^2 + ky^2 + kz^2) - 1) exp(-ky^2 d^2/2)."""
    def f(ky):
        k2 = kx * kx + ky * ky + kz * kz
        return (4 * math.pi / 3) * (3 * kz * kz / k2 - 1) * math.exp(-ky * ky * d * d / 2) / (2 * math.pi)
    val, _ = integrate.quad(f, -np.inf, np.inf, epsabs=1e-13, epsrel=1e-12, limit=400)
    assert abs(oracle.q2dxz_value(kx, kz, d) - val) < 1e-10 * max(1.0, abs(val))


@pytest.mark.parametrize("d", [0.3, 0.5, 1.0])
def test_quasi2d_xz_identities(d):
    """Exact consequences of the definition.  With kz = 0 the in-plane term
    vanishes: U(kx, 0) = -(4pi/3)/(sqrt(2pi) d) for every kx.  At kx = 0, kz = k
    the XZ integrand is 3 k^2/(k^2 + ky^2) - 1 and the XY kernel's (dipoles
    along the integrated axis) is 3 ky^2/(k^2 + ky^2) - 1; their sum is 1, so
    U_XZ(0, k) + U_XY(k) = (4pi/3)/(sqrt(2pi) d)."""
    pref = (4 * math.pi / 3) / (math.sqrt(2 * math.pi) * d)
    for kx in (0.0, 0.1, 1.0, 7.0, 40.0):
        assert abs(oracle.q2dxz_value(kx, 0.0, d) + pref) < 1e-13 * pref
    for k in (0.05, 0.5, 2.0, 9.0, 30.0):
        assert abs(oracle.q2dxz_value(0.0, k, d) + oracle.q2d_value(k, d) - pref) < 1e-12 * pref


def test_quasi2d_xz_single_modes():
    """Fourier modes along z and along x on the (x, z) grid."""
    n, h, d = (24, 20), (0.2, 0.3), 0.5
    Z, X = _grid(n, h)
    kz = 2 * math.pi * 2 / (n[1] * h[1])
    kx = 2 * math.pi * 3 / (n[0] * h[0])
    p = oracle.Params(dim=2, n=n, h=h, nu=(1, 1), kernel="quasi2d_xz", qd=d)
    dens = 1.0 + 0.2 * np.cos(kz * Z) + 0.1 * np.cos(kx * X)
    phi = oracle.dipolar_potential(p, dens)
    U0 = oracle.q2dxz_value(0.0, 0.0, d)
    ref = U0 + 0.2 * oracle.q2dxz_value(0.0, kz, d) * np.cos(kz * Z) + 0.1 * oracle.q2dxz_value(kx, 0.0, d) * np.cos(kx * X)
    assert np.max(np.abs(phi - ref)) < 1e-12
    # dipoles along z in the plane: the kernel is positive for wave vectors
    # along the dipoles and negative across them
    assert oracle.q2dxz_value(0.0, kz, d) > 0 > oracle.q2dxz_value(kx, 0.0, d)


@pytest.mark.parametrize("u", [0.0, 1e-3, 0.5, 3.0, 10.0, 24.0, 24.999, 25.0, 25.001, 26.0, 30.0, 45.0,
                               88.9, 300.0, 1e4])
def test_erfcx_vs_library(u):
    """exp(u^2) erfc(u) of the quasi-2D kernels against scipy's erfcx on both
    sides of u = 25, where the oracle switches from the direct product to the
    asymptotic series.  Near u = 25 the direct product carries the rounding
    of u^2 in exp (about 625 x 1.1e-16 relative); above it the series is
    held to 2e-15, which its sixth term (2.7e-15 at u = 25) still exceeds."""
    ref = special.erfcx(u)
    assert abs(oracle.erfcx(u) - ref) <= (2e-13 if u < 25.0 else 2e-15) * ref


@pytest.mark.parametrize("d", [0.5, 1.0])
def test_quasi2d_kernels_continuous_at_branch(d):
    """Both kernels are smooth in k: just below and just above the k where
    u = k d / sqrt(2) crosses 25 the values agree to the derivative times the
    gap (a dropped or mis-signed term of the series would leave a jump of
    3 pref / q^2 ~ 2e-3 relative, the third term one of ~2e-6)."""
    k0 = 25.0 * math.sqrt(2.0) / d
    dk = 1e-12 * k0  # slope x gap: ~1e-14 relative
    lo, hi = oracle.q2d_value(k0 - dk, d), oracle.q2d_value(k0 + dk, d)
    assert abs(hi - lo) < 3e-13 * abs(lo)
    for ang in (0.3, 0.8, 1.2):  # XZ on rays through the branch circle
        a = (k0 - dk) * math.cos(ang), (k0 - dk) * math.sin(ang)
        b = (k0 + dk) * math.cos(ang), (k0 + dk) * math.sin(ang)
        lo, hi = oracle.q2dxz_value(*a, d), oracle.q2dxz_value(*b, d)
        assert abs(hi - lo) < 3e-13 * max(abs(lo), (4 * math.pi / 3) / (math.sqrt(2 * math.pi) * d))


def test_asymptotic_region_carries_weight_on_128_grid():
    """The GPU parity case on a 128^2 grid at h = 0.05, d = 0.5 checks the
    asymptotic branch only if the density has weight where u >= 25.  Planting
    mistakes in the oracle's U table there (on the CPU) shows it does: a
    flipped 1/q^2 term moves Phi_d by > 1e-5 (the FP32-bulk bound) and a 1e-6
    relative error by > 1e-10 (far above the FP64 bound)."""
    n, h, d = (128, 128), (0.05, 0.05), 0.5
    psi = synth.gaussian_state(n, h, (1.0, 1.5), 0.05, 11)
    dens = np.abs(psi) ** 2
    U = oracle.kernel_q2d(n, h, d)
    kx = 2 * np.pi * np.fft.fftfreq(n[0], h[0])
    ky = 2 * np.pi * np.fft.fftfreq(n[1], h[1])
    KX, KY = np.meshgrid(kx, ky)
    q = np.hypot(KX, KY) * d
    mask = q / math.sqrt(2) >= 25
    assert 0.05 < mask.mean() < 0.2
    pref = (4 * math.pi / 3) / (math.sqrt(2 * math.pi) * d)
    F = np.fft.fft2(dens)
    phi = np.real(np.fft.ifft2(U * F))
    bad = U.copy()
    bad[mask] -= pref * 6 / q[mask] ** 2
    assert np.linalg.norm(np.real(np.fft.ifft2(bad * F)) - phi) > 1e-5 * np.linalg.norm(phi)
    bad = U.copy()
    bad[mask] *= 1 + 1e-6
    assert np.linalg.norm(np.real(np.fft.ifft2(bad * F)) - phi) > 1e-10 * np.linalg.norm(phi)
