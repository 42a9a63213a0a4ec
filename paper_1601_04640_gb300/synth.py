"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the solver's arithmetic: only the random-number
generator and the analytic initial states the workloads start from.

Random numbers: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) gives 64-bit
words; the top 53 bits make a uniform double in [0, 1); the Box-Muller
transform turns pairs of uniforms into pairs of independent standard normals.
Everything is generated on the host in FP64 so both sides see the same bits.
"""
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Words offset .. offset+count-1 of the SplitMix64 stream for `seed`."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each word."""
    w = splitmix64(seed, count, offset)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal_pairs(seed: int, count: int):
    """`count` pairs (xi, eta) of independent N(0, 1) values (Box-Muller)."""
    u = uniform(seed, 2 * count)
    u1 = 1.0 - u[0::2]          # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    return r * np.cos(2.0 * math.pi * u2), r * np.sin(2.0 * math.pi * u2)


def axis(n: int, h: float) -> np.ndarray:
    """Grid coordinates x_i = (i - n/2) h."""
    return (np.arange(n, dtype=np.float64) - (n // 2)) * h


def gaussian_state(n, h, a, noise=0.0, seed=0, amplitude=None):
    """psi0 = A exp(-sum_i a_i x_i^2 / 2) (1 + noise (xi + i eta)).

    n, h, a: per-axis (x, y[, z]) sizes, spacings and width coefficients.
    A defaults to the continuum normalisation prod_i (a_i / pi)^(1/4), so the
    envelope has unit integral of |psi|^2 on an infinite domain.
    Returns complex128 of shape (nz, ny, nx) or (ny, nx)."""
    dim = len(n)
    if amplitude is None:
        amplitude = 1.0
        for ai in a:
            amplitude *= (ai / math.pi) ** 0.25
    env = None
    for ax in range(dim):
        x = axis(n[ax], h[ax])
        f = np.exp(-0.5 * a[ax] * x * x)
        shape = [1] * dim
        shape[dim - 1 - ax] = n[ax]
        f = f.reshape(shape)
        env = f if env is None else env * f
    env = amplitude * env
    shape = tuple(reversed(list(n)))
    psi = np.broadcast_to(env, shape).astype(np.complex128)
    if noise:
        xi, eta = normal_pairs(seed, psi.size)
        psi = psi * (1.0 + noise * (xi + 1j * eta)).reshape(shape)
    return np.ascontiguousarray(psi)


def trap_modulation(seed: int, M: int = 8, amp: float = 0.05) -> np.ndarray:
    """c_1..c_M ~ U(-amp, amp) for V(t) = V0 (1 + sum_m c_m sin(m t))."""
    return (2.0 * uniform(seed, M) - 1.0) * amp


BATCH_SIZES = (64, 96, 128, 160, 256, 384, 512)


def batched_problems(seed: int, count: int, sizes=BATCH_SIZES, h=0.2, dt=1e-3,
                     qd=0.5):
    """Parameter sweep for independent 2D XY problems.

    Size uniform over `sizes`; nu_x = 1, nu_y ~ U[0.5, 2]; g ~ U[10, 200];
    g_dd = g * U[0, 0.8]; even index -> imaginary time, odd -> real time."""
    u = uniform(seed, 5 * count).reshape(count, 5)
    out = []
    for i in range(count):
        n = sizes[min(int(u[i, 0] * len(sizes)), len(sizes) - 1)]
        nuy = 0.5 + 1.5 * u[i, 1]
        g = 10.0 + 190.0 * u[i, 2]
        gdd = g * 0.8 * u[i, 3]
        out.append(dict(n=(n, n), h=(h, h), nu=(1.0, nuy), g=g, gdd=gdd,
                        dt=dt, imag=(i % 2 == 0), qd=qd,
                        seed=int(splitmix64(seed ^ 0x5EED, 1, i)[0] >> np.uint64(1))))
    return out
