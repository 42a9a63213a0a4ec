"""Write divergence_64.json: how fast the 256^3 workload's dynamics amplify a
rounding-sized difference, measured on the oracle alone.

The real-time workload (g = 150, g_dd = 60 after the quench, cigar trap
nu = (1, 1, 0.5), dt = 5e-4) has eps_dd = (4 pi / 3) g_dd / g = 1.68 > 1 in a
trap elongated along the dipoles, so its evolution is dynamically unstable.
This script runs the FP64 oracle on a 64^3 grid over the same box (h = 0.2)
from the seed-9 Gaussian, once unperturbed and then with rounding-sized
perturbations, and records the relative L2 distance between each perturbed run
and the unperturbed one at the checkpoints:
  * "initial": psi0 (1 + eps xi) once, xi ~ N(0, 1) per site (real, seed 77);
  * "every_step": psi <- psi (1 + eps xi_s) after every step s, a fresh xi_s
    per step (seed 77 + s), which models a solver whose arithmetic rounds
    differently from the oracle's in every step;
with eps = 2^-53 (FP64 rounding) and eps = 2^-24 (FP32 rounding).  The GPU
tests compare their own error against the oracle with these curves: an error
that tracks the oracle's own amplification of rounding-sized differences
comes from the dynamics, not from the kernels.

Calls only oracle/ and the seeded input generator.  Run from the repository
root:  python tests/golden/make_divergence.py   (about 8 minutes on 8 cores)
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1601_04640_gb300 import synth  # noqa: E402

N, H, NU = (64, 64, 64), (0.2, 0.2, 0.2), (1.0, 1.0, 0.5)
G, GDD, DT = 150.0, 60.0, 5e-4
WIDTHS, SEED, PSEED = (0.8, 0.8, 0.4), 9, 77
CHECKPOINTS = [100, 250, 500, 750, 1000, 1250, 1500, 1750, 2000]
EPS = {"fp64_rounding": 2.0 ** -53, "fp32_rounding": 2.0 ** -24}


def run(psi, op, eps_step=0.0):
    out, s = [], 0
    for c in CHECKPOINTS:
        if eps_step == 0.0:
            psi = oracle.step(op, psi, s, c - s)
            s = c
        while s < c:
            psi = oracle.step(op, psi, s, 1)
            xi, _ = synth.normal_pairs(PSEED + s, psi.size)
            psi = psi * (1.0 + eps_step * xi.reshape(psi.shape))
            s += 1
        out.append(psi.copy())
    return out


def main():
    op = oracle.Params(dim=3, n=N, h=H, nu=NU, g=G, gdd=GDD, dt=DT, imag=False, kernel="dipolar3d")
    psi0 = synth.gaussian_state(N, H, WIDTHS, 0.01, SEED)
    xi, _ = synth.normal_pairs(PSEED, psi0.size)
    base = run(psi0, op)
    res = {"workload": "64^3, h=0.2, nu=(1,1,0.5), g=150, g_dd=60, dt=5e-4, real time, seed-9 Gaussian "
                       "(widths 0.8, 0.8, 0.4, 1% noise); perturbations: initial psi0 (1 + eps xi), xi from seed 77; "
                       "every_step psi (1 + eps xi_s) after step s, xi_s from seed 77 + s",
           "checkpoints": CHECKPOINTS,
           "norm_rel_drift": [float(np.sum(np.abs(b) ** 2) / np.sum(np.abs(psi0) ** 2) - 1) for b in base]}
    for name, eps in EPS.items():
        res[name] = {"eps": eps}
        for kind in ("initial", "every_step"):
            if kind == "initial":
                pert = run(psi0 * (1.0 + eps * xi.reshape(psi0.shape)), op)
            else:
                pert = run(psi0, op, eps)
            res[name][kind] = [float(np.linalg.norm(p - b) / np.linalg.norm(b)) for p, b in zip(pert, base)]
            print(name, kind, res[name][kind], flush=True)
    with open(os.path.join(HERE, "divergence_64.json"), "w") as f:
        json.dump(res, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
