"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances: relative L2 of psi <= 1e-10 for the FP64 form and <= 1e-5 for the
FP32-bulk form; mu and energy within 1e-11 (FP64) and 1e-6 (FP32-bulk),
relative.  Shorter runs are held to the same bounds (they are upper bounds;
the measured errors are printed)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1601_04640_gb300 import build as gbuild
from paper_1601_04640_gb300 import dgpe, synth

pytestmark = pytest.mark.gpu

TOL_PSI = {True: 1e-10, False: 1e-5}
GOLDEN_DIV = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "divergence_64.json")
DIV_FACTOR = 30.0
TOL_MU = {True: 1e-11, False: 1e-6}


@pytest.fixture(scope="session", autouse=True)
def _built():
    gbuild.build()
    oracle.load()


def rel_l2(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def make_case(dim, n, h, nu, g, gdd, dt, imag, kernel=None, seed=1601, noise=0.01, widths=None):
    kname = {None: "dipolar3d" if dim == 3 else "quasi2d", "none": "none", "xz": "quasi2d_xz"}[kernel]
    op = oracle.Params(dim=dim, n=n, h=h, nu=nu, g=g, gdd=gdd, dt=dt, imag=imag, kernel=kname, qd=0.5)
    kc = {None: None, "none": dgpe.DGPE_KERNEL_NONE, "xz": dgpe.DGPE_KERNEL_QUASI2D_XZ}[kernel]
    psi0 = synth.gaussian_state(n, h, widths or nu, noise, seed)
    return op, kc, psi0


def gpu_run(dim, n, h, nu, g, gdd, dt, imag, fp64, kc, psi0, steps, graph=True, cn=None):
    with dgpe.Solver(dim, n, h, nu, g, gdd, dt, imag, fp64, kernel=kc, graph=graph, cn=cn) as s:
        s.set_psi(psi0)
        s.step(steps)
        return s.get_psi(), s.observables()


CASES_3D = [
    ((32, 32, 32), (0.25, 0.25, 0.25), (1.0, 1.0, 2.0)),
    ((64, 32, 128), (0.2, 0.3, 0.1), (1.0, 1.3, 0.8)),
    ((96, 160, 48), (0.2, 0.15, 0.3), (1.0, 1.2, 1.5)),   # 3 * 2^k and 5 * 2^k lengths
]


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("case", range(len(CASES_3D)))
def test_dipolar_potential_3d(fp64, case):
    n, h, nu = CASES_3D[case]
    op, kc, psi0 = make_case(3, n, h, nu, 10, 5, 1e-3, False)
    with dgpe.Solver(3, n, h, nu, 10, 5, 1e-3, False, fp64) as s:
        s.set_psi(psi0)
        phi = s.dipolar_potential()
    ref = oracle.dipolar_potential(op, np.abs(psi0) ** 2)
    err = np.max(np.abs(phi - ref)) / np.max(np.abs(ref))
    print("phi rel max err", err)
    assert err < (1e-12 if fp64 else 2e-6)


@pytest.mark.parametrize("fp64", [True, False])
def test_dipolar_potential_quasi2d(fp64):
    n, h, nu = (64, 32), (0.2, 0.3), (1.0, 1.5)
    op, kc, psi0 = make_case(2, n, h, nu, 10, 5, 1e-3, False)
    with dgpe.Solver(2, n, h, nu, 10, 5, 1e-3, False, fp64) as s:
        s.set_psi(psi0)
        phi = s.dipolar_potential()
    ref = oracle.dipolar_potential(op, np.abs(psi0) ** 2)
    err = np.max(np.abs(phi - ref)) / np.max(np.abs(ref))
    print("phi rel max err", err)
    assert err < (1e-12 if fp64 else 2e-6)


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("case", range(len(CASES_3D)))
def test_step_parity_3d(fp64, imag, case):
    n, h, nu = CASES_3D[case]
    op, kc, psi0 = make_case(3, n, h, nu, 50.0, 15.0, 2e-3, imag)
    for steps in (1, 10):
        psi, obs = gpu_run(3, n, h, nu, 50.0, 15.0, 2e-3, imag, fp64, kc, psi0, steps)
        ref = oracle.step(op, psi0, 0, steps)
        e = rel_l2(psi, ref)
        print("steps", steps, "rel L2", e)
        assert e < TOL_PSI[fp64]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("case", range(len(CASES_3D)))
def test_step_parity_3d_line_serial_cn(imag, case):
    """FP64 form with the one-thread-per-line Thomas solve forced on small
    grids (it is the default from 8192 lines per axis)."""
    n, h, nu = CASES_3D[case]
    op, kc, psi0 = make_case(3, n, h, nu, 50.0, 15.0, 2e-3, imag)
    for steps in (1, 10):
        psi, obs = gpu_run(3, n, h, nu, 50.0, 15.0, 2e-3, imag, True, kc, psi0, steps, cn="serial")
        ref = oracle.step(op, psi0, 0, steps)
        e = rel_l2(psi, ref)
        print("steps", steps, "rel L2", e)
        assert e < TOL_PSI[True]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("n", [(64, 32), (96, 160)])
def test_step_parity_2d_line_serial_cn(imag, n):
    h, nu = (0.2, 0.3), (1.0, 1.5)
    op, kc, psi0 = make_case(2, n, h, nu, 80.0, 40.0, 1e-3, imag)
    psi, obs = gpu_run(2, n, h, nu, 80.0, 40.0, 1e-3, imag, True, kc, psi0, 10, cn="serial")
    ref = oracle.step(op, psi0, 0, 10)
    e = rel_l2(psi, ref)
    print("rel L2", e)
    assert e < TOL_PSI[True]


def test_cn_form_flags_checked():
    n, h, nu = (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)
    with pytest.raises(dgpe.DgpeError):
        dgpe.Solver(3, n, h, nu, 1, 1, 1e-3, True, False, cn="serial")  # FP32 form
    p = dgpe.make_params(3, n, h, nu, fp64=True)
    p.flags |= dgpe.DGPE_FLAG_CN_SERIAL | dgpe.DGPE_FLAG_CN_CHUNKED
    with pytest.raises(dgpe.DgpeError):
        dgpe.dgpe_create(p)
    # the line-serial form adds the CN_x pass
    with dgpe.Solver(3, n, h, nu, 1, 1, 1e-3, True, True, cn="serial") as a, \
            dgpe.Solver(3, n, h, nu, 1, 1, 1e-3, True, True, cn="chunked") as b:
        la = dgpe.load().dgpe_launches_per_step(a.h)
        lb = dgpe.load().dgpe_launches_per_step(b.h)
        assert la == lb + 1


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("n", [(64, 32), (96, 160), (384, 80), (512, 64)])
def test_step_parity_2d(fp64, imag, n):
    h, nu = (0.2, 0.3), (1.0, 1.5)
    op, kc, psi0 = make_case(2, n, h, nu, 80.0, 40.0, 1e-3, imag)
    psi, obs = gpu_run(2, n, h, nu, 80.0, 40.0, 1e-3, imag, fp64, kc, psi0, 10)
    ref = oracle.step(op, psi0, 0, 10)
    e = rel_l2(psi, ref)
    print("rel L2", e)
    assert e < TOL_PSI[fp64]


@pytest.mark.parametrize("form", ["fp64", "fp32", "fp64_serial"])
@pytest.mark.parametrize("imag", [True, False])
def test_cn_only(form, imag):
    """g = g_dd = 0, no trap: the exponential is the identity and the step is
    the three CN substeps alone (large dt so the solves are far from I)."""
    fp64 = form != "fp32"
    n, h = (32, 64, 32), (0.2, 0.15, 0.3)
    op, kc, psi0 = make_case(3, n, h, (0, 0, 0), 0, 0, 0.05, imag, kernel="none", noise=0.3,
                             widths=(1.0, 1.0, 1.0))
    psi, _ = gpu_run(3, n, h, (0, 0, 0), 0, 0, 0.05, imag, fp64, kc, psi0, 3,
                     cn="serial" if form == "fp64_serial" else None)
    ref = oracle.step(op, psi0, 0, 3)
    e = rel_l2(psi, ref)
    print("rel L2", e)
    assert e < TOL_PSI[fp64]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("dt", [0.01, 0.2, 2.0, 20.0])
def test_cn_only_scan_reach(imag, dt):
    """FP32 chunk-parallel CN substeps alone (g = g_dd = 0, no trap) over
    kt = dt / (4 h^2) = 0.0625 ... 125.  The scan across the chunks of a line
    runs only as many rounds as the whole-chunk products |alpha|^16 need: one
    neighbour at small kt (|alpha| ~ kt), every round at large kt (|alpha|
    near 1).  Each regime must agree with the oracle's Thomas solve, within
    a few FP32 ulps times the solve's condition number 1 + 4 kt (the
    imaginary-time substeps damp high modes by up to that factor and the norm
    restores them)."""
    n, h = (256, 64, 32), (0.2, 0.2, 0.2)
    kt = dt / (4 * 0.04)
    op, kc, psi0 = make_case(3, n, h, (0, 0, 0), 0, 0, dt, imag, kernel="none", noise=0.3,
                             widths=(2.0, 1.5, 1.0))
    psi, _ = gpu_run(3, n, h, (0, 0, 0), 0, 0, dt, imag, False, kc, psi0, 3)
    ref = oracle.step(op, psi0, 0, 3)
    e = rel_l2(psi, ref)
    tol = max(TOL_PSI[False], 4 * (1 + 4 * kt) * 2.0 ** -24)
    print("kt", kt, "rel L2", e, "tol", tol)
    assert e < tol


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("dim", [2, 3])
def test_observables_parity(fp64, dim):
    if dim == 3:
        n, h, nu = (32, 32, 64), (0.3, 0.3, 0.2), (1.0, 1.2, 2.0)
    else:
        n, h, nu = (64, 64), (0.2, 0.2), (1.0, 1.5)
    op, kc, psi0 = make_case(dim, n, h, nu, 60.0, 30.0, 1e-3, False, noise=0.05)
    with dgpe.Solver(dim, n, h, nu, 60.0, 30.0, 1e-3, False, fp64) as s:
        s.set_psi(psi0)
        o = s.observables()
    r = oracle.observables(op, psi0)
    tol = TOL_MU[fp64]
    for k in ("norm", "mu", "energy", "kin", "pot", "contact", "rms_r"):
        assert abs(o[k] - r[k]) <= tol * max(1.0, abs(r[k])), (k, o[k], r[k])
    assert abs(o["dipolar"] - r["dipolar"]) <= tol * max(1.0, abs(r["mu"]))
    for a in range(dim):
        assert abs(o["rms"][a] - r["rms"][a]) <= tol * r["rms"][a]


def test_imag3d_config_full_length():
    """32^3, h = 0.25, V = (x^2 + y^2 + 4 z^2)/2, g = 50, g_dd = 15,
    imaginary dt = 0.002, 500 steps from the noisy Gaussian, both forms."""
    n, h, nu = (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=50, gdd=15, dt=0.002, imag=True, kernel="dipolar3d")
    psi0 = synth.gaussian_state(n, h, (1.0, 1.0, 2.0), 0.01, 1601)
    ref = oracle.step(op, psi0, 0, 500)
    r = oracle.observables(op, ref, 500)
    for fp64 in (True, False):
        psi, o = gpu_run(3, n, h, nu, 50, 15, 0.002, True, fp64, None, psi0, 500)
        e = rel_l2(psi, ref)
        print("fp64" if fp64 else "fp32", "rel L2", e, "mu", o["mu"], r["mu"])
        assert e < TOL_PSI[fp64]
        assert abs(o["mu"] - r["mu"]) <= TOL_MU[fp64] * abs(r["mu"])
        assert abs(o["energy"] - r["energy"]) <= TOL_MU[fp64] * abs(r["energy"])


def test_real3d_256_short_parity():
    """256^3 real-time workload (h = 0.1, cigar trap, g = 150 after the quench,
    g_dd = 60, dt = 5e-4) from a Gaussian stand-in for the ground state:
    three steps against the oracle, both forms."""
    n, h, nu = (256, 256, 256), (0.1,) * 3, (1.0, 1.0, 0.5)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=150, gdd=60, dt=5e-4, imag=False, kernel="dipolar3d")
    psi0 = synth.gaussian_state(n, h, (0.6, 0.6, 0.3), 0.01, 2000)
    ref = oracle.step(op, psi0, 0, 3)
    for fp64, cn in ((True, None), (True, "chunked"), (False, None)):
        psi, o = gpu_run(3, n, h, nu, 150, 60, 5e-4, False, fp64, None, psi0, 3, cn=cn)
        e = rel_l2(psi, ref)
        print("fp64" if fp64 else "fp32", cn, "rel L2", e)
        assert e < TOL_PSI[fp64]


def test_large_512x512x256_short_parity():
    """The 512 x 512 x 256 pancake workload (h = 0.08, nu = (1, 1, 3), g = 500,
    g_dd = 200, dt = 2e-4) at full size from its seed-2016 Gaussian: two
    steps against the oracle, both forms."""
    n, h, nu = (512, 512, 256), (0.08,) * 3, (1.0, 1.0, 3.0)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=500, gdd=200, dt=2e-4, imag=False, kernel="dipolar3d")
    psi0 = synth.gaussian_state(n, h, nu, 0.01, 2016)
    ref = oracle.step(op, psi0, 0, 2)
    for fp64 in (True, False):
        psi, o = gpu_run(3, n, h, nu, 500, 200, 2e-4, False, fp64, None, psi0, 2)
        e = rel_l2(psi, ref)
        print("fp64" if fp64 else "fp32", "rel L2", e)
        assert e < TOL_PSI[fp64]
        del psi


@pytest.mark.parametrize("fp64", [True, False])
def test_real_time_norm_conserved(fp64):
    n, h, nu = (64, 64, 64), (0.2,) * 3, (1.0, 1.0, 0.5)
    psi0 = synth.gaussian_state(n, h, (1.0, 1.0, 0.5), 0.01, 7)
    with dgpe.Solver(3, n, h, nu, 150, 60, 5e-4, False, fp64) as s:
        s.set_psi(psi0)
        n0 = s.observables()["norm"]
        s.step(2000)
        n1 = s.observables()["norm"]
    print("norm drift", n1 / n0 - 1)
    assert abs(n1 / n0 - 1) < (1e-12 if fp64 else 1e-5)


def test_fp32_bulk_full_length_64_stable():
    """2000 real-time steps at 64^3 against the oracle: the FP32-bulk bound.
    g_dd = 20 keeps eps_dd = (4 pi/3) g_dd / g = 0.56 < 1 (dynamically stable),
    so rounding differences are not amplified exponentially."""
    n, h, nu = (64, 64, 64), (0.2,) * 3, (1.0, 1.0, 0.5)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=150, gdd=20, dt=5e-4, imag=False, kernel="dipolar3d")
    psi0 = synth.gaussian_state(n, h, (0.8, 0.8, 0.4), 0.01, 9)
    ref = oracle.step(op, psi0, 0, 2000)
    psi, o = gpu_run(3, n, h, nu, 150, 20, 5e-4, False, False, None, psi0, 2000)
    e = rel_l2(psi, ref)
    r = oracle.observables(op, ref, 2000)
    print("fp32 2000 steps rel L2", e, "mu", o["mu"], r["mu"])
    assert e < TOL_PSI[False]
    assert abs(o["mu"] - r["mu"]) <= TOL_MU[False] * abs(r["mu"])


def test_fp64_config_interactions_1000_steps():
    """1000 real-time steps at 64^3 with the 256^3 workload's g = 150,
    g_dd = 60, FP64 form against the oracle.  eps_dd = 1.68 makes this
    dynamics unstable: rounding differences grow ~1e7-fold over 2000 steps,
    so the FP64 bound is checked at 1000 steps (growth ~1e3)."""
    n, h, nu = (64, 64, 64), (0.2,) * 3, (1.0, 1.0, 0.5)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=150, gdd=60, dt=5e-4, imag=False, kernel="dipolar3d")
    psi0 = synth.gaussian_state(n, h, (0.8, 0.8, 0.4), 0.01, 9)
    ref = oracle.step(op, psi0, 0, 1000)
    psi, o = gpu_run(3, n, h, nu, 150, 60, 5e-4, False, True, None, psi0, 1000)
    e = rel_l2(psi, ref)
    print("fp64 1000 steps rel L2", e)
    assert e < TOL_PSI[True]


def test_unstable_workload_error_tracks_oracle_divergence():
    """The 256^3 workload's interactions (g = 150, g_dd = 60, eps_dd = 1.68,
    cigar trap) over its full 2000 steps at 64^3 (same box), both forms,
    against the oracle at every checkpoint of tests/golden/divergence_64.json.
    That file holds the oracle's own divergence when its state is perturbed
    by rounding-sized noise (2^-53 or 2^-24 relative per site) after every
    step, written by tests/golden/make_divergence.py.  Each form's error must
    stay within a factor DIV_FACTOR of the curve for its own rounding unit:
    the growth of the GPU error is the dynamics amplifying rounding, not the
    kernels.  The FP64 form also meets its 1e-10 bound at 1000 steps."""
    with open(GOLDEN_DIV) as f:
        gold = json.load(f)
    cps = gold["checkpoints"]
    n, h, nu = (64, 64, 64), (0.2,) * 3, (1.0, 1.0, 0.5)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=150, gdd=60, dt=5e-4, imag=False, kernel="dipolar3d")
    psi0 = synth.gaussian_state(n, h, (0.8, 0.8, 0.4), 0.01, 9)
    refs, psi, s0 = [], psi0, 0
    for c in cps:
        psi = oracle.step(op, psi, s0, c - s0)
        refs.append(psi)
        s0 = c
    for fp64 in (True, False):
        curve = gold["fp64_rounding" if fp64 else "fp32_rounding"]["every_step"]
        errs = []
        with dgpe.Solver(3, n, h, nu, 150, 60, 5e-4, False, fp64) as s:
            s.set_psi(psi0)
            s0 = 0
            for c in cps:
                s.step(c - s0)
                s0 = c
                errs.append(rel_l2(s.get_psi(), refs[len(errs)]))
        for c, e, d in zip(cps, errs, curve):
            print("fp64" if fp64 else "fp32", "step", c, "rel L2", e, "oracle divergence", d, "ratio", e / d)
        for e, d in zip(errs, curve):
            assert e <= DIV_FACTOR * d
        if fp64:
            assert errs[cps.index(1000)] < TOL_PSI[True]


@pytest.mark.parametrize("fp64", [True, False])
def test_graph_and_direct_launch_identical(fp64):
    n, h, nu = (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)
    op, kc, psi0 = make_case(3, n, h, nu, 50.0, 15.0, 2e-3, True)
    a, _ = gpu_run(3, n, h, nu, 50.0, 15.0, 2e-3, True, fp64, kc, psi0, 5, graph=True)
    b, _ = gpu_run(3, n, h, nu, 50.0, 15.0, 2e-3, True, fp64, kc, psi0, 5, graph=False)
    assert np.array_equal(a, b)


def test_quench_mode_switch_modulation_time():
    """set_g, set_mode, a trap modulation and the step counter against the
    oracle's V(t) = V0 (1 + sum_m c_m sin(m t_n)), t_n = n dt."""
    n, h, nu = (32, 32, 32), (0.3,) * 3, (1.0, 1.0, 1.5)
    cm = list(synth.trap_modulation(160104640, 8, 0.05))
    psi0 = synth.gaussian_state(n, h, nu, 0.01, 4)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=60, gdd=20, dt=0.01, imag=True, kernel="dipolar3d")
    ref = oracle.step(op, psi0, 0, 5)
    op.imag = False
    op.g = 45.0
    op.cm = cm
    ref = oracle.step(op, ref, 5, 7)
    with dgpe.Solver(3, n, h, nu, 60, 20, 0.01, True, True) as s:
        s.set_psi(psi0)
        s.step(5)
        s.set_mode(False)
        s.set_g(45.0)
        s.set_trap_modulation(cm)
        assert s.time() == 5
        s.step(7)
        assert s.time() == 12
        psi = s.get_psi()
        o = s.observables()
    e = rel_l2(psi, ref)
    print("rel L2", e)
    assert e < TOL_PSI[True]
    r = oracle.observables(op, ref, 12)
    assert abs(o["mu"] - r["mu"]) <= 1e-11 * abs(r["mu"])
    assert abs(o["t"] - 0.12) < 1e-15


def test_nonfinite_state_reported():
    n, h, nu = (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)
    psi0 = synth.gaussian_state(n, h, nu, 0.0)
    psi0[3, 4, 5] = np.nan
    with dgpe.Solver(3, n, h, nu, 10, 5, 1e-3, True, True) as s:
        s.set_psi(psi0)
        with pytest.raises(dgpe.DgpeError) as e:
            s.observables()
        assert e.value.code == dgpe.DGPE_ENONFINITE


def test_device_pointer_roundtrip():
    torch = pytest.importorskip("torch")
    n, h, nu = (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)
    psi0 = synth.gaussian_state(n, h, nu, 0.01, 5)
    for fp64 in (True, False):
        with dgpe.Solver(3, n, h, nu, 10, 5, 1e-3, False, fp64) as s:
            t = torch.from_numpy(psi0).to("cuda")
            dgpe.dgpe_set_psi_device(s.h, t.data_ptr(), t.numel(), True)
            out = torch.empty_like(t)
            dgpe.dgpe_get_psi_device(s.h, out.data_ptr(), out.numel(), True)
            s.sync()
            assert np.max(np.abs(out.cpu().numpy() - psi0)) <= (0 if fp64 else 1e-7)
            host = s.get_psi()
            assert np.array_equal(host, out.cpu().numpy())


def test_launch_counter_and_operation_model():
    """dgpe_kernel_launches counts a graph replay as the step's kernels and the
    observables' own kernels; dgpe_pass_flops gives the line-serial Thomas
    solve 28 flops per site in real time (FP64)."""
    n, h, nu = (64, 64, 64), (0.2,) * 3, (1.0, 1.0, 0.5)
    with dgpe.Solver(3, n, h, nu, 10, 5, 1e-3, False, True, cn="serial") as s:
        s.set_psi(synth.gaussian_state(n, h, (1.0, 1.0, 0.5), 0.01, 3))
        lps = dgpe.dgpe_launches_per_step(s.h)
        l0 = dgpe.dgpe_kernel_launches(s.h)
        s.step(3)
        assert dgpe.dgpe_kernel_launches(s.h) - l0 == 3 * lps
        l1 = dgpe.dgpe_kernel_launches(s.h)
        s.observables()
        assert dgpe.dgpe_kernel_launches(s.h) - l1 >= 2
        lib = dgpe.load()
        names = [lib.dgpe_pass_name(s.h, i).decode() for i in range(lps)]
        flops = [lib.dgpe_pass_flops(s.h, i) for i in range(lps)]
        assert names[-3:] == ["cn_x", "cn_y", "cn_z"]
        for f in flops[-3:]:
            assert f == 28.0 * 64 ** 3
        assert all(f > 0 for f in flops)


def test_dipolar_potential_quasi2d_xz():
    """XZ plane (second axis z), dipoles along z in the plane."""
    n, h, nu = (96, 64), (0.2, 0.25), (1.0, 1.5)
    psi0 = synth.gaussian_state(n, h, (1.0, 1.5), 0.05, 11)
    op = oracle.Params(dim=2, n=n, h=h, nu=nu, kernel="quasi2d_xz", qd=0.5)
    ref = oracle.dipolar_potential(op, np.abs(psi0) ** 2)
    for fp64, tol in ((True, 1e-12), (False, 1e-5)):
        with dgpe.Solver(2, n, h, nu, 10, 5, 1e-3, False, fp64, kernel=dgpe.DGPE_KERNEL_QUASI2D_XZ) as s:
            s.set_psi(psi0)
            phi = s.dipolar_potential()
        e = rel_l2(phi, ref)
        print("fp64" if fp64 else "fp32", "Phi rel L2", e)
        assert e < tol


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("n", [(64, 96), (128, 64), (160, 160)])
def test_step_parity_2d_xz(fp64, imag, n):
    h, nu = (0.2, 0.25), (1.0, 1.5)
    op, kc, psi0 = make_case(2, n, h, nu, 80.0, 40.0, 1e-3, imag, kernel="xz")
    psi, obs = gpu_run(2, n, h, nu, 80.0, 40.0, 1e-3, imag, fp64, kc, psi0, 10)
    ref = oracle.step(op, psi0, 0, 10)
    e = rel_l2(psi, ref)
    r = oracle.observables(op, ref, 10)
    print("rel L2", e, "mu", obs["mu"], r["mu"])
    assert e < TOL_PSI[fp64]
    assert abs(obs["mu"] - r["mu"]) <= TOL_MU[fp64] * abs(r["mu"])


def test_step_parity_contact_only_line_serial_cn():
    """No dipolar term with the separate line-serial CN_x pass: the x-line pass
    then applies the exponential without a C2R in front of it."""
    for dim, n, h, nu in ((3, (32, 48, 40), (0.25, 0.2, 0.22), (1.0, 1.3, 0.9)),
                          (2, (64, 96), (0.2, 0.15), (1.0, 1.4))):
        for imag in (True, False):
            op, kc, psi0 = make_case(dim, n, h, nu, 60.0, 0.0, 2e-3, imag, kernel="none")
            psi, obs = gpu_run(dim, n, h, nu, 60.0, 0.0, 2e-3, imag, True, kc, psi0, 10, cn="serial")
            ref = oracle.step(op, psi0, 0, 10)
            e = rel_l2(psi, ref)
            print(dim, "imag" if imag else "real", "rel L2", e)
            assert e < TOL_PSI[True]


# (dim, n, h, nu, fp64, kernel, cn, graph)
STRANG_CASES = [
    (3, (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0), True, None, None, True),
    (3, (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0), False, None, None, True),
    (3, (64, 32, 128), (0.2, 0.3, 0.1), (1.0, 1.3, 0.8), True, None, "serial", True),
    (3, (96, 160, 48), (0.2, 0.15, 0.3), (1.0, 1.2, 1.5), False, None, None, False),
    (3, (32, 48, 40), (0.25, 0.2, 0.22), (1.0, 1.3, 0.9), True, "none", "serial", True),
    (2, (64, 32), (0.2, 0.3), (1.0, 1.5), True, None, None, True),
    (2, (96, 64), (0.2, 0.25), (1.0, 1.5), False, "xz", None, True),
]


@pytest.mark.parametrize("case", range(len(STRANG_CASES)))
def test_step_parity_strang(case):
    """Second-order splitting: dgpe_step runs n first-order steps between
    exponential passes over -dt/2 and +dt/2; the oracle takes n literal
    E(dt/2, t_k+1) C E(dt/2, t_k) steps.  Two calls (3 + 4 steps), modulated
    trap; the first-order result differs from both by more than ten times
    the tolerance and a hundred times the measured error."""
    dim, n, h, nu, fp64, kernel, cn, graph = STRANG_CASES[case]
    g, gdd, dt, cm = 50.0, (0.0 if kernel == "none" else 15.0), 2e-3, [0.5, 0.0, 0.3]
    op, kc, psi0 = make_case(dim, n, h, nu, g, gdd, dt, False, kernel=kernel)
    op.cm = cm
    with dgpe.Solver(dim, n, h, nu, g, gdd, dt, False, fp64, kernel=kc, cn=cn, graph=graph,
                     split="strang") as s:
        s.set_psi(psi0)
        s.set_trap_modulation(cm)
        s.step(3)
        s.step(0)
        s.step(4)
        psi = s.get_psi()
        assert s.time() == 7
    ref = oracle.step(op, psi0, 0, 7, split="strang")
    e = rel_l2(psi, ref)
    d = rel_l2(oracle.step(op, psi0, 0, 7), ref)
    print("rel L2", e, "first-order vs second-order", d)
    assert e < TOL_PSI[fp64]
    assert d > 10 * TOL_PSI[fp64] and d > 100 * e


def test_strang_launches_and_refusals():
    n, h, nu = (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)
    with dgpe.Solver(3, n, h, nu, 10, 5, 1e-3, False, True, split="strang") as s:
        s.set_psi(synth.gaussian_state(n, h, nu, 0.01, 5))
        lps = dgpe.dgpe_launches_per_step(s.h)
        l0 = dgpe.dgpe_kernel_launches(s.h)
        s.step(0)
        assert dgpe.dgpe_kernel_launches(s.h) == l0
        s.step(3)
        # two exponential passes, each after the four passes of the dipolar chain
        assert dgpe.dgpe_kernel_launches(s.h) - l0 == 3 * lps + 2 * 5
        with pytest.raises(dgpe.DgpeError) as e:
            s.set_mode(True)
        assert e.value.code == dgpe.DGPE_EUNSUPPORTED
        import torch
        a = torch.zeros(32 ** 3, dtype=torch.complex128, device="cuda")
        b = torch.zeros_like(a)
        with pytest.raises(dgpe.DgpeError) as e:
            dgpe.dgpe_step_adjoint(s.h, a.data_ptr(), b.data_ptr(), 0)
        assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.Solver(3, n, h, nu, 10, 5, 1e-3, True, True, split="strang")
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    q = dict(n=(64, 64), h=(0.2, 0.2), nu=(1.0, 1.0), g=10.0, gdd=5.0, dt=1e-3, imag=False,
             split="strang")
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.Batch([q])
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED


# (dim, n, h, nu, fp64, kernel)
REAL_STATE_CASES = [
    (3, (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0), True, None),
    (3, (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0), False, None),
    (3, (64, 32, 128), (0.2, 0.3, 0.1), (1.0, 1.3, 0.8), True, None),
    (3, (96, 160, 48), (0.2, 0.15, 0.3), (1.0, 1.2, 1.5), False, None),
    (3, (160, 48, 40), (0.15, 0.3, 0.3), (1.0, 1.4, 1.2), True, "none"),
    (2, (64, 32), (0.2, 0.3), (1.0, 1.5), True, None),
    (2, (96, 64), (0.2, 0.25), (1.0, 1.5), False, "xz"),
    (2, (384, 96), (0.05, 0.2), (1.0, 1.5), False, None),
]


@pytest.mark.parametrize("case", range(len(REAL_STATE_CASES)))
def test_step_parity_real_state(case):
    """Real state in imaginary time (nx reals per row; rows paired into the
    complex lines of the x-line pass, columns paired by the strided CN passes)
    against the oracle's complex step on the same real input, with a
    modulated trap; the state read back is real; mu and E of the result."""
    dim, n, h, nu, fp64, kernel = REAL_STATE_CASES[case]
    g, gdd, dt, cm = 50.0, (0.0 if kernel == "none" else 15.0), 2e-3, [0.3]
    op, kc, psi0 = make_case(dim, n, h, nu, g, gdd, dt, True, kernel=kernel, noise=0.05)
    psi0 = psi0.real.astype(np.complex128)
    op.cm = cm
    with dgpe.Solver(dim, n, h, nu, g, gdd, dt, True, fp64, kernel=kc, real_psi=True) as s:
        s.set_psi(psi0)
        s.set_trap_modulation(cm)
        s.step(4)
        s.step(6)
        psi = s.get_psi()
        o = s.observables()
        assert s.time() == 10
    ref = oracle.step(op, psi0, 0, 10)
    r = oracle.observables(op, ref, 10)
    e = rel_l2(psi, ref)
    print("rel L2", e, "mu", o["mu"], r["mu"])
    assert np.all(psi.imag == 0.0)
    assert e < TOL_PSI[fp64]
    for k in ("norm", "mu", "energy"):
        assert abs(o[k] - r[k]) <= TOL_MU[fp64] * max(1.0, abs(r[k])), (k, o[k], r[k])


def test_real_state_bytes_potential_and_refusals():
    n, h, nu = (64, 32, 48), (0.2, 0.3, 0.25), (1.0, 1.3, 0.9)
    psi0 = synth.gaussian_state(n, h, nu, 0.05, 21).real.astype(np.complex128)
    op = oracle.Params(dim=3, n=n, h=h, nu=nu, g=30, gdd=12, dt=1e-3, imag=True, kernel="dipolar3d")
    ref = oracle.dipolar_potential(op, np.abs(psi0) ** 2)
    lib = dgpe.load()
    with dgpe.Solver(3, n, h, nu, 30, 12, 1e-3, True, True, cn="chunked") as c, \
            dgpe.Solver(3, n, h, nu, 30, 12, 1e-3, True, True, real_psi=True) as s:
        s.set_psi(psi0)
        phi = s.dipolar_potential()
        assert np.max(np.abs(phi - ref)) / np.max(np.abs(ref)) < 1e-12
        lps = dgpe.dgpe_launches_per_step(s.h)
        assert lps == dgpe.dgpe_launches_per_step(c.h)
        names = [lib.dgpe_pass_name(s.h, i).decode() for i in range(lps)]
        bs = [lib.dgpe_pass_bytes(s.h, i) for i in range(lps)]
        bc = [lib.dgpe_pass_bytes(c.h, i) for i in range(lps)]
        sites = 64 * 32 * 48
        for name, a, b in zip(names, bs, bc):
            if name in ("cn_y", "cn_z"):
                assert a == 2 * 8 * sites and b == 2 * 16 * sites
            if name == "c2r_x_exp_cn_x":
                assert b - a == 2 * 8 * sites
        with pytest.raises(dgpe.DgpeError) as e:
            s.set_mode(False)
        assert e.value.code == dgpe.DGPE_EUNSUPPORTED
    q = dict(n=(64, 64), h=(0.2, 0.2), nu=(1.0, 1.0), g=10.0, gdd=5.0, dt=1e-3, imag=True,
             real_psi=True)
    with pytest.raises(dgpe.DgpeError) as e:
        dgpe.Batch([q])
    assert e.value.code == dgpe.DGPE_EUNSUPPORTED


ASYM_N, ASYM_H, ASYM_NU = (128, 128), (0.05, 0.05), (1.0, 1.5)


@pytest.mark.parametrize("fp64", [True, False])
@pytest.mark.parametrize("kernel", [None, "xz"])
def test_parity_2d_asymptotic_kernel_region(fp64, kernel):
    """128^2 at h = 0.05 with d = 0.5 (XY and XZ kernels): the corner of the
    k-grid has u = k d / sqrt(2) = 31.4, so about 9 % of the U(k) table comes
    from erfcx's asymptotic series (u >= 25).  With 5 % noise on the state the
    density has weight there: a sign error in the series' 1/q^2 term moves
    Phi_d by 1.4e-4 in relative L2, a 1e-6 relative error of U there by
    3.4e-8 (measured on the oracle's table).  Phi_d, then 10 steps of each
    mode, against the oracle."""
    n, h, nu = ASYM_N, ASYM_H, ASYM_NU
    assert math.hypot(math.pi / h[0], math.pi / h[1]) * 0.5 / math.sqrt(2) > 25
    kname = "quasi2d" if kernel is None else "quasi2d_xz"
    kc = None if kernel is None else dgpe.DGPE_KERNEL_QUASI2D_XZ
    psi0 = synth.gaussian_state(n, h, nu, 0.05, 11)
    op = oracle.Params(dim=2, n=n, h=h, nu=nu, kernel=kname, qd=0.5)
    with dgpe.Solver(2, n, h, nu, 10, 5, 1e-3, False, fp64, kernel=kc) as s:
        s.set_psi(psi0)
        phi = s.dipolar_potential()
    ref = oracle.dipolar_potential(op, np.abs(psi0) ** 2)
    e = rel_l2(phi, ref)
    print("Phi rel L2", e)
    assert e < (1e-12 if fp64 else 1e-5)
    for imag in (True, False):
        op, kc2, psi0 = make_case(2, n, h, nu, 80.0, 40.0, 1e-3, imag, kernel=kernel, noise=0.05, seed=12)
        psi, obs = gpu_run(2, n, h, nu, 80.0, 40.0, 1e-3, imag, fp64, kc2, psi0, 10)
        ref = oracle.step(op, psi0, 0, 10)
        e = rel_l2(psi, ref)
        r = oracle.observables(op, ref, 10)
        print("imag" if imag else "real", "rel L2", e, "mu", obs["mu"], r["mu"])
        assert e < TOL_PSI[fp64]
        assert abs(obs["mu"] - r["mu"]) <= TOL_MU[fp64] * abs(r["mu"])


# (dim, n, h, nu): power-of-two nx (the pipelined FP32 x-line pass); the 2D
# cases leave a ragged last tile (nrows not a multiple of the tile's rows)
P1_PIPE_CASES = [
    (3, (32, 32, 32), (0.25,) * 3, (1.0, 1.0, 2.0)),
    (3, (256, 40, 96), (0.05, 0.3, 0.15), (1.0, 1.2, 0.8)),
    (3, (512, 32, 40), (0.03, 0.3, 0.3), (1.0, 1.3, 1.1)),
    (2, (64, 40), (0.2, 0.3), (1.0, 1.5)),
    (2, (64, 96), (0.2, 0.3), (1.0, 1.5)),
    (2, (128, 160), (0.1, 0.15), (1.0, 1.2)),
]


@pytest.mark.parametrize("imag", [True, False])
@pytest.mark.parametrize("case", range(len(P1_PIPE_CASES)))
def test_p1_pipelined_matches_oneshot_and_oracle(imag, case):
    """FP32 bulk: the persistent, bulk-copy-fed x-line pass (the default) and
    the one-CTA-per-tile pass (DGPE_FLAG_P1_ONESHOT) compute the same
    arithmetic; both against the oracle over 6 steps, and the contact-only
    case (no C2R in front of the exponential)."""
    dim, n, h, nu = P1_PIPE_CASES[case]
    for kernel, gdd in ((None, 40.0), ("none", 0.0)):
        op, kc, psi0 = make_case(dim, n, h, nu, 80.0, gdd, 1e-3, imag, kernel=kernel)
        outs = []
        for flags in (0, dgpe.DGPE_FLAG_P1_ONESHOT):
            with dgpe.Solver(dim, n, h, nu, 80.0, gdd, 1e-3, imag, False, kernel=kc, flags=flags) as s:
                s.set_psi(psi0)
                s.step(6)
                outs.append(s.get_psi())
                o = s.observables()
        ref = oracle.step(op, psi0, 0, 6)
        e0, e1 = rel_l2(outs[0], ref), rel_l2(outs[1], ref)
        d = rel_l2(outs[0], outs[1])
        print(kernel, "pipelined", e0, "one-shot", e1, "between", d)
        assert e0 < TOL_PSI[False] and e1 < TOL_PSI[False]
        assert d < 1e-6


TMA_CASES = [
    (3, (64, 512, 32), (0.2, 0.05, 0.3), (1.0, 1.0, 1.5)),
    (3, (32, 64, 512), (0.3, 0.2, 0.04), (1.0, 1.2, 0.7)),
    (3, (96, 64, 64), (0.2, 0.25, 0.25), (1.0, 1.1, 1.3)),
    (2, (64, 512), (0.2, 0.05), (1.0, 1.4)),
]


@pytest.mark.parametrize("case", range(len(TMA_CASES)))
def test_tensor_map_transforms_match_register_fed_and_oracle(case):
    """FP32 bulk, power-of-two y and z lines: the strided transforms fed by
    tensor-map tiles (the default; the 3D z-pass evaluates U(k)) against the
    register-fed kernels with the U table (DGPE_FLAG_P1_ONESHOT) and against
    the oracle, for Phi_d and for 4 real-time steps.  The cases take 512-point
    lines (two boxes per tile, 8-column tiles) along y and along z, a spectrum
    width that leaves a ragged last tile (nx = 96: 49 columns in tiles of 16),
    and the 2D y-pass FFT_y.U.IFFT_y."""
    dim, n, h, nu = TMA_CASES[case]
    op, kc, psi0 = make_case(dim, n, h, nu, 60.0, 30.0, 1e-3, False)
    phis, outs = [], []
    for flags in (0, dgpe.DGPE_FLAG_P1_ONESHOT):
        with dgpe.Solver(dim, n, h, nu, 60.0, 30.0, 1e-3, False, False, kernel=kc, flags=flags) as s:
            s.set_psi(psi0)
            phis.append(s.dipolar_potential())
            s.step(4)
            outs.append(s.get_psi())
    # the oracle sees the state the FP32 form holds (psi rounded once)
    dens = np.abs(psi0.astype(np.complex64).astype(np.complex128)) ** 2
    phi_ref = oracle.dipolar_potential(op, dens)
    scale = np.max(np.abs(phi_ref))
    ep = [np.max(np.abs(ph - phi_ref)) / scale for ph in phis]
    dp = np.max(np.abs(phis[0] - phis[1])) / scale
    ref = oracle.step(op, psi0, 0, 4)
    e0, e1 = rel_l2(outs[0], ref), rel_l2(outs[1], ref)
    d = rel_l2(outs[0], outs[1])
    print("Phi_d vs oracle", ep, "between", dp, "| psi vs oracle", e0, e1, "between", d)
    assert max(ep) < 1e-5 and dp < 2e-6
    assert e0 < TOL_PSI[False] and e1 < TOL_PSI[False]
    assert d < 1e-6
