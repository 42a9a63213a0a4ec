"""Benchmark: 3D split-step site-updates/s of the dipolar GP solver (FP64 and
FP32-bulk forms) and the fraction of the HBM roofline of the dominant kernel.

Workload (default): real-time 256^3 grid, spacing 0.1, cigar trap
V = (x^2 + y^2 + 0.25 z^2)/2, g_dd = 60, dt = 5e-4; the state is relaxed
towards the ground state at g = 200 by 400 imaginary-time steps (FP32 bulk,
dt = 2e-3, on the GPU, untimed; not converged) and g is quenched to 150 before
the timed steps.  One step = one full split step over
the grid (all passes).  Inputs are synthetic (seeded Gaussian + 1% noise).

`python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]`
prints one JSON line.  Under torchrun (N > 1) every rank runs an independent
replica (the single-grid step does not shard); value = all ranks' site updates
/ the slowest rank's time.  `--impl reference` times the FP64 CPU oracle on
the host cores instead (rank 0 only).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "real3d": dict(n=(256, 256, 256), h=(0.1, 0.1, 0.1), nu=(1.0, 1.0, 0.5), g_prep=200.0, g=150.0,
                   gdd=60.0, dt=5e-4, widths=(1.0, 1.0, 0.5), seed=2016, prep_steps=400,
                   desc="real3d 256^3, h=0.1, cigar nu=(1,1,0.5), g 200->150 quench, g_dd=60, dt=5e-4, "
                        "real time from a 400-step imaginary-time relaxation at g=200 (not converged)"),
    "large": dict(n=(512, 512, 256), h=(0.08, 0.08, 0.08), nu=(1.0, 1.0, 3.0), g_prep=None, g=500.0,
                  gdd=200.0, dt=2e-4, widths=(1.0, 1.0, 3.0), seed=2016, prep_steps=0,
                  desc="large real3d 512x512x256, h=0.08, pancake nu=(1,1,3), g=500, g_dd=200, "
                       "dt=2e-4, from a seeded Gaussian"),
    "batched2d": dict(n=None, desc="batched 2D: 512 independent XY problems, square grids from "
                      "{64,96,128,160,256,384,512}^2, h=0.2, nu_y in [0.5,2], g in [10,200], g_dd/g in "
                      "[0,0.8], quasi-2D kernel d=0.5, half imaginary / half real time, dt=1e-3, "
                      "FP32-bulk, one persistent kernel launch per call (seed 4640)"),
    "adjoint": dict(n=(128, 128, 128), h=(0.15, 0.15, 0.15), nu=(1.0, 1.0, 0.5), g=200.0, gdd=60.0,
                    dt=1e-3, widths=(1.0, 1.0, 0.5), seed=160104640, g_prep=None, prep_steps=0,
                    desc="adjoint real3d 128^3, h=0.15, FP32-bulk, dt=1e-3, 1000 steps, V(t)=V0(1+sum "
                         "c_m sin(m t)), c_m~U(-0.05,0.05); fidelity gradient w.r.t. c_1..c_8 and g, "
                         "checkpoint every 32 steps"),
    "xz2d": dict(n=(512, 512), h=(0.05, 0.05), nu=(1.0, 2.0), g_prep=200.0, g=150.0, gdd=60.0, dt=5e-4,
                 widths=(1.0, 2.0), seed=2017, prep_steps=200, kernel="quasi2d_xz", qd=0.5,
                 metric="2D XZ split-step site-updates/s (FP64 vs FP32-bulk) and % of HBM roofline",
                 desc="2D XZ plane 512x512, h=0.05, nu=(1,2), dipoles along z in the plane, quasi-2D "
                      "XZ kernel d=0.5, g 200->150 quench, g_dd=60, dt=5e-4, real time from the "
                      "200-step imaginary-time relaxation at g=200 (not converged)"),
    "imag256": dict(n=(256, 256, 256), h=(0.1, 0.1, 0.1), nu=(1.0, 1.0, 0.5), g_prep=None, g=200.0,
                    gdd=60.0, dt=2e-3, widths=(1.0, 1.0, 0.5), seed=2018, prep_steps=0, imag=True,
                    real_init=True,
                    metric="3D imaginary-time split-step site-updates/s (complex vs real state)",
                    desc="imag3d 256^3, h=0.1, cigar nu=(1,1,0.5), g=200, g_dd=60, imaginary dt=0.002, "
                         "from a real seeded Gaussian (ground-state search)"),
    "imag3d": dict(n=(32, 32, 32), h=(0.25, 0.25, 0.25), nu=(1.0, 1.0, 2.0), g_prep=None, g=50.0,
                   gdd=15.0, dt=2e-3, widths=(1.0, 1.0, 2.0), seed=1601, prep_steps=0, imag=True,
                   desc="imag3d 32^3, h=0.25, nu=(1,1,2), g=50, g_dd=15, imaginary dt=0.002"),
}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def fp64_peak():
    """FP64 arithmetic peak from unit counts and clocks: 152 SMs x 2 FP64
    FMA per SM per clock (ncu's sm__sass_thread_inst_executed_op_dfma_pred_on
    peak_sustained = 304 per clock for the GPU) x 2 flop x the maximum SM
    clock (MEASURED_PEAKS.json sm_max_mhz, else the nominal 2070 MHz)."""
    mhz = 2070.0
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mhz = float(json.load(f).get("sm_max_mhz", mhz))
    except Exception:
        pass
    return 152 * 2 * 2 * mhz * 1e6 / 1e12


def source_hash():
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1601_04640_gb300", "csrc")
    files = []
    for dp, _, fs in os.walk(d):
        files += [os.path.join(dp, f) for f in fs]
    for f in sorted(files):
        with open(f, "rb") as fh:
            h.update(os.path.relpath(f, d).encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, form, workload):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources (else None)."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get("%s/%s/%s" % (workload, form, kernel))
    if not e or e.get("source_hash") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons."""
    Q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def workload_config(wl, form, world=1):
    """The `config` dict of a 3D/2D step workload, the same on both arms."""
    n = wl["n"]
    sites = int(np.prod(n))
    fits = 16 * sites < (256 << 20)
    return {"workload": wl["desc"], "grid": list(n), "sites": sites, "form": form,
            "l2": ("inputs larger than L2: psi %d MB (FP64) / %d MB (FP32) vs 129 MB L2" % (
                16 * sites >> 20, 8 * sites >> 20)) if not fits else
                  "L2 flushed before every timed step (256 MB write outside the step's events); "
                  "the state (%.1f MB FP64) fits in L2" % (16 * sites / 2 ** 20),
            "parallelism": "replicas" if world > 1 else "single GPU",
            "prep_imag_steps": wl["prep_steps"] if wl.get("g_prep") is not None else 0}


def run_oracle_sample(wl, seconds=12.0, max_steps=3):
    """The FP64 oracle, as it stands, on a bounded sample of the workload."""
    import oracle
    from paper_1601_04640_gb300 import synth
    n = wl["n"]
    p = oracle.Params(dim=len(n), n=n, h=wl["h"], nu=wl["nu"], g=wl["g"], gdd=wl["gdd"], dt=wl["dt"],
                      imag=wl.get("imag", False), kernel=wl.get("kernel", "dipolar3d"), qd=wl.get("qd", 0.5))
    psi = synth.gaussian_state(n, wl["h"], wl["widths"], 0.01, wl["seed"])
    if wl.get("real_init"):
        psi = psi.real.astype(np.complex128)
    sites = int(np.prod(n))
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        psi = oracle.step(p, psi, steps, 1)
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": sites * steps / dt, "unit": "site-updates/s", "cores": oracle.threads(),
            "kind": "oracle", "sample": "%d full step(s) of the %s workload, FP64 C oracle" % (
                steps, "x".join(str(v) for v in n))}, steps, dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="real3d", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the cuFFT comparison step")
    ap.add_argument("--no-strang", action="store_true", help="skip the second-order splitting leg")
    ap.add_argument("--no-real-psi", action="store_true", help="skip the real-state leg (imaginary time)")
    ap.add_argument("--no-launch-cmp", action="store_true",
                    help="skip the graph-replay vs direct-launch comparison (states that fit in L2)")
    ap.add_argument("--cn", default="auto", choices=["auto", "serial", "chunked"],
                    help="Crank-Nicolson solve form of the FP64 form (auto: the library's default "
                         "for the grid size); the FP32 form always uses the chunk-parallel solve")
    ap.add_argument("--forms", default="both", choices=["both", "fp64", "fp32"],
                    help="precision forms to time (the first listed is the top-level line)")
    ap.add_argument("--prep-steps", type=int, default=None,
                    help="imaginary-time preparation steps (default: the workload's)")
    ap.add_argument("--problems", type=int, default=512,
                    help="batched2d: the first K problems of the seeded sweep (default: all 512; a smaller K "
                         "is a profiling case, not the workload)")
    args = ap.parse_args()
    args.steps_default = "--steps" not in " ".join(sys.argv[1:])
    wl = dict(WORKLOADS[args.workload])
    if args.prep_steps is not None:
        wl["prep_steps"] = args.prep_steps
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    n = wl["n"]
    sites = int(np.prod(n)) if n else 0
    dim = len(n) if n else 3
    metric = wl.get("metric", "3D split-step site-updates/s (FP64 vs FP32-bulk) and % of HBM roofline")

    if args.impl == "reference":
        if rank != 0:
            return
        if args.workload in ("batched2d", "adjoint"):
            print(json.dumps({"impl": "reference", "unavailable": "the oracle reference arm times the 3D step workloads only"}))
            return
        import oracle.build
        oracle.build.build()
        # the W warm-up steps (untimed; bounded at about 30 s of CPU time), then K timed steps
        W = 0
        if args.warmup > 0:
            _, W, _ = run_oracle_sample(wl, seconds=30.0, max_steps=args.warmup)
        cb, steps, dt = run_oracle_sample(wl, seconds=1e9, max_steps=max(1, args.steps))
        line = {"impl": "reference", "metric": metric, "value": cb["value"], "unit": "site-updates/s",
                "n_gpus": 0, "steps": steps, "warmup": W, "ms_per_step": 1e3 * dt / steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(wl, "fp64" if args.forms != "fp32" else "fp32_bulk"),
                "start": "seeded Gaussian of the workload (the oracle's cost per step does not depend on the "
                         "state; the GPU arm starts from its prepared state)",
                "cpu_baseline": {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")},
                "e2e": {"value": cb["value"], "unit": "site-updates/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_1601_04640_gb300 import build as gbuild
    from paper_1601_04640_gb300 import dgpe, shard, synth
    if args.workload == "batched2d":
        return bench_batched(args, wl, world, rank, local)
    if args.workload == "adjoint":
        return bench_adjoint(args, wl, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    gbuild.build()
    dgpe.load()
    stream = torch.cuda.Stream()
    hbm_peak, peak_kind = peaks()
    imag = wl.get("imag", False)

    # relaxation towards the ground state (imaginary time at g_prep), FP32-bulk
    psi0 = synth.gaussian_state(n, wl["h"], wl["widths"], 0.01, wl["seed"])
    if wl.get("real_init"):
        psi0 = psi0.real.astype(np.complex128)
    kcode = {"dipolar3d": dgpe.DGPE_KERNEL_DIPOLAR_3D, "quasi2d": dgpe.DGPE_KERNEL_QUASI2D_XY,
             "quasi2d_xz": dgpe.DGPE_KERNEL_QUASI2D_XZ}[wl.get("kernel", "dipolar3d")]
    qd = wl.get("qd", 0.5)
    prep = None
    if wl["g_prep"] is not None and wl["prep_steps"] > 0:
        with dgpe.Solver(dim, n, wl["h"], wl["nu"], wl["g_prep"], wl["gdd"], 2e-3, True, False,
                         kernel=kcode, qd=qd, stream=stream.cuda_stream) as s:
            s.set_psi(psi0)
            s.step(wl["prep_steps"])
            prep = s.observables()
            psi0 = s.get_psi()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    forms = {}
    order = {"both": (True, False), "fp64": (True,), "fp32": (False,)}[args.forms]
    # L2 is 129 MB: a state that fits is evicted before every timed step
    flush = None
    if 16 * sites < (256 << 20):
        flush = torch.zeros(64 << 20, dtype=torch.float32, device="cuda")
    for fp64 in order:
        name = "fp64" if fp64 else "fp32_bulk"
        S = dgpe.Solver(dim, n, wl["h"], wl["nu"], wl["g"], wl["gdd"], wl["dt"], imag, fp64, kernel=kcode, qd=qd,
                        stream=stream.cuda_stream, cn=None if (args.cn == "auto" or not fp64) else args.cn)
        S.set_psi(psi0)
        S.step(args.warmup)
        barrier()
        clk = Clocks(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        l0 = dgpe.dgpe_kernel_launches(S.h)
        if flush is None:
            e0.record(stream)
            S.step(args.steps)
            e1.record(stream)
        else:
            # the state fits in L2: every timed step starts after a 256 MB write
            # (outside its events) has evicted it
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            with torch.cuda.stream(stream):
                for a0, a1 in evs:
                    flush.add_(1.0)
                    a0.record(stream)
                    S.step(1)
                    a1.record(stream)
        launches = dgpe.dgpe_kernel_launches(S.h) - l0
        barrier()
        clocks = clk.stop()
        ms = e0.elapsed_time(e1) if flush is None else sum(a0.elapsed_time(a1) for a0, a1 in evs)
        ms_max = shard.max_over_ranks(ms)
        obs = S.observables()
        # per-pass durations (passes launched one by one, events between them)
        if flush is None:
            passes = dgpe.dgpe_profile_steps(S.h, max(3, args.steps // 2))
        else:
            # one profiled step per L2 flush, averaged
            runs = []
            for _ in range(max(3, min(args.steps, 20))):
                with torch.cuda.stream(stream):
                    flush.add_(1.0)
                runs.append(dgpe.dgpe_profile_steps(S.h, 1))
            passes = [(r0[0], sum(r[i][1] for r in runs) / len(runs), r0[2], r0[3])
                      for i, r0 in enumerate(runs[0])]
        tot = sum(p[1] for p in passes)
        top = max(passes, key=lambda p: p[1])
        achieved = top[2] / (top[1] * 1e-3) / 1e9
        roof = {"bound": "hbm", "kernel": top[0], "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                "traffic": ncu_traffic(top[0], name, args.workload),
                "algorithmic_bytes_per_launch": top[2], "ms_per_launch": top[1]}
        step_bytes = sum(p[2] for p in passes)
        step_flops = sum(p[3] for p in passes)
        roof_alu = None
        if fp64:
            # the FP64 form is limited by the FP64 pipe: its roofline is the
            # FP64 arithmetic peak (unit counts x clock)
            pk = fp64_peak()
            ach = top[3] / (top[1] * 1e-3) / 1e12
            roof_alu = {"bound": "alu", "kernel": top[0], "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                        "frac": ach / pk, "peak_kind": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x max SM clock",
                        "traffic": roof["traffic"], "algorithmic_flops_per_launch": top[3],
                        "ms_per_launch": top[1]}
        f = {"value": world * sites * args.steps / (ms_max * 1e-3), "ms_per_step": ms_max / args.steps,
             "dtype": "f64" if fp64 else "f32 (FP64 reductions/tables)",
             "roofline": roof_alu if roof_alu else roof,
             "roofline_hbm": roof,
             "step_hbm": {"algorithmic_bytes_per_step": step_bytes,
                          "achieved_GBps": step_bytes / (ms_max / args.steps * 1e-3) / 1e9,
                          "frac": step_bytes / (ms_max / args.steps * 1e-3) / 1e9 / hbm_peak},
             "step_flops": {"flops_per_step": step_flops,
                            "achieved_TFLOPs": step_flops / (ms_max / args.steps * 1e-3) / 1e12},
             "passes": [{"kernel": p[0], "ms": p[1], "share": p[1] / tot, "GBps": p[2] / (p[1] * 1e-3) / 1e9,
                         "TFLOPs": p[3] / (p[1] * 1e-3) / 1e12}
                        for p in passes],
             "gpu_launches": launches, "clocks": clocks,
             "observables_after": {"norm": obs["norm"], "mu": obs["mu"], "energy": obs["energy"]}}
        # end to end through the C ABI with host buffers: every step copies
        # the state in from pinned host memory and reads it back
        if not args.no_e2e:
            host_in = torch.from_numpy(psi0.view(np.float64).copy()).pin_memory()
            host_out = torch.empty_like(host_in).pin_memory()
            lib = dgpe.load()
            ke = max(2, min(args.steps, 10))
            for _ in range(2):
                dgpe._check(lib.dgpe_set_psi(S.h, host_in.data_ptr(), sites), S.h)
                S.step(1)
                dgpe._check(lib.dgpe_get_psi(S.h, host_out.data_ptr(), sites), S.h)
            barrier()
            t0 = time.perf_counter()
            for _ in range(ke):
                dgpe._check(lib.dgpe_set_psi(S.h, host_in.data_ptr(), sites), S.h)
                S.step(1)
                dgpe._check(lib.dgpe_get_psi(S.h, host_out.data_ptr(), sites), S.h)
            barrier()
            te = time.perf_counter() - t0
            f["e2e"] = {"value": world * sites * ke / shard.max_over_ranks(te), "unit": "site-updates/s",
                        "h2d_bytes_per_step": 16 * sites, "d2h_bytes_per_step": 16 * sites,
                        "steps": ke}
        S.close()
        forms[name] = f

    # launch-bound sizes (the state fits in L2): steps/s with the step replayed
    # as one CUDA graph against its kernels launched one by one, back to back
    # and with an L2 flush before every step
    launch_cmp = None
    if flush is not None and not args.no_launch_cmp:
        launch_cmp = {}
        for fp64 in order:
            name = "fp64" if fp64 else "fp32_bulk"
            row = {}
            for graph in (True, False):
                key = "graph" if graph else "direct"
                with dgpe.Solver(dim, n, wl["h"], wl["nu"], wl["g"], wl["gdd"], wl["dt"], imag, fp64, kernel=kcode,
                                 qd=qd, stream=stream.cuda_stream, graph=graph) as S4:
                    S4.set_psi(psi0)
                    S4.step(args.warmup)
                    barrier()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    S4.step(args.steps)
                    e1.record(stream)
                    barrier()
                    b2b = shard.max_over_ranks(e0.elapsed_time(e1)) / args.steps
                    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                           for _ in range(args.steps)]
                    with torch.cuda.stream(stream):
                        for a0, a1 in evs:
                            flush.add_(1.0)
                            a0.record(stream)
                            S4.step(1)
                            a1.record(stream)
                    barrier()
                    fl = shard.max_over_ranks(sum(a0.elapsed_time(a1) for a0, a1 in evs)) / args.steps
                row[key] = {"ms_per_step_back_to_back": b2b, "steps_per_s_back_to_back": 1e3 / b2b,
                            "ms_per_step_l2_flushed": fl, "steps_per_s_l2_flushed": 1e3 / fl}
            row["graph_speedup_back_to_back"] = row["direct"]["ms_per_step_back_to_back"] / row["graph"]["ms_per_step_back_to_back"]
            launch_cmp[name] = row

    # second-order (Strang) splitting on the same workload and state: one
    # dgpe_step(K) call runs K first-order steps between two exponential
    # passes over -dt/2 and +dt/2
    strang = None
    if not imag and not args.no_strang:
        if flush is not None:
            strang = {"unavailable": "timed on states larger than L2 only (one call of K steps)"}
        else:
            strang = {}
            for fp64 in order:
                name = "fp64" if fp64 else "fp32_bulk"
                with dgpe.Solver(dim, n, wl["h"], wl["nu"], wl["g"], wl["gdd"], wl["dt"], False, fp64,
                                 kernel=kcode, qd=qd, stream=stream.cuda_stream, split="strang",
                                 cn=None if (args.cn == "auto" or not fp64) else args.cn) as S2:
                    S2.set_psi(psi0)
                    S2.step(args.warmup)
                    barrier()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    l0 = dgpe.dgpe_kernel_launches(S2.h)
                    e0.record(stream)
                    S2.step(args.steps)
                    e1.record(stream)
                    barrier()
                    launches = dgpe.dgpe_kernel_launches(S2.h) - l0
                    ms = shard.max_over_ranks(e0.elapsed_time(e1))
                strang[name] = {"value": world * sites * args.steps / (ms * 1e-3),
                                "ms_per_step": ms / args.steps,
                                "time_vs_first_order": (ms / args.steps) / forms[name]["ms_per_step"],
                                "gpu_launches": launches}

    # imaginary time with a real state (half the bytes of psi), same workload;
    # the real state may fit in L2, so every timed step follows a 256 MB write
    real_state = None
    if imag and not args.no_real_psi:
        real_state = {"timing": "L2 flushed before every timed step (256 MB write outside the step's events)"}
        lib = dgpe.load()
        rs_flush = flush if flush is not None else torch.zeros(64 << 20, dtype=torch.float32, device="cuda")
        for fp64 in order:
            name = "fp64" if fp64 else "fp32_bulk"
            with dgpe.Solver(dim, n, wl["h"], wl["nu"], wl["g"], wl["gdd"], wl["dt"], True, fp64,
                             kernel=kcode, qd=qd, stream=stream.cuda_stream, real_psi=True) as S3:
                S3.set_psi(psi0.real.astype(np.complex128))
                S3.step(args.warmup)
                barrier()
                l0 = dgpe.dgpe_kernel_launches(S3.h)
                evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(args.steps)]
                with torch.cuda.stream(stream):
                    for a0, a1 in evs:
                        rs_flush.add_(1.0)
                        a0.record(stream)
                        S3.step(1)
                        a1.record(stream)
                barrier()
                ms = sum(a0.elapsed_time(a1) for a0, a1 in evs)
                launches = dgpe.dgpe_kernel_launches(S3.h) - l0
                ms = shard.max_over_ranks(ms)
                lps = dgpe.dgpe_launches_per_step(S3.h)
                sb = sum(lib.dgpe_pass_bytes(S3.h, i) for i in range(lps))
                o3 = S3.observables()
            real_state[name] = {"value": world * sites * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps,
                                "speedup_vs_complex": forms[name]["ms_per_step"] / (ms / args.steps),
                                "algorithmic_bytes_per_step": sb,
                                "achieved_GBps": sb / (ms / args.steps * 1e-3) / 1e9,
                                "gpu_launches": launches, "mu_after": o3["mu"]}

    # the paper's design (separate kernels + cuFFT R2C/C2R, one thread per CN
    # line), same workload and state, timed the same way: comparison only
    plain = None
    if not args.no_plain and not imag and dim == 3:
        try:
            from paper_1601_04640_gb300 import plain as pl
            gbuild.build_plain()
            plain = {}
            for fp64 in order:
                name = "fp64" if fp64 else "fp32"
                with pl.PlainSolver(3, n, wl["h"], wl["nu"], wl["g"], wl["gdd"], wl["dt"], fp64,
                                    stream=stream.cuda_stream) as P:
                    P.set_psi(psi0)
                    P.step(args.warmup)
                    barrier()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    P.step(args.steps)
                    e1.record(stream)
                    barrier()
                    ms = e0.elapsed_time(e1)
                plain[name] = {"value": world * sites * args.steps / (ms * 1e-3), "ms_per_step": ms / args.steps}
                ours = forms["fp64" if fp64 else "fp32_bulk"]
                plain[name]["fused_speedup"] = ours["value"] / plain[name]["value"]
        except Exception as ex:  # the comparison leg must not hide the main result
            plain = {"unavailable": str(ex)[:200]}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle.build
        oracle.build.build()
        run_oracle_sample(wl, seconds=0.0, max_steps=1)  # untimed warm-up step (thread pool, first touch)
        cpu, _, _ = run_oracle_sample(wl)
        # the paper's baseline is one CPU core: the same oracle on one thread
        import oracle
        allc = oracle.threads()
        oracle.set_threads(1)
        try:
            one, _, _ = run_oracle_sample(wl, seconds=15.0, max_steps=1)
        finally:
            oracle.set_threads(allc)
        cpu["single_core"] = {k: one[k] for k in ("value", "cores", "sample")}
    a = forms["fp64"] if "fp64" in forms else forms["fp32_bulk"]
    b = forms.get("fp32_bulk") if "fp64" in forms else None
    line = {
        "metric": metric, "value": a["value"], "unit": "site-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": a["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": a["dtype"],
        "data": "synthetic",
        "config": workload_config(wl, "fp64" if "fp64" in forms else "fp32_bulk", world),
        "prep": None if prep is None else {"imag_steps": wl["prep_steps"], "g": wl["g_prep"],
                                           "mu": prep["mu"]},
        "roofline": a["roofline"], "roofline_hbm": a["roofline_hbm"], "step_hbm": a["step_hbm"],
        "step_flops": a["step_flops"], "passes": a["passes"],
        "cpu_baseline": cpu, "e2e": a.get("e2e"),
        "gpu_launches": a["gpu_launches"],
        "clocks": a["clocks"], "observables_after": a["observables_after"],
        "fp32_bulk": b,
        "cufft_plain_step": plain,
        "strang_split": strang,
        "graph_vs_direct": launch_cmp,
        "real_state": real_state,
        "speedup_fp32_bulk_vs_fp64": (b["value"] / a["value"]) if b else None,
        "source_hash": source_hash(),
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def _peak_line(metric, value, unit, steps, warmup, ms, dtype, cfg, world, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg}
    line.update(extra)
    return line


def bench_batched(args, wl, world, rank, local):
    """512 independent 2D problems stepped by one persistent kernel launch.  With
    N ranks the sweep is partitioned by cost (shard.partition): each rank steps
    its share, the only exchange is a host-side gather of the results."""
    import torch
    from paper_1601_04640_gb300 import build as gbuild
    from paper_1601_04640_gb300 import dgpe, shard, synth
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    gbuild.build()
    stream = torch.cuda.Stream()
    sweep = synth.batched_problems(4640, 512)[:max(1, min(512, args.problems))]
    parts = shard.partition(sweep, world)
    mine = parts[rank]
    probs = [sweep[i] for i in mine]
    sweep_sites = sum(q["n"][0] * q["n"][1] for q in sweep)
    hbm_peak, peak_kind = peaks()
    states = []
    for q in probs:
        noise = 0.01 if q["imag"] else 0.0
        states.append(synth.gaussian_state(q["n"], q["h"], (1.0, q["nu"][1]), noise, q["seed"]))
    t0 = time.perf_counter()
    B = dgpe.Batch(probs, stream=stream.cuda_stream)
    t_create = time.perf_counter() - t0
    info = B.info()
    for i, st in enumerate(states):
        B.set_psi(i, st)
    B.step(args.warmup)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = Clocks(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    B.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    ms = shard.max_over_ranks(ms)
    sites = info["sites"]
    per_step = ms / args.steps
    gbs = info["bytes_per_step"] / (per_step * 1e-3) / 1e9
    sizes = {}
    for q in sweep:
        sizes[q["n"][0]] = sizes.get(q["n"][0], 0) + 1
    # end to end: every step copies all 512 states in from the host and back
    ke = 2
    t0 = time.perf_counter()
    for _ in range(ke):
        for i, st in enumerate(states):
            B.set_psi(i, st)
        B.step(1)
        outs = [B.get_psi(i) for i in range(len(probs))]
    te = time.perf_counter() - t0
    te = shard.max_over_ranks(te)
    mus = {}
    for j, i in enumerate(mine):
        mus[i] = B.observables(j)["mu"]
    obs0 = B.observables(0)
    B.close()
    # comparison: the same sweep as per-size-class batched kernels in one graph
    Bc = dgpe.Batch(probs, stream=stream.cuda_stream, classes=True)
    for i, st in enumerate(states):
        Bc.set_psi(i, st)
    Bc.step(args.warmup)
    torch.cuda.synchronize()
    c0 = torch.cuda.Event(enable_timing=True)
    c1 = torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    Bc.step(args.steps)
    c1.record(stream)
    torch.cuda.synchronize()
    per_class = {"ms_per_step": shard.max_over_ranks(c0.elapsed_time(c1)) / args.steps,
                 "launches_per_step": Bc.info()["launches_per_step"]}
    Bc.close()
    mus = shard.gather(mus)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle
        import oracle.build
        oracle.build.build()
        t0, done, steps = time.perf_counter(), 0, 0
        for i, q in enumerate(probs[:64]):
            op = oracle.Params(dim=2, n=q["n"], h=q["h"], nu=q["nu"], g=q["g"], gdd=q["gdd"], dt=q["dt"],
                               imag=q["imag"], kernel="quasi2d", qd=q["qd"])
            oracle.step(op, states[i], 0, 2)
            done += 2 * q["n"][0] * q["n"][1]
            if time.perf_counter() - t0 > 15:
                break
        dtc = time.perf_counter() - t0
        cpu = {"value": done / dtc, "unit": "site-updates/s", "cores": oracle.threads(), "kind": "oracle",
               "sample": "2 steps of each of the first %d problems of the sweep" % (i + 1)}
    line = _peak_line("2D batched split-step site-updates/s and % of HBM roofline",
                      sweep_sites * args.steps / (ms * 1e-3), "site-updates/s", args.steps, args.warmup,
                      per_step, "f32 (FP64 reductions/tables)",
                      {"workload": wl["desc"], "problems": len(sweep), "sites": sweep_sites, "sizes": sizes,
                       "classes": info["classes"], "l2": "inputs larger than L2 (%d MB of state)" % (8 * sites >> 20),
                       "parallelism": ("sweep partitioned by cost over %d GPUs (rank 0: %d problems, %d sites; "
                                       "imbalance %.3f); results gathered on the host" % (
                                           world, len(probs), sites, shard.imbalance(sweep, parts)))
                       if world > 1 else "single GPU",
                       "results_gathered": len(mus)},
                      world, scaling="strong" if world > 1 else "weak",
                      roofline={"bound": "hbm", "kernel": "whole batched step", "achieved": gbs,
                                "peak": hbm_peak, "unit": "GB/s", "frac": gbs / hbm_peak, "peak_kind": peak_kind,
                                "traffic": None, "algorithmic_bytes_per_step": info["bytes_per_step"]},
                      e2e={"value": sweep_sites * ke / te, "unit": "site-updates/s",
                           "h2d_bytes_per_step": 16 * sweep_sites, "d2h_bytes_per_step": 16 * sweep_sites},
                      gpu_launches=info["launches_per_step"], clocks=clocks, cpu_baseline=cpu,
                      create_s=t_create, observables_problem0={"mu": obs0["mu"], "norm": obs0["norm"]},
                      per_class_graph=per_class)
    print(json.dumps(line))


def bench_adjoint(args, wl, world, rank, local):
    """One fidelity + gradient evaluation (forward with checkpoints, reverse sweep)."""
    import torch
    from paper_1601_04640_gb300 import build as gbuild
    from paper_1601_04640_gb300 import dgpe, synth
    torch.cuda.set_device(local)
    gbuild.build()
    n, h = wl["n"], wl["h"]
    cm = list(synth.trap_modulation(wl["seed"], 8, 0.05))
    psi0 = synth.gaussian_state(n, h, wl["widths"], 0.01, 1)
    target = synth.gaussian_state(n, h, (1.1, 0.9, 0.5), 0.01, 2)
    K = 1000 if args.steps_default else args.steps  # the adjoint workload's 1000 steps unless --steps
    every = 32
    out = {}
    for fp64 in (False, True):
        if fp64 and K > 200:
            Kf = 200
        else:
            Kf = K
        with dgpe.Solver(3, n, h, wl["nu"], wl["g"], wl["gdd"], wl["dt"], False, fp64) as s:
            s.set_trap_modulation(cm)
            dgpe.dgpe_fidelity_gradient(s.h, psi0, target, 2 * every, every, len(cm))  # warm-up
            torch.cuda.synchronize()
            l0 = dgpe.dgpe_kernel_launches(s.h)
            t0 = time.perf_counter()
            F, dg, dc = dgpe.dgpe_fidelity_gradient(s.h, psi0, target, Kf, every, len(cm))
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            nl = dgpe.dgpe_kernel_launches(s.h) - l0
        sites = n[0] * n[1] * n[2]
        out["fp64" if fp64 else "fp32_bulk"] = {"steps": Kf, "seconds": dt, "value": sites * Kf / dt,
                                                 "F": F, "dF_dg": dg, "dF_dc": dc, "gpu_launches": nl}
    a = out["fp32_bulk"]
    line = _peak_line("adjoint: forward+reverse site-updates/s of one fidelity gradient", a["value"],
                      "site-updates/s", a["steps"], 1, 1e3 * a["seconds"] / a["steps"],
                      "f32 (FP64 reductions/tables)", {"workload": wl["desc"], "grid": list(n)}, 1,
                      forms=out, gpu_launches=a["gpu_launches"])
    print(json.dumps(line))


if __name__ == "__main__":
    main()
