#!/usr/bin/env python3
"""Throughput benchmark of the GB300 FCN z-step (Nr*Nt*z-steps per second).

Workload (ours): the filamentation-regime grid Nr = 1024, Nt = 4096 (w0 = 2 mm,
tp = 50 fs, 5 P_cr, n2 + n4, 1 % seeded amplitude noise, dz = 2 mm), run in the
FP32-mixed precision form.  Each GPU advances a batch of independent pulses
of that grid (noise seeds rank*B .. rank*B+B-1), so that the field (B x 33.5 MB)
is larger than the 129 MB L2 between timed steps.  One bench step is one
z-step of the whole batch: Strang step = nonlinear half step, FFT along tau,
Crank-Nicolson column solve, inverse FFT, nonlinear half step.

Also reported on the same line: the kernel roofline of the dominant kernel
(CUDA-event durations of a profiled replay of the timed steps), the
end-to-end figure through the C-ABI with host buffers, the plain FP64 path on
the same batch, the FP32-vs-FP64 field difference after the full 1000-step
run of one pulse, SM clocks sampled during the timed region, the FP64
CPU oracle timed on a bounded sample (rank 0, N = 1), and the Cartesian
(3D+1) grid: config 1's pulse on 255 x 255 x 256 nodes, 200 steps of 1 cm,
FP32-mixed against FP64, with its own kernel fractions and roofline.

--impl reference times that oracle (the deliberately slow CPU program the
CUDA path is checked against) on the same metric.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Nr*Nt*z-steps/sec on 1 GB300, chosen form vs plain FP64 FCN at <=1e-4 rel-L2"
UNIT = "point-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--pulses", type=int, default=8, help="pulses per GPU")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-cfg4", action="store_true")
    ap.add_argument("--cfg4-steps", type=int, default=500)
    ap.add_argument("--no-cartesian", action="store_true")
    ap.add_argument("--no-chosen", action="store_true", help="skip the adaptive chosen-form leg")
    ap.add_argument("--chosen-z", type=float, default=1.0, help="metres of the chosen-form leg")
    ap.add_argument("--oracle-scaling", action="store_true",
                    help="only run the oracle's thread-scaling table on the paper's grid (CPU)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (copy, burst)"
    return 6800.0, "fallback 6.8 TB/s"


class ClockSampler:
    """nvidia-smi clocks sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def reduce_max(x: float, pg, device) -> float:
    """Maximum of x over the ranks of process group pg (x itself if None)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(world: int, points_per_rank: int, steps: int, t_max_ms: float) -> float:
    """Whole-job throughput: every rank advances points_per_rank points by
    steps z-steps; the job takes as long as the slowest rank."""
    return world * points_per_rank * steps / (t_max_ms * 1e-3)


def rel_l2(a, b):
    import numpy as np
    return float(np.sqrt(np.sum(np.abs(a - b) ** 2) / np.sum(np.abs(b) ** 2)))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_sample(wl, budget_s=15.0):
    """Times the FP64 CPU oracle on one pulse of the bench grid: the paper's
    row/column thread decomposition on all host cores for as many whole
    z-steps as fit in ~budget_s, and one single-threaded step beside it."""
    import oracle
    pb = oracle.Problem(**wl.physics())
    cores = host_cores()
    a = wl.field()
    t0 = time.perf_counter()
    a, _ = oracle.run(pb, wl.dz, 1, a, threads=cores)
    t1 = time.perf_counter() - t0
    n = max(1, int(budget_s / max(t1, 1e-3)) - 1)
    t0 = time.perf_counter()
    oracle.run(pb, wl.dz, n, a, threads=cores)
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.run(pb, wl.dz, 1, a)
    dt1 = time.perf_counter() - t0
    return {"value": wl.points * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} z-steps of one {wl.nr}x{wl.nt} pulse (after 1 untimed), FP64 C oracle, "
                      f"row/column threads on {cores} cores, {dt:.1f} s",
            "single_thread_value": wl.points / dt1}


def cpu_oracle_sample_xy(wl, budget_s=12.0):
    """Times the FP64 CPU oracle on the Cartesian workload: rows and
    frequency bins split over all host cores (the paper's decomposition
    carried to this grid) for as many whole z-steps as fit in ~budget_s
    after one untimed step, and one single-threaded step beside it."""
    import oracle
    pb = oracle.Problem(**wl.physics())
    g = oracle.GridXY(**wl.grid())
    cores = host_cores()
    a = wl.field()
    t0 = time.perf_counter()
    a, _ = oracle.xy_run(pb, g, wl.dz, 1, a, threads=cores)
    t1 = time.perf_counter() - t0
    n = max(1, int(budget_s / max(t1, 1e-3)) - 1)
    t0 = time.perf_counter()
    a, _ = oracle.xy_run(pb, g, wl.dz, n, a, threads=cores)
    dt = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.xy_run(pb, g, wl.dz, 1, a)
    dt1 = time.perf_counter() - t0
    return {"value": wl.points * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} z-steps of the {wl.nx}x{wl.ny}x{wl.nt} field (after 1 untimed), FP64 C "
                      f"oracle, row/bin threads on {cores} cores, {dt:.1f} s",
            "single_thread_value": wl.points / dt1}


def run_reference(args, budget_s=150.0):
    """The oracle as the reference arm: whole z-steps of one cfg2 pulse with
    the paper's thread decomposition on all host cores; the timed steps are
    capped by a time budget (the sample states how many ran)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1507_05988_gb300 import workloads as W
    import oracle
    wl = W.config2(seed=0)
    pb = oracle.Problem(**wl.physics())
    cores = host_cores()
    a = wl.field()
    for _ in range(max(1, min(args.warmup, 3))):
        t0 = time.perf_counter()
        a, _ = oracle.run(pb, wl.dz, 1, a, threads=cores)
        t_one = time.perf_counter() - t0
    k = max(1, min(args.steps, int(budget_s / max(t_one, 1e-3))))
    t0 = time.perf_counter()
    a, _ = oracle.run(pb, wl.dz, k, a, threads=cores)
    dt = time.perf_counter() - t0
    v = wl.points * k / dt
    sample = (f"{k} of {args.steps} requested z-steps of one {wl.nr}x{wl.nt} pulse (time budget "
              f"{budget_s:.0f} s), FP64 C oracle, row/column threads on {cores} cores")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / k,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"cfg2 {wl.nr}x{wl.nt} one pulse (seed 0), dz=2 mm, FP64 CPU oracle"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def oracle_thread_scaling(steps=3):
    """The paper's thread-scaling experiment (Sec. 5, Table 2: Nr = 2112,
    Nt = 2048) with the FP64 oracle's row/column thread decomposition on this
    host's cores: seconds per z-step and speedup over one thread for 1, 2, 4,
    8, 12, 16, ... threads (up to the core count).  Context only: the paper's
    machine (24-core Xeon) is not this one, and the oracle is a plain
    restatement, not the paper's code."""
    from paper_1507_05988_gb300 import workloads as W
    import oracle
    wl = W.config1().with_(nr=2112, nt=2048, name="paper_table2_2112x2048")
    pb = oracle.Problem(**wl.physics())
    a0 = wl.field()
    cores = host_cores()
    counts = [t for t in (1, 2, 4, 8, 12, 16, 20, 24, 32, 48, 64) if t <= cores]
    if cores not in counts:
        counts.append(cores)
    rows = []
    for t in counts:
        a, _ = oracle.run(pb, wl.dz, 1, a0, threads=t)            # untimed first step
        t0 = time.perf_counter()
        oracle.run(pb, wl.dz, steps, a, threads=t)
        rows.append((t, (time.perf_counter() - t0) / steps))
    base = rows[0][1]
    out = {"experiment": "oracle thread scaling on the paper's Table 2 grid",
           "grid": f"{wl.nr}x{wl.nt}", "steps_timed": steps, "host_cores": cores,
           "rows": [{"threads": t, "s_per_step": dt, "speedup": base / dt, "efficiency": base / dt / t}
                    for t, dt in rows],
           "paper": "Table 2: 20 threads 19.23x (96 % efficiency) on a 24-core Xeon E7-4807"}
    print(json.dumps(out), flush=True)
    return 0


PERTURB_DEVICE = "cuda"      # where the conditioning reference's perturbation is drawn


def accuracy_leg(fcn, wl, field, dz, make=None, checkpoints=None):
    """FP32-mixed against the FP64 GPU path over the full fixed-step run, at
    checkpoints; beside it the same FP64 path with its field multiplied by
    (1 + 6e-8 xi), xi uniform in [-1, 1] per point, after every step (a
    perturbation of FP32 rounding size entering at every step, the way FP32
    rounding does): where that run drifts as far from the unperturbed one as
    FP32 does, the difference is the problem's conditioning, not the
    arithmetic.  make(precision) builds the solver (default: a radial Solver
    of wl); both solver kinds take the perturbation through their device
    field entry points."""
    if make is None:
        def make(prec):
            return fcn.Solver(wl.physics(), precision=prec)
    if checkpoints is None:
        checkpoints = [c for c in (100, 200, 300, 400, 500, 750, 1000) if c <= wl.nsteps]
        if wl.nsteps not in checkpoints:
            checkpoints.append(wl.nsteps)

    def run(prec, visit, perturb=False):
        import torch
        s = make(prec)
        s.set_field(field)
        done = 0
        if perturb:
            gen = torch.Generator(device=PERTURB_DEVICE)
            gen.manual_seed(12345)
            buf = torch.empty(field.shape, dtype=torch.complex128, device=PERTURB_DEVICE)
        for c in checkpoints:
            if perturb:
                for _ in range(c - done):
                    s.step(dz, 1)
                    s.get_field_device(buf)
                    xi = torch.rand(field.shape, generator=gen, device=PERTURB_DEVICE, dtype=torch.float64)
                    buf.mul_(1.0 + 6e-8 * (2.0 * xi - 1.0))
                    s.set_field_device(buf)
            else:
                s.step(dz, c - done)
            done = c
            visit(c, s.get_field(), s.diag()["energy"])
        s.close()

    ref = {}
    run(fcn.FCN_FP64, lambda c, a, e: ref.__setitem__(c, (a, e)))
    table = {c: {"steps": c} for c in checkpoints}
    for name, prec, pt in (("fp32", fcn.FCN_FP32_MIXED, False), ("fp64_perturbed", fcn.FCN_FP64, True)):
        def visit(c, a, e, name=name):
            table[c][name + "_field_rel_l2"] = rel_l2(a, ref[c][0])
            table[c][name + "_energy_rel"] = abs(e / ref[c][1] - 1)
        run(prec, visit, perturb=pt)
    for c in checkpoints:
        ref_d = table[c]["fp64_perturbed_field_rel_l2"]
        table[c]["fp32_over_reference"] = table[c]["fp32_field_rel_l2"] / ref_d if ref_d > 0 else None
    table = [table[c] for c in checkpoints]
    last = table[-1]
    return {"field_rel_l2": last["fp32_field_rel_l2"], "energy_rel": last["fp32_energy_rel"],
            "run": f"{checkpoints[-1]} steps of dz = {dz} m, FP32-mixed vs FP64 GPU path",
            "checkpoints": table,
            "conditioning": ("fp64_perturbed_*: the FP64 path with its field multiplied by "
                             "(1 + 6e-8 xi), xi ~ U[-1, 1] per point, after every step, against the "
                             "unperturbed FP64 path")}


def energy_drift_leg(fcn, W, steps=300):
    """Energy change per step of the loss-free parts of the step, where the
    exact discrete step conserves the energy: the config-2 pulse (1024 x
    4096, dz = 2 mm) with diffraction + dispersion only, and with the Kerr
    terms (n2, n4: pure phases) added, over `steps` steps in FP32-mixed and
    in FP64.  (E_n / E_0 - 1) / n; FP32 rounding that perturbs the discrete
    operator the same way at every step shows here as a steady drift."""
    wl = W.config2(seed=0)
    f = wl.field()
    out = {"workload": f"cfg2 pulse {wl.nr}x{wl.nt}, {steps} steps of {wl.dz} m"}
    for tag, flags in (("linear", fcn.FCN_DIFFRACTION | fcn.FCN_DISPERSION),
                       ("linear_kerr", fcn.FCN_DIFFRACTION | fcn.FCN_DISPERSION | fcn.FCN_KERR)):
        phys = dict(wl.physics(), flags=flags)
        row = {}
        for prec, name in ((fcn.FCN_FP32_MIXED, "fp32"), (fcn.FCN_FP64, "fp64")):
            s = fcn.Solver(phys, precision=prec)
            s.set_field(f)
            e0 = s.diag()["energy"]
            s.step(wl.dz, steps)
            row[name] = (s.diag()["energy"] / e0 - 1.0) / steps
            s.close()
        out[tag] = row
    return out


def chosen_form_leg(fcn, W, z_len, pulses=8, rtol=1e-4):
    """The chosen form against the plain FP64 GPU path at the metric's
    accuracy: config-2 pulses (noise seeds 0..pulses-1) propagated over
    z_len metres by step doubling at rtol, in
      - fp32_batched_plain:   FP32-mixed, all pulses in one adaptive batch
                              (one dz, one launch per stage), the law's dz;
      - fp32_batched_learned: the same with the learned dz proposals
                              (weights trained by learned_dz.py with this
                              library's kernels; skipped if the file is absent);
      - fp32_single_plain:    FP32-mixed, pulse 0 alone;
      - fp64_single_plain:    the plain FP64 GPU path, pulse 0 alone.
    Throughput counts accepted steps: pulses x Nr x Nt x accepted / wall
    time (the host loop synchronises every attempt, so wall time is the
    honest clock); raw counts all Strang substeps.  Pulse 0's final field
    and energy of every FP32 run are compared with the FP64 run's."""
    import numpy as np
    wls = [W.config2(seed=i) for i in range(pulses)]
    pts = wls[0].points
    dz0 = 2e-3
    wpath = os.path.join(ROOT, "paper_1507_05988_gb300", "learned_dz_weights.npy")
    weights = np.load(wpath) if os.path.exists(wpath) else None
    fields = [w.field() for w in wls]
    out = {"workload": f"{pulses} cfg2 pulses 1024x4096 (noise seeds 0..{pulses - 1}), "
                       f"0 -> {z_len} m, step doubling at rtol {rtol}",
           "z_m": z_len, "rtol": rtol, "pulses": pulses}

    def run(name, prec, n, controller):
        s = fcn.Solver([w.physics() for w in wls[:n]] if n > 1 else wls[0].physics(), precision=prec)
        if controller == 1:
            s.mlp_set(weights)
        for i in range(n):
            s.set_field(fields[i], pulse=i)
        s.propagate(3 * dz0, dz0, rtol=rtol, controller=controller)   # tuning and first tables
        for i in range(n):
            s.set_field(fields[i], pulse=i)
        t0 = time.perf_counter()
        st = s.propagate(z_len, dz0, rtol=rtol, controller=controller, max_reject=40)
        wall = time.perf_counter() - t0
        a0, e0 = s.get_field(0), s.diag(0)["energy"]
        s.close()
        out[name] = {"pulses": n, "wall_s": wall, "accepted": st["accepted"], "rejected": st["rejected"],
                     "substeps": st["substeps"], "mlp_proposals": st["mlp_proposals"],
                     "accepted_point_steps_per_s": n * pts * st["accepted"] / wall,
                     "raw_point_steps_per_s": n * pts * st["substeps"] / wall}
        return a0, e0

    res = {}
    res["fp64_single_plain"] = run("fp64_single_plain", fcn.FCN_FP64, 1, 0)
    res["fp32_single_plain"] = run("fp32_single_plain", fcn.FCN_FP32_MIXED, 1, 0)
    res["fp32_batched_plain"] = run("fp32_batched_plain", fcn.FCN_FP32_MIXED, pulses, 0)
    if weights is not None:
        res["fp32_batched_learned"] = run("fp32_batched_learned", fcn.FCN_FP32_MIXED, pulses, 1)
    else:
        out["fp32_batched_learned"] = {"skipped": "no trained weights (learned_dz.py --save)"}
    a64, e64 = res["fp64_single_plain"]
    v64 = out["fp64_single_plain"]["accepted_point_steps_per_s"]
    for name, (a, e) in res.items():
        if name == "fp64_single_plain":
            continue
        out[name]["pulse0_field_rel_l2_vs_fp64"] = rel_l2(a, a64)
        out[name]["pulse0_energy_rel_vs_fp64"] = abs(e / e64 - 1)
        out[name]["speedup_over_fp64"] = out[name]["accepted_point_steps_per_s"] / v64
    best = "fp32_batched_learned" if weights is not None else "fp32_batched_plain"
    out["chosen"] = best
    return out


def cartesian_leg(fcn, W, pg, world, accuracy=True, cpu=True):
    """Config 1's pulse on the 255 x 255 x 256 Cartesian grid (x and y
    Crank-Nicolson factors): the full 200-step run timed in FP32-mixed and in
    FP64 (CUDA events on the launch stream), the FP32 field and energy
    against the FP64 path at checkpoints (accuracy_leg), and per-kernel CUDA-event times of
    a profiled replay with their algorithmic HBM fractions (one complex64
    field read and write per point and launch), and the FP64 oracle timed on
    the host beside it (cpu_oracle_sample_xy)."""
    import torch
    wl = W.cartesian_config1()
    pts, K = wl.points, wl.nsteps
    f = wl.field()
    out = {"workload": f"{wl.name}: {wl.nx}x{wl.ny}x{wl.nt} nodes over 10 w0 x 10 w0 x 16 tp "
                       f"(w0=1 mm, tp=100 fs, 3 Pcr, n2), {K} steps of {wl.dz} m",
           "points": pts, "steps": K,
           "l2": f"field {pts * 8 / 1e6:.0f} MB complex64 vs 129 MB L2"}
    for prec, name in ((fcn.FCN_FP32_MIXED, "fp32"), (fcn.FCN_FP64, "fp64")):
        s = fcn.SolverXY(wl.grid(), wl.physics(), precision=prec)
        s.set_field(f)
        s.step(wl.dz, 3)                         # warm-up (and variant timing)
        s.set_field(f)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        s.step(wl.dz, K)
        b.record()
        torch.cuda.synchronize()
        t = reduce_max(a.elapsed_time(b), pg, "cuda")
        out[name] = {"value": weak_scaling_value(world, pts, K, t), "ms_per_step": t / K,
                     "variants": {"row": s.variants()[0], "line": s.variants()[1]}}
        if name == "fp32":
            s.profile(True)
            s.step(wl.dz, K)
            prof = s.profile_read(reset=True)
            s.profile(False)
            peak, peak_src = measured_peaks()
            kernels = {}
            for k, (ms, n) in prof.items():
                gbps = n * 2 * pts * 8 / (ms * 1e-3) / 1e9 if ms else None
                kernels[k] = {"launches": n, "total_ms": ms, "avg_us": (ms / n * 1e3 if n else None),
                              "alg_GBps": gbps, "frac_of_hbm_peak": (gbps / peak if gbps else None)}
            dom = max(prof.items(), key=lambda kv: kv[1][0])[0]
            traffic = None
            tpath = os.path.join(ROOT, "profiles", "traffic.json")
            if os.path.exists(tpath):
                with open(tpath) as fh:
                    traffic = json.load(fh).get("cart_" + dom)
            out["gpu_launches"] = int(sum(n for _, n in prof.values()))
            out["kernels"] = kernels
            out["roofline"] = {"bound": "hbm", "achieved": kernels[dom]["alg_GBps"], "peak": peak,
                               "unit": "GB/s", "frac": kernels[dom]["alg_GBps"] / peak,
                               "traffic": traffic, "kernel": dom, "peak_source": peak_src,
                               "algorithmic_bytes_per_launch": 2 * pts * 8}
        s.close()
    out["speedup_fp32_over_fp64"] = out["fp32"]["value"] / out["fp64"]["value"]
    if accuracy:
        out["accuracy_vs_fp64"] = accuracy_leg(
            fcn, wl, f, wl.dz, make=lambda prec: fcn.SolverXY(wl.grid(), wl.physics(), precision=prec),
            checkpoints=[25, 50, 100, 150, K])
    if cpu:
        out["cpu_baseline"] = cpu_oracle_sample_xy(wl)
    return out


def run_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    from paper_1507_05988_gb300 import build
    build.build()
    from paper_1507_05988_gb300 import fcn, workloads as W

    B = args.pulses
    wls = [W.config2(seed=rank * B + i) for i in range(B)]
    wl0 = wls[0]
    pts = wl0.points
    dz = wl0.dz
    solver = fcn.Solver([w.physics() for w in wls], precision=fcn.FCN_FP32_MIXED)
    fields = [w.field() for w in wls]
    for i, f in enumerate(fields):
        solver.set_field(f, pulse=i)
    solver.step(dz, args.warmup)
    torch.cuda.synchronize()
    variants = {"row": solver.variants(0)[0], "column": solver.variants(0)[1],
                "paired_columns": solver.pairing(),
                "sequential_columns_all_pulses": solver.sequential_columns()}

    def barrier():
        if pg:
            pg.barrier()

    # ---- timed region: K z-steps of the whole batch, device-resident ----
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    solver.step(dz, args.steps)
    e1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    t_ms = reduce_max(e0.elapsed_time(e1), pg, "cuda")
    value = weak_scaling_value(world, B * pts, args.steps, t_ms)

    # ---- kernel roofline: the same steps replayed from graphs that carry an
    # event node before and after every kernel (the launch structure of the
    # timed region; one synchronisation per replayed block of steps) ----
    # the replay starts from the state the timed region started from (the
    # row stage's work depends on the field: wing rows skip work)
    for i, f in enumerate(fields):
        solver.set_field(f, pulse=i)
    solver.step(dz, args.warmup)
    solver.profile(2)
    solver.step(dz, args.steps)
    prof = solver.profile_read(reset=True)
    solver.profile(False)
    launches = int(sum(n for _, n in prof.values()))
    # algorithmic bytes: one field read + one write (complex64) per point and
    # stage execution; per pulse a K-step call runs 1 head, K-1 middle and
    # 1 tail row stage and K column stages
    execs = {"row_head": 1, "row_mid": args.steps - 1, "row_tail": 1, "column": args.steps}
    stage_bytes = 2 * pts * 8
    peak, peak_src = measured_peaks()
    kernels = {}
    for k, (ms, n) in prof.items():
        tot = B * execs[k] * stage_bytes
        gbps = tot / (ms * 1e-3) / 1e9 if ms else None
        kernels[k] = {"launches": n, "total_ms": ms, "avg_us": (ms / n * 1e3 if n else None),
                      "alg_GBps": gbps, "frac_of_hbm_peak": (gbps / peak if gbps else None)}
    dom_name = max(prof.items(), key=lambda kv: kv[1][0])[0]
    achieved = kernels[dom_name]["alg_GBps"]
    # a launch processes one pulse, two (paired column stage, two-pulse row
    # launch) or the whole batch (batched stage): the pulses it covers on average
    units = B * execs[dom_name] / prof[dom_name][1]
    bytes_per_launch = stage_bytes * units
    # measured DRAM bytes (ncu) per pulse of the row stage, per paired column
    # launch (two pulses) of the column stage, scaled to this launch's pulses
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if dom_name == "column" and variants["paired_columns"] == 1 and \
                variants["sequential_columns_all_pulses"] != 1:
            t = tj.get("column_pair")
            traffic = t * units / 2 if t else None
        else:
            t = tj.get(dom_name)
            traffic = t * units if t else None

    # ---- end to end through the C-ABI with pinned host buffers ----
    # every step: each pulse's field uploaded from pinned host memory, one
    # z-step, each pulse's field read back; host buffers in complex64 (the
    # FP32-mixed form's own state, fcn_set/get_field_c64) and, for
    # comparison, complex128 (fcn_set/get_field, converted on the device)
    import ctypes as C
    K2 = max(1, min(args.steps, 10))

    def e2e_run(dtype, setf, getf, ptr):
        host_in = [torch.from_numpy(f.astype(dtype)).pin_memory() for f in fields]
        host_out = [torch.empty_like(h).pin_memory() for h in host_in]

        def one_step():
            for i in range(B):
                fcn.check(setf(solver.ctx, i, C.cast(host_in[i].data_ptr(), ptr)), solver.ctx)
            solver.step(dz, 1)
            for i in range(B):
                fcn.check(getf(solver.ctx, i, C.cast(host_out[i].data_ptr(), ptr)), solver.ctx)

        for _ in range(3):       # untimed warm-up (first touch of the pinned buffers)
            one_step()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        for _ in range(K2):
            one_step()
        torch.cuda.synchronize()
        return reduce_max(time.perf_counter() - t0, pg, "cuda")

    t_e2e = e2e_run(np.complex64, fcn.fcn_set_field_c64, fcn.fcn_get_field_c64, fcn._F)
    t_e2e128 = e2e_run(np.complex128, fcn.fcn_set_field, fcn.fcn_get_field, fcn._D)
    e2e = {"value": weak_scaling_value(world, B * pts, K2, t_e2e * 1e3), "unit": UNIT,
           "h2d_bytes_per_step": B * pts * 8, "d2h_bytes_per_step": B * pts * 8,
           "steps": K2, "note": "per step: fcn_set_field_c64 of every pulse (pinned host complex64), "
                                "fcn_step(dz, 1), fcn_get_field_c64 of every pulse",
           "complex128_host_buffers": {
               "value": weak_scaling_value(world, B * pts, K2, t_e2e128 * 1e3),
               "h2d_bytes_per_step": B * pts * 16, "d2h_bytes_per_step": B * pts * 16,
               "note": "fcn_set_field / fcn_get_field (host complex128, converted on the device)"}}
    solver.close()

    # ---- batched form on 64 uneven pulses (config-4 draws) ----
    cfg4 = None
    if not args.no_cfg4:
        w4 = W.config4()
        s4 = fcn.Solver([w.physics() for w in w4], precision=fcn.FCN_FP32_MIXED)
        for i, w in enumerate(w4):
            s4.set_field(w.field(), pulse=i)
        pts4 = sum(w.points for w in w4)
        cfg4 = {"pulses": len(w4), "points": pts4, "dz_m": w4[0].dz, "steps": args.cfg4_steps}
        for mode, name in ((1, "batched_one_launch_per_stage"), (0, "per_pulse_launches")):
            s4.set_batching(mode)
            s4.step(w4[0].dz, 2)
            torch.cuda.synchronize()
            a4, b4 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a4.record()
            s4.step(w4[0].dz, args.cfg4_steps)
            b4.record()
            torch.cuda.synchronize()
            cfg4[name] = pts4 * args.cfg4_steps / (a4.elapsed_time(b4) * 1e-3)
        s4.close()

    # ---- Cartesian transverse grid (3D+1) ----
    cart = None if args.no_cartesian else cartesian_leg(
        fcn, W, pg, world, accuracy=rank == 0 and not args.no_accuracy,
        cpu=rank == 0 and world == 1 and not args.no_cpu_baseline)

    # ---- plain FP64 FCN on the same batch ----
    K64 = max(2, min(args.steps, 6))
    s64 = fcn.Solver([w.physics() for w in wls], precision=fcn.FCN_FP64)
    for i, f in enumerate(fields):
        s64.set_field(f, pulse=i)
    s64.step(dz, 1)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    s64.step(dz, K64)
    b.record()
    torch.cuda.synchronize()
    v64 = weak_scaling_value(world, B * pts, K64, reduce_max(a.elapsed_time(b), pg, "cuda"))
    s64.close()
    # the FP64 path is bound by FP64 arithmetic: flops per point-step from the
    # ncu instruction counts of its row and column kernels (2 DFMA + DADD +
    # DMUL: 346 + 96 per point, profiles/fp64_kernels_cfg2.md) against the
    # FP64 FMA rate measured here by the library's microkernel
    fp64_flops_per_point_step = 442.0
    fp64_peak = fcn.alu_peak(0)
    fp64_roof = {"bound": "alu", "achieved": fp64_flops_per_point_step * v64 / world / 1e12,
                 "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                 "frac": fp64_flops_per_point_step * v64 / world / fp64_peak,
                 "flops_per_point_step": fp64_flops_per_point_step,
                 "peak_source": "fcn_alu_peak(0): this library's FP64 FMA microkernel, measured in this run",
                 "fp32_fma_peak_tflops": fcn.alu_peak(1) / 1e12}

    # ---- the chosen form (FP32 + learned dz + batched, adaptive) against the
    # plain FP64 path at the metric's rtol ----
    chosen = None
    if rank == 0 and not args.no_chosen:
        chosen = chosen_form_leg(fcn, W, args.chosen_z)

    # ---- accuracy of the chosen form against the FP64 path, full 1000-step run ----
    acc = None
    if rank == 0 and not args.no_accuracy:
        acc = accuracy_leg(fcn, wl0, fields[0], dz)
        acc["loss_free_energy_drift_per_step"] = energy_drift_leg(fcn, W)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_sample(wl0)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {
                "workload": f"cfg2 {wl0.nr}x{wl0.nt} (w0=2 mm, tp=50 fs, 5 Pcr, n2+n4, 1% noise), "
                            f"dz=2 mm, FP32-mixed, {B} pulses per GPU",
                "nr": wl0.nr, "nt": wl0.nt, "pulses_per_gpu": B, "dz_m": dz,
                "l2": f"inputs larger than L2: {B} x {pts * 8 / 1e6:.1f} MB complex64 field "
                      f"per GPU vs 129 MB L2",
                "timed": f"one fcn_step(dz, {args.steps}) call (CUDA graphs), CUDA events on "
                         "the launch stream",
                "kernel_variants": variants,
            },
            "ms_per_z_step_per_pulse": t_ms / args.steps / B,
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": dom_name, "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "note": "achieved = algorithmic bytes / mean CUDA-event launch time"},
            "kernels": kernels,
            "batched_cfg4": cfg4,
            "cartesian_3d1": cart,
            "fp64_gpu": {"value": v64, "unit": UNIT, "steps": K64,
                         "speedup_of_fp32_mixed": value / v64, "roofline": fp64_roof},
            "accuracy_vs_fp64": acc,
            "chosen_form": chosen,
            "clocks": clk,
            "e2e": e2e,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.oracle_scaling:
        return oracle_thread_scaling()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
