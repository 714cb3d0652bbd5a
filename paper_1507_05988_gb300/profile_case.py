"""Runs a few z-steps of one pulse with fixed kernel variants, for profilers.

    python -m paper_1507_05988_gb300.profile_case --config 2 --precision fp32 \
        --steps 3 --row-variant 0 --col-variant 0

The pulse is one of the seeded workloads (config 1: 128 x 256, config 2:
1024 x 4096, config 3: 2048 x 8192), or with --cartesian config 1's pulse on
the 255 x 255 x 256 Cartesian grid (--nxy for another node count per axis;
row variant, then line variant).  With variants given the autotuner does
not run, so a profiler sees exactly one fused middle row launch and one
column launch per step after the first step (which adds the opening row
launch).  Steps run without CUDA graphs unless --graph is given.
"""
from __future__ import annotations

import argparse

import numpy as np

from . import fcn, workloads


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--pulses", type=int, default=1)
    ap.add_argument("--row-variant", type=int, default=-1)
    ap.add_argument("--col-variant", type=int, default=-1)
    ap.add_argument("--graph", action="store_true")
    ap.add_argument("--branches", type=int, default=1, help="graph branches (pulse groups run concurrently)")
    ap.add_argument("--multi", type=int, default=2, help="multi-pulse row launch mode (0, 1, 2)")
    ap.add_argument("--seq", type=int, default=-1,
                    help="sequential column kernel over all pulses: 1 on, 0 off, -1 decided by "
                         "timing, 2..4 on with ring shape 0..2")
    ap.add_argument("--time", type=int, default=0,
                    help="then time this many graph-replayed steps (wall clock around a "
                         "synchronising call) and as many steps replayed from graphs with "
                         "event nodes around every kernel")
    ap.add_argument("--cartesian", action="store_true")
    ap.add_argument("--nxy", type=int, default=255,
                    help="Cartesian nodes per transverse axis (the walls stay at +-5 w0)")
    a = ap.parse_args(argv)
    if a.cartesian:
        return _cartesian(a)
    make = {1: workloads.config1, 2: workloads.config2, 3: workloads.config3}[a.config]
    wls = [make(seed=k) if a.config == 2 else make() for k in range(a.pulses)]
    prec = fcn.FCN_FP32_MIXED if a.precision == "fp32" else fcn.FCN_FP64
    s = fcn.Solver([w.physics() for w in wls] if a.pulses > 1 else wls[0].physics(), precision=prec)
    if a.row_variant >= 0 or a.col_variant >= 0:
        s.set_variants(a.row_variant, a.col_variant)
    for k, w in enumerate(wls):
        s.set_field(w.field(), pulse=k)
    if a.branches > 1:
        s.set_graph_branches(a.branches)
    s.set_multi_launch(a.multi)
    if a.pulses > 1:
        s.set_sequential_columns(a.seq)
        if a.seq >= 1:
            s.set_pairing(0)      # no pairing decision: the column launches are the step's own
    dz = wls[0].dz if wls[0].nsteps else 2e-3
    s.step(dz, a.steps, graph=a.graph)
    d = s.diag(0)
    ok = np.isfinite(d["energy"]) and d["nonfinite"] == 0
    if a.time > 0:
        import time
        s.step(dz, 16)
        s.diag(0)
        t0 = time.perf_counter()
        s.step(dz, a.time)
        s.diag(0)
        dt = time.perf_counter() - t0
        print(f"profile_case: graph replay {1e6 * dt / (a.time * a.pulses):.2f} us per pulse-step "
              f"({a.pulses} pulses, {a.branches} graph branches, "
              f"multi-pulse row launch mode {a.multi})")
        s.profile(2)
        s.step(dz, a.time)
        s.diag(0)
        for k, (ms, n) in s.profile_read().items():
            if n:
                print(f"profile_case: {k} {n} launches, {1e3 * ms / n:.2f} us per launch "
                      "(event nodes in the graphs)")
        s.profile(False)
    print(f"profile_case: config {a.config} {a.precision} steps {a.steps} variants {s.variants(0)} "
          f"energy {d['energy']:.6e}")
    s.close()
    return 0 if ok else 1


def _cartesian(a) -> int:
    import time
    wl = workloads.cartesian_config1()
    if a.nxy != wl.nx:
        wl = wl.with_(nx=a.nxy, ny=a.nxy, name=f"cart_cfg1_{a.nxy}x{a.nxy}x{wl.nt}")
    prec = fcn.FCN_FP32_MIXED if a.precision == "fp32" else fcn.FCN_FP64
    s = fcn.SolverXY(wl.grid(), wl.physics(), precision=prec)
    if a.row_variant >= 0 or a.col_variant >= 0:
        s.set_variants(a.row_variant, a.col_variant)
    s.set_field(wl.field())
    s.step(wl.dz, a.steps, graph=a.graph)
    d = s.diag()
    ok = np.isfinite(d["energy"]) and d["nonfinite"] == 0
    if a.time > 0:
        s.step(wl.dz, 16)
        s.diag()
        t0 = time.perf_counter()
        s.step(wl.dz, a.time)
        s.diag()
        dt = time.perf_counter() - t0
        print(f"profile_case: cartesian graph replay {1e6 * dt / a.time:.2f} us per step "
              f"({wl.points / (dt / a.time):.3e} point-steps/s)")
        s.profile(True)
        s.step(wl.dz, a.time)
        s.diag()
        for k, (ms, n) in s.profile_read().items():
            if n:
                print(f"profile_case: {k} {n} launches, {1e3 * ms / n:.2f} us per launch (events)")
        s.profile(False)
    print(f"profile_case: cartesian {wl.nx}x{wl.ny}x{wl.nt} {a.precision} steps {a.steps} "
          f"variants {s.variants()} energy {d['energy']:.6e}")
    s.close()
    return 0 if ok else 1


if __name__ == "__main__":
    raise SystemExit(main())
