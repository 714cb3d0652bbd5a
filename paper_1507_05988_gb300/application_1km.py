"""The paper's 1.1 km application run (Sec. 5, Fig. 4) on one GPU.

    python -m paper_1507_05988_gb300.application_1km --every 10000 --json out.json

Nr = 1350, Nt = 1024, 1.1e6 fixed steps of 1 mm (FP32-mixed by default),
from the Gaussian of Eq. (gauss) with peak intensity 3.14e14 W/m^2,
r0 = 18 mm, tau0 = 300 fs.  Every --every steps it records the quantities of
Fig. 4: the on-axis peak intensity, the peak intensity and electron density
anywhere, the energy, and the fluence F(r) = int |A|^2 dtau of that z.  The
paper reports the run (20 threads) as taking under three days; this prints
the wall time of the GPU run.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import fcn, workloads as W


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=1_100_000)
    ap.add_argument("--every", type=int, default=10_000)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--json", default="")
    a = ap.parse_args(argv)
    wl = W.application_1km()
    prec = fcn.FCN_FP32_MIXED if a.precision == "fp32" else fcn.FCN_FP64
    s = fcn.Solver(wl.physics(), precision=prec)
    s.set_field(wl.field())
    r = np.arange(wl.nr) * wl.r_max / (wl.nr - 1)
    rec = []
    t0 = time.perf_counter()
    done = 0
    while done < a.steps:
        n = min(a.every, a.steps - done)
        s.step(wl.dz, n)
        done += n
        d = s.diag(0)
        _, flu = s.profiles(0)
        rec.append({"z_m": done * wl.dz, "onaxis_peak_W_m2": d["onaxis_peak"],
                    "peak_W_m2": d["peak_intensity"], "peak_rho_m3": d["peak_rho"],
                    "energy_J": d["energy"], "nonfinite": d["nonfinite"],
                    "fluence_J_m2": [float(flu[i]) for i in range(0, wl.nr, max(1, wl.nr // 54))]})
        if d["nonfinite"]:
            break
    wall = time.perf_counter() - t0
    s.close()
    out = {"workload": f"{wl.name}: Nr {wl.nr}, Nt {wl.nt}, dz {wl.dz} m, {done} steps, "
                       f"P = {wl.p_over_pcr:.1f} P_cr, {a.precision}",
           "wall_s": wall, "point_steps_per_s": wl.nr * wl.nt * done / wall,
           "fluence_r_m": [float(r[i]) for i in range(0, wl.nr, max(1, wl.nr // 54))],
           "records": rec}
    print(json.dumps({k: v for k, v in out.items() if k != "records"}), flush=True)
    for x in rec[:: max(1, len(rec) // 12)]:
        print(f"z {x['z_m']:8.1f} m  on-axis peak {x['onaxis_peak_W_m2']:.3e}  peak {x['peak_W_m2']:.3e} "
              f"W/m^2  peak rho {x['peak_rho_m3']:.3e} m^-3  energy {x['energy_J']:.4e} J", flush=True)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(out, f)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
