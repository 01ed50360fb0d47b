"""Long-run conservation check of the two state forms on one workload.

    python -m paper_2405_03980_gb300.stress --workload cyl_2525900_lowT \
        --steps 10000 --every 1000 --forms mixed,fp64 [--fp64-steps 2000]

Advances the workload in each form and records, every `every` steps, the
FP64 diagnostics: the total mass change (exactly zero expected), the
angular-momentum budget residual |L_z(t) - L_z(0) - J_z(t)| / |L_z(0)| (the
walls' torque impulse J_z is the only external torque), the kinetic and spin
energy, and the extrema of the density and speed.  Prints one JSON line.

--margin widens the cell grid to R + margin (in dx): fluid particles that
diffuse through the two wall layers over long runs then stay on the grid
instead of ending the run with SPH_ERR_ESCAPED.  A run that stops on a
latched error reports the error and the last step reached.
"""
from __future__ import annotations

import argparse
import json
import time

from . import _binding as B
from . import synth
from .sim import Simulation


def run_form(c, precision, steps, every):
    sim = Simulation(c, precision=precision)
    d0 = sim.diagnostics()
    Lz0 = d0["L_orb"][2] + d0["L_spin"][2]
    rows = []
    t0 = time.perf_counter()
    done = 0
    error = None
    while done < steps:
        k = min(every, steps - done)
        try:
            sim.step(k)
            done += k
            d = sim.diagnostics()
        except B.SphError as e:
            error = f"{e} within steps {done + 1}..{done + k}"
            break
        Lz = d["L_orb"][2] + d["L_spin"][2]
        rows.append({"step": d["step"], "mass_change": d["mass"] - d0["mass"],
                     "Lz_budget_residual": (Lz - Lz0 - d["J_wall"][2]) / abs(Lz0),
                     "Lz_rel_change": (Lz - Lz0) / abs(Lz0),
                     "E_kin": d["E_kin"], "E_rot": d["E_rot"], "rho_min": d["rho_min"],
                     "rho_max": d["rho_max"], "v_max": d["v_max"]})
    secs = time.perf_counter() - t0
    sim.close()
    return {"seconds": secs, "Lz0": Lz0, "steps_done": done, "error": error, "trace": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="cyl_2525900_lowT")
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--fp64-steps", type=int, default=0, help="0 = same as --steps")
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--forms", default="mixed,fp64")
    ap.add_argument("--margin", type=float, default=0.0,
                    help="widen the cell grid to R + margin dx (0: the workload's box)")
    args = ap.parse_args()
    c = synth.workload(args.workload)
    if args.margin > 0:
        ext = c.R + args.margin
        c.params = dict(c.params, box_lo=(-ext, -ext, 0.0), box_hi=(ext, ext, float(c.H)))
    out = {"workload": args.workload, "particles": c.n, "grid_margin": args.margin}
    for f in [x.strip() for x in args.forms.split(",") if x.strip()]:
        steps = args.steps if (f == "mixed" or not args.fp64_steps) else args.fp64_steps
        out[f] = run_form(c, B.SPH_MIXED if f == "mixed" else B.SPH_FP64, steps,
                          min(args.every, steps))
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
