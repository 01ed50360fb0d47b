"""Force breakdown of a workload: the share of each pair term.

    python -m paper_2405_03980_gb300.breakdown --workload paper_8802016 \
        --steps 200 --every 50 --form mixed

Advances the workload and prints, every `every` steps, sum_i |f_i^term| of the
pressure, interfacial (temperature-gradient), shear, rotational and local
interaction (mutual friction) terms and their shares of the total, the
quantity the paper reports for its runs (Sec. 4).  Its magnitudes depend on
C_T and C_l, which the paper does not print; the workloads carry the recipe of
`synth.workload_params`.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import time

from . import _binding as B
from . import synth
from .sim import Simulation

TERMS = ("pressure", "interfacial", "shear", "rotational", "local_interaction")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper_2534800")
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--every", type=int, default=50)
    ap.add_argument("--form", choices=("mixed", "fp64"), default="mixed")
    args = ap.parse_args()
    c = synth.workload(args.workload)
    sim = Simulation(c, precision=B.SPH_MIXED if args.form == "mixed" else B.SPH_FP64)
    rows = []
    done = 0
    t0 = time.perf_counter()
    while True:
        mag = sim.force_breakdown()
        tot = float(mag.sum())
        rows.append({"step": done, "sum_abs_force": dict(zip(TERMS, map(float, mag))),
                     "share": {t: float(m) / tot for t, m in zip(TERMS, mag)}})
        if done >= args.steps:
            break
        k = min(args.every, args.steps - done)
        sim.step(k)
        done += k
    sim.check()
    secs = time.perf_counter() - t0
    sim.close()
    print(json.dumps({"workload": args.workload, "particles": c.n, "fluid": c.n_fluid,
                      "form": args.form, "seconds": secs, "trace": rows}), flush=True)


if __name__ == "__main__":
    main()
