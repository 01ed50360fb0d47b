"""Benchmark: particle-steps/s of the two-fluid spin-SPH step on one GB300.

Default workload: the 20,100,112-particle rotating cylinder (R = 146 dx,
H = 292 layers, 19.55M fluid + 0.55M wall particles; the 19.6M resolution of
Sec. 3), synthetic jittered-lattice input (paper_2405_03980_gb300.synth).
A "step" is one full kick-drift-kick time step: cell keys, counting sort,
reorder, density + Tait pressure, the fused pair pass, kick, wall-torque
reduction.  Inputs (~6 GB of state) are far larger than L2 (129 MB), so no L2
flush is needed between steps.

Forms timed: the FP64 form (and the mixed FP32 form once available); the
headline `value` is the fastest form that is built.  Under torchrun every rank
advances its own replica of the cylinder (no exchange: weak scaling).

`--impl reference` times the CPU FP64 oracle (O(N^2), all host cores) on a
bounded sample of the same workload: a compact cluster of fluid particles
whose density, pressure and pair forces are evaluated against all N particles;
the per-row costs give the time of a full step (N density rows and N_fluid
force rows), and value = N / that time.  The cpu_baseline leg of the GPU arm
reports the same quantity.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s at 19.6M particles"
UNIT = "particle-steps/s"

# Length of each workload's whole job in steps, as its configuration states it
# (the 2.4M cylinder: 1000 steps; the 19.6M cylinder: 200; the uneven ensemble:
# 100; the low-temperature stress: 10,000).  The end-to-end leg runs one whole
# job from host state to host state, so the upload of the initial state and the
# read-back of the final one are spread over the steps the job really takes.
JOB_STEPS = {"cyl_2525900": 1000, "cyl_20100112": 200, "ensemble64": 100,
             "cyl_2525900_lowT": 10000}


def e2e_steps(workload, steps, override=0):
    """Steps of the end-to-end leg: the override if given, else the workload's
    job length, never fewer than the device-timed steps."""
    if override > 0:
        return override
    return max(steps, JOB_STEPS.get(workload, steps))

# Algorithmic work is counted per UNIQUE interacting pair with at least one
# fluid particle: a fluid-fluid pair once (the gather evaluates it from both
# sides; that second evaluation is implementation work, not algorithmic), a
# fluid-wall pair once.  The counts come from sph_pair_census, which sorts
# the ordered (fluid row, neighbour) pairs of the lists into species classes:
# unique = fluid-fluid / 2 + fluid-wall.
# Operations per pair of the pair pass, counted from the kernel source
# (add/sub/mul = 1, fused multiply-add = 2, sqrt/rsqrt/div = 1), by the terms
# a pair carries (Eqs. 1-2 as the model reads them): two inviscid particles
# the pressure term alone; unlike species (walls count as viscous) pressure,
# interfacial and local interaction with its torque; two viscous particles
# pressure, shear and rotational with its torque.  The FP64 form's pair pass
# runs one specialised loop per class and these are its counts.  For the
# mixed form the same terms cost 6 more (the pair vector from the cell
# offsets: a subtraction and a fused multiply-add per axis where the FP64
# form subtracts) plus its compensated sums (4 operations per sum per group
# of 8 neighbours: 1.5 per pair for the force alone, 3 with the torque); its
# pair pass, bound by L1 throughput and gather latency, runs one loop that
# evaluates every term for every pair (96 operations), the rest being
# implementation work (specialised loops measured slower there).
FORCE_FLOPS_BY_CLASS = {"fp64": {"II": 23, "IX": 76, "VV": 79},
                        "mixed": {"II": 30.5, "IX": 85, "VV": 88}}
# Density pass: operations per pair of the density sum (pair vector, r^2,
# sqrt, Wendland W, accumulation; the mixed form adds the cell offsets and
# the Kahan update).  W_ij = W_ji, so a pair is algorithmic work once.  The
# candidate tests that find the neighbours, rejected ones included, are not
# algorithmic work.
DENSITY_FLOPS_PER_PAIR = {"fp64": 18, "mixed": 29}
# Algorithmic DRAM bytes per particle of the two neighbour passes: each must
# read a particle's own record once and write its results once; neighbour
# records are re-reads that a good kernel serves on chip.  Density: the
# position record in, rho and P (and V, P/rho^2 for the pair pass) out.  Pair
# pass: position, velocity, spin, V and P/rho^2 in, a and alpha out.
ALGO_BYTES_PER_PARTICLE = {"k_density_mixed": 4 + 16 + 16, "k_density_fp64": 32 + 32,
                           "k_forces_mixed": 4 + 48 + 32, "k_forces_mixed_x2": 4 + 48 + 32,
                           "k_forces_fp64": 96 + 64}
# Optional steps of Algorithm 1 (--extras).  The pressure filter streams each
# fluid/inner-wall row's neighbour list and the kernel shapes the density
# pass stored beside it (4 B + 4 B mixed, 4 B + 8 B FP64 per neighbour) and
# gathers (V, P) from chip-resident records: an HBM-bound pass whose
# algorithmic bytes are those streams plus, per particle, its count, its own
# (V, P) and the P and P/rho^2 it writes.  The collision model puts one add
# per pair in the pair pass (the products of the rare colliding pairs are
# not counted).
FILTER_BYTES_PER_PAIR = {"fp64": 12, "mixed": 8}
FILTER_BYTES_PER_PARTICLE = {"fp64": 4 + 16 + 8 + 8, "mixed": 4 + 8 + 4 + 4}
# its arithmetic: two fused multiply-adds per neighbour (FP64 form, which
# stores V and V P), three operations plus a compensated sum per group of 8
# (mixed); on GB300's FP64 pipe the FP64 form's two FMAs outweigh its bytes.
FILTER_FLOPS_PER_PAIR = {"fp64": 4, "mixed": 3}
COLLISION_FLOPS_PER_PAIR = 1
EXTRAS = {"pfilter": 128, "collision": 256}
# Neighbour search: FP32 operations per candidate test (pair vector, r^2; the
# mixed form adds the cell displacement).  Its implementation work is the
# candidate tests of the 27-cell stencil of every particle that keeps a list
# (fluid and inner wall), counted on the host from the initial positions
# (candidate_tests); reported beside the roofline, not as algorithmic work.
# Its algorithmic work is reading each particle's position record once.
SEARCH_FLOPS_PER_TEST = {"fp64": 8, "mixed": 11}
SEARCH_ALGO_BYTES_PER_PARTICLE = {"fp64": 16, "mixed": 16}

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per particle of
# one launch, from the ncu captures summarised in profiles/ (2,525,900-particle
# cylinder; the traffic grows with the particle count).  Each figure holds
# only while the kernel's sources hash to the values recorded with it; after
# any change the roofline reports traffic null until it is re-measured.
DRAM_BYTES_PER_PARTICLE = {
    "k_cell_search<true>": (222.4, {"sph_search.cu": "cf8572358b743c10",
                                    "sph_internal.h": "1756e1381f18b6ad"}),
    "k_cell_search<false>": (None, {}),
    "k_density_mixed": (769.9, {"sph_mixed.cu": "701e6e1044459c54",
                                "sph_internal.h": "1756e1381f18b6ad"}),
    "k_forces_mixed": (None, {}),
    "k_forces_mixed_x2": (416.8, {"sph_mixed.cu": "701e6e1044459c54",
                                  "sph_internal.h": "1756e1381f18b6ad"}),
    "k_density_fp64": (646.8, {"sph_fp64.cu": "2b1a99c0f5cfa53b",
                               "sph_internal.h": "1756e1381f18b6ad"}),
    "k_forces_fp64": (860.5, {"sph_fp64.cu": "2b1a99c0f5cfa53b",
                              "sph_internal.h": "1756e1381f18b6ad"}),
}


# Algorithmic DRAM bytes per particle of the streaming stages (plain, mixed):
# the state each reads and writes once (section 8 of the design notes).
STREAM_BYTES_PER_PARTICLE = {
    "kick_drift_keys": {"fp64": 224, "mixed": 120},
    "cell_scan": {"fp64": 0, "mixed": 0},            # 8 B per cell, below
    "scatter_cell_sort": {"fp64": 16, "mixed": 16},
    "reorder": {"fp64": 240, "mixed": 144},
    "kick": {"fp64": 192, "mixed": 96},
    "wall_torque": {"fp64": 32, "mixed": 16},
}


def step_roofline(stage_ms, form, n_particles, n_cells, pairs, unique, peak_alu, hbm_gbs,
                  extras=(), force_flops=None):
    """Lower bound of one step: every stage at its own roof (the streaming
    stages and the neighbour search at the measured HBM bandwidth with their
    algorithmic bytes, the density and pair passes at the measured FMA rate
    with their algorithmic flops per unique pair), summed, and the fraction of
    it the measured step reaches.  pairs: ordered fluid-row pairs (what the
    filter streams); unique: unique pairs with a fluid particle."""
    bound = {}
    for st, b in STREAM_BYTES_PER_PARTICLE.items():
        by = b[form] * n_particles + (8 * n_cells if st == "cell_scan" else 0)
        bound[st] = by / (hbm_gbs * 1e9) * 1e3
    bound["cell_search"] = SEARCH_ALGO_BYTES_PER_PARTICLE[form] * n_particles / (hbm_gbs * 1e9) * 1e3
    flops = {"density": DENSITY_FLOPS_PER_PAIR[form] * unique,
             "forces": force_flops}
    if "pfilter" in extras:
        by = filter_bytes(form, pairs, n_particles)
        fl = FILTER_FLOPS_PER_PAIR[form] * pairs
        bound["pressure_filter"] = max(by / (hbm_gbs * 1e9), fl / (peak_alu[form] * 1e12)) * 1e3
    for st, fl in flops.items():
        bound[st] = fl / (peak_alu[form] * 1e12) * 1e3
    tb = sum(bound.values())
    tm = sum(stage_ms.values())
    return {"bound_ms": tb, "measured_ms": tm, "frac": tb / tm,
            "per_stage_bound_ms": bound, "hbm_gbs": hbm_gbs,
            "note": "sum over stages of algorithmic bytes / measured HBM bandwidth or "
                    "algorithmic flops (per unique pair) / measured FMA rate; the neighbour "
                    "search counts only its position reads (its candidate tests, rejected "
                    "ones included, are not algorithmic work); measured_ms sums the "
                    "per-stage event times"}


def hbm_peak():
    """Measured HBM copy bandwidth of this machine's GPUs (GB/s)."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6695.5


def filter_bytes(form, pairs, n_particles):
    return FILTER_BYTES_PER_PAIR[form] * pairs + FILTER_BYTES_PER_PARTICLE[form] * n_particles


def ratio(traffic, algorithmic):
    """Measured DRAM bytes over algorithmic bytes (None without a capture)."""
    return None if traffic is None or not algorithmic else traffic / algorithmic


# What the same captures show binding each pass (its busiest unit); reported
# beside the FMA-rate fraction under the same source-hash condition as the
# traffic.
BINDING = {
    "k_forces_mixed_x2": "L1 data path of the neighbour gathers: L1 throughput 81 %, issue "
                         "58 %, FMA pipe 45 % (ncu, 2,525,900-particle cylinder); each pair is "
                         "evaluated from both sides",
    "k_density_mixed": "L1 data path of the offset gathers: L1 throughput 84 %, issue 57 %, "
                       "FMA pipe 26 % (ncu, 2,525,900-particle cylinder)",
    "k_forces_fp64": "FP64 pipe 89 % busy (ncu, 2,525,900-particle cylinder); each pair is "
                     "evaluated from both sides",
    "k_density_fp64": "FP64 pipe 85 % busy (ncu, 2,525,900-particle cylinder)",
}


def sources_match(kernel):
    """The kernel's sources hash to the values recorded with its capture."""
    import hashlib
    per, srcs = DRAM_BYTES_PER_PARTICLE.get(kernel, (None, {}))
    if per is None:
        return False
    for f, h in srcs.items():
        path = os.path.join(ROOT, "paper_2405_03980_gb300", "csrc", f)
        if hashlib.sha256(open(path, "rb").read()).hexdigest()[:16] != h:
            return False
    return True


def measured_traffic(kernel, n_particles):
    """Per-launch DRAM bytes of kernel at n_particles, or None when no capture
    matches the current sources."""
    if not sources_match(kernel):
        return None
    return DRAM_BYTES_PER_PARTICLE[kernel][0] * n_particles


def pair_classes(census):
    """Unique pairs by class from the ordered census [II, unlike fluid,
    VV, inviscid-wall, viscous-wall]: fluid-fluid pairs halved, fluid-wall
    pairs once (walls count as viscous)."""
    c = [int(x) for x in census]
    return {"II": c[0] // 2, "IX": c[1] // 2 + c[3], "VV": c[2] // 2 + c[4]}


def candidate_tests(insts):
    """Sum over the particles that keep a neighbour list of the particle count
    of their 27 surrounding grid cells (cell side >= 2h, the grid of the
    library: floor(L / 2h) cells per axis, periodic in z)."""
    total = 0
    for c in insts:
        p = c.params
        lo = np.array(p["box_lo"], dtype=np.float64)
        hi = np.array(p["box_hi"], dtype=np.float64)
        ncell = np.maximum(np.floor((hi - lo) / (2.0 * p["h"])), 1).astype(np.int64)
        side = (hi - lo) / ncell
        idx = np.clip(np.floor((c.pos - lo) / side).astype(np.int64), 0, ncell - 1)
        cnt = np.zeros(tuple(ncell + 2), dtype=np.int64)  # one ghost layer per side
        np.add.at(cnt, (idx[:, 0] + 1, idx[:, 1] + 1, idx[:, 2] + 1), 1)
        if p.get("periodic_z", 1):
            cnt[:, :, 0] = cnt[:, :, -2]
            cnt[:, :, -1] = cnt[:, :, 1]
        nb = np.zeros_like(cnt)
        for ox in (-1, 0, 1):
            for oy in (-1, 0, 1):
                for oz in (-1, 0, 1):
                    nb[1:-1, 1:-1, 1:-1] += cnt[1 + ox:cnt.shape[0] - 1 + ox,
                                                1 + oy:cnt.shape[1] - 1 + oy,
                                                1 + oz:cnt.shape[2] - 1 + oz]
        keep = c.species != 3
        total += int(nb[idx[keep, 0] + 1, idx[keep, 1] + 1, idx[keep, 2] + 1].sum())
    return total


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cyl_20100112")
    ap.add_argument("--forms", default="mixed,fp64")
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0,
                    help="steps of the end-to-end leg (0: the workload's whole job, "
                         "at least --steps)")
    ap.add_argument("--extras", default="",
                    help="optional steps of Algorithm 1 to switch on: pfilter, collision "
                         "(comma list; the default step has neither)")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="skin of the mixed form's reused neighbour lists in dx (0: the "
                         "library default; < 0: rebuild every step)")
    ap.add_argument("--cpu-sample", type=int, default=0,
                    help="fluid particles in the oracle sample (0 = size for ~15 s)")
    return ap.parse_args()


# ---------------------------------------------------------------- distributed

class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = torch.device("cuda", self.local) if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        # the raw samples go to SPH_CLOCKS_DIR if set (to keep them), else to
        # the temporary directory
        out = os.environ.get("SPH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"sph_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax),
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- CPU oracle leg

def oracle_sample(c, target_s: float = 15.0, n_sample: int = 0):
    """Bounded oracle sample: a compact cluster S of fluid particles near
    mid-radius and every particle R within 2h (+1 dx) of its bounding box.
    One sample step = oracle density+pressure for the rows R and pair forces
    for the rows S, each row evaluated against all N particles (the oracle is
    O(N) per row), timed separately so that a full step can be estimated
    from the per-row costs (full_step_seconds)."""
    import oracle
    p = oracle.make_params(c.params)
    fluid = np.nonzero(c.species < 2)[0]
    centre = np.array([0.5 * c.R, 0.0, 0.5 * c.H])
    d = np.abs(c.pos[fluid] - centre).max(1)
    order = fluid[np.argsort(d, kind="stable")]

    def rows_for(k):
        S = np.sort(order[:k])
        lo = c.pos[S].min(0) - (2 * p.h + 1.0)
        hi = c.pos[S].max(0) + (2 * p.h + 1.0)
        inside = np.all((c.pos >= lo) & (c.pos <= hi), axis=1)
        return S, np.nonzero(inside)[0]

    def run(S, R):
        """Seconds per density row and per force row of one sample step."""
        t0 = time.perf_counter()
        rho, P = oracle.density(p, c.pos, c.species, rows=R)
        t1 = time.perf_counter()
        oracle.forces(p, c.pos, c.vel, c.spin, c.species, rho, P, rows=S)
        t2 = time.perf_counter()
        return (t1 - t0) / len(R), (t2 - t1) / len(S), t2 - t0

    # at least 32 force rows per host thread, so that the rows keep every
    # thread of the oracle's OpenMP loop busy and the per-row costs are
    # throughput figures, independent of the sample's size
    k_min = min(len(order), 32 * cores_used())
    if n_sample:
        S, R = rows_for(max(n_sample, k_min))
        return p, S, R, run
    # calibrate the cost per evaluated row on the smallest cluster, then size
    # the cluster so that one sample step costs about target_s seconds
    S, R = rows_for(k_min)
    t = run(S, R)[2]
    rows_per_s = (len(R) + len(S)) / max(t, 1e-4)
    want = target_s * rows_per_s
    k = k_min
    while k < len(order):
        k2 = min(len(order), int(k * 1.5) + 1)
        S2, R2 = rows_for(k2)
        if len(R2) + len(S2) > want:
            break
        k = k2
    S, R = rows_for(k)
    return p, S, R, run


def full_step_seconds(c, t_density_row, t_force_row):
    """Oracle seconds for one whole step of instance c from the per-row costs:
    a density row for every fluid and inner-wall particle (outer walls keep
    rho0) and a force row for every fluid particle; the O(N) kick, drift and
    wall placement are negligible beside these O(N) rows."""
    n_density = int((c.species != 3).sum())
    n_force = int((c.species < 2).sum())
    return n_density * t_density_row + n_force * t_force_row


def cores_used() -> int:
    try:
        n = len(os.sched_getaffinity(0))
    except Exception:
        n = os.cpu_count() or 1
    return int(os.environ.get("OMP_NUM_THREADS", n))


def cpu_baseline(c, n_sample=0):
    _, S, R, run = oracle_sample(c, target_s=10.0, n_sample=n_sample)
    best = min((run(S, R) for _ in range(2)), key=lambda r: r[2])
    td, tf, t = best
    T = full_step_seconds(c, td, tf)
    return {"value": c.n / T, "unit": UNIT, "cores": cores_used(), "kind": "oracle",
            "sample": (f"{len(S)} fluid particles of the {c.n}-particle cylinder: oracle "
                       f"density+pressure rows for the {len(R)} particles within 2h of them "
                       f"({td * 1e3:.2f} ms per row) and pair-force rows for the {len(S)} "
                       f"({tf * 1e3:.2f} ms per row), each row against all {c.n} particles; "
                       f"best of 2 sample steps of {t:.2f} s; value = N / (N_density_rows x "
                       f"t_density_row + N_fluid x t_force_row), a full step being "
                       f"{T:.3g} s")}


def run_reference(args, dist):
    if dist.rank != 0:
        return
    # the oracle is O(N) per row: the sample is drawn from the largest instance
    c = max(load_workload(args.workload), key=lambda x: x.n)
    target = min(10.0, max(1.0, 90.0 / max(1, args.steps + args.warmup)))
    _, S, R, run = oracle_sample(c, target_s=target, n_sample=args.cpu_sample)
    for _ in range(args.warmup):
        run(S, R)
    full, wall = 0.0, 0.0
    for _ in range(args.steps):
        td, tf, t = run(S, R)
        full += full_step_seconds(c, td, tf)
        wall += t
    v = c.n * args.steps / full
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * wall / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "particles": c.n,
                       "sample_particles": int(len(S)), "sample_rows": int(len(R)),
                       "ms_per_step": "wall time of one sample step; value is N over the "
                                      "full-step time estimated from its per-row costs",
                       "full_step_seconds": full / args.steps,
                       "l2": "inputs larger than L2 (not applicable on CPU)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "kind": "oracle", "cores": cores_used(),
                             "sample": f"{len(S)} force rows and {len(R)} density rows of the "
                                       f"{c.n}-particle cylinder per step, each row against "
                                       f"all N particles, scaled to a full step by the "
                                       f"per-row costs"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU leg

def time_form(insts, precision, args, dist, dev):
    import torch
    from paper_2405_03980_gb300 import _binding as B
    from paper_2405_03980_gb300.sim import Simulation

    sim = Simulation(insts, precision=precision, device=f"cuda:{dev}")
    stream = sim.stream
    if not args.no_autotune:
        sim.autotune(2)
    blocks = sim.launch_config()
    sim.step(args.warmup)
    sim.check()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    dist.barrier()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    ck = clocks.stop()
    sim.check()
    ms = e0.elapsed_time(e1) / args.steps
    ms = dist.max(ms)
    diag = sim.diagnostics()
    diag["n_pairs"] = sum(sim.diagnostics(k)["n_pairs"] for k in range(len(insts)))
    # the mixed form rebuilds its lists only every few steps: the per-stage
    # times are means over a window of steps, and the list-build stages are
    # also reported per build
    census = np.sum([sim.pair_census(k) for k in range(len(insts))], axis=0)
    b0 = sum(sim.list_builds(k) for k in range(len(insts)))
    nprof = args.profile_steps if precision == B.SPH_FP64 else max(args.profile_steps, 16)
    stages = sim.profile(nprof)
    builds = (sum(sim.list_builds(k) for k in range(len(insts))) - b0) / len(insts)
    launches = sim.launches_per_step()
    out = {"ms_per_step": ms, "diag": diag, "stages": stages, "clocks": ck,
           "launches_per_step": launches, "sim": sim, "blocks": blocks,
           "profile_steps": nprof, "list_builds_per_step": builds / nprof,
           "census": [int(x) for x in census]}
    return out


def e2e_buffers(insts):
    """Pinned host copies of the inputs and of the state read back."""
    import torch

    def pinned(parts):
        t = torch.from_numpy(np.ascontiguousarray(np.concatenate(parts))).pin_memory()
        return t

    pos = pinned([c.pos for c in insts])
    vel = pinned([c.vel for c in insts])
    spin = pinned([c.spin for c in insts])
    sp = pinned([c.species for c in insts])
    n = sum(c.n for c in insts)
    out_pos, out_vel, out_spin = (torch.empty((n, 3), dtype=torch.float64).pin_memory()
                                  for _ in range(3))
    return pos, vel, spin, sp, out_pos, out_vel, out_spin


def parse_extras(spec):
    ex = tuple(e.strip() for e in spec.split(",") if e.strip())
    bad = [e for e in ex if e not in EXTRAS]
    if bad:
        raise SystemExit(f"unknown --extras {bad}; choose from {sorted(EXTRAS)}")
    return ex


def load_workload(name, extras=()):
    """A named cylinder, or "ensembleK": K uneven cylinders advanced together;
    extras switch on optional steps of Algorithm 1 in every instance."""
    from paper_2405_03980_gb300 import _binding as B
    from paper_2405_03980_gb300 import synth
    if name.startswith("ensemble"):
        insts = synth.ensemble(int(name[len("ensemble"):] or 64))
    else:
        insts = [synth.workload(name, seed=0)]
    if extras:
        fl = B.SPH_FLAGS_DEFAULT
        for e in extras:
            fl |= EXTRAS[e]
        for c in insts:
            c.params = dict(c.params, flags=fl)
    return insts


def run_ours(args, dist):
    import torch
    from paper_2405_03980_gb300 import _binding as B
    from paper_2405_03980_gb300 import synth

    dev = dist.local
    torch.cuda.set_device(dev)
    B.lib(build_if_missing=True)
    extras = parse_extras(args.extras)
    insts = load_workload(args.workload, extras)
    if args.skin:
        for c in insts:
            c.params = dict(c.params, skin=args.skin)
    n_part = sum(c.n for c in insts)
    forms = [f.strip() for f in args.forms.split(",") if f.strip()]
    prec = {"fp64": B.SPH_FP64, "mixed": B.SPH_MIXED}
    results = {}
    for f in forms:
        results[f] = time_form(insts, prec[f], args, dist, dev)
    best = min(results, key=lambda f: results[f]["ms_per_step"])
    r = results[best]
    n_total = n_part * dist.world
    value = n_total / (r["ms_per_step"] * 1e-3)
    pairs = r["diag"]["n_pairs"]

    # roofline of the dominant kernel (the pair pass), timed with CUDA events
    # on the library's stream inside the profiled steps
    st = r["stages"]
    dom = max(st, key=st.get)
    peaks = {"fp64": B.sph_fma_peak(B.SPH_FP64, 1 << 15),
             "mixed": B.sph_fma_peak(B.SPH_MIXED, 1 << 20)}
    roofs = {}
    tests = candidate_tests(insts)
    census = {}
    for f in results:
        pr = results[f]["diag"]["n_pairs"]
        cls = pair_classes(results[f]["census"])
        uq = sum(cls.values())
        census[f] = {"ordered_fluid_row_pairs": pr, "ordered_by_class": results[f]["census"],
                     "unique_by_class": cls, "unique_pairs": uq, "candidate_tests": tests}
        unit = "FP64" if f == "fp64" else "FP32"
        byc = FORCE_FLOPS_BY_CLASS[f]
        fl_forces = sum(byc[k] * cls[k] for k in cls) + (
            COLLISION_FLOPS_PER_PAIR * uq if "collision" in extras else 0)
        # the mixed form's default pair pass takes two neighbours per step in
        # packed FP32; with the collision model it runs the one-neighbour loop
        fkern = ("k_forces_mixed_x2" if f == "mixed" and "collision" not in extras
                 else f"k_forces_{f}")
        stages = [("forces", fkern, fl_forces / max(uq, 1), uq,
                   "unique pairs with a fluid particle (" +
                   ", ".join(f"{cls[k]} {k} at {byc[k]}" for k in cls) + " flop)", unit),
                  ("density", f"k_density_{f}", DENSITY_FLOPS_PER_PAIR[f], uq,
                   "unique pairs with a fluid particle", unit)]
        # the neighbour search: algorithmic work is its position reads; in the
        # mixed form it runs in the steps that rebuild the lists, so its
        # launch time is the stage's mean over the profiled steps divided by
        # the builds per step
        bps = results[f]["list_builds_per_step"]
        t = results[f]["stages"]["cell_search"] / (bps if bps > 0 else 1.0)
        kern = f"k_cell_search<{str(f == 'mixed').lower()}>"
        by = SEARCH_ALGO_BYTES_PER_PARTICLE[f] * n_part
        ach = by / (t * 1e-3) / 1e9
        roofs.setdefault(f, {})["cell_search"] = {
            "kernel": kern, "bound": "hbm", "achieved": ach, "peak": hbm_peak(), "unit": "GB/s",
            "frac": ach / hbm_peak(), "peak_source": "MEASURED_PEAKS.json hbm_gbs, of measured",
            "traffic": measured_traffic(kern, n_part), "traffic_unit": "bytes per launch",
            "traffic_ratio": ratio(measured_traffic(kern, n_part), by),
            "work": f"{SEARCH_ALGO_BYTES_PER_PARTICLE[f]} B x {n_part} particles per launch "
                    "(position records read once); the candidate tests are implementation "
                    "work, not algorithmic",
            "candidate_tests": tests,
            "candidate_test_tflops": SEARCH_FLOPS_PER_TEST[f] * tests / (t * 1e-3) / 1e12,
            "launch_ms": t, "list_builds_per_step": bps}
        if "pfilter" in extras:
            t = results[f]["stages"]["pressure_filter"]
            by = filter_bytes(f, pr, n_part)
            fl = FILTER_FLOPS_PER_PAIR[f] * pr
            pk = peaks["mixed"] if f == "mixed" else peaks["fp64"]
            ent = {"kernel": f"k_pfilter_{f}",
                   "traffic": measured_traffic(f"k_pfilter_{f}", n_part),
                   "traffic_unit": "bytes per launch", "launch_ms": t}
            if by / (hbm_peak() * 1e9) >= fl / (pk * 1e12):  # the HBM roof is the higher
                ach = by / (t * 1e-3) / 1e9
                ent.update(bound="hbm", achieved=ach, peak=hbm_peak(), unit="GB/s",
                           frac=ach / hbm_peak(),
                           peak_source="MEASURED_PEAKS.json hbm_gbs, of measured",
                           work=f"{FILTER_BYTES_PER_PAIR[f]} B x {pr} fluid neighbour pairs + "
                                f"{FILTER_BYTES_PER_PARTICLE[f]} B x {n_part} particles per launch")
            else:
                ach = fl / (t * 1e-3) / 1e12
                ent.update(bound="alu", achieved=ach, peak=pk, unit="TFLOP/s", frac=ach / pk,
                           peak_source=f"measured {unit} FMA-chain rate of this GPU "
                                       "(sph_fma_peak), of measured",
                           work=f"{FILTER_FLOPS_PER_PAIR[f]} {unit} flop x {pr} fluid neighbour "
                                "pairs per launch")
            roofs.setdefault(f, {})["pressure_filter"] = ent
        for stage, kern, fpp, units, what, u in stages:
            pk = peaks["mixed"] if u == "FP32" else peaks["fp64"]
            src = f"measured {u} FMA-chain rate of this GPU (sph_fma_peak), of measured"
            t = results[f]["stages"][stage] * 1e-3
            ach = fpp * units / t / 1e12
            tr = measured_traffic(kern, n_part)
            roofs.setdefault(f, {})[stage] = {
                "kernel": kern, "bound": "alu", "achieved": ach, "peak": pk,
                "unit": "TFLOP/s", "frac": ach / pk,
                "traffic": tr, "traffic_unit": "bytes per launch",
                "algorithmic_bytes": ALGO_BYTES_PER_PARTICLE[kern] * n_part,
                "traffic_ratio": ratio(tr, ALGO_BYTES_PER_PARTICLE[kern] * n_part),
                "peak_source": src,
                "work": f"{fpp:.2f} {u} flop x {units} {what} per launch",
                "binding": BINDING.get(kern) if sources_match(kern) else None,
                "launch_ms": results[f]["stages"][stage]}
    dom_stage = max(("forces", "density", "cell_search"), key=lambda k: st[k])
    roof = roofs[best][dom_stage]
    hbm = hbm_peak()
    n_cells = sum(float((np.floor((np.array(c.params["box_hi"]) - np.array(c.params["box_lo"]))
                                  / (2.0 * c.params["h"])) + [2, 2, 0]).prod()) for c in insts)
    steps_roof = {f: step_roofline(results[f]["stages"], f, n_part, n_cells,
                                   results[f]["diag"]["n_pairs"], census[f]["unique_pairs"],
                                   peaks, hbm, extras,
                                   force_flops=roofs[f]["forces"]["achieved"] * 1e12 *
                                   roofs[f]["forces"]["launch_ms"] * 1e-3)
                  for f in results}

    # end-to-end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        sim = r["sim"]
        pos, vel, spin, sp, opos, ovel, ospin = e2e_buffers(insts)
        ke = e2e_steps(args.workload, args.steps, args.e2e_steps)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        sim.reinit(pos, vel, spin, sp)
        for _ in range(ke):
            sim.step(1)
            sim.diagnostics()
        B.sph_get_state(sim.ctx, opos, ovel, ospin)
        t = time.perf_counter() - t0
        t = dist.max(t)
        h2d = n_part * (3 * 3 * 8 + 1)
        d2h = ke * 8 * 33 + n_part * 3 * 3 * 8
        e2e = {"value": n_total * ke / t, "unit": UNIT, "steps": ke, "seconds": t,
               "h2d_bytes_per_step": h2d / ke, "d2h_bytes_per_step": d2h / ke,
               "includes": "one whole job of the workload: sph_init from pinned host state "
                           "(initial density+forces), steps x (sph_step + sph_diagnostics "
                           "read-back), sph_get_state"}
    for f in results:
        results[f]["sim"].close()

    cpu = None
    # (the oracle sample times the default step, so none with extras)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline and not extras:
        cpu = cpu_baseline(max(insts, key=lambda c: c.n), n_sample=args.cpu_sample)

    if dist.rank == 0:
        forms_out = {f: {"ms_per_step": results[f]["ms_per_step"],
                         "particle_steps_per_s": n_total / (results[f]["ms_per_step"] * 1e-3),
                         "pair_interactions_per_s":
                             results[f]["diag"]["n_pairs"] * dist.world /
                             (results[f]["ms_per_step"] * 1e-3),
                         "stage_ms": results[f]["stages"],
                         "stage_ms_note": f"mean per step over {results[f]['profile_steps']} "
                                          "eager steps (the list-build stages run only in "
                                          "the steps that rebuild)",
                         "list_builds_per_step": results[f]["list_builds_per_step"],
                         "launch_config": results[f]["blocks"]} for f in results}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if best == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "particles": n_part,
                       "fluid": sum(c.n_fluid for c in insts), "instances": len(insts),
                       "R": insts[0].R if len(insts) == 1 else None,
                       "H": insts[0].H if len(insts) == 1 else None,
                       "form": best, "parallelism": "replicas",
                       "extras": list(extras), "skin": args.skin or "default",
                       "l2": "inputs larger than L2 (state of GBs), no flush"},
            "pair_interactions_per_s": pairs * dist.world / (r["ms_per_step"] * 1e-3),
            "forms": forms_out,
            "roofline": roof,
            "pair_census": census[best],
            "step_roofline": steps_roof,
            "roofline_by_form": roofs,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": r["clocks"],
            # (mixed form: sph_step(k) runs k step graphs, each one launch short
            # of sph_step(1)'s count, then one closing half kick)
            "gpu_launches": ((r["launches_per_step"] - 1) * args.steps + 1 if best == "mixed"
                             else r["launches_per_step"] * args.steps),
            "dominant_stage": dom,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    dist = Dist()
    if args.impl == "reference":
        # the CPU oracle runs on rank 0 only; other ranks exit without work
        run_reference(args, dist)
        return
    dist.init("nccl")
    try:
        run_ours(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
