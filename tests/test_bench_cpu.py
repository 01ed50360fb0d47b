"""Host-side accounting of bench.py, checked by hand on small numbers: the
unique-pair classes from the ordered census, the per-class flop counts, the
step's lower bound, the CPU baseline's full-step estimate, the source-hash
guard of the recorded DRAM traffic and the end-to-end leg's job length."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2405_03980_gb300 import synth  # noqa: E402


def test_pair_classes_halve_fluid_pairs_and_count_wall_pairs_once():
    # ordered census [II, unlike fluid, VV, inviscid-wall, viscous-wall]
    cls = bench.pair_classes([10, 6, 4, 3, 2])
    assert cls == {"II": 5, "IX": 3 + 3, "VV": 2 + 2}


def test_class_flops_weight_the_pair_pass_work():
    cls = {"II": 100, "IX": 50, "VV": 10}
    for form in ("fp64", "mixed"):
        byc = bench.FORCE_FLOPS_BY_CLASS[form]
        total = sum(byc[k] * cls[k] for k in cls)
        assert total == pytest.approx(100 * byc["II"] + 50 * byc["IX"] + 10 * byc["VV"])
        # a pressure-only pair is the cheapest class, two viscous ones the dearest
        assert byc["II"] < byc["IX"] < byc["VV"]
    # the mixed form adds the pair vector from the cell offsets and the
    # compensated sums to every class
    for k in ("II", "IX", "VV"):
        assert bench.FORCE_FLOPS_BY_CLASS["mixed"][k] > bench.FORCE_FLOPS_BY_CLASS["fp64"][k]


def test_step_roofline_sums_the_stage_bounds():
    stage_ms = {k: 1.0 for k in bench.STREAM_BYTES_PER_PARTICLE}
    stage_ms.update(cell_search=1.0, density=2.0, forces=3.0)
    n, cells, unique = 1_000_000, 50_000, 40_000_000
    peaks = {"fp64": 1.0, "mixed": 80.0}
    r = bench.step_roofline(stage_ms, "mixed", n, cells, 2 * unique, unique, peaks, 6000.0,
                            force_flops=60.0 * unique)
    b = r["per_stage_bound_ms"]
    assert r["bound_ms"] == pytest.approx(sum(b.values()))
    assert r["measured_ms"] == pytest.approx(sum(stage_ms.values()))
    assert r["frac"] == pytest.approx(r["bound_ms"] / r["measured_ms"])
    # the pair pass at the FMA rate, the search at its position reads
    assert b["forces"] == pytest.approx(60.0 * unique / 80e12 * 1e3)
    assert b["cell_search"] == pytest.approx(
        bench.SEARCH_ALGO_BYTES_PER_PARTICLE["mixed"] * n / 6000e9 * 1e3)


def test_cpu_baseline_full_step_counts_rows_by_species():
    c = synth.workload("cyl_8960")
    t = bench.full_step_seconds(c, 2.0, 3.0)
    n_density = int((c.species != 3).sum())
    n_force = int((c.species < 2).sum())
    assert t == pytest.approx(2.0 * n_density + 3.0 * n_force)
    assert 0 < n_force < n_density < c.n


def test_traffic_needs_matching_sources(monkeypatch):
    tab = dict(bench.DRAM_BYTES_PER_PARTICLE)
    tab["k_probe"] = (100.0, {"sph_mixed.cu": "0" * 16})
    monkeypatch.setattr(bench, "DRAM_BYTES_PER_PARTICLE", tab)
    assert bench.measured_traffic("k_probe", 10) is None
    assert not bench.sources_match("k_probe")
    # recorded figures scale with the particle count while their sources match
    for k, (per, srcs) in bench.DRAM_BYTES_PER_PARTICLE.items():
        if per is not None and bench.sources_match(k):
            assert bench.measured_traffic(k, 2000) == pytest.approx(2 * bench.measured_traffic(k, 1000))
    assert bench.ratio(None, 5.0) is None
    assert bench.ratio(10.0, 5.0) == pytest.approx(2.0)


def test_e2e_runs_the_workloads_whole_job():
    # the 19.6M cylinder's job is 200 steps, the 2.4M cylinder's 1000
    assert bench.e2e_steps("cyl_20100112", 20) == 200
    assert bench.e2e_steps("cyl_2525900", 20) == 1000
    # never fewer steps than the device-timed run, and an explicit count wins
    assert bench.e2e_steps("cyl_20100112", 500) == 500
    assert bench.e2e_steps("cyl_20100112", 20, override=7) == 7
    # a workload without a stated job length runs the device-timed steps
    assert bench.e2e_steps("paper_2534800", 20) == 20
    for name in bench.JOB_STEPS:
        assert name in synth.WORKLOADS or name.startswith("ensemble")
