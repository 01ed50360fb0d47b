"""The multi-process path of bench.py on CPU (gloo, world size 2): the
barrier and the max-over-ranks reduction used for the timed region, the
replicas-only scaling (no data-path collective), and the reference arm, which
runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


_WORKER = r"""
import os, sys, json
sys.path.insert(0, {root!r})
import bench
d = bench.Dist()
d.init("gloo")
v = d.max(float(d.rank) * 10.0 + 1.0)
d.barrier()
print(json.dumps({{"rank": d.rank, "world": d.world, "max": v}}), flush=True)
d.close()
"""


def test_two_rank_gloo_barrier_and_max():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", _WORKER.format(root=ROOT)],
                                      env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                      text=True))
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e[-2000:]
    res = [json.loads(o.strip().splitlines()[-1]) for o, _ in outs]
    assert sorted(r["rank"] for r in res) == [0, 1]
    assert all(r["world"] == 2 and r["max"] == 11.0 for r in res)


def test_reference_arm_prints_on_rank_zero_only():
    outs = []
    for r in range(2):
        env = dict(os.environ, WORLD_SIZE="2", RANK=str(r), LOCAL_RANK=str(r),
                   OMP_NUM_THREADS="2", CUDA_VISIBLE_DEVICES="")
        p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                            "--gpus", "2", "--workload", "cyl_8960", "--steps", "1",
                            "--warmup", "0", "--cpu-sample", "8"],
                           env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
        assert p.returncode == 0, p.stderr[-2000:]
        outs.append(p.stdout.strip())
    assert outs[1] == ""
    line = json.loads(outs[0].splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0


def test_candidate_test_count_matches_brute_force():
    """bench.candidate_tests (the work unit of the neighbour-search roofline)
    equals a direct count: for every particle that keeps a list, the
    particles whose grid cell lies within one cell of its own on each axis
    (periodic in z), itself included."""
    import numpy as np
    sys.path.insert(0, ROOT)
    import bench
    from paper_2405_03980_gb300 import synth
    c = synth.workload("cyl_8960")
    p = c.params
    lo = np.array(p["box_lo"], dtype=float)
    hi = np.array(p["box_hi"], dtype=float)
    ncell = np.maximum(np.floor((hi - lo) / (2.0 * p["h"])), 1).astype(int)
    cell = np.clip(np.floor((c.pos - lo) / ((hi - lo) / ncell)).astype(int), 0, ncell - 1)
    rows = np.nonzero(c.species != 3)[0]
    total = 0
    for k in range(0, len(rows), 512):  # blocks of rows keep the memory small
        d = np.abs(cell[rows[k:k + 512], None, :] - cell[None, :, :]).astype(np.int32)
        d[:, :, 2] = np.minimum(d[:, :, 2], ncell[2] - d[:, :, 2])
        total += int((d <= 1).all(axis=2).sum())
    assert bench.candidate_tests([c]) == total
