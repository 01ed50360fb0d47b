"""Parity of the pressure filter and the collision model (the two optional
steps of Algorithm 1, flags SPH_PFILTER and SPH_COLLISION) with the CPU FP64
oracle, through the C ABI: the FP64 form to 1e-12 per field (max error over
the max reference value), the mixed form within its one-step relative-L2
target of 2e-5.  The workload is the 8,960-particle cylinder with a collision
distance of 0.95 dx, so that the +-0.05 dx lattice jitter brings many pairs
(fluid-fluid and fluid-wall) inside it."""
import numpy as np
import pytest

import oracle
from paper_2405_03980_gb300 import _binding as B
from paper_2405_03980_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12
L2_TOL = 2e-5
BOTH = B.SPH_PFILTER | B.SPH_COLLISION


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_03980_gb300 import build
    build.build()
    yield


def sim_of(instances, **kw):
    from paper_2405_03980_gb300.sim import Simulation
    return Simulation(instances, **kw)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.abs(a - b).max() / np.abs(b).max()


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def workload(extra, seed=0):
    c = synth.workload("cyl_8960", seed=seed)
    flags = B.SPH_FLAGS_DEFAULT | extra
    c.params = dict(c.params, col_dist=0.95, col_e=0.2, flags=flags)
    return c, flags


def colliding_pairs(c, pos, vel):
    """Approaching fluid-row pairs closer than col_dist, by brute force."""
    p = oracle.make_params(c.params)
    off, nbr = oracle.neighbors(p, pos)
    n_ff = n_fw = 0
    for i in np.nonzero(c.species < 2)[0]:
        js = nbr[off[i]:off[i + 1]]
        d = pos[i] - pos[js]
        d[:, 2] -= c.H * np.round(d[:, 2] / c.H)
        close = (d * d).sum(1) < c.params["col_dist"] ** 2
        appr = ((vel[i] - vel[js]) * d).sum(1) < 0.0
        hit = js[close & appr]
        n_ff += int((c.species[hit] < 2).sum())
        n_fw += int((c.species[hit] >= 2).sum())
    return n_ff, n_fw


@pytest.mark.parametrize("extra", [B.SPH_PFILTER, B.SPH_COLLISION, BOTH])
def test_fp64_extras_match_oracle(extra):
    c, flags = workload(extra)
    sim = sim_of(c)
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species, flags=flags)
    fluid = c.species < 2
    for k in (0, 5):
        if k:
            sim.step(k)
            o.step(k)
        st = sim.state_arrays()
        errs = {"rho": rel(st["rho"], o.rho), "P": rel(st["P"], o.P),
                "acc": rel(st["acc"][fluid], o.acc[fluid]),
                "dspin": rel(st["dspin"][fluid], o.dspin[fluid]),
                "pos": rel(st["pos"], o.pos), "vel": rel(st["vel"], o.vel),
                "spin": rel(st["spin"], o.spin)}
        print(f"extras {extra} after {k} steps, FP64 max relative errors", errs)
        bad = {f: v for f, v in errs.items() if not v <= TOL}
        assert not bad, (k, bad)
    d, od = sim.diagnostics(), o.diagnostics()
    assert d["J_wall"][2] == pytest.approx(od["J_wall"][2], rel=1e-10, abs=1e-10)
    if extra & B.SPH_COLLISION:
        n_ff, n_fw = colliding_pairs(c, o.pos, o.vel)
        assert n_ff > 50 and n_fw > 5, (n_ff, n_fw)
    sim.close()


def test_extras_change_the_result():
    """The options are live: the filtered pressure and the collision force
    differ from the default step's by far more than the tolerance."""
    base = synth.workload("cyl_8960")
    ref = sim_of(base)
    c, _ = workload(BOTH)
    sim = sim_of(c)
    a, b = ref.state_arrays(), sim.state_arrays()
    fluid = base.species < 2
    assert rel(b["P"], a["P"]) > 1e-3
    assert rel(b["acc"][fluid], a["acc"][fluid]) > 1e-3
    assert np.array_equal(b["rho"], a["rho"])
    ref.close()
    sim.close()


@pytest.mark.parametrize("extra", [B.SPH_PFILTER, B.SPH_COLLISION, BOTH])
def test_mixed_extras_within_target(extra):
    c, flags = workload(extra)
    fluid = c.species < 2
    sim = sim_of(c, precision=B.SPH_MIXED)
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species, flags=flags)
    errs = {}
    for k in (0, 1):
        if k:
            sim.step(1)
            o.step(1)
        st = sim.state_arrays()
        errs[k] = {"rho": rel_l2(st["rho"], o.rho), "P": rel_l2(st["P"], o.P),
                   "acc": rel_l2(st["acc"][fluid], o.acc[fluid]),
                   "dspin": rel_l2(st["dspin"][fluid], o.dspin[fluid]),
                   "vel": rel_l2(st["vel"][fluid], o.vel[fluid])}
    print(f"extras {extra}, mixed relative L2 errors", errs)
    bad = {(k, f): v for k in errs for f, v in errs[k].items() if not v <= L2_TOL}
    assert not bad, bad
    sim.close()


def test_mixed_collisions_keep_momentum_in_a_periodic_box():
    """The collision force is bitwise antisymmetric per pair, like the other
    pair terms: the total force of a periodic block vanishes up to the
    rounding of the per-particle sums."""
    pos, vel, spin, sp = synth.periodic_block(8, 8, 8, seed=4, f_v=0.4, vel_sigma=0.2)
    prm = synth.workload_params(4.0, 8, 0.1)
    prm.update(box_lo=(-2.0, -2.0, 0.0), box_hi=(10.0, 10.0, 8.0), C_T=0.5, C_l=0.3,
               col_dist=1.0, col_e=0.3, mass_ratio=2.0,
               flags=B.SPH_FLAGS_DEFAULT | B.SPH_COLLISION)
    c = synth.Cylinder(R=4.0, H=8, dx=1.0, Omega=0.1, f_v=0.4, seed=4, pos=pos, vel=vel,
                       spin=spin, species=sp, params=prm)
    for prec in (B.SPH_MIXED, B.SPH_FP64):
        sim = sim_of(c, precision=prec)
        st = sim.state_arrays()
        p = oracle.make_params(prm)
        m = np.where(sp == 0, oracle.mass(p, 0), oracle.mass(p, 1))[:, None]
        F = st["acc"] * m
        tot = F.sum(0)
        assert np.all(np.abs(tot) < 1e-6 * np.abs(F).sum(0)), (prec, tot)
        sim.close()


def test_batch_with_and_without_extras_matches_solo_runs():
    """One batch mixing an instance with both options and one without runs
    the option-carrying kernels for both.  The instance with the options
    equals its solo run bit for bit (same compiled kernels); the one without
    runs compiled code that differs from its solo run's only in the
    compiler's multiply-add contractions, so it agrees to rounding."""
    c1, _ = workload(BOTH)
    c2 = synth.cylinder(R=5.2, H=10, Omega=0.12, f_v=0.3, seed=11)
    for prec in (B.SPH_FP64, B.SPH_MIXED):
        batch = sim_of([c1, c2], precision=prec)
        batch.step(3)
        bst = batch.state_arrays()
        off = 0
        for k, c in enumerate((c1, c2)):
            solo = sim_of(c, precision=prec)
            solo.step(3)
            s = solo.state_arrays()
            for f in ("pos", "vel", "spin", "rho", "P", "acc", "dspin"):
                got = bst[f][off:off + c.n]
                if k == 0:
                    assert np.array_equal(got, s[f]), (prec, f)
                else:
                    tol = 1e-13 if prec == B.SPH_FP64 else 1e-5
                    assert rel(got, s[f]) <= tol, (prec, f, rel(got, s[f]))
            solo.close()
            off += c.n
        batch.close()
