"""Parity of the FP64 CUDA path with the CPU FP64 oracle, through the C ABI.

Tolerance: the FP64 path must match the oracle to 1e-12 per field, measured as
max_i |x_gpu,i - x_oracle,i| / max_i |x_oracle,i| (the two sum in different
orders and the GPU contracts multiply-adds, so only round-off may differ), and
its neighbour sets must equal the oracle's brute-force sets exactly.

Fields whose pair sums nearly cancel (the acceleration of an interior
particle) are also held to a per-particle bound on the same state:
|a_gpu,i - a_oracle,i| <= 1e-12 sum_j |f_ij| / m_i and the same for the spin
change with sum_j |tau_ij| / I_i, the oracle computing both sums; the
pressure of each particle within 1e-12 of its Tait sensitivity
alpha_P p0 (rho_i / rho0)^alpha_P (the pressure error a relative density
error of 1 would cause).  A reordered summation in FP64 stays about 30 times
below these bars (the oracle against itself on a permuted particle order).
Every field of sph_diagnostics is compared with the oracle's diagnostics.
"""
import numpy as np
import pytest

import oracle
from paper_2405_03980_gb300 import _binding as B
from paper_2405_03980_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-12


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
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.abs(b).max()
    if scale == 0.0:
        return np.abs(a).max()
    return np.abs(a - b).max() / scale


def check_fields(st, o, fluid, tol=TOL, fields=("pos", "vel", "spin", "rho", "P", "acc", "dspin")):
    ref = {"pos": o.pos, "vel": o.vel, "spin": o.spin, "rho": o.rho, "P": o.P,
           "acc": o.acc, "dspin": o.dspin}
    errs = {}
    for k in fields:
        a, b = st[k], ref[k]
        if k in ("acc", "dspin"):
            a, b = a[fluid], b[fluid]
        errs[k] = rel(a, b)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"fields above {tol}: {bad} (all: {errs})"
    return errs


def per_particle_check(st, c, after_steps, tol=TOL):
    """Per-particle parity on the GPU's own state: the oracle re-derives the
    density, pressure and pair forces from the returned positions and (after
    steps) the half-step velocities v - dt/2 a that the last pair pass used.
    Returns the largest error of each field relative to its per-row bound."""
    p = oracle.make_params(c.params)
    pos = st["pos"]
    rho, P = oracle.density(p, pos, c.species)
    fl = c.species < 2
    vh, wh = st["vel"].copy(), st["spin"].copy()
    if after_steps:
        hdt = 0.5 * c.params["dt"]
        vh[fl] -= hdt * st["acc"][fl]
        wh[fl] -= hdt * st["dspin"][fl]
    acc, dsp, _, sc = oracle.forces(p, pos, vh, wh, c.species, rho, P, scale=True)
    eos = p.alpha_P * p.p0 * (rho / p.rho0) ** p.alpha_P
    worst = {
        "rho": (np.abs(st["rho"] - rho) / rho).max(),
        "P": (np.abs(st["P"] - P) / eos).max(),
        "acc": (np.linalg.norm(st["acc"][fl] - acc[fl], axis=1) / sc[fl, 0]).max(),
        "dspin": (np.linalg.norm(st["dspin"][fl] - dsp[fl], axis=1) / sc[fl, 1]).max(),
    }
    bad = {k: v for k, v in worst.items() if not v <= tol}
    assert not bad, f"per-particle bounds above {tol}: {bad} (all: {worst})"
    return worst


def check_diagnostics(d, od, st, c, tol=TOL):
    """Every sph_diagnostics field against orc_diagnostics: scalar sums and
    extrema relative to themselves, vector sums relative to the sum of the
    magnitudes they add (so near-zero totals such as the linear momentum are
    held to round-off of their terms)."""
    fl = c.species < 2
    p = oracle.make_params(c.params)
    m = np.where(c.species == 0, oracle.mass(p, 0), oracle.mass(p, 1))[fl]
    I = p.inertia_coef * m * p.dx ** 2
    r, v, w = st["pos"][fl], st["vel"][fl], st["spin"][fl]
    scales = {"mom": (m * np.linalg.norm(v, axis=1)).sum(),
              "L_orb": (m * np.linalg.norm(np.cross(r, v), axis=1)).sum(),
              "L_spin": (I * np.linalg.norm(w, axis=1)).sum()}
    for k in ("mass", "mass_s", "mass_n", "E_kin", "E_rot", "E_int", "rho_min", "rho_max",
              "v_max"):
        assert d[k] == pytest.approx(od[k], rel=tol, abs=1e-300), k
    for k, sc in scales.items():
        assert np.all(np.abs(np.subtract(d[k], od[k])) <= tol * sc), (k, d[k], od[k])
    assert d["n_pairs"] == od["n_pairs"]
    tw = np.abs(od["T_wall"]).max()
    assert np.allclose(d["T_wall"], od["T_wall"], rtol=0, atol=1e-11 * tw), "T_wall"
    jw = np.abs(od["J_wall"]).max()
    assert np.allclose(d["J_wall"], od["J_wall"], rtol=0, atol=1e-10 * jw + 1e-300), "J_wall"


def compare_neighbours(sim, species, p):
    st = sim.state_arrays()
    sim.density()
    off_g, nbr_g = sim.neighbors()
    off_o, nbr_o = oracle.neighbors(p, st["pos"])
    n = len(species)
    outer = species == 3
    for i in range(n):
        g = nbr_g[off_g[i]:off_g[i + 1]]
        if outer[i]:
            assert len(g) == 0
            continue
        o = nbr_o[off_o[i]:off_o[i + 1]]
        assert np.array_equal(g, o), f"particle {i}: {len(g)} vs {len(o)} neighbours"


def test_initial_evaluation_matches_oracle():
    c = synth.workload("cyl_8960")
    sim = sim_of(c)
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    st = sim.state_arrays()
    fluid = c.species < 2
    errs = check_fields(st, o, fluid)
    print("t=0 errors", errs)
    print("t=0 per-particle", per_particle_check(st, c, after_steps=False))
    # FP64 sums over 6,320 fluid particles in another order: 1e-12 relative
    check_diagnostics(sim.diagnostics(), o.diagnostics(), st, c)
    sim.close()


def test_neighbour_sets_bit_exact():
    c = synth.workload("cyl_8960")
    sim = sim_of(c)
    p = oracle.make_params(c.params)
    compare_neighbours(sim, c.species, p)
    sim.step(3)
    compare_neighbours(sim, c.species, p)
    sim.close()


def test_ten_steps_match_oracle():
    c = synth.workload("cyl_8960")
    sim = sim_of(c)
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    sim.step(10)
    o.step(10)
    st = sim.state_arrays()
    errs = check_fields(st, o, c.species < 2)
    print("10-step errors", errs)
    print("10-step per-particle", per_particle_check(st, c, after_steps=True))
    d = sim.diagnostics()
    od = o.diagnostics()
    assert d["step"] == 10
    assert d["theta"] == pytest.approx(o.theta.value, rel=0, abs=0)
    # the two trajectories differ by round-off, so the diagnostics of the
    # oracle's own state are compared at the state's 1e-12 agreement
    check_diagnostics(d, od, st, c, tol=1e-11)
    for a in range(3):
        assert d["L_orb"][a] + d["L_spin"][a] == pytest.approx(
            od["L_orb"][a] + od["L_spin"][a], rel=1e-11, abs=1e-9)
        assert d["J_wall"][a] == pytest.approx(od["J_wall"][a], rel=1e-10, abs=1e-10)
    # angular-momentum budget of the driven vessel on the GPU itself
    d0 = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species).diagnostics()
    Lz0 = d0["L_orb"][2] + d0["L_spin"][2]
    Lz = d["L_orb"][2] + d["L_spin"][2]
    assert Lz - Lz0 == pytest.approx(d["J_wall"][2], rel=1e-8)
    sim.close()


@pytest.mark.parametrize("flags", [B.SPH_TERM_P, B.SPH_TERM_T | B.SPH_HPROJ, B.SPH_TERM_T,
                                   B.SPH_TERM_SH, B.SPH_TERM_ROT, B.SPH_TERM_SN,
                                   B.SPH_TERM_SN | B.SPH_SN_LITERAL, B.SPH_FLAGS_DEFAULT])
def test_each_term_matches_oracle(flags):
    c = synth.workload("cyl_8960", seed=3)
    prm = dict(c.params, C_l=0.5, C_T=2.0, flags=flags)
    c.params = prm
    sim = sim_of(c)
    o = oracle.Sim(prm, c.pos, c.vel, c.spin, c.species, flags=flags)
    sim.step(2)
    o.step(2)
    check_fields(sim.state_arrays(), o, c.species < 2)
    sim.close()


def test_small_ragged_instance_and_open_z():
    # a 4-cell-wide cylinder with a non-periodic z: ragged cells, empty cells,
    # particles touching the grid ghosts' neighbours
    c = synth.cylinder(R=3.3, H=7, Omega=0.2, f_v=0.5, seed=5)
    prm = dict(c.params, periodic_z=0, box_lo=(c.params["box_lo"][0], c.params["box_lo"][1], -3.0),
               box_hi=(c.params["box_hi"][0], c.params["box_hi"][1], 10.0))
    c.params = prm
    sim = sim_of(c)
    o = oracle.Sim(prm, c.pos, c.vel, c.spin, c.species)
    sim.step(4)
    o.step(4)
    check_fields(sim.state_arrays(), o, c.species < 2)
    sim.close()


def test_batch_equals_solo_runs_bitwise():
    cs = [synth.cylinder(R=r, H=h, Omega=om, f_v=fv, seed=s)
          for r, h, om, fv, s in [(4.2, 9, 0.15, 0.2, 1), (7.0, 12, 0.08, 0.45, 2),
                                  (3.1, 8, 0.19, 0.05, 3)]]
    batch = sim_of(cs)
    batch.step(5)
    bst = batch.state_arrays()
    off = 0
    for k, c in enumerate(cs):
        solo = sim_of(c)
        solo.step(5)
        s = solo.state_arrays()
        for f in ("pos", "vel", "spin", "rho", "P", "acc", "dspin"):
            assert np.array_equal(bst[f][off:off + c.n], s[f]), (k, f)
        db = batch.diagnostics(k)
        ds = solo.diagnostics(0)
        for key in ("mass", "E_kin", "E_int", "L_orb", "J_wall", "theta", "step", "n_pairs"):
            assert db[key] == ds[key], (k, key)
        solo.close()
        off += c.n
    batch.close()


@pytest.mark.parametrize("precision", [B.SPH_FP64, B.SPH_MIXED])
def test_rerun_is_deterministic(precision):
    """Reruns and split step calls give the same bits.  (The mixed form's step
    graphs leave each step's closing half kick to the next step's drift and
    the call's end: one call of 6 steps, two of 3 and six of 1 must agree.)"""
    c = synth.workload("cyl_8960", seed=7)
    a = sim_of(c, precision=precision)
    a.step(6)
    b = sim_of(c, precision=precision)
    b.step(3)
    b.step(3)
    d = sim_of(c, precision=precision)
    for _ in range(6):
        d.step(1)
    sa, sb, sd = a.state_arrays(), b.state_arrays(), d.state_arrays()
    for f in sa:
        assert np.array_equal(sa[f], sb[f]), f
        assert np.array_equal(sa[f], sd[f]), f
    for s in (a, b, d):
        s.close()


def test_device_errors_are_latched_not_trapped():
    c = synth.workload("cyl_8960")
    fluid = np.nonzero(c.species < 2)[0]
    # a fluid particle far outside the cell grid: clamped, reported as escaped
    pos = c.pos.copy()
    pos[fluid[5]] = [1e3, 0.0, 1.0]
    bad = synth.Cylinder(**{**c.__dict__, "pos": pos})
    with pytest.raises(B.SphError) as e:
        sim_of(bad)
    assert e.value.status == -5
    # a NaN velocity of a fluid particle: reported as non-finite (the initial
    # force evaluation already propagates it)
    vel = c.vel.copy()
    vel[fluid[7], 1] = np.nan
    bad = synth.Cylinder(**{**c.__dict__, "vel": vel})
    sim = None
    with pytest.raises(B.SphError) as e:
        sim = sim_of(bad)
        sim.step(1)
        sim.check()
    assert e.value.status in (-6, -5)
    # the context stays usable: a fresh simulation on the same device works
    ok = sim_of(c)
    ok.step(1)
    ok.check()
    ok.close()


@pytest.mark.parametrize("precision,tol", [(B.SPH_FP64, 1e-10), (B.SPH_MIXED, 1e-4)])
def test_force_breakdown_matches_oracle(precision, tol):
    """sph_force_breakdown: sum_i |f_i^term| of the pressure, interfacial,
    shear, rotational and local-interaction terms (the force breakdown of
    Sec. 4) equals the oracle's term sums for the same state.  The FP64 form
    agrees to round-off; the mixed form's state is FP32, read the same way by
    both sides, and its neighbour sets differ from the FP64 ones only at the
    cutoff, where the terms vanish."""
    c = synth.workload("cyl_8960")
    sim = sim_of(c, precision=precision)
    sim.step(3)
    got = sim.force_breakdown()
    st = sim.state_arrays()
    p = oracle.make_params(c.params)
    _, _, _, mag = oracle.forces(p, st["pos"], st["vel"], st["spin"], c.species, st["rho"],
                                 st["P"], term_mag=True)
    sim.close()
    assert np.all(mag > 0)
    assert np.all(np.abs(got - mag) <= tol * mag), (got, mag)


@pytest.mark.parametrize("precision", [B.SPH_FP64, B.SPH_MIXED])
def test_neighbour_overflows_are_latched(precision):
    """About 80 neighbours against a list capacity of 64, and a cluster whose
    27-cell stencil holds more particles than the candidate table (1024):
    both are reported as SPH_ERR_NEIGHBORS, without a fault, and the context
    stays usable."""
    c = synth.workload("cyl_8960")
    with pytest.raises(B.SphError) as e:
        s = sim_of(c, precision=precision, nbr_cap=64)
        s.check()
    assert e.value.status == -9
    if precision == B.SPH_FP64:
        # 1200 fluid particles packed into one cell of side 2h at the centre
        rng = np.random.default_rng(3)
        pos = c.pos.copy()
        fluid = np.nonzero(c.species < 2)[0][:1200]
        h = c.params["h"]
        pos[fluid] = rng.uniform(-0.9 * h, 0.9 * h, size=(len(fluid), 3)) + [0.0, 0.0, 10.0]
        dense = synth.Cylinder(**{**c.__dict__, "pos": pos})
        with pytest.raises(B.SphError) as e:
            s = sim_of(dense, precision=precision, nbr_cap=1024)
            s.check()
        assert e.value.status == -9
    ok = sim_of(c, precision=precision)
    ok.step(1)
    ok.check()
    ok.close()


@pytest.mark.parametrize("precision", [B.SPH_FP64, B.SPH_MIXED])
@pytest.mark.parametrize("extras", [0, B.SPH_PFILTER | B.SPH_COLLISION])
def test_autotune_leaves_state_and_results_unchanged(precision, extras):
    """The autotuner times launch shapes on the current state; per-particle
    results do not depend on the block size, so the state after tuning and the
    trajectory that follows are bit-identical to an untuned run (also with
    the pressure filter and the collision model on)."""
    c = synth.workload("cyl_8960", seed=4)
    if extras:
        c.params = dict(c.params, col_dist=0.95, flags=B.SPH_FLAGS_DEFAULT | extras)
    a = sim_of(c, precision=precision)
    b = sim_of(c, precision=precision)
    a.step(2)
    b.step(2)
    bd, bf = b.autotune(2)
    assert bd in (32, 64, 128) and bf in (64, 128, 256)
    sa, sb = a.state_arrays(), b.state_arrays()
    for f in sa:
        assert np.array_equal(sa[f], sb[f]), f
    a.step(3)
    b.step(3)
    sa, sb = a.state_arrays(), b.state_arrays()
    for f in sa:
        assert np.array_equal(sa[f], sb[f]), f
    a.close()
    b.close()


@pytest.mark.parametrize("precision", [B.SPH_FP64, B.SPH_MIXED])
def test_checkpoint_resume_is_bit_identical(precision, tmp_path):
    """Saving after 4 steps and resuming in a fresh context gives, after 5
    more steps, exactly the state, diagnostics and wall budget of the
    uninterrupted run; mismatched contexts and corrupt checkpoints are
    refused without touching the target."""
    c = synth.workload("cyl_8960", seed=2)
    a = sim_of(c, precision=precision)
    a.step(4)
    path = str(tmp_path / "ck.bin")
    ck = a.save_checkpoint(path)
    assert ck.nbytes == B.sph_checkpoint_bytes(a.ctx)
    a.step(5)
    sa, da = a.state_arrays(), a.diagnostics()
    b = sim_of(c, precision=precision)
    b.step(1)  # a context with another history: the load replaces all of it
    b.load_checkpoint(path)
    b.step(5)
    sb, db = b.state_arrays(), b.diagnostics()
    for f in sa:
        assert np.array_equal(sa[f], sb[f]), f
    for k in ("step", "theta", "J_wall", "T_wall", "L_orb", "L_spin", "E_kin", "mass"):
        assert da[k] == db[k], k
    assert da["step"] == 9
    # another parameter set, another precision, a truncated or corrupt buffer
    other = synth.workload("cyl_8960", seed=2)
    other.params = dict(other.params, C_T=2.0 * other.params["C_T"])
    o = sim_of(other, precision=precision)
    with pytest.raises(B.SphError):
        o.load_checkpoint(ck)
    with pytest.raises(B.SphError):
        b.load_checkpoint(ck[:-8])
    bad = ck.copy()
    bad[0] ^= 0xFF
    with pytest.raises(B.SphError):
        b.load_checkpoint(bad)
    q = sim_of(c, precision=B.SPH_MIXED if precision == B.SPH_FP64 else B.SPH_FP64)
    with pytest.raises(B.SphError):
        q.load_checkpoint(ck)
    # the refused loads left b as it was
    assert np.array_equal(b.state_arrays()["pos"], sb["pos"])
    for s in (a, b, o, q):
        s.close()


@pytest.mark.parametrize("precision", [B.SPH_FP64, B.SPH_MIXED])
def test_search_mappings_give_identical_results(precision):
    """The thread-per-particle neighbour search writes the same masks and
    candidate tables as the warp-per-cell one (both classify a candidate with
    the same FP32 expression), so neighbour lists, fields and the trajectory
    are bit-identical; on the periodic 8,960 cylinder and on a small ragged
    cylinder with an open z range."""
    rag = synth.cylinder(R=3.3, H=7, Omega=0.2, f_v=0.5, seed=5)
    rag.params = dict(rag.params, periodic_z=0,
                      box_lo=(rag.params["box_lo"][0], rag.params["box_lo"][1], -3.0),
                      box_hi=(rag.params["box_hi"][0], rag.params["box_hi"][1], 10.0))
    for c in (synth.workload("cyl_8960", seed=7), rag):
        a = sim_of(c, precision=precision)  # 4 cells per block, depth 512
        others = [sim_of(c, precision=precision) for _ in range(2)]
        others[0].set_launch_config(64, 128, 0)         # thread per particle
        others[1].set_launch_config(32, 256, 2, 256)    # 2 cells per block, depth 256
        assert others[0].launch_config()["search_warps"] == 0
        assert others[1].launch_config()["search_depth"] == 256
        for _ in range(2):
            a.step(2)
            sa = a.state_arrays()
            for b in others:
                b.step(2)
                sb = b.state_arrays()
                for f in sa:
                    assert np.array_equal(sa[f], sb[f]), f
        oa, na = a.neighbors()
        for b in others:
            ob, nb = b.neighbors()
            assert np.array_equal(oa, ob) and np.array_equal(na, nb)
        with pytest.raises(B.SphError):
            others[0].set_launch_config(64, 128, 3)
        with pytest.raises(B.SphError):
            others[0].set_launch_config(64, 128, 4, 384)
        for s_ in [a] + others:
            s_.close()
