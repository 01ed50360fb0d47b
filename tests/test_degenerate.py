"""Degenerate inputs: an isolated particle, two coincident particles, a pair
exactly at the support radius 2h, a pair that meets only across the periodic
z boundary, and a system of one particle.

The CPU tests pin the oracle on these cases to closed forms: a particle with
no neighbour has the density of its own kernel term, rho = m W(0), and feels
no force (Sec. 2.1: every force of Eqs. 1-2 is a sum over neighbour pairs);
coincident particles count W(0) for each other in the density summation but
exert no pair force (the pair direction r_ij / |r_ij| does not exist; the
discrete forces are all proportional to r_ij or to F_ij (I - e e) u_ij with
no radial direction); a pair at distance exactly 2h is not a pair (the
Wendland C2 kernel has compact support r < 2h).  The GPU tests then run the
same instances through the C ABI in both state forms and compare every field
with the oracle: FP64 to 1e-12 of the largest value, mixed within the
2e-5 relative L2 bar of the mixed form (max-normalised here, since several
fields are zero for most of these particles).
"""
import numpy as np
import pytest

import oracle
from paper_2405_03980_gb300 import synth

INV, VIS = synth.INVISCID, synth.VISCOUS


def sparse_instance():
    """Eight fluid particles in a 16 x 16 x 12 box, periodic in z (h = 1.3):
    0 and 1 at distance exactly 2h (doubling h is exact, so r^2 equals the
    cut-off (2h)^2 bit for bit and the pair is excluded); 2 alone; 3 and 4 at
    the same point, with 5 at distance 1.1 of both; 6 and 7 at distance 0.8
    across the z period only."""
    prm = synth.workload_params(5.0, 12, 0.1)
    h = prm["h"]
    prm.update(box_lo=(-8.0, -8.0, 0.0), box_hi=(8.0, 8.0, 12.0), periodic_z=1,
               C_T=0.05 * prm["p0"], C_l=0.2)
    pos = np.array([
        [0.0, -5.0, 2.0],
        [2.0 * h, -5.0, 2.0],
        [-5.0, -5.0, 8.0],
        [3.0, 3.0, 6.0],
        [3.0, 3.0, 6.0],
        [4.1, 3.0, 6.0],
        [-5.0, 5.0, 0.3],
        [-5.0, 5.0, 11.5],
    ])
    species = np.array([INV, VIS, VIS, INV, VIS, VIS, INV, VIS], dtype=np.uint8)
    rng = np.random.Generator(np.random.PCG64(11))
    vel = rng.normal(0.0, 0.05, size=(8, 3))
    spin = rng.normal(0.0, 0.05, size=(8, 3))
    return synth.Cylinder(R=5.0, H=12, dx=1.0, Omega=0.1, f_v=0.5, seed=11, pos=pos,
                          vel=vel, spin=spin, species=species, params=prm)


def single_instance():
    """One fluid particle in a periodic box."""
    c = sparse_instance()
    return synth.Cylinder(R=c.R, H=c.H, dx=c.dx, Omega=c.Omega, f_v=c.f_v, seed=c.seed,
                          pos=c.pos[2:3].copy(), vel=c.vel[2:3].copy(),
                          spin=c.spin[2:3].copy(), species=c.species[2:3].copy(),
                          params=dict(c.params))


def _self_density(p, species):
    return oracle.mass(p, int(species)) * oracle.W(p, 0.0)


def test_oracle_neighbours_of_the_degenerate_instance():
    c = sparse_instance()
    p = oracle.make_params(c.params)
    off, nbr = oracle.neighbors(p, c.pos)
    sets = [sorted(nbr[off[i]:off[i + 1]].tolist()) for i in range(c.n)]
    assert sets == [[], [], [], [4, 5], [3, 5], [3, 4], [7], [6]]


def test_oracle_isolated_and_cutoff_particles_are_free():
    c = sparse_instance()
    p = oracle.make_params(c.params)
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    for i in (0, 1, 2):
        assert o.rho[i] == pytest.approx(_self_density(p, c.species[i]), rel=1e-15)
        assert np.all(o.acc[i] == 0.0) and np.all(o.dspin[i] == 0.0)
    # a free particle moves ballistically with a constant spin
    x0, v0, w0 = o.pos[2].copy(), o.vel[2].copy(), o.spin[2].copy()
    o.step(3)
    assert np.allclose(o.pos[2], x0 + 3 * p.dt * v0, rtol=0, atol=1e-14)
    assert np.array_equal(o.vel[2], v0) and np.array_equal(o.spin[2], w0)


def test_oracle_coincident_pair_counts_for_density_only():
    c = sparse_instance()
    p = oracle.make_params(c.params)
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    r = 1.1
    w0 = oracle.W(p, 0.0)
    for i, j in ((3, 4), (4, 3)):
        want = (oracle.mass(p, int(c.species[i])) * w0 + oracle.mass(p, int(c.species[j])) * w0
                + oracle.mass(p, int(c.species[5])) * oracle.W(p, r))
        assert o.rho[i] == pytest.approx(want, rel=1e-14)
    # without 5 the coincident pair alone feels nothing
    keep = [3, 4]
    o2 = oracle.Sim(c.params, c.pos[keep], c.vel[keep], c.spin[keep], c.species[keep])
    assert np.all(o2.acc == 0.0) and np.all(o2.dspin == 0.0)
    assert o2.rho[0] == pytest.approx(2 * oracle.mass(p, INV) * w0, rel=1e-15)


def test_oracle_pair_across_the_z_period_matches_the_direct_pair():
    """Particles 6 and 7 meet only through the periodic image; moving 7 to
    its image position (z - 12) gives the same pair in an open box."""
    c = sparse_instance()
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    keep = [6, 7]
    pos = c.pos[keep].copy()
    pos[1, 2] -= 12.0
    prm = dict(c.params, periodic_z=0, box_lo=(-8.0, -8.0, -6.0), box_hi=(8.0, 8.0, 6.0))
    o2 = oracle.Sim(prm, pos, c.vel[keep], c.spin[keep], c.species[keep])
    for a, b in ((o.rho[keep], o2.rho), (o.P[keep], o2.P), (o.acc[keep], o2.acc),
                 (o.dspin[keep], o2.dspin)):
        assert np.allclose(a, b, rtol=1e-13, atol=1e-15)
    assert np.any(o2.acc != 0.0)


def test_oracle_single_particle():
    c = single_instance()
    p = oracle.make_params(c.params)
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    assert o.rho[0] == pytest.approx(_self_density(p, c.species[0]), rel=1e-15)
    assert np.all(o.acc == 0.0) and np.all(o.dspin == 0.0)


# ---------------------------------------------------------------- GPU parity

def _gpu_ready():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_03980_gb300 import build
    build.build()


def _max_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    s = np.abs(b).max()
    return np.abs(a - b).max() / s if s > 0 else np.abs(a).max()


@pytest.mark.gpu
@pytest.mark.parametrize("make", [sparse_instance, single_instance])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("mixed", 2e-5)])
def test_degenerate_instances_match_oracle(make, precision, tol):
    _gpu_ready()
    from paper_2405_03980_gb300 import _binding as B
    from paper_2405_03980_gb300.sim import Simulation
    c = make()
    prec = B.SPH_FP64 if precision == "fp64" else B.SPH_MIXED
    sim = Simulation(c, precision=prec, device="cuda:0")
    o = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    for steps in (0, 3):
        if steps:
            sim.step(steps)
            o.step(steps)
        st = sim.state_arrays()
        ref = {"pos": o.pos, "vel": o.vel, "spin": o.spin, "rho": o.rho, "P": o.P,
               "acc": o.acc, "dspin": o.dspin}
        errs = {k: _max_rel(st[k], r) for k, r in ref.items()}
        bad = {k: v for k, v in errs.items() if not v <= tol}
        assert not bad, f"{precision} after {steps} steps: {bad} (all: {errs})"
        # particles without a neighbour feel exactly nothing in either form
        free = [2] if c.n == 8 else [0]
        assert np.all(st["acc"][free] == 0.0) and np.all(st["dspin"][free] == 0.0)
    sim.close()
