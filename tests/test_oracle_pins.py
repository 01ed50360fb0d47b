"""Pins of the CPU FP64 oracle against what the paper and the mathematics fix.

Each test pins one part of the oracle to something other than itself: a
quadrature, a finite difference, a k-d tree, a closed-form lattice count, a
conservation law the paper asserts (Sec. 2.1: total mass M = M_s + M_n; the
interfacial forces of Eqs. 1-2 act in opposite directions on the two
components; F_sn acts with its reaction on the other species; rigid rotation
produces no rotational stress), the continuum limit of Eq. 2, or a property of
the velocity Verlet integrator (Sec. 2.3).  A plausible slip in the oracle (a
dropped term, a wrong sign, factor or index) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2405_03980_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(h_over_dx=1.3, periodic_z=1, Hz=20.0, dx=1.0, **kw):
    p = synth.workload_params(10.0, Hz, 0.1, dx=dx, h_over_dx=h_over_dx)
    p.update(periodic_z=periodic_z, box_lo=(-50.0, -50.0, 0.0), box_hi=(50.0, 50.0, Hz))
    p.update(kw)
    return p


def _lattice(n, spacing=1.0):
    g = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return (g.astype(np.float64) - (n - 1) / 2.0) * spacing


# ---------------------------------------------------------------- kernel (M0)

@pytest.mark.parametrize("h", [0.7, 1.3, 2.1])
def test_kernel_normalised_by_quadrature(h):
    from scipy.integrate import quad
    p = oracle.make_params(_params(h_over_dx=h))
    val, _ = quad(lambda r: 4.0 * math.pi * r * r * oracle.W(p, r), 0.0, 2.0 * h,
                  epsabs=1e-14, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-12
    assert oracle.W(p, 2.0 * h) == 0.0 and oracle.W(p, 2.0 * h * 1.0001) == 0.0


def test_kernel_gradient_matches_finite_difference():
    p = oracle.make_params(_params())
    for r in np.linspace(0.05, 2.55, 37):
        eps = 1e-6
        dW = (oracle.W(p, r + eps) - oracle.W(p, r - eps)) / (2 * eps)
        assert oracle.F(p, r) == pytest.approx(-dW / r, rel=1e-7, abs=1e-12)
        assert oracle.F(p, r) >= 0.0


def test_lattice_sum_golden_and_neighbour_count():
    # Golden: sum_n W(|n| dx) on the unit cubic lattice at h = 1.3 dx, evaluated
    # independently when the workload was specified (tests/golden/lattice_sum.txt).
    with open(os.path.join(GOLDEN, "lattice_sum.txt")) as f:
        golden = float([l for l in f if not l.startswith("#")][0])
    p = oracle.make_params(_params())
    assert oracle.lattice_sum(p) == pytest.approx(golden, rel=1e-14)
    # closed form: integer points with |n|^2 < (2h)^2 = 6.76 -> 1+6+12+8+6+24+24 = 81
    pos = _lattice(9)
    off, nbr = oracle.neighbors(oracle.make_params(_params(periodic_z=0)), pos)
    c = int(np.argmin((pos ** 2).sum(1)))
    assert off[c + 1] - off[c] == 80


def test_rest_density_on_unjittered_lattice():
    """M1 with the lattice mass: interior particles have rho = rho0 exactly,
    and the mass of a particle is rho0 / lattice sum (Sec. 2.1 equal volumes)."""
    p = oracle.make_params(_params(periodic_z=0))
    pos = _lattice(9)
    sp = np.ones(len(pos), np.uint8)
    rho, P = oracle.density(p, pos, sp)
    interior = np.all(np.abs(pos) <= 1.0 + 1e-9, axis=1)
    assert np.allclose(rho[interior], 1.0, rtol=0, atol=4e-15)
    assert np.allclose(P[interior], 0.0, atol=1e-12 * p.p0)
    # particles on the outer shell see fewer neighbours (no wall): lower density
    shell = np.abs(pos).max(1) >= 4.0
    assert rho[shell].max() < 1.0
    # density with unequal species masses counts the mass of each neighbour
    p2 = oracle.make_params(_params(periodic_z=0, mass_ratio=5.0))
    sp2 = np.zeros(len(pos), np.uint8)
    rho2, _ = oracle.density(p2, pos, sp2)
    assert rho2[interior] == pytest.approx(5.0 * rho[interior], rel=1e-14)
    # one inviscid particle among viscous ones: its neighbours bring m_n each
    # and only the self term carries m_s, so rho = rho0 + (m_s - m_n) W(0)
    c = int(np.argmin((pos ** 2).sum(1)))
    sp3 = np.ones(len(pos), np.uint8)
    sp3[c] = 0
    rho3, _ = oracle.density(p2, pos, sp3)
    m_s, m_n = oracle.mass(p2, 0), oracle.mass(p2, 1)
    assert rho3[c] == pytest.approx(1.0 + (m_s - m_n) * oracle.W(p2, 0.0), rel=1e-13)
    # walls are particles of the normal fluid (Sec. 3): as neighbours, inner
    # and outer walls alike bring m_n, and a lattice of inner walls alone sits
    # at rho0 whatever the species mass ratio
    sp4 = np.where(np.arange(len(pos)) % 2 == 0, 2, 3).astype(np.uint8)
    sp4[c] = 0
    rho4, _ = oracle.density(p2, pos, sp4)
    assert rho4[c] == pytest.approx(1.0 + (m_s - m_n) * oracle.W(p2, 0.0), rel=1e-13)
    rho5, _ = oracle.density(p2, pos, np.full(len(pos), 2, np.uint8))
    assert np.allclose(rho5[interior], 1.0, rtol=0, atol=4e-15)


def test_neighbours_match_kdtree_with_periodic_z():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(7)
    Hz = 9.0
    n = 600
    pos = np.column_stack([rng.uniform(0, 8, n), rng.uniform(0, 8, n), rng.uniform(0, Hz, n)])
    p = oracle.make_params(_params(Hz=Hz))
    off, nbr = oracle.neighbors(p, pos)
    tree = cKDTree(pos + np.array([100.0, 100.0, 0.0]), boxsize=[1000.0, 1000.0, Hz])
    pairs = tree.query_pairs(2.0 * p.h, output_type="ndarray")
    want = set(map(tuple, pairs)) | set((b, a) for a, b in pairs)
    got = set((i, int(j)) for i in range(n) for j in nbr[off[i]:off[i + 1]])
    assert got == want
    # a pair exactly at the cutoff distance is not a neighbour (strict r < 2h)
    two = np.array([[0.0, 0.0, 1.0], [2.0 * p.h, 0.0, 1.0]])
    o2, _ = oracle.neighbors(p, two)
    assert o2[-1] == 0


def test_z_minimum_image():
    p = oracle.make_params(_params(Hz=12.0))
    a = np.array([[0.3, 0.1, 0.4], [0.9, -0.2, 11.5]])    # across z = 0 / H
    b = a.copy()
    b[:, 2] = [6.4, 5.5]                                   # same pair, interior
    sp = np.array([0, 1], np.uint8)
    ra, Pa = oracle.density(p, a, sp)
    rb, Pb = oracle.density(p, b, sp)
    assert np.allclose(ra, rb, rtol=1e-15)
    v = np.array([[0.1, 0.0, 0.2], [-0.1, 0.3, 0.0]])
    w = np.array([[0.0, 0.1, 0.0], [0.2, 0.0, -0.1]])
    fa = oracle.forces(p, a, v, w, sp, ra, Pa)
    fb = oracle.forces(p, b, v, w, sp, rb, Pb)
    for x, y in zip(fa[:2], fb[:2]):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ EOS (M2)

def test_tait_eos_binomial_form():
    """Eq. 4 with beta_P = p0 (Sec. 2.1): P(rho0) = 0 and
    P = p0 * delta (7 + 21 d + 35 d^2 + 35 d^3 + 21 d^4 + 7 d^5 + d^6)."""
    p = oracle.make_params(_params(periodic_z=0))
    m = oracle.mass(p, 1)
    for r in [0.4, 1.0, 1.7, 2.3]:
        pos = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
        sp = np.array([1, 1], np.uint8)
        rho, P = oracle.density(p, pos, sp)
        d = rho[0] / p.rho0 - 1.0
        binom = p.p0 * d * (7 + d * (21 + d * (35 + d * (35 + d * (21 + d * (7 + d))))))
        assert P[0] == pytest.approx(binom, rel=1e-10)
        assert rho[0] == pytest.approx(m * (oracle.W(p, 0.0) + oracle.W(p, r)), rel=1e-15)
    # outer walls keep the initial density and pressure
    pos = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    rho, P = oracle.density(p, pos, np.array([3, 2], np.uint8))
    assert rho[0] == p.rho0 and P[0] == 0.0 and rho[1] != p.rho0


# ------------------------------------------------------ pairwise forces (M3-M8)

def _block(nx=6, ny=6, nz=6, seed=3, f_v=0.4):
    return synth.periodic_block(nx, ny, nz, seed=seed, f_v=f_v, vel_sigma=0.2)


def test_linear_momentum_zero_sum_periodic():
    pos, vel, spin, sp = _block()
    p = oracle.make_params(_params(Hz=6.0, C_T=0.3, C_l=0.7), flags=oracle.TERMS_ALL | oracle.HPROJ)
    rho, P = oracle.density(p, pos, sp)
    acc, dsp, _ = oracle.forces(p, pos, vel, spin, sp, rho, P)
    m = np.where(sp == 0, oracle.mass(p, 0), oracle.mass(p, 1))[:, None]
    tot = (m * acc).sum(0)
    scale = np.abs(m * acc).sum()
    assert np.all(np.abs(tot) < 1e-13 * scale)


def _angular_residual(flags):
    pos, vel, spin, sp = _block(seed=11)
    pos = pos - pos.mean(0)
    p = oracle.make_params(_params(periodic_z=0, C_T=0.3, C_l=0.7, mass_ratio=2.0), flags=flags)
    rho, P = oracle.density(p, pos, sp)
    acc, dsp, _ = oracle.forces(p, pos, vel, spin, sp, rho, P)
    m = np.where(sp == 0, oracle.mass(p, 0), oracle.mass(p, 1))[:, None]
    I = p.inertia_coef * m * p.dx ** 2
    orb = np.cross(pos, m * acc).sum(0)
    spn = (I * dsp).sum(0)
    scale = np.abs(np.cross(pos, m * acc)).sum()
    return orb + spn, scale


def test_angular_momentum_orbital_plus_spin_free_cluster():
    res, scale = _angular_residual(oracle.TERMS_ALL)
    assert np.all(np.abs(res) < 1e-12 * scale)
    # the horizontal projection of the interfacial force keeps only L_z
    res, scale = _angular_residual(oracle.TERMS_ALL | oracle.HPROJ)
    assert abs(res[2]) < 1e-12 * scale
    assert np.abs(res[:2]).max() > 1e-6 * scale


@pytest.mark.parametrize("dx", [1.0, 0.5])
def test_angular_momentum_constant_over_kdk_steps(dx):
    """Orbital plus spin momentum is constant over KDK steps; at dx != 1 the
    spin inertia m dx^2 (a length squared, so the spin momentum is counted in
    the same units as r x m v) must be the same in the torque update and in
    the reported L_spin, or the sum drifts."""
    pos, vel, spin, sp = _block(5, 5, 5, seed=5)
    pos = (pos - pos.mean(0)) * dx
    vel = vel * dx
    prm = _params(periodic_z=0, C_T=0.3, C_l=0.5, dt=0.01, dx=dx)
    s = oracle.Sim(prm, pos, vel, spin, sp, flags=oracle.TERMS_ALL)
    d0 = s.diagnostics()
    L0 = np.add(d0["L_orb"], d0["L_spin"])
    s.step(60)
    d1 = s.diagnostics()
    L1 = np.add(d1["L_orb"], d1["L_spin"])
    scale = np.abs(d0["L_orb"]).max() + 1.0
    assert np.all(np.abs(L1 - L0) < 1e-11 * scale)
    assert np.allclose(d1["mom"], d0["mom"], atol=1e-11)
    assert d1["mass"] == d0["mass"]
    assert d0["mass"] == pytest.approx(d0["mass_s"] + d0["mass_n"], rel=1e-15)


def test_walls_act_on_the_fluid_as_viscous_particles():
    """Walls are particles of the normal fluid (Sec. 3): on a fluid particle a
    wall neighbour acts as a viscous particle with the same position,
    velocity, spin, density and pressure would, in every pair term, also at
    unequal species masses."""
    c = synth.workload("cyl_8960")
    p = oracle.make_params(dict(c.params, mass_ratio=3.0, C_T=0.3, C_l=0.5))
    rng = np.random.Generator(np.random.PCG64(21))
    spin = c.spin + rng.normal(0.0, 0.05, size=c.spin.shape)
    rho, P = oracle.density(p, c.pos, c.species)
    fluid = np.nonzero(c.species < 2)[0]
    acc, dsp, _ = oracle.forces(p, c.pos, c.vel, spin, c.species, rho, P, rows=fluid)
    as_viscous = np.where(c.species >= 2, 1, c.species).astype(np.uint8)
    acc2, dsp2, _ = oracle.forces(p, c.pos, c.vel, spin, as_viscous, rho, P, rows=fluid)
    # a good share of the fluid rows has wall neighbours
    assert (np.hypot(c.pos[fluid, 0], c.pos[fluid, 1]) > c.R - 2.0 * p.h).sum() > 1000
    assert np.allclose(acc2[fluid], acc[fluid], rtol=1e-13, atol=1e-13 * np.abs(acc).max())
    assert np.allclose(dsp2[fluid], dsp[fluid], rtol=1e-13, atol=1e-13 * np.abs(dsp).max())
    # likewise in the pressure filter's weights (outer walls stay out of it)
    Pn = P + rng.normal(0.0, 0.1 * p.p0, size=P.shape)
    Pf = oracle.pressure_filter(p, c.pos, c.species, rho, Pn, rows=fluid)
    inner_as_viscous = np.where(c.species == 2, 1, c.species).astype(np.uint8)
    Pf2 = oracle.pressure_filter(p, c.pos, inner_as_viscous, rho, Pn, rows=fluid)
    assert np.allclose(Pf2[fluid], Pf[fluid], rtol=1e-13, atol=1e-13 * p.p0)
    assert not np.allclose(Pf[fluid], Pn[fluid])


def test_drift_keeps_positions_in_the_z_period():
    """z is periodic (the slip top and bottom of Sec. 3): a particle that
    drifts across z = H re-enters at z = 0, so the state stays in [0, H)."""
    Hz = 4.0
    pos, vel, spin, sp = _block(4, 4, 4, seed=7)
    vel[:, 2] += 3.0  # 0.15 per step: most particles cross z = H in 10 steps
    prm = _params(Hz=Hz, periodic_z=1, dt=0.05)
    s = oracle.Sim(prm, pos, vel, spin, sp, flags=oracle.TERMS_ALL)
    s.step(10)
    assert np.all((s.pos[:, 2] >= 0.0) & (s.pos[:, 2] < Hz))
    # the particles whose free flight ends well past z = H (a quarter of them)
    # are found near the bottom of the period
    crossed = pos[:, 2] + 10 * 0.05 * vel[:, 2] >= Hz + 0.25
    assert crossed.sum() >= len(pos) // 4
    assert np.all(s.pos[crossed, 2] < 2.0)


def test_spin_energy_is_half_spin_times_spin_momentum():
    """For one spin w0 shared by every fluid particle, E_rot = 1/2 sum I w0^2
    and L_spin = sum I w0, so E_rot = 1/2 w0 . L_spin whatever the inertia;
    likewise E_kin = 1/2 v0 . P for one velocity v0."""
    c = synth.workload("cyl_8960")
    p = oracle.make_params(dict(c.params, mass_ratio=3.0))
    w0 = np.array([0.2, -0.1, 0.35])
    v0 = np.array([0.05, 0.3, -0.2])
    spin = np.tile(w0, (c.n, 1))
    vel = np.tile(v0, (c.n, 1))
    rho, _ = oracle.density(p, c.pos, c.species)
    d = oracle.diagnostics(p, c.pos, vel, spin, c.species, rho)
    assert d["E_rot"] == pytest.approx(0.5 * np.dot(w0, d["L_spin"]), rel=1e-12)
    assert d["E_kin"] == pytest.approx(0.5 * np.dot(v0, d["mom"]), rel=1e-12)
    assert d["E_rot"] > 0.0 and d["E_kin"] > 0.0


def test_rigid_rotation_with_placed_walls_has_no_rotational_stress():
    """The rotating walls move as a rigid body (Sec. 3): placed by the oracle at
    any phase they carry v = Omega z x r and the spin Omega z, so a fluid in
    rigid co-rotation next to them feels no shear, rotational or local
    interaction force and no spin torque."""
    c = synth.workload("cyl_8960")
    Om = c.params["Omega"]
    p = oracle.make_params(dict(c.params, C_l=2.0),
                           flags=oracle.TERM_SH | oracle.TERM_ROT | oracle.TERM_SN)
    pos = np.ascontiguousarray(c.pos.copy())
    vel = np.ascontiguousarray(np.cross([0.0, 0.0, Om], pos))
    spin = np.ascontiguousarray(np.tile([0.0, 0.0, Om], (c.n, 1)))
    wall = c.species >= 2
    vel[wall] = 0.0
    spin[wall] = 0.0
    oracle.place_walls(p, c.species, c.pos[:, :2], 0.7, pos, vel, spin)
    # rotate the fluid by the same phase: the whole vessel is one rigid body
    ct, st = math.cos(0.7), math.sin(0.7)
    fl = ~wall
    x, y = c.pos[fl, 0].copy(), c.pos[fl, 1].copy()
    pos[fl, 0], pos[fl, 1] = ct * x - st * y, st * x + ct * y
    vel[fl] = np.cross([0.0, 0.0, Om], pos[fl])
    assert np.allclose(spin[wall], [0.0, 0.0, Om], rtol=0, atol=0)
    rho, P = oracle.density(p, pos, c.species)
    r_xy = np.hypot(pos[:, 0], pos[:, 1])
    rows = np.nonzero(fl & (r_xy > r_xy[fl].max() - 2.6))[0]  # fluid next to the walls
    acc, dsp, _ = oracle.forces(p, pos, vel, spin, c.species, rho, P, rows=rows)
    # the same rows with the walls' spin dropped feel O(1) forces
    spin2 = spin.copy()
    spin2[wall] = 0.0
    acc2, dsp2, _ = oracle.forces(p, pos, vel, spin2, c.species, rho, P, rows=rows)
    ref = np.abs(acc2[rows]).max() + np.abs(dsp2[rows]).max()
    assert ref > 1e-3
    assert np.abs(acc[rows]).max() < 1e-9 * ref
    assert np.abs(dsp[rows]).max() < 1e-9 * ref


def test_rigid_rotation_has_no_viscous_or_local_force():
    """Rigid co-rotation (curl u = 2 w0) gives no rotational stress (Sec. 2.1);
    the shear, rotational and local-interaction pair terms all vanish."""
    c = synth.workload("cyl_8960")
    Om = np.array([0.0, 0.0, 0.37])
    vel = np.cross(Om, c.pos)
    spin = np.tile(Om, (c.n, 1))
    prm = dict(c.params, C_l=2.0)
    p = oracle.make_params(prm, flags=oracle.TERM_SH | oracle.TERM_ROT | oracle.TERM_SN)
    rho, P = oracle.density(p, c.pos, c.species)
    rows = np.arange(0, c.n, 7)
    acc, dsp, _ = oracle.forces(p, c.pos, vel, spin, c.species, rho, P, rows=rows)
    # same configuration with the rigid rotation broken gives O(1) forces
    acc2, dsp2, _ = oracle.forces(p, c.pos, vel, np.zeros_like(spin), c.species, rho, P, rows=rows)
    ref = np.abs(acc2[rows]).max() + np.abs(dsp2[rows]).max()
    assert ref > 1e-3
    assert np.abs(acc[rows]).max() < 1e-12 * ref * 1e3
    assert np.abs(dsp[rows]).max() < 1e-12 * ref * 1e3


@pytest.fixture(scope="module")
def lattice21():
    pos = _lattice(21)
    c = int(np.argmin((pos ** 2).sum(1)))
    return pos, c


def _visc_density(lattice, eta, etar, v, w, flags=oracle.TERM_SH | oracle.TERM_ROT):
    pos, c = lattice
    prm = _params(h_over_dx=2.6, periodic_z=0, eta_bar=eta, eta_r=etar)
    p = oracle.make_params(prm, flags=flags)
    sp = np.ones(len(pos), np.uint8)
    rho, P = oracle.density(p, pos, sp)
    a, b, _ = oracle.forces(p, pos, v, w, sp, rho, P, rows=[c])
    m = oracle.mass(p, 1)
    V = m / rho[c]
    return a[c] * m / V, b[c] * p.inertia_coef * m * p.dx ** 2 / V


def test_viscous_terms_reproduce_eq2_continuum(lattice21):
    """M5 + M6 -> (eta + eta_r) lap v + 2 eta_r curl w for div v = 0, and the
    spin torque -> 2 eta_r (curl v - 2 w): the third and fifth terms of Eq. 2
    and the rigid-rotation strain of Sec. 2.1.  Smooth fields on a fine
    unjittered lattice; the lattice error at h = 2.6 dx is below 0.6 %."""
    pos, c = lattice21
    x, y, z = pos.T
    zero = np.zeros_like(pos)
    tol = 1.5e-2
    # shear only and rotational only, v = (y^2, 0, 0): lap v = (2, 0, 0)
    v = np.column_stack([y * y, 0 * x, 0 * x])
    for eta, etar in [(1.0, 0.0), (0.0, 1.0), (0.7, 0.3)]:
        f, _ = _visc_density(lattice21, eta, etar, v, zero)
        assert f[0] == pytest.approx(2.0 * (eta + etar), rel=tol)
        assert abs(f[1]) + abs(f[2]) < 1e-10
    v = np.column_stack([z * z, x * x, y * y])
    f, _ = _visc_density(lattice21, 1.0, 1.0, v, zero)
    assert np.allclose(f, 4.0, rtol=tol)
    # spin gradient: w = (0, 0, x) -> curl w = (0, -1, 0) -> force 2 eta_r (0, -1, 0)
    w = np.column_stack([0 * x, 0 * x, x])
    f, tq = _visc_density(lattice21, 1.0, 0.8, zero, w)
    assert f[1] == pytest.approx(-1.6, rel=tol) and abs(f[0]) + abs(f[2]) < 1e-10
    # torque: v = s(-y, x, 0), w = (0, 0, w0) -> 2 eta_r (2 s - 2 w0) z
    s, w0 = 0.3, 0.1
    v = np.column_stack([-s * y, s * x, 0 * x])
    w = np.column_stack([0 * x, 0 * x, w0 + 0 * x])
    f, tq = _visc_density(lattice21, 1.0, 0.8, v, w)
    assert tq[2] == pytest.approx(2 * 0.8 * (2 * s - 2 * w0), rel=tol)
    assert np.abs(f).max() < 1e-10


def test_dissipative_terms_never_raise_energy():
    """Shear, rotational and local-interaction terms are dissipative: the
    kinetic + spin energy decreases monotonically without pressure."""
    pos, vel, spin, sp = _block(6, 6, 6, seed=9)
    prm = _params(Hz=6.0, C_l=0.5, dt=0.005, eta_bar=0.3, eta_r=0.2)
    s = oracle.Sim(prm, pos, vel, spin, sp,
                   flags=oracle.TERM_SH | oracle.TERM_ROT | oracle.TERM_SN)
    e = []
    for _ in range(12):
        d = s.diagnostics()
        e.append(d["E_kin"] + d["E_rot"])
        s.step(1)
    de = np.diff(e)
    assert np.all(de < 0.0)
    assert e[-1] < 0.97 * e[0]


def test_pressure_energy_conserved_to_second_order():
    """Pressure-only WCSPH is Hamiltonian: E_kin + E_int is conserved by the
    velocity Verlet integrator up to O(dt^2)."""
    pos, vel, spin, sp = _block(6, 6, 6, seed=4)
    vel *= 0.05

    def drift(dt, T):
        prm = _params(Hz=6.0, dt=dt)
        prm["p0"] = prm["beta_P"] = 2.0
        s = oracle.Sim(prm, pos, vel, spin, sp, flags=oracle.TERM_P)
        d = s.diagnostics()
        e0 = d["E_kin"] + d["E_int"]
        err = 0.0
        for _ in range(int(round(T / dt))):
            s.step(1)
            d = s.diagnostics()
            err = max(err, abs(d["E_kin"] + d["E_int"] - e0))
        return err, e0

    e1, _ = drift(0.04, 1.6)
    e2, _ = drift(0.02, 1.6)
    assert 3.0 < e1 / e2 < 5.5


def test_interfacial_force_sign_projection_and_reaction():
    """Eqs. 1-2: +/- rho_s sigma grad T act oppositely on the two components,
    only in the horizontal plane (Sec. 2.1); C_T > 0 pushes unlike species
    apart; like species feel nothing."""
    p = oracle.make_params(_params(periodic_z=0, C_T=1.0), flags=oracle.TERM_T | oracle.HPROJ)
    pos = np.array([[0.0, 0.0, 0.0], [0.9, 0.4, 0.7]])
    zero = np.zeros_like(pos)
    for sp, expect in [([0, 1], True), ([1, 0], True), ([0, 0], False), ([1, 1], False),
                       ([0, 2], True)]:
        sp = np.array(sp, np.uint8)
        rho, P = oracle.density(p, pos, sp)
        acc, _, _ = oracle.forces(p, pos, zero, zero, sp, rho, P)
        m = np.where(sp == 0, oracle.mass(p, 0), oracle.mass(p, 1))[:, None]
        f = m * acc
        if not expect:
            assert np.all(f == 0.0)
            continue
        d = pos[0] - pos[1]
        assert f[0, 2] == 0.0
        assert np.dot(f[0, :2], d[:2]) > 0.0            # repulsive
        if sp[1] < 2:
            assert np.allclose(f[0], -f[1], rtol=1e-15)  # reaction
    # without the projection the force lies along r_ij
    p.flags = oracle.TERM_T
    sp = np.array([0, 1], np.uint8)
    rho, P = oracle.density(p, pos, sp)
    acc, _, _ = oracle.forces(p, pos, zero, zero, sp, rho, P)
    assert np.allclose(np.cross(acc[0], pos[0] - pos[1]), 0.0, atol=1e-15)


def _interface_column(p, axis):
    """Unjittered lattice of 12 x 13 x 13 points split by the plane x_axis = 0
    (inviscid below, viscous above); rows: the column of points on the axis
    below the plane.  Returns the summed force on those rows."""
    G = np.stack(np.meshgrid(*[np.arange(-6, 7)] * 3, indexing="ij"), -1).reshape(-1, 3)
    G = G[G[:, axis] <= 5].astype(np.float64)
    G[:, axis] += 0.5
    sp = np.where(G[:, axis] < 0.0, 0, 1).astype(np.uint8)
    others = [k for k in range(3) if k != axis]
    rows = np.where((G[:, others[0]] == 0) & (G[:, others[1]] == 0) & (G[:, axis] < 0))[0]
    rho = np.full(len(G), p.rho0)  # rest density: V_j = m_j / rho0 for every j
    zero = np.zeros_like(G)
    acc, _, _ = oracle.forces(p, G, zero, zero, sp, rho, np.zeros(len(G)), rows=rows)
    return (oracle.mass(p, 0) * acc[rows]).sum(0)


@pytest.mark.parametrize("h_over_dx", [1.3, 2.6])
def test_interfacial_force_planar_interface_closed_form(h_over_dx):
    """Scale and radial factor of the interfacial force (Eqs. 1-2).  The pair
    form is the gradient estimate sum_j V_j (T_j - T_i) grad_i W_ij of a
    temperature that jumps by dT across the species interface, times
    -/+ rho_s sigma V_i.  On a lattice split by a plane, the pairs that cross
    it from one column give, by counting the pairs at each separation s,
        sum_i f_i = -C_T V^2 dx sum_{s>=1} s^2 sum_{p,q} F(dx |(s,p,q)|)
                  = -(C_T V^2 dx / 2) sum_{n in Z^3} n_x^2 F(|n| dx),
    and the second moment of the kernel gradient, int x^2 F d^3x = 1 (by
    parts from int W = 1), makes that -C_T / 2 per unit interface area in
    the continuum: half the jump acts on each side.  With the horizontal
    projection of Sec. 2.1 a horizontal interface feels nothing."""
    p = oracle.make_params(_params(h_over_dx=h_over_dx, periodic_z=0, C_T=1.7, rho0=2.0),
                           flags=oracle.TERM_T | oracle.HPROJ)
    m = int(math.ceil(2.0 * h_over_dx)) + 1
    g = np.arange(-m, m + 1, dtype=np.float64)
    n = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    moment = sum(nx * nx * oracle.F(p, r) for nx, r in zip(n[:, 0], np.sqrt((n * n).sum(1))))
    # continuum second moment of F, to the lattice's accuracy at this h
    assert moment * p.dx ** 5 == pytest.approx(1.0, abs=2e-4 if h_over_dx > 2 else 3e-2)
    V = oracle.mass(p, 0) / p.rho0
    expect = -0.5 * p.C_T * V * V * p.dx * moment
    for axis in (0, 1):  # vertical interfaces: normal x, then y
        f = _interface_column(p, axis)
        assert f[axis] == pytest.approx(expect, rel=1e-12)
        assert f[2] == 0.0
        assert abs(f[1 - axis]) < 1e-14 * abs(expect)
        if h_over_dx > 2:
            assert f[axis] / p.dx ** 2 == pytest.approx(-0.5 * p.C_T, rel=3e-4)
    # horizontal interface: no force under the projection, the same law without it
    f = _interface_column(p, 2)
    assert np.all(f == 0.0) or np.abs(f).max() < 1e-14 * abs(expect)
    assert f[2] == 0.0
    p.flags = oracle.TERM_T
    f = _interface_column(p, 2)
    assert f[2] == pytest.approx(expect, rel=1e-12)


def test_force_scale_is_the_absolute_pair_sum():
    """The per-row scale the parity tests use, sum_j |f_ij| / m_i and
    sum_j |tau_ij| / I_i: for a lone pair it is |a| and |alpha| themselves,
    and on every row it bounds them (triangle inequality)."""
    p = oracle.make_params(_params(periodic_z=0, C_T=0.4, C_l=0.6),
                           flags=oracle.TERMS_ALL | oracle.HPROJ)
    pos = np.array([[0.0, 0.0, 0.0], [0.8, -0.5, 0.9]])
    vel = np.array([[0.1, 0.3, -0.2], [-0.4, 0.2, 0.1]])
    spin = np.array([[0.2, -0.1, 0.3], [0.0, 0.5, -0.2]])
    sp = np.array([0, 1], np.uint8)
    rho, P = oracle.density(p, pos, sp)
    P = P + np.array([0.3, -0.1])
    acc, dsp, _, sc = oracle.forces(p, pos, vel, spin, sp, rho, P, scale=True)
    assert sc[:, 0] == pytest.approx(np.linalg.norm(acc, axis=1), rel=1e-15)
    assert sc[:, 1] == pytest.approx(np.linalg.norm(dsp, axis=1), rel=1e-15)
    pos, vel, spin, sp = _block(6, 6, 6, seed=13)
    p = oracle.make_params(_params(Hz=6.0, C_T=0.3, C_l=0.7), flags=oracle.TERMS_ALL | oracle.HPROJ)
    rho, P = oracle.density(p, pos, sp)
    acc, dsp, _, sc = oracle.forces(p, pos, vel, spin, sp, rho, P, scale=True)
    assert np.all(np.linalg.norm(acc, axis=1) <= sc[:, 0] * (1 + 1e-14))
    assert np.all(np.linalg.norm(dsp, axis=1) <= sc[:, 1] * (1 + 1e-14))
    assert np.all(sc[:, 0] > 0) and np.all(sc[:, 1] > 0)


def test_local_interaction_opposes_relative_velocity():
    """F_sn = C_l v_sn acts between unlike species with its reaction on the
    other species (Sec. 2.1), decelerating their relative motion."""
    p = oracle.make_params(_params(periodic_z=0, C_l=1.0),
                           flags=oracle.TERM_SN | oracle.SN_LITERAL)
    pos = np.array([[0.0, 0.0, 0.0], [1.1, 0.3, -0.2]])
    vel = np.array([[0.5, -0.2, 0.1], [-0.1, 0.3, 0.0]])
    zero = np.zeros_like(pos)
    sp = np.array([0, 1], np.uint8)
    rho, P = oracle.density(p, pos, sp)
    acc, dsp, _ = oracle.forces(p, pos, vel, zero, sp, rho, P)
    m = oracle.mass(p, 0)
    f = m * acc
    vrel = vel[0] - vel[1]
    assert np.allclose(np.cross(f[0], vrel), 0.0, atol=1e-15) and np.dot(f[0], vrel) < 0
    assert np.allclose(f[0], -f[1], rtol=1e-15)
    assert np.all(dsp == 0.0)                              # literal: no torque
    # ratio at two distances follows the kernel W (local average weight)
    pos2 = pos.copy()
    pos2[1] *= 1.4
    rho2, P2 = oracle.density(p, pos2, sp)
    acc2, _, _ = oracle.forces(p, pos2, vel, zero, sp, rho2, P2)
    r1, r2 = np.linalg.norm(pos[1]), np.linalg.norm(pos2[1])
    ratio = (np.linalg.norm(acc[0]) * rho[0] * rho[1]) / (np.linalg.norm(acc2[0]) * rho2[0] * rho2[1])
    assert ratio == pytest.approx(oracle.W(p, r1) / oracle.W(p, r2), rel=1e-12)
    same = np.array([1, 1], np.uint8)
    acc3, _, _ = oracle.forces(p, pos, vel, zero, same, rho, P)
    assert np.all(acc3 == 0.0)


def test_pressure_sign():
    """Compressed fluid (rho > rho0, P > 0) pushes outwards; a dilute cluster
    (P < 0) pulls inwards."""
    p = oracle.make_params(_params(periodic_z=0), flags=oracle.TERM_P)
    for spacing, outward in [(0.7, True), (1.6, False)]:
        pos = _lattice(5, spacing)
        sp = np.ones(len(pos), np.uint8)
        rho, P = oracle.density(p, pos, sp)
        zero = np.zeros_like(pos)
        acc, _, _ = oracle.forces(p, pos, zero, zero, sp, rho, P)
        corner = int(np.argmax(pos.sum(1)))
        radial = np.dot(acc[corner], pos[corner])
        assert (P[len(pos) // 2] > 0) == outward
        assert (radial > 0) == outward


# ------------------------------------------------------- integrator, walls (M9)

def test_kdk_is_time_reversible():
    pos, vel, spin, sp = _block(5, 5, 5, seed=2)
    prm = _params(Hz=5.0, dt=0.02)
    prm["p0"] = prm["beta_P"] = 1.5
    s = oracle.Sim(prm, pos, vel * 0.3, spin, sp, flags=oracle.TERM_P | oracle.TERM_T)
    x0, v0 = s.pos.copy(), s.vel.copy()
    s.step(25)
    assert np.abs(s.pos - x0).max() > 1e-2
    s.vel *= -1.0
    s.acc *= 1.0
    s.step(25)
    dz = s.pos - x0
    dz[:, 2] -= 5.0 * np.round(dz[:, 2] / 5.0)
    assert np.abs(dz).max() < 1e-9
    assert np.abs(s.vel + v0).max() < 1e-9


def test_rotating_walls_and_angular_momentum_budget():
    c = synth.workload("cyl_8960")
    s = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    ref = s.wall_ref.copy()
    d0 = s.diagnostics()
    s.step(3)
    th = 0.0
    for _ in range(3):
        th += c.params["Omega"] * c.params["dt"]
    assert s.theta.value == th
    w = c.species >= 2
    ct, st = math.cos(th), math.sin(th)
    want = np.column_stack([ct * ref[w, 0] - st * ref[w, 1], st * ref[w, 0] + ct * ref[w, 1], ref[w, 2]])
    assert np.array_equal(s.pos[w], want)
    assert np.allclose(s.vel[w], np.cross([0, 0, c.params["Omega"]], s.pos[w]), rtol=1e-15)
    assert np.all(s.rho[c.species == 3] == 1.0) and np.all(s.P[c.species == 3] == 0.0)
    inner = c.species == 2
    assert np.all(s.rho[inner] != 1.0)
    d1 = s.diagnostics()
    # L_z(t) - L_z(0) equals the torque impulse of the walls (internal pair
    # forces and spin torques cancel), to round-off
    dL = (d1["L_orb"][2] + d1["L_spin"][2]) - (d0["L_orb"][2] + d0["L_spin"][2])
    assert dL == pytest.approx(d1["J_wall"][2], rel=1e-9, abs=1e-9 * abs(d0["L_orb"][2]))
    assert d1["mass"] == d0["mass"]
    fl = c.species < 2
    assert np.all(s.pos[fl, 2] >= 0.0) and np.all(s.pos[fl, 2] < c.H)


# ------------------------------------------- pressure filter (Algorithm 1)
# The filter's formula is not printed; the oracle reads it as the zeroth-order
# kernel average Pf_i = sum_j V_j P_j W_ij / sum_j V_j W_ij (i itself included,
# outer walls excluded).  These pins fix what that reading implies.

def test_pressure_filter_keeps_constant_and_linear_fields():
    c = synth.workload("cyl_8960")
    p = oracle.make_params(c.params)
    rho, _ = oracle.density(p, c.pos, c.species)
    keep = c.species != 3
    # a constant field is a fixed point for any positive weights
    Pc = np.full(c.n, 0.37)
    Pf = oracle.pressure_filter(p, c.pos, c.species, rho, Pc)
    assert np.abs(Pf[keep] - 0.37).max() < 1e-15 * 0.37 * 8
    # on an unjittered lattice with uniform volumes, the neighbourhood of an
    # interior particle is point-symmetric, so a linear field is kept exactly
    q = oracle.make_params(_params(periodic_z=0))
    pos = _lattice(11)
    sp = np.ones(len(pos), np.uint8)
    P = 0.3 * pos[:, 0] - 1.1 * pos[:, 1] + 0.7 * pos[:, 2] + 2.0
    Pf = oracle.pressure_filter(q, pos, sp, np.ones(len(pos)), P)
    inner = np.all(np.abs(pos) <= 2.0 + 1e-9, axis=1)
    assert inner.sum() == 125
    assert np.abs(Pf[inner] - P[inner]).max() < 1e-13
    # the boundary rows see a one-sided neighbourhood and move (the field's
    # slope is not symmetric there): the test above is not vacuous
    assert np.abs(Pf - P).max() > 1e-2


def test_pressure_filter_unit_impulse_response_on_lattice():
    """P = 1 at one lattice particle, 0 elsewhere, uniform density: with the
    lattice mass m = rho0 / sum_n W(|n| dx) the weights of every interior row
    sum to one, so the filtered field is (m / rho0) W(r) around the impulse:
    (m / rho0) W(0) at the impulse itself and zero beyond 2h."""
    q = oracle.make_params(_params(periodic_z=0, rho0=2.5))
    pos = _lattice(13)
    n = len(pos)
    sp = np.ones(n, np.uint8)
    k = int(np.argmin((pos ** 2).sum(1)))
    P = np.zeros(n)
    P[k] = 1.0
    Pf = oracle.pressure_filter(q, pos, sp, np.full(n, 2.5), P)
    r = np.sqrt((pos ** 2).sum(1))
    S = oracle.lattice_sum(q)
    near = r < 2.0 * q.h
    want = np.array([oracle.W(q, x) for x in r[near]]) / S
    assert np.abs(Pf[near] - want).max() < 1e-15
    assert Pf[k] == pytest.approx(oracle.W(q, 0.0) / S, rel=1e-14)
    assert np.all(Pf[~near] == 0.0)


def test_pressure_filter_bounds_and_outer_wall_exclusion():
    c = synth.workload("cyl_8960")
    p = oracle.make_params(c.params)
    rho, _ = oracle.density(p, c.pos, c.species)
    rng = np.random.default_rng(4)
    P = rng.normal(size=c.n)
    P[c.species == 3] = 0.0
    Pf = oracle.pressure_filter(p, c.pos, c.species, rho, P)
    off, nbr = oracle.neighbors(p, c.pos)
    for i in range(0, c.n, 37):
        if c.species[i] == 3:
            assert Pf[i] == P[i]
            continue
        js = np.append(nbr[off[i]:off[i + 1]], i)
        js = js[c.species[js] != 3]
        assert P[js].min() - 1e-14 <= Pf[i] <= P[js].max() + 1e-14
    # the outer-wall pressures do not enter any row
    P2 = P.copy()
    P2[c.species == 3] = 1e3
    Pf2 = oracle.pressure_filter(p, c.pos, c.species, rho, P2)
    keep = c.species != 3
    assert np.array_equal(Pf2[keep], Pf[keep])


# -------------------------------------------- collision model (Algorithm 1)
# Read as the binary inelastic collision of two spheres along the line of
# centres, for pairs closer than col_dist that approach; the velocity change
# enters the pair pass as the force m_i dv_i / dt.

def _two_body(mass_ratio=3.0, e=0.3, d=0.7, flip=False, seed=8):
    rng = np.random.default_rng(seed)
    prm = _params(periodic_z=0, mass_ratio=mass_ratio, col_dist=0.9, col_e=e, dt=0.01)
    p = oracle.make_params(prm, flags=oracle.COLLISION)
    n_hat = rng.normal(size=3)
    n_hat /= np.linalg.norm(n_hat)
    pos = np.array([[0.0, 0.0, 0.0], d * n_hat]) + 5.0
    vel = rng.normal(size=(2, 3))
    vn = (vel[0] - vel[1]) @ (pos[0] - pos[1])
    if (vn > 0) != flip:  # make the pair approach (or separate, if flip)
        vel = vel[::-1].copy()
    spin = rng.normal(size=(2, 3))
    sp = np.array([0, 1], np.uint8)
    rho = np.array([1.3, 0.8])
    acc, dsp, _ = oracle.forces(p, pos, vel, spin, sp, rho, np.zeros(2))
    m = np.array([oracle.mass(p, 0), oracle.mass(p, 1)])
    return p, pos, vel, acc, dsp, m


def test_collision_two_body_law():
    """Textbook binary collision: after dv = a dt the normal relative velocity
    is -e times the one before, the tangential one is unchanged, momentum is
    conserved and no spin torque arises."""
    p, pos, vel, acc, dsp, m = _two_body()
    assert m[0] == pytest.approx(3.0 * m[1], rel=1e-15)
    dv = acc * p.dt
    e_hat = (pos[0] - pos[1]) / np.linalg.norm(pos[0] - pos[1])
    v0 = vel[0] - vel[1]
    v1 = (vel[0] + dv[0]) - (vel[1] + dv[1])
    assert v0 @ e_hat < 0.0
    assert v1 @ e_hat == pytest.approx(-p.col_e * (v0 @ e_hat), rel=1e-12)
    t0 = v0 - (v0 @ e_hat) * e_hat
    t1 = v1 - (v1 @ e_hat) * e_hat
    assert np.abs(t1 - t0).max() < 1e-13
    assert np.abs(m[0] * dv[0] + m[1] * dv[1]).max() < 1e-15
    assert np.all(dsp == 0.0)
    # kinetic energy does not grow (restitution below one)
    E0 = 0.5 * (m * (vel ** 2).sum(1)).sum()
    E1 = 0.5 * (m * ((vel + dv) ** 2).sum(1)).sum()
    assert E1 < E0


def test_collision_only_for_close_approaching_pairs():
    _, _, _, acc, _, _ = _two_body(flip=True)
    assert np.all(acc == 0.0)
    _, _, _, acc, _, _ = _two_body(d=0.95)
    assert np.all(acc == 0.0)
    _, _, _, acc, _, _ = _two_body(e=1.0)
    assert np.abs(acc).max() > 0.0


def test_collision_conserves_momentum_and_angular_momentum():
    pos, vel, spin, sp = _block(5, 5, 5, seed=21)
    pos = pos - pos.mean(0)
    prm = _params(periodic_z=0, mass_ratio=2.0, col_dist=1.02, col_e=0.2)
    p = oracle.make_params(prm, flags=oracle.COLLISION)
    rho, P = oracle.density(p, pos, sp)
    acc, dsp, _ = oracle.forces(p, pos, vel, spin, sp, rho, P)
    m = np.where(sp == 0, oracle.mass(p, 0), oracle.mass(p, 1))[:, None]
    f = m * acc
    hit = np.any(acc != 0.0, axis=1)
    assert hit.sum() > 20
    scale = np.abs(f).sum()
    assert np.abs(f.sum(0)).max() < 1e-13 * scale
    assert np.abs(np.cross(pos, f).sum(0)).max() < 1e-13 * np.abs(np.cross(pos, f)).sum()
    assert np.all(dsp == 0.0)


def test_filter_and_collision_keep_the_wall_budget():
    """With the pressure filter and the collision model on, fluid-wall
    collisions act on the walls too: L_z(t) - L_z(0) still equals the torque
    impulse of the walls."""
    c = synth.workload("cyl_8960")
    prm = dict(c.params, col_dist=0.95, col_e=0.2)
    fl = oracle.DEFAULT_FLAGS | oracle.PFILTER | oracle.COLLISION
    s = oracle.Sim(prm, c.pos, c.vel, c.spin, c.species, flags=fl)
    base = oracle.Sim(c.params, c.pos, c.vel, c.spin, c.species)
    d0 = s.diagnostics()
    s.step(3)
    base.step(3)
    d1 = s.diagnostics()
    dL = (d1["L_orb"][2] + d1["L_spin"][2]) - (d0["L_orb"][2] + d0["L_spin"][2])
    assert dL == pytest.approx(d1["J_wall"][2], rel=1e-9, abs=1e-9 * abs(d0["L_orb"][2]))
    # both optional steps changed the state
    assert np.abs(s.P - base.P).max() > 1e-6 * np.abs(base.P).max()
    assert np.abs(s.vel - base.vel).max() > 0.0
