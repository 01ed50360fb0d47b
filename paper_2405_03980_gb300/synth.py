"""Seeded synthetic inputs for the rotating-cylinder two-fluid SPH workload.

This module only *places* particles and draws the random numbers of the
initial condition; it contains none of the SPH arithmetic (no kernel, no
density, no force, no integrator).  Both the CPU oracle and the CUDA library
consume exactly the arrays produced here.

Geometry (Sec. 3, the cylindrical vessel rotating about z; the initial state
draws the two species at random in proportion to their share):

* lattice points at ((i+1/2)dx, (j+1/2)dx, (k+1/2)dx), axis of the cylinder at
  x = y = 0, k = 0 .. H-1 so that z spans [0, H) and is periodic;
* fluid where r_xy < R, inner wall layer R <= r_xy < R+dx, then the outer
  (dummy) layers R+dx <= r_xy < R+(1+d)dx, d = dummy_layers: one by default
  (two wall layers in all), two for the long runs, so that the kernel support
  of every inner-wall particle (2h = 2.6 dx) lies inside wall particles;
* fluid points jittered by U(-0.05, 0.05) dx per axis; walls are not jittered;
* each fluid particle is viscous with probability f_v, otherwise inviscid;
* velocity Omega z^ x r (+ N(0, 1e-3) per component for the fluid), spin zero
  for the fluid and Omega z^ for the rigid walls.

Species codes: 0 inviscid, 1 viscous, 2 inner wall, 3 outer wall.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

INVISCID, VISCOUS, WALL_INNER, WALL_OUTER = 0, 1, 2, 3


@dataclass
class Cylinder:
    """One synthetic rotating-cylinder instance (all arrays float64 / uint8)."""

    R: float
    H: int
    dx: float
    Omega: float
    f_v: float
    seed: int
    pos: np.ndarray          # (n, 3) float64
    vel: np.ndarray          # (n, 3) float64
    spin: np.ndarray         # (n, 3) float64
    species: np.ndarray      # (n,) uint8
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.species.shape[0])

    @property
    def n_fluid(self) -> int:
        return int((self.species < WALL_INNER).sum())


def workload_params(R: float, H: float, Omega: float, dx: float = 1.0,
                    h_over_dx: float = 1.3, rho0: float = 1.0, gamma: int = 7,
                    Re: float = 100.0, cs_factor: float = 10.0,
                    dt_factor: float = 0.25, wall_layers: int = 2) -> dict:
    """Dimensionless parameter recipe of the benchmark workloads.

    c_s = 10 Omega R, p0 = beta_P = rho0 c_s^2 / gamma (so P(rho0) = 0),
    eta_bar = eta_r = rho0 Omega R^2 / Re, dt = 0.25 h / c_s,
    C_T = 0.01 p0, C_l = 1e-3 rho0 Omega, C_omega = 0.016 (recorded only),
    unit species mass ratio and spin inertia I = 0.1 m dx^2; for the optional
    collision model (off unless its flag is set) a collision distance of
    0.8 dx and a restitution coefficient of 0.2.
    These are workload choices (the paper prints no dimensionless values).
    """
    h = h_over_dx * dx
    cs = cs_factor * Omega * R
    p0 = rho0 * cs * cs / gamma
    eta = rho0 * Omega * R * R / Re
    margin = wall_layers * dx + 2.0 * h
    ext = R + margin
    return dict(
        dx=dx, h=h, rho0=rho0, alpha_P=float(gamma), p0=p0, beta_P=p0,
        eta_bar=eta, eta_r=eta, xi_bar=0.0, C_l=1e-3 * rho0 * Omega,
        C_T=0.01 * p0, C_omega=0.016, mass_ratio=1.0, inertia_coef=0.1,
        Omega=Omega, dt=dt_factor * h / cs, col_dist=0.8 * dx, col_e=0.2,
        box_lo=(-ext, -ext, 0.0), box_hi=(ext, ext, float(H)), periodic_z=1,
    )


def cylinder(R: float, H: int, Omega: float = 0.1, f_v: float = 0.3,
             seed: int = 0, dx: float = 1.0, jitter: float = 0.05,
             vel_noise: float = 1e-3, dummy_layers: int = 1, **param_kw) -> Cylinder:
    """Jittered-lattice cylinder of radius R and H layers with one inner wall
    layer and `dummy_layers` outer (dummy) layers."""
    if dummy_layers < 1:
        raise ValueError("at least one dummy layer")
    rng = np.random.Generator(np.random.PCG64(seed))
    outer = (1 + dummy_layers) * dx
    m = int(math.ceil((R + outer) / dx)) + 1
    ax = (np.arange(-m, m, dtype=np.float64) + 0.5) * dx
    X, Y = np.meshgrid(ax, ax, indexing="ij")
    X = X.ravel()
    Y = Y.ravel()
    rxy = np.sqrt(X * X + Y * Y)
    kind = np.full(X.shape, -1, dtype=np.int8)
    kind[rxy < R] = 0
    kind[(rxy >= R) & (rxy < R + dx)] = WALL_INNER
    kind[(rxy >= R + dx) & (rxy < R + outer)] = WALL_OUTER
    keep = kind >= 0
    X, Y, kind = X[keep], Y[keep], kind[keep]
    nl = X.shape[0]
    Z = (np.arange(H, dtype=np.float64) + 0.5) * dx
    pos = np.empty((nl * H, 3), dtype=np.float64)
    pos[:, 0] = np.tile(X, H)
    pos[:, 1] = np.tile(Y, H)
    pos[:, 2] = np.repeat(Z, nl)
    kind = np.tile(kind, H)
    fluid = kind == 0
    nf = int(fluid.sum())
    species = kind.astype(np.uint8)
    draw = rng.random(nf)
    species[fluid] = np.where(draw < f_v, VISCOUS, INVISCID).astype(np.uint8)
    pos[fluid] += rng.uniform(-jitter * dx, jitter * dx, size=(nf, 3))
    vel = np.zeros_like(pos)
    vel[:, 0] = -Omega * pos[:, 1]
    vel[:, 1] = Omega * pos[:, 0]
    vel[fluid] += rng.normal(0.0, vel_noise, size=(nf, 3))
    spin = np.zeros_like(pos)
    spin[~fluid, 2] = Omega
    params = workload_params(R, H, Omega, dx=dx, wall_layers=1 + dummy_layers, **param_kw)
    return Cylinder(R=R, H=H, dx=dx, Omega=Omega, f_v=f_v, seed=seed, pos=pos,
                    vel=vel, spin=spin, species=species, params=params)


# Named workloads: the 8,960-particle parity cylinder, the 2.4M and the 19.6M
# cylinders (R:H = 1:2), and the near-inviscid low-temperature stress case,
# whose 10,000 steps need the inner wall's kernel support covered by wall
# particles (two dummy layers: 2,592,020 particles in all).
# The paper_* cylinders have the paper's vessel shape (Sec. 3: diameter five
# times the height, R:H = 2.5:1) at its three resolutions, 2.45M, 8.62M and
# 19.6M fluid particles (2,454,000, 8,620,224 and 19,636,400 here), with the
# species drawn in proportion to the density ratio rho_s / rho_n = 5 (a
# viscous particle with probability 1/6, equal particle masses).
WORKLOADS = {
    "cyl_8960": dict(R=10.0, H=20, Omega=0.1, f_v=0.3),
    "cyl_2525900": dict(R=72.5, H=145, Omega=0.1, f_v=0.3),
    "cyl_20100112": dict(R=146.0, H=292, Omega=0.1, f_v=0.3),
    "cyl_2525900_lowT": dict(R=72.5, H=145, Omega=0.2, f_v=0.01, dummy_layers=2),
    "paper_2534800": dict(R=125.0, H=50, Omega=0.1, f_v=1.0 / 6.0),
    "paper_8802016": dict(R=190.0, H=76, Omega=0.1, f_v=1.0 / 6.0),
    "paper_19949600": dict(R=250.0, H=100, Omega=0.1, f_v=1.0 / 6.0),
}


def workload(name: str, seed: int = 0) -> Cylinder:
    return cylinder(seed=seed, **WORKLOADS[name])


def ensemble(k: int = 64, seed: int = 1234, n_lo: float = 2e4,
             n_hi: float = 5e5) -> list[Cylinder]:
    """Uneven ensemble: N_fluid log-uniform in [n_lo, n_hi], Omega ~ U(0.05, 0.2),
    f_v ~ U(0.02, 0.5), R/H ~ U(0.25, 1), R = (N (R/H) / pi)^(1/3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for t in range(k):
        nf = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        om = rng.uniform(0.05, 0.2)
        fv = rng.uniform(0.02, 0.5)
        rh = rng.uniform(0.25, 1.0)
        R = (nf * rh / math.pi) ** (1.0 / 3.0)
        H = max(8, int(round(R / rh)))
        out.append(cylinder(R=R, H=H, Omega=om, f_v=fv, seed=seed * 1000 + t))
    return out


def periodic_block(nx: int, ny: int, nz: int, seed: int = 0, jitter: float = 0.05,
                   f_v: float = 0.3, vel_sigma: float = 0.1, dx: float = 1.0):
    """Fluid-only jittered lattice filling [0,nx)x[0,ny)x[0,nz) (for box tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
    pos = (g + 0.5) * dx
    n = pos.shape[0]
    pos += rng.uniform(-jitter * dx, jitter * dx, size=(n, 3))
    species = np.where(rng.random(n) < f_v, VISCOUS, INVISCID).astype(np.uint8)
    vel = rng.normal(0.0, vel_sigma, size=(n, 3))
    spin = rng.normal(0.0, vel_sigma, size=(n, 3))
    return pos, vel, spin, species
