"""Per-rank arithmetic for the slab decomposition tests: the CPU oracle's
density, pressure and pair forces on a rank's local set, and the velocity
Verlet kicks and drift as the oracle's own step takes them (test
infrastructure: the decomposition module itself holds no SPH arithmetic)."""
import numpy as np

import oracle


class OracleEngine:
    def kick_drift(self, own, p):
        f = own.species < 2
        hdt, dt = 0.5 * p["dt"], p["dt"]
        H = p["box_hi"][2] - p["box_lo"][2]
        own.vel[f] += hdt * own.acc[f]
        own.spin[f] += hdt * own.dspin[f]
        own.pos[f] += dt * own.vel[f]
        z = own.pos[:, 2]
        z[f & (z >= H)] -= H
        z[f & (z < 0.0)] += H

    def place_walls(self, own, p, theta):
        q = oracle.make_params(p)
        for k in ("pos", "vel", "spin"):
            setattr(own, k, np.ascontiguousarray(getattr(own, k)))
        oracle.place_walls(q, own.species, own.wref, theta, own.pos, own.vel, own.spin)

    def evaluate(self, local, p):
        q = oracle.make_params(p)
        rho, P = oracle.density(q, local.pos, local.species)
        acc, dspin, wt = oracle.forces(q, local.pos, local.vel, local.spin, local.species, rho, P)
        return rho, P, acc, dspin, wt

    def kick(self, own, p):
        f = own.species < 2
        hdt = 0.5 * p["dt"]
        own.vel[f] += hdt * own.acc[f]
        own.spin[f] += hdt * own.dspin[f]
