"""Spatial decomposition of one rotating cylinder over ranks: z-slabs with a
halo (the paper's domain decomposition with halo exchange, Sec. 2.3 and
Algorithm 1; its own runs used a 4 x 8 slice grid on 32 GPUs).

Rank r owns the particles whose z lies in its slab [z_r, z_{r+1}) of the
period [0, H) (split evenly).  Before each density and pair-force evaluation
it receives from its two neighbours (periodic in z) every particle within
`halo` of its slab's faces as ghosts.  With halo = 2 x the kernel support
(4h), the ghosts within 2h of the slab have every one of their own
neighbours present too, so their density and pressure come out of the local
evaluation exactly and one exchange per step suffices; the owned rows' forces
then need nothing else.  After the drift, particles whose z left the slab
migrate to the rank that owns it.  The conservation sums are FP64 all-reduces
over the owned particles.

One step (kick-drift-kick, the same sequence as the single-domain step):
    1. half kick and drift of the owned fluid particles, z folded into [0, H);
       the wall phase advances and the owned walls are placed at it
    2. migration to the owning ranks
    3. halo exchange (position, velocity, spin, species, global index)
    4. density, pressure and pair forces of the local set (owned + ghosts),
       kept for the owned rows
    5. second half kick of the owned fluid particles; the wall torque of the
       owned rows, summed over ranks, enters the torque impulse

The arithmetic of steps 1, 4 and 5 is delegated to an engine object
(`kick_drift`, `place_walls`, `evaluate`, `kick`); this module only moves
particles between ranks.  Collectives go through torch.distributed
(point-to-point send/recv to the two neighbours, all_reduce for the sums),
gloo on the CPU or NCCL on GPUs.
"""
from __future__ import annotations

import numpy as np

FIELDS = ("pos", "vel", "spin", "wref", "acc", "dspin")   # (n, 3) float64 each


class SlabLayout:
    """Even split of the z period [0, H) over `world` ranks."""

    def __init__(self, H: float, world: int, halo: float):
        if world < 1:
            raise ValueError("world must be positive")
        self.H, self.world, self.halo = float(H), int(world), float(halo)
        self.edges = np.linspace(0.0, self.H, self.world + 1)
        if world > 1 and np.diff(self.edges).min() < self.halo:
            raise ValueError(f"slabs of {H / world:.3g} are thinner than the halo {halo:.3g}")

    def owner(self, z: np.ndarray) -> np.ndarray:
        """Rank owning each z (z folded into [0, H))."""
        r = np.searchsorted(self.edges, z, side="right") - 1
        return np.clip(r, 0, self.world - 1)

    def slab(self, rank: int) -> tuple[float, float]:
        return float(self.edges[rank]), float(self.edges[rank + 1])

    def halo_sends(self, z: np.ndarray, rank: int):
        """Owned particles to copy to the rank below and to the rank above,
        with the z shift that places them next to the receiver's slab
        (+H or -H across the period)."""
        lo, hi = self.slab(rank)
        down = np.nonzero(z < lo + self.halo)[0]
        up = np.nonzero(z >= hi - self.halo)[0]
        shift_down = self.H if rank == 0 else 0.0
        shift_up = -self.H if rank == self.world - 1 else 0.0
        return (down, shift_down), (up, shift_up)


class Particles:
    """Arrays of one rank's particles (owned or ghosts), row-aligned."""

    def __init__(self, gid, species, **fields):
        self.gid = np.asarray(gid, dtype=np.int64)
        self.species = np.asarray(species, dtype=np.uint8)
        n = len(self.gid)
        for k in FIELDS:
            v = fields.get(k)
            setattr(self, k, np.zeros((n, 3)) if v is None else np.array(v, dtype=np.float64))

    @property
    def n(self) -> int:
        return len(self.gid)

    def take(self, idx) -> "Particles":
        return Particles(self.gid[idx], self.species[idx],
                         **{k: getattr(self, k)[idx] for k in FIELDS})

    @staticmethod
    def concat(parts) -> "Particles":
        return Particles(np.concatenate([p.gid for p in parts]),
                         np.concatenate([p.species for p in parts]),
                         **{k: np.concatenate([getattr(p, k) for p in parts]) for k in FIELDS})

    def pack(self) -> np.ndarray:
        """One float64 row per particle: gid, species, then the fields."""
        return np.concatenate([self.gid[:, None].astype(np.float64),
                               self.species[:, None].astype(np.float64)] +
                              [getattr(self, k) for k in FIELDS], axis=1)

    @staticmethod
    def unpack(buf: np.ndarray) -> "Particles":
        buf = buf.reshape(-1, 2 + 3 * len(FIELDS))
        f = {k: buf[:, 2 + 3 * j:5 + 3 * j] for j, k in enumerate(FIELDS)}
        return Particles(buf[:, 0].astype(np.int64), buf[:, 1].astype(np.uint8), **f)


class Comm:
    """Neighbour exchange and sums over torch.distributed (world 1: local)."""

    def __init__(self, dist=None):
        self.dist = dist
        self.rank = dist.get_rank() if dist else 0
        self.world = dist.get_world_size() if dist else 1

    def sendrecv(self, to_rank: int, payload: np.ndarray, from_rank: int) -> np.ndarray:
        """Send a float64 matrix to one rank and receive one from another
        (count first, then the rows)."""
        if self.world == 1:
            return payload
        import torch
        width = payload.shape[1]
        cnt_out = torch.tensor([payload.shape[0]], dtype=torch.int64)
        cnt_in = torch.zeros(1, dtype=torch.int64)
        reqs = [self.dist.isend(cnt_out, to_rank), self.dist.irecv(cnt_in, from_rank)]
        for q in reqs:
            q.wait()
        out = torch.from_numpy(np.ascontiguousarray(payload, dtype=np.float64))
        inc = torch.zeros((int(cnt_in.item()), width), dtype=torch.float64)
        reqs = []
        if out.shape[0]:
            reqs.append(self.dist.isend(out, to_rank))
        if inc.shape[0]:
            reqs.append(self.dist.irecv(inc, from_rank))
        for q in reqs:
            q.wait()
        return inc.numpy()

    def allreduce(self, x: np.ndarray) -> np.ndarray:
        if self.world == 1:
            return np.asarray(x, dtype=np.float64)
        import torch
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).clone()
        self.dist.all_reduce(t)
        return t.numpy()


class DecomposedCylinder:
    """One cylinder advanced by `comm.world` ranks, each owning a z-slab.

    params: the instance parameters (dict as synth.workload_params makes);
    pos, vel, spin, species: the whole initial state (every rank passes the
    same arrays and keeps its own slab); engine: the per-rank arithmetic
    (kick_drift(p, P), place_walls(p, theta), evaluate(local, params) ->
    (rho, P, acc, dspin, wall_torque) for every local row, kick(p)).
    """

    def __init__(self, params: dict, pos, vel, spin, species, engine, comm: Comm,
                 halo: float | None = None):
        self.p = dict(params)
        self.engine = engine
        self.comm = comm
        H = float(self.p["box_hi"][2] - self.p["box_lo"][2])
        self.halo = 4.0 * self.p["h"] if halo is None else float(halo)
        self.layout = SlabLayout(H, comm.world, self.halo)
        pos = np.asarray(pos, dtype=np.float64)
        n = pos.shape[0]
        gid = np.arange(n)
        mine = self.layout.owner(pos[:, 2]) == comm.rank
        allp = Particles(gid, species, pos=pos, vel=vel, spin=spin, wref=pos)
        self.own = allp.take(np.nonzero(mine)[0])
        self.theta = 0.0
        self.T = np.zeros(3)
        self.J = np.zeros(3)
        self.step_count = 0
        self.engine.place_walls(self.own, self.p, self.theta)
        self.T = self._evaluate()

    # -- exchanges ------------------------------------------------------------

    def _neighbours(self):
        w, r = self.comm.world, self.comm.rank
        return (r - 1) % w, (r + 1) % w

    def _migrate(self):
        """Owned particles whose z left the slab go to the neighbour owning it
        (a particle moves less than a slab per step)."""
        if self.comm.world == 1:
            return
        own = self.layout.owner(self.own.pos[:, 2])
        below, above = self._neighbours()
        r = self.comm.rank
        if np.any((own != r) & (own != below) & (own != above)):
            raise RuntimeError("a particle moved further than one slab in one step")
        to_below = np.nonzero(own == below)[0] if below != r else np.zeros(0, np.int64)
        to_above = np.nonzero((own == above) & (own != below))[0]
        # the count, then the rows, to each neighbour; from the other side the
        # neighbour's own leavers towards this rank
        got = [self.comm.sendrecv(below, self.own.take(to_below).pack(), above),
               self.comm.sendrecv(above, self.own.take(to_above).pack(), below)]
        parts = [self.own.take(np.nonzero(own == r)[0])]
        parts += [Particles.unpack(g) for g in got if g.shape[0]]
        self.own = Particles.concat(parts)

    def _ghosts(self) -> Particles:
        """Halo copies from the two neighbours, z shifted next to this slab."""
        if self.comm.world == 1:
            return Particles(np.zeros(0, np.int64), np.zeros(0, np.uint8))
        (d, sd), (u, su) = self.layout.halo_sends(self.own.pos[:, 2], self.comm.rank)
        below, above = self._neighbours()
        down = self.own.take(d)
        down.pos = down.pos.copy()
        down.pos[:, 2] += sd
        up = self.own.take(u)
        up.pos = up.pos.copy()
        up.pos[:, 2] += su
        from_above = self.comm.sendrecv(below, down.pack(), above)
        from_below = self.comm.sendrecv(above, up.pack(), below)
        parts = [Particles.unpack(g) for g in (from_above, from_below) if g.shape[0]]
        if not parts:
            return Particles(np.zeros(0, np.int64), np.zeros(0, np.uint8))
        return Particles.concat(parts)

    # -- evaluation and step ----------------------------------------------------

    def _local_params(self) -> dict:
        """Open z over this slab and its halo (the period is handled by the
        ghosts' z shifts) when there is more than one rank."""
        if self.comm.world == 1:
            return self.p
        lo, hi = self.layout.slab(self.comm.rank)
        q = dict(self.p)
        q["periodic_z"] = 0
        q["box_lo"] = (self.p["box_lo"][0], self.p["box_lo"][1], lo - self.halo - 1.0)
        q["box_hi"] = (self.p["box_hi"][0], self.p["box_hi"][1], hi + self.halo + 1.0)
        return q

    def _evaluate(self) -> np.ndarray:
        """Density, pressure and forces of the owned rows; returns the wall
        torque on the owned fluid particles summed over all ranks."""
        ghosts = self._ghosts()
        local = Particles.concat([self.own, ghosts]) if ghosts.n else self.own
        rho, P, acc, dspin, wt = self.engine.evaluate(local, self._local_params())
        n = self.own.n
        self.own.acc = acc[:n].copy()
        self.own.dspin = dspin[:n].copy()
        self.rho, self.P = rho[:n].copy(), P[:n].copy()
        fluid = self.own.species < 2
        return self.comm.allreduce(wt[:n][fluid].sum(axis=0))

    def step(self, k: int = 1):
        dt = float(self.p["dt"])
        for _ in range(k):
            self.engine.kick_drift(self.own, self.p)
            self.theta += float(self.p["Omega"]) * dt
            self.engine.place_walls(self.own, self.p, self.theta)
            self._migrate()
            T_old = self.T
            self.T = self._evaluate()
            self.engine.kick(self.own, self.p)
            self.J = self.J + 0.5 * dt * (T_old + self.T)
            self.step_count += 1

    def gather(self) -> dict:
        """The whole state by global index (every rank receives it)."""
        if self.comm.world == 1:
            parts = [self.own]
            rhos, Ps = [self.rho], [self.P]
        else:
            import torch
            buf = np.concatenate([self.own.pack(), self.rho[:, None], self.P[:, None]], axis=1)
            cnt = torch.tensor([buf.shape[0]], dtype=torch.int64)
            cnts = [torch.zeros(1, dtype=torch.int64) for _ in range(self.comm.world)]
            self.comm.dist.all_gather(cnts, cnt)
            m = max(int(c.item()) for c in cnts)
            pad = np.zeros((m, buf.shape[1]))
            pad[:buf.shape[0]] = buf
            outs = [torch.zeros((m, buf.shape[1]), dtype=torch.float64)
                    for _ in range(self.comm.world)]
            self.comm.dist.all_gather(outs, torch.from_numpy(pad))
            parts, rhos, Ps = [], [], []
            for c, o in zip(cnts, outs):
                a = o.numpy()[:int(c.item())]
                parts.append(Particles.unpack(a[:, :-2]))
                rhos.append(a[:, -2])
                Ps.append(a[:, -1])
        allp = Particles.concat(parts)
        order = np.argsort(allp.gid)
        return {"gid": allp.gid[order], "pos": allp.pos[order], "vel": allp.vel[order],
                "spin": allp.spin[order], "acc": allp.acc[order], "dspin": allp.dspin[order],
                "rho": np.concatenate(rhos)[order], "P": np.concatenate(Ps)[order],
                "species": allp.species[order]}
