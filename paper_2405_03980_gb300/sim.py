"""Convenience wrapper: torch owns the device buffers, the C ABI does the work.

``Simulation`` sizes the state and workspace buffers with
``sph_state_bytes``/``sph_workspace_bytes``, allocates them as torch uint8
tensors on the chosen device, and forwards every call to the library on the
current torch stream.  No step of the method runs in Python.
"""
from __future__ import annotations

import numpy as np

from . import _binding as B


class Simulation:
    def __init__(self, instances, precision: int = B.SPH_FP64, flags: int = B.SPH_FLAGS_DEFAULT,
                 nbr_cap: int = 160, device: str = "cuda:0", stream=None, host_pinned=False):
        import torch

        self.torch = torch
        self.device = torch.device(device)
        if not isinstance(instances, (list, tuple)):
            instances = [instances]
        self.params = []
        self.counts = []
        for c in instances:
            p = dict(c.params)
            p.setdefault("precision", precision)
            p.setdefault("flags", flags)
            p.setdefault("nbr_cap", nbr_cap)
            self.params.append(B.params_from_dict(p))
            self.counts.append(int(c.species.shape[0]))
        self.n = int(sum(self.counts))
        pos = np.ascontiguousarray(np.concatenate([c.pos for c in instances]), dtype=np.float64)
        vel = np.ascontiguousarray(np.concatenate([c.vel for c in instances]), dtype=np.float64)
        spin = np.ascontiguousarray(np.concatenate([c.spin for c in instances]), dtype=np.float64)
        sp = np.ascontiguousarray(np.concatenate([c.species for c in instances]), dtype=np.uint8)
        self.state_bytes = B.sph_state_bytes(self.params, self.counts)
        self.ws_bytes = B.sph_workspace_bytes(self.params, self.counts)
        if self.state_bytes == 0 or self.ws_bytes == 0:
            raise B.SphError(-1, "sph_state_bytes/sph_workspace_bytes")
        self.ctx = None
        with torch.cuda.device(self.device):
            self.state = torch.empty(self.state_bytes, dtype=torch.uint8, device=self.device)
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.reinit(pos, vel, spin, sp)

    def reinit(self, pos, vel, spin, species):
        """(Re)initialise on the already-allocated device buffers from arrays in
        input order (numpy / pinned host memory or device tensors)."""
        self.close()
        with self.torch.cuda.device(self.device):
            self.ctx = B.sph_init_batch(self.params, self.counts, pos, vel, spin, species,
                                        self.state, self.state_bytes, self.ws, self.ws_bytes,
                                        self.stream.cuda_stream)

    # -- stepping ---------------------------------------------------------
    def step(self, k: int = 1):
        B.sph_step(self.ctx, k)

    def build_cells(self):
        B.sph_build_cells(self.ctx)

    def density(self):
        B.sph_density(self.ctx)

    def forces(self):
        B.sph_forces(self.ctx)

    def check(self):
        B.sph_check(self.ctx)

    # -- read-out ---------------------------------------------------------
    def diagnostics(self, inst: int = 0) -> dict:
        return B.sph_diagnostics(self.ctx, inst)

    def force_breakdown(self, inst: int = 0):
        return B.sph_force_breakdown(self.ctx, inst)

    def state_arrays(self) -> dict:
        n = self.n
        out = {k: np.zeros((n, 3)) for k in ("pos", "vel", "spin", "acc", "dspin")}
        out["rho"] = np.zeros(n)
        out["P"] = np.zeros(n)
        B.sph_get_state(self.ctx, out["pos"], out["vel"], out["spin"], out["rho"], out["P"],
                        out["acc"], out["dspin"])
        return out

    def neighbors(self):
        return B.sph_get_neighbors(self.ctx, self.n)

    def profile(self, nsteps: int) -> dict:
        return B.sph_profile_steps(self.ctx, nsteps)

    def autotune(self, reps: int = 3) -> tuple[int, int]:
        return B.sph_autotune(self.ctx, reps)

    def launch_config(self) -> dict:
        return B.sph_get_launch_config(self.ctx)

    def set_launch_config(self, block_density: int = 128, block_forces: int = 128,
                          search_warps: int = 4, search_depth: int = 512):
        B.sph_set_launch_config(self.ctx, block_density, block_forces, search_warps,
                                search_depth)

    def launches_per_step(self) -> int:
        return B.sph_launches_per_step(self.ctx)

    def pair_census(self, inst: int = 0):
        return B.sph_pair_census(self.ctx, inst)

    def list_builds(self, inst: int = 0) -> int:
        return B.sph_list_builds(self.ctx, inst)

    # -- checkpoint / resume ----------------------------------------------
    def save_checkpoint(self, path: str | None = None):
        """The complete persistent state as a host uint8 array (also written
        to path if given); restore it with load_checkpoint on a Simulation
        of the same instances, parameters and precision."""
        buf = B.sph_save_checkpoint(self.ctx)
        if path is not None:
            buf.tofile(path)
        return buf

    def load_checkpoint(self, src):
        """Restore a checkpoint (array from save_checkpoint, or a file path)."""
        buf = np.fromfile(src, dtype=np.uint8) if isinstance(src, str) else src
        B.sph_load_checkpoint(self.ctx, buf)

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
