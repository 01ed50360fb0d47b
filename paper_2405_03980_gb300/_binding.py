"""ctypes binding of the C ABI in ``include/sph.h`` (argument marshalling only).

Every function keeps the C name.  Array arguments accept numpy arrays (host
memory) or torch tensors (``data_ptr()``, host or device); the library itself
decides where a pointer lives.  There is no fallback: if the sm_103a library
is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

SPH_OK = 0
STATUS = {0: "SPH_OK", -1: "SPH_ERR_ARG", -2: "SPH_ERR_CUDA", -3: "SPH_ERR_WORKSPACE",
          -4: "SPH_ERR_GRID_OVERFLOW", -5: "SPH_ERR_ESCAPED", -6: "SPH_ERR_NONFINITE",
          -7: "SPH_ERR_TIMEOUT", -8: "SPH_ERR_STATE", -9: "SPH_ERR_NEIGHBORS",
          -10: "SPH_ERR_BOUNDS"}
SPH_TERM_P, SPH_TERM_T, SPH_TERM_SH, SPH_TERM_ROT, SPH_TERM_SN = 1, 2, 4, 8, 16
SPH_HPROJ, SPH_SN_LITERAL, SPH_FLAGS_DEFAULT = 32, 64, 63
SPH_PFILTER, SPH_COLLISION = 128, 256
SPH_FP64, SPH_MIXED = 0, 1


class SphError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


class SphParams(C.Structure):
    _fields_ = [(k, C.c_double) for k in (
        "dx", "h", "rho0", "alpha_P", "p0", "beta_P", "eta_bar", "eta_r", "xi_bar",
        "C_l", "C_T", "C_omega", "mass_ratio", "inertia_coef", "Omega", "dt")] + [
        ("box_lo", C.c_double * 3), ("box_hi", C.c_double * 3),
        ("periodic_z", C.c_int32), ("precision", C.c_int32), ("flags", C.c_uint32),
        ("nbr_cap", C.c_int32), ("col_dist", C.c_double), ("col_e", C.c_double),
        ("skin", C.c_double)]


class SphDiag(C.Structure):
    _fields_ = [("mass", C.c_double), ("mass_s", C.c_double), ("mass_n", C.c_double),
                ("mom", C.c_double * 3), ("L_orb", C.c_double * 3), ("L_spin", C.c_double * 3),
                ("E_kin", C.c_double), ("E_rot", C.c_double), ("E_int", C.c_double),
                ("T_wall", C.c_double * 3), ("J_wall", C.c_double * 3),
                ("rho_min", C.c_double), ("rho_max", C.c_double), ("v_max", C.c_double),
                ("n_pairs", C.c_int64), ("step", C.c_int64), ("theta", C.c_double)]

    def as_dict(self) -> dict:
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if not isinstance(v, (int, float)) else v
        return out


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Load the sm_103a library (building it with nvcc if it is absent).

    With SPH_CHECKED=1 in the environment the checked variant is loaded
    instead (device bounds checks that latch SPH_ERR_BOUNDS)."""
    global _lib
    with _lock:
        if _lib is None:
            checked = os.environ.get("SPH_CHECKED", "") == "1"
            path = _build.LIB_CHECKED if checked else _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise RuntimeError(f"CUDA library missing: {path}")
                _build.build(checked=checked)
            L = C.CDLL(path)
            vp, P, i64p = C.c_void_p, C.POINTER(SphParams), C.POINTER(C.c_int64)
            sig = {
                "sph_params_default": (C.c_int, [P, C.c_double, C.c_double, C.c_double]),
                "sph_state_bytes": (C.c_size_t, [C.c_int32, P, i64p]),
                "sph_workspace_bytes": (C.c_size_t, [C.c_int32, P, i64p]),
                "sph_init": (C.c_int, [C.POINTER(vp), P, C.c_int64, vp, vp, vp, vp, vp,
                                       C.c_size_t, vp, C.c_size_t, vp]),
                "sph_init_batch": (C.c_int, [C.POINTER(vp), C.c_int32, P, i64p, vp, vp, vp, vp,
                                             vp, C.c_size_t, vp, C.c_size_t, vp]),
                "sph_build_cells": (C.c_int, [vp]),
                "sph_density": (C.c_int, [vp]),
                "sph_forces": (C.c_int, [vp]),
                "sph_step": (C.c_int, [vp, C.c_int32]),
                "sph_diagnostics": (C.c_int, [vp, C.c_int32, C.POINTER(SphDiag)]),
                "sph_force_breakdown": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_double)]),
                "sph_get_state": (C.c_int, [vp] + [vp] * 7),
                "sph_get_neighbors": (C.c_int, [vp, i64p, i64p, C.c_int64]),
                "sph_check": (C.c_int, [vp]),
                "sph_launches_per_step": (C.c_int32, [vp]),
                "sph_list_builds": (C.c_int, [vp, C.c_int32, i64p]),
                "sph_pair_census": (C.c_int, [vp, C.c_int32, i64p]),
                "sph_profile_steps": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_double), C.c_int32]),
                "sph_stage_count": (C.c_int32, []),
                "sph_autotune": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_int32),
                                           C.POINTER(C.c_int32)]),
                "sph_get_launch_config": (C.c_int, [vp, C.POINTER(C.c_int32),
                                                    C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                                    C.POINTER(C.c_int32)]),
                "sph_stage_name": (C.c_char_p, [C.c_int32]),
                "sph_fma_peak": (C.c_int, [C.c_int32, C.c_int32, C.POINTER(C.c_double)]),
                "sph_diag_sums_noalloc": (C.c_int, [P, C.c_int64, vp, vp, vp, vp, vp, vp, vp]),
                "sph_set_launch_config": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32,
                                                    C.c_int32]),
                "sph_checkpoint_bytes": (C.c_size_t, [vp]),
                "sph_save_checkpoint": (C.c_int, [vp, vp, C.c_size_t]),
                "sph_load_checkpoint": (C.c_int, [vp, vp, C.c_size_t]),
                "sph_destroy": (C.c_int, [vp]),
                "sph_status_string": (C.c_char_p, [C.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def exported_symbols() -> list[str]:
    """Names this binding expects the library to export."""
    return ["sph_params_default", "sph_state_bytes", "sph_workspace_bytes", "sph_init",
            "sph_init_batch", "sph_build_cells", "sph_density", "sph_forces", "sph_step",
            "sph_diagnostics", "sph_force_breakdown", "sph_get_state", "sph_get_neighbors", "sph_check",
            "sph_launches_per_step", "sph_list_builds", "sph_pair_census",
            "sph_profile_steps", "sph_stage_count", "sph_stage_name",
            "sph_autotune", "sph_get_launch_config", "sph_set_launch_config",
            "sph_fma_peak", "sph_diag_sums_noalloc", "sph_checkpoint_bytes",
            "sph_save_checkpoint", "sph_load_checkpoint", "sph_destroy", "sph_status_string"]


def _ck(st: int, where: str):
    if st != SPH_OK:
        raise SphError(st, where)


def _ptr(a):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported array type {type(a)}")


def params_from_dict(p: dict, precision: int = SPH_FP64, flags: int = SPH_FLAGS_DEFAULT,
                     nbr_cap: int = 160) -> SphParams:
    s = SphParams()
    for k in ("dx", "h", "rho0", "alpha_P", "p0", "beta_P", "eta_bar", "eta_r", "xi_bar",
              "C_l", "C_T", "C_omega", "mass_ratio", "inertia_coef", "Omega", "dt"):
        setattr(s, k, float(p[k]))
    for a in range(3):
        s.box_lo[a] = float(p["box_lo"][a])
        s.box_hi[a] = float(p["box_hi"][a])
    s.periodic_z = int(p.get("periodic_z", 1))
    s.precision = int(p.get("precision", precision))
    s.flags = int(p.get("flags", flags))
    s.nbr_cap = int(p.get("nbr_cap", nbr_cap))
    s.col_dist = float(p.get("col_dist", 0.8 * float(p["dx"])))
    s.col_e = float(p.get("col_e", 0.2))
    s.skin = float(p.get("skin", 0.0))
    return s


def _param_array(params):
    if isinstance(params, SphParams):
        params = [params]
    arr = (SphParams * len(params))(*params)
    return arr, len(params)


def sph_params_default(R: float, H: float, Omega: float) -> SphParams:
    p = SphParams()
    _ck(lib().sph_params_default(C.byref(p), R, H, Omega), "sph_params_default")
    return p


def sph_state_bytes(params, counts) -> int:
    arr, k = _param_array(params)
    cnt = (C.c_int64 * k)(*[int(c) for c in counts])
    return int(lib().sph_state_bytes(k, arr, cnt))


def sph_workspace_bytes(params, counts) -> int:
    arr, k = _param_array(params)
    cnt = (C.c_int64 * k)(*[int(c) for c in counts])
    return int(lib().sph_workspace_bytes(k, arr, cnt))


def sph_init_batch(params, counts, pos, vel, spin, species, dev_state, state_bytes,
                   dev_workspace, workspace_bytes, stream=0):
    arr, k = _param_array(params)
    cnt = (C.c_int64 * k)(*[int(c) for c in counts])
    ctx = C.c_void_p()
    _ck(lib().sph_init_batch(C.byref(ctx), k, arr, cnt, _ptr(pos), _ptr(vel), _ptr(spin),
                             _ptr(species), _ptr(dev_state), int(state_bytes),
                             _ptr(dev_workspace), int(workspace_bytes), stream or None),
        "sph_init_batch")
    return ctx


def sph_init(params, n, pos, vel, spin, species, dev_state, state_bytes, dev_workspace,
             workspace_bytes, stream=0):
    ctx = C.c_void_p()
    _ck(lib().sph_init(C.byref(ctx), C.byref(params), int(n), _ptr(pos), _ptr(vel), _ptr(spin),
                       _ptr(species), _ptr(dev_state), int(state_bytes), _ptr(dev_workspace),
                       int(workspace_bytes), stream or None), "sph_init")
    return ctx


def sph_build_cells(ctx):
    _ck(lib().sph_build_cells(ctx), "sph_build_cells")


def sph_density(ctx):
    _ck(lib().sph_density(ctx), "sph_density")


def sph_forces(ctx):
    _ck(lib().sph_forces(ctx), "sph_forces")


def sph_step(ctx, nsteps: int = 1):
    _ck(lib().sph_step(ctx, int(nsteps)), "sph_step")


def sph_diagnostics(ctx, inst: int = 0) -> dict:
    d = SphDiag()
    _ck(lib().sph_diagnostics(ctx, int(inst), C.byref(d)), "sph_diagnostics")
    return d.as_dict()


def sph_force_breakdown(ctx, inst: int = 0) -> np.ndarray:
    """sum_i |f_i^term| for the pressure, interfacial, shear, rotational and
    local-interaction terms of instance inst (FP64, current state)."""
    out = (C.c_double * 5)()
    _ck(lib().sph_force_breakdown(ctx, int(inst), out), "sph_force_breakdown")
    return np.array(out[:], dtype=np.float64)


def sph_get_state(ctx, pos=None, vel=None, spin=None, rho=None, P=None, acc=None, dspin=None):
    _ck(lib().sph_get_state(ctx, _ptr(pos), _ptr(vel), _ptr(spin), _ptr(rho), _ptr(P),
                            _ptr(acc), _ptr(dspin)), "sph_get_state")


def sph_get_neighbors(ctx, n: int):
    off = np.zeros(n + 1, dtype=np.int64)
    st = lib().sph_get_neighbors(ctx, off.ctypes.data_as(C.POINTER(C.c_int64)), None, 0)
    if st not in (SPH_OK, -1):
        _ck(st, "sph_get_neighbors")
    tot = int(off[-1])
    nbr = np.zeros(max(tot, 1), dtype=np.int64)
    _ck(lib().sph_get_neighbors(ctx, off.ctypes.data_as(C.POINTER(C.c_int64)),
                                nbr.ctypes.data_as(C.POINTER(C.c_int64)), tot),
        "sph_get_neighbors")
    return off, nbr[:tot]


def sph_check(ctx):
    _ck(lib().sph_check(ctx), "sph_check")


def sph_launches_per_step(ctx) -> int:
    return int(lib().sph_launches_per_step(ctx))


def sph_pair_census(ctx, inst: int = 0) -> np.ndarray:
    out = np.zeros(5, dtype=np.int64)
    _ck(lib().sph_pair_census(ctx, inst, out.ctypes.data_as(C.POINTER(C.c_int64))),
        "sph_pair_census")
    return out


def sph_list_builds(ctx, inst: int = 0) -> int:
    n = C.c_int64(0)
    _ck(lib().sph_list_builds(ctx, inst, C.byref(n)), "sph_list_builds")
    return int(n.value)


def sph_profile_steps(ctx, nsteps: int) -> dict:
    k = int(lib().sph_stage_count())
    ms = (C.c_double * k)()
    _ck(lib().sph_profile_steps(ctx, int(nsteps), ms, k), "sph_profile_steps")
    return {lib().sph_stage_name(i).decode(): ms[i] for i in range(k)}


def sph_fma_peak(precision: int, iters: int = 1 << 16) -> float:
    t = C.c_double()
    _ck(lib().sph_fma_peak(int(precision), int(iters), C.byref(t)), "sph_fma_peak")
    return t.value


SPH_DIAG_SUMS = 19


def sph_diag_sums_noalloc(params, n, pos, vel, spin, species, rho, out, stream=0):
    """Conservation totals of device-resident arrays with no device allocation
    (see include/sph.h); out: SPH_DIAG_SUMS doubles, host or device."""
    _ck(lib().sph_diag_sums_noalloc(C.byref(params), int(n), _ptr(pos), _ptr(vel), _ptr(spin),
                                    _ptr(species), _ptr(rho), _ptr(out), stream or None),
        "sph_diag_sums_noalloc")


def sph_autotune(ctx, reps: int = 3) -> tuple[int, int]:
    bd, bf = C.c_int32(), C.c_int32()
    _ck(lib().sph_autotune(ctx, int(reps), C.byref(bd), C.byref(bf)), "sph_autotune")
    return bd.value, bf.value


def sph_get_launch_config(ctx) -> dict:
    a, b, w, d = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _ck(lib().sph_get_launch_config(ctx, C.byref(a), C.byref(b), C.byref(w), C.byref(d)),
        "sph_get_launch_config")
    return {"block_density": a.value, "block_forces": b.value, "search_warps": w.value,
            "search_depth": d.value}


def sph_checkpoint_bytes(ctx) -> int:
    return int(lib().sph_checkpoint_bytes(ctx))


def sph_save_checkpoint(ctx, buf=None):
    """Write a checkpoint of ctx into buf (a uint8 numpy array or tensor of at
    least sph_checkpoint_bytes; a new host array if None) and return buf."""
    nb = sph_checkpoint_bytes(ctx)
    if buf is None:
        buf = np.empty(nb, dtype=np.uint8)
    _ck(lib().sph_save_checkpoint(ctx, _ptr(buf), _nbytes(buf)), "sph_save_checkpoint")
    return buf


def sph_load_checkpoint(ctx, buf):
    _ck(lib().sph_load_checkpoint(ctx, _ptr(buf), _nbytes(buf)), "sph_load_checkpoint")


def _nbytes(a) -> int:
    if isinstance(a, np.ndarray):
        return int(a.nbytes)
    return int(a.numel() * a.element_size())


def sph_set_launch_config(ctx, block_density: int, block_forces: int, search_warps: int,
                          search_depth: int = 512):
    _ck(lib().sph_set_launch_config(ctx, int(block_density), int(block_forces),
                                    int(search_warps), int(search_depth)),
        "sph_set_launch_config")


def sph_destroy(ctx):
    _ck(lib().sph_destroy(ctx), "sph_destroy")


def sph_status_string(st: int) -> str:
    return lib().sph_status_string(int(st)).decode()
