"""CPU FP64 oracle of the two-fluid spin-SPH step (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg import this package.  It wraps the plain C implementation in
``sph_oracle.c`` (built here with gcc, ``-ffp-contract=off``, OpenMP over the
rows) through ctypes; nothing here is shared with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None

TERM_P, TERM_T, TERM_SH, TERM_ROT, TERM_SN = 1, 2, 4, 8, 16
HPROJ, SN_LITERAL = 32, 64
PFILTER, COLLISION = 128, 256
TERMS_ALL = 31
DEFAULT_FLAGS = TERMS_ALL | HPROJ


class OrcParams(C.Structure):
    _fields_ = [(k, C.c_double) for k in (
        "dx", "h", "rho0", "alpha_P", "p0", "beta_P", "eta_bar", "eta_r",
        "xi_bar", "C_l", "C_T", "C_omega", "mass_ratio", "inertia_coef",
        "Omega", "dt", "col_dist", "col_e", "Hz")] + [("periodic_z", C.c_int),
                                                      ("flags", C.c_uint)]


class OrcDiag(C.Structure):
    _fields_ = [("mass", C.c_double), ("mass_s", C.c_double), ("mass_n", C.c_double),
                ("mom", C.c_double * 3), ("L_orb", C.c_double * 3),
                ("L_spin", C.c_double * 3), ("E_kin", C.c_double),
                ("E_rot", C.c_double), ("E_int", C.c_double),
                ("T_wall", C.c_double * 3), ("J_wall", C.c_double * 3),
                ("rho_min", C.c_double), ("rho_max", C.c_double),
                ("v_max", C.c_double), ("n_pairs", C.c_int64)]

    def as_dict(self) -> dict:
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if not isinstance(v, (int, float)) else v
        return out


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (idempotent).

    ``SPH_ORACLE_LIB`` may name an already-built variant (the mutation tests
    load deliberately broken copies of the oracle through it)."""
    alt = os.environ.get("SPH_ORACLE_LIB")
    if alt:
        return alt
    src = os.path.join(_HERE, "sph_oracle.c")
    hdr = os.path.join(_HERE, "sph_oracle.h")
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            u8p = C.POINTER(C.c_uint8)
            i64p = C.POINTER(C.c_int64)
            P = C.POINTER(OrcParams)
            L.orc_W.restype = C.c_double
            L.orc_W.argtypes = [P, C.c_double]
            L.orc_F.restype = C.c_double
            L.orc_F.argtypes = [P, C.c_double]
            L.orc_lattice_sum.restype = C.c_double
            L.orc_lattice_sum.argtypes = [P]
            L.orc_mass.restype = C.c_double
            L.orc_mass.argtypes = [P, C.c_int]
            L.orc_neighbors.restype = C.c_int64
            L.orc_neighbors.argtypes = [P, C.c_int64, dp, i64p, i64p, C.c_int64]
            L.orc_density.restype = None
            L.orc_density.argtypes = [P, C.c_int64, dp, u8p, i64p, C.c_int64, dp, dp]
            L.orc_pressure_filter.restype = None
            L.orc_pressure_filter.argtypes = [P, C.c_int64, dp, u8p, dp, dp, i64p, C.c_int64,
                                              dp]
            L.orc_forces.restype = None
            L.orc_forces.argtypes = [P, C.c_int64, dp, dp, dp, u8p, dp, dp, i64p,
                                     C.c_int64, dp, dp, dp, dp]
            L.orc_forces_ex.restype = None
            L.orc_forces_ex.argtypes = [P, C.c_int64, dp, dp, dp, u8p, dp, dp, i64p,
                                        C.c_int64, dp, dp, dp, dp, dp]
            L.orc_place_walls.restype = None
            L.orc_place_walls.argtypes = [P, C.c_int64, u8p, dp, C.c_double, dp, dp, dp]
            L.orc_init.restype = None
            L.orc_init.argtypes = [P, C.c_int64, dp, dp, dp, u8p, dp, C.c_double,
                                   dp, dp, dp, dp, dp]
            L.orc_step.restype = None
            L.orc_step.argtypes = [P, C.c_int64, dp, dp, dp, u8p, dp, dp, dp, dp,
                                   dp, dp, dp, dp]
            L.orc_diagnostics.restype = None
            L.orc_diagnostics.argtypes = [P, C.c_int64, dp, dp, dp, u8p, dp, dp, dp,
                                          C.POINTER(OrcDiag)]
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _u8(a):
    return a.ctypes.data_as(C.POINTER(C.c_uint8))


def _i64(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int64))


def make_params(p: dict, flags: int = DEFAULT_FLAGS) -> OrcParams:
    o = OrcParams()
    for k in ("dx", "h", "rho0", "alpha_P", "p0", "beta_P", "eta_bar", "eta_r",
              "xi_bar", "C_l", "C_T", "C_omega", "mass_ratio", "inertia_coef",
              "Omega", "dt"):
        setattr(o, k, float(p[k]))
    o.col_dist = float(p.get("col_dist", 0.0))
    o.col_e = float(p.get("col_e", 0.0))
    o.Hz = float(p["box_hi"][2] - p["box_lo"][2])
    o.periodic_z = int(p.get("periodic_z", 1))
    o.flags = int(p.get("flags", flags))
    return o


def W(p: OrcParams, r: float) -> float:
    return lib().orc_W(C.byref(p), float(r))


def F(p: OrcParams, r: float) -> float:
    return lib().orc_F(C.byref(p), float(r))


def lattice_sum(p: OrcParams) -> float:
    return lib().orc_lattice_sum(C.byref(p))


def mass(p: OrcParams, species: int) -> float:
    return lib().orc_mass(C.byref(p), int(species))


def neighbors(p: OrcParams, pos: np.ndarray):
    """Brute-force CSR neighbour lists (j ascending) for every particle."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    off = np.zeros(n + 1, dtype=np.int64)
    cap = max(1, n * 200)
    nbr = np.zeros(cap, dtype=np.int64)
    tot = lib().orc_neighbors(C.byref(p), n, _d(pos), _i64(off), _i64(nbr), cap)
    if tot > cap:
        nbr = np.zeros(tot, dtype=np.int64)
        lib().orc_neighbors(C.byref(p), n, _d(pos), _i64(off), _i64(nbr), tot)
    return off, nbr[:tot]


def density(p: OrcParams, pos, species, rows=None):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.uint8)
    n = pos.shape[0]
    rho = np.zeros(n)
    P = np.zeros(n)
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if rows is None else r.shape[0]
    lib().orc_density(C.byref(p), n, _d(pos), _u8(species), _i64(r), nr, _d(rho), _d(P))
    return rho, P


def pressure_filter(p: OrcParams, pos, species, rho, P, rows=None):
    """Filtered pressure of the listed rows (others are returned unchanged)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    species = np.ascontiguousarray(species, dtype=np.uint8)
    rho, P = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, P))
    n = pos.shape[0]
    Pf = P.copy()
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if rows is None else r.shape[0]
    lib().orc_pressure_filter(C.byref(p), n, _d(pos), _u8(species), _d(rho), _d(P), _i64(r),
                              nr, _d(Pf))
    return Pf


def forces(p: OrcParams, pos, vel, spin, species, rho, P, rows=None, term_mag=False,
           scale=False):
    """Pair forces of the listed rows: (acc, dspin, wall torque[, term sums]
    [, scale]).  scale (n, 2): sum_j |f_ij| / m_i and sum_j |tau_ij| / I_i of
    each listed fluid row, the bound on what summation order can change."""
    pos, vel, spin = (np.ascontiguousarray(a, dtype=np.float64) for a in (pos, vel, spin))
    species = np.ascontiguousarray(species, dtype=np.uint8)
    rho, P = (np.ascontiguousarray(a, dtype=np.float64) for a in (rho, P))
    n = pos.shape[0]
    acc = np.zeros((n, 3))
    dspin = np.zeros((n, 3))
    wT = np.zeros((n, 3))
    mag = np.zeros(5)
    sc = np.zeros((n, 2))
    r = None if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    nr = n if rows is None else r.shape[0]
    lib().orc_forces_ex(C.byref(p), n, _d(pos), _d(vel), _d(spin), _u8(species), _d(rho),
                        _d(P), _i64(r), nr, _d(acc), _d(dspin), _d(wT), _d(mag), _d(sc))
    out = (acc, dspin, wT)
    if term_mag:
        out += (mag,)
    if scale:
        out += (sc,)
    return out


def place_walls(p: OrcParams, species, wall_ref, theta: float, pos, vel, spin):
    """Walls at phase theta from their reference positions, in place."""
    for a in (pos, vel, spin):
        assert a.flags["C_CONTIGUOUS"] and a.dtype == np.float64
    species = np.ascontiguousarray(species, dtype=np.uint8)
    wall_ref = np.ascontiguousarray(wall_ref, dtype=np.float64)
    lib().orc_place_walls(C.byref(p), pos.shape[0], _u8(species), _d(wall_ref), float(theta),
                          _d(pos), _d(vel), _d(spin))


def diagnostics(p: OrcParams, pos, vel, spin, species, rho, T_wall=None, J_wall=None) -> dict:
    """FP64 conservation diagnostics of a given state (orc_diagnostics)."""
    pos, vel, spin = (np.ascontiguousarray(a, dtype=np.float64) for a in (pos, vel, spin))
    species = np.ascontiguousarray(species, dtype=np.uint8)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    T = np.zeros(3) if T_wall is None else np.ascontiguousarray(T_wall, dtype=np.float64)
    J = np.zeros(3) if J_wall is None else np.ascontiguousarray(J_wall, dtype=np.float64)
    d = OrcDiag()
    lib().orc_diagnostics(C.byref(p), pos.shape[0], _d(pos), _d(vel), _d(spin), _u8(species),
                          _d(rho), _d(T), _d(J), C.byref(d))
    return d.as_dict()


class Sim:
    """Full-state oracle time stepper (kick-drift-kick, rotating walls)."""

    def __init__(self, params: dict, pos, vel, spin, species, flags=None, theta=0.0):
        self.p = make_params(params) if flags is None else make_params(params, flags)
        if flags is not None:
            self.p.flags = flags
        self.pos = np.array(pos, dtype=np.float64, order="C")
        self.vel = np.array(vel, dtype=np.float64, order="C")
        self.spin = np.array(spin, dtype=np.float64, order="C")
        self.species = np.array(species, dtype=np.uint8, order="C")
        self.wall_ref = self.pos.copy()
        self.n = self.pos.shape[0]
        self.rho = np.zeros(self.n)
        self.P = np.zeros(self.n)
        self.acc = np.zeros((self.n, 3))
        self.dspin = np.zeros((self.n, 3))
        self.T = np.zeros(3)
        self.J = np.zeros(3)
        self.theta = C.c_double(theta)
        self.step_count = 0
        lib().orc_init(C.byref(self.p), self.n, _d(self.pos), _d(self.vel), _d(self.spin),
                       _u8(self.species), _d(self.wall_ref), self.theta.value,
                       _d(self.rho), _d(self.P), _d(self.acc), _d(self.dspin), _d(self.T))

    def step(self, k: int = 1):
        for _ in range(k):
            lib().orc_step(C.byref(self.p), self.n, _d(self.pos), _d(self.vel),
                           _d(self.spin), _u8(self.species), _d(self.wall_ref),
                           C.byref(self.theta), _d(self.rho), _d(self.P), _d(self.acc),
                           _d(self.dspin), _d(self.T), _d(self.J))
            self.step_count += 1

    def diagnostics(self) -> dict:
        d = OrcDiag()
        lib().orc_diagnostics(C.byref(self.p), self.n, _d(self.pos), _d(self.vel),
                              _d(self.spin), _u8(self.species), _d(self.rho),
                              _d(self.T), _d(self.J), C.byref(d))
        return d.as_dict()
