"""ctypes front end of the C oracle (TEST INFRASTRUCTURE, see __init__.py).

build() compiles oracle/lbm_oracle.c with gcc into oracle/_build/ (FP64,
-ffp-contract=off so that no multiply-add is fused, OpenMP over rows).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

from . import lattice as _lat

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Lattice(C.Structure):
    _fields_ = [("Q", C.c_int), ("ex", C.POINTER(C.c_int)), ("ey", C.POINTER(C.c_int)),
                ("w", C.POINTER(C.c_double)), ("r", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("Nx", C.c_int), ("Ny", C.c_int), ("eq_order", C.c_int),
                ("thermal", C.c_int), ("Kn", C.c_double), ("tau", C.c_double),
                ("mu_exp", C.c_double), ("u_wall", C.c_double * 2),
                ("T_wall", C.c_double * 2), ("accom", C.c_double * 2),
                ("vn", C.c_double * 2)]


class _WallStats(C.Structure):
    _fields_ = [("m_in", C.c_double * 2), ("m_out", C.c_double * 2),
                ("holes_unfilled", C.c_longlong), ("slots_doubled", C.c_longlong),
                ("m_lost", C.c_double * 2)]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        lib.orc_equilibrium.argtypes = [C.POINTER(_Lattice), C.c_int, C.c_double, C.c_double,
                                        C.c_double, C.c_double, dp]
        lib.orc_moments.argtypes = [C.POINTER(_Lattice), C.c_int, dp, C.c_long, dp, dp, dp, dp]
        lib.orc_collide.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params), dp]
        lib.orc_wall_distribution.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params),
                                              C.c_int, dp]
        lib.orc_wall_distribution.restype = C.c_double
        lib.orc_run.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params), dp, C.c_long,
                                C.POINTER(_WallStats)]
        lib.orc_init_fields.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params), dp, dp, dp,
                                        dp, dp]
        lib.orc_macros.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params), dp, dp, dp, dp, dp]
        lib.orc_macros_kinetic.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params), dp, dp, dp,
                                           dp, dp]
        lib.orc_set_num_threads.argtypes = [C.c_int]
        lib.orc_set_num_threads.restype = None
        lib.orc_fluxes.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params), dp, dp, dp, dp, dp,
                                   dp]
        lib.orc_run_to_residual.argtypes = [C.POINTER(_Lattice), C.POINTER(_Params), dp,
                                            C.c_double, C.c_long, C.c_int,
                                            C.POINTER(C.c_long), dp]
        lib.orc_num_threads.restype = C.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Problem:
    """One Couette problem: lattice + grid + physical parameters."""
    lattice: str = "D2Q25"
    Nx: int = 1
    Ny: int = 64
    eq_order: int = 2
    thermal: bool = False
    Kn: float = 0.1
    tau: float = 0.0
    mu_exp: float = 1.0
    u_wall: tuple = (-0.1, 0.1)
    T_wall: tuple = (1.0, 1.0)
    accom: tuple = (1.0, 1.0)
    vn: tuple = (0.0, 0.0)      # normal wall velocity u_w . n / r, cells per step
    lat: _lat.OracleLattice = field(init=False, repr=False)

    def __post_init__(self):
        self.lat = _lat.get(self.lattice)
        self._ex = np.ascontiguousarray(self.lat.e[:, 0], dtype=np.int32)
        self._ey = np.ascontiguousarray(self.lat.e[:, 1], dtype=np.int32)
        self._w = np.ascontiguousarray(self.lat.w, dtype=np.float64)
        ip = C.POINTER(C.c_int)
        self._cl = _Lattice(self.lat.Q, self._ex.ctypes.data_as(ip),
                            self._ey.ctypes.data_as(ip), _dp(self._w), float(self.lat.r))
        self._cp = _Params(self.Nx, self.Ny, self.eq_order, int(self.thermal), self.Kn,
                           self.tau, self.mu_exp, (C.c_double * 2)(*self.u_wall),
                           (C.c_double * 2)(*self.T_wall), (C.c_double * 2)(*self.accom),
                           (C.c_double * 2)(*self.vn))

    @property
    def Q(self) -> int:
        return self.lat.Q

    def new_state(self) -> np.ndarray:
        return np.zeros((self.Q, self.Ny, self.Nx), dtype=np.float64)


def set_num_threads(n: int) -> None:
    _load().orc_set_num_threads(int(n))


def num_threads() -> int:
    return int(_load().orc_num_threads())


def equilibrium(p: Problem, rho, ux, uy, T, order=None) -> np.ndarray:
    out = np.empty(p.Q)
    _load().orc_equilibrium(C.byref(p._cl), p.eq_order if order is None else order,
                            rho, ux, uy, T, _dp(out))
    return out


def moments(p: Problem, fa: np.ndarray):
    fa = np.ascontiguousarray(fa, dtype=np.float64)
    r = [C.c_double() for _ in range(4)]
    _load().orc_moments(C.byref(p._cl), int(p.thermal), _dp(fa), 1, *[C.byref(v) for v in r])
    return tuple(v.value for v in r)


def wall_distribution(p: Problem, wall: int):
    gw = np.empty(p.Q)
    den = _load().orc_wall_distribution(C.byref(p._cl), C.byref(p._cp), wall, _dp(gw))
    return gw, den


def init_fields(p: Problem, rho, ux=None, uy=None, T=None) -> np.ndarray:
    f = p.new_state()
    fld = [None if a is None else np.ascontiguousarray(np.broadcast_to(a, (p.Ny, p.Nx)),
                                                       dtype=np.float64)
           for a in (rho, ux, uy, T)]
    _load().orc_init_fields(C.byref(p._cl), C.byref(p._cp), *[_dp(a) for a in fld], _dp(f))
    return f


def collide(p: Problem, f: np.ndarray) -> np.ndarray:
    g = np.ascontiguousarray(f, dtype=np.float64).copy()
    _load().orc_collide(C.byref(p._cl), C.byref(p._cp), _dp(g))
    return g


def run(p: Problem, f: np.ndarray, nsteps: int, stats: bool = False):
    """Advance pre-collision f~ by nsteps (in place); returns wall stats."""
    assert f.shape == (p.Q, p.Ny, p.Nx) and f.dtype == np.float64 and f.flags.c_contiguous
    st = _WallStats()
    rc = _load().orc_run(C.byref(p._cl), C.byref(p._cp), _dp(f), int(nsteps), C.byref(st))
    if rc != 0:
        raise RuntimeError(f"oracle run failed: {rc}")
    if stats:
        return dict(m_in=tuple(st.m_in), m_out=tuple(st.m_out), m_lost=tuple(st.m_lost),
                    holes_unfilled=st.holes_unfilled, slots_doubled=st.slots_doubled)
    return None


def macros(p: Problem, f: np.ndarray):
    out = [np.empty((p.Ny, p.Nx)) for _ in range(4)]
    _load().orc_macros(C.byref(p._cl), C.byref(p._cp), _dp(np.ascontiguousarray(f)),
                       *[_dp(a) for a in out])
    return tuple(out)


def macros_kinetic(p: Problem, f: np.ndarray):
    """Like macros(), with the kinetic temperature also for isothermal runs."""
    out = [np.empty((p.Ny, p.Nx)) for _ in range(4)]
    _load().orc_macros_kinetic(C.byref(p._cl), C.byref(p._cp), _dp(np.ascontiguousarray(f)),
                               *[_dp(a) for a in out])
    return tuple(out)


def fluxes(p: Problem, f: np.ndarray):
    """Stress (sigma_xx, sigma_xy, sigma_yy) and heat flux (q_x, q_y) planes
    [Ny][Nx] of the distribution behind the pre-collision f~ (Sec. II)."""
    out = [np.empty((p.Ny, p.Nx)) for _ in range(5)]
    _load().orc_fluxes(C.byref(p._cl), C.byref(p._cp), _dp(np.ascontiguousarray(f)),
                       *[_dp(a) for a in out])
    return tuple(out)


def run_to_residual(p: Problem, f: np.ndarray, tol: float, max_steps: int,
                    check_every: int = 100):
    steps = C.c_long()
    res = C.c_double()
    rc = _load().orc_run_to_residual(C.byref(p._cl), C.byref(p._cp), _dp(f), tol,
                                     int(max_steps), int(check_every), C.byref(steps),
                                     C.byref(res))
    if rc < 0:
        raise RuntimeError(f"oracle run_to_residual failed: {rc}")
    return rc == 0, steps.value, res.value
