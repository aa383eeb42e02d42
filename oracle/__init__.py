"""FP64 CPU oracle for the improved axisymmetric lattice Boltzmann scheme.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import this package.  It shares no code with the CUDA library
and imports nothing from it; it accepts any object with the attributes of
``paper_1003_0282_gb300.inputs.Problem``.

The arithmetic lives in ``axlbm_oracle.c`` (plain C, double precision, one
node at a time, two lattices); this module compiles it with gcc on first use
and marshals numpy arrays.  Array layout: [population][k][j] float64;
macroscopic fields [5][k][j] = rho, u_r, u_z, u_theta, T.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "axlbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

INNER = {"axis": 0, "wall": 1, "axis_node": 2}
ZKIND = {"periodic": 0, "wall": 1, "free": 2, "mixed": 3, "nee": 4}
OUTER = {"wall": 0, "nee": 1, "zou_he": 2}
FACES = ("inner", "outer", "lo", "hi")


class _Params(ctypes.Structure):
    _fields_ = [
        ("nr", ctypes.c_int32), ("nz", ctypes.c_int32), ("inner", ctypes.c_int32),
        ("z_lo", ctypes.c_int32), ("z_hi", ctypes.c_int32), ("swirl", ctypes.c_int32),
        ("temperature", ctypes.c_int32), ("t_dirichlet", ctypes.c_int32 * 4),
        ("outer", ctypes.c_int32), ("r0", ctypes.c_double), ("tau_s", ctypes.c_double),
        ("tau_t_s", ctypes.c_double), ("rho0", ctypes.c_double), ("az0", ctypes.c_double),
        ("omega_t", ctypes.c_double), ("gbeta", ctypes.c_double), ("t_ref", ctypes.c_double),
        ("r_split", ctypes.c_double), ("omega_w", ctypes.c_double * 4),
        ("t_w", ctypes.c_double * 4), ("collision", ctypes.c_int32), ("pad2", ctypes.c_int32),
        ("s_eps", ctypes.c_double), ("s_q", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, no -march)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        # AXLBM_ORACLE_LIB lets the mutation test load a deliberately broken copy
        path = os.environ.get("AXLBM_ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER(_Params)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_validate.argtypes = [P]
        lib.orc_step.argtypes = [P, ctypes.c_int64, ctypes.c_int64, dp, dp, dp]
        lib.orc_moments.argtypes = [P, ctypes.c_int64, dp, dp, dp, dp]
        lib.orc_equilibrium.argtypes = [P, dp, dp, dp, dp]
        lib.orc_stats.argtypes = [P, ctypes.c_int64, dp, dp, dp, dp, dp, dp]
        lib.orc_collide_cell.argtypes = [P, ctypes.c_double, ctypes.c_double, dp, dp, dp,
                                         dp, dp, dp, dp]
        lib.orc_collide_cell.restype = None
        lib.orc_stream.argtypes = [P, dp, dp, dp, dp, dp, dp]
        lib.orc_stream.restype = None
        lib.orc_mrt_matrix.argtypes = [dp]
        lib.orc_mrt_matrix.restype = None
        _lib = lib
    return _lib


def params(pb) -> _Params:
    """Translate a Problem into the oracle's parameter block."""
    p = _Params()
    p.nr, p.nz = int(pb.nr), int(pb.nz)
    p.inner = INNER[pb.inner]
    p.z_lo, p.z_hi = ZKIND[pb.z_lo], ZKIND[pb.z_hi]
    p.outer = OUTER[getattr(pb, "outer", "wall")]
    p.swirl, p.temperature = int(bool(pb.swirl)), int(bool(pb.temperature))
    for i, face in enumerate(FACES):
        p.t_dirichlet[i] = int(face in pb.t_wall)
        p.t_w[i] = float(pb.t_wall.get(face, 0.0))
        p.omega_w[i] = float(pb.omega.get(face, 0.0))
    p.r0, p.tau_s, p.tau_t_s, p.rho0 = float(pb.r0), float(pb.tau), float(pb.tau_t), float(pb.rho0)
    p.az0, p.omega_t = float(pb.az0), float(pb.omega_t)
    p.gbeta, p.t_ref, p.r_split = float(pb.gbeta), float(pb.t_ref), float(pb.r_split)
    p.collision = {"bgk": 0, "mrt": 1}[getattr(pb, "collision", "bgk")]
    p.s_eps, p.s_q = float(getattr(pb, "s_eps", 0.0)), float(getattr(pb, "s_q", 0.0))
    return p


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class State:
    """Populations of one domain at time t: f [9][nz][nr], g [4][nz][nr], h [4][nz][nr]."""

    def __init__(self, pb, f=None, g=None, h=None, t: int = 0):
        self.pb = pb
        shape = (pb.nz, pb.nr)
        self.f = np.zeros((9,) + shape) if f is None else np.ascontiguousarray(f, dtype=np.float64)
        self.g = np.zeros((4,) + shape) if g is None else np.ascontiguousarray(g, dtype=np.float64)
        self.h = np.zeros((4,) + shape) if h is None else np.ascontiguousarray(h, dtype=np.float64)
        self.t = int(t)

    def copy(self) -> "State":
        return State(self.pb, self.f.copy(), self.g.copy(), self.h.copy(), self.t)


def validate(pb) -> bool:
    p = params(pb)
    return _load().orc_validate(ctypes.byref(p)) == 0


def equilibrium(pb, fields: np.ndarray, t: int = 0) -> State:
    """Equilibrium populations (Eqs. 6 and 54) for macroscopic fields [5][nz][nr]."""
    p = params(pb)
    fields = np.ascontiguousarray(fields, dtype=np.float64)
    assert fields.shape == (5, pb.nz, pb.nr)
    st = State(pb, t=t)
    rc = _load().orc_equilibrium(ctypes.byref(p), _ptr(fields), _ptr(st.f), _ptr(st.g), _ptr(st.h))
    if rc:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return st


def rest_state(pb, t_init: float = None) -> State:
    """Fluid at rest with rho = rho0 and uniform temperature (t_ref unless given)."""
    fields = np.zeros((5, pb.nz, pb.nr))
    fields[0] = pb.rho0
    fields[4] = pb.t_ref if t_init is None else t_init
    return equilibrium(pb, fields)


def step(st: State, n: int) -> State:
    """Advance st by n time steps in place; returns st."""
    p = params(st.pb)
    rc = _load().orc_step(ctypes.byref(p), st.t, int(n), _ptr(st.f), _ptr(st.g), _ptr(st.h))
    if rc:
        raise ValueError(f"oracle step failed (code {rc})")
    st.t += int(n)
    return st


def moments(st: State) -> np.ndarray:
    """Macroscopic fields [5][nz][nr] (rho, u_r, u_z, u_theta, T) at time st.t."""
    p = params(st.pb)
    out = np.empty((5, st.pb.nz, st.pb.nr))
    rc = _load().orc_moments(ctypes.byref(p), st.t, _ptr(st.f), _ptr(st.g), _ptr(st.h), _ptr(out))
    if rc:
        raise ValueError(f"oracle moments failed (code {rc})")
    return out


def stats(st: State):
    """(mass, budget, speed[nz][nr]) at time st.t; see orc_stats."""
    p = params(st.pb)
    mass = ctypes.c_double()
    budget = ctypes.c_double()
    speed = np.empty((st.pb.nz, st.pb.nr))
    rc = _load().orc_stats(ctypes.byref(p), st.t, _ptr(st.f), _ptr(st.g), _ptr(st.h),
                           ctypes.byref(mass), ctypes.byref(budget), _ptr(speed))
    if rc:
        raise ValueError(f"oracle stats failed (code {rc})")
    return mass.value, budget.value, speed


def collide_cell(pb, r: float, a_t: float, f, g=None, h=None):
    """Post-collision populations of one node; returns (f*, g*, h*, moments)."""
    p = params(pb)
    fi = np.ascontiguousarray(f, dtype=np.float64)
    gi = np.ascontiguousarray(np.zeros(4) if g is None else g, dtype=np.float64)
    hi = np.ascontiguousarray(np.zeros(4) if h is None else h, dtype=np.float64)
    fo, go, ho, mom = np.zeros(9), np.zeros(4), np.zeros(4), np.zeros(5)
    _load().orc_collide_cell(ctypes.byref(p), float(r), float(a_t), _ptr(fi), _ptr(gi), _ptr(hi),
                             _ptr(fo), _ptr(go), _ptr(ho), _ptr(mom))
    return fo, go, ho, mom


def stream(pb, fp, gp=None, hp=None):
    """Streaming (with boundary rules) of post-collision lattices; returns (f, g, h)."""
    p = params(pb)
    shape = (pb.nz, pb.nr)
    fp = np.ascontiguousarray(fp, dtype=np.float64)
    gp = np.ascontiguousarray(np.zeros((4,) + shape) if gp is None else gp, dtype=np.float64)
    hp = np.ascontiguousarray(np.zeros((4,) + shape) if hp is None else hp, dtype=np.float64)
    fn = np.full((9,) + shape, np.nan)
    gn = np.full((4,) + shape, np.nan) if pb.swirl else np.zeros((4,) + shape)
    hn = np.full((4,) + shape, np.nan) if pb.temperature else np.zeros((4,) + shape)
    _load().orc_stream(ctypes.byref(p), _ptr(fp), _ptr(gp), _ptr(hp), _ptr(fn), _ptr(gn), _ptr(hn))
    return fn, gn, hn


def node_radii(pb) -> np.ndarray:
    return pb.r0 + np.arange(pb.nr) + (0.0 if pb.inner == "axis_node" else 0.5)


def mrt_matrix() -> np.ndarray:
    """The oracle's MRT moment basis M (9 x 9), rows as in Eq. 38."""
    out = np.empty(81)
    _load().orc_mrt_matrix(_ptr(out))
    return out.reshape(9, 9)
