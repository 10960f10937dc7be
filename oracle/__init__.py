"""FP64 CPU oracle of the D2Q9 moving-solid lattice-Boltzmann step.

TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
CPU-baseline leg of the benchmark may import this module.  The CUDA library
never calls it; the two implementations share no code.

The arithmetic lives in ``lbm_oracle.c`` (plain C, FP64, floating-point
contraction off).  This module builds it with gcc on first use and wraps it
with ctypes.  Every function cites the passage of Wen et al.,
arXiv:1303.0625, that it follows; see the C file's header for the step order
and for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liblbm_oracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, WALL, OPEN = 0, 1, 2
PRESCRIBED, FREE = 0, 1
RHOW_CONST, RHOW_LOCAL = 0, 1
REFILL_A1, REFILL_A2, REFILL_A3 = 1, 2, 3
CME, GME = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, FP64, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP for the per-node loops where the compiler has it; else one thread
        if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
            subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


class Config(ctypes.Structure):
    """Mirror of ``ora_config`` in lbm_oracle.c."""

    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
        ("u0x", ctypes.c_double), ("u0y", ctypes.c_double),
        ("wall_ux", ctypes.c_double * 2),
        ("body_fx", ctypes.c_double), ("body_fy", ctypes.c_double),
        ("inflow_umax", ctypes.c_double),
        ("gravity_x", ctypes.c_double), ("gravity_y", ctypes.c_double),
        ("lub_range", ctypes.c_double),
        ("rho_w_mode", ctypes.c_int32), ("refill", ctypes.c_int32),
        ("motion_cme", ctypes.c_int32), ("relative_changes", ctypes.c_int32),
        ("collision", ctypes.c_int32), ("boundary", ctypes.c_int32),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P, D, I32, I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        sig = {
            "ora_create": (P, [ctypes.POINTER(Config)]),
            "ora_destroy": (None, [P]),
            "ora_add_disk": (ctypes.c_int, [P, D, D, D, D, D, D, D, ctypes.c_int]),
            "ora_step": (None, [P, I64, dp]),
            "ora_time": (I64, [P]),
            "ora_nsolid": (ctypes.c_int, [P]),
            "ora_get_f": (None, [P, dp]),
            "ora_set_f": (None, [P, dp]),
            "ora_get_owner": (None, [P, ip]),
            "ora_fields": (None, [P, dp, dp, dp]),
            "ora_solid_state": (None, [P, ctypes.c_int, dp]),
            "ora_set_solid_state": (None, [P, ctypes.c_int, dp]),
            "ora_links": (I64, [P, I64, ip]),
            "ora_refill_probe": (None, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]),
            "ora_feq": (None, [D, D, D, dp]),
            "ora_link_force": (None, [ctypes.c_int, D, D, D, D, dp]),
            "ora_pending": (None, [P, dp]),
            "ora_mrt_node": (None, [dp, dp, dp]),
            "ora_set_threads": (ctypes.c_int, [ctypes.c_int]),
            "ora_link_fraction": (ctypes.c_double, [P, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                    ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def feq(rho: float, ux: float, uy: float) -> np.ndarray:
    """Eq. 8 equilibrium populations (9,) in the D2Q9 order of Sec. III.C."""
    out = np.empty(9)
    _load().ora_feq(rho, ux, uy, _dp(out))
    return out


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's per-node loops (n < 1: all cores); returns the
    count in effect (1 when the oracle was built without OpenMP)."""
    return int(_load().ora_set_threads(int(n)))


def mrt_node(f, s) -> np.ndarray:
    """One MRT collision of a node's populations f (9,) with moment rates s
    (9,) in the basis (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    out = np.empty(9)
    _load().ora_mrt_node(_dp(f), _dp(s), _dp(out))
    return out


MRT_RATES = (0.0, 1.64, 1.54, 0.0, 1.9, 0.0, 1.9)  # then 1/tau twice (Sec. IV)


def link_force(i: int, fi: float, fbb: float, vx: float, vy: float) -> np.ndarray:
    """Per-link force on the solid: [Eq. 4 x, Eq. 4 y, Eq. 5 x, Eq. 5 y].

    ``fi`` streams from the fluid node into the boundary along e_i, ``fbb``
    streams out of the boundary along -e_i; (vx, vy) is the boundary velocity
    at the intersection point (Sec. III.A-B)."""
    out = np.empty(4)
    _load().ora_link_force(int(i), fi, fbb, vx, vy, _dp(out))
    return out


class Oracle:
    """One D2Q9 domain with rigid disks, advanced step by step in FP64."""

    def __init__(self, nx, ny, tau, *, rho0=1.0, u0=(0.0, 0.0), bc_x=PERIODIC, bc_y=PERIODIC,
                 wall_ux=(0.0, 0.0), body_force=(0.0, 0.0), inflow_umax=0.0,
                 gravity=(0.0, 0.0), lub_range=0.0, rho_w_mode=RHOW_CONST, refill=REFILL_A1,
                 motion_cme=0, relative_changes=0, collision=0, boundary=0):
        lib = _load()
        c = Config()
        c.nx, c.ny, c.bc_x, c.bc_y = int(nx), int(ny), int(bc_x), int(bc_y)
        c.tau, c.rho0 = float(tau), float(rho0)
        c.u0x, c.u0y = float(u0[0]), float(u0[1])
        c.wall_ux[0], c.wall_ux[1] = float(wall_ux[0]), float(wall_ux[1])
        c.body_fx, c.body_fy = float(body_force[0]), float(body_force[1])
        c.inflow_umax = float(inflow_umax)
        c.gravity_x, c.gravity_y = float(gravity[0]), float(gravity[1])
        c.lub_range = float(lub_range)
        c.rho_w_mode, c.refill = int(rho_w_mode), int(refill)
        c.motion_cme = int(motion_cme)
        c.relative_changes = int(relative_changes)
        c.collision = int(collision)
        c.boundary = int(boundary)
        self._lib = lib
        self._h = lib.ora_create(ctypes.byref(c))
        if not self._h:
            raise ValueError("invalid oracle configuration")
        self.nx, self.ny = int(nx), int(ny)
        self._radius = []

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.ora_destroy(h)
            self._h = None

    @property
    def t(self) -> int:
        return int(self._lib.ora_time(self._h))

    @property
    def nsolid(self) -> int:
        return int(self._lib.ora_nsolid(self._h))

    def add_disk(self, cx, cy, r, vx=0.0, vy=0.0, omega=0.0, rho_s=1.0, motion=PRESCRIBED) -> int:
        self._radius.append(float(r))
        return int(self._lib.ora_add_disk(self._h, cx, cy, r, vx, vy, omega, rho_s, int(motion)))

    def step(self, n: int = 1, record: bool = True):
        """Advance n steps; returns forces [n][nsolid][2 (Eq. 4, Eq. 5)][Fx, Fy, T]."""
        n = int(n)
        if record:
            rec = np.zeros((n, max(self.nsolid, 1), 2, 3))
            self._lib.ora_step(self._h, n, _dp(rec))
            return rec[:, : self.nsolid]
        self._lib.ora_step(self._h, n, None)
        return None

    def get_f(self) -> np.ndarray:
        out = np.empty((9, self.ny, self.nx))
        self._lib.ora_get_f(self._h, _dp(out))
        return out

    def set_f(self, f: np.ndarray) -> None:
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(9, self.ny, self.nx)
        self._lib.ora_set_f(self._h, _dp(f))

    def owner(self) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=np.int32)
        self._lib.ora_get_owner(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return out

    def fields(self):
        rho = np.empty((self.ny, self.nx))
        ux = np.empty_like(rho)
        uy = np.empty_like(rho)
        self._lib.ora_fields(self._h, _dp(rho), _dp(ux), _dp(uy))
        return rho, ux, uy

    def solid_state(self, s: int) -> np.ndarray:
        """[x, y, vx, vy, omega] of solid s at the current time."""
        out = np.empty(5)
        self._lib.ora_solid_state(self._h, int(s), _dp(out))
        return out

    def link_fraction(self, s: int, x: int, y: int, i: int) -> float:
        """Fraction of the link from node (x, y) along e_i at which it meets disk s."""
        return float(self._lib.ora_link_fraction(self._h, int(s), int(x), int(y), int(i)))

    def solid_radius(self, s: int) -> float:
        return float(self._radius[s])

    def set_solid_state(self, s: int, state) -> None:
        st = np.ascontiguousarray(state, dtype=np.float64)
        self._lib.ora_set_solid_state(self._h, int(s), _dp(st))

    def links(self) -> np.ndarray:
        """All fluid-solid links as rows (x_f, y_f, i, solid), raster order."""
        n = int(self._lib.ora_links(self._h, 0, None))
        out = np.zeros((max(n, 1), 4), dtype=np.int32)
        self._lib.ora_links(self._h, n, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        return out[:n]

    def pending(self) -> np.ndarray:
        """Momentum [nsolid][Fx, Fy, T] booked for the next force record."""
        out = np.zeros((max(self.nsolid, 1), 3))
        self._lib.ora_pending(self._h, _dp(out))
        return out[: self.nsolid]

    def refill_probe(self, x: int, y: int, s: int = -1) -> np.ndarray:
        out = np.empty(9)
        self._lib.ora_refill_probe(self._h, int(x), int(y), int(s), _dp(out))
        return out
