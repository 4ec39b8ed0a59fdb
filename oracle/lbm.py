"""ctypes front end of the plain FP64 C oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY (tests, ``__graft_entry__.smoke()``, bench CPU-baseline legs).
The C source follows Sec. 3 (BGK lattice Boltzmann, D2Q9) and Sec. 8.1/8.2 (cylinder
and Taylor-Green set-ups) of arXiv 2508.13867; see the header of ``lbm_oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle_lbm.so")

TGV, CHANNEL, TGV_PERTURBED = 0, 1, 2
HALFWAY, BOUZIDI = 0, 1  # obstacle schemes of the channel case
FACE, INTERPOLATED = 0, 1  # inlet/outlet schemes of the channel case


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags only; OpenMP across samples)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fopenmp", "-fPIC", "-shared",
               _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Case(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("steps", ctypes.c_int64), ("nu", ctypes.c_double), ("u0", ctypes.c_double),
                ("amp2", ctypes.c_double), ("amp3", ctypes.c_double), ("u_ref", ctypes.c_double),
                ("cyl_cx", ctypes.c_double), ("cyl_cy", ctypes.c_double),
                ("cyl_r", ctypes.c_double), ("ramp_steps", ctypes.c_int64),
                ("qoi_every", ctypes.c_int64), ("steady_tol", ctypes.c_double), ("pert", ctypes.c_double * 4),
                ("obstacle_bc", ctypes.c_int32), ("inout_bc", ctypes.c_int32)]


_P = ctypes.POINTER(ctypes.c_double)


class _Out(ctypes.Structure):
    _fields_ = [("u", _P), ("v", _P), ("rho", _P), ("series", _P), ("series_cl", _P),
                ("series_len", ctypes.c_int64), ("scalars", ctypes.c_double * 8)]


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.oracle_run_batch.argtypes = [ctypes.POINTER(_Case), ctypes.POINTER(_Out),
                                          ctypes.c_int64, ctypes.c_int]
        _lib.oracle_run_batch.restype = ctypes.c_int
        _lib.oracle_obstacle_mask.argtypes = [ctypes.POINTER(_Case), ctypes.c_void_p]
        _lib.oracle_obstacle_mask.restype = ctypes.c_int
        _lib.oracle_num_threads.restype = ctypes.c_int
        _lib.oracle_link_fraction.argtypes = [ctypes.POINTER(_Case), ctypes.c_int, ctypes.c_int, ctypes.c_int]
        _lib.oracle_link_fraction.restype = ctypes.c_double
    return _lib


@dataclass
class Case:
    """One deterministic run.  Lattice units throughout; tau = 3 nu + 1/2."""
    kind: int
    nx: int
    ny: int
    steps: int
    nu: float
    u0: float
    amp2: float = 0.0
    amp3: float = 0.0
    u_ref: float = 0.01
    cyl_cx: float = 0.0
    cyl_cy: float = 0.0
    cyl_r: float = 0.0
    ramp_steps: int = 0
    qoi_every: int = 0
    steady_tol: float = 0.0
    pert: tuple = (0.0, 0.0, 0.0, 0.0)
    obstacle_bc: int = HALFWAY
    inout_bc: int = FACE

    def _c(self) -> _Case:
        return _Case(self.kind, self.nx, self.ny, self.steps, self.nu, self.u0, self.amp2,
                     self.amp3, self.u_ref, self.cyl_cx, self.cyl_cy, self.cyl_r,
                     self.ramp_steps, self.qoi_every, self.steady_tol, (ctypes.c_double * 4)(*self.pert),
                     self.obstacle_bc, self.inout_bc)


@dataclass
class Result:
    u: np.ndarray
    v: np.ndarray
    rho: np.ndarray
    series: np.ndarray
    series_cl: np.ndarray
    k_final: float
    mass: float
    mom_x: float
    mom_y: float
    cd: float
    cl: float
    steps_run: int


def run(cases: list[Case], threads: int = 0) -> list[Result]:
    """Run independent samples (OpenMP across samples).  threads = 0: OpenMP default."""
    lib = _load()
    n = len(cases)
    carr = (_Case * n)(*[c._c() for c in cases])
    oarr = (_Out * n)()
    keep = []
    for i, c in enumerate(cases):
        nn = c.nx * c.ny
        u, v, rho = np.zeros(nn), np.zeros(nn), np.zeros(nn)
        ns = (c.steps // c.qoi_every + 1) if c.qoi_every > 0 else 0
        ser, ser_cl = np.full(max(ns, 1), np.nan), np.full(max(ns, 1), np.nan)
        keep.append((u, v, rho, ser, ser_cl))
        oarr[i].u = u.ctypes.data_as(_P)
        oarr[i].v = v.ctypes.data_as(_P)
        oarr[i].rho = rho.ctypes.data_as(_P)
        oarr[i].series = ser.ctypes.data_as(_P)
        oarr[i].series_cl = ser_cl.ctypes.data_as(_P)
        oarr[i].series_len = ns
    rc = lib.oracle_run_batch(carr, oarr, n, int(threads))
    if rc != 0:
        raise RuntimeError(f"oracle_run_batch failed with status {rc}")
    res = []
    for i, c in enumerate(cases):
        u, v, rho, ser, ser_cl = keep[i]
        s = list(oarr[i].scalars)
        shape = (c.ny, c.nx)
        res.append(Result(u.reshape(shape), v.reshape(shape), rho.reshape(shape), ser, ser_cl,
                          s[0], s[1], s[2], s[3], s[4], s[5], int(s[6])))
    return res


def obstacle_mask(case: Case) -> np.ndarray:
    """The oracle's staircase obstacle mask, [ny, nx] uint8 (1 = solid)."""
    lib = _load()
    m = np.zeros(case.nx * case.ny, dtype=np.uint8)
    c = case._c()
    if lib.oracle_obstacle_mask(ctypes.byref(c), m.ctypes.data) != 0:
        raise RuntimeError("oracle_obstacle_mask failed")
    return m.reshape(case.ny, case.nx)


def link_fraction(case: Case, x: int, y: int, i: int) -> float:
    """Fraction q of the link from node (x, y) along D2Q9 direction i at which it enters the
    obstacle circle (the oracle's Bouzidi geometry)."""
    c = case._c()
    return float(_load().oracle_link_fraction(ctypes.byref(c), x, y, i))


def num_threads() -> int:
    return int(_load().oracle_num_threads())
