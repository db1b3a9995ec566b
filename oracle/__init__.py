"""FP64 CPU oracle for the ARK explicit step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never uses it.

The arithmetic lives in ``ark_oracle.c`` (plain loops, FP64, optional
OpenMP); this module builds it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ark_oracle.c")
_LIB = os.path.join(_HERE, "libark_oracle.so")
_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("lo", ctypes.c_double * 3),
        ("dx", ctypes.c_double * 3),
        ("gamma", ctypes.c_double),
        ("g", ctypes.c_double * 3),
        ("mu", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("K", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("low_mach", ctypes.c_int),
        ("bc_lo", ctypes.c_int * 3),
        ("bc_hi", ctypes.c_int * 3),
        ("T_lo", ctypes.c_double * 3),
        ("T_hi", ctypes.c_double * 3),
        ("energy_form", ctypes.c_int),
        ("phi", ctypes.POINTER(ctypes.c_double)),
        ("p_inf", ctypes.c_double),
        ("b", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.POINTER(_Problem)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_step.argtypes = [P, dp, ctypes.c_double, dp]
        lib.orc_step.restype = ctypes.c_int
        lib.orc_step_window.argtypes = [P, dp, ctypes.c_double, ip, ip, dp]
        lib.orc_step_window.restype = ctypes.c_int
        lib.orc_dt.argtypes = [P, dp]
        lib.orc_dt.restype = ctypes.c_double
        lib.orc_diagnostics.argtypes = [P, dp, dp]
        lib.orc_diagnostics.restype = None
        lib.orc_cell_at.argtypes = [P, dp, ip, dp]
        lib.orc_cell_at.restype = None
        lib.orc_face.argtypes = [P, dp, dp, ctypes.c_int, dp]
        lib.orc_face.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (it is single-file plain C)."""
    _load().orc_set_threads(int(n))


def _struct(prob) -> _Problem:
    s = _Problem()
    s.dim = prob.dim
    dx = prob.dx
    for d in range(3):
        s.n[d] = int(prob.n[d]) if d < prob.dim else 1
        s.lo[d] = float(prob.lo[d])
        s.dx[d] = float(dx[d])
        s.g[d] = 0.0
        s.bc_lo[d] = int(prob.bc_lo[d])
        s.bc_hi[d] = int(prob.bc_hi[d])
        s.T_lo[d] = float(prob.T_lo[d])
        s.T_hi[d] = float(prob.T_hi[d])
    s.g[prob.dim - 1] = float(prob.g)
    s.gamma = float(prob.gamma)
    s.mu = float(prob.mu)
    s.kappa = float(prob.kappa)
    s.K = float(prob.K)
    s.cfl = float(prob.cfl)
    s.low_mach = int(prob.low_mach)
    s.energy_form = int(getattr(prob, "energy_form", 0))
    s.p_inf = float(getattr(prob, "p_inf", 0.0))
    s.b = float(getattr(prob, "b", 0.0))
    phi = getattr(prob, "phi", None)
    if phi is not None:
        arr = np.ascontiguousarray(phi, dtype=np.float64)
        if arr.shape != tuple(prob.shape):
            raise ValueError("phi must have the shape of one field")
        s._phi_keep = arr                      # the array outlives the call through the struct
        s.phi = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    else:
        s.phi = ctypes.POINTER(ctypes.c_double)()
    return s


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c64(U: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(U, dtype=np.float64)


def step(prob, U: np.ndarray, dt: float) -> np.ndarray:
    lib = _load()
    U = _c64(U)
    out = np.empty_like(U)
    rc = lib.orc_step(ctypes.byref(_struct(prob)), _dptr(U), float(dt), _dptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_step failed ({rc})")
    return out


def step_window(prob, U: np.ndarray, dt: float, wlo: Sequence[int], whi: Sequence[int]) -> np.ndarray:
    """Updated values of the cells in [wlo, whi) (x, y[, z] order), shape (nf, ...)."""
    lib = _load()
    U = _c64(U)
    lo = (ctypes.c_int * 3)(*(list(wlo) + [0] * (3 - len(wlo))))
    hi = (ctypes.c_int * 3)(*(list(whi) + [1] * (3 - len(whi))))
    ext = [hi[d] - lo[d] for d in range(prob.dim)]
    out = np.empty((prob.nfields,) + tuple(reversed(ext)), dtype=np.float64)
    rc = lib.orc_step_window(ctypes.byref(_struct(prob)), _dptr(U), float(dt), lo, hi, _dptr(out))
    if rc != 0:
        raise RuntimeError(f"orc_step_window failed ({rc})")
    return out


def dt(prob, U: np.ndarray) -> float:
    lib = _load()
    U = _c64(U)
    return float(lib.orc_dt(ctypes.byref(_struct(prob)), _dptr(U)))


DIAG_NAMES = ("mass", "mom_x", "mom_y", "mom_z", "energy", "kinetic", "max_speed", "mean_abs_v_last",
              "min_rho", "min_p")


def diagnostics(prob, U: np.ndarray) -> dict:
    lib = _load()
    U = _c64(U)
    out = np.zeros(10)
    lib.orc_diagnostics(ctypes.byref(_struct(prob)), _dptr(U), _dptr(out))
    return dict(zip(DIAG_NAMES, out.tolist()))


CELL_NAMES = ("rho", "m_x", "m_y", "m_z", "W", "u", "v", "w", "p", "T", "c", "phi")


def cell_at(prob, U: np.ndarray, ijk: Sequence[int]) -> dict:
    lib = _load()
    U = _c64(U)
    idx = (ctypes.c_int * 3)(*(list(ijk) + [0] * (3 - len(ijk))))
    out = np.zeros(12)
    lib.orc_cell_at(ctypes.byref(_struct(prob)), _dptr(U), idx, _dptr(out))
    return dict(zip(CELL_NAMES, out.tolist()))


def face(prob, left: Sequence[float], right: Sequence[float], d: int) -> dict:
    """Acoustic face values between primitive states (rho, u, v, w, p, phi)."""
    lib = _load()
    L = np.asarray(left, dtype=np.float64)
    R = np.asarray(right, dtype=np.float64)
    out = np.zeros(5)
    lib.orc_face(ctypes.byref(_struct(prob)), _dptr(L), _dptr(R), int(d), _dptr(out))
    return dict(zip(("a", "S", "ustar", "theta", "Pistar"), out.tolist()))


def run(prob, U: np.ndarray, nsteps: int, dt_fixed: float | None = None, t_end: float | None = None,
        return_dt: bool = False):
    """Advance ``nsteps`` steps (or until ``t_end``) with CFL time steps."""
    U = _c64(U).copy()
    t = 0.0
    dts = []
    for _ in range(nsteps):
        h = dt_fixed if dt_fixed is not None else dt(prob, U)
        if t_end is not None:
            if t >= t_end:
                break
            h = min(h, t_end - t)
        U = step(prob, U, h)
        t += h
        dts.append(h)
    if return_dt:
        return U, t, dts
    return U, t
