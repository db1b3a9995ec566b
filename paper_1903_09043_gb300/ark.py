"""Thin ctypes binding of libark.so (include/ark.h): argument marshalling only.

Every step of the method runs in the CUDA kernels of ``libark.so``; this
module translates a :class:`paper_1903_09043_gb300.inputs.Problem` into
``ark_params``, passes host arrays (numpy) or device tensors (torch, via
``data_ptr``) and CUDA streams (``torch.cuda.Stream.cuda_stream``) through,
and raises :class:`ArkError` on any non-OK status.  There is no CPU path: if
the library is missing, importing this module fails.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libark.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

ARK_OK = 0
ARK_ERR_INVALID_ARG = 1
ARK_ERR_CUDA = 2
ARK_ERR_NONPHYSICAL = 3
ARK_ERR_TIMEOUT = 4
ARK_ERR_UNSUPPORTED = 5
ARK_ERR_ALLOC = 6

ARK_BC_PERIODIC = 0
ARK_BC_REFLECT_HYDRO = 1
ARK_BC_NOSLIP_FIXED_T = 2
ARK_BC_OUTFLOW = 3
ARK_BC_HALO = 4

ARK_F64 = 0
ARK_F32 = 1
ARK_F32_SPLIT = 2

ARK_EOS_STIFFENED_GAS = 0
ARK_EOS_NOBLE_ABEL = 1
PRECISIONS = {"f64": ARK_F64, "f32": ARK_F32, "f32split": ARK_F32_SPLIT}


class ark_grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3)]


class ark_eos(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("p_inf", ctypes.c_double), ("law", ctypes.c_int),
                ("b", ctypes.c_double)]


class ark_gravity(ctypes.Structure):
    _fields_ = [("g", ctypes.c_double), ("phi", ctypes.POINTER(ctypes.c_double))]


class ark_bc(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_int * 3), ("hi", ctypes.c_int * 3), ("T_lo", ctypes.c_double * 3),
                ("T_hi", ctypes.c_double * 3)]


class ark_params(ctypes.Structure):
    _fields_ = [("grid", ark_grid), ("eos", ark_eos), ("gravity", ark_gravity), ("mu", ctypes.c_double),
                ("kappa", ctypes.c_double), ("low_mach", ctypes.c_int), ("K", ctypes.c_double),
                ("cfl", ctypes.c_double), ("bc", ark_bc), ("precision", ctypes.c_int),
                ("energy_form", ctypes.c_int)]


class ark_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("momentum", ctypes.c_double * 3), ("energy", ctypes.c_double),
                ("kinetic", ctypes.c_double), ("max_speed", ctypes.c_double), ("mean_abs_v_last", ctypes.c_double),
                ("min_rho", ctypes.c_double), ("min_p", ctypes.c_double), ("t", ctypes.c_double),
                ("step", ctypes.c_longlong), ("dt", ctypes.c_double), ("status", ctypes.c_uint)]


_H = ctypes.c_void_p
_st = ctypes.c_int
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

_SIGS = {
    "ark_create": (_st, [ctypes.POINTER(ark_params), ctypes.c_void_p, ctypes.POINTER(_H)]),
    "ark_destroy": (_st, [_H]),
    "ark_set_state": (_st, [_H, ctypes.c_void_p, ctypes.c_int]),
    "ark_get_state": (_st, [_H, ctypes.c_void_p, ctypes.c_int]),
    "ark_compute_dt": (_st, [_H, _dp]),
    "ark_step": (_st, [_H, ctypes.c_int, ctypes.c_double]),
    "ark_diagnostics": (_st, [_H, ctypes.POINTER(ark_diag)]),
    "ark_sync": (_st, [_H, ctypes.c_double]),
    "ark_time": (_st, [_H, _dp, _dp]),
    "ark_state_device_ptr": (_st, [_H, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_size_t)]),
    "ark_get_halo": (_st, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "ark_set_halo": (_st, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "ark_launch_shape": (_st, [_H, _ip, _ip, _ip, _ip, _ip]),
    "ark_compute_dt_noalloc": (_st, [ctypes.POINTER(ark_params), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "ark_batch_create": (_st, [ctypes.c_int, ctypes.POINTER(ark_params), ctypes.c_void_p, ctypes.POINTER(_H)]),
    "ark_batch_set_state": (_st, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "ark_batch_get_state": (_st, [_H, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "ark_batch_tune": (_st, [_H, ctypes.c_int, _ip, _ip]),
    "ark_batch_step": (_st, [_H, ctypes.c_int]),
    "ark_batch_diagnostics": (_st, [_H, ctypes.c_int, ctypes.POINTER(ark_diag)]),
    "ark_batch_shape": (_st, [_H, _ip, _ip, _ip, _ip]),
    "ark_batch_destroy": (_st, [_H]),
    "ark_batch_last_error": (ctypes.c_char_p, [_H]),
    "ark_last_error": (ctypes.c_char_p, [_H]),
    "ark_status_string": (ctypes.c_char_p, [ctypes.c_int]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

# The same names as the C ABI.
ark_create = _lib.ark_create
ark_destroy = _lib.ark_destroy
ark_set_state = _lib.ark_set_state
ark_get_state = _lib.ark_get_state
ark_compute_dt = _lib.ark_compute_dt
ark_step = _lib.ark_step
ark_diagnostics = _lib.ark_diagnostics
ark_sync = _lib.ark_sync
ark_time = _lib.ark_time
ark_state_device_ptr = _lib.ark_state_device_ptr
ark_get_halo = _lib.ark_get_halo
ark_set_halo = _lib.ark_set_halo
ark_launch_shape = _lib.ark_launch_shape
ark_compute_dt_noalloc = _lib.ark_compute_dt_noalloc
ark_last_error = _lib.ark_last_error
ark_status_string = _lib.ark_status_string
ark_batch_create = _lib.ark_batch_create
ark_batch_set_state = _lib.ark_batch_set_state
ark_batch_get_state = _lib.ark_batch_get_state
ark_batch_tune = _lib.ark_batch_tune
ark_batch_step = _lib.ark_batch_step
ark_batch_diagnostics = _lib.ark_batch_diagnostics
ark_batch_shape = _lib.ark_batch_shape
ark_batch_destroy = _lib.ark_batch_destroy
ark_batch_last_error = _lib.ark_batch_last_error


class ArkError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


def params_from_problem(prob, precision: int = ARK_F64) -> ark_params:
    p = ark_params()
    p.grid.dim = prob.dim
    for d in range(3):
        p.grid.n[d] = int(prob.n[d]) if d < prob.dim else 1
        p.grid.lo[d] = float(prob.lo[d])
        p.grid.hi[d] = float(prob.hi[d])
        p.bc.lo[d] = int(prob.bc_lo[d])
        p.bc.hi[d] = int(prob.bc_hi[d])
        p.bc.T_lo[d] = float(prob.T_lo[d])
        p.bc.T_hi[d] = float(prob.T_hi[d])
    p.eos.gamma = float(prob.gamma)
    p.eos.p_inf = float(getattr(prob, "p_inf", 0.0))
    b = float(getattr(prob, "b", 0.0))
    p.eos.law = ARK_EOS_NOBLE_ABEL if b != 0.0 else ARK_EOS_STIFFENED_GAS
    p.eos.b = b
    p.gravity.g = float(prob.g)
    phi = getattr(prob, "phi", None)
    if phi is not None:   # caller-supplied potential: a host array ark_create copies
        arr = np.ascontiguousarray(phi, dtype=np.float64)
        p._phi_keep = arr
        p.gravity.phi = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        p.gravity.g = 0.0
    p.mu = float(prob.mu)
    p.kappa = float(prob.kappa)
    p.low_mach = int(prob.low_mach)
    p.K = float(prob.K)
    p.cfl = float(prob.cfl)
    p.precision = int(precision)
    p.energy_form = int(getattr(prob, "energy_form", 0))
    return p


def _ptr(x):
    """(address, on_device) of a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("state arrays must be C-contiguous float64")
        return x.ctypes.data, 0
    import torch
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise ValueError("state tensors must be contiguous float64")
    return x.data_ptr(), 1 if x.is_cuda else 0


class Solver:
    """One grid behind the C ABI (ark_create ... ark_destroy)."""

    def __init__(self, prob, precision="f64", stream: Optional[int] = None):
        self.prob = prob
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        self.precision = prec
        self.params = params_from_problem(prob, prec)
        h = _H()
        st = ark_create(ctypes.byref(self.params), ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != ARK_OK:
            raise ArkError(st, f"ark_create: {ark_status_string(st).decode()}")
        self.h = h

    def _check(self, st: int, what: str):
        if st != ARK_OK:
            raise ArkError(st, f"{what}: {ark_last_error(self.h).decode()}")

    def set_state(self, U) -> None:
        addr, dev = _ptr(U)
        self._check(ark_set_state(self.h, ctypes.c_void_p(addr), dev), "ark_set_state")

    def get_state(self, out=None):
        if out is None:
            out = np.empty((self.prob.nfields,) + self.prob.shape, dtype=np.float64)
        addr, dev = _ptr(out)
        self._check(ark_get_state(self.h, ctypes.c_void_p(addr), dev), "ark_get_state")
        return out

    def compute_dt(self) -> float:
        dt = ctypes.c_double(0.0)
        self._check(ark_compute_dt(self.h, ctypes.byref(dt)), "ark_compute_dt")
        return dt.value

    def step(self, nsteps: int = 1, dt: float = -1.0) -> None:
        self._check(ark_step(self.h, int(nsteps), float(dt)), "ark_step")

    def diagnostics(self, check: bool = True) -> dict:
        d = ark_diag()
        st = ark_diagnostics(self.h, ctypes.byref(d))
        if check:
            self._check(st, "ark_diagnostics")
        return {"mass": d.mass, "mom_x": d.momentum[0], "mom_y": d.momentum[1], "mom_z": d.momentum[2],
                "energy": d.energy, "kinetic": d.kinetic, "max_speed": d.max_speed,
                "mean_abs_v_last": d.mean_abs_v_last, "min_rho": d.min_rho, "min_p": d.min_p, "t": d.t,
                "step": d.step, "dt": d.dt, "status": d.status}

    def time(self):
        t = ctypes.c_double(0.0)
        dt = ctypes.c_double(0.0)
        self._check(ark_time(self.h, ctypes.byref(t), ctypes.byref(dt)), "ark_time")
        return t.value, dt.value

    def sync(self, timeout_s: float = 60.0) -> None:
        self._check(ark_sync(self.h, float(timeout_s)), "ark_sync")

    def launch_shape(self) -> dict:
        v = [ctypes.c_int(0) for _ in range(5)]
        self._check(ark_launch_shape(self.h, *[ctypes.byref(x) for x in v]), "ark_launch_shape")
        return dict(zip(("tx", "ty", "planes", "threads", "blocks"), [x.value for x in v]))

    def halo_shape(self):
        """Shape of a halo buffer: (fields, planes of the last axis, rows of y (1 in 2D), 2 layers)."""
        p = self.prob
        return (p.nfields, p.n[p.dim - 1], p.n[1] if p.dim == 3 else 1, 2)

    def get_halo(self, side: int, out=None):
        """The two cell layers next to x side ``side`` (0 low, 1 high), layer 0 at the side."""
        if out is None:
            out = np.empty(self.halo_shape(), dtype=np.float64)
        addr, dev = _ptr(out)
        self._check(ark_get_halo(self.h, int(side), ctypes.c_void_p(addr), dev), "ark_get_halo")
        return out

    def set_halo(self, side: int, layers) -> None:
        """Ghost layers beyond the ARK_BC_HALO side ``side`` (layer 0 adjacent to the side)."""
        addr, dev = _ptr(layers)
        self._check(ark_set_halo(self.h, int(side), ctypes.c_void_p(addr), dev), "ark_set_halo")

    def state_device_ptr(self):
        p = ctypes.c_void_p()
        n = ctypes.c_size_t()
        self._check(ark_state_device_ptr(self.h, ctypes.byref(p), ctypes.byref(n)), "ark_state_device_ptr")
        return p.value, n.value

    def close(self) -> None:
        if getattr(self, "h", None):
            ark_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _diag_dict(d: ark_diag) -> dict:
    return {"mass": d.mass, "mom_x": d.momentum[0], "mom_y": d.momentum[1], "mom_z": d.momentum[2],
            "energy": d.energy, "kinetic": d.kinetic, "max_speed": d.max_speed,
            "mean_abs_v_last": d.mean_abs_v_last, "min_rho": d.min_rho, "min_p": d.min_p, "t": d.t,
            "step": d.step, "dt": d.dt, "status": d.status}


class Batch:
    """An ensemble of independent 2D runs (ark_batch_create ... ark_batch_destroy)."""

    def __init__(self, probs, precision="f32split", stream: Optional[int] = None):
        self.probs = list(probs)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        arr = (ark_params * len(self.probs))(*[params_from_problem(p, prec) for p in self.probs])
        self._params = arr
        h = _H()
        st = ark_batch_create(len(self.probs), arr, ctypes.c_void_p(stream or 0), ctypes.byref(h))
        if st != ARK_OK:
            raise ArkError(st, f"ark_batch_create: {ark_status_string(st).decode()}")
        self.h = h

    def _check(self, st: int, what: str):
        if st != ARK_OK:
            raise ArkError(st, f"{what}: {ark_batch_last_error(self.h).decode()}")

    def set_state(self, i: int, U) -> None:
        addr, dev = _ptr(U)
        self._check(ark_batch_set_state(self.h, int(i), ctypes.c_void_p(addr), dev), "ark_batch_set_state")

    def get_state(self, i: int, out=None):
        if out is None:
            p = self.probs[i]
            out = np.empty((p.nfields,) + p.shape, dtype=np.float64)
        addr, dev = _ptr(out)
        self._check(ark_batch_get_state(self.h, int(i), ctypes.c_void_p(addr), dev), "ark_batch_get_state")
        return out

    def tune(self, reps: int = 3):
        tx = ctypes.c_int(0)
        pl = ctypes.c_int(0)
        self._check(ark_batch_tune(self.h, int(reps), ctypes.byref(tx), ctypes.byref(pl)), "ark_batch_tune")
        return tx.value, pl.value

    def step(self, nsteps: int = 1) -> None:
        self._check(ark_batch_step(self.h, int(nsteps)), "ark_batch_step")

    def diagnostics(self, i: int, check: bool = True) -> dict:
        d = ark_diag()
        st = ark_batch_diagnostics(self.h, int(i), ctypes.byref(d))
        if check:
            self._check(st, "ark_batch_diagnostics")
        return _diag_dict(d)

    def shape(self) -> dict:
        v = [ctypes.c_int(0) for _ in range(4)]
        self._check(ark_batch_shape(self.h, *[ctypes.byref(x) for x in v]), "ark_batch_shape")
        return dict(zip(("tx", "planes", "items", "blocks"), [x.value for x in v]))

    def close(self) -> None:
        if getattr(self, "h", None):
            ark_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
