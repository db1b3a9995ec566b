"""ark_compute_dt_noalloc: the CFL time step of a caller's FP64 device state
without any device allocation, against the handle-based ark_compute_dt.

Callers that cannot allocate device memory when they need a time step (a
memory pool or arena that owns the device, a thread that must not trigger an
allocation) use this entry point; its only scratch is a fixed array inside
the library.  The file name makes pytest collect it last.
"""
import ctypes
import math

import numpy as np
import pytest

from paper_1903_09043_gb300 import inputs as I
from parity import F64_TOL

MAX_CELLS = 67_108_864
CELLS_PER_SLOT = 4096


def _ark():
    from paper_1903_09043_gb300 import ark
    return ark


def test_noalloc_rejects_grids_beyond_its_scratch():
    """Rejected before any device work, so this runs without a GPU."""
    ark = _ark()
    prob, _ = I.random_periodic(3, (4, 4, 4))
    p = ark.params_from_problem(prob.replace(n=(1024, 1024, 65)), ark.ARK_F64)
    assert 1024 * 1024 * 65 > MAX_CELLS
    fake = ctypes.c_void_p(16)   # never dereferenced: the checks come before any launch
    assert ark.ark_compute_dt_noalloc(ctypes.byref(p), fake, fake, None) == ark.ARK_ERR_INVALID_ARG
    p32 = ark.params_from_problem(prob, ark.ARK_F32)
    assert ark.ark_compute_dt_noalloc(ctypes.byref(p32), fake, fake, None) == ark.ARK_ERR_INVALID_ARG
    assert ark.ark_compute_dt_noalloc(None, fake, fake, None) == ark.ARK_ERR_INVALID_ARG


def test_noalloc_rejects_what_ark_create_rejects():
    """Non-finite box corners, gravity or coefficients, and a potential array,
    are refused before any device work."""
    ark = _ark()
    prob, _ = I.random_periodic(2, (8, 8), mu=0.1, kappa=0.1)
    fake = ctypes.c_void_p(16)
    for field, value in (("hi", math.inf), ("lo", -math.inf), ("mu", math.nan), ("kappa", math.inf),
                         ("cfl", math.inf), ("gamma", math.inf), ("K", math.nan)):
        p = ark.params_from_problem(prob, ark.ARK_F64)
        if field in ("hi", "lo"):
            getattr(p.grid, field)[0] = value
        elif field == "gamma":
            p.eos.gamma = value
        else:
            setattr(p, field, value)
        assert ark.ark_compute_dt_noalloc(ctypes.byref(p), fake, fake, None) == ark.ARK_ERR_INVALID_ARG, field
    sp, _ = I.stratified_random(2, (8, 8))
    p = ark.params_from_problem(sp, ark.ARK_F64)
    p.gravity.g = math.inf
    assert ark.ark_compute_dt_noalloc(ctypes.byref(p), fake, fake, None) == ark.ARK_ERR_INVALID_ARG
    pp, _ = I.periodic_potential_state(2, (8, 8))
    p = ark.params_from_problem(pp, ark.ARK_F64)
    assert ark.ark_compute_dt_noalloc(ctypes.byref(p), fake, fake, None) == ark.ARK_ERR_UNSUPPORTED


def _noalloc(ark, prob, Ud, out, stream):
    p = ark.params_from_problem(prob, ark.ARK_F64)
    return ark.ark_compute_dt_noalloc(ctypes.byref(p), ctypes.c_void_p(Ud.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))


def _handle_dt(ark, prob, U, stream):
    with ark.Solver(prob, "f64", stream=stream) as s:
        s.set_state(U)
        return s.compute_dt()


@pytest.mark.gpu
def test_noalloc_dt_matches_handle_dt_on_consecutive_calls():
    import torch
    ark = _ark()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [I.rayleigh_benard(3, (40, 36, 24), amp=1e-3),
             I.atmosphere((128, 128)),
             I.random_periodic(2, (300, 7), seed=4, mu=0.5, kappa=0.2),
             I.random_periodic(3, (17, 9, 13), seed=6, mu=0.3, kappa=0.4),   # 3D viscous, rate from dissipation
             I.random_periodic(2, (64, 64), seed=8),                         # exactly one scratch slot
             I.random_periodic(2, (5, 3), seed=9),                           # a single partial slot
             I.rayleigh_benard(3, (128, 128, 64), amp=1e-3)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for prob, U in cases:
        ref = _handle_dt(ark, prob, U, stream)
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        for _ in range(2):
            out.fill_(-1.0)
            assert _noalloc(ark, prob, Ud, out, stream) == ark.ARK_OK
            torch.cuda.synchronize()
            assert out.item() == pytest.approx(ref, rel=F64_TOL)


@pytest.mark.gpu
def test_noalloc_at_its_largest_grid():
    """512 x 512 x 256 = 67,108,864 cells fills every scratch slot."""
    import torch
    ark = _ark()
    stream = torch.cuda.current_stream().cuda_stream
    prob, U = I.rayleigh_benard(3, (512, 512, 256), m=0.1, chi=1.1, Ra=1e7, amp=1e-3, seed=4)
    assert prob.ncells == MAX_CELLS
    ref = _handle_dt(ark, prob, U, stream)
    Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
    del U
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        out.fill_(-1.0)
        assert _noalloc(ark, prob, Ud, out, stream) == ark.ARK_OK
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=F64_TOL)


@pytest.mark.gpu
def test_noalloc_reports_a_bad_state_as_nan():
    """One NaN cell, or one cell with rho <= 0, gives a NaN time step rather
    than a finite step from the healthy cells; the next call on a healthy
    state gives the handle's time step again."""
    import torch
    ark = _ark()
    stream = torch.cuda.current_stream().cuda_stream
    prob, U = I.rayleigh_benard(3, (64, 40, 48), amp=1e-3)
    ref = _handle_dt(ark, prob, U, stream)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    nf = prob.nfields
    plants = [(nf - 1, (7, 3, 11), np.nan),     # NaN energy: NaN rate
              (0, (40, 39, 63), -1.0),           # negative density
              (nf - 1, (0, 0, 0), -1e3),         # negative pressure
              (0, (47, 0, 5), np.nan)]           # NaN density in the last block
    for f, (k, j, i), v in plants:
        B = np.array(U, copy=True)
        B[f, k, j, i] = v
        Bd = torch.from_numpy(B).cuda()
        out.fill_(1.0)
        assert _noalloc(ark, prob, Bd, out, stream) == ark.ARK_OK
        torch.cuda.synchronize()
        assert math.isnan(out.item()), (f, k, j, i, v, out.item())
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        out.fill_(-1.0)
        assert _noalloc(ark, prob, Ud, out, stream) == ark.ARK_OK
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref, rel=F64_TOL)
