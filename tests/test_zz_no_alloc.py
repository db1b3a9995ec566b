"""ark_compute_dt_noalloc: the CFL time step of a caller's FP64 device state
without any device allocation, against the handle-based ark_compute_dt.

Callers that cannot allocate device memory when they need a time step (a
memory pool or arena that owns the device, a thread that must not trigger an
allocation) use this entry point; its only scratch is a fixed array inside
the library.  The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

from paper_1903_09043_gb300 import inputs as I
from parity import F64_TOL

MAX_CELLS = 67_108_864


def _ark():
    from paper_1903_09043_gb300 import ark
    return ark


def test_noalloc_rejects_grids_beyond_its_scratch():
    """Rejected before any device work, so this runs without a GPU."""
    ark = _ark()
    prob, _ = I.random_periodic(3, (4, 4, 4))
    p = ark.params_from_problem(prob.replace(n=(1024, 1024, 65)), ark.ARK_F64)
    assert 1024 * 1024 * 65 > MAX_CELLS
    fake = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    assert ark.ark_compute_dt_noalloc(ctypes.byref(p), fake, fake, None) == ark.ARK_ERR_INVALID_ARG
    p32 = ark.params_from_problem(prob, ark.ARK_F32)
    assert ark.ark_compute_dt_noalloc(ctypes.byref(p32), fake, fake, None) == ark.ARK_ERR_INVALID_ARG
    assert ark.ark_compute_dt_noalloc(None, fake, fake, None) == ark.ARK_ERR_INVALID_ARG


@pytest.mark.gpu
def test_noalloc_dt_matches_handle_dt_on_consecutive_calls():
    import torch
    ark = _ark()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [I.rayleigh_benard(3, (40, 36, 24), amp=1e-3),
             I.atmosphere((128, 128)),
             I.random_periodic(2, (300, 7), seed=4, mu=0.5, kappa=0.2),
             I.rayleigh_benard(3, (128, 128, 64), amp=1e-3)]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for prob, U in cases:
        with ark.Solver(prob, "f64", stream=stream) as s:
            s.set_state(U)
            ref = s.compute_dt()
        Ud = torch.from_numpy(np.ascontiguousarray(U)).cuda()
        p = ark.params_from_problem(prob, ark.ARK_F64)
        for _ in range(2):
            out.fill_(-1.0)
            st = ark.ark_compute_dt_noalloc(ctypes.byref(p), ctypes.c_void_p(Ud.data_ptr()),
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
            assert st == ark.ARK_OK
            torch.cuda.synchronize()
            assert out.item() == pytest.approx(ref, rel=F64_TOL)
