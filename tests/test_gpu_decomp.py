"""Slab decomposition along x on the GPU (ARK_BC_HALO, ark_get_halo,
ark_set_halo; Sec. 3.2: regular domain decomposition with ghost zones
refreshed from the neighbours every step).

Every slab is an ordinary handle; the halo layers move between handles
before each step and all slabs take the minimum of their CFL steps.  The
joined slabs equal the undivided grid (FP64: to the last bit of the cell
size, which a slab forms from its own box) and the oracle, and in the FP32
forms stay within their budget.  The decomposition is unmeasured on more
than one GPU: here the slabs share one."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1903_09043_gb300 import inputs as I
from paper_1903_09043_gb300.decomp import DecomposedSolver, SlabDecomposition, advance_local, combine_diagnostics
from parity import F32_STEP_TOL, F64_TOL, field_errors

pytestmark = pytest.mark.gpu


def _ark():
    from paper_1903_09043_gb300 import ark
    return ark


def _walls_in_y():
    """3D layer with reflective walls across y and outflow ends in x (gravity
    along z): the corner ghosts beyond a slab boundary come from the y wall
    rule applied to halo cells."""
    prob, U = I.stratified_random(3, (48, 10, 9), mu=0.01, kappa=0.02, walls=I.REFLECT_HYDRO)
    lo, hi = list(prob.bc_lo), list(prob.bc_hi)
    lo[0] = hi[0] = I.OUTFLOW
    lo[1] = hi[1] = I.REFLECT_HYDRO
    return prob.replace(bc_lo=tuple(lo), bc_hi=tuple(hi)), U


CASES = {
    "2d_rb_three_slabs": (lambda: I.rayleigh_benard(2, (96, 32), amp=1e-2), 3),
    "3d_walls_in_y_outflow_x": (_walls_in_y, 3),
    "2d_shock_tube_outflow_x": (lambda: I.sod(90, axis=0), 3),
    "3d_strat_noslip_visc": (lambda: I.stratified_random(3, (70, 33, 12), mu=0.005, kappa=0.005), 2),
    "3d_periodic_noble_abel": (lambda: (lambda pu: (pu[0].replace(b=0.3), pu[1]))(
        I.random_periodic(3, (48, 9, 11), seed=6, mu=0.02, kappa=0.03)), 3),
}


def _run_slabs(prob, U, parts, precision, nsteps):
    import torch
    ark = _ark()
    dec = SlabDecomposition(prob, parts)
    stream = torch.cuda.current_stream().cuda_stream
    solvers = [ark.Solver(dec.sub_problem(r), precision, stream=stream) for r in range(parts)]
    try:
        for s, V in zip(solvers, dec.split(U)):
            s.set_state(V)
        dt = advance_local(dec, solvers, nsteps)
        out = dec.join([s.get_state() for s in solvers])
        diag = combine_diagnostics([s.diagnostics(check=False) for s in solvers], [dec.cells(r) for r in range(parts)])
    finally:
        for s in solvers:
            s.close()
    return out, dt, diag


def _check_diagnostics(got, want, tol):
    """Whole-grid diagnostics combined from the slabs against the oracle's
    of the undivided grid (momenta relative to the mass scale)."""
    for k, v in want.items():
        scale = max(abs(v), abs(want["mass"]) if k.startswith("mom") else abs(v), 1e-300)
        assert abs(got[k] - v) <= tol * scale, (k, got[k], v)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("precision", ["f64", "f32", "f32split"])
def test_slabs_on_one_gpu_match_undivided_grid_and_oracle(case, precision):
    make, parts = CASES[case]
    prob, U = make()
    n = 12
    V, dt, diag = _run_slabs(prob, U, parts, precision, n)
    assert diag["status"] == 0
    ref, t, dts = O.run(prob, U, n, return_dt=True)
    errs = field_errors(prob, V, ref)
    assert max(errs) <= (F64_TOL if precision == "f64" else n * F32_STEP_TOL), errs
    if precision == "f64":
        ark = _ark()
        import torch
        with ark.Solver(prob, "f64", stream=torch.cuda.current_stream().cuda_stream) as s:
            s.set_state(U)
            s.step(n)
            W = s.get_state()
        assert max(field_errors(prob, V, W)) <= 1e-14
        assert dt == pytest.approx(dts[-1], rel=1e-14)
        _check_diagnostics(diag, O.diagnostics(prob, ref), 1e-12)


def test_halo_calls_reject_a_side_without_halo():
    ark = _ark()
    prob, U = I.sod(40, axis=0)
    with ark.Solver(prob, "f64") as s:
        s.set_state(U)
        lay = s.get_halo(1)                 # any side may be read
        assert lay.shape == (4, 1, 1, 2)
        assert np.array_equal(lay[:, 0, 0, 0], U[:, 0, -1]) and np.array_equal(lay[:, 0, 0, 1], U[:, 0, -2])
        with pytest.raises(ark.ArkError) as ei:
            s.set_halo(0, lay)              # an outflow side takes no halo
        assert ei.value.status == ark.ARK_ERR_INVALID_ARG


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nsteps, q):
    import torch
    import torch.distributed as dist
    from paper_1903_09043_gb300 import ark
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob, U = I.rayleigh_benard(2, (96, 32), amp=1e-2)
        dec = SlabDecomposition(prob, world)
        with ark.Solver(dec.sub_problem(rank), "f64") as s:
            s.set_state(dec.split(U)[rank])
            ds = DecomposedSolver(dec, rank, s)
            dt = ds.step(nsteps)
            q.put((rank, s.get_state(), dt, ds.global_diagnostics()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharing_the_gpu():
    """One process per slab, halos and the time step exchanged over gloo (host
    buffers); the kernels of the two processes never wait on each other."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, 10, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (V, dt, dg)) for r, V, dt, dg in (q.get(timeout=300) for _ in range(2)))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    prob, U = I.rayleigh_benard(2, (96, 32), amp=1e-2)
    dec = SlabDecomposition(prob, 2)
    ref, t, dts = O.run(prob, U, 10, return_dt=True)
    assert max(field_errors(prob, dec.join([got[0][0], got[1][0]]), ref)) <= F64_TOL
    assert got[0][1] == pytest.approx(dts[-1], rel=1e-14) and got[1][1] == got[0][1]
    for r in range(2):
        _check_diagnostics(got[r][2], O.diagnostics(prob, ref), 1e-12)
