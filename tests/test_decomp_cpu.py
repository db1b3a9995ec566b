"""Slab decomposition along x, host side (Sec. 3.2: regular domain
decomposition, ghost zones refreshed from the neighbours every step).

The split, the neighbour map, the halo exchange over gloo ranks and the
allreduce-min time step are checked with a stand-in for each slab's solver:
the oracle stepping the slab extended by the ghost layers it received (the
step's stencil reaches two cells, so the slab's own cells are exact).  The
ranks' slabs, joined, must equal the undivided oracle run to rounding: a
slab's cell size (hi - lo) / n, formed from its own box, may differ from the
whole grid's in the last bit."""
import os
import socket

import numpy as np
import pytest

import oracle as O
from paper_1903_09043_gb300 import inputs as I
from paper_1903_09043_gb300.decomp import HALO, DecomposedSolver, SlabDecomposition, combine_diagnostics, slab_bounds
from parity import field_errors

TOL = 1e-14


class OracleSlab:
    """A slab's solver for the host-side test: the state in FP64 and the
    oracle on the slab plus its ghost layers."""

    def __init__(self, prob, U):
        self.prob = prob
        self.U = np.array(U, dtype=np.float64)
        self.ghost = [None, None]

    def halo_shape(self):
        p = self.prob
        return (p.nfields, p.n[p.dim - 1], p.n[1] if p.dim == 3 else 1, 2)

    def get_halo(self, side, out=None):
        L = self.U[..., 0:2] if side == 0 else self.U[..., ::-1][..., 0:2]   # layer 0 at the side
        return np.ascontiguousarray(L).reshape(self.halo_shape())

    def set_halo(self, side, layers):
        self.ghost[side] = np.asarray(layers).reshape(self.U.shape[:-1] + (2,))

    def _plain(self):
        p = self.prob
        lo = tuple(I.OUTFLOW if b == HALO else b for b in p.bc_lo)
        hi = tuple(I.OUTFLOW if b == HALO else b for b in p.bc_hi)
        return p.replace(bc_lo=lo, bc_hi=hi)

    def compute_dt(self):
        return O.dt(self._plain(), self.U)

    def diagnostics(self, check=False):
        d = O.diagnostics(self._plain(), self.U)
        d.update(t=0.0, step=0, dt=0.0, status=0)
        return d

    def step(self, n, dt):
        p = self._plain()
        for _ in range(n):
            parts, a = [], 0
            if self.prob.bc_lo[0] == HALO:
                parts.append(self.ghost[0][..., ::-1])      # x = -2, -1
                a = 2
            parts.append(self.U)
            if self.prob.bc_hi[0] == HALO:
                parts.append(self.ghost[1])                 # x = nx, nx + 1
            E = np.ascontiguousarray(np.concatenate(parts, axis=-1))
            dx = (p.hi[0] - p.lo[0]) / p.n[0]
            ext = p.replace(n=(E.shape[-1],) + tuple(p.n[1:]), lo=(p.lo[0] - a * dx,) + tuple(p.lo[1:]),
                            hi=(p.lo[0] + (E.shape[-1] - a) * dx,) + tuple(p.hi[1:]))
            self.U = np.ascontiguousarray(O.step(ext, E, dt)[..., a:a + self.U.shape[-1]])


CASES = {
    "2d_periodic_visc": lambda: I.random_periodic(2, (20, 13), seed=2, mu=0.02, kappa=0.03),
    "2d_rb_walls_in_y": lambda: I.rayleigh_benard(2, (24, 12), amp=1e-2),
    "2d_shock_tube_outflow_x": lambda: I.sod(30, axis=0),
    "3d_periodic_visc": lambda: I.random_periodic(3, (12, 7, 5), seed=3, mu=0.02, kappa=0.03),
    "3d_walls_in_y_outflow_x": lambda: _walls_in_y(),
}


def _walls_in_y():
    prob, U = I.stratified_random(3, (12, 6, 5), mu=0.01, kappa=0.02, walls=I.REFLECT_HYDRO)
    lo, hi = list(prob.bc_lo), list(prob.bc_hi)
    lo[0] = hi[0] = I.OUTFLOW
    lo[1] = hi[1] = I.REFLECT_HYDRO
    return prob.replace(bc_lo=tuple(lo), bc_hi=tuple(hi)), U


def test_slab_bounds_and_sub_problems():
    assert slab_bounds(10, 3) == [(0, 4), (4, 7), (7, 10)]
    with pytest.raises(ValueError):
        slab_bounds(5, 3)
    prob, U = I.sod(30, axis=0)
    dec = SlabDecomposition(prob, 3)
    assert [dec.neighbours(r) for r in range(3)] == [(None, 1), (0, 2), (1, None)]
    s0, s2 = dec.sub_problem(0), dec.sub_problem(2)
    assert s0.bc_lo[0] == I.OUTFLOW and s0.bc_hi[0] == HALO
    assert s2.bc_lo[0] == HALO and s2.bc_hi[0] == I.OUTFLOW
    assert s0.dx[0] == pytest.approx(prob.dx[0]) and s2.hi[0] == pytest.approx(prob.hi[0])
    assert np.array_equal(dec.join(dec.split(U)), U)
    per, _ = I.random_periodic(2, (20, 13))
    d2 = SlabDecomposition(per, 2)
    assert d2.neighbours(0) == (1, 1) and d2.neighbours(1) == (0, 0)
    assert d2.sub_problem(0).bc_lo[0] == HALO and d2.sub_problem(1).bc_hi[0] == HALO
    assert SlabDecomposition(per, 1).sub_problem(0).bc_lo[0] == I.PERIODIC


def test_local_stand_in_equals_undivided_oracle():
    """Without ranks: the stand-in slabs with halos moved by hand equal the
    undivided grid (the stand-in itself is right)."""
    prob, U = CASES["2d_rb_walls_in_y"]()
    dec = SlabDecomposition(prob, 3)
    slabs = [OracleSlab(dec.sub_problem(r), V) for r, V in enumerate(dec.split(U))]
    for _ in range(4):
        halos = [(s.get_halo(0), s.get_halo(1)) for s in slabs]
        for r, s in enumerate(slabs):
            left, right = dec.neighbours(r)
            s.set_halo(0, halos[left][1])
            s.set_halo(1, halos[right][0])
        dt = min(s.compute_dt() for s in slabs)
        for s in slabs:
            s.step(1, dt)
    ref, _ = O.run(prob, U, 4)
    assert max(field_errors(prob, dec.join([s.U for s in slabs]), ref)) <= TOL
    _check_diagnostics(combine_diagnostics([s.diagnostics() for s in slabs], [dec.cells(r) for r in range(3)]),
                       O.diagnostics(prob, ref))


def _check_diagnostics(got, want):
    """Whole-grid diagnostics from the slabs against the undivided grid's
    (sums in another order, and each slab's cell size formed from its own box)."""
    for k, v in want.items():
        scale = max(abs(v), abs(want["mass"]) if k.startswith("mom") else abs(v), 1e-300)
        assert abs(got[k] - v) <= 1e-12 * scale, (k, got[k], v)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, case, nsteps, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        prob, U = CASES[case]()
        dec = SlabDecomposition(prob, world)
        slab = OracleSlab(dec.sub_problem(rank), dec.split(U)[rank])
        ds = DecomposedSolver(dec, rank, slab)
        dt = ds.step(nsteps)
        q.put((rank, slab.U, dt, ds.global_diagnostics()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,world", [("2d_periodic_visc", 2), ("2d_rb_walls_in_y", 3),
                                        ("2d_shock_tube_outflow_x", 3), ("3d_periodic_visc", 2),
                                        ("3d_walls_in_y_outflow_x", 3)])
def test_gloo_ranks_equal_undivided_grid(case, world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, case, 5, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict((r, (V, dt, dg)) for r, V, dt, dg in (q.get(timeout=120) for _ in range(world)))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    prob, U = CASES[case]()
    dec = SlabDecomposition(prob, world)
    ref, t, dts = O.run(prob, U, 5, return_dt=True)
    assert max(field_errors(prob, dec.join([got[r][0] for r in range(world)]), ref)) <= TOL
    assert all(got[r][1] == pytest.approx(dts[-1], rel=1e-14) for r in range(world))
    want = O.diagnostics(prob, ref)
    for r in range(world):   # every rank holds the whole grid's diagnostics
        _check_diagnostics(got[r][2], want)


def test_combined_diagnostics_of_uneven_slabs():
    """Five slabs of 5, 5, 5, 5 and 4 columns: the integrals add up, the mean
    |v| is weighted by each slab's cells, extremes are the grid's."""
    prob, U = I.rayleigh_benard(2, (24, 12), amp=1e-2)
    dec = SlabDecomposition(prob, 5)
    assert sorted({dec.cells(r) for r in range(5)}) == [4 * 12, 5 * 12]
    slabs = [OracleSlab(dec.sub_problem(r), V) for r, V in enumerate(dec.split(U))]
    parts = [s.diagnostics() for s in slabs]
    got = combine_diagnostics(parts, [dec.cells(r) for r in range(5)])
    _check_diagnostics(got, O.diagnostics(prob, U))
    unweighted = sum(d["mean_abs_v_last"] for d in parts) / 5
    assert abs(unweighted - got["mean_abs_v_last"]) > 1e-6 * got["mean_abs_v_last"]
    parts[3]["status"] = 4
    assert combine_diagnostics(parts, [dec.cells(r) for r in range(5)])["status"] == 4
