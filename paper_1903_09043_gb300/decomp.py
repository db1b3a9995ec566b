"""Slab decomposition of one grid along x (Sec. 3.2, Implementation).

The paper runs one process per subdomain of a regular domain decomposition;
each subdomain keeps ghost zones per direction and side, refreshed from its
neighbours every step.  Here a subdomain is an ordinary solver handle whose
inner x sides are ``ARK_BC_HALO`` (include/ark.h): its two ghost layers on
such a side are the neighbour's two boundary layers, moved by the caller
with ``ark_get_halo`` / ``ark_set_halo`` before every step.  All subdomains
then advance with the same time step, the minimum of their CFL steps, which
is the CFL step of the whole grid.  With FP64 state the decomposed run equals
the undivided one.

This module splits a problem and its state into slabs and drives the
exchange:

* :func:`advance_local` -- several subdomains in one process (one GPU), halos
  moved device to device;
* :class:`DecomposedSolver` -- one subdomain per rank of a
  ``torch.distributed`` process group: every step each rank sends the layers
  at its x sides to the neighbours on those sides, takes theirs as its ghost
  layers, and joins an allreduce-min of the time step.  Halos travel as host
  arrays (gloo) or device tensors (nccl).  Whole-grid diagnostics are the
  slabs' own, combined by allreduce (sums, maxima, minima);
* :func:`combine_diagnostics` -- the same combination for slabs in one process.

Only uniform gravity along the last axis is decomposed (the slab boundary is
then free of potential jumps), as the library requires for ``ARK_BC_HALO``.
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import numpy as np

from .inputs import PERIODIC

HALO = 4   # ARK_BC_HALO: the x side borders a neighbouring slab

# diagnostics that add up over slabs (integrals over the cells); the mean |v|
# of the last axis adds up once weighted by the slab's cells
SUMMED = ("mass", "mom_x", "mom_y", "mom_z", "energy", "kinetic")
STATUS_BITS = (1, 2, 4)   # nonphysical rho/p, L~ <= 0, NaN


def slab_bounds(nx: int, parts: int) -> List[Tuple[int, int]]:
    """Cell ranges [i0, i1) of ``parts`` slabs of ``nx`` cells, sizes differing by at most one."""
    if parts < 1 or nx < 2 * parts:
        raise ValueError("each slab needs at least two cells along x")
    base, extra = divmod(nx, parts)
    out, i0 = [], 0
    for r in range(parts):
        i1 = i0 + base + (1 if r < extra else 0)
        out.append((i0, i1))
        i0 = i1
    return out


class SlabDecomposition:
    """A problem split along x into ``parts`` slabs, slab r owned by rank r."""

    def __init__(self, prob, parts: int):
        if getattr(prob, "phi", None) is not None:
            raise ValueError("slab decomposition takes uniform gravity only")
        self.prob = prob
        self.parts = int(parts)
        self.bounds = slab_bounds(prob.n[0], self.parts)
        self.periodic = prob.bc_lo[0] == PERIODIC

    def neighbours(self, r: int) -> Tuple[Optional[int], Optional[int]]:
        """Ranks owning the slabs beyond the low and high x sides of slab r (None: a physical side)."""
        if self.parts == 1:
            return None, None
        left = r - 1 if r > 0 else (self.parts - 1 if self.periodic else None)
        right = r + 1 if r < self.parts - 1 else (0 if self.periodic else None)
        return left, right

    def sub_problem(self, r: int):
        """The problem of slab r: its cells, box and x boundary rules (ARK_BC_HALO toward neighbours)."""
        p = self.prob
        i0, i1 = self.bounds[r]
        dx = (p.hi[0] - p.lo[0]) / p.n[0]
        left, right = self.neighbours(r)
        bc_lo, bc_hi = list(p.bc_lo), list(p.bc_hi)
        if left is not None:
            bc_lo[0] = HALO
        if right is not None:
            bc_hi[0] = HALO
        n = (i1 - i0,) + tuple(p.n[1:])
        lo = (p.lo[0] + i0 * dx,) + tuple(p.lo[1:])
        hi = (p.lo[0] + i1 * dx,) + tuple(p.hi[1:])
        return p.replace(n=n, lo=lo, hi=hi, bc_lo=tuple(bc_lo), bc_hi=tuple(bc_hi))

    def split(self, U: np.ndarray) -> List[np.ndarray]:
        """Slab states of a whole state (x is the last array axis)."""
        return [np.ascontiguousarray(U[..., i0:i1]) for i0, i1 in self.bounds]

    def join(self, parts: Sequence[np.ndarray]) -> np.ndarray:
        return np.concatenate(list(parts), axis=-1)

    def cells(self, r: int) -> int:
        """Cells of slab r."""
        i0, i1 = self.bounds[r]
        return (i1 - i0) * int(np.prod(self.prob.n[1:]))


def combine_diagnostics(parts: Sequence[dict], cells: Sequence[int]) -> dict:
    """Whole-grid diagnostics from the slabs' own (``parts[r]`` of a slab of
    ``cells[r]`` cells, keys as ``Solver.diagnostics``): integrals summed, the
    mean |v| weighted by cells, the largest speed, the smallest rho and p,
    status bits or-ed; time, step and dt are the first slab's (all slabs
    advance together)."""
    out = dict(parts[0])
    for k in SUMMED:
        out[k] = sum(d[k] for d in parts)
    out["mean_abs_v_last"] = sum(d["mean_abs_v_last"] * n for d, n in zip(parts, cells)) / sum(cells)
    out["max_speed"] = max(d["max_speed"] for d in parts)
    out["min_rho"] = min(d["min_rho"] for d in parts)
    out["min_p"] = min(d["min_p"] for d in parts)
    status = 0
    for d in parts:
        status |= int(d.get("status", 0))
    out["status"] = status
    return out


def advance_local(decomp: SlabDecomposition, solvers: Sequence, nsteps: int) -> float:
    """Advance every subdomain of ``decomp`` (solver r on slab r, all in this
    process) by ``nsteps`` steps: halos moved device to device, the time step
    the minimum of the subdomains' CFL steps.  Returns the last time step.
    The solvers must share one CUDA stream (the halo buffers are written by
    one handle's kernels and read by another's, in stream order)."""
    import torch
    dt = 0.0
    out = [(torch.empty(s.halo_shape(), dtype=torch.float64, device="cuda"),
            torch.empty(s.halo_shape(), dtype=torch.float64, device="cuda")) for s in solvers]
    for _ in range(nsteps):
        for r, s in enumerate(solvers):
            s.get_halo(0, out[r][0])
            s.get_halo(1, out[r][1])
        for r, s in enumerate(solvers):
            left, right = decomp.neighbours(r)
            if left is not None:
                s.set_halo(0, out[left][1])    # the left slab's layers at its high side
            if right is not None:
                s.set_halo(1, out[right][0])   # the right slab's layers at its low side
        dt = min(s.compute_dt() for s in solvers)
        for s in solvers:
            s.step(1, dt)
    return dt


class DecomposedSolver:
    """Rank ``rank``'s slab of ``decomp``, advanced together with the other
    ranks of a ``torch.distributed`` process group.

    ``solver`` is the slab's solver (an :class:`~paper_1903_09043_gb300.ark.Solver`
    on ``decomp.sub_problem(rank)``, or any object with ``get_halo``,
    ``set_halo``, ``halo_shape``, ``compute_dt`` and ``step``).  With the
    gloo backend halos travel as host arrays, with nccl as device tensors.
    Device halos are written and read on the solver's stream, while NCCL
    orders its work after torch's current stream, so in device mode the
    solver's stream is synchronised before a send and the current stream
    after the receives."""

    TAG_FROM_LOW, TAG_FROM_HIGH = 0, 1   # which side of the sender the layers come from

    def __init__(self, decomp: SlabDecomposition, rank: int, solver, group=None, device: str = "cpu"):
        self.decomp = decomp
        self.rank = rank
        self.solver = solver
        self.group = group
        self.device = device
        self.left, self.right = decomp.neighbours(rank)

    def _buffer(self):
        import torch
        return torch.empty(self.solver.halo_shape(), dtype=torch.float64, device=self.device)

    def _fill(self, side: int):
        import torch
        if self.device == "cpu":
            return torch.from_numpy(self.solver.get_halo(side))
        buf = self._buffer()
        self.solver.get_halo(side, buf)
        sync = getattr(self.solver, "sync", None)
        if sync is not None:
            sync()          # the layers are in buf before the collective reads it
        return buf

    def exchange(self) -> None:
        """Send the layers at each x side to the neighbour beyond it and take
        the neighbours' layers as this slab's ghost layers."""
        import torch.distributed as dist
        sends, recvs = [], []
        if self.left is not None:
            sends.append(dist.isend(self._fill(0), self.left, group=self.group, tag=self.TAG_FROM_LOW))
        if self.right is not None:
            sends.append(dist.isend(self._fill(1), self.right, group=self.group, tag=self.TAG_FROM_HIGH))
        got_lo = got_hi = None
        if self.left is not None:       # the left neighbour's layers at its high side
            got_lo = self._buffer()
            recvs.append(dist.irecv(got_lo, self.left, group=self.group, tag=self.TAG_FROM_HIGH))
        if self.right is not None:      # the right neighbour's layers at its low side
            got_hi = self._buffer()
            recvs.append(dist.irecv(got_hi, self.right, group=self.group, tag=self.TAG_FROM_LOW))
        for w in recvs + sends:
            w.wait()
        if self.device != "cpu" and recvs:
            import torch
            torch.cuda.current_stream().synchronize()   # received layers complete before the solver's stream reads them
        if got_lo is not None:
            self.solver.set_halo(0, got_lo.numpy() if self.device == "cpu" else got_lo)
        if got_hi is not None:
            self.solver.set_halo(1, got_hi.numpy() if self.device == "cpu" else got_hi)

    def global_diagnostics(self) -> dict:
        """Diagnostics of the whole grid, the same on every rank (one allreduce
        each for the sums, the maxima and the minima)."""
        import torch
        import torch.distributed as dist
        d = dict(self.solver.diagnostics(check=False))
        n = self.decomp.cells(self.rank)
        total = sum(self.decomp.cells(r) for r in range(self.decomp.parts))
        st = int(d.get("status", 0))
        sums = torch.tensor([d[k] for k in SUMMED] + [d["mean_abs_v_last"] * n], dtype=torch.float64, device=self.device)
        maxs = torch.tensor([d["max_speed"]] + [1.0 if st & b else 0.0 for b in STATUS_BITS], dtype=torch.float64,
                            device=self.device)
        mins = torch.tensor([d["min_rho"], d["min_p"]], dtype=torch.float64, device=self.device)
        dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=self.group)
        dist.all_reduce(maxs, op=dist.ReduceOp.MAX, group=self.group)
        dist.all_reduce(mins, op=dist.ReduceOp.MIN, group=self.group)
        sums, maxs, mins = sums.tolist(), maxs.tolist(), mins.tolist()
        for i, k in enumerate(SUMMED):
            d[k] = sums[i]
        d["mean_abs_v_last"] = sums[len(SUMMED)] / total
        d["max_speed"] = maxs[0]
        d["status"] = sum(b for b, on in zip(STATUS_BITS, maxs[1:]) if on > 0.5)
        d["min_rho"], d["min_p"] = mins
        return d

    def global_dt(self) -> float:
        """Minimum of the ranks' CFL time steps: the CFL step of the whole grid."""
        import torch
        import torch.distributed as dist
        t = torch.tensor([self.solver.compute_dt()], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MIN, group=self.group)
        return float(t.item())

    def step(self, nsteps: int = 1) -> float:
        dt = 0.0
        for _ in range(nsteps):
            self.exchange()
            dt = self.global_dt()
            self.solver.step(1, dt)
        return dt
