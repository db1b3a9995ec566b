"""Seeded synthetic inputs: problem descriptions and FP64 initial states.

This module holds no step arithmetic.  It builds the initial data of the
paper's test problems (Sec. 4) and of the benchmark workloads, as plain
numpy arrays, plus the :class:`Problem` record that both the CUDA library
binding and the CPU oracle translate into their own parameter structs.

State layout everywhere: ``U[f, z, y, x]`` (``U[f, y, x]`` in 2D) with the
fields ``rho, m_x, m_y[, m_z], rho*calE`` where ``rho*calE = rho e + rho
|u|^2/2 + rho Phi`` (Sec. 1, Eq. 6 conservation_of_energy) and ``Phi = -g
x_last`` (uniform gravity along the last axis).

Hydrostatic initial profiles use the discrete balance of Eq. 18
(well_balanced_formula) as the paper prescribes for its atmosphere and
Rayleigh-Benard set-ups (Sec. 4.3 and Sec. 4.5): starting from the exact
profile in the bottom cell, ``p_{j+1} = (p_j - rho_j dPhi/2) / (1 + dPhi /
(2 T_{j+1}))`` with ``rho = p / T``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

PERIODIC = 0
REFLECT_HYDRO = 1
NOSLIP_FIXED_T = 2
OUTFLOW = 3

RA_CRITICAL_RIGID = 1707.76   # rigid-rigid Boussinesq onset (textbook linear stability)


@dataclasses.dataclass
class Problem:
    dim: int
    n: Tuple[int, int, int]
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    gamma: float = 5.0 / 3.0
    g: float = 0.0                 # gravity along the last axis (Phi = -g * x_last)
    mu: float = 0.0
    kappa: float = 0.0
    K: float = 1.1
    cfl: float = 0.8
    low_mach: int = 1
    bc_lo: Tuple[int, int, int] = (PERIODIC, PERIODIC, PERIODIC)
    bc_hi: Tuple[int, int, int] = (PERIODIC, PERIODIC, PERIODIC)
    T_lo: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    T_hi: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    energy_form: int = 0           # 0: rho*calE with rho*Phi (Sec. 2); 1: rho E, gravity as a source (Appendix B)
    # caller-supplied potential at the cell centres (shape of one field); None: Phi = -g * x_last
    phi: np.ndarray | None = dataclasses.field(default=None, compare=False, repr=False)
    # stiffened-gas constant: p = (gamma - 1) rho e - gamma p_inf, T = (p + p_inf) / rho; 0: ideal gas
    p_inf: float = 0.0
    # covolume of the Noble-Abel stiffened gas: p = (gamma - 1) rho e / (1 - b rho) - gamma p_inf,
    # T = (p + p_inf)(1 - b rho) / rho; 0: the stiffened gas
    b: float = 0.0

    @property
    def nfields(self) -> int:
        return self.dim + 2

    @property
    def shape(self) -> Tuple[int, ...]:
        """Array shape of one field, slowest axis first."""
        if self.dim == 2:
            return (self.n[1], self.n[0])
        return (self.n[2], self.n[1], self.n[0])

    @property
    def ncells(self) -> int:
        return int(np.prod(self.shape))

    @property
    def dx(self) -> Tuple[float, float, float]:
        return tuple((self.hi[d] - self.lo[d]) / self.n[d] if d < self.dim else 1.0
                     for d in range(3))

    def centers(self, d: int) -> np.ndarray:
        return self.lo[d] + (np.arange(self.n[d]) + 0.5) * self.dx[d]

    def potential(self) -> np.ndarray:
        """Phi at every cell centre (shape of one field)."""
        if self.phi is not None:
            return np.asarray(self.phi, dtype=np.float64)
        v = -self.g * self.centers(self.dim - 1)
        return np.broadcast_to(v.reshape((-1,) + (1,) * (self.dim - 1)), self.shape)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


# ---------------------------------------------------------------------------
# helpers (no step arithmetic: EOS closure of the initial data only)
# ---------------------------------------------------------------------------
def _assemble(prob: Problem, rho: np.ndarray, vel: Sequence[np.ndarray], p: np.ndarray) -> np.ndarray:
    """Conserved state from (rho, u, p) with rho*calE including rho*Phi."""
    shape = prob.shape
    rho = np.broadcast_to(rho, shape).astype(np.float64)
    p = np.broadcast_to(p, shape).astype(np.float64)
    vel = [np.broadcast_to(v, shape).astype(np.float64) for v in vel]
    phi = prob.potential()
    U = np.empty((prob.nfields,) + shape, dtype=np.float64)
    U[0] = rho
    ke = np.zeros(shape)
    for d in range(prob.dim):
        U[1 + d] = rho * vel[d]
        ke += 0.5 * rho * vel[d] * vel[d]
    rho_e = (p + prob.gamma * prob.p_inf) * (1.0 - prob.b * rho) / (prob.gamma - 1.0)
    U[prob.dim + 1] = rho_e + ke + (rho * phi if prob.energy_form == 0 else 0.0)
    return U


def _last_axis_centers(prob: Problem) -> np.ndarray:
    x = prob.centers(prob.dim - 1)
    return x.reshape((-1,) + (1,) * (prob.dim - 1))


def hydrostatic_profile(phi: np.ndarray, T: np.ndarray, p0: float,
                        p_inf: float = 0.0, b: float = 0.0) -> Tuple[np.ndarray, np.ndarray]:
    """Discrete hydrostatic column (Eq. 18) from the bottom cell upward, with
    rho = (p + p_inf) / T (p_inf = 0: the ideal gas), or with a covolume b,
    rho = (p + p_inf) / (T + b (p + p_inf)); then each step solves the
    quadratic b q^2 + (T - b K + dPhi / 2) q - K T = 0 for q = p + p_inf,
    K = q_below - rho_below dPhi / 2 (its positive root)."""
    n = len(phi)
    q = np.empty(n)    # p + p_inf
    rho = np.empty(n)
    q[0] = p0 + p_inf
    rho[0] = q[0] / (T[0] + b * q[0])
    for j in range(n - 1):
        dphi = phi[j + 1] - phi[j]
        if b == 0.0:
            q[j + 1] = (q[j] - 0.5 * rho[j] * dphi) / (1.0 + dphi / (2.0 * T[j + 1]))
        else:
            K = q[j] - 0.5 * rho[j] * dphi
            B = T[j + 1] - b * K + 0.5 * dphi
            q[j + 1] = 2.0 * K * T[j + 1] / (B + math.sqrt(B * B + 4.0 * b * K * T[j + 1]))
        rho[j + 1] = q[j + 1] / (T[j + 1] + b * q[j + 1])
    return rho, q - p_inf


def to_energy_form(prob: Problem, U: np.ndarray, form: int) -> Tuple[Problem, np.ndarray]:
    """The same physical state with the energy variable of ``form`` (adds or
    removes rho*Phi; no step arithmetic)."""
    V = np.array(U, dtype=np.float64, copy=True)
    phi = prob.potential()
    if prob.energy_form == 0 and form == 1:
        V[prob.dim + 1] -= V[0] * phi
    elif prob.energy_form == 1 and form == 0:
        V[prob.dim + 1] += V[0] * phi
    return prob.replace(energy_form=form), V


def _bcast_profile(prob: Problem, prof: np.ndarray) -> np.ndarray:
    return np.broadcast_to(prof.reshape((-1,) + (1,) * (prob.dim - 1)), prob.shape)


# ---------------------------------------------------------------------------
# test problems of the paper (Sec. 4) and the workloads built on them
# ---------------------------------------------------------------------------
def atmosphere(n: Sequence[int] = (128, 128), height: float = 1.0, width: float = 1.0,
               low_mach: int = 1, gamma: float = 5.0 / 3.0, cfl: float = 0.8,
               p_inf: float = 0.0, b: float = 0.0) -> Tuple[Problem, np.ndarray]:
    """Isothermal atmosphere at rest, p = rho = exp(-y), T = 1, g = -1 (Sec. 4.3).

    2D, periodic in x, reflective hydrostatic walls in y.  With ``p_inf`` > 0
    the fluid is a stiffened gas (a liquid-like column, rho = (p + p_inf) / T)
    built by the same discrete balance from p = exp(-y) in the bottom cell."""
    prob = Problem(dim=2, n=(n[0], n[1], 1), lo=(0.0, 0.0, 0.0), hi=(width, height, 1.0),
                   gamma=gamma, g=-1.0, low_mach=low_mach, cfl=cfl, p_inf=p_inf, b=b,
                   bc_lo=(PERIODIC, REFLECT_HYDRO, PERIODIC), bc_hi=(PERIODIC, REFLECT_HYDRO, PERIODIC))
    y = prob.centers(1)
    phi = -prob.g * y
    rho, p = hydrostatic_profile(phi, np.ones_like(y), math.exp(-y[0]), p_inf, b)
    zero = np.zeros(prob.shape)
    return prob, _assemble(prob, _bcast_profile(prob, rho), [zero, zero], _bcast_profile(prob, p))


def polytrope_base(chi: float, m: float):
    """Polytropic layer T = z, rho = z^m, p = z^(m+1) with z = z0 + 1 - y (y up, height 1)."""
    z0 = 1.0 / (chi ** (1.0 / m) - 1.0)
    return z0


def rb_viscosity(chi: float, m: float, gamma: float, Ra: float, Pr: float) -> Tuple[float, float]:
    """(mu, kappa) from the Rayleigh number evaluated at mid-depth.

    Ra = g (beta - g/c_p) rho_mid^2 Pr / (T_mid mu^2), beta = |dT/dy| = 1,
    g = m + 1, c_p = gamma / (gamma - 1), kappa = mu c_p / Pr."""
    z0 = polytrope_base(chi, m)
    zmid = z0 + 0.5
    rho_mid = zmid ** m
    T_mid = zmid
    g = m + 1.0
    cp = gamma / (gamma - 1.0)
    mu = rho_mid * math.sqrt(g * (1.0 - g / cp) * Pr / (T_mid * Ra))
    return mu, mu * cp / Pr


def rayleigh_benard(dim: int = 2, n: Sequence[int] = (256, 128), chi: float = 1.1, m: float = 1.3,
                    Ra: float = 1.1 * RA_CRITICAL_RIGID, Pr: float = 1.0, amp: float = 1e-4, seed: int = 2,
                    gamma: float = 5.0 / 3.0, low_mach: int = 1, cfl: float = 0.8,
                    rng: np.random.Generator | None = None, roll: bool = False) -> Tuple[Problem, np.ndarray]:
    """Rayleigh-Benard layer on a polytrope (Sec. 4.5): box 2 x 1 (2D) or 2 x 2 x 1 (3D),
    periodic horizontally, no-slip fixed-temperature walls at bottom and top.

    Velocity perturbation: every component uniform in (-amp, amp), drawn from
    ``numpy.random.default_rng(seed)`` (or ``rng``) over the cells in C order;
    with ``roll`` (2D), instead the single convection roll pair that fits the
    box, stream function amp sin(pi x) sin(pi y) / pi: u = amp sin(pi x) cos(pi y),
    v = -amp cos(pi x) sin(pi y)."""
    z0 = polytrope_base(chi, m)
    mu, kappa = rb_viscosity(chi, m, gamma, Ra, Pr)
    g = -(m + 1.0)
    if dim == 2:
        nn = (n[0], n[1], 1)
        hi = (2.0, 1.0, 1.0)
        bc_lo = (PERIODIC, NOSLIP_FIXED_T, PERIODIC)
        bc_hi = (PERIODIC, NOSLIP_FIXED_T, PERIODIC)
        T_lo = (0.0, z0 + 1.0, 0.0)
        T_hi = (0.0, z0, 0.0)
    else:
        nn = (n[0], n[1], n[2])
        hi = (2.0, 2.0, 1.0)
        bc_lo = (PERIODIC, PERIODIC, NOSLIP_FIXED_T)
        bc_hi = (PERIODIC, PERIODIC, NOSLIP_FIXED_T)
        T_lo = (0.0, 0.0, z0 + 1.0)
        T_hi = (0.0, 0.0, z0)
    prob = Problem(dim=dim, n=nn, lo=(0.0, 0.0, 0.0), hi=hi, gamma=gamma, g=g, mu=mu, kappa=kappa,
                   low_mach=low_mach, cfl=cfl, bc_lo=bc_lo, bc_hi=bc_hi, T_lo=T_lo, T_hi=T_hi)
    y = prob.centers(dim - 1)
    T = z0 + 1.0 - y
    phi = -g * y
    rho, p = hydrostatic_profile(phi, T, T[0] ** (m + 1.0))
    if roll:
        if dim != 2:
            raise ValueError("roll perturbation is 2D")
        xc = prob.centers(0)[None, :]
        yc = y[:, None]
        vel = [amp * np.sin(np.pi * xc) * np.cos(np.pi * yc), -amp * np.cos(np.pi * xc) * np.sin(np.pi * yc)]
    else:
        if rng is None:
            rng = np.random.default_rng(seed)
        vel = [rng.uniform(-amp, amp, size=prob.shape) for _ in range(dim)] if amp > 0 else \
            [np.zeros(prob.shape) for _ in range(dim)]
    return prob, _assemble(prob, _bcast_profile(prob, rho), vel, _bcast_profile(prob, p))


def gresho(n: int = 1024, mach: float = 1e-2, gamma: float = 5.0 / 3.0, low_mach: int = 1,
           cfl: float = 0.8) -> Tuple[Problem, np.ndarray]:
    """Gresho vortex (Sec. 4.2) on the periodic unit square, centre (0.5, 0.5),
    rho0 = 1, p0 = 1 / (gamma Ma^2)."""
    prob = Problem(dim=2, n=(n, n, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), gamma=gamma,
                   low_mach=low_mach, cfl=cfl)
    x = prob.centers(0)[None, :]
    y = prob.centers(1)[:, None]
    dx, dy = x - 0.5, y - 0.5
    r = np.sqrt(dx * dx + dy * dy)
    p0 = 1.0 / (gamma * mach * mach)
    ut = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    with np.errstate(divide="ignore"):
        p = np.where(r < 0.2, p0 + 12.5 * r * r,
                     np.where(r < 0.4, p0 + 12.5 * r * r + 4.0 - 20.0 * r + 4.0 * np.log(np.maximum(5.0 * r, 1e-300)),
                              p0 - 2.0 + 4.0 * math.log(2.0)))
    with np.errstate(invalid="ignore", divide="ignore"):
        sin_t = np.where(r > 0, dy / np.where(r > 0, r, 1.0), 0.0)
        cos_t = np.where(r > 0, dx / np.where(r > 0, r, 1.0), 0.0)
    u = -ut * sin_t
    v = ut * cos_t
    return prob, _assemble(prob, np.ones(prob.shape), [u, v], p)


def gresho_velocity(prob: Problem) -> Tuple[np.ndarray, np.ndarray]:
    """Exact (stationary) Gresho velocity field at the cell centres."""
    x = prob.centers(0)[None, :]
    y = prob.centers(1)[:, None]
    dx, dy = x - 0.5, y - 0.5
    r = np.sqrt(dx * dx + dy * dy)
    ut = np.where(r < 0.2, 5.0 * r, np.where(r < 0.4, 2.0 - 5.0 * r, 0.0))
    rs = np.where(r > 0, r, 1.0)
    return -ut * dy / rs, ut * dx / rs


def sod(n: int = 100, gamma: float = 1.4, low_mach: int = 1, axis: int = 0,
        cfl: float = 0.8, left: Tuple[float, float] = (1.0, 1.0), right: Tuple[float, float] = (0.125, 0.1),
        p_inf: float = 0.0, b: float = 0.0) -> Tuple[Problem, np.ndarray]:
    """Sod shock tube (Sec. 4.1) on [0, 1] along ``axis`` (0 = x, 1 = y) of a 2D
    grid that is one cell wide and periodic across; zero-gradient ends.
    ``left`` / ``right``: (rho, p) of the two states at rest (Sod's by default);
    ``p_inf`` > 0 makes it a stiffened-gas shock tube, ``b`` > 0 a Noble-Abel one."""
    if axis == 0:
        nn, hi = (n, 1, 1), (1.0, 1.0 / n, 1.0)
        bc_lo, bc_hi = (OUTFLOW, PERIODIC, PERIODIC), (OUTFLOW, PERIODIC, PERIODIC)
    else:
        nn, hi = (1, n, 1), (1.0 / n, 1.0, 1.0)
        bc_lo, bc_hi = (PERIODIC, OUTFLOW, PERIODIC), (PERIODIC, OUTFLOW, PERIODIC)
    prob = Problem(dim=2, n=nn, lo=(0.0, 0.0, 0.0), hi=hi, gamma=gamma, low_mach=low_mach, cfl=cfl,
                   bc_lo=bc_lo, bc_hi=bc_hi, p_inf=p_inf, b=b)
    x = prob.centers(axis)
    is_left = x < 0.5
    rho = np.where(is_left, left[0], right[0])
    p = np.where(is_left, left[1], right[1])
    rho = rho[None, :] if axis == 0 else rho[:, None]
    p = p[None, :] if axis == 0 else p[:, None]
    zero = np.zeros(prob.shape)
    return prob, _assemble(prob, rho, [zero, zero], p)


def well_balanced_column(n: int = 128, low_mach: int = 1, gamma: float = 5.0 / 3.0) -> Tuple[Problem, np.ndarray]:
    """The paper's well-balanced column (Sec. 4.3, Table 1): isothermal, height 3,
    one cell wide and periodic across, reflective hydrostatic walls."""
    prob = Problem(dim=2, n=(1, n, 1), lo=(0.0, 0.0, 0.0), hi=(3.0 / n, 3.0, 1.0), gamma=gamma, g=-1.0,
                   low_mach=low_mach, bc_lo=(PERIODIC, REFLECT_HYDRO, PERIODIC),
                   bc_hi=(PERIODIC, REFLECT_HYDRO, PERIODIC))
    y = prob.centers(1)
    rho, p = hydrostatic_profile(y.copy(), np.ones_like(y), math.exp(-y[0]))
    zero = np.zeros(prob.shape)
    return prob, _assemble(prob, _bcast_profile(prob, rho), [zero, zero], _bcast_profile(prob, p))


def rayleigh_taylor(n: Sequence[int] = (200, 600), C: float = 0.01, g: float = -0.1, p0: float = 2.5,
                    gamma: float = 1.4, low_mach: int = 1, cfl: float = 0.8) -> Tuple[Problem, np.ndarray]:
    """Rayleigh-Taylor instability (Sec. 4.4) on [-0.25, 0.25] x [-0.75, 0.75]:
    rho = 2 above y = 0 and 1 below, at rest in hydrostatic balance
    p = p0 + rho g y (the printed p = rho g y is negative; the pressure offset
    p0 = 2.5 and g = -0.1 make it the standard set-up), vertical velocity
    v = C/4 (1 + cos(2 pi x / Lx)) (1 + cos(2 pi y / Ly)).  Periodic in x,
    reflective hydrostatic walls in y.  With the interface on a face (even
    ny) the state at rest is a discrete equilibrium of the scheme: in each
    fluid p_{j+1} - p_j equals the source S, and across the interface both are
    -(1 + 2)/2 |g| dy."""
    nx, ny = int(n[0]), int(n[1])
    prob = Problem(dim=2, n=(nx, ny, 1), lo=(-0.25, -0.75, 0.0), hi=(0.25, 0.75, 1.0), gamma=gamma, g=g,
                   low_mach=low_mach, cfl=cfl, bc_lo=(PERIODIC, REFLECT_HYDRO, PERIODIC),
                   bc_hi=(PERIODIC, REFLECT_HYDRO, PERIODIC))
    x = prob.centers(0)[None, :]
    y = prob.centers(1)[:, None]
    rho = np.where(y >= 0.0, 2.0, 1.0) * np.ones((1, nx))
    p = p0 + rho * g * y
    Lx, Ly = 0.5, 1.5
    v = 0.25 * C * (1.0 + np.cos(2.0 * np.pi * x / Lx)) * (1.0 + np.cos(2.0 * np.pi * y / Ly))
    return prob, _assemble(prob, rho, [np.zeros((ny, nx)), v], p)


def tilted_atmosphere(n: Sequence[int] = (24, 20), gx: float = -0.3, gy: float = -1.0, T: float = 1.0,
                      low_mach: int = 1, gamma: float = 5.0 / 3.0) -> Tuple[Problem, np.ndarray]:
    """Isothermal atmosphere at rest under gravity (gx, gy) that is not along an
    axis, given as a potential array Phi = -gx x - gy y, in a box with
    reflective hydrostatic walls on all sides.  Built as the discrete
    equilibrium of Eq. 18 along both axes: for T constant the pressure ratio
    across a face depends only on that face's Phi step, so
    p_{i,j} = p_{0,0} r_x^i r_y^j with r = (1 - dPhi / (2T)) / (1 + dPhi / (2T))."""
    nx, ny = int(n[0]), int(n[1])
    prob = Problem(dim=2, n=(nx, ny, 1), lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), gamma=gamma, low_mach=low_mach,
                   bc_lo=(REFLECT_HYDRO, REFLECT_HYDRO, PERIODIC), bc_hi=(REFLECT_HYDRO, REFLECT_HYDRO, PERIODIC))
    x = prob.centers(0)[None, :]
    y = prob.centers(1)[:, None]
    phi = -gx * x - gy * y
    prob = prob.replace(phi=np.ascontiguousarray(phi * np.ones((ny, nx))))
    p = np.empty((ny, nx))
    p[0, 0] = 1.0
    for i in range(1, nx):
        dphi = prob.phi[0, i] - prob.phi[0, i - 1]
        p[0, i] = p[0, i - 1] * (1.0 - dphi / (2.0 * T)) / (1.0 + dphi / (2.0 * T))
    for j in range(1, ny):
        dphi = prob.phi[j, :] - prob.phi[j - 1, :]
        p[j, :] = p[j - 1, :] * (1.0 - dphi / (2.0 * T)) / (1.0 + dphi / (2.0 * T))
    rho = p / T
    return prob, _assemble(prob, rho, [np.zeros((ny, nx)), np.zeros((ny, nx))], p)


def row_potential_state(dim: int = 2, n: Sequence[int] = (20, 16), seed: int = 11, amp: float = 1e-2,
                        mu: float = 0.0, kappa: float = 0.0, low_mach: int = 1, walls: int = NOSLIP_FIXED_T,
                        g0: float = -2.0, curv: float = 1.5, T0: float = 3.0, beta: float = 1.0,
                        gamma: float = 5.0 / 3.0, p_inf: float = 0.0, b: float = 0.0) -> Tuple[Problem, np.ndarray]:
    """Layer under a non-uniform gravity given as a potential array that
    varies along the last axis only, Phi = -g0 y + curv y^2 (the pull weakens
    with height), walls at both ends of that axis, periodic across.  The
    column T = T0 - beta y is the discrete equilibrium of Eq. 18 for that
    potential; density, pressure and velocity carry a random disturbance of
    relative size ``amp`` (0: at rest)."""
    nn = tuple(int(v) for v in n) + (1,) * (3 - len(n))
    last = dim - 1
    bc_lo = [PERIODIC] * 3
    bc_hi = [PERIODIC] * 3
    bc_lo[last] = walls
    bc_hi[last] = walls
    T_lo = [0.0] * 3
    T_hi = [0.0] * 3
    T_lo[last] = T0
    T_hi[last] = T0 - beta
    prob = Problem(dim=dim, n=nn, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), gamma=gamma, mu=mu, kappa=kappa,
                   low_mach=low_mach, bc_lo=tuple(bc_lo), bc_hi=tuple(bc_hi), T_lo=tuple(T_lo), T_hi=tuple(T_hi),
                   p_inf=p_inf, b=b)
    y = prob.centers(last)
    prof = -g0 * y + curv * y * y
    prob = prob.replace(phi=np.ascontiguousarray(_bcast_profile(prob, prof)))
    T = T0 - beta * y
    rho, p = hydrostatic_profile(prof, T, T[0] ** 2, p_inf, b)
    rng = np.random.default_rng(seed)
    rhof = _bcast_profile(prob, rho) * (1.0 + amp * rng.uniform(-1, 1, size=prob.shape))
    pf = _bcast_profile(prob, p) * (1.0 + amp * rng.uniform(-1, 1, size=prob.shape))
    vel = [amp * rng.uniform(-1, 1, size=prob.shape) for _ in range(dim)]
    return prob, _assemble(prob, rhof, vel, pf)


def periodic_potential_state(dim: int = 2, n: Sequence[int] = (24, 20), seed: int = 7, amp: float = 0.05,
                             A: float = 0.3, mu: float = 0.0, kappa: float = 0.0,
                             low_mach: int = 1) -> Tuple[Problem, np.ndarray]:
    """Fully periodic box with the potential Phi = A sin(2 pi x) cos(2 pi y)
    [cos(2 pi z)] given as an array, and a smooth random state (density,
    velocity, pressure perturbed by sinusoids of random phase)."""
    nn = tuple(int(v) for v in n) + (1,) * (3 - len(n))
    prob = Problem(dim=dim, n=nn, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), mu=mu, kappa=kappa, low_mach=low_mach)
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[prob.centers(d) for d in reversed(range(dim))], indexing="ij")[::-1]   # x, y[, z]
    phi = A * np.sin(2 * np.pi * grids[0]) * np.cos(2 * np.pi * grids[1])
    if dim == 3:
        phi = phi * np.cos(2 * np.pi * grids[2])
    prob = prob.replace(phi=np.ascontiguousarray(phi))

    def smooth():
        ph = rng.uniform(0, 2 * np.pi, size=dim)
        return np.prod([np.sin(2 * np.pi * grids[d] + ph[d]) for d in range(dim)], axis=0)

    rho = 1.0 + amp * smooth()
    p = 1.0 + amp * smooth()
    vel = [amp * smooth() for _ in range(dim)]
    return prob, _assemble(prob, rho, vel, p)


def random_periodic(dim: int = 2, n: Sequence[int] = (24, 20), seed: int = 0, amp: float = 0.1,
                    gamma: float = 1.4, mu: float = 0.0, kappa: float = 0.0, low_mach: int = 1,
                    cfl: float = 0.5) -> Tuple[Problem, np.ndarray]:
    """Smooth random state on a fully periodic unit box without gravity."""
    nn = tuple(n) + (1,) * (3 - len(n))
    prob = Problem(dim=dim, n=nn, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), gamma=gamma, mu=mu, kappa=kappa,
                   low_mach=low_mach, cfl=cfl)
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[prob.centers(d) for d in reversed(range(dim))], indexing="ij")
    coords = list(reversed(grids))   # coords[d] has the field shape

    def smooth():
        out = np.zeros(prob.shape)
        for _ in range(3):
            k = rng.integers(1, 3, size=dim)
            ph = rng.uniform(0, 2 * np.pi, size=dim)
            term = np.ones(prob.shape)
            for d in range(dim):
                term = term * np.sin(2 * np.pi * k[d] * coords[d] + ph[d])
            out += rng.uniform(-1, 1) * term
        return out / 3.0

    rho = 1.0 + amp * smooth()
    p = 1.0 + amp * smooth()
    vel = [amp * smooth() for _ in range(dim)]
    return prob, _assemble(prob, rho, vel, p)


def stratified_random(dim: int = 2, n: Sequence[int] = (20, 16), seed: int = 1, amp: float = 1e-2,
                      mu: float = 0.0, kappa: float = 0.0, low_mach: int = 1, walls: int = NOSLIP_FIXED_T,
                      chi: float = 3.0, m: float = 1.0, gamma: float = 5.0 / 3.0,
                      cfl: float = 0.8, p_inf: float = 0.0, b: float = 0.0) -> Tuple[Problem, np.ndarray]:
    """Polytropic layer with gravity along the last axis, walls at both ends of it,
    periodic across, and a random velocity and pressure disturbance.  With
    ``p_inf`` > 0 the fluid is a stiffened gas, rho = (p + p_inf) / T; with a
    covolume ``b`` a Noble-Abel stiffened gas, rho = (p + p_inf) / (T + b (p + p_inf))."""
    z0 = polytrope_base(chi, m)
    g = -(m + 1.0)
    nn = tuple(n) + (1,) * (3 - len(n))
    last = dim - 1
    bc_lo = [PERIODIC] * 3
    bc_hi = [PERIODIC] * 3
    bc_lo[last] = walls
    bc_hi[last] = walls
    T_lo = [0.0] * 3
    T_hi = [0.0] * 3
    T_lo[last] = z0 + 1.0
    T_hi[last] = z0
    hi = [1.0, 1.0, 1.0]
    prob = Problem(dim=dim, n=nn, lo=(0.0, 0.0, 0.0), hi=tuple(hi), gamma=gamma, g=g, mu=mu, kappa=kappa,
                   low_mach=low_mach, cfl=cfl, bc_lo=tuple(bc_lo), bc_hi=tuple(bc_hi), T_lo=tuple(T_lo),
                   T_hi=tuple(T_hi), p_inf=p_inf, b=b)
    y = prob.centers(last)
    T = z0 + 1.0 - y
    rho, p = hydrostatic_profile(-g * y, T, T[0] ** (m + 1.0), p_inf, b)
    rng = np.random.default_rng(seed)
    rhof = _bcast_profile(prob, rho) * (1.0 + amp * rng.uniform(-1, 1, size=prob.shape))
    pf = _bcast_profile(prob, p) * (1.0 + amp * rng.uniform(-1, 1, size=prob.shape))
    vel = [amp * rng.uniform(-1, 1, size=prob.shape) for _ in range(dim)]
    return prob, _assemble(prob, rhof, vel, pf)


def ensemble(count: int = 256, seed: int = 5, amp: float = 1e-4, chi: float = 1.1, m: float = 1.3,
             nmin: int = 64, nmax: int = 512) -> List[Tuple[Problem, np.ndarray]]:
    """Ensemble of independent 2D Rayleigh-Benard runs: nx = 16 round(exp(U(ln 64, ln 512)) / 16),
    ny = nx / 2, Ra = exp(U(ln 1e3, ln 1e6)); one generator ``default_rng(seed)`` draws the sizes,
    Rayleigh numbers and perturbations in run order."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        nx = int(16 * round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) / 16))
        nx = max(nmin, min(nmax, nx))
        ny = nx // 2
        Ra = math.exp(rng.uniform(math.log(1e3), math.log(1e6)))
        out.append(rayleigh_benard(dim=2, n=(nx, ny), chi=chi, m=m, Ra=Ra, amp=amp, rng=rng))
    return out
