"""Pins of the oracle's diagnostics (mass, momenta, energy, kinetic energy,
max |u|, mean |u_last|, min rho, min p) against closed forms.

The sums are the cell averages times the cell volume over the interior (the
finite-volume totals whose conservation Sec. 2 of the scheme guarantees);
the extrema are over the cells.  Each case has sums a plain formula gives
exactly:

* the isothermal column of Sec. 4.3 built by the discrete balance of Eq. 18:
  with T = 1 and a uniform Phi step h, every cell's pressure (and density) is
  the one below it times r = (1 - h/2) / (1 + h/2), so the totals are
  geometric and arithmetico-geometric series;
* a uniform flow with three distinct velocity components on a box of
  non-unit volume, under gravity (rho Phi in the energy sums to rho0 (-g)
  z_mid V because the cell centres average to the box midpoint);
* a checkerboard vertical velocity (its momentum cancels, its mean |v| does
  not);
* the Appendix B energy variable (no rho Phi) and a linear caller potential;
* a stiffened-gas column under tension (min p below zero).

A dropped cell-volume factor, a swapped momentum component, a missing or
doubled rho Phi term, or a pressure formed without p_inf fails one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1903_09043_gb300 import inputs as I

REL = 1e-12


def _close(a, b, scale=None, rel=REL):
    s = abs(b) if scale is None else scale
    assert abs(a - b) <= rel * max(s, 1e-300), (a, b)


def _column_sums(n, h, q0, y0, p_inf=0.0, gamma=5.0 / 3.0):
    """Sum over the column of rho and of rho*calE, for q_j = q0 r^j (q = p + p_inf,
    rho = q / T with T = 1) and Phi_j = y0 + j h."""
    r = (1.0 - 0.5 * h) / (1.0 + 0.5 * h)
    S0 = (1.0 - r ** n) / (1.0 - r)
    S1 = r * (1.0 - n * r ** (n - 1) + (n - 1) * r ** n) / (1.0 - r) ** 2
    mass = q0 * S0
    # rho e = (p + gamma p_inf) / (gamma - 1) = q / (gamma - 1) + p_inf
    energy = q0 * ((1.0 / (gamma - 1.0) + y0) * S0 + h * S1) + n * p_inf
    return mass, energy, q0 * r ** (n - 1) - p_inf


@pytest.mark.parametrize("p_inf", [0.0, 2.5])
def test_isothermal_column_totals(p_inf):
    nx, ny, width, height = 7, 33, 2.5, 3.0
    prob, U = I.atmosphere((nx, ny), height=height, width=width, p_inf=p_inf)
    h = height / ny
    y0 = 0.5 * h
    col_mass, col_energy, pmin = _column_sums(ny, h, math.exp(-y0) + p_inf, y0, p_inf)
    d = O.diagnostics(prob, U)
    _close(d["mass"], width * h * col_mass)
    _close(d["energy"], width * h * col_energy)
    for k in ("mom_x", "mom_y", "mom_z", "kinetic", "max_speed", "mean_abs_v_last"):
        assert d[k] == 0.0, k
    _close(d["min_rho"], (math.exp(-y0) + p_inf) * ((1 - 0.5 * h) / (1 + 0.5 * h)) ** (ny - 1))
    _close(d["min_p"], pmin, scale=max(abs(pmin), 1.0))


def _uniform_3d(energy_form=0, g=-0.7):
    prob = I.Problem(dim=3, n=(5, 4, 3), lo=(0.0, -1.0, 0.5), hi=(2.0, 0.5, 3.5), gamma=1.4, g=g,
                     bc_lo=(I.PERIODIC, I.PERIODIC, I.REFLECT_HYDRO), bc_hi=(I.PERIODIC, I.PERIODIC, I.REFLECT_HYDRO),
                     energy_form=energy_form)
    rho0, p0, u = 1.3, 2.1, (0.7, -0.2, 0.45)
    z = prob.centers(2).reshape(-1, 1, 1)
    U = np.empty((5,) + prob.shape)
    U[0] = rho0
    for d in range(3):
        U[1 + d] = rho0 * u[d]
    ke = 0.5 * rho0 * sum(v * v for v in u)
    U[4] = p0 / (prob.gamma - 1.0) + ke + (rho0 * (-g) * z if energy_form == 0 else 0.0)
    return prob, U, rho0, p0, u, ke


@pytest.mark.parametrize("energy_form", [0, 1])
def test_uniform_flow_totals_under_gravity(energy_form):
    prob, U, rho0, p0, u, ke = _uniform_3d(energy_form)
    V = 2.0 * 1.5 * 3.0
    z_mid = 0.5 * (0.5 + 3.5)
    d = O.diagnostics(prob, U)
    _close(d["mass"], rho0 * V)
    for k, name in enumerate(("mom_x", "mom_y", "mom_z")):
        _close(d[name], rho0 * u[k] * V)
    _close(d["kinetic"], ke * V)
    grav = rho0 * 0.7 * z_mid if energy_form == 0 else 0.0
    _close(d["energy"], (p0 / 0.4 + ke + grav) * V)
    _close(d["max_speed"], math.sqrt(sum(v * v for v in u)))
    _close(d["mean_abs_v_last"], abs(u[2]))
    _close(d["min_rho"], rho0)
    _close(d["min_p"], p0)


def test_checkerboard_vertical_velocity():
    prob = I.Problem(dim=2, n=(6, 5, 1), lo=(0.0, 0.0, 0.0), hi=(3.0, 0.5, 1.0), gamma=5.0 / 3.0)
    rho0, p0, u0, v0 = 0.8, 1.7, 0.3, 0.55
    sign = np.where(np.arange(6) % 2 == 0, 1.0, -1.0).reshape(1, -1)
    U = np.empty((4,) + prob.shape)
    U[0] = rho0
    U[1] = rho0 * u0
    U[2] = rho0 * v0 * sign
    ke = 0.5 * rho0 * (u0 * u0 + v0 * v0)
    U[3] = p0 / (prob.gamma - 1.0) + ke
    V = 1.5
    d = O.diagnostics(prob, U)
    _close(d["mass"], rho0 * V)
    _close(d["mom_x"], rho0 * u0 * V)
    assert abs(d["mom_y"]) <= 1e-15
    _close(d["kinetic"], ke * V)
    _close(d["energy"], (p0 / (prob.gamma - 1.0) + ke) * V)
    _close(d["mean_abs_v_last"], v0)
    _close(d["max_speed"], math.hypot(u0, v0))
    _close(d["min_p"], p0)


def test_linear_potential_array_energy():
    prob = I.Problem(dim=2, n=(8, 6, 1), lo=(-1.0, 0.0, 0.0), hi=(1.0, 3.0, 1.0), gamma=1.4)
    a, b, c = 0.25, -0.6, 1.1
    x = prob.centers(0).reshape(1, -1)
    y = prob.centers(1).reshape(-1, 1)
    phi = a + b * x + c * y + 0.0 * x * y
    prob = prob.replace(phi=phi)
    rho0, p0, u0, v0 = 1.1, 0.9, -0.35, 0.2
    U = np.empty((4,) + prob.shape)
    U[0] = rho0
    U[1] = rho0 * u0
    U[2] = rho0 * v0
    ke = 0.5 * rho0 * (u0 * u0 + v0 * v0)
    U[3] = p0 / 0.4 + ke + rho0 * phi
    V = 6.0
    d = O.diagnostics(prob, U)
    _close(d["energy"], (p0 / 0.4 + ke + rho0 * (a + b * 0.0 + c * 1.5)) * V)
    _close(d["min_p"], p0)
    _close(d["mom_x"], rho0 * u0 * V)
    _close(d["mom_y"], rho0 * v0 * V)
