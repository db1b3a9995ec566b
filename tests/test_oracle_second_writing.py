"""The C oracle against an independent NumPy writing of the same 2D step
(oracle/numpy_step.py) on grids of at most 16 x 16 cells: every boundary
rule, gravity, dissipation, the low-Mach correction on and off, both energy
variables (Sec. 2 and Appendix B), the stiffened gas and the Noble-Abel
stiffened gas.  Two writings of one
specification, with different mechanisms (recursive per-cell ghosts and
face arrays in C, padded whole-array expressions in NumPy), agree to
rounding."""
import numpy as np
import pytest

import oracle as O
from oracle import numpy_step as NS
from paper_1903_09043_gb300 import inputs as I
from parity import field_errors

TOL = 1e-13

CASES = {
    "periodic_visc": lambda: I.random_periodic(2, (16, 12), seed=2, mu=0.02, kappa=0.03),
    "periodic_theta1": lambda: I.random_periodic(2, (13, 9), seed=3, mu=0.02, kappa=0.03, low_mach=0),
    "atmosphere_reflect": lambda: I.atmosphere((11, 16)),
    "strat_noslip_visc": lambda: I.stratified_random(2, (16, 11), mu=0.01, kappa=0.02),
    "strat_reflect": lambda: I.stratified_random(2, (9, 14), walls=I.REFLECT_HYDRO),
    "strat_reflect_visc": lambda: I.stratified_random(2, (10, 13), walls=I.REFLECT_HYDRO, mu=0.05, kappa=0.04),
    "sod_x_outflow": lambda: I.sod(16, axis=0),
    "sod_y_outflow": lambda: I.sod(16, axis=1),
    "rb_chi21": lambda: I.rayleigh_benard(2, (16, 16), chi=21.0, amp=1e-2),
    "rb": lambda: I.rayleigh_benard(2, (16, 8), amp=1e-2),
    "rayleigh_taylor": lambda: I.rayleigh_taylor((8, 16)),
    "walls_n2": lambda: I.stratified_random(2, (5, 2), mu=0.01, kappa=0.01, chi=1.2),
    "stiffened_column": lambda: I.atmosphere((6, 16), p_inf=2.5),
    "noble_abel_column": lambda: I.atmosphere((6, 16), p_inf=0.5, b=0.3),
    "noble_abel_strat_noslip_visc": lambda: I.stratified_random(2, (16, 11), mu=0.01, kappa=0.02, p_inf=0.2, b=0.2),
    "noble_abel_sod_x": lambda: I.sod(16, axis=0, p_inf=0.3, b=0.4),
    "noble_abel_periodic_visc": lambda: (lambda pu: (pu[0].replace(b=0.3), pu[1]))(
        I.random_periodic(2, (12, 10), seed=4, mu=0.02, kappa=0.03)),
    "noble_abel_sod_y_inflow": lambda: _inflow(I.sod(16, axis=1, p_inf=0.3, b=0.4), -0.3),
}


def _inflow(pu, u):
    """The tube with every cell moving at u along its axis (flow enters through one end)."""
    prob, U = pu
    axis = 0 if prob.n[0] > 1 else 1
    U = np.array(U)
    U[1 + axis] = U[0] * u
    U[3] += 0.5 * U[0] * u * u
    return prob, U


def _cases():
    out = []
    for name in sorted(CASES):
        out.append((name, 0))
        if name in ("strat_noslip_visc", "atmosphere_reflect", "rb"):
            out.append((name, 1))
    return out


@pytest.mark.parametrize("name,form", _cases())
def test_numpy_writing_equals_c_oracle(name, form):
    prob, U = CASES[name]()
    if form == 1:
        prob, U = I.to_energy_form(prob, U, 1)
    assert prob.n[0] <= 16 and prob.n[1] <= 16
    for _ in range(3):
        dt = O.dt(prob, U)
        A = NS.step(prob, U, dt)
        B = O.step(prob, U, dt)
        errs = field_errors(prob, A, B)
        assert max(errs) <= TOL, errs
        U = B


def test_numpy_writing_sees_a_planted_sign_flip():
    """The comparison is sharp enough to see a one-term change: a heat flux
    with the printed (anti-diffusive) sign differs at order dt kappa."""
    prob, U = I.stratified_random(2, (12, 10), mu=0.0, kappa=0.05)
    dt = O.dt(prob, U)
    B = O.step(prob, U, dt)
    A = NS.step(prob.replace(kappa=-prob.kappa), U, dt)
    assert max(field_errors(prob, A, B)) > 1e-8
