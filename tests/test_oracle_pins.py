"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them:

* printed values: Table 1 of Sec. 4.3 (tests/golden/well_balanced_table1.txt);
* closed forms: uniform-state face values and time step, the linear-acoustics
  Riemann solution (characteristic invariants), shear-wave and entropy-mode
  decay rates, exact Sod solution (Toro Ch. 4);
* invariants: well-balanced rest state, exact conservation of mass, momentum
  and total energy, transverse momentum with gravity, x/y symmetry, bitwise
  preservation of uniform flow;
* special cases that reduce to a textbook routine: first-order upwind advection
  of a density bump at uniform velocity and pressure;
* the paper's qualitative results: Gresho error flat in Mach with the low-Mach
  correction and growing without it (Sec. 4.2), Sod insensitive to it (Sec. 4.1).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1903_09043_gb300 import inputs as I

from riemann_exact import sample as riemann_sample

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

O.set_threads(1)


def _prim(prob, U):
    dim = prob.dim
    rho = U[0]
    vel = [U[1 + d] / rho for d in range(dim)]
    ke = 0.5 * sum(rho * v * v for v in vel)
    phi = -prob.g * prob.centers(dim - 1).reshape((-1,) + (1,) * (dim - 1))
    p = (prob.gamma - 1.0) * (U[dim + 1] - ke - rho * phi)
    return rho, vel, p


# --------------------------------------------------------------------------
# primitives, ghosts, faces
# --------------------------------------------------------------------------
def test_primitives_remove_gravitational_energy():
    """rho*calE includes rho*Phi (Eq. 6): a state at rest built with p and Phi
    must give back p exactly up to rounding, and T = p / rho, c^2 = gamma p / rho."""
    prob, U = I.atmosphere((4, 6))
    for j in range(6):
        c = O.cell_at(prob, U, (1, j))
        y = prob.centers(1)[j]
        assert c["phi"] == pytest.approx(y, rel=0, abs=1e-15)
        p_exact = U[0, j, 1]   # T = 1 so p = rho
        assert c["p"] == pytest.approx(p_exact, rel=1e-14)
        assert c["T"] == pytest.approx(1.0, rel=1e-14)
        assert c["c"] == pytest.approx(math.sqrt(prob.gamma), rel=1e-14)


def test_hydrostatic_wall_ghosts_satisfy_discrete_balance():
    """Wall ghosts extend the discrete equilibrium of Eq. 18 and mirror the
    normal velocity; a fixed-temperature ghost averages to the wall value."""
    prob, U = I.stratified_random(2, (6, 8), walls=I.NOSLIP_FIXED_T, amp=1e-2)
    for i in range(6):
        for (a, b, Tw) in ((0, -1, prob.T_lo[1]), (-1, -2, None), (7, 8, prob.T_hi[1]), (8, 9, None)):
            A = O.cell_at(prob, U, (i, a))
            G = O.cell_at(prob, U, (i, b))
            lhs = G["p"] - A["p"]
            rhs = -0.5 * (A["rho"] + G["rho"]) * (G["phi"] - A["phi"])
            assert lhs == pytest.approx(rhs, rel=1e-12, abs=1e-14)
        # fixed-temperature wall: mean of ghost and mirror T is the wall temperature
        c0, g1 = O.cell_at(prob, U, (i, 0)), O.cell_at(prob, U, (i, -1))
        assert 0.5 * (c0["T"] + g1["T"]) == pytest.approx(prob.T_lo[1], rel=1e-13)
        # no-slip: every component flipped
        assert g1["u"] == pytest.approx(-c0["u"], abs=1e-16)
        assert g1["v"] == pytest.approx(-c0["v"], abs=1e-16)
    prob, U = I.stratified_random(2, (6, 8), walls=I.REFLECT_HYDRO, amp=1e-2)
    c0, g1 = O.cell_at(prob, U, (2, 0)), O.cell_at(prob, U, (2, -1))
    assert g1["v"] == pytest.approx(-c0["v"], abs=1e-16)   # normal flipped
    assert g1["u"] == pytest.approx(c0["u"], abs=1e-16)    # tangential kept
    assert g1["T"] == pytest.approx(c0["T"], rel=1e-14)    # isothermal mirror
    # periodic: wrapped; corner ghosts follow x then y
    c = O.cell_at(prob, U, (-1, 3))
    assert c["rho"] == U[0, 3, 5]
    corner = O.cell_at(prob, U, (-1, -1))
    edge = O.cell_at(prob, U, (5, -1))
    assert corner["rho"] == edge["rho"]


@pytest.mark.parametrize("low_mach", [0, 1])
def test_face_matches_linear_acoustics_riemann_solution(low_mach):
    """With theta = 1 the face state (u*, Pi*) is the linear-acoustics Riemann
    solution with impedance a: the right-going invariant p + a u is carried
    from the left, the left-going p - a u from the right, each shifted by S/2
    for the gravity source (integral consistency).  Solved here as a 2x2 system."""
    prob = I.Problem(dim=2, n=(4, 4, 1), lo=(0, 0, 0), hi=(1, 1, 1), gamma=1.4, low_mach=0, K=1.3)
    rng = np.random.default_rng(7)
    for _ in range(20):
        L = [rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), 0.0, rng.uniform(0.5, 2), rng.uniform(0, 1)]
        R = [rng.uniform(0.5, 2), rng.uniform(-1, 1), rng.uniform(-1, 1), 0.0, rng.uniform(0.5, 2), rng.uniform(0, 1)]
        for d in (0, 1):
            f = O.face(prob, L, R, d)
            cL = math.sqrt(1.4 * L[4] / L[0])
            cR = math.sqrt(1.4 * R[4] / R[0])
            a = 1.3 * max(L[0] * cL, R[0] * cR)
            S = -0.5 * (L[0] + R[0]) * (R[5] - L[5])
            A = np.array([[1.0, a], [1.0, -a]])
            rhs = np.array([L[4] + a * L[1 + d] + 0.5 * S, R[4] - a * R[1 + d] - 0.5 * S])
            Pi, us = np.linalg.solve(A, rhs)
            assert f["a"] == pytest.approx(a, rel=1e-14)
            assert f["S"] == pytest.approx(S, rel=1e-14, abs=1e-15)
            assert f["ustar"] == pytest.approx(us, rel=1e-12, abs=1e-13)
            assert f["Pistar"] == pytest.approx(Pi, rel=1e-12)
    # low-Mach correction (Eq. 16): theta in [0, 1]; it scales only the
    # velocity-jump part of Pi*, so equal velocities give the same Pi*; a
    # supersonic face has theta = 1.
    p2 = prob.replace(low_mach=low_mach)
    f = O.face(p2, [1, 0.3, 0, 0, 1, 0], [0.5, 0.3, 0, 0, 2, 0], 0)
    assert 0.0 <= f["theta"] <= 1.0
    assert f["Pistar"] == pytest.approx(1.5, rel=1e-15)
    fs = O.face(p2, [1, 5.0, 0, 0, 1, 0], [1, 4.0, 0, 0, 1, 0], 0)
    assert fs["theta"] == 1.0
    fsub = O.face(p2, [1, 0.01, 0, 0, 1, 0], [1, -0.01, 0, 0, 1, 0], 0)
    if low_mach:
        assert fsub["theta"] < 0.02
        assert abs(fsub["Pistar"] - 1.0) < 0.02 * abs(O.face(prob, [1, 0.01, 0, 0, 1, 0], [1, -0.01, 0, 0, 1, 0], 0)["Pistar"] - 1.0) + 1e-15
    else:
        assert fsub["theta"] == 1.0


def test_face_sign_high_pressure_pushes_fluid_out():
    prob = I.Problem(dim=2, n=(4, 4, 1), lo=(0, 0, 0), hi=(1, 1, 1), gamma=1.4, low_mach=0)
    f = O.face(prob, [1, 0, 0, 0, 2.0, 0], [1, 0, 0, 0, 1.0, 0], 0)
    assert f["ustar"] > 0
    f = O.face(prob, [1, 0, 0, 0, 1.0, 0], [1, 0, 0, 0, 2.0, 0], 1)
    assert f["ustar"] < 0


# --------------------------------------------------------------------------
# time step
# --------------------------------------------------------------------------
def test_dt_uniform_state_closed_form():
    prob, U = I.random_periodic(2, (8, 6), amp=0.0, gamma=1.4)
    U[1] = 0.5 * U[0]
    U[2] = -0.25 * U[0]
    U[3] += 0.5 * U[0] * (0.25 + 0.0625)
    dx, dy = prob.dx[0], prob.dx[1]
    c = math.sqrt(1.4)
    expect = prob.cfl / ((0.5 + c) / dx + (0.25 + c) / dy)
    assert O.dt(prob, U) == pytest.approx(expect, rel=1e-14)
    # a large viscosity switches to the parabolic bound
    pv = prob.replace(mu=10.0, kappa=0.0)
    expect_p = prob.cfl / (2 * (4 * 10.0 / 3.0) * (1 / dx ** 2 + 1 / dy ** 2))
    assert O.dt(pv, U) == pytest.approx(expect_p, rel=1e-14)
    # ... and a large conductivity to the thermal one, kappa (gamma - 1) / rho (R3),
    # which wins over the viscous one when it is the larger diffusivity
    rho = float(U[0].flat[0])
    assert np.all(U[0] == rho)
    pk = prob.replace(mu=0.0, kappa=20.0)
    expect_k = prob.cfl / (2 * (20.0 * 0.4 / rho) * (1 / dx ** 2 + 1 / dy ** 2))
    assert O.dt(pk, U) == pytest.approx(expect_k, rel=1e-14)
    pb = prob.replace(mu=1.0, kappa=20.0)
    assert O.dt(pb, U) == pytest.approx(expect_k, rel=1e-14)


# --------------------------------------------------------------------------
# invariants of the step
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, (9, 7)), (3, (5, 6, 4))])
def test_uniform_flow_preserved_bitwise(dim, n):
    prob, U = I.random_periodic(dim, n, amp=0.0, mu=0.01, kappa=0.01)
    for d in range(dim):
        U[1 + d] = (0.3 - 0.2 * d) * U[0]
    U[dim + 1] = 1.0 / 0.4 + 0.5 * sum((0.3 - 0.2 * d) ** 2 for d in range(dim))
    V = U.copy()
    for _ in range(5):
        V = O.step(prob, V, O.dt(prob, V))
    assert np.array_equal(V, U)


@pytest.mark.parametrize("low_mach", [0, 1])
def test_hydrostatic_atmosphere_stays_at_rest(low_mach):
    """Config: 2D 128 x 128 isothermal atmosphere, 1000 steps (Sec. 2.1.6
    well-balanced property); mass and total energy conserved."""
    prob, U = I.atmosphere((128, 128), low_mach=low_mach)
    d0 = O.diagnostics(prob, U)
    V, t = O.run(prob, U, 1000)
    d = O.diagnostics(prob, V)
    assert d["max_speed"] < 1e-12
    assert abs(d["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d["energy"] - d0["energy"]) <= 1e-13 * d0["energy"]


def test_polytrope_with_diffusion_stays_at_rest():
    """Linear temperature profile: constant conductive flux, zero divergence;
    the no-slip fixed-temperature walls keep the discrete equilibrium."""
    prob, U = I.rayleigh_benard(2, (32, 16), amp=0.0)
    V, t = O.run(prob, U, 300)
    assert O.diagnostics(prob, V)["max_speed"] < 1e-12


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "well_balanced_table1.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            n, a, b = line.split()
            rows.append((int(n), float(a), float(b)))
    return rows


@pytest.mark.parametrize("row", _table1()[:3], ids=lambda r: f"n{r[0]}")
def test_paper_table1_well_balanced_column(row):
    """Sec. 4.3 Table 1: isothermal column on [0, 3] at t = 10.  The printed
    max velocity with theta = 1 is reproduced within a factor 3 (round-off
    values depend on operation order); with theta = Ma the paper reports a
    boundary-induced shift that the wall ghosts used here do not show, so it
    is an upper bound."""
    n, v_theta1, v_thetaMa = row
    for low_mach, ref in ((0, v_theta1), (1, v_thetaMa)):
        prob, U = I.well_balanced_column(n, low_mach=low_mach)
        V, t = O.run(prob, U, 10 ** 7, t_end=10.0)
        assert t == pytest.approx(10.0)
        vmax = O.diagnostics(prob, V)["max_speed"]
        if low_mach == 0:
            assert ref / 3 <= vmax <= 3 * ref, (n, vmax, ref)
        else:
            assert vmax <= ref


@pytest.mark.parametrize("dim,n", [(2, (24, 20)), (3, (10, 9, 8))])
def test_conservation_periodic_with_diffusion(dim, n):
    prob, U = I.random_periodic(dim, n, mu=0.01, kappa=0.02)
    d0 = O.diagnostics(prob, U)
    V, _ = O.run(prob, U, 50)
    d = O.diagnostics(prob, V)
    assert abs(d["mass"] - d0["mass"]) <= 2e-15 * n[0] * d0["mass"]
    assert abs(d["energy"] - d0["energy"]) <= 2e-15 * n[0] * d0["energy"]
    for k in ("mom_x", "mom_y", "mom_z"):
        assert abs(d[k] - d0[k]) <= 1e-16 * n[0]


@pytest.mark.parametrize("dim,n", [(2, (20, 16)), (3, (8, 7, 10))])
def test_conservation_with_gravity_and_walls(dim, n):
    """Mass, total energy rho*calE and the transverse momenta are conserved
    to machine precision with gravity and reflective hydrostatic walls
    (abstract; Sec. 2.1.5)."""
    prob, U = I.stratified_random(dim, n, walls=I.REFLECT_HYDRO)
    d0 = O.diagnostics(prob, U)
    V, _ = O.run(prob, U, 100)
    d = O.diagnostics(prob, V)
    assert abs(d["mass"] - d0["mass"]) <= 1e-14 * d0["mass"]
    assert abs(d["energy"] - d0["energy"]) <= 1e-14 * d0["energy"]
    names = ("mom_x", "mom_y", "mom_z")[: dim - 1]
    for k in names:
        assert abs(d[k] - d0[k]) <= 1e-17 * np.prod(n)
    # the vertical momentum does change (gravity acts): the test is not vacuous
    vert = ("mom_x", "mom_y", "mom_z")[dim - 1]
    assert abs(d[vert] - d0[vert]) > 1e-8


def test_xy_symmetry_transpose():
    prob, U = I.random_periodic(2, (12, 10), seed=3, mu=0.01, kappa=0.01)
    probT = prob.replace(n=(10, 12, 1))
    UT = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    dt = O.dt(prob, U)
    assert O.dt(probT, UT) == pytest.approx(dt, rel=1e-15)
    V = O.step(prob, U, dt)
    VT = O.step(probT, UT, dt)
    back = np.stack([VT[0].T, VT[2].T, VT[1].T, VT[3].T])
    assert np.max(np.abs(back - V)) <= 1e-14 * np.max(np.abs(V))


def test_xyz_symmetry_3d_permutation():
    prob, U = I.random_periodic(3, (6, 5, 4), seed=4, mu=0.01, kappa=0.01)
    # cyclic permutation x->y->z->x
    probP = prob.replace(n=(4, 6, 5))
    P = lambda a: np.transpose(a, (1, 2, 0))    # (z, y, x) -> (y, x, z) index order of new (z', y', x')
    UP = np.stack([P(U[0]), P(U[3]), P(U[1]), P(U[2]), P(U[4])])
    dt = O.dt(prob, U)
    V = O.step(prob, U, dt)
    VP = O.step(probP, UP, dt)
    expect = np.stack([P(V[0]), P(V[3]), P(V[1]), P(V[2]), P(V[4])])
    assert np.max(np.abs(VP - expect)) <= 1e-14 * np.max(np.abs(V))


def test_uniform_velocity_and_pressure_reduce_to_upwind_advection():
    """At uniform u and p the face values are u* = u, Pi* = p exactly, so the
    step is first-order upwind advection of rho (and of m, W)."""
    n = 40
    prob = I.Problem(dim=2, n=(n, 1, 1), lo=(0, 0, 0), hi=(1, 1.0 / n, 1), gamma=1.4)
    x = prob.centers(0)[None, :]
    rho = 1.0 + 0.5 * np.exp(-100 * (x - 0.5) ** 2)
    for u in (0.7, -0.4):
        U = I._assemble(prob, rho, [np.full_like(rho, u), np.zeros_like(rho)], np.ones_like(rho))
        dt = 0.3 * prob.dx[0] / (abs(u) + 2.0)
        V = O.step(prob, U, dt)
        nu = u * dt / prob.dx[0]
        r = rho[0]
        up = r - nu * (r - np.roll(r, 1)) if u > 0 else r - nu * (np.roll(r, -1) - r)
        np.testing.assert_allclose(V[0, 0], up, rtol=1e-14)
        _, vel, p = _prim(prob, V)
        np.testing.assert_allclose(p, 1.0, rtol=1e-13)
        np.testing.assert_allclose(vel[0], u, rtol=1e-13)


# --------------------------------------------------------------------------
# dissipative fluxes (Sec. 2.2)
# --------------------------------------------------------------------------
def test_shear_wave_decays_at_viscous_rate():
    n, eps, mu = 64, 1e-3, 0.01
    prob = I.Problem(dim=2, n=(1, n, 1), lo=(0, 0, 0), hi=(1.0 / n, 1, 1), gamma=5 / 3, mu=mu)
    y = prob.centers(1)[:, None]
    u = eps * np.sin(2 * np.pi * y)
    U = I._assemble(prob, np.ones((n, 1)), [u, np.zeros((n, 1))], np.ones((n, 1)))
    V, t = O.run(prob, U, 10 ** 6, t_end=5.0)
    amp = 2 * np.mean(V[1] / V[0] * np.sin(2 * np.pi * y))
    rate = math.log(amp / eps) / t
    assert rate == pytest.approx(-mu * (2 * np.pi) ** 2, rel=2e-3)


def test_entropy_mode_decays_at_isobaric_conduction_rate():
    """A temperature ripple at uniform pressure decays at kappa k^2 / (rho c_p)
    (slow-mode limit; acoustic coupling gives < 1 % here)."""
    n, eps, kappa, g = 64, 1e-3, 0.01, 5 / 3
    prob = I.Problem(dim=2, n=(n, 1, 1), lo=(0, 0, 0), hi=(1, 1.0 / n, 1), gamma=g, kappa=kappa)
    x = prob.centers(0)[None, :]
    T = 1 + eps * np.sin(2 * np.pi * x)
    U = I._assemble(prob, 1.0 / T, [np.zeros_like(T)] * 2, np.ones_like(T))
    V, t = O.run(prob, U, 10 ** 6, t_end=5.0)
    rho, vel, p = _prim(prob, V)
    T2 = p / rho
    amp = 2 * np.mean((T2 - T2.mean()) * np.sin(2 * np.pi * x))
    rate = math.log(amp / eps) / t
    cp = g / (g - 1)
    assert rate == pytest.approx(-kappa * (2 * np.pi) ** 2 / cp, rel=2e-2)


# --------------------------------------------------------------------------
# shocks and the low-Mach regime (Sec. 4.1, 4.2)
# --------------------------------------------------------------------------
def test_sod_converges_to_exact_riemann_solution():
    errs = {}
    for low_mach in (0, 1):
        e = []
        for n in (100, 200, 400):
            prob, U = I.sod(n, low_mach=low_mach)
            V, t = O.run(prob, U, 10 ** 6, t_end=0.2)
            ex = riemann_sample(prob.centers(0), 0.2, 0.5, (1, 0, 1), (0.125, 0, 0.1), 1.4)
            e.append(np.mean(np.abs(V[0, 0] - ex[0])))
        assert e[0] < 0.03
        assert e[0] > e[1] > e[2]
        assert math.log2(e[0] / e[2]) / 2 > 0.5
        errs[low_mach] = e
    # the correction barely changes the shock tube (Sec. 4.1)
    assert errs[1][0] == pytest.approx(errs[0][0], rel=0.3)


def test_sod_same_along_x_and_y():
    px, Ux = I.sod(100, axis=0)
    py, Uy = I.sod(100, axis=1)
    Vx, _ = O.run(px, Ux, 10 ** 6, t_end=0.2)
    Vy, _ = O.run(py, Uy, 10 ** 6, t_end=0.2)
    np.testing.assert_array_equal(Vx[0, 0, :], Vy[0, :, 0])
    np.testing.assert_array_equal(Vx[1, 0, :], Vy[2, :, 0])


def test_gresho_low_mach_correction():
    """Sec. 4.2: with the correction the velocity error does not grow as Ma
    decreases; without it, it grows roughly like 1/Ma."""
    err = {}
    for low_mach in (0, 1):
        for mach in (1e-2, 1e-3):
            prob, U = I.gresho(32, mach=mach, low_mach=low_mach)
            V, _ = O.run(prob, U, 10 ** 6, t_end=2e-3)
            ue, ve = I.gresho_velocity(prob)
            err[(low_mach, mach)] = np.mean(np.abs(V[1] / V[0] - ue) + np.abs(V[2] / V[0] - ve))
    assert 0.8 < err[(1, 1e-3)] / err[(1, 1e-2)] < 1.25
    assert err[(0, 1e-3)] / err[(0, 1e-2)] > 3.0
    assert err[(0, 1e-3)] > 20 * err[(1, 1e-3)]


# --------------------------------------------------------------------------
# window evaluation (used for sampled checks at full size)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,n", [(2, (13, 11)), (3, (7, 6, 9))])
def test_window_equals_full_step(dim, n):
    prob, U = I.stratified_random(dim, n, walls=I.NOSLIP_FIXED_T, mu=0.02, kappa=0.03)
    dt = O.dt(prob, U)
    V = O.step(prob, U, dt)
    lo = [1, 2, 3][:dim]
    hi = [n[0] - 2, n[1], n[2] - 1][:dim] if dim == 3 else [n[0] - 2, n[1]]
    W = O.step_window(prob, U, dt, lo, hi)
    sl = tuple(slice(lo[d], hi[d]) for d in reversed(range(dim)))
    np.testing.assert_array_equal(W, V[(slice(None),) + sl])


def test_sound_wave_viscous_damping_uses_stokes_hypothesis():
    """Classical (Stokes) absorption: with eta = -2 mu / 3 (Eq. 4) a standing
    sound wave loses acoustic energy at (4/3) mu k^2 / rho; the scheme's own
    numerical damping is removed by differencing two runs at one fixed dt."""
    g, n, eps, mu = 5 / 3, 64, 1e-4, 0.01

    def energy_ratio(mu_, dt):
        prob = I.Problem(dim=2, n=(n, 1, 1), lo=(0, 0, 0), hi=(1, 1.0 / n, 1), gamma=g, mu=mu_)
        x = prob.centers(0)[None, :]
        u = eps * np.sin(2 * np.pi * x)
        U = I._assemble(prob, np.ones_like(u), [u, np.zeros_like(u)], np.ones_like(u))
        V, t = O.run(prob, U, int(round(2.0 / dt)), dt_fixed=dt)
        rho, vel, p = _prim(prob, V)
        E = np.sum(0.5 * rho * vel[0] ** 2 + (p - 1) ** 2 / (2 * g))
        return E / np.sum(0.5 * u * u), t

    prob = I.Problem(dim=2, n=(n, 1, 1), lo=(0, 0, 0), hi=(1, 1.0 / n, 1), gamma=g, mu=2 * mu)
    dt = O.dt(prob, I._assemble(prob, np.ones((1, n)), [np.zeros((1, n))] * 2, np.ones((1, n))))
    e0, t = energy_ratio(0.0, dt)
    e1, _ = energy_ratio(mu, dt)
    rate = math.log(e1 / e0) / t
    assert rate == pytest.approx(-(4.0 / 3.0) * mu * (2 * np.pi) ** 2, rel=5e-2)


def test_diagonal_shear_wave_uses_tangential_derivatives():
    """A divergence-free shear wave along the diagonal decays at nu |k|^2; its
    stress involves the cross (tangential) derivatives at every face."""
    n, eps, mu = 32, 1e-3, 0.01
    prob = I.Problem(dim=2, n=(n, n, 1), lo=(0, 0, 0), hi=(1, 1, 1), gamma=5 / 3, mu=mu)
    x = prob.centers(0)[None, :]
    y = prob.centers(1)[:, None]
    s = eps * np.sin(2 * np.pi * (x + y))
    U = I._assemble(prob, np.ones_like(s), [s / np.sqrt(2), -s / np.sqrt(2)], np.ones_like(s))
    V, t = O.run(prob, U, 10 ** 6, t_end=2.0)
    amp = 2 * np.mean((V[1] / V[0]) * np.sqrt(2) * np.sin(2 * np.pi * (x + y)))
    assert math.log(amp / eps) / t == pytest.approx(-mu * 2 * (2 * np.pi) ** 2, rel=5e-3)


def test_viscous_heating_is_second_order_local():
    """Kinetic energy lost to viscosity reappears locally as mu (du/dy)^2 of
    internal energy, to second order in the grid size (shear flow, one tiny step)."""
    errs = []
    for n in (32, 64):
        mu, eps, k = 0.01, 0.1, 2 * np.pi
        prob = I.Problem(dim=2, n=(1, n, 1), lo=(0, 0, 0), hi=(1.0 / n, 1, 1), gamma=5 / 3, mu=mu)
        y = prob.centers(1)[:, None]
        u = eps * np.sin(k * y)
        U = I._assemble(prob, np.ones((n, 1)), [u, np.zeros((n, 1))], np.ones((n, 1)))
        dt = 1e-3 * O.dt(prob, U)
        V = O.step(prob, U, dt)
        rhoe = lambda A: A[3] - 0.5 * (A[1] ** 2 + A[2] ** 2) / A[0]
        heat = (rhoe(V) - rhoe(U)) / dt
        exact = mu * (eps * k * np.cos(k * y)) ** 2
        errs.append(np.max(np.abs(heat - exact)) / np.max(exact))
    assert errs[0] < 0.02
    assert errs[0] / errs[1] > 3.5     # second order


def test_low_mach_theta_never_exceeds_either_side_mach_number():
    """Eq. 16 uses the larger sound speed of the two cells: theta <= |u*| / c on both sides."""
    prob = I.Problem(dim=2, n=(4, 4, 1), lo=(0, 0, 0), hi=(1, 1, 1), gamma=1.4, low_mach=1)
    rng = np.random.default_rng(11)
    for _ in range(50):
        L = [rng.uniform(0.2, 3), rng.uniform(-0.3, 0.3), 0, 0, rng.uniform(0.2, 3), 0]
        R = [rng.uniform(0.2, 3), rng.uniform(-0.3, 0.3), 0, 0, rng.uniform(0.2, 3), 0]
        f = O.face(prob, L, R, 0)
        for s in (L, R):
            c = math.sqrt(1.4 * s[4] / s[0])
            assert f["theta"] <= abs(f["ustar"]) / c * (1 + 1e-14)
        cmax = max(math.sqrt(1.4 * L[4] / L[0]), math.sqrt(1.4 * R[4] / R[0]))
        assert f["theta"] == pytest.approx(min(abs(f["ustar"]) / cmax, 1.0), rel=1e-14)


# --------------------------------------------------------------------------
# Appendix B: non-conservative energy form (rho E without rho Phi, gravity
# work as the source dt/dx (uS)_i)
# --------------------------------------------------------------------------
def test_appendix_b_equals_sec2_scheme_without_gravity():
    """With a constant potential both energy forms are the same scheme (S = 0)."""
    prob, U = I.random_periodic(2, (20, 16), mu=0.01, kappa=0.01)
    p1, U1 = I.to_energy_form(prob, U, 1)
    A, _ = O.run(prob, U, 20)
    B, _ = O.run(p1, U1, 20)
    assert np.array_equal(A, B)


def test_appendix_b_keeps_atmosphere_at_rest():
    prob, U = I.atmosphere((64, 64))
    p1, U1 = I.to_energy_form(prob, U, 1)
    V, _ = O.run(p1, U1, 500)
    assert O.diagnostics(p1, V)["max_speed"] < 1e-13


def test_appendix_b_converges_to_the_conservative_form():
    """Both forms discretise the same equations: on a smooth stratified flow
    their difference shrinks at first order with the grid (a wrong sign or
    factor in the (uS) source leaves an O(1) gap)."""
    gaps = []
    for n in (16, 32, 64):
        prob, Ub = I.stratified_random(2, (n, n), seed=3, amp=0.0)
        x = prob.centers(0)[None, :]
        y = prob.centers(1)[:, None]
        pert = 0.05 * np.sin(2 * np.pi * x) * np.sin(np.pi * y)
        U = Ub.copy()
        U[2] = Ub[0] * pert
        U[3] = Ub[3] + 0.5 * Ub[0] * pert ** 2
        p1, U1 = I.to_energy_form(prob, U, 1)
        A, _ = O.run(prob, U, 10 ** 6, t_end=0.2)
        B, _ = O.run(p1, U1, 10 ** 6, t_end=0.2)
        _, B0 = I.to_energy_form(p1, B, 0)
        gaps.append(max(np.max(np.abs(A[f] - B0[f])) / np.max(np.abs(A[f])) for f in (0, 2, 3)))
    assert gaps[0] < 0.02
    assert math.log2(gaps[0] / gaps[1]) > 0.8 and math.log2(gaps[1] / gaps[2]) > 0.8


# --------------------------------------------------------------------------
# Rayleigh-Taylor set-up (Sec. 4.4) and strong stratification (Sec. 4.5)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("low_mach", [1, 0])
def test_rayleigh_taylor_rest_state_is_a_discrete_equilibrium(low_mach):
    """The two-fluid state at rest (density jump 1 -> 2 on a face) stays at rest
    to round-off without any well-balanced reconstruction: the source S of
    every face, the interface included, equals the pressure jump (Sec. 4.4)."""
    prob, U = I.rayleigh_taylor((20, 60), C=0.0, low_mach=low_mach)
    V, _ = O.run(prob, U, 500)
    d = O.diagnostics(prob, V)
    assert d["max_speed"] < 1e-12
    assert np.max(np.abs(V[0] - U[0])) < 1e-12


def test_rayleigh_taylor_interface_is_unstable_and_conserves_mass():
    """Heavy over light is unstable: the seeded mode grows, mass and energy
    are conserved between the reflective walls."""
    prob, U = I.rayleigh_taylor((20, 60), C=0.01)
    V, t = O.run(prob, U, 10 ** 6, t_end=6.0)
    d0, d1 = O.diagnostics(prob, U), O.diagnostics(prob, V)
    assert d1["max_speed"] > 2.0 * d0["max_speed"]
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-13)
    assert d1["energy"] == pytest.approx(d0["energy"], rel=1e-13)


def test_strongly_stratified_polytrope_stays_at_rest():
    """chi = 21 (density contrast 21 across the layer, Sec. 4.5): the discrete
    polytrope at rest with the no-slip fixed-temperature walls and heat
    conduction stays at rest (linear T: uniform conductive flux)."""
    prob, U = I.rayleigh_benard(2, (16, 40), chi=21.0, amp=0.0)
    # rho = T^m with T = z0 + 1 - y: the wall densities differ by chi
    assert (prob.T_lo[1] / prob.T_hi[1]) ** 1.3 == pytest.approx(21.0, rel=1e-12)
    V, _ = O.run(prob, U, 300)
    assert O.diagnostics(prob, V)["max_speed"] < 1e-10



# --------------------------------------------------------------------------
# Caller-supplied potential Phi at the cell centres (R20)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("low_mach", [1, 0])
def test_tilted_gravity_atmosphere_is_a_discrete_equilibrium(low_mach):
    """Gravity not along an axis (a Phi array with steps in x and y, walls on
    all sides): the isothermal state built by Eq. 18 along both axes stays at
    rest -- the source S of the in-plane faces balances their pressure jumps."""
    prob, U = I.tilted_atmosphere((24, 20), gx=-0.3, gy=-1.0, low_mach=low_mach)
    V, _ = O.run(prob, U, 500)
    assert O.diagnostics(prob, V)["max_speed"] < 1e-12


@pytest.mark.parametrize("walls", [I.NOSLIP_FIXED_T, I.REFLECT_HYDRO])
def test_non_uniform_gravity_column_is_a_discrete_equilibrium(walls):
    """A potential that varies along the last axis only, Phi = 2 y + 1.5 y^2
    (non-uniform gravity), with the column T = 3 - y built by Eq. 18 for it:
    the state stays at rest, in 2D and 3D, with either wall rule."""
    for dim, n in ((2, (12, 16)), (3, (6, 5, 16))):
        prob, U = I.row_potential_state(dim, n, amp=0.0, walls=walls)
        V, _ = O.run(prob, U, 300)
        assert O.diagnostics(prob, V)["max_speed"] < 1e-13


def test_potential_array_equal_to_uniform_gravity_gives_the_same_steps():
    """Phi given as an array equal to -g y reproduces the uniform-gravity steps
    (to rounding: the wall ghosts of the array extend Phi linearly instead of
    evaluating -g y)."""
    prob, U = I.stratified_random(2, (12, 16), mu=0.01, kappa=0.02)
    probA = prob.replace(phi=np.ascontiguousarray(np.array(prob.potential())), g=0.0)
    A, _ = O.run(prob, U, 30)
    B, _ = O.run(probA, U, 30)
    assert np.max(np.abs(A - B)) <= 1e-13 * np.max(np.abs(A))


def test_gravity_along_x_is_the_transposed_gravity_along_y():
    """Gravity along x through a Phi array, walls in x, equals the transposed
    run of the built-in gravity along y: pins S, the momentum source and the
    hydrostatic wall ghosts on in-plane faces against the gravity axis."""
    prob, U = I.stratified_random(2, (10, 14), mu=0.01, kappa=0.02)
    n = 20
    V, _ = O.run(prob, U, n)
    probT = I.Problem(dim=2, n=(14, 10, 1), lo=(0.0, 0.0, 0.0), hi=(prob.hi[1], prob.hi[0], 1.0), gamma=prob.gamma,
                      mu=prob.mu, kappa=prob.kappa, low_mach=prob.low_mach,
                      bc_lo=(prob.bc_lo[1], prob.bc_lo[0], I.PERIODIC), bc_hi=(prob.bc_hi[1], prob.bc_hi[0], I.PERIODIC),
                      T_lo=(prob.T_lo[1], prob.T_lo[0], 0.0), T_hi=(prob.T_hi[1], prob.T_hi[0], 0.0),
                      phi=np.ascontiguousarray(np.array(prob.potential()).T))
    UT = np.stack([U[0].T, U[2].T, U[1].T, U[3].T])
    VT, _ = O.run(probT, UT, n)
    back = np.stack([VT[0].T, VT[2].T, VT[1].T, VT[3].T])
    assert np.max(np.abs(back - V)) <= 1e-13 * np.max(np.abs(V))


def test_periodic_potential_conserves_mass_and_energy():
    """Time-independent Phi in a periodic box: mass and rho*calE telescope
    exactly (Sec. 2.1); the momentum changes (the potential exerts a force)."""
    prob, U = I.periodic_potential_state(2, (24, 20), A=0.3)
    d0 = O.diagnostics(prob, U)
    V, _ = O.run(prob, U, 200)
    d1 = O.diagnostics(prob, V)
    assert d1["mass"] == pytest.approx(d0["mass"], rel=1e-13)
    assert d1["energy"] == pytest.approx(d0["energy"], rel=1e-13)
    assert abs(d1["mom_x"] - d0["mom_x"]) > 1e-6


def test_ghost_potential_extends_a_linear_potential_exactly():
    """R20 on a linear Phi: the ghost values of both layers, at sides, edges
    and corners, across walls and outflow, are the values of the same linear
    function at the ghost centres (and wrap across periodic sides)."""
    g = (-0.7, -1.3)
    prob = I.Problem(dim=2, n=(6, 5, 1), lo=(0.0, 0.0, 0.0), hi=(1.2, 0.5, 1.0),
                     bc_lo=(I.OUTFLOW, I.REFLECT_HYDRO, I.PERIODIC), bc_hi=(I.REFLECT_HYDRO, I.OUTFLOW, I.PERIODIC))
    xs = lambda d, i: prob.lo[d] + (i + 0.5) * prob.dx[d]
    lin = lambda i, j: -g[0] * xs(0, i) - g[1] * xs(1, j)
    phi = np.array([[lin(i, j) for i in range(6)] for j in range(5)])
    probA = prob.replace(phi=phi)
    U = I._assemble(probA, np.ones((5, 6)), [np.zeros((5, 6))] * 2, np.ones((5, 6)))
    for i in range(-2, 8):
        for j in range(-2, 7):
            c = O.cell_at(probA, U, (i, j, 0))
            assert c["phi"] == pytest.approx(lin(i, j), rel=0, abs=1e-14), (i, j)
    # periodic side: the value wraps
    probP = probA.replace(bc_lo=(I.PERIODIC, I.REFLECT_HYDRO, I.PERIODIC), bc_hi=(I.PERIODIC, I.OUTFLOW, I.PERIODIC))
    assert O.cell_at(probP, U, (-1, 2, 0))["phi"] == phi[2, 5]
    assert O.cell_at(probP, U, (7, 1, 0))["phi"] == phi[1, 1]


# --------------------------------------------------------------------------
# stiffened-gas equation of state (Sec. 4 admits another equation of state;
# R21: p = (gamma-1) rho e - gamma p_inf, T = (p + p_inf)/rho)
# --------------------------------------------------------------------------
def _stiffened_cases():
    walls, Uw = I.stratified_random(2, (14, 12), seed=11, amp=2e-2, mu=0.02, kappa=0.03,
                                    walls=I.NOSLIP_FIXED_T, p_inf=3.0)
    refl, Ur = I.stratified_random(3, (7, 6, 8), seed=12, amp=2e-2, mu=0.01, kappa=0.01,
                                   walls=I.REFLECT_HYDRO, p_inf=2.0, low_mach=0)
    tube, Ut = I.sod(40, gamma=4.4, p_inf=6.0, left=(1.0, 8.0), right=(0.8, 0.1))
    pb, Ub = I.to_energy_form(walls, Uw, 1)
    pot, Up = I.periodic_potential_state(2, (12, 10), seed=13, mu=0.01, kappa=0.02)
    pot = pot.replace(p_inf=4.0)
    Up = np.array(Up)
    Up[pot.dim + 1] += 4.0 * pot.gamma / (pot.gamma - 1.0)   # the same (rho, u, p) as a stiffened gas
    return {"noslip_viscous_2d": (walls, Uw), "reflect_3d": (refl, Ur), "outflow_tube": (tube, Ut),
            "appendix_b": (pb, Ub), "potential_array": (pot, Up)}


@pytest.mark.parametrize("case", list(_stiffened_cases()))
def test_stiffened_gas_is_the_ideal_gas_of_the_shifted_energy(case):
    """A change of variables, exact in exact arithmetic: with pi = p + p_inf a
    stiffened gas has rho e - p_inf = pi / (gamma-1), c^2 = gamma pi / rho and
    T = pi / rho, all ideal-gas relations in pi.  The scheme reads pressures
    only through differences (u*, [Pi*], the wall balance of Eq. 18 written in
    pi), through c and T, and through the energy flux (W~ + Pi*) u*, where the
    shift of Pi* by -p_inf cancels that of W~ by +p_inf (L~ = 1 + lambda
    [u*]).  So a step of the stiffened gas on U equals a step of the ideal gas
    on U - p_inf e_W, plus p_inf e_W, for every boundary rule, with the
    dissipative fluxes, in both energy forms, and the time steps agree."""
    prob, U = _stiffened_cases()[case]
    s = prob.p_inf
    e = prob.dim + 1
    ideal = prob.replace(p_inf=0.0)
    Ui = np.array(U)
    Ui[e] -= s
    assert O.dt(prob, U) == pytest.approx(O.dt(ideal, Ui), rel=1e-14)
    dt = 0.5 * O.dt(prob, U)
    V, Vi = np.array(U), np.array(Ui)
    for _ in range(20):
        V = O.step(prob, V, dt)
        Vi = O.step(ideal, Vi, dt)
    Vi[e] += s
    scale = [np.max(np.abs(U[0]))] + [np.max(np.abs(U[0])) * 2.0] * prob.dim + [np.max(np.abs(U[e]))]
    for f in range(prob.nfields):
        assert np.max(np.abs(V[f] - Vi[f])) <= 5e-14 * scale[f], (case, f)
    # not vacuous: an ideal gas with the same (rho, u, p) steps differently (the
    # stratified cases hold too little pressure to be ideal-gas columns)
    if case in ("outflow_tube", "potential_array"):
        Ug = np.array(U)
        Ug[e] -= s * prob.gamma / (prob.gamma - 1.0)
        assert np.max(np.abs(O.step(ideal, Ug, dt)[1:e] - O.step(prob, U, dt)[1:e])) > 1e-7


def test_stiffened_shock_tube_converges_to_exact_riemann_solution():
    """Water-like stiffened gas (gamma = 4.4, p_inf = 6) shock tube against the
    exact solution, which is the ideal-gas solution in the shifted pressure
    p + p_inf (Ivings, Causon and Toro 1998): density L1 error falls with the
    grid (t = 0.04, before any wave leaves [0, 1]), pressure and velocity
    follow the exact profiles."""
    g, pinf = 4.4, 6.0
    L, R = (1.0, 8.0), (0.8, 0.1)
    e = []
    for n in (100, 200, 400):
        prob, U = I.sod(n, gamma=g, p_inf=pinf, left=L, right=R)
        V, t = O.run(prob, U, 10 ** 6, t_end=0.04)
        assert t == pytest.approx(0.04)
        ex = riemann_sample(prob.centers(0), 0.04, 0.5, (L[0], 0.0, L[1] + pinf), (R[0], 0.0, R[1] + pinf), g)
        e.append(np.mean(np.abs(V[0, 0] - ex[0])))
        if n == 400:
            rho = V[0, 0]
            u = V[1, 0] / rho
            p = (g - 1.0) * (V[3, 0] - 0.5 * rho * u * u) - g * pinf
            assert np.mean(np.abs(p - (ex[2] - pinf))) < 0.005 * (L[1] + pinf)
            assert np.mean(np.abs(u - ex[1])) < 0.05 * np.max(np.abs(ex[1]))
    assert e[0] < 0.005
    assert e[0] > e[1] > e[2]
    assert math.log2(e[0] / e[2]) / 2 > 0.5


@pytest.mark.parametrize("low_mach", [0, 1])
def test_stiffened_liquid_column_stays_at_rest(low_mach):
    """An isothermal stiffened-gas column (p_inf = 5) built by the discrete
    balance of Eq. 18 in p + p_inf is a discrete equilibrium with the
    reflective hydrostatic walls (Sec. 2.1.6); mass and energy conserved.
    The upper part is under tension (p < 0 < p + p_inf), which a stiffened
    gas allows."""
    prob, U = I.atmosphere((32, 64), low_mach=low_mach, p_inf=5.0)
    d0 = O.diagnostics(prob, U)
    assert d0["min_p"] < 0.0
    V, t = O.run(prob, U, 1000)
    d = O.diagnostics(prob, V)
    assert d["max_speed"] < 1e-12
    assert abs(d["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
    assert abs(d["energy"] - d0["energy"]) <= 1e-13 * d0["energy"]


def test_stiffened_gas_zero_constant_is_the_ideal_gas_bitwise():
    prob, U = I.stratified_random(2, (12, 10), seed=3, mu=0.01, kappa=0.02)
    assert prob.p_inf == 0.0
    a = O.step(prob, U, 1e-3)
    b = O.step(prob.replace(p_inf=-0.0), U, 1e-3)
    assert np.array_equal(a, b)


# --------------------------------------------------------------------------
# Noble-Abel stiffened gas (covolume b; R22): p = (gamma-1) rho e / (1 - b rho)
# - gamma p_inf, T = (p + p_inf)(1 - b rho)/rho, c^2 = gamma (p + p_inf)/(rho (1 - b rho))
# --------------------------------------------------------------------------
def test_noble_abel_shock_tube_converges_to_exact_riemann_solution():
    """Shock tube of a Noble-Abel stiffened gas (gamma = 1.4, p_inf = 0.3,
    b = 0.4: the left state fills 40 % of its volume with covolume) against
    the exact solution (the covolume gas of Toro, Ch. 4.7, in p + p_inf):
    density L1 error falls with the grid, pressure and velocity follow the
    exact profiles.  The waves' positions depend on the sound speed
    c^2 = gamma (p + p_inf) / (rho (1 - b rho)) and the star state on the
    energy law, so a law without the covolume fails."""
    from riemann_exact import sample_covolume
    g, pinf, b = 1.4, 0.3, 0.4
    L, R = (1.0, 1.0), (0.125, 0.1)
    t_end = 0.1
    e = []
    for n in (100, 200, 400):
        prob, U = I.sod(n, gamma=g, p_inf=pinf, b=b, left=L, right=R)
        V, t = O.run(prob, U, 10 ** 6, t_end=t_end)
        assert t == pytest.approx(t_end)
        ex = sample_covolume(prob.centers(0), t_end, 0.5, (L[0], 0.0, L[1]), (R[0], 0.0, R[1]), g, pinf, b)
        e.append(np.mean(np.abs(V[0, 0] - ex[0])))
        if n == 400:
            rho = V[0, 0]
            u = V[1, 0] / rho
            p = (g - 1.0) * (V[3, 0] - 0.5 * rho * u * u) / (1.0 - b * rho) - g * pinf
            assert np.mean(np.abs(p - ex[2])) < 0.01 * L[1]
            assert np.mean(np.abs(u - ex[1])) < 0.05 * np.max(np.abs(ex[1]))
    assert e[0] < 0.02
    assert e[0] > e[1] > e[2]
    assert math.log2(e[0] / e[2]) / 2 > 0.5
    # the same tube read with the stiffened-gas law (no covolume) is far off
    prob, U = I.sod(400, gamma=g, p_inf=pinf, b=b, left=L, right=R)
    V, _ = O.run(prob.replace(b=0.0), U, 10 ** 6, t_end=t_end)
    ex = sample_covolume(prob.centers(0), t_end, 0.5, (L[0], 0.0, L[1]), (R[0], 0.0, R[1]), g, pinf, b)
    assert np.mean(np.abs(V[0, 0] - ex[0])) > 3 * e[2]


@pytest.mark.parametrize("low_mach", [0, 1])
def test_noble_abel_columns_stay_at_rest(low_mach):
    """Columns of a Noble-Abel stiffened gas built by the discrete balance of
    Eq. 18 with rho = (p + p_inf) / (T + b (p + p_inf)) are discrete
    equilibria: an isothermal column between reflective hydrostatic walls
    (2D) and a viscous polytrope between them (3D), and a conducting, viscous
    polytrope (linear T) between fixed-temperature no-slip walls, whose heat
    flux is uniform only if T is the law's temperature.  Mass and energy are
    conserved."""
    cases = [I.atmosphere((16, 48), low_mach=low_mach, p_inf=0.5, b=0.3),
             I.stratified_random(2, (12, 40), amp=0.0, mu=0.02, kappa=0.05, low_mach=low_mach, p_inf=0.2, b=0.2),
             # reflective walls are adiabatic: viscous, but not conducting, to stay at rest
             I.stratified_random(3, (5, 4, 24), amp=0.0, mu=0.02, kappa=0.0, low_mach=low_mach, b=0.25,
                                 walls=I.REFLECT_HYDRO)]
    for prob, U in cases:
        assert np.max(prob.b * U[0]) > 0.05      # the covolume matters
        d0 = O.diagnostics(prob, U)
        V, _ = O.run(prob, U, 500)
        d = O.diagnostics(prob, V)
        assert d["max_speed"] < 1e-12, d["max_speed"]
        assert abs(d["mass"] - d0["mass"]) <= 1e-13 * d0["mass"]
        assert abs(d["energy"] - d0["energy"]) <= 1e-13 * abs(d0["energy"])


def test_noble_abel_conserves_mass_energy_and_momentum():
    """A disturbed Noble-Abel gas in a periodic box (no gravity): the totals of
    mass, momentum and energy are unchanged to round-off (telescoping fluxes)."""
    prob, U = I.random_periodic(2, (24, 20), seed=5, amp=0.2, mu=0.01, kappa=0.02)
    prob = prob.replace(b=0.35, p_inf=0.4)
    rho = U[0]
    ke = 0.5 * (U[1] ** 2 + U[2] ** 2) / rho
    p = (prob.gamma - 1.0) * (U[3] - ke)          # the pressure U was built with (ideal gas)
    U = np.array(U)
    U[3] = (p + prob.gamma * prob.p_inf) * (1.0 - prob.b * rho) / (prob.gamma - 1.0) + ke
    d0 = O.diagnostics(prob, U)
    V, _ = O.run(prob, U, 200)
    d = O.diagnostics(prob, V)
    for k in ("mass", "energy"):
        assert abs(d[k] - d0[k]) <= 1e-13 * abs(d0[k]), k
    for k in ("mom_x", "mom_y"):
        assert abs(d[k] - d0[k]) <= 1e-13 * d0["mass"], k
    assert d["max_speed"] > 1e-3     # it moved


def test_noble_abel_zero_covolume_is_the_stiffened_gas_bitwise():
    prob, U = I.stratified_random(2, (12, 10), seed=3, mu=0.01, kappa=0.02, p_inf=0.7)
    assert prob.b == 0.0
    a = O.step(prob, U, 1e-3)
    b = O.step(prob.replace(b=-0.0), U, 1e-3)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("axis", [0, 1])
def test_noble_abel_uniform_flow_through_outflow_ends_stays_uniform(axis):
    """A uniform Noble-Abel flow entering through one zero-gradient end and
    leaving through the other: the inflow face carries the ghost's upwind
    energy (rho e of the ghost from its p, with the covolume), so the state
    stays uniform to round-off only if the ghost's energy follows the law."""
    prob, U = I.sod(16, axis=axis, p_inf=0.3, b=0.4, left=(1.2, 0.8), right=(1.2, 0.8))
    u = -0.35
    U = np.array(U)
    U[1 + axis] = U[0] * u
    U[3] += 0.5 * U[0] * u * u
    V, _ = O.run(prob, U, 50)
    assert np.max(np.abs(V - U)) <= 1e-13 * np.max(np.abs(U))
