"""Second writing of one 2D step of the scheme, in NumPy -- TEST
INFRASTRUCTURE ONLY (only ``tests/`` imports it).

A tiny, independent restatement of the explicit step of arXiv:1903.09043,
Sec. 2, used on grids of at most 16 x 16 cells to cross-check the C oracle
(``ark_oracle.c``): two writings of one specification.  It shares no code with
the C oracle or with the CUDA library.  Where the C oracle evaluates every
ghost cell through a recursive per-cell rule, this writing fills whole
padded arrays of primitives, x ghosts on the interior rows first and then y
ghosts over the x-extended rows, and forms every face and cell quantity as
array expressions.

What it covers: 2D, uniform gravity along y (Phi = -g y at the centres,
ghosts included), the Noble-Abel stiffened-gas equation of state (covolume b
and p_inf; b = p_inf = 0 is the ideal gas of Sec. 4), both energy variables (Sec. 2 and Appendix B), every boundary
rule (periodic, reflective hydrostatic wall, no-slip fixed-temperature wall,
outflow), the low-Mach correction on and off, and the first-order viscous
and heat fluxes of Sec. 2.2.  The readings of the paper are the same as the C
oracle's: unsplit multi-D sums, a = K max(rho c), dissipative fluxes from
U^n in the same update with the physical heat-flux sign, the two-point and
averaged-tangential viscous stencil, upwind tie u* = 0 to the left, wall
ghosts from the discrete balance of Eq. 18.
"""
from __future__ import annotations

import numpy as np

PERIODIC, REFLECT, NOSLIP, OUTFLOW = 0, 1, 2, 3
G = 2   # ghost layers


def _eos_prims(prob, rho, mx, my, W, phi):
    """Primitives of conserved values (equation of state, Sec. 1 Eq. 6 with
    the stiffened gas of p_inf): u, v, p, T, c."""
    u, v = mx / rho, my / rho
    rho_e = W - 0.5 * rho * (u * u + v * v) - (rho * phi if prob.energy_form == 0 else 0.0)
    p = (prob.gamma - 1.0) * rho_e / (1.0 - prob.b * rho) - prob.gamma * prob.p_inf
    return u, v, p


def _pad_prims(prob, U):
    """Ghost-padded arrays (ny + 4, nx + 4) of rho, u, v, p and Phi."""
    nx, ny = prob.n[0], prob.n[1]
    dy = (prob.hi[1] - prob.lo[1]) / ny
    rows = prob.lo[1] + (np.arange(-G, ny + G) + 0.5) * dy
    phi = np.broadcast_to((-prob.g * rows)[:, None], (ny + 2 * G, nx + 2 * G)).copy()
    Q = {k: np.zeros((ny + 2 * G, nx + 2 * G)) for k in ("rho", "u", "v", "p")}
    inner = (slice(G, G + ny), slice(G, G + nx))
    rho = U[0]
    u, v, p = _eos_prims(prob, rho, U[1], U[2], U[3], phi[inner])
    Q["rho"][inner], Q["u"][inner], Q["v"][inner], Q["p"][inner] = rho, u, v, p
    _fill_axis(prob, Q, phi, axis=1, rows=slice(G, G + ny))   # x ghosts on the interior rows
    _fill_axis(prob, Q, phi, axis=0, rows=slice(None))         # y ghosts on the x-extended rows
    return Q, phi


def _fill_axis(prob, Q, phi, axis, rows):
    """Ghost layers of one axis of the padded arrays (axis 1: x columns,
    axis 0: y rows); ``rows`` restricts the other axis."""
    d = 0 if axis == 1 else 1          # direction of the normal velocity
    n = prob.n[d]
    normal = "u" if d == 0 else "v"
    pinf = prob.p_inf

    def take(k, idx):
        a = Q[k] if k != "phi" else phi
        return a[rows, idx] if axis == 1 else a[idx, :]

    def put(k, idx, val):
        if axis == 1:
            Q[k][rows, idx] = val
        else:
            Q[k][idx, :] = val

    for side in (0, 1):
        bc = (prob.bc_lo if side == 0 else prob.bc_hi)[d]
        Tw = (prob.T_lo if side == 0 else prob.T_hi)[d]
        for layer in (1, 2):
            g = G - layer if side == 0 else G + n - 1 + layer       # ghost index
            if bc == PERIODIC:
                src = g + n if side == 0 else g - n
                for k in Q:
                    put(k, g, take(k, src))
                continue
            if bc == OUTFLOW:
                src = G if side == 0 else G + n - 1
                for k in Q:
                    put(k, g, take(k, src))
                continue
            mirror = G + layer - 1 if side == 0 else G + n - layer
            inner = g + 1 if side == 0 else g - 1                   # neighbour toward the interior
            rho_m, p_m = take("rho", mirror), take("p", mirror)
            T_m = (p_m + pinf) * (1.0 - prob.b * rho_m) / rho_m
            uu, vv = take("u", mirror), take("v", mirror)
            if bc == REFLECT:
                Tg = T_m
                uu, vv = (-uu, vv) if normal == "u" else (uu, -vv)
            else:
                Tg = 2.0 * Tw - T_m
                uu, vv = -uu, -vv
            dphi = take("phi", g) - take("phi", inner)
            K = take("p", inner) + pinf - 0.5 * take("rho", inner) * dphi
            if prob.b == 0.0:
                qg = K / (1.0 + dphi / (2.0 * Tg))
            else:   # rho_g = q_g / (T_g + b q_g): the balance is a quadratic in q_g
                Bq = Tg - prob.b * K + 0.5 * dphi
                qg = 2.0 * K * Tg / (Bq + np.sqrt(Bq * Bq + 4.0 * prob.b * K * Tg))
            put("rho", g, qg / (Tg + prob.b * qg))
            put("p", g, qg - pinf)
            put("u", g, uu)
            put("v", g, vv)


def _faces(prob, Q, phi, axis):
    """Acoustic face values between neighbours along ``axis`` of the padded
    arrays (Sec. 2.1.2; theta of Eq. 16): a, S, u*, Pi*."""
    sl_L = (slice(None), slice(0, -1)) if axis == 1 else (slice(0, -1), slice(None))
    sl_R = (slice(None), slice(1, None)) if axis == 1 else (slice(1, None), slice(None))
    un = Q["u"] if axis == 1 else Q["v"]
    rho, p = Q["rho"], Q["p"]
    c = np.sqrt(prob.gamma * (p + prob.p_inf) / (rho * (1.0 - prob.b * rho)))
    a = prob.K * np.maximum(rho[sl_L] * c[sl_L], rho[sl_R] * c[sl_R])
    S = -0.5 * (rho[sl_L] + rho[sl_R]) * (phi[sl_R] - phi[sl_L])
    us = 0.5 * (un[sl_L] + un[sl_R]) - (p[sl_R] - p[sl_L] - S) / (2.0 * a)
    if prob.low_mach:
        theta = np.minimum(np.abs(us) / np.maximum(c[sl_L], c[sl_R]), 1.0)
    else:
        theta = np.ones_like(us)
    Pi = 0.5 * (p[sl_L] + p[sl_R]) - 0.5 * a * theta * (un[sl_R] - un[sl_L])
    return us, Pi, S


def step(prob, U, dt):
    """U^{n+1} of a 2D state U (fields rho, m_x, m_y, energy; shape (4, ny, nx))."""
    assert prob.dim == 2 and getattr(prob, "phi", None) is None
    nx, ny = prob.n[0], prob.n[1]
    dx = (prob.hi[0] - prob.lo[0]) / nx
    dy = (prob.hi[1] - prob.lo[1]) / ny
    lx, ly = dt / dx, dt / dy
    Q, phi = _pad_prims(prob, U)
    rho, u, v, p = Q["rho"], Q["u"], Q["v"], Q["p"]
    # conserved values of every padded cell (ghosts from their primitives)
    mx, my = rho * u, rho * v
    W = (p + prob.gamma * prob.p_inf) * (1.0 - prob.b * rho) / (prob.gamma - 1.0) + 0.5 * rho * (u * u + v * v)
    if prob.energy_form == 0:
        W = W + rho * phi
    usx, Pix, Sx = _faces(prob, Q, phi, axis=1)   # (ny+4, nx+3): face between columns i, i+1
    usy, Piy, Sy = _faces(prob, Q, phi, axis=0)   # (ny+3, nx+4)

    # acoustic step: L~ and tilde states on the interior plus one ghost layer
    # (padded rows / columns 1 .. n + 2); the faces of cell (j, i) are
    # x: [j, i - 1] (low) and [j, i] (high), y: [j - 1, i] and [j, i]
    J = slice(1, ny + 3)
    I_ = slice(1, nx + 3)
    Jm, Im = slice(0, ny + 2), slice(0, nx + 2)
    xp = (J, I_)           # high x face of the cells (j, i) in J x I_
    xm = (J, Im)
    yp = (J, I_)
    ym = (Jm, I_)
    ell = lx * (usx[xp] - usx[xm]) + ly * (usy[yp] - usy[ym])
    Lt = 1.0 + ell
    m_t = mx[J, I_] - lx * (Pix[xp] - Pix[xm]) + lx * 0.5 * (Sx[xp] + Sx[xm])
    n_t = my[J, I_] - ly * (Piy[yp] - Piy[ym]) + ly * 0.5 * (Sy[yp] + Sy[ym])
    W_t = W[J, I_] - lx * (Pix[xp] * usx[xp] - Pix[xm] * usx[xm]) - ly * (Piy[yp] * usy[yp] - Piy[ym] * usy[ym])
    if prob.energy_form == 1:   # Appendix B: the gravity work of the acoustic step
        W_t = W_t + lx * 0.5 * (usx[xp] * Sx[xp] + usx[xm] * Sx[xm]) + ly * 0.5 * (usy[yp] * Sy[yp] + usy[ym] * Sy[ym])
    tilde = np.stack([rho[J, I_], m_t, n_t, W_t]) / Lt      # indices shifted by one: tilde[:, j-1, i-1]

    # transport step (Sec. 2.1.3) on the interior: upwind b~ on u*, tie to the left
    jj, ii = slice(1, ny + 1), slice(1, nx + 1)             # interior in tilde indexing
    bt = tilde[:, jj, ii]
    out = bt.copy()
    fx = usx[G:G + ny, G - 1:G + nx]                        # x faces left of interior cell i, .. right of the last
    fy = usy[G - 1:G + ny, G:G + nx]
    tx = tilde[:, jj, 0:nx + 2]                              # interior rows, columns -1 .. nx
    ty = tilde[:, 0:ny + 2, ii]
    upx = np.where(fx >= 0.0, tx[:, :, :-1], tx[:, :, 1:])  # upwind value at each x face
    upy = np.where(fy >= 0.0, ty[:, :-1, :], ty[:, 1:, :])
    Fx, Fy = upx * fx, upy * fy
    out -= lx * (Fx[:, :, 1:] - Fx[:, :, :-1]) + ly * (Fy[:, 1:, :] - Fy[:, :-1, :])
    out += bt * (lx * (fx[:, 1:] - fx[:, :-1]) + ly * (fy[1:, :] - fy[:-1, :]))

    # first-order dissipative fluxes (Sec. 2.2) from U^n
    if prob.mu != 0.0 or prob.kappa != 0.0:
        mu, eta = prob.mu, -2.0 / 3.0 * prob.mu
        T = (p + prob.p_inf) * (1.0 - prob.b * rho) / rho
        for axis in (1, 0):
            dn, dt_ = (dx, dy) if axis == 1 else (dy, dx)
            # normal (n) and tangential (t) velocity components for this face direction
            un_, ut_ = (u, v) if axis == 1 else (v, u)
            if axis == 1:   # faces between columns c, c + 1 over the interior rows, c = G-1 .. G+nx-1
                L = lambda a, s=0: a[G + s:G + ny + s, G - 1:G + nx]
                R = lambda a, s=0: a[G + s:G + ny + s, G:G + nx + 1]
            else:           # faces between rows r, r + 1 over the interior columns
                L = lambda a, s=0: a[G - 1:G + ny, G + s:G + nx + s]
                R = lambda a, s=0: a[G:G + ny + 1, G + s:G + nx + s]
            dnn = (R(un_) - L(un_)) / dn      # d u_n / d n
            dnt = (R(ut_) - L(ut_)) / dn      # d u_t / d n
            dtn = 0.25 * ((L(un_, 1) - L(un_, -1)) + (R(un_, 1) - R(un_, -1))) / dt_   # d u_n / d t
            dtt = 0.25 * ((L(ut_, 1) - L(ut_, -1)) + (R(ut_, 1) - R(ut_, -1))) / dt_   # d u_t / d t
            tau_nn = 2.0 * mu * dnn + eta * (dnn + dtt)
            tau_nt = mu * (dtn + dnt)
            work = tau_nn * 0.5 * (L(un_) + R(un_)) + tau_nt * 0.5 * (L(ut_) + R(ut_))
            heat = prob.kappa * (R(T) - L(T)) / dn
            lam = dt / dn
            if axis == 1:
                out[1] += lam * (tau_nn[:, 1:] - tau_nn[:, :-1])
                out[2] += lam * (tau_nt[:, 1:] - tau_nt[:, :-1])
                out[3] += lam * ((work + heat)[:, 1:] - (work + heat)[:, :-1])
            else:
                out[2] += lam * (tau_nn[1:, :] - tau_nn[:-1, :])
                out[1] += lam * (tau_nt[1:, :] - tau_nt[:-1, :])
                out[3] += lam * ((work + heat)[1:, :] - (work + heat)[:-1, :])
    return out
