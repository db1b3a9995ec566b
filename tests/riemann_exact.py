"""Exact solution of the ideal-gas Riemann problem (test helper).

Textbook method: Newton iteration on the pressure function
f(p) = f_L(p) + f_R(p) + (u_R - u_L) with the shock / rarefaction branches of
E. F. Toro, *Riemann Solvers and Numerical Methods for Fluid Dynamics*,
3rd ed., Ch. 4 (Secs. 4.2-4.5).  Used to pin the oracle's Sod results; it
shares nothing with the scheme under test.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        f = (p - pk) * s
        df = s * (1.0 - 0.5 * (p - pk) / (B + p))
    else:        # rarefaction
        f = 2.0 * ck / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * ck) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rhoL, uL, pL, rhoR, uR, pR, g):
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    p = max(1e-12, 0.5 * (pL + pR))
    for _ in range(100):
        fL, dL = _fk(p, rhoL, pL, cL, g)
        fR, dR = _fk(p, rhoR, pR, cR, g)
        f = fL + fR + (uR - uL)
        pn = max(1e-12, p - f / (dL + dR))
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _fk(p, rhoL, pL, cL, g)
    fR, _ = _fk(p, rhoR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(x, t, x0, left, right, g):
    """(rho, u, p) of the exact solution at positions x and time t > 0."""
    rhoL, uL, pL = left
    rhoR, uR, pR = right
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, g)
    cL = math.sqrt(g * pL / rhoL)
    cR = math.sqrt(g * pR / rhoR)
    gm = (g - 1.0) / (g + 1.0)
    out = np.zeros((3, len(x)))
    for i, xi in enumerate(x):
        S = (xi - x0) / t
        if S <= us:   # left of contact
            if ps > pL:   # left shock
                SL = uL - cL * math.sqrt((g + 1.0) / (2.0 * g) * ps / pL + (g - 1.0) / (2.0 * g))
                if S <= SL:
                    r, u, p = rhoL, uL, pL
                else:
                    r = rhoL * (ps / pL + gm) / (gm * ps / pL + 1.0)
                    u, p = us, ps
            else:         # left rarefaction
                csL = cL * (ps / pL) ** ((g - 1.0) / (2.0 * g))
                SHL, STL = uL - cL, us - csL
                if S <= SHL:
                    r, u, p = rhoL, uL, pL
                elif S >= STL:
                    r = rhoL * (ps / pL) ** (1.0 / g)
                    u, p = us, ps
                else:
                    u = 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * uL + S)
                    c = 2.0 / (g + 1.0) * (cL + (g - 1.0) / 2.0 * (uL - S))
                    r = rhoL * (c / cL) ** (2.0 / (g - 1.0))
                    p = pL * (c / cL) ** (2.0 * g / (g - 1.0))
        else:         # right of contact
            if ps > pR:   # right shock
                SR = uR + cR * math.sqrt((g + 1.0) / (2.0 * g) * ps / pR + (g - 1.0) / (2.0 * g))
                if S >= SR:
                    r, u, p = rhoR, uR, pR
                else:
                    r = rhoR * (ps / pR + gm) / (gm * ps / pR + 1.0)
                    u, p = us, ps
            else:         # right rarefaction
                csR = cR * (ps / pR) ** ((g - 1.0) / (2.0 * g))
                SHR, STR = uR + cR, us + csR
                if S >= SHR:
                    r, u, p = rhoR, uR, pR
                elif S <= STR:
                    r = rhoR * (ps / pR) ** (1.0 / g)
                    u, p = us, ps
                else:
                    u = 2.0 / (g + 1.0) * (-cR + (g - 1.0) / 2.0 * uR + S)
                    c = 2.0 / (g + 1.0) * (cR - (g - 1.0) / 2.0 * (uR - S))
                    r = rhoR * (c / cR) ** (2.0 / (g - 1.0))
                    p = pR * (c / cR) ** (2.0 * g / (g - 1.0))
        out[:, i] = (r, u, p)
    return out
