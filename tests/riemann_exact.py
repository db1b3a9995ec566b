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


def sample_covolume(x, t, x0, left, right, g, p_inf=0.0, b=0.0):
    """(rho, u, p) of the exact Riemann solution for the Noble-Abel stiffened
    gas, rho e = (p + g p_inf)(1 - b rho)/(g - 1), c^2 = g (p + p_inf)/(rho (1 - b rho)).

    In the variables pi = p + p_inf and v' = 1/rho - b the energy, the
    Hugoniot, the isentropes pi v'^g = const and the Riemann invariants are
    those of an ideal gas of density rho' = 1/v' (the covolume gas of Toro,
    Ch. 4.7, shifted as the stiffened gas of Ivings, Causon and Toro), so the
    star pressure and velocity are the ideal solver's.  Wave speeds use the
    real specific volume: a shock moves at u_K -+ m v_K (m the mass flux), a
    characteristic at u -+ c with c = c' (1 + b rho'), c' = sqrt(g pi / rho');
    inside a fan the state solves u -+ c = x / t on the invariant, by bisection."""
    def mapped(state):
        r, u, p = state
        rp = r / (1.0 - b * r)
        return rp, u, p + p_inf

    rL, uL, qL = mapped(left)
    rR, uR, qR = mapped(right)
    qs, us = star_state(rL, uL, qL, rR, uR, qR, g)
    gm = (g - 1.0) / (g + 1.0)

    def real(rp, u, q):
        return rp / (1.0 + b * rp), u, q - p_inf

    def cp(rp, q):
        return math.sqrt(g * q / rp)

    def side(S, rK, uK, qK, sgn):
        """sgn = -1: left wave family; +1: right."""
        cK = cp(rK, qK)
        if qs > qK:   # shock
            rs = rK * (qs / qK + gm) / (gm * qs / qK + 1.0)
            m = math.sqrt((qs - qK) / (1.0 / rK - 1.0 / rs))
            vK = 1.0 / rK + b
            SK = uK + sgn * m * vK
            if (S - SK) * sgn >= 0.0:
                return real(rK, uK, qK)
            return real(rs, us, qs)
        rs = rK * (qs / qK) ** (1.0 / g)
        head = uK + sgn * cK * (1.0 + b * rK)
        tail = us + sgn * cp(rs, qs) * (1.0 + b * rs)
        if (S - head) * sgn >= 0.0:
            return real(rK, uK, qK)
        if (S - tail) * sgn <= 0.0:
            return real(rs, us, qs)
        # inside the fan: u = uK + sgn 2 (c'(rho') - cK) / (g - 1), u + sgn c = S
        def resid(rp):
            c1 = cK * (rp / rK) ** ((g - 1.0) / 2.0)
            u = uK + sgn * 2.0 * (c1 - cK) / (g - 1.0)
            return u + sgn * c1 * (1.0 + b * rp) - S
        lo_r, hi_r = min(rs, rK), max(rs, rK)
        f_lo = resid(lo_r)
        for _ in range(200):
            mid = 0.5 * (lo_r + hi_r)
            fm = resid(mid)
            if (fm > 0) == (f_lo > 0):
                lo_r, f_lo = mid, fm
            else:
                hi_r = mid
        rp = 0.5 * (lo_r + hi_r)
        c1 = cK * (rp / rK) ** ((g - 1.0) / 2.0)
        u = uK + sgn * 2.0 * (c1 - cK) / (g - 1.0)
        q = qK * (rp / rK) ** g
        return real(rp, u, q)

    out = np.zeros((3, len(x)))
    for i, xi in enumerate(x):
        S = (xi - x0) / t
        out[:, i] = side(S, rL, uL, qL, -1.0) if S <= us else side(S, rR, uR, qR, 1.0)
    return out
