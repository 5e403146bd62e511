"""Exact Riemann solver of the 1-D Euler equations for a calorically perfect gas
(test infrastructure for the dry-flux pin of the oracle).

Godunov's exact solution: the star pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0,
with f_K the shock (Rankine-Hugoniot) or rarefaction (isentropic) branch of side K, by
Newton iteration from the two-rarefaction guess; the solution at x/t is then sampled from
the wave pattern.  Pinned by the textbook star states of Toro's tests (tests/golden/).
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    pr = p / pk
    f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(left, right, g=1.4, tol=1e-14):
    """(p*, u*) of the Riemann problem left=(rho, u, p), right=(rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, cl, g)
        fr, dfr = _fk(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, tol)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, g)
    fr, _ = _fk(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, xi, g=1.4):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t (array)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, g)
    cl, cr = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=float)
    out = np.zeros((3, xi.size))
    gm = (g - 1.0) / (g + 1.0)
    for n, s in enumerate(xi.ravel()):
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
                sl = ul - cl * math.sqrt((g + 1.0) / (2.0 * g) * ps / pl + (g - 1.0) / (2.0 * g))
                out[:, n] = (rl, ul, pl) if s <= sl else (rs, us, ps)
            else:  # left rarefaction
                rs = rl * (ps / pl) ** (1.0 / g)
                cs = cl * (ps / pl) ** ((g - 1.0) / (2.0 * g))
                sh, st = ul - cl, us - cs
                if s <= sh:
                    out[:, n] = (rl, ul, pl)
                elif s >= st:
                    out[:, n] = (rs, us, ps)
                else:
                    f = 2.0 / (g + 1.0) + (g - 1.0) / ((g + 1.0) * cl) * (ul - s)
                    rho = rl * f ** (2.0 / (g - 1.0))
                    u = 2.0 / (g + 1.0) * (cl + 0.5 * (g - 1.0) * ul + s)
                    out[:, n] = (rho, u, pl * f ** (2.0 * g / (g - 1.0)))
        else:  # right of contact
            if ps > pr:  # right shock
                rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
                sr = ur + cr * math.sqrt((g + 1.0) / (2.0 * g) * ps / pr + (g - 1.0) / (2.0 * g))
                out[:, n] = (rr, ur, pr) if s >= sr else (rs, us, ps)
            else:  # right rarefaction
                rs = rr * (ps / pr) ** (1.0 / g)
                cs = cr * (ps / pr) ** ((g - 1.0) / (2.0 * g))
                sh, st = ur + cr, us + cs
                if s >= sh:
                    out[:, n] = (rr, ur, pr)
                elif s <= st:
                    out[:, n] = (rs, us, ps)
                else:
                    f = 2.0 / (g + 1.0) - (g - 1.0) / ((g + 1.0) * cr) * (ur - s)
                    rho = rr * f ** (2.0 / (g - 1.0))
                    u = 2.0 / (g + 1.0) * (-cr + 0.5 * (g - 1.0) * ur + s)
                    out[:, n] = (rho, u, pr * f ** (2.0 * g / (g - 1.0)))
    return out
