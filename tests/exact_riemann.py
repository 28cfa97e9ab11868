"""Exact solution of the 1D Euler Riemann problem for an ideal gas.

Test-only helper, written from the textbook equations (E. F. Toro, "Riemann
Solvers and Numerical Methods for Fluid Dynamics", ch. 4: the pressure
function f_K(p), shock and rarefaction branches, and the self-similar
sampling).  It shares nothing with the oracle's two-shock Newton solver and is
used to pin it.
"""
import numpy as np


def _fK(p, rho, pK, g):
    A = 2.0 / ((g + 1.0) * rho)
    B = (g - 1.0) / (g + 1.0) * pK
    c = np.sqrt(g * pK / rho)
    if p > pK:  # shock
        f = (p - pK) * np.sqrt(A / (p + B))
        df = np.sqrt(A / (B + p)) * (1.0 - 0.5 * (p - pK) / (B + p))
    else:  # rarefaction
        f = 2.0 * c / (g - 1.0) * ((p / pK) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * c) * (p / pK) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star(rl, ul, pl, rr, ur, pr, g=1.4):
    """Star pressure and velocity by Newton on f_L + f_R + du = 0 (to 1e-15)."""
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _fK(p, rl, pl, g)
        fr, dfr = _fK(p, rr, pr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, 1e-14)
        if abs(pn - p) <= 1e-15 * pn:
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, g)
    fr, _ = _fK(p, rr, pr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, rl, ul, pl, rr, ur, pr, g=1.4):
    """Exact (rho, u, p) at similarity coordinate xi = x/t."""
    ps, us = star(rl, ul, pl, rr, ur, pr, g)
    cl = np.sqrt(g * pl / rl); cr = np.sqrt(g * pr / rr)
    gm = (g - 1.0) / (g + 1.0)
    if xi <= us:  # left of contact
        if ps > pl:
            rs = rl * (ps / pl + gm) / (gm * ps / pl + 1.0)
            S = ul - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
            return (rl, ul, pl) if xi <= S else (rs, us, ps)
        rs = rl * (ps / pl) ** (1.0 / g)
        cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
        sh, st = ul - cl, us - cs
        if xi <= sh:
            return (rl, ul, pl)
        if xi >= st:
            return (rs, us, ps)
        u = 2.0 / (g + 1) * (cl + (g - 1) / 2 * ul + xi)
        c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (ul - xi))
        r = rl * (c / cl) ** (2.0 / (g - 1))
        return (r, u, pl * (c / cl) ** (2 * g / (g - 1)))
    if ps > pr:
        rs = rr * (ps / pr + gm) / (gm * ps / pr + 1.0)
        S = ur + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        return (rr, ur, pr) if xi >= S else (rs, us, ps)
    rs = rr * (ps / pr) ** (1.0 / g)
    cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
    sh, st = ur + cr, us + cs
    if xi >= sh:
        return (rr, ur, pr)
    if xi <= st:
        return (rs, us, ps)
    u = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * ur + xi)
    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (ur - xi))
    r = rr * (c / cr) ** (2.0 / (g - 1))
    return (r, u, pr * (c / cr) ** (2 * g / (g - 1)))
