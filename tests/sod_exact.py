"""Exact solution of the Riemann problem for the 1D Euler equations (ideal gas).

Textbook construction (pressure function + Newton iteration for the star
pressure, then sampling of the self-similar fan), used to pin the oracle's
finite-volume Euler scheme on the Sod shock tube.  Test helper only.
"""
import math

import numpy as np


def _fk(p, rho, pk, gamma):
    """Pressure function of one side and its derivative."""
    c = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    f = 2.0 * c / (gamma - 1.0) * ((p / pk) ** e - 1.0)
    df = 1.0 / (rho * c) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma=1.4):
    rl, ul, pl = left
    rr, ur, pr = right
    p = 0.5 * (pl + pr)
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, gamma)
        fr, dfr = _fk(p, rr, pr, gamma)
        f = fl + fr + (ur - ul)
        dp = f / (dfl + dfr)
        p_new = max(p - dp, 1e-12)
        if abs(p_new - p) < 1e-15 * (p_new + p):
            p = p_new
            break
        p = p_new
    fl, _ = _fk(p, rl, pl, gamma)
    fr, _ = _fk(p, rr, pr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(xi, left, right, gamma=1.4):
    """(rho, u, p) at similarity coordinate xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    g = gamma
    if xi <= us:  # left of contact
        cl = math.sqrt(g * pl / rl)
        if ps > pl:  # left shock
            sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
            if xi <= sl:
                return rl, ul, pl
            r = rl * ((ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1))
            return r, us, ps
        # left rarefaction
        cs = cl * (ps / pl) ** ((g - 1) / (2 * g))
        head, tail = ul - cl, us - cs
        if xi <= head:
            return rl, ul, pl
        if xi >= tail:
            return rl * (ps / pl) ** (1 / g), us, ps
        u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + xi)
        c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - xi))
        r = rl * (c / cl) ** (2 / (g - 1))
        return r, u, pl * (c / cl) ** (2 * g / (g - 1))
    # right of contact
    cr = math.sqrt(g * pr / rr)
    if ps > pr:  # right shock
        sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
        if xi >= sr:
            return rr, ur, pr
        r = rr * ((ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1))
        return r, us, ps
    cs = cr * (ps / pr) ** ((g - 1) / (2 * g))
    head, tail = ur + cr, us + cs
    if xi >= head:
        return rr, ur, pr
    if xi <= tail:
        return rr * (ps / pr) ** (1 / g), us, ps
    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + xi)
    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - xi))
    r = rr * (c / cr) ** (2 / (g - 1))
    return r, u, pr * (c / cr) ** (2 * g / (g - 1))


def sod_density(x, t, x0=0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1), gamma=1.4):
    return np.array([sample((xx - x0) / t, left, right, gamma)[0] for xx in x])
