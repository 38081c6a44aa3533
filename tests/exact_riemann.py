"""Exact solution of the Riemann problem for the 1D Euler equations of an ideal
gas (textbook two-rarefaction/two-shock construction: pressure function
f_L(p) + f_R(p) + (u_R - u_L) = 0 for the star pressure, then sampling x/t).

Used as an independent pin for the coarse Rusanov solver and for the Euler
limit of the kinetic solver (monoatomic gas, gamma = 5/3, Eq. 5 with d_v = 3).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq


def _fk(p, rho, pk, gamma):
    c = math.sqrt(gamma * pk / rho)
    if p > pk:
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        return (p - pk) * math.sqrt(A / (p + B))
    return 2.0 * c / (gamma - 1.0) * ((p / pk) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)


def star_state(left, right, gamma):
    rl, ul, pl = left
    rr, ur, pr = right

    def F(p):
        return _fk(p, rl, pl, gamma) + _fk(p, rr, pr, gamma) + (ur - ul)

    lo, hi = 1e-12, 10.0 * max(pl, pr) + 10.0
    while F(hi) < 0:
        hi *= 2.0
    ps = brentq(F, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    us = 0.5 * (ul + ur) + 0.5 * (_fk(ps, rr, pr, gamma) - _fk(ps, rl, pl, gamma))
    return ps, us


def sample(left, right, gamma, s):
    """Return (rho, u, p) at similarity coordinate s = (x - x0)/t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    if s <= us:  # left of the contact
        cl = math.sqrt(gamma * pl / rl)
        if ps > pl:  # left shock
            sl = ul - cl * math.sqrt((gamma + 1) / (2 * gamma) * ps / pl + (gamma - 1) / (2 * gamma))
            if s <= sl:
                return rl, ul, pl
            rho = rl * (ps / pl + g1) / (g1 * ps / pl + 1.0)
            return rho, us, ps
        # left rarefaction
        rho_s = rl * (ps / pl) ** (1.0 / gamma)
        cs = cl * (ps / pl) ** ((gamma - 1) / (2 * gamma))
        head, tail = ul - cl, us - cs
        if s <= head:
            return rl, ul, pl
        if s >= tail:
            return rho_s, us, ps
        u = 2.0 / (gamma + 1) * (cl + (gamma - 1) / 2 * ul + s)
        c = 2.0 / (gamma + 1) * (cl + (gamma - 1) / 2 * (ul - s))
        rho = rl * (c / cl) ** (2.0 / (gamma - 1))
        return rho, u, pl * (c / cl) ** (2.0 * gamma / (gamma - 1))
    cr = math.sqrt(gamma * pr / rr)
    if ps > pr:  # right shock
        sr = ur + cr * math.sqrt((gamma + 1) / (2 * gamma) * ps / pr + (gamma - 1) / (2 * gamma))
        if s >= sr:
            return rr, ur, pr
        rho = rr * (ps / pr + g1) / (g1 * ps / pr + 1.0)
        return rho, us, ps
    rho_s = rr * (ps / pr) ** (1.0 / gamma)
    cs = cr * (ps / pr) ** ((gamma - 1) / (2 * gamma))
    head, tail = ur + cr, us + cs
    if s >= head:
        return rr, ur, pr
    if s <= tail:
        return rho_s, us, ps
    u = 2.0 / (gamma + 1) * (-cr + (gamma - 1) / 2 * ur + s)
    c = 2.0 / (gamma + 1) * (cr - (gamma - 1) / 2 * (ur - s))
    rho = rr * (c / cr) ** (2.0 / (gamma - 1))
    return rho, u, pr * (c / cr) ** (2.0 * gamma / (gamma - 1))


def density_profile(left, right, gamma, x, x0, t):
    return np.array([sample(left, right, gamma, (xi - x0) / t)[0] for xi in x])
