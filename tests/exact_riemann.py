"""Exact solution of the Riemann problem for the 1-D Euler equations of an ideal
gas (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
3rd ed., ch. 4: pressure function, Newton iteration for p*, wave sampling).

Independent of the oracle: it is the textbook solution that pins the oracle's
reconstruction + HLLE + RK2 on the Sod shock tube.
"""
from __future__ import annotations

import math

import numpy as np


def _fk(p, rho, pk, ck, gamma):
    """Toro's f_K(p) and its derivative."""
    if p > pk:  # shock
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction
    e = (gamma - 1.0) / (2.0 * gamma)
    return (2.0 * ck / (gamma - 1.0)) * ((p / pk) ** e - 1.0), (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)) / (rho * ck)


def star_state(left, right, gamma):
    """(p*, u*) for left/right primitive states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr))
    for _ in range(100):
        fl, dfl = _fk(p, rl, pl, cl, gamma)
        fr, dfr = _fk(p, rr, pr, cr, gamma)
        f = fl + fr + (ur - ul)
        pn = max(1e-14, p - f / (dfl + dfr))
        if abs(pn - p) <= 1e-14 * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fk(p, rl, pl, cl, gamma)
    fr, _ = _fk(p, rr, pr, cr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(left, right, gamma, xi):
    """Primitive state (rho, u, p) at similarity coordinate xi = x/t (arrays)."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(left, right, gamma)
    cl = math.sqrt(gamma * pl / rl)
    cr = math.sqrt(gamma * pr / rr)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for n, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pl + (gamma - 1.0) / (2.0 * gamma))
                if s <= sl:
                    rho[n], u[n], p[n] = rl, ul, pl
                else:
                    rho[n] = rl * ((ps / pl + g1) / (g1 * ps / pl + 1.0))
                    u[n], p[n] = us, ps
            else:  # left rarefaction
                shl = ul - cl
                cml = cl * (ps / pl) ** ((gamma - 1.0) / (2.0 * gamma))
                stl = us - cml
                if s <= shl:
                    rho[n], u[n], p[n] = rl, ul, pl
                elif s >= stl:
                    rho[n] = rl * (ps / pl) ** (1.0 / gamma)
                    u[n], p[n] = us, ps
                else:
                    c = 2.0 / (gamma + 1.0) + g1 / cl * (ul - s)
                    rho[n] = rl * c ** (2.0 / (gamma - 1.0))
                    u[n] = 2.0 / (gamma + 1.0) * (cl + (gamma - 1.0) / 2.0 * ul + s)
                    p[n] = pl * c ** (2.0 * gamma / (gamma - 1.0))
        else:  # right of the contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((gamma + 1.0) / (2.0 * gamma) * ps / pr + (gamma - 1.0) / (2.0 * gamma))
                if s >= sr:
                    rho[n], u[n], p[n] = rr, ur, pr
                else:
                    rho[n] = rr * ((ps / pr + g1) / (g1 * ps / pr + 1.0))
                    u[n], p[n] = us, ps
            else:  # right rarefaction
                shr = ur + cr
                cmr = cr * (ps / pr) ** ((gamma - 1.0) / (2.0 * gamma))
                str_ = us + cmr
                if s >= shr:
                    rho[n], u[n], p[n] = rr, ur, pr
                elif s <= str_:
                    rho[n] = rr * (ps / pr) ** (1.0 / gamma)
                    u[n], p[n] = us, ps
                else:
                    c = 2.0 / (gamma + 1.0) - g1 / cr * (ur - s)
                    rho[n] = rr * c ** (2.0 / (gamma - 1.0))
                    u[n] = 2.0 / (gamma + 1.0) * (-cr + (gamma - 1.0) / 2.0 * ur + s)
                    p[n] = pr * c ** (2.0 * gamma / (gamma - 1.0))
    return rho, u, p
