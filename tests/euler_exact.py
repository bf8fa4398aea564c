"""Exact solution of the Riemann problem of the 1D Euler equations for a polytropic gas,
used to pin the oracle on the shock tubes of Sec. 5.6.

The star-region pressure p* solves f_L(p) + f_R(p) + (v_R - v_L) = 0, where f_K is the
shock (Rankine-Hugoniot) branch for p > p_K and the isentropic rarefaction branch
otherwise; v* follows from the same functions.  The solution at x / t is then read off
the wave pattern (left wave, contact, right wave).  This is the textbook construction
(Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics", ch. 4), written here
from its equations; nothing is shared with the oracle or the library.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import brentq


def _f(p, rho, pk, g):
    """Velocity jump across the wave that connects state K to pressure p."""
    c = np.sqrt(g * pk / rho)
    if p > pk:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        return (p - pk) * np.sqrt(A / (p + B))
    return 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)


def star_state(left, right, g=1.4):
    """(p*, v*, rho*_L, rho*_R) of the Riemann problem with primitive states (rho, v, p)."""
    rl, vl, pl = left
    rr, vr, pr = right
    fn = lambda p: _f(p, rl, pl, g) + _f(p, rr, pr, g) + (vr - vl)
    hi = max(pl, pr)
    while fn(hi) < 0:
        hi *= 2.0
    ps = brentq(fn, 1e-14, hi, xtol=1e-15, rtol=1e-15, maxiter=500)
    vs = 0.5 * (vl + vr) + 0.5 * (_f(ps, rr, pr, g) - _f(ps, rl, pl, g))

    def rho_star(rho, pk):
        if ps > pk:
            r = ps / pk
            k = (g - 1.0) / (g + 1.0)
            return rho * (r + k) / (k * r + 1.0)
        return rho * (ps / pk) ** (1.0 / g)

    return ps, vs, rho_star(rl, pl), rho_star(rr, pr)


def sample(left, right, xi, g=1.4):
    """Primitive (rho, v, p) arrays of the self-similar solution at xi = (x - x0) / t."""
    rl, vl, pl = left
    rr, vr, pr = right
    ps, vs, rsl, rsr = star_state(left, right, g)
    cl, cr = np.sqrt(g * pl / rl), np.sqrt(g * pr / rr)
    xi = np.asarray(xi, dtype=np.float64)
    out = np.zeros((3,) + xi.shape)
    for idx, s in np.ndenumerate(xi):
        if s <= vs:      # left of the contact
            if ps > pl:  # left shock
                S = vl - cl * np.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                st = (rl, vl, pl) if s <= S else (rsl, vs, ps)
            else:        # left rarefaction
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                head, tail = vl - cl, vs - csl
                if s <= head:
                    st = (rl, vl, pl)
                elif s >= tail:
                    st = (rsl, vs, ps)
                else:
                    v = 2.0 / (g + 1) * (cl + (g - 1) / 2 * vl + s)
                    c = 2.0 / (g + 1) * (cl + (g - 1) / 2 * (vl - s))
                    rho = rl * (c / cl) ** (2.0 / (g - 1))
                    st = (rho, v, pl * (c / cl) ** (2.0 * g / (g - 1)))
        else:
            if ps > pr:  # right shock
                S = vr + cr * np.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                st = (rr, vr, pr) if s >= S else (rsr, vs, ps)
            else:        # right rarefaction
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                head, tail = vr + cr, vs + csr
                if s >= head:
                    st = (rr, vr, pr)
                elif s <= tail:
                    st = (rsr, vs, ps)
                else:
                    v = 2.0 / (g + 1) * (-cr + (g - 1) / 2 * vr + s)
                    c = 2.0 / (g + 1) * (cr - (g - 1) / 2 * (vr - s))
                    rho = rr * (c / cr) ** (2.0 / (g - 1))
                    st = (rho, v, pr * (c / cr) ** (2.0 * g / (g - 1)))
        out[(slice(None),) + idx] = st
    return out


def conservative(prim, g=1.4):
    rho, v, p = prim
    return np.array([rho, rho * v, p / (g - 1.0) + 0.5 * rho * v * v])
