"""Exact solution of the one-dimensional Riemann problem for the Euler
equations of an ideal gas.

TEST INFRASTRUCTURE: the reference solution for the shock-tube check of the
oracle (the paper compares its shock tube with the analytical solution,
Sec. 5.2).  Written from the standard construction: the star pressure is the
root of f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is the shock
(Rankine-Hugoniot) branch for p > p_K and the rarefaction (isentropic,
Riemann invariant) branch otherwise; the root is found by Newton iteration,
then the self-similar solution is sampled at xi = (x - x0) / t.
"""
from __future__ import annotations

import math

import numpy as np


def _f_and_df(p, rho, pk, ck, gamma):
    if p > pk:  # shock branch
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction branch
    e = (gamma - 1.0) / (2.0 * gamma)
    f = 2.0 * ck / (gamma - 1.0) * ((p / pk) ** e - 1.0)
    df = (1.0 / (rho * ck)) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma))
    return f, df


def star_state(left, right, gamma=1.4, tol=1e-14, maxit=100):
    """(p*, u*, rho*_L, rho*_R) for left/right states (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    p = max(tol, 0.5 * (pl + pr))
    for _ in range(maxit):
        fl, dfl = _f_and_df(p, rl, pl, cl, gamma)
        fr, dfr = _f_and_df(p, rr, pr, cr, gamma)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(pn, tol)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, cl, gamma)
    fr, _ = _f_and_df(p, rr, pr, cr, gamma)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    if p > pl:
        rsl = rl * (p / pl + g1) / (g1 * p / pl + 1.0)
    else:
        rsl = rl * (p / pl) ** (1.0 / gamma)
    if p > pr:
        rsr = rr * (p / pr + g1) / (g1 * p / pr + 1.0)
    else:
        rsr = rr * (p / pr) ** (1.0 / gamma)
    return p, u, rsl, rsr


def sample(left, right, xi, gamma=1.4):
    """rho, u, p of the self-similar solution at the points xi = (x - x0) / t."""
    rl, ul, pl = left
    rr, ur, pr = right
    cl, cr = math.sqrt(gamma * pl / rl), math.sqrt(gamma * pr / rr)
    ps, us, rsl, rsr = star_state(left, right, gamma)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi); u = np.empty_like(xi); p = np.empty_like(xi)
    gm1, gp1 = gamma - 1.0, gamma + 1.0
    for k, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pl:
                sl = ul - cl * math.sqrt(gp1 / (2 * gamma) * ps / pl + gm1 / (2 * gamma))
                st = (rl, ul, pl) if s <= sl else (rsl, us, ps)
            else:
                csl = cl * (ps / pl) ** (gm1 / (2 * gamma))
                head, tail = ul - cl, us - csl
                if s <= head:
                    st = (rl, ul, pl)
                elif s >= tail:
                    st = (rsl, us, ps)
                else:
                    uu = 2.0 / gp1 * (cl + 0.5 * gm1 * ul + s)
                    cc = 2.0 / gp1 * (cl + 0.5 * gm1 * (ul - s))
                    rr_ = rl * (cc / cl) ** (2.0 / gm1)
                    st = (rr_, uu, pl * (cc / cl) ** (2.0 * gamma / gm1))
        else:  # right of the contact
            if ps > pr:
                sr = ur + cr * math.sqrt(gp1 / (2 * gamma) * ps / pr + gm1 / (2 * gamma))
                st = (rr, ur, pr) if s >= sr else (rsr, us, ps)
            else:
                csr = cr * (ps / pr) ** (gm1 / (2 * gamma))
                head, tail = ur + cr, us + csr
                if s >= head:
                    st = (rr, ur, pr)
                elif s <= tail:
                    st = (rsr, us, ps)
                else:
                    uu = 2.0 / gp1 * (-cr + 0.5 * gm1 * ur + s)
                    cc = 2.0 / gp1 * (cr - 0.5 * gm1 * (ur - s))
                    rr_ = rr * (cc / cr) ** (2.0 / gm1)
                    st = (rr_, uu, pr * (cc / cr) ** (2.0 * gamma / gm1))
        rho[k], u[k], p[k] = st
    return rho, u, p
