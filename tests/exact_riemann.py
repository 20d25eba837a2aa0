"""Exact solution of the 1-D Riemann problem for an ideal gas (independent
test helper used to pin the oracle's HLLC / MUSCL-Hancock path).

Pressure in the star region from the root of f(p) = f_L(p) + f_R(p) + du,
with the shock branch from the Rankine-Hugoniot conditions and the
rarefaction branch from the isentropic relations, solved by Newton's
method; the solution is then sampled along x/t.
"""
import math


def _f(p, rho, pk, ck, g):
    if p > pk:  # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    pr = p / pk
    return 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0), 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))


def star(rL, uL, pL, rR, uR, pR, g=1.4):
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    p = max(1e-8, 0.5 * (pL + pR))
    for _ in range(100):
        fL, dL = _f(p, rL, pL, cL, g)
        fR, dR = _f(p, rR, pR, cR, g)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(1e-12, p - dp)
        if abs(pn - p) < 1e-14 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _f(p, rL, pL, cL, g)
    fR, _ = _f(p, rR, pR, cR, g)
    u = 0.5 * (uL + uR) + 0.5 * (fR - fL)
    return p, u


def sample(rL, uL, pL, rR, uR, pR, s, g=1.4):
    """(rho, u, p) at similarity coordinate s = x/t."""
    ps, us = star(rL, uL, pL, rR, uR, pR, g)
    cL, cR = math.sqrt(g * pL / rL), math.sqrt(g * pR / rR)
    if s <= us:
        if ps > pL:
            SL = uL - cL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
            if s <= SL:
                return rL, uL, pL
            return rL * ((ps / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pL + 1)), us, ps
        cs = cL * (ps / pL) ** ((g - 1) / (2 * g))
        if s <= uL - cL:
            return rL, uL, pL
        if s >= us - cs:
            return rL * (ps / pL) ** (1 / g), us, ps
        u = 2 / (g + 1) * (cL + (g - 1) / 2 * uL + s)
        c = 2 / (g + 1) * (cL + (g - 1) / 2 * (uL - s))
        r = rL * (c / cL) ** (2 / (g - 1))
        return r, u, pL * (c / cL) ** (2 * g / (g - 1))
    if ps > pR:
        SR = uR + cR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
        if s >= SR:
            return rR, uR, pR
        return rR * ((ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1)), us, ps
    cs = cR * (ps / pR) ** ((g - 1) / (2 * g))
    if s >= uR + cR:
        return rR, uR, pR
    if s <= us + cs:
        return rR * (ps / pR) ** (1 / g), us, ps
    u = 2 / (g + 1) * (-cR + (g - 1) / 2 * uR + s)
    c = 2 / (g + 1) * (cR - (g - 1) / 2 * (uR - s))
    r = rR * (c / cR) ** (2 / (g - 1))
    return r, u, pR * (c / cR) ** (2 * g / (g - 1))
