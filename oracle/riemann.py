"""Exact solution of the one-dimensional Riemann problem of an ideal gas, the
analytic reference of the Sod shock tube (CRK-HACC Sec. 4, the Sod test).

TEST INFRASTRUCTURE ONLY: imported by tests/ and the bench's Sod report,
never by the product path.

The solution is the textbook one for the Euler equations (e.g. E. F. Toro,
Riemann Solvers and Numerical Methods for Fluid Dynamics, ch. 4): the star
pressure p* solves f_L(p) + f_R(p) + (u_R - u_L) = 0 with, for side K,
  a shock (p > p_K):       f_K = (p - p_K) sqrt(A_K / (p + B_K)),
                           A_K = 2 / ((gamma+1) rho_K), B_K = (gamma-1)/(gamma+1) p_K,
  a rarefaction (p <= p_K): f_K = 2 c_K/(gamma-1) ((p/p_K)^((gamma-1)/(2 gamma)) - 1),
u* = (u_L + u_R)/2 + (f_R(p*) - f_L(p*))/2, and the self-similar profile is
sampled at xi = (x - x0)/t: left state, left wave (shock or fan), left star
state, contact at u*, right star state, right wave, right state.
"""
import numpy as np


def _f(p, rho, pK, c, g):
    if p > pK:
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pK
        q = np.sqrt(A / (p + B))
        return (p - pK) * q, q * (1.0 - 0.5 * (p - pK) / (B + p))
    r = p / pK
    return (2.0 * c / (g - 1.0) * (r ** ((g - 1.0) / (2.0 * g)) - 1.0),
            r ** (-(g + 1.0) / (2.0 * g)) / (rho * c))


def star(left, right, gamma=5.0 / 3.0, tol=1e-15):
    """(p*, u*) of left = (rho, u, p), right = (rho, u, p)."""
    (rL, uL, pL), (rR, uR, pR) = left, right
    cL, cR = np.sqrt(gamma * pL / rL), np.sqrt(gamma * pR / rR)
    if 2.0 * (cL + cR) / (gamma - 1.0) <= uR - uL:
        raise ValueError("the states produce a vacuum")
    p = max(0.5 * (pL + pR), 1e-12)
    for _ in range(200):
        fL, dL = _f(p, rL, pL, cL, gamma)
        fR, dR = _f(p, rR, pR, cR, gamma)
        dp = (fL + fR + uR - uL) / (dL + dR)
        pn = max(p - dp, 1e-3 * p)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fL, _ = _f(p, rL, pL, cL, gamma)
    fR, _ = _f(p, rR, pR, cR, gamma)
    return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)


def sample(xi, left, right, gamma=5.0 / 3.0):
    """Density, velocity and pressure of the self-similar solution at
    xi = (x - x0)/t (array); left/right = (rho, u, p)."""
    g = gamma
    (rL, uL, pL), (rR, uR, pR) = left, right
    ps, us = star(left, right, g)
    cL, cR = np.sqrt(g * pL / rL), np.sqrt(g * pR / rR)
    xi = np.asarray(xi, np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    gm = (g - 1.0) / (g + 1.0)
    for side, (rK, uK, pK, cK, s) in (("L", (rL, uL, pL, cL, -1.0)), ("R", (rR, uR, pR, cR, 1.0))):
        m = (xi < us) if side == "L" else (xi >= us)
        x = xi[m]
        if ps > pK:   # shock: speed from the mass flux, star density from the Hugoniot
            S = uK + s * cK * np.sqrt((g + 1.0) / (2.0 * g) * ps / pK + (g - 1.0) / (2.0 * g))
            rs = rK * (ps / pK + gm) / (gm * ps / pK + 1.0)
            out = (x < S) if side == "L" else (x > S)
            rho[m] = np.where(out, rK, rs)
            u[m] = np.where(out, uK, us)
            p[m] = np.where(out, pK, ps)
        else:         # rarefaction: isentropic fan between head and tail
            rs = rK * (ps / pK) ** (1.0 / g)
            cs = cK * (ps / pK) ** ((g - 1.0) / (2.0 * g))
            head, tail = uK + s * cK, us + s * cs
            out = (x < head) if side == "L" else (x > head)
            inner = (x > tail) if side == "L" else (x < tail)
            # inside the fan: u - s c = x, with u + s 2c/(g-1) the Riemann invariant of the far state
            uf = 2.0 / (g + 1.0) * (-s * cK + (g - 1.0) / 2.0 * uK + x)
            cf = -s * (uf - x)
            rf = rK * (cf / cK) ** (2.0 / (g - 1.0))
            pf = pK * (cf / cK) ** (2.0 * g / (g - 1.0))
            rho[m] = np.where(out, rK, np.where(inner, rs, rf))
            u[m] = np.where(out, uK, np.where(inner, us, uf))
            p[m] = np.where(out, pK, np.where(inner, ps, pf))
    return rho, u, p
