"""Exact solution of the Riemann problem of the 1D Euler equations for an ideal gas
(the textbook construction: pressure functions for shock / rarefaction branches,
bisection for the star pressure, then sampling in x/t).  Used as the
reference for the Sod shock tube (paper Sec. III.B)."""
from __future__ import annotations

import math

import numpy as np


def star_state(rho_l, u_l, p_l, rho_r, u_r, p_r, gamma=1.4, tol=1e-14):
    """(p*, u*, rho*_L, rho*_R) of the exact solution."""
    c_l = math.sqrt(gamma * p_l / rho_l)
    c_r = math.sqrt(gamma * p_r / rho_r)

    def f(p, rho_k, p_k, c_k):
        if p > p_k:
            A = 2.0 / ((gamma + 1.0) * rho_k)
            B = (gamma - 1.0) / (gamma + 1.0) * p_k
            return (p - p_k) * math.sqrt(A / (p + B))
        return 2.0 * c_k / (gamma - 1.0) * ((p / p_k) ** ((gamma - 1.0) / (2.0 * gamma)) - 1.0)

    def F(p):
        return f(p, rho_l, p_l, c_l) + f(p, rho_r, p_r, c_r) + (u_r - u_l)

    # bracket and bisect-polish (robust and plenty fast for a test)
    lo, hi = 1e-12, max(p_l, p_r) * 10.0
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if F(mid) > 0.0:
            hi = mid
        else:
            lo = mid
        if hi - lo < tol * max(1.0, mid):
            break
    p = 0.5 * (lo + hi)
    u = 0.5 * (u_l + u_r) + 0.5 * (f(p, rho_r, p_r, c_r) - f(p, rho_l, p_l, c_l))
    g1 = (gamma - 1.0) / (gamma + 1.0)

    def rho_star(rho_k, p_k):
        if p > p_k:
            return rho_k * (p / p_k + g1) / (g1 * p / p_k + 1.0)
        return rho_k * (p / p_k) ** (1.0 / gamma)

    return p, u, rho_star(rho_l, p_l), rho_star(rho_r, p_r)


def sample(xi, rho_l, u_l, p_l, rho_r, u_r, p_r, gamma=1.4):
    """(rho, u, p) at similarity coordinates xi = (x - x0)/t (array)."""
    ps, us, rl, rr = star_state(rho_l, u_l, p_l, rho_r, u_r, p_r, gamma)
    c_l = math.sqrt(gamma * p_l / rho_l)
    c_r = math.sqrt(gamma * p_r / rho_r)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    g1 = (gamma - 1.0) / (gamma + 1.0)
    for k, s in enumerate(xi.ravel()):
        if s <= us:  # left of contact
            if ps > p_l:  # left shock
                S = u_l - c_l * math.sqrt((gamma + 1) / (2 * gamma) * ps / p_l + (gamma - 1) / (2 * gamma))
                st = (rl, us, ps) if s >= S else (rho_l, u_l, p_l)
            else:  # left rarefaction
                c_s = c_l * (ps / p_l) ** ((gamma - 1) / (2 * gamma))
                head, tail = u_l - c_l, us - c_s
                if s <= head:
                    st = (rho_l, u_l, p_l)
                elif s >= tail:
                    st = (rl, us, ps)
                else:
                    fac = 2 / (gamma + 1) + g1 / c_l * (u_l - s)
                    st = (rho_l * fac ** (2 / (gamma - 1)),
                          2 / (gamma + 1) * (c_l + (gamma - 1) / 2 * u_l + s),
                          p_l * fac ** (2 * gamma / (gamma - 1)))
        else:
            if ps > p_r:  # right shock
                S = u_r + c_r * math.sqrt((gamma + 1) / (2 * gamma) * ps / p_r + (gamma - 1) / (2 * gamma))
                st = (rr, us, ps) if s <= S else (rho_r, u_r, p_r)
            else:
                c_s = c_r * (ps / p_r) ** ((gamma - 1) / (2 * gamma))
                head, tail = u_r + c_r, us + c_s
                if s >= head:
                    st = (rho_r, u_r, p_r)
                elif s <= tail:
                    st = (rr, us, ps)
                else:
                    fac = 2 / (gamma + 1) - g1 / c_r * (u_r - s)
                    st = (rho_r * fac ** (2 / (gamma - 1)),
                          2 / (gamma + 1) * (-c_r + (gamma - 1) / 2 * u_r + s),
                          p_r * fac ** (2 * gamma / (gamma - 1)))
        rho.ravel()[k], u.ravel()[k], p.ravel()[k] = st
    return rho, u, p
