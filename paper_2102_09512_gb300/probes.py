"""Post-processing probes of the shock-vortex interaction (paper Sec. III.C) on
fields extracted from a solver (host numpy arrays, lattice units).

The sound pressure is Delta P = (P - P_s) / P_s with P = rho T (R = 1) and P_s the
pressure behind the shock; it is read along a ray from the vortex centre at an angle
theta (the paper uses theta = -45 degrees at t* = t c_s,l / r_v = 6, 8, 10).
"""
from __future__ import annotations

import math

import numpy as np


def bilinear(field: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Bilinear interpolation of a (ny, nx) node field at points (x, y); points are
    clamped to the grid."""
    ny, nx = field.shape
    x = np.clip(np.asarray(x, dtype=np.float64), 0.0, nx - 1.0)
    y = np.clip(np.asarray(y, dtype=np.float64), 0.0, ny - 1.0)
    x0 = np.minimum(np.floor(x).astype(np.int64), nx - 2)
    y0 = np.minimum(np.floor(y).astype(np.int64), ny - 2)
    fx, fy = x - x0, y - y0
    return ((1 - fx) * (1 - fy) * field[y0, x0] + fx * (1 - fy) * field[y0, x0 + 1]
            + (1 - fx) * fy * field[y0 + 1, x0] + fx * fy * field[y0 + 1, x0 + 1])


def vorticity(u: np.ndarray) -> np.ndarray:
    """omega_z = d u_y / d x - d u_x / d y of a (2, ny, nx) velocity field by central
    differences (one-sided at the edges)."""
    return np.gradient(u[1], axis=1) - np.gradient(u[0], axis=0)


def vortex_centre(u: np.ndarray, guess, half_width: int) -> tuple:
    """Centre of the vortex core near `guess` = (x, y): the extremum of the vorticity
    magnitude in a square window, refined by a parabola through its axis neighbours."""
    w = np.abs(vorticity(u))
    ny, nx = w.shape
    gx, gy = int(round(guess[0])), int(round(guess[1]))
    xa, xb = max(1, gx - half_width), min(nx - 1, gx + half_width + 1)
    ya, yb = max(1, gy - half_width), min(ny - 1, gy + half_width + 1)
    win = w[ya:yb, xa:xb]
    j, i = np.unravel_index(int(np.argmax(win)), win.shape)
    x, y = xa + i, ya + j

    def vertex(m, c, p):
        d = m - 2.0 * c + p
        return 0.0 if d == 0.0 else 0.5 * (m - p) / d

    return (x + vertex(w[y, x - 1], w[y, x], w[y, x + 1]), y + vertex(w[y - 1, x], w[y, x], w[y + 1, x]))


def radial_sound_pressure(rho: np.ndarray, T: np.ndarray, centre, theta_deg: float, r: np.ndarray,
                          P_s: float) -> np.ndarray:
    """Delta P = (rho T - P_s) / P_s at distances r from `centre` along the angle
    theta (degrees, counter-clockwise from +x; y grows with the row index)."""
    th = math.radians(theta_deg)
    x = centre[0] + np.asarray(r) * math.cos(th)
    y = centre[1] + np.asarray(r) * math.sin(th)
    return (bilinear(rho * T, x, y) - P_s) / P_s
