"""Post-processing probes on fields extracted from a solver (lattice units): the
shock-vortex interaction (paper Sec. III.C) and the energy spectrum of decaying
turbulence (Sec. III.D).

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


def energy_spectrum(u) -> tuple:
    """Shell-summed kinetic energy spectrum E(k) of a periodic (3, n, n, n) velocity
    field (numpy or torch; torch tensors are transformed on their device):
    E(k) = sum over integer shells |k| in [k - 1/2, k + 1/2) of |u_hat|^2 / 2, with
    u_hat the FFT normalised by n^3, so that sum_k E(k) = <u.u>/2.  Returns (k, E)
    as numpy arrays over every shell, k = 0 .. round(sqrt(3) n/2) (shells above n/2 are
    only partly inside the transform's cube)."""
    n = u.shape[-1]
    nk = int(round(math.sqrt(3.0) * (n // 2))) + 1
    try:
        import torch
        is_torch = isinstance(u, torch.Tensor)
    except ImportError:
        is_torch = False
    kk = np.fft.fftfreq(n, d=1.0 / n)
    kr = np.fft.rfftfreq(n, d=1.0 / n)
    if is_torch:
        dev = u.device
        kz = torch.as_tensor(kk, device=dev).view(n, 1, 1)
        ky = torch.as_tensor(kk, device=dev).view(1, n, 1)
        kx = torch.as_tensor(kr, device=dev).view(1, 1, -1)
        shell = torch.round(torch.sqrt(kx * kx + ky * ky + kz * kz)).long()
        # the half-spectrum counts every k_x > 0 (except the Nyquist plane) twice
        wgt = torch.full((1, 1, kr.size), 2.0, device=dev, dtype=torch.float64)
        wgt[..., 0] = 1.0
        if n % 2 == 0:
            wgt[..., -1] = 1.0
        E = torch.zeros(nk, dtype=torch.float64, device=dev)
        for a in range(3):
            uh = torch.fft.rfftn(u[a].to(torch.float64), dim=(0, 1, 2)) / float(n) ** 3
            e = 0.5 * (uh.real ** 2 + uh.imag ** 2) * wgt
            E.index_add_(0, shell.reshape(-1), e.reshape(-1))
            del uh, e
        E = E.cpu().numpy()
    else:
        kz, ky, kx = np.meshgrid(kk, kk, kr, indexing="ij")
        shell = np.rint(np.sqrt(kx * kx + ky * ky + kz * kz)).astype(np.int64)
        wgt = np.full(kr.size, 2.0)
        wgt[0] = 1.0
        if n % 2 == 0:
            wgt[-1] = 1.0
        E = np.zeros(nk)
        for a in range(3):
            uh = np.fft.rfftn(np.asarray(u[a], dtype=np.float64)) / float(n) ** 3
            np.add.at(E, shell.ravel(), (0.5 * np.abs(uh) ** 2 * wgt).ravel())
    return np.arange(nk), E
