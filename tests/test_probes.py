"""Host probes of the shock-vortex interaction (Sec. III.C): interpolation, vortex
centre and radial sound pressure on synthetic fields with known answers."""
import math

import numpy as np
import pytest

from paper_2102_09512_gb300 import cases as C
from paper_2102_09512_gb300 import probes as PR


def test_bilinear_is_exact_on_linear_fields():
    y, x = np.mgrid[0:20, 0:30].astype(np.float64)
    f = 0.3 * x - 1.7 * y + 2.0
    px = np.array([0.0, 3.25, 17.5, 28.9])
    py = np.array([0.0, 11.75, 2.5, 18.2])
    assert np.allclose(PR.bilinear(f, px, py), 0.3 * px - 1.7 * py + 2.0, atol=1e-12)


def test_vortex_centre_of_the_isentropic_vortex():
    """The vorticity extremum of the set-up's vortex is its centre, also off the grid
    points (centre shifted by a fraction of a node)."""
    c = C.isentropic_vortex(L=64, U0=0.2, Ma_v=0.25, r_v=5.0)
    u = c.u[:, 0]
    x, y = PR.vortex_centre(u, (30, 34), 8)
    assert abs(x - 32.0) < 0.05 and abs(y - 32.0) < 0.05
    c2 = C.shock_vortex(nx=160, ny=96, r_v=6.0, Ma_s=1.2)
    x, y = PR.vortex_centre(c2.u[:, 0], (c2.extra["x_v"] + 3, c2.extra["y_v"] - 2), 8)
    assert abs(x - c2.extra["x_v"]) < 0.05 and abs(y - c2.extra["y_v"]) < 0.05


def test_radial_sound_pressure_along_the_ray():
    """On a radially symmetric pressure field the profile along any angle is that
    radial function; theta = -45 degrees walks towards +x, -y."""
    y, x = np.mgrid[0:101, 0:101].astype(np.float64)
    rr = np.hypot(x - 50.0, y - 50.0)
    P_s = 2.0
    T = np.full_like(rr, 0.5)
    rho = P_s * (1.0 + 0.01 * np.cos(0.3 * rr)) / T
    r = np.linspace(0.0, 40.0, 41)
    dp = PR.radial_sound_pressure(rho, T, (50.0, 50.0), -45.0, r, P_s)
    assert np.allclose(dp, 0.01 * np.cos(0.3 * r), atol=2e-4)   # bilinear error only
    # the ray at -45 degrees passes through (50 + 10/sqrt 2, 50 - 10/sqrt 2)
    marker = np.zeros_like(rr)
    marker[43, 57] = 1.0
    hit = PR.radial_sound_pressure(marker + 1.0, np.ones_like(rr), (50.0, 50.0), -45.0,
                                   np.array([7.0 * math.sqrt(2.0)]), 1.0)
    assert hit[0] == 1.0


def test_energy_spectrum_of_single_modes():
    """A Fourier mode of wavenumber (3, 4, 0) (|k| = 5) puts all its energy <u.u>/2 in
    shell 5; a uniform flow puts its energy in shell 0; the sum is <u.u>/2."""
    n = 16
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    u = np.zeros((3, n, n, n))
    u[2] = 0.3 * np.cos(2 * np.pi * (3 * x + 4 * y) / n + 0.7)
    u[0] = 0.1
    k, E = PR.energy_spectrum(u)
    assert k[5] == 5
    assert E[5] == pytest.approx(0.5 * np.mean(u[2] ** 2), rel=1e-12)
    assert E[0] == pytest.approx(0.5 * 0.01, rel=1e-12)
    assert E.sum() == pytest.approx(0.5 * np.mean((u ** 2).sum(0)), rel=1e-12)


def test_energy_spectrum_torch_matches_numpy():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    u = rng.standard_normal((3, 12, 12, 12))
    k1, E1 = PR.energy_spectrum(u)
    k2, E2 = PR.energy_spectrum(torch.as_tensor(u))
    assert np.array_equal(k1, k2)
    assert np.allclose(E1, E2, rtol=1e-12, atol=1e-15)
    assert E1.sum() == pytest.approx(0.5 * np.mean((u ** 2).sum(0)), rel=1e-12)
