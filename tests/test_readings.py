"""CPU checks, in the FP64 oracle, of two readings where the configured parameters and
the paper part ways (readings R9 and R13 of the design notes):

- Sod tube (Sec. III.B) on 800 x 4 nodes: the configured mu = 1e-3 drives omega to
  about 1.99 at T = 0.12-0.15 and the run leaves the physical range within a few dozen
  steps; the paper's own mu = 0.015 stays physical over the configured 500 steps.
- Shock-vortex interaction (Sec. III.C): mu taken from Re = 800 on a scaled-down vortex
  radius (0.0026 at r_v = 8, 0.0053 at r_v = 16; 0.0106 at the configured r_v = 32)
  makes the initial standing shock diverge; the paper's viscosity, Re = 800 on its own
  r_v = 60 (mu = 0.0198), keeps it physical.  The oracle runs a reduced 256 x 128 grid
  (r_v = 8) here; the configured 1024 x 1024 grid (r_v = 32) is checked on the GPU in
  tests/test_gpu_shock_vortex.py and tests/test_gpu_parity.py.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from paper_2102_09512_gb300 import cases as C


def _params(c):
    return O.Params(D=c.D, nx=c.nx, ny=c.ny, nz=c.nz, gamma=c.gamma, Pr=c.Pr, mu0=c.mu0, T0=c.T0,
                    mu_exp=c.mu_exp, bc=c.bc, fixed=c.fixed, cv=c.cv)


def _physical_steps(c, nmax, every):
    """Steps (in multiples of `every`) until rho, u or T stops being finite or rho or T
    stops being positive; None if the state stays physical for nmax steps."""
    s = O.init(_params(c), c.rho, c.u, c.T)
    n = 0
    while n < nmax:
        O.step(s, every)
        n += every
        r, u, T = O.fields(s)
        if not (np.isfinite(r).all() and np.isfinite(u).all() and np.isfinite(T).all()
                and r.min() > 0.0 and T.min() > 0.0):
            return n
    return None


def test_sod_configured_viscosity_diverges():
    n = _physical_steps(C.sod(nx=800, ny=4, mu=1e-3), 150, 5)
    assert n is not None and n < 150


def test_sod_paper_viscosity_stays_physical():
    assert _physical_steps(C.sod(nx=800, ny=4, mu=0.015), 500, 50) is None


def test_shock_vortex_viscosity_from_scaled_radius_diverges():
    c = C.shock_vortex(nx=256, ny=128, r_v=8.0, r_v_mu=8.0)
    n = _physical_steps(c, 200, 25)
    assert n is not None and n <= 100


def test_shock_vortex_paper_viscosity_stays_physical():
    c = C.shock_vortex(nx=256, ny=128, r_v=8.0)
    assert abs(c.mu0 - 0.0198431) < 1e-6
    assert _physical_steps(c, 200, 50) is None
