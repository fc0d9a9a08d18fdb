"""Runs of the paper's Sec. III test cases through the solver, returning the
diagnostics the paper plots (histories, spectra, probe profiles).  Thin drivers:
every time step runs in the CUDA kernels; the diagnostics come from the device
statistics (elbm_turbulence_stats) and the host probes (probes.py).

  decaying_turbulence   Sec. III.D: K, dissipation <mu omega^2>, Re_lambda, theta_rms,
                        rho_rms, Ma_t histories against t* = t u_rms,0 / L_I, and energy
                        spectra (on the device with torch.fft).
  shock_vortex_sound    Sec. III.C: vortex track and radial sound pressure Delta P
                        along theta from the vortex centre at t* = t c_s,l / r_v.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import cases as C
from . import elbm as E
from . import probes as PR


def decaying_turbulence(n: int = 768, Ma_t: float = 0.488, Re_lambda: float = 175.0, k0: float = 4.0,
                        store: str = "f32", t_end: float = 3.0, samples_per_tau: int = 4,
                        spectra_at=(0.0, 1.0, 3.0), deriv: int = 0, seed: int = 20210218) -> dict:
    """Decaying compressible turbulence on an n^3 periodic D3Q27 box (Sec. III.D; the
    paper's high-Reynolds run is n = 768, Ma_t = 0.488, Re_lambda = 175, kappa_0 = 4).
    tau = L_I / u_rms,0 with L_I = sqrt(2 pi)/kappa_0 (in lattice units n / (kappa_0
    sqrt(2 pi))).  Statistics every tau / samples_per_tau; spectra at the sample
    closest to each requested t*."""
    import torch

    c = C.hit(n, seed=seed, k0=k0, Ma_t=Ma_t, Re_lambda=Re_lambda, dtype=np.float32 if n > 256 else np.float64)
    u_rms0 = c.extra["u_rms"]
    tau = n / (k0 * math.sqrt(2.0 * math.pi)) / u_rms0
    dt = max(1, int(round(tau / samples_per_tau)))
    g = E.Solver.from_case(c, store=store, deriv=deriv)
    c.rho = c.u = c.T = None   # the host copy is not needed any more
    hist, spectra = [], {}

    def spectrum():
        dev = torch.device("cuda")
        rho = torch.empty(n ** 3, dtype=torch.float64, device=dev)
        u = torch.empty(3 * n ** 3, dtype=torch.float64, device=dev)
        T = torch.empty(n ** 3, dtype=torch.float64, device=dev)
        g.fields_device(rho, u, T)
        del rho, T
        k, Ek = PR.energy_spectrum(u.view(3, n, n, n))
        del u
        torch.cuda.empty_cache()
        return k, Ek

    want = sorted(spectra_at)
    t, wall = 0, 0.0
    try:
        while True:
            s = g.turbulence_stats()
            ts = t / tau
            s["t_star"] = ts
            s["Ma_t"] = math.sqrt(3.0) * s["u_rms"] / math.sqrt(c.gamma * s["T_mean"])
            hist.append(s)
            while want and ts >= want[0] - 0.5 / samples_per_tau:
                spectra[want.pop(0)] = spectrum()
            if ts >= t_end - 0.5 * dt / tau:   # the sample nearest to t_end
                break
            t0 = time.perf_counter()
            g.step(dt)
            g.sync()
            wall += time.perf_counter() - t0
            t += dt
    finally:
        g.close()
    return dict(n=n, tau=tau, dt=dt, steps=t, step_seconds=wall, hist=hist, spectra=spectra, mu0=c.mu0)


def shock_vortex_sound(nx: int = 1680, ny: int = 1440, r_v: float = 60.0, Ma_s: float = 1.2,
                       Ma_v: float = 0.25, times=(6.0, 8.0, 10.0), theta_deg: float = -45.0,
                       store: str = "f64", r_max: float = 8.0) -> dict:
    """Shock-vortex interaction with a supersonic inflow on -x (Sec. III.C; the paper's
    run is the default).  At each t* the vortex centre (vorticity extremum near the
    position advected at u_l to the shock and u_s behind it) and Delta P along
    theta_deg out to r_max r_v."""
    c = C.shock_vortex(nx, ny, r_v=r_v, Ma_s=Ma_s, Ma_v=Ma_v, inflow=True)
    rv, cs, P_s, u_s, u_l = c.extra["r_v"], c.extra["cs_l"], c.extra["P_s"], c.extra["u_s"], c.fixed[1]
    xv, yv, xs = c.extra["x_v"], c.extra["y_v"], c.extra["x_s"]
    t_hit = (xs - xv) / u_l
    r = np.arange(0.0, r_max * rv + 0.5, 1.0)
    g = E.Solver.from_case(c, store=store)
    out, t = {}, 0
    try:
        for ts in times:
            steps = int(round(ts * rv / cs))
            g.step(steps - t)
            t = steps
            rho, u, T = g.fields()
            rho, T, u = rho.reshape(ny, nx), T.reshape(ny, nx), u.reshape(2, ny, nx)
            pred = (xv + u_l * t if t < t_hit else xs + u_s * (t - t_hit), yv)
            centre = PR.vortex_centre(u, pred, int(1.5 * rv))
            out[ts] = dict(steps=steps, predicted=pred, centre=centre, r_over_rv=r / rv,
                           delta_p=PR.radial_sound_pressure(rho, T, centre, theta_deg, r, P_s))
    finally:
        g.close()
    return dict(case=c.extra, results=out)
