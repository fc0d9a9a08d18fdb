"""Runs of the paper's Sec. III test cases through the solver, returning the
diagnostics the paper plots (histories, spectra, probe profiles).  Thin drivers:
every time step runs in the CUDA kernels; the diagnostics come from the device
statistics (elbm_turbulence_stats) and the host probes (probes.py).

  decaying_turbulence   Sec. III.D: K, dissipation <mu omega^2>, Re_lambda, theta_rms,
                        rho_rms, Ma_t histories against t* = t u_rms,0 / L_I, and energy
                        spectra (on the device with torch.fft).
  shock_vortex_sound    Sec. III.C: vortex track and radial sound pressure Delta P
                        along theta from the vortex centre at t* = t c_s,l / r_v.
  precision_study       reduced-precision population stores (FP32, FP16 and BF16
                        deviations) against a GPU FP64 run of the same decaying-turbulence
                        field: relative L2 errors of rho, u, T and statistics drift.
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


def _rel_l2(a, b) -> float:
    import torch
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def precision_study(n: int = 256, steps: int = 100, stores=("f32", "f16dev", "bf16dev"), every: int = 10,
                    survive: int = 0, seed: int = 20210218, k0: float = 4.0, Ma_t: float = 0.5,
                    Re_lambda: float = 72.0) -> dict:
    """The decaying-turbulence field of Sec. III.D on an n^3 periodic D3Q27 box (the
    bench workload at n = 256) run with the FP64 store and with each store in
    `stores`.  For every store, after `steps` steps: the relative L2 error of rho, u
    (all components) and T against the FP64 run, the same for the fluctuations
    rho - <rho> and T - <T> (the plain metric is lenient because of the means), and the
    K(t) and theta_rms(t) histories (sampled every `every` steps) with their relative
    deviation from FP64's; the largest deviation is taken over t > 0 (the initial
    dilatation is near zero, so its relative deviation says nothing).  Every run then
    continues to `survive` steps (if larger) and reports the last sample at which its
    state was still physical.  Errors are computed on the device."""
    import torch

    c = C.hit(n, seed=seed, k0=k0, Ma_t=Ma_t, Re_lambda=Re_lambda, dtype=np.float32 if n > 256 else np.float64)
    N = n ** 3
    dev = torch.device("cuda")
    t_end = max(steps, survive)

    def run(store):
        g = E.Solver.from_case(c, store=store)
        hist, t, wall, fields, last_ok = [], 0, 0.0, None, 0
        try:
            while True:
                s = g.turbulence_stats()   # synchronises; raises if the state is non-physical
                last_ok = t
                hist.append((t, s["K"], s["theta_rms"]))
                if t == steps:
                    rho = torch.empty(N, dtype=torch.float64, device=dev)
                    u = torch.empty(3 * N, dtype=torch.float64, device=dev)
                    T = torch.empty(N, dtype=torch.float64, device=dev)
                    g.fields_device(rho, u, T)
                    g.sync()
                    fields = (rho, u, T)
                if t >= t_end:
                    break
                k = min(every, (steps if t < steps else t_end) - t)
                t0 = time.perf_counter()
                g.step(k)
                g.sync()
                wall += time.perf_counter() - t0
                t += k
        except E.ElbmError:
            pass
        finally:
            g.close()
            del g
            torch.cuda.empty_cache()
        return dict(hist=np.array(hist), fields=fields, physical_to=last_ok, s_per_step=wall / max(t, 1))

    ref = run("f64")
    if ref["fields"] is None:
        raise RuntimeError(f"the FP64 run turned non-physical before step {steps} (last physical: "
                           f"{ref['physical_to']})")
    r_rho, r_u, r_T = ref["fields"]
    hr = ref["hist"]
    out = {"n": n, "steps": steps, "mu0": c.mu0, "every": every,
           "f64": {"s_per_step": ref["s_per_step"], "physical_to": ref["physical_to"],
                   "K": hr[:, 1].tolist(), "theta_rms": hr[:, 2].tolist()}}
    for store in stores:
        r = run(store)
        e = {"s_per_step": r["s_per_step"], "physical_to": r["physical_to"]}
        if r["fields"] is not None:
            rho, u, T = r["fields"]
            e.update(rho=_rel_l2(rho, r_rho), u=_rel_l2(u, r_u), T=_rel_l2(T, r_T),
                     rho_fluct=_rel_l2(rho - rho.mean(), r_rho - r_rho.mean()),
                     T_fluct=_rel_l2(T - T.mean(), r_T - r_T.mean()))
            m = min(len(r["hist"]), len(hr))
            h = r["hist"][:m]
            dK = np.abs(h[:, 1] - hr[:m, 1]) / hr[:m, 1]
            dth = np.abs(h[:, 2] - hr[:m, 2]) / hr[:m, 2]
            upto = h[:, 0] <= steps
            e["K_dev"] = dK.tolist()
            e["theta_dev"] = dth.tolist()
            e["K_drift"] = float(np.max(dK[1:][upto[1:]])) if m > 1 else 0.0
            e["theta_drift"] = float(np.max(dth[1:][upto[1:]])) if m > 1 else 0.0
            del rho, u, T
        r["fields"] = None
        torch.cuda.empty_cache()
        out[store] = e
    return out


def _turbulence_report(out: dict, fit=(6, 16)) -> dict:
    """Histories of a decaying_turbulence run relative to their initial values, and the
    spectral slope fitted over integer shells fit[0] .. fit[1] at each spectrum time."""
    h = out["hist"]
    K0 = h[0]["K"]
    rows = [dict(t_star=s["t_star"], K_over_K0=s["K"] / K0, dissipation=s["dissipation"],
                 Re_lambda=s["Re_lambda"], theta_rms=s["theta_rms"], rho_rms=s["rho_rms"], Ma_t=s["Ma_t"])
            for s in h]
    slopes = {}
    for ts, (k, Ek) in out["spectra"].items():
        sel = (k >= fit[0]) & (k <= fit[1]) & (Ek > 0)
        slopes[ts] = float(np.polyfit(np.log(k[sel]), np.log(Ek[sel]), 1)[0])
        peak = int(k[1:][np.argmax(Ek[1:])])
        slopes[f"peak_shell_t{ts}"] = peak
    return dict(n=out["n"], tau_steps=out["tau"], steps=out["steps"], step_seconds=out["step_seconds"],
                mu0=out["mu0"], glups=out["n"] ** 3 * out["steps"] / max(out["step_seconds"], 1e-9) / 1e9,
                history=rows, spectral_slopes=slopes, fit_shells=list(fit))


if __name__ == "__main__":
    # python -m paper_2102_09512_gb300.studies decaying_turbulence N [out.json]
    #   decaying compressible turbulence on an N^3 box (Sec. III.D; N = 768 is the paper's
    #   Re_lambda = 175, Ma_t = 0.488 run), FP32 store, statistics every tau/4 to t* = 3,
    #   spectra at t* = 0, 1, 3; prints (and writes) the histories and spectral slopes.
    import json
    import sys

    if len(sys.argv) < 3 or sys.argv[1] != "decaying_turbulence":
        raise SystemExit("usage: python -m paper_2102_09512_gb300.studies decaying_turbulence N [out.json]")
    rep = _turbulence_report(decaying_turbulence(n=int(sys.argv[2])))
    txt = json.dumps(rep, indent=1)
    print(txt)
    if len(sys.argv) > 3:
        with open(sys.argv[3], "w") as fh:
            fh.write(txt)
