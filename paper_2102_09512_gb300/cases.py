"""Seeded synthetic initial conditions (rho, u, T) for the model's workloads.

This module holds only problem set-ups: no step of the lattice Boltzmann method
itself.  Both the CUDA path and the FP64 oracle are fed from here, so it must stay
free of the method's arithmetic (equilibria, moments, collision, streaming).

Array conventions: ``rho`` and ``T`` are float64 arrays of shape ``(nz, ny, nx)``
(``nz = 1`` in 2D), ``u`` is ``(D, nz, ny, nx)``.  Flattened in C order they give
node index ``n = x + nx*(y + ny*z)``.  Lattice units throughout: dx = dt = 1, R = 1.

Set-ups (paper Sec. III):
  - :func:`sod`           Sod shock tube (Sec. III.B)
  - :func:`shock_vortex`  Rankine-Hugoniot standing shock + isentropic vortex (Sec. III.C)
  - :func:`hit`           solenoidal random field with E(k) ~ k^4 exp(-2 (k/k0)^2)
                          (Sec. III.D), with mu0 from Re_lambda
  - :func:`ensemble`      uneven 2D instances (Sod / shock-vortex mix)
  - :func:`isentropic_vortex`  vortex carried by a uniform flow (translation pin)
  - :func:`shear_wave`, :func:`sound_wave`, :func:`thermal_wave`, :func:`random_smooth`
                          small-amplitude and random fields for tests
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Case:
    """Initial fields plus the physical parameters that go with them."""
    name: str
    D: int
    nx: int
    ny: int
    nz: int
    rho: np.ndarray = field(repr=False)
    u: np.ndarray = field(repr=False)
    T: np.ndarray = field(repr=False)
    gamma: float = 1.4
    Pr: float = 0.71
    mu0: float = 1e-3
    T0: float = 0.15
    mu_exp: float = 0.0
    bc: tuple = (0, 0, 0, 0, 0, 0)      # per face -x,+x,-y,+y,-z,+z: 0 periodic, 1 zero-gradient, 2 fixed
    extra: dict = field(default_factory=dict)
    fixed: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)   # (rho, u_x, u_y, u_z, T) of the fixed-state faces
    cv: tuple = None   # None: Cv = 1/(gamma-1); else Cv(T) = cv[0] + cv[1] T + cv[2] T^2 + cv[3] T^3

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz


def _empty(D, nx, ny, nz):
    shape = (nz, ny, nx)
    return np.zeros(shape), np.zeros((D,) + shape), np.zeros(shape)


def sod(nx: int = 800, ny: int = 4, rho_l: float = 1.0, T_l: float = 0.15,
        rho_r: float = 0.125, T_r: float = 0.12, gamma: float = 1.4, Pr: float = 0.71,
        mu: float = 0.015) -> Case:
    """Sod shock tube on D2Q9: left (x < nx/2) rho_l, T_l; right rho_r, T_r; u = 0.
    Pressures P = rho T give 0.15 | 0.015 (ratio 10).  y periodic, x zero-gradient.
    mu defaults to the paper's 0.015 (mu = 1e-3 diverges within ~100 steps)."""
    rho, u, T = _empty(2, nx, ny, 1)
    left = np.arange(nx) < nx // 2
    rho[..., left] = rho_l
    rho[..., ~left] = rho_r
    T[..., left] = T_l
    T[..., ~left] = T_r
    return Case("sod", 2, nx, ny, 1, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu, T0=T_l,
                bc=(1, 1, 0, 0, 0, 0))


def rankine_hugoniot(Ma: float, gamma: float = 1.4):
    """Normal-shock jump ratios (rho2/rho1, p2/p1, T2/T1, u2/u1) for upstream Mach Ma."""
    M2 = Ma * Ma
    r = (gamma + 1.0) * M2 / ((gamma - 1.0) * M2 + 2.0)
    pr = 1.0 + 2.0 * gamma / (gamma + 1.0) * (M2 - 1.0)
    return r, pr, pr / r, 1.0 / r


def shock_vortex(nx: int = 1024, ny: int = 1024, Ma_s: float = 1.2, Ma_v: float = 0.25,
                 r_v: float = 32.0, Re: float = 800.0, Pr: float = 0.75, gamma: float = 1.4,
                 T_l: float = 0.05, rho_l: float = 1.0, r_v_mu: float = 60.0,
                 inflow: bool = False) -> Case:
    """Standing normal shock at x_s = 8 r_v (left state rho_l, T_l, u = Ma_s sqrt(gamma T_l),
    right state by Rankine-Hugoniot) with an isentropic vortex of Mach Ma_v and radius
    r_v centred at (6 r_v, ny/2) superposed on the local base state.
    mu = rho_l c_s,l r_v_mu / Re: by default the viscosity of the paper's run (r_v = 60,
    Re = 800) is kept when the domain is scaled down; a smaller mu (e.g. Re = 800 on
    r_v = 32) makes the initial shock diverge within a few hundred steps.
    y periodic; x zero-gradient, or with inflow=True the -x face holds the upstream
    state fixed (a supersonic inflow) and +x stays zero-gradient.  The paper's run is
    shock_vortex(1680, 1440, r_v=60, inflow=True) (Sec. III.C)."""
    rho, u, T = _empty(2, nx, ny, 1)
    cs_l = math.sqrt(gamma * T_l)
    ux_l = Ma_s * cs_l
    r_rho, r_p, r_T, r_u = rankine_hugoniot(Ma_s, gamma)
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    xs = 8.0 * r_v
    left = (x < xs)
    rho_inf = np.where(left, rho_l, rho_l * r_rho) * np.ones_like(y)
    P_inf = np.where(left, rho_l * T_l, rho_l * T_l * r_p) * np.ones_like(y)
    ux_inf = np.where(left, ux_l, ux_l * r_u) * np.ones_like(y)
    xv, yv = 6.0 * r_v, ny / 2.0
    r2 = ((x - xv) ** 2 + (y - yv) ** 2) / (r_v * r_v)
    base = 1.0 - 0.5 * (gamma - 1.0) * Ma_v * Ma_v * np.exp(1.0 - r2)
    rho2 = rho_inf * base ** (1.0 / (gamma - 1.0))
    P2 = P_inf * base ** (gamma / (gamma - 1.0))
    amp = cs_l * Ma_v * np.exp(0.5 * (1.0 - r2))
    ux = ux_inf + amp * (y - yv) / r_v
    uy = -amp * (x - xv) / r_v
    rho[0] = rho2
    T[0] = P2 / rho2
    u[0, 0] = ux
    u[1, 0] = uy
    mu = rho_l * cs_l * r_v_mu / Re
    return Case("shock_vortex", 2, nx, ny, 1, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu, T0=T_l,
                bc=(2 if inflow else 1, 1, 0, 0, 0, 0),
                extra=dict(Ma_s=Ma_s, Ma_v=Ma_v, r_v=r_v, Re=Re, x_s=xs, x_v=xv, y_v=yv, cs_l=cs_l,
                           P_s=rho_l * T_l * r_p, u_s=ux_l * r_u),
                fixed=(rho_l, ux_l, 0.0, 0.0, T_l))


def _rfftn(a: np.ndarray) -> np.ndarray:
    """Real 3D FFT, on all host cores when scipy is present (same transform as numpy's)."""
    try:
        import scipy.fft as sf
        return sf.rfftn(a, workers=-1)
    except ImportError:
        return np.fft.rfftn(a)


def _irfftn(a: np.ndarray, shape) -> np.ndarray:
    try:
        import scipy.fft as sf
        return sf.irfftn(a, s=shape, axes=(0, 1, 2), workers=-1)
    except ImportError:
        return np.fft.irfftn(a, s=shape, axes=(0, 1, 2))


def _central_dx(a: np.ndarray, axis: int) -> np.ndarray:
    return 0.5 * (np.roll(a, -1, axis=axis) - np.roll(a, 1, axis=axis))


def hit(n: int = 128, seed: int = 20210218, k0: float = 4.0, Ma_t: float = 0.5,
        Re_lambda: float = 72.0, T0: float = 0.15, gamma: float = 1.4, Pr: float = 0.7,
        rho0: float = 1.0, mu_exp: float = 0.76, dtype=np.float64) -> Case:
    """Decaying-turbulence initial field on an n^3 periodic D3Q27 box.

    Gaussian white noise is filtered in Fourier space to the shell spectrum
    E(k) ~ k^4 exp(-2 (k/k0)^2) (k in integer wavenumbers), projected onto
    divergence-free fields, and scaled so that Ma_t = sqrt(<u.u>)/sqrt(gamma T0).
    rho = rho0, T = T0.  mu0 = <rho> u_rms lambda / Re_lambda with
    u_rms = sqrt(<u.u>/3) and lambda = sqrt(<u_x^2>/<(d_x u_x)^2>) (central
    differences).  mu = mu0 (T/T0)^mu_exp.
    """
    rng = np.random.default_rng(seed)
    shape = (n, n, n)
    m = np.fft.fftfreq(n, d=1.0 / n)            # integer wavenumbers
    mr = np.fft.rfftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(m, m, mr, indexing="ij")
    k2 = kx * kx + ky * ky + kz * kz
    kmag = np.sqrt(k2)
    # |u_hat(k)| ~ sqrt(E(k) / (4 pi k^2)) ~ k exp(-(k/k0)^2); white noise carries the phases
    amp = kmag * np.exp(-(kmag / k0) ** 2)
    amp[0, 0, 0] = 0.0
    with np.errstate(invalid="ignore", divide="ignore"):
        inv_k2 = np.where(k2 > 0, 1.0 / np.where(k2 > 0, k2, 1.0), 0.0)
    w = [_rfftn(rng.standard_normal(shape).astype(dtype)) * amp for _ in range(3)]
    kv = (kx, ky, kz)
    div = (kv[0] * w[0] + kv[1] * w[1] + kv[2] * w[2]) * inv_k2
    uh = [w[a] - kv[a] * div for a in range(3)]
    del w, div
    u = np.stack([_irfftn(uh[a], shape) for a in range(3)]).astype(np.float64)
    del uh
    # u[a] has axes (z, y, x); component 0 is u_x
    usq = float(np.mean(u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
    scale = Ma_t * math.sqrt(gamma * T0) / math.sqrt(usq)
    u *= scale
    usq *= scale * scale
    u_rms = math.sqrt(usq / 3.0)
    dux = _central_dx(u[0], axis=2)
    lam = math.sqrt(float(np.mean(u[0] ** 2)) / float(np.mean(dux ** 2)))
    mu0 = rho0 * u_rms * lam / Re_lambda
    rho = np.full((n, n, n), rho0)
    T = np.full((n, n, n), T0)
    return Case("hit", 3, n, n, n, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu0, T0=T0,
                mu_exp=mu_exp, bc=(0, 0, 0, 0, 0, 0),
                extra=dict(seed=seed, k0=k0, Ma_t=Ma_t, Re_lambda=Re_lambda, u_rms=u_rms,
                           lambda_=lam))


def ensemble(n: int = 64, seed: int = 7, side_min: int = 256, side_max: int = 1024,
             side_step: int = 128, Ma_range=(1.1, 1.5)):
    """Specifications of n uneven 2D instances: square sides drawn uniformly from
    {side_min, side_min+side_step, ..., side_max}; even instances are Sod tubes,
    odd ones shock-vortex cases with Ma_s ~ U[Ma_range] and r_v = side/32.
    Returns a list of dicts (kind, side, Ma_s); build each with :func:`build_instance`."""
    rng = np.random.default_rng(seed)
    sides = np.arange(side_min, side_max + 1, side_step)
    out = []
    for k in range(n):
        side = int(rng.choice(sides))
        Ma = float(rng.uniform(*Ma_range))
        out.append(dict(kind="sod" if k % 2 == 0 else "shock_vortex", side=side, Ma_s=Ma))
    return out


def build_instance(spec: dict) -> Case:
    side = spec["side"]
    if spec["kind"] == "sod":
        return sod(nx=side, ny=side)
    return shock_vortex(nx=side, ny=side, Ma_s=spec["Ma_s"], r_v=side / 32.0)


def _grid(D, nx, ny, nz):
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return x.astype(np.float64), y.astype(np.float64), z.astype(np.float64)


def shear_wave(D: int = 2, L: int = 64, A: float = 1e-4, U0: float = 0.0, rho0: float = 1.0,
               T0: float = 0.15, mu: float = 0.01, Pr: float = 0.71, gamma: float = 1.4,
               n_other: int = 1) -> Case:
    """Transverse wave u_y = A sin(2 pi x / L) on a uniform state advected with u_x = U0.
    Periodic box L x n_other (x n_other in 3D)."""
    nz = n_other if D == 3 else 1
    rho, u, T = _empty(D, L, n_other, nz)
    x, _, _ = _grid(D, L, n_other, nz)
    rho[:] = rho0
    T[:] = T0
    u[0] = U0
    u[1] = A * np.sin(2.0 * math.pi * x / L)
    return Case("shear_wave", D, L, n_other, nz, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu, T0=T0)


def sound_wave(D: int = 2, L: int = 64, A: float = 1e-4, U0: float = 0.0, rho0: float = 1.0,
               T0: float = 0.15, mu: float = 0.002, Pr: float = 0.71, gamma: float = 1.4,
               n_other: int = 1) -> Case:
    """Right-running isentropic acoustic wave along x on a state advected with u_x = U0:
    rho' = A rho0 cos(kx), u_x' = A c_s cos(kx), T'/T0 = (gamma-1) rho'/rho0."""
    nz = n_other if D == 3 else 1
    rho, u, T = _empty(D, L, n_other, nz)
    x, _, _ = _grid(D, L, n_other, nz)
    cs = math.sqrt(gamma * T0)
    s = A * np.cos(2.0 * math.pi * x / L)
    rho[:] = rho0 * (1.0 + s)
    T[:] = T0 * (1.0 + (gamma - 1.0) * s)
    u[0] = U0 + cs * s
    return Case("sound_wave", D, L, n_other, nz, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu, T0=T0)


def thermal_wave(D: int = 2, L: int = 64, A: float = 1e-4, rho0: float = 1.0, T0: float = 0.15,
                 mu: float = 0.01, Pr: float = 0.71, gamma: float = 1.4, n_other: int = 1) -> Case:
    """Isobaric temperature wave T = T0 (1 + A cos(kx)), rho = rho0 T0 / T, u = 0."""
    nz = n_other if D == 3 else 1
    rho, u, T = _empty(D, L, n_other, nz)
    x, _, _ = _grid(D, L, n_other, nz)
    T[:] = T0 * (1.0 + A * np.cos(2.0 * math.pi * x / L))
    rho[:] = rho0 * T0 / T
    return Case("thermal_wave", D, L, n_other, nz, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu, T0=T0)


def isentropic_vortex(L: int = 48, U0: float = 0.2, Ma_v: float = 0.2, r_v: float = 6.0,
                      rho0: float = 1.0, T0: float = 0.15, mu: float = 1e-3, Pr: float = 0.71,
                      gamma: float = 1.4) -> Case:
    """Isentropic vortex of Mach Ma_v and radius r_v (the vortex of Sec. III.C) at the
    centre of a periodic L x L box, carried by a uniform flow u_x = U0.  The Euler
    solution translates it unchanged: after t steps its centre is at
    (L/2 + U0 t, L/2) modulo L."""
    rho, u, T = _empty(2, L, L, 1)
    x, y, _ = _grid(2, L, L, 1)
    xv = yv = L / 2.0
    cs = math.sqrt(gamma * T0)
    r2 = ((x - xv) ** 2 + (y - yv) ** 2) / (r_v * r_v)
    base = 1.0 - 0.5 * (gamma - 1.0) * Ma_v * Ma_v * np.exp(1.0 - r2)
    rho[:] = rho0 * base ** (1.0 / (gamma - 1.0))
    T[:] = T0 * base
    amp = cs * Ma_v * np.exp(0.5 * (1.0 - r2))
    u[0] = U0 + amp * (y - yv) / r_v
    u[1] = -amp * (x - xv) / r_v
    return Case("isentropic_vortex", 2, L, L, 1, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu, T0=T0,
                extra=dict(U0=U0, x_v=xv, y_v=yv, r_v=r_v))


def random_smooth(D: int, nx: int, ny: int, nz: int = 1, seed: int = 0, rho0: float = 1.0,
                  T0: float = 0.15, drho: float = 0.05, du: float = 0.08, dT: float = 0.02,
                  modes: int = 4, gamma: float = 1.4, Pr: float = 0.71, mu0: float = 0.01,
                  mu_exp: float = 0.0, bc=(0, 0, 0, 0, 0, 0), u0=(0.0, 0.0, 0.0)) -> Case:
    """Smooth seeded random fields: each of rho, u_a, T is its base value (u0 for the
    velocity) plus a sum of `modes` random Fourier modes (periodic on the box) scaled
    so that the perturbation never exceeds the given amplitude.  With |u0_a| > du every
    velocity component keeps one sign everywhere."""
    rng = np.random.default_rng(seed)
    if D == 2:
        nz = 1
    x, y, z = _grid(D, nx, ny, nz)

    def field_(amp):
        acc = np.zeros((nz, ny, nx))
        for _ in range(modes):
            kx, ky = rng.integers(0, 3, size=2)
            kz = rng.integers(0, 3) if D == 3 else 0
            ph = rng.uniform(0, 2 * math.pi)
            acc += np.cos(2 * math.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + ph)
        return amp * acc / modes

    rho = rho0 + field_(drho)
    T = T0 + field_(dT)
    u = np.stack([u0[a] + field_(du) for a in range(D)])
    return Case("random_smooth", D, nx, ny, nz, rho, u, T, gamma=gamma, Pr=Pr, mu0=mu0, T0=T0,
                mu_exp=mu_exp, bc=tuple(bc))
