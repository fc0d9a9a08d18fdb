"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by
element on the same seeded inputs.

Tolerances (relative L2 over all nodes, all components for u): FP64 store 1e-12,
FP32 1e-5, FP16 deviation store 1e-3, over the stated number of steps.  The BF16
deviation store keeps 8 significand bits against FP16's 11, so its unit roundoff,
and with it the storage error, is 8x FP16's (3.5e-3 in u where FP16 gives 4e-4); it
is held to the FP16 bound times that ratio, 8e-3, above the 1e-3 that FP16 meets.
Grids are chosen ragged against the 32 x 8 tiles of the fused kernels and, in 3D,
against the z segments.

The upwind derivative (Sec. III.A) branches on the sign of u_a at the node.  Where
u_a is within rounding of zero, FP32 and FP64 may take different branches, which
changes D_a by a second difference: a legitimate, discrete divergence rather than
an arithmetic error.  The reduced-precision cases therefore use flows whose
velocity components keep one sign everywhere (a mean flow larger than the
perturbation), so every upwind decision is the same on both sides; flows with
zero crossings are compared at FP64, where both sides decide identically.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from paper_2102_09512_gb300 import cases as C

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5, "f16dev": 1e-3, "bf16dev": 8e-3}


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2102_09512_gb300 import build as B
    B.build()
    O.build()
    O.set_threads(0)
    from paper_2102_09512_gb300 import elbm
    return elbm


def oparams(c, **kw):
    d = dict(D=c.D, nx=c.nx, ny=c.ny, nz=c.nz, gamma=c.gamma, Pr=c.Pr, mu0=c.mu0, T0=c.T0,
             mu_exp=c.mu_exp, bc=c.bc, fixed=c.fixed, cv=c.cv)
    d.update(kw)
    return O.Params(**d)


_ORACLE = {}


def oracle_fields(key, c, steps, **kw):
    if key not in _ORACLE:
        s = O.init(oparams(c, **kw), c.rho, c.u, c.T)
        O.step(s, steps)
        _ORACLE[key] = O.fields(s)
    return _ORACLE[key]


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def gpu_fields(E, c, steps, store, kernel=0, deriv=0, tz=None):
    g = E.Solver.from_case(c, store=store, deriv=deriv)
    g.set_kernel(kernel)
    if tz is not None:
        g.set_tile_z(tz)
    g.step(steps)
    out = g.fields()
    g.close()
    return out


def assert_parity(got, ref, tol, label=""):
    names = ("rho", "u", "T")
    errs = {n: rel_l2(a, b) for n, a, b in zip(names, got, ref)}
    for n in names:
        assert errs[n] <= tol, (label, errs)
    return errs


U0_2D = (0.09, -0.07, 0.0)
U0_3D = (0.09, -0.07, 0.06)
CASES_2D = {
    # zero-mean flows: upwind ties possible, FP64 only
    "periodic-zm": lambda: C.random_smooth(2, 37, 29, 1, seed=11, mu0=0.01),
    "zerograd-zm": lambda: C.random_smooth(2, 45, 19, 1, seed=12, mu0=0.01, bc=(1, 1, 1, 1, 0, 0)),
    # one-signed velocity components: all stores
    "periodic": lambda: C.random_smooth(2, 37, 29, 1, seed=13, mu0=0.01, du=0.05, u0=U0_2D),
    "zerograd": lambda: C.random_smooth(2, 45, 19, 1, seed=14, mu0=0.01, du=0.05, u0=U0_2D,
                                        bc=(1, 1, 1, 1, 0, 0)),
}
CASES_3D = {
    "periodic-zm": lambda: C.random_smooth(3, 37, 21, 19, seed=21, mu0=0.01),
    "zerograd-zm": lambda: C.random_smooth(3, 20, 13, 17, seed=22, mu0=0.01, bc=(1, 1, 0, 0, 1, 1)),
    "periodic": lambda: C.random_smooth(3, 37, 21, 19, seed=23, mu0=0.01, du=0.05, u0=U0_3D),
    "zerograd": lambda: C.random_smooth(3, 20, 13, 17, seed=24, mu0=0.01, du=0.05, u0=U0_3D,
                                        bc=(1, 1, 0, 0, 1, 1)),
}
PAIRS = [(case, store) for case in ("periodic", "zerograd") for store in TOL] + \
        [("periodic-zm", "f64"), ("zerograd-zm", "f64")]


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("case,store", PAIRS)
def test_d2q9_parity(E, case, store, kernel):
    c = CASES_2D[case]()
    steps = 100
    ref = oracle_fields(("2d", case), c, steps)
    assert_parity(gpu_fields(E, c, steps, store, kernel), ref, TOL[store], (case, kernel, store))


MARCH_2D = {
    "periodic": lambda: C.random_smooth(2, 301, 45, 1, seed=15, mu0=0.01, du=0.05, u0=U0_2D),
    "zerograd": lambda: C.random_smooth(2, 260, 33, 1, seed=16, mu0=0.01, du=0.05, u0=U0_2D,
                                        bc=(1, 1, 1, 1, 0, 0)),
    "periodic-zm": lambda: C.random_smooth(2, 301, 45, 1, seed=17, mu0=0.01),
}


@pytest.mark.parametrize("tz", [1, 2, 7, 16, None])
@pytest.mark.parametrize("case,store", [("periodic", "f64"), ("periodic", "f32"), ("periodic", "f16dev"),
                                        ("zerograd", "f64"), ("zerograd", "f32"), ("zerograd", "f16dev"),
                                        ("periodic", "bf16dev"), ("periodic-zm", "f64")])
def test_d2q9_row_march_segments(E, case, store, tz):
    """The D2Q9 row march over grids of several strips (128 nodes for FP64 and FP32, 256
    for the 16-bit stores; the last one ragged) and row segments of 1, 2, 7 and 16 rows or
    the length chosen for the device, 100 steps: segments of one and two rows run only the
    prologue and the last-row paths."""
    c = MARCH_2D[case]()
    ref = oracle_fields(("2d-march", case), c, 100)
    assert_parity(gpu_fields(E, c, 100, store, 0, tz=tz), ref, TOL[store], (case, store, tz))


@pytest.mark.parametrize("kernel", [0, 1, 2])
@pytest.mark.parametrize("case,store", PAIRS)
def test_d3q27_parity(E, case, store, kernel):
    """Every store (BF16 included) on small ragged grids over 40 steps; the 100-step
    window follows in test_d3q27_parity_100_steps."""
    c = CASES_3D[case]()
    steps = 40
    ref = oracle_fields(("3d", case), c, steps)
    assert_parity(gpu_fields(E, c, steps, store, kernel), ref, TOL[store], (case, kernel, store))


# 100-step D3Q27 parity on a grid ragged against the 32 x 8 tiles (40 x 27) and long in z
# (80 planes), marched in the z segments the bench workload uses on 152 SMs (64 planes for
# the FP32 store, 37 for FP16): several segments, one of them the full-length pipeline.
LONG_3D = {
    "periodic": lambda: C.random_smooth(3, 40, 27, 80, seed=121, mu0=0.01, du=0.05, u0=U0_3D),
    "zerograd": lambda: C.random_smooth(3, 40, 27, 80, seed=122, mu0=0.01, du=0.05, u0=U0_3D,
                                        bc=(1, 1, 0, 0, 1, 1)),
    "periodic-zm": lambda: C.random_smooth(3, 40, 27, 80, seed=123, mu0=0.01),
    "zerograd-zm": lambda: C.random_smooth(3, 40, 27, 80, seed=124, mu0=0.01, bc=(1, 1, 0, 0, 1, 1)),
}
LONG_PAIRS = [(case, store) for case in ("periodic", "zerograd") for store in ("f64", "f32", "f16dev")] + \
             [("periodic-zm", "f64"), ("zerograd-zm", "f64")]
PRODUCTION_TZ = {"f64": None, "f32": 64, "f16dev": 37}


@pytest.mark.parametrize("kernel", [0, 1, 2, 3])
@pytest.mark.parametrize("case,store", LONG_PAIRS)
def test_d3q27_parity_100_steps(E, case, store, kernel):
    """FP64 to 1e-12, FP32 to 1e-5 and the FP16 deviation store to 1e-3 over 100 steps, in
    the fused (cp.async), two-pass, re-read and tensor-copy (TMA) schedules (the last has
    no FP64 form)."""
    if kernel == 3 and store == "f64":
        pytest.skip("the tensor-copy schedule runs the FP32-arithmetic stores only")
    c = LONG_3D[case]()
    steps = 100
    ref = oracle_fields(("3d-long", case), c, steps)
    tz = PRODUCTION_TZ[store] if kernel in (0, 3) else None
    assert_parity(gpu_fields(E, c, steps, store, kernel, tz=tz), ref, TOL[store], (case, kernel, store))


INNER_3D = {
    # tiles of 32 x 8 with two nodes of margin to every x and y face (x0 = 32, 64; y0 = 8, 16):
    # their pull addresses skip the boundary maps on the planes away from the z faces
    "periodic": lambda: C.random_smooth(3, 100, 30, 12, seed=131, mu0=0.01, du=0.05, u0=U0_3D),
    "zerograd": lambda: C.random_smooth(3, 100, 30, 12, seed=132, mu0=0.01, du=0.05, u0=U0_3D,
                                        bc=(1, 1, 1, 1, 1, 1)),
}


@pytest.mark.parametrize("kernel", [0, 3])
@pytest.mark.parametrize("case,store", [(c, s) for c in INNER_3D for s in ("f64", "f32", "f16dev")])
def test_d3q27_inner_tiles(E, case, store, kernel):
    if kernel == 3 and store == "f64":
        pytest.skip("the tensor-copy schedule runs the FP32-arithmetic stores only")
    c = INNER_3D[case]()
    ref = oracle_fields(("inner", case), c, 60)
    assert_parity(gpu_fields(E, c, 60, store, kernel), ref, TOL[store], (case, store, kernel))


@pytest.mark.parametrize("store", ["f64", "f32", "f16dev"])
@pytest.mark.parametrize("tz", [1, 2, 5, 7, 64])
def test_d3q27_z_segments(E, tz, store):
    """The z-segment length of the fused kernels changes nothing but the schedule
    (segments of 1 and 2 planes exercise the pipeline prologue and epilogue)."""
    c = CASES_3D["periodic"]()
    ref = oracle_fields(("3d", "periodic"), c, 40)
    assert_parity(gpu_fields(E, c, 40, store, 0, tz=tz), ref, TOL[store], (tz, store))


@pytest.mark.parametrize("D", [2, 3])
def test_central_derivative_variant(E, D):
    c = C.random_smooth(D, 33, 17, 9 if D == 3 else 1, seed=31, mu0=0.01, du=0.05, u0=U0_3D)
    ref = oracle_fields(("central", D), c, 30, deriv=1)
    for store in ("f64", "f32"):
        assert_parity(gpu_fields(E, c, 30, store, 0, deriv=1), ref, TOL[store], store)


def test_power_law_viscosity(E):
    c = C.random_smooth(3, 24, 17, 10, seed=41, mu0=0.01, mu_exp=0.76, dT=0.04, du=0.05, u0=U0_3D)
    ref = oracle_fields(("powerlaw",), c, 30)
    for store in ("f64", "f32"):
        assert_parity(gpu_fields(E, c, 30, store, 0), ref, TOL[store], store)


def test_sod_tube_fp64_parity_and_exact_solution(E):
    """Sod tube (Sec. III.B), 800 x 4, 500 steps, FP64: oracle parity, and the GPU
    profile against the exact Riemann solution."""
    import exact_riemann as R
    c = C.sod(nx=800, ny=4, mu=0.015)
    ref = oracle_fields(("sod",), c, 500)
    got = gpu_fields(E, c, 500, "f64", 0)
    assert_parity(got, ref, TOL["f64"])
    rho = got[0].reshape(4, 800)[0]
    ux = got[1][0].reshape(4, 800)[0]
    xi = (np.arange(800) + 0.5 - 400.0) / 500.0
    re, ue, _ = R.sample(xi, 1.0, 0.0, 0.15, 0.125, 0.0, 0.015)
    assert np.mean(np.abs(rho - re)) < 4.5e-3
    assert np.mean(np.abs(ux - ue)) < 2.0e-3


@pytest.mark.parametrize("D", [2, 3])
def test_conservation_totals(E, D):
    """FP64 totals of the GPU state equal the oracle's; the totals accumulated inside
    the step kernel equal the totals of the state the step produced; under
    periodic boundaries they do not drift."""
    c = C.random_smooth(D, 37, 21, 19 if D == 3 else 1, seed=51, mu0=0.01)
    s = O.init(oparams(c), c.rho, c.u, c.T)
    t0 = O.conservation(s)
    g = E.Solver.from_case(c, store="f64")
    assert np.allclose(g.conservation(), t0, rtol=1e-14, atol=1e-14 * abs(t0[0]))
    for kernel in (0, 1):
        g.set_kernel(kernel)
        g.step(1)
        assert np.allclose(g.step_totals(), g.conservation(), rtol=1e-13, atol=1e-13 * abs(t0[0]))
    g.step(20)
    t1 = g.conservation()
    scale = np.array([t0[0]] * 4 + [t0[4]])
    assert np.all(np.abs(t1 - t0) / scale < 1e-13)
    g.close()


def test_checkpoint_restart_is_bitwise(E):
    c = C.random_smooth(3, 21, 13, 9, seed=61, mu0=0.01)
    for store in ("f64", "f32", "f16dev"):
        a = E.Solver.from_case(c, store=store)
        a.step(10)
        snap = a.get_populations()
        a.step(10)
        ref = a.fields()
        b = E.Solver.from_case(c, store=store)
        b.set_populations(snap)
        b.step(10)
        got = b.fields()
        for x, y in zip(got, ref):
            assert np.array_equal(x, y), store
        a.close()
        b.close()


def test_fused_and_twopass_agree(E):
    """The three schedules compute the same arithmetic per node in different kernels;
    compiler contraction choices differ at the last bit, which FP64 and FP32 keep at
    rounding level and FP16 storage can turn into one-ulp differences per step."""
    c = CASES_3D["periodic"]()
    for store, tol in (("f64", 1e-14), ("f32", 1e-6), ("f16dev", TOL["f16dev"])):
        a = gpu_fields(E, c, 20, store, 0)
        for kernel in (1, 2):
            b = gpu_fields(E, c, 20, store, kernel)
            for x, y in zip(a, b):
                assert rel_l2(x, y) <= tol, (store, kernel)


def test_nonphysical_state_is_reported_and_recoverable(E):
    """A negative temperature (host-side fault injection) is latched on the device and
    reported as ELBM_ERR_NONPHYSICAL; the handle and the context stay usable."""
    c = C.random_smooth(2, 40, 24, 1, seed=71, mu0=0.01)
    g = E.Solver.from_case(c, store="f32")
    T = c.T.copy()
    T.reshape(-1)[123] = -0.1
    with pytest.raises(E.ElbmError) as ei:
        g.set_fields(c.rho, c.u, T)
    assert ei.value.code == E.ELBM_ERR_NONPHYSICAL
    g.set_fields(c.rho, c.u, c.T)
    g.step(5)
    g.sync()
    rho, _, _ = g.fields()
    assert np.all(np.isfinite(rho))
    g.close()


def test_device_field_entry_points(E):
    import torch
    c = C.random_smooth(3, 19, 11, 7, seed=81, mu0=0.01)
    g = E.Solver.from_case(c, store="f32")
    rho = torch.tensor(c.rho.reshape(-1), device="cuda")
    u = torch.tensor(c.u.reshape(-1), device="cuda")
    T = torch.tensor(c.T.reshape(-1), device="cuda")
    g.set_fields(rho, u, T)
    g.step(3)
    r2, u2, T2 = torch.empty_like(rho), torch.empty_like(u), torch.empty_like(T)
    g.fields_device(r2, u2, T2)
    h = g.fields()
    torch.cuda.synchronize()
    assert np.array_equal(r2.cpu().numpy(), h[0])
    assert np.array_equal(T2.cpu().numpy(), h[2])
    g.close()


def _center_after_one_step(c, x, y, z):
    """Oracle value at (x, y, z) after one step, computed on the 5^3 neighbourhood
    (one step at a node depends on nodes at most two apart)."""
    n = c.nx
    idx = [(np.arange(-2, 3) + v) % n for v in (x, y, z)]
    sub_rho = c.rho[np.ix_(idx[2], idx[1], idx[0])]
    sub_T = c.T[np.ix_(idx[2], idx[1], idx[0])]
    sub_u = np.stack([c.u[a][np.ix_(idx[2], idx[1], idx[0])] for a in range(3)])
    p = O.Params(D=3, nx=5, ny=5, nz=5, gamma=c.gamma, Pr=c.Pr, mu0=c.mu0, T0=c.T0,
                 mu_exp=c.mu_exp, bc=(1, 1, 1, 1, 1, 1))
    s = O.init(p, sub_rho, sub_u, sub_T)
    O.step(s, 1)
    r, u, T = O.fields(s)
    k = 2 + 5 * (2 + 5 * 2)
    return r[k], u[:, k], T[k]


@pytest.mark.parametrize("kernel", [0, 3])
@pytest.mark.parametrize("store,tol,drift", [("f32", 2e-6, 1e-6), ("f16dev", 2e-4, 1e-5), ("bf16dev", 4e-3, 8e-5)])
def test_full_size_256_sampled_nodes(E, store, tol, drift, kernel):
    """At the bench's full size (D3Q27, 256^3, decaying-turbulence field; the fused
    cp.async kernel the bench times, and the tensor-copy one) sampled nodes after one
    step equal the oracle's one-by-one values, and the totals are conserved over 5
    steps (FP16: up to the storage rounding, 2^-11 of deviations that are a few
    percent of the populations).  BF16 keeps 8 significand bits: each stored deviation
    carries a relative rounding of up to 2^-9 and the deviations of a node sum in
    magnitude to at most about 2 rho, so rho, T and rho u move by up to about
    2 * 2^-9 = 3.9e-3 (relative): the bound is 4e-3 for rho and T, 2e-3 for u."""
    c = C.hit(256, seed=20210218)
    g = E.Solver.from_case(c, store=store)
    g.set_kernel(kernel)
    t0 = g.conservation()
    g.step(1)
    rho, u, T = g.fields()
    rng = np.random.default_rng(5)
    pts = rng.integers(0, 256, size=(12, 3))
    pts[0] = (0, 0, 0)
    pts[1] = (255, 255, 255)
    for x, y, z in pts:
        n = x + 256 * (y + 256 * z)
        r_o, u_o, T_o = _center_after_one_step(c, x, y, z)
        assert abs(rho[n] - r_o) <= tol * abs(r_o)
        assert abs(T[n] - T_o) <= tol * abs(T_o)
        assert np.max(np.abs(u[:, n] - u_o)) <= tol * 0.5
    g.step(4)
    t1 = g.conservation()
    assert abs(t1[0] - t0[0]) / t0[0] < drift
    assert abs(t1[4] - t0[4]) / t0[4] < drift
    assert np.max(np.abs(t1[1:4] - t0[1:4])) / t0[0] < drift
    g.close()


@pytest.mark.parametrize("store", ["f64", "f32"])
def test_shock_vortex_parity(E, store):
    """Standing Ma_s = 1.2 shock with an isentropic vortex (Sec. III.C) on a reduced
    256 x 128 D2Q9 grid (r_v = 8), 150 steps: oracle parity.  The vortex makes u_y
    change sign, where FP32 and FP64 may take different upwind branches (a second
    difference of Q~ at that node), so the FP32 store is held to 1e-4 here; the
    one-signed cases above hold it to 1e-5."""
    c = C.shock_vortex(nx=256, ny=128, r_v=8.0, Ma_s=1.2)
    ref = oracle_fields(("shock_vortex",), c, 150)
    got = gpu_fields(E, c, 150, store, 0)
    assert_parity(got, ref, TOL["f64"] if store == "f64" else 1e-4, store)


def _center_after_one_step_2d(c, x, y):
    """Oracle value at interior node (x, y) after one step from its 5 x 5 neighbourhood."""
    sub = (slice(0, 1), slice(y - 2, y + 3), slice(x - 2, x + 3))
    p = O.Params(D=2, nx=5, ny=5, nz=1, gamma=c.gamma, Pr=c.Pr, mu0=c.mu0, T0=c.T0, mu_exp=c.mu_exp,
                 bc=(1, 1, 1, 1, 0, 0))
    s = O.init(p, c.rho[sub], np.stack([c.u[0][sub], c.u[1][sub]]), c.T[sub])
    O.step(s, 1)
    r, u, T = O.fields(s)
    return r[12], u[:, 12], T[12]


@pytest.mark.parametrize("store,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_shock_vortex_full_size_sampled(E, store, tol):
    """At the configured 1024 x 1024 (r_v = 32) sampled interior nodes after one step
    equal the oracle's one-by-one values (one step depends on nodes at most two away)."""
    c = C.shock_vortex(nx=1024, ny=1024, r_v=32.0, Ma_s=1.2)
    g = E.Solver.from_case(c, store=store)
    g.step(1)
    rho, u, T = g.fields()
    rng = np.random.default_rng(7)
    pts = list(rng.integers(3, 1021, size=(10, 2))) + [(256, 512), (192, 512)]   # shock, vortex centre
    for x, y in pts:
        n = x + 1024 * y
        r_o, u_o, T_o = _center_after_one_step_2d(c, x, y)
        assert abs(rho[n] - r_o) <= tol * abs(r_o)
        assert abs(T[n] - T_o) <= tol * abs(T_o)
        assert np.max(np.abs(u[:, n] - u_o)) <= tol
    g.close()


# --------------------------------------------------------------------------
# isentropic vortex carried by a uniform flow (Euler translation, Sec. III.C vortex)
# --------------------------------------------------------------------------
def _circular_centre(d, L):
    th = 2.0 * math.pi * np.arange(L) / L
    out = []
    for w in (d.sum(axis=0), d.sum(axis=1)):
        ang = math.atan2(float((w * np.sin(th)).sum()), float((w * np.cos(th)).sum()))
        out.append((ang * L / (2.0 * math.pi)) % L)
    return out


@pytest.mark.parametrize("kernel", [0, 1])
def test_vortex_translation_parity_f64(E, kernel):
    """Quarter period of the translating vortex (u_y changes sign: FP64 only)."""
    c = C.isentropic_vortex(L=48, U0=0.1, Ma_v=0.1, r_v=6.0, T0=0.15, mu=0.002)
    steps = 120
    ref = oracle_fields(("vortex",), c, steps)
    assert_parity(gpu_fields(E, c, steps, "f64", kernel), ref, TOL["f64"], ("vortex", kernel))


@pytest.mark.parametrize("store", ["f32", "f16dev"])
def test_vortex_translation_reduced_precision(E, store):
    """The reduced-precision stores carry the vortex to L/2 + U0 t like the Euler
    solution (the same property the oracle is pinned to)."""
    c = C.isentropic_vortex(L=48, U0=0.1, Ma_v=0.1, r_v=6.0, T0=0.15, mu=0.002)
    L, U0, steps = c.nx, c.extra["U0"], 120
    rho, _, T = gpu_fields(E, c, steps, store)
    x, y = _circular_centre(c.T0 - (rho * T).reshape(L, L), L)
    assert abs(x - (L / 2 + U0 * steps) % L) < 0.1 and abs(y - L / 2) < 0.1


# --------------------------------------------------------------------------
# fixed-state face: supersonic inflow upstream of the shock (Sec. III.C)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("store,kernel", [("f64", 0), ("f64", 1), ("f64", 2), ("f32", 0), ("f16dev", 0)])
def test_shock_vortex_inflow_parity(E, store, kernel):
    """The shock-vortex case with the -x face holding the upstream state fixed, on a
    grid ragged against the tiles (150 x 70, r_v = 8), 150 steps, against the oracle.
    u_y changes sign around the vortex, so the reduced-precision stores are held to
    10x their one-signed bounds, as in test_shock_vortex_parity."""
    c = C.shock_vortex(nx=150, ny=70, r_v=8.0, Ma_s=1.2, inflow=True)
    ref = oracle_fields(("shock_vortex_inflow",), c, 150)
    got = gpu_fields(E, c, 150, store, kernel, tz=16 if kernel == 0 else None)
    tol = TOL["f64"] if store == "f64" else 10 * TOL[store]
    assert_parity(got, ref, tol, (store, kernel))


@pytest.mark.parametrize("bc", [(2, 1, 2, 1, 0, 0), (2, 1, 1, 2, 0, 0)])
@pytest.mark.parametrize("kernel,tz", [(0, 16), (0, 1), (1, None), (2, None)])
def test_fixed_state_faces_on_both_axes(E, bc, kernel, tz):
    """Fixed-state ghosts on the -x face and on one y face (the row march's first or last
    row borders the fixed state), FP64 against the oracle over 150 steps.  The flow keeps
    u_x and u_y positive everywhere (0.03 <= u_y <= 0.1 over the run), so every upwind
    decision is the same on both sides.  (A tangential flow along a fixed y face, such as
    the shock-vortex case with its inflow state on a y face, has u_y within rounding of
    zero at the wall: GPU and oracle sums that differ in the last bit then take different
    upwind branches there and the runs part by 1e-3 within five steps, in every schedule
    alike.)"""
    c = C.random_smooth(2, 150, 70, 1, seed=18, mu0=0.01, du=0.05, u0=(0.09, 0.07, 0.0))
    c.bc = bc
    c.fixed = (1.0, 0.09, 0.07, 0.0, 0.15)
    ref = oracle_fields(("fixed-xy", bc), c, 150)
    assert_parity(gpu_fields(E, c, 150, "f64", kernel, tz=tz), ref, TOL["f64"], (bc, kernel, tz))
    if kernel == 0:
        assert_parity(gpu_fields(E, c, 150, "f32", kernel, tz=tz), ref, TOL["f32"], (bc, kernel, tz, "f32"))


# --------------------------------------------------------------------------
# general caloric equation of state (Eqs. U, E): cubic Cv(T)
# --------------------------------------------------------------------------
CV_POLY = (1.0, 4.0, -4.0, 5.0)


@pytest.mark.parametrize("D,kernel", [(2, 0), (2, 1), (3, 0), (3, 1), (3, 2)])
@pytest.mark.parametrize("store", list(TOL))
def test_caloric_eos_parity(E, D, kernel, store):
    """Cv(T) = 1 + 4T - 4T^2 + 5T^3: every store and schedule against the oracle (the
    one-signed flow of the cases above, 60 steps)."""
    c = (CASES_2D if D == 2 else CASES_3D)["periodic"]()
    c.cv = CV_POLY
    steps = 60
    ref = oracle_fields(("caloric", D), c, steps)
    assert_parity(gpu_fields(E, c, steps, store, kernel), ref, TOL[store], (D, kernel, store))


# --------------------------------------------------------------------------
# D3Q27 schedule with tensor-copy (TMA) plane staging: ELBM_KERNEL_FUSED_TMA
# --------------------------------------------------------------------------
TMA_CASES = {
    # periodic; tiles (32, 8) and (32, 16) take the tensor-copy path, the others (at the
    # x and y faces, or ragged) the per-pair cp.async path
    "periodic": lambda: C.random_smooth(3, 80, 27, 13, seed=25, mu0=0.01, du=0.05, u0=U0_3D),
    # zero-gradient on every face, with tensor-copy tiles inside
    "zerograd": lambda: C.random_smooth(3, 72, 26, 11, seed=28, mu0=0.01, du=0.05, u0=U0_3D,
                                        bc=(1, 1, 1, 1, 1, 1)),
    # x periodic, zero-gradient y and z faces, every tile at a face (cp.async path only)
    "zerograd-yz": lambda: C.random_smooth(3, 40, 13, 17, seed=26, mu0=0.01, du=0.05, u0=U0_3D,
                                           bc=(0, 0, 1, 1, 1, 1)),
    # fewer rows than a box (5 < 10)
    "thin-y": lambda: C.random_smooth(3, 64, 5, 9, seed=27, mu0=0.01, du=0.05, u0=U0_3D),
}
TMA_STORES = ["f32", "f16dev", "bf16dev"]


@pytest.mark.parametrize("store", TMA_STORES)
@pytest.mark.parametrize("case", list(TMA_CASES))
def test_d3q27_tma_parity(E, case, store):
    c = TMA_CASES[case]()
    steps = 40
    ref = oracle_fields(("tma", case), c, steps)
    got = gpu_fields(E, c, steps, store, E.ELBM_KERNEL_FUSED_TMA)
    assert_parity(got, ref, TOL[store], (case, store))


@pytest.mark.parametrize("store", ["f32", "f16dev"])
@pytest.mark.parametrize("tz", [1, 2, 5])
def test_d3q27_tma_z_segments(E, tz, store):
    """Segments of 1 and 2 planes run only the prologue and the last-plane paths of
    the TMA pipeline."""
    c = TMA_CASES["periodic"]()
    ref = oracle_fields(("tma", "periodic"), c, 40)
    got = gpu_fields(E, c, 40, store, E.ELBM_KERNEL_FUSED_TMA, tz=tz)
    assert_parity(got, ref, TOL[store], (tz, store))


@pytest.mark.parametrize("store", TMA_STORES)
def test_d3q27_tma_caloric_eos(E, store):
    c = TMA_CASES["periodic"]()
    c.cv = CV_POLY
    ref = oracle_fields(("tma-caloric",), c, 60)
    got = gpu_fields(E, c, 60, store, E.ELBM_KERNEL_FUSED_TMA)
    assert_parity(got, ref, TOL[store], store)


def test_d3q27_tma_agrees_with_cp_async_kernel(E):
    """The TMA-staged and the per-pair cp.async schedules run the same per-node
    arithmetic on the same pulled values."""
    for case in ("periodic", "zerograd"):
        c = TMA_CASES[case]()
        for store, tol in (("f32", 1e-6), ("f16dev", TOL["f16dev"])):
            a = gpu_fields(E, c, 20, store, E.ELBM_KERNEL_FUSED)
            b = gpu_fields(E, c, 20, store, E.ELBM_KERNEL_FUSED_TMA)
            for x, y in zip(a, b):
                assert rel_l2(x, y) <= tol, (case, store)


def test_d3q27_tma_step_totals(E):
    """The totals the TMA kernel accumulates equal those of the state it produced."""
    c = TMA_CASES["periodic"]()
    g = E.Solver.from_case(c, store="f32")
    g.set_kernel(E.ELBM_KERNEL_FUSED_TMA)
    g.step(3)
    t = g.step_totals()
    ref = g.conservation()
    assert np.allclose(t, ref, rtol=1e-6, atol=1e-6 * abs(ref[0]))
    g.close()


def test_tma_wait_timeout_is_reported_and_recoverable(E):
    """Failure path of the TMA-staged schedule, exercised without a GPU fault: with the
    fault injection on, the tile that requests its planes by tensor copies (the one at
    (32, 8) of this 96 x 24 x 4 grid) waits for 16 bytes that never come.  Its bounded
    waits run out (about a second each), the step reports ELBM_ERR_TIMEOUT at the next
    synchronising call, and afterwards the same handle and context run normal steps
    that match the oracle."""
    c = C.random_smooth(3, 96, 24, 4, seed=29, mu0=0.01, du=0.05, u0=U0_3D)
    g = E.Solver.from_case(c, store="f32")
    g.set_kernel(E.ELBM_KERNEL_FUSED_TMA)
    E.elbm_inject_wait_timeout(g.h, 1)
    g.step(1)
    with pytest.raises(E.ElbmError) as ei:
        g.sync()
    assert ei.value.code == E.ELBM_ERR_TIMEOUT
    E.elbm_inject_wait_timeout(g.h, 0)
    g.set_fields(c.rho, c.u, c.T)
    g.step(10)
    ref = oracle_fields(("tma-timeout",), c, 10)
    assert_parity(g.fields(), ref, TOL["f32"])
    g.close()


DEGENERATE = {
    # one and two planes in z (the pulled planes z - 1 and z + 1 are the plane itself or
    # the other one), one row in y, and zero-gradient faces on a single plane
    "nz1": lambda: C.random_smooth(3, 40, 12, 1, seed=91, mu0=0.01, du=0.05, u0=U0_3D),
    "nz2": lambda: C.random_smooth(3, 40, 12, 2, seed=92, mu0=0.01, du=0.05, u0=U0_3D),
    "ny1": lambda: C.random_smooth(3, 40, 1, 7, seed=93, mu0=0.01, du=0.05, u0=U0_3D),
    "nz1-zerograd": lambda: C.random_smooth(3, 36, 9, 1, seed=94, mu0=0.01, du=0.05, u0=U0_3D,
                                            bc=(1, 1, 1, 1, 1, 1)),
    "2d-ny1": lambda: C.random_smooth(2, 40, 1, 1, seed=95, mu0=0.01, du=0.05, u0=U0_2D),
}


@pytest.mark.parametrize("store", ["f64", "f32"])
@pytest.mark.parametrize("case", list(DEGENERATE))
def test_degenerate_grids(E, case, store):
    """Degenerate extents against the oracle in every schedule that applies."""
    c = DEGENERATE[case]()
    steps = 30
    ref = oracle_fields(("degenerate", case), c, steps)
    kernels = [0, 1] if c.D == 2 else ([0, 1, 2, 3] if store == "f32" else [0, 1, 2])
    for kernel in kernels:
        assert_parity(gpu_fields(E, c, steps, store, kernel), ref, TOL[store], (case, store, kernel))


@pytest.mark.parametrize("D,store,kernel", [(2, "f32", 0), (2, "f32", 1), (2, "f16dev", 0), (3, "f32", 1),
                                            (3, "f16dev", 1)])
def test_step_totals_of_the_fp32_arithmetic_paths(E, D, store, kernel):
    """The step totals of the kernels that sum each warp's node values in FP32 before
    the FP64 sum over warps equal the FP64 totals of the state they produced, to the
    rounding of the FP32 node values."""
    c = C.random_smooth(D, 45, 23, 9 if D == 3 else 1, seed=97, mu0=0.01)
    g = E.Solver.from_case(c, store=store)
    g.set_kernel(kernel)
    g.step(3)
    t = g.step_totals()
    ref = g.conservation()
    assert np.allclose(t, ref, rtol=2e-6, atol=2e-6 * abs(ref[0])), (t, ref)
    g.close()


def test_shock_vortex_1024_full_run_fp32_against_fp64(E):
    """The configured shock-vortex case (1024 x 1024, r_v = 32, Ma_s = 1.2) over its
    4000 steps: the FP64 and FP32 stores stay physical and the FP32 fields stay within
    5e-4 (relative L2) of the FP64 ones (measured: u 1.6e-4, rho 1.2e-4, T 6.5e-5; the
    vortex's u_y sign changes make FP32 and FP64 take different upwind branches at a
    few nodes, so the bound is above the one-signed cases' 1e-5)."""
    c = C.shock_vortex(nx=1024, ny=1024, r_v=32.0, Ma_s=1.2)
    out = {}
    for store in ("f64", "f32"):
        g = E.Solver.from_case(c, store=store)
        g.step(4000)
        g.sync()
        out[store] = g.fields()
        g.close()
    for a, b in zip(out["f32"], out["f64"]):
        assert np.all(np.isfinite(a))
        assert rel_l2(a, b) <= 5e-4



@pytest.mark.parametrize("store,tol", [("f32", 2e-6), ("f16dev", 2e-4)])
def test_full_size_512_sampled_nodes(E, store, tol):
    """The 512^3 decaying-turbulence grid (134 M nodes, the larger size of the
    reduced-precision study): sampled nodes after one step of the default fused kernel
    equal the oracle's one-by-one values."""
    c = C.hit(512, seed=20210218, dtype=np.float32)
    g = E.Solver.from_case(c, store=store)
    g.step(1)
    import torch
    n3 = 512 ** 3
    rho = torch.empty(n3, dtype=torch.float64, device="cuda")
    u = torch.empty(3 * n3, dtype=torch.float64, device="cuda")
    T = torch.empty(n3, dtype=torch.float64, device="cuda")
    g.fields_device(rho, u, T)
    g.sync()
    rng = np.random.default_rng(9)
    pts = rng.integers(0, 512, size=(8, 3))
    pts[0] = (0, 0, 0)
    pts[1] = (511, 511, 511)
    for x, y, z in pts:
        n = int(x + 512 * (y + 512 * z))
        r_o, u_o, T_o = _center_after_one_step(c, x, y, z)
        assert abs(float(rho[n]) - r_o) <= tol * abs(r_o)
        assert abs(float(T[n]) - T_o) <= tol * abs(T_o)
        assert max(abs(float(u[a * n3 + n]) - u_o[a]) for a in range(3)) <= tol * 0.5
    g.close()
