"""The shock-vortex interaction at the paper's size (Sec. III.C): 1680 x 1440 D2Q9,
r_v = 60, Ma_s = 1.2, Ma_v = 0.25, Re = 800, Pr = 0.75, the upstream state held
fixed on the -x face (supersonic inflow), +x zero-gradient, y periodic.  FP64 store
(the reduced-precision stores do not stay stable on this case: rounding noise grows
in the supersonic vortex, where the upwind-corrected scheme is at its stability edge).

The paper compares the radial sound pressure Delta P = (P - P_s)/P_s at theta = -45
degrees with DNS data that is not available here; these tests check what the
physics fixes: the vortex is carried at the upstream speed to the shock and at the
post-shock speed after it, and the sound wave it radiates runs outwards at the
sound speed behind the shock, with an amplitude of the order of the paper's ~1 %."""
import math

import numpy as np
import pytest

from paper_2102_09512_gb300 import cases as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2102_09512_gb300 import build as B
    B.build()
    from paper_2102_09512_gb300 import elbm
    return elbm


@pytest.fixture(scope="module")
def run(E):
    from paper_2102_09512_gb300 import studies
    out = studies.shock_vortex_sound(times=(6.0, 8.0), store="f64")
    res = {int(ts): dict(pred=e["predicted"], centre=e["centre"], r=e["r_over_rv"], dp=e["delta_p"])
           for ts, e in out["results"].items()}
    return out["case"], res


def test_vortex_track(run):
    """The vortex centre (vorticity extremum) sits within a few nodes (r_v = 60) of the
    position advected at u_l up to the shock and at u_s behind it."""
    c, out = run
    for ts, e in out.items():
        assert abs(e["centre"][0] - e["pred"][0]) < 5.0, (ts, e["centre"], e["pred"])
        assert abs(e["centre"][1] - e["pred"][1]) < 6.0, (ts, e["centre"], e["pred"])


def test_sound_wave_runs_at_the_post_shock_sound_speed(run):
    """The leading compression of Delta P along theta = -45 degrees moves by
    2 c_s,r / c_s,l r_v between t* = 6 and 8 (c_s,r / c_s,l = sqrt(T_r / T_l)); its
    amplitude is a fraction of a percent to a few percent."""
    c, out = run
    _, _, r_T, _ = C.rankine_hugoniot(1.2)
    expect = 2.0 * math.sqrt(r_T)
    peaks = {}
    for ts, e in out.items():
        m = e["r"] > 1.5
        k = int(np.argmax(np.where(m, e["dp"], -1.0)))
        peaks[ts] = (e["r"][k], e["dp"][k])
        assert 1e-3 < e["dp"][k] < 3e-2, (ts, peaks[ts])
    assert abs((peaks[8][0] - peaks[6][0]) - expect) < 0.3, (peaks, expect)


def test_configured_grid_with_viscosity_from_its_radius_diverges(E):
    """The configured 1024 x 1024 case with mu from Re = 800 on r_v = 32 (mu = 0.0106)
    leaves the physical range within 500 steps (FP64 store); with the paper's mu = 0.0198
    the same grid stays physical over its 4000 steps (tests/test_gpu_parity.py)."""
    c = C.shock_vortex(nx=1024, ny=1024, r_v=32.0, Ma_s=1.2, r_v_mu=32.0)
    assert abs(c.mu0 - 0.0105830) < 1e-6
    g = E.Solver.from_case(c, store="f64")
    status = E.ELBM_OK
    for _ in range(10):
        g.step(50)
        status = E.elbm_sync(g.h)
        if status != E.ELBM_OK:
            break
    g.close()
    assert status == E.ELBM_ERR_NONPHYSICAL
