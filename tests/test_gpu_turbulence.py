"""Turbulence statistics (paper Sec. III.D) on the GPU: the device reduction against
the same statistics computed on the host from the extracted fields, and the long-run
histories of kinetic energy and rms dilatation of the reduced-precision stores
against the FP64 store (within 1 %)."""
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


def host_stats(c, rho, u, T):
    n = c.nx
    r = rho.reshape(c.nz, c.ny, c.nx)
    U = u.reshape(3, c.nz, c.ny, c.nx)
    Tt = T.reshape(c.nz, c.ny, c.nx)
    d = lambda a, ax: 0.5 * (np.roll(a, -1, axis=ax) - np.roll(a, 1, axis=ax))
    theta = d(U[0], 2) + d(U[1], 1) + d(U[2], 0)
    uu = (U ** 2).sum(0)
    return dict(rho_mean=r.mean(), rho_rms=r.std(), K=0.5 * (r * uu).mean(), u_rms=np.sqrt(uu.mean() / 3),
                theta_rms=np.sqrt((theta ** 2).mean()), T_mean=Tt.mean(), T_rms=Tt.std(),
                dudx2=(d(U[0], 2) ** 2).mean())


def test_device_statistics_match_host(E):
    c = C.hit(48, seed=5)
    g = E.Solver.from_case(c, store="f64")
    g.step(20)
    dev = g.turbulence_stats()
    ref = host_stats(c, *g.fields())
    for k, v in ref.items():
        assert dev[k] == pytest.approx(v, rel=1e-10, abs=1e-14), k
    g.close()


def test_long_run_statistics_reduced_precision(E):
    """Decaying turbulence (64^3, Ma_t = 0.5): K(t) and theta_rms(t) of the FP32 and
    FP16-deviation stores stay within 1 % of the FP64 store over 600 steps."""
    c = C.hit(64)
    hist = {}
    for store in ("f64", "f32", "f16dev"):
        g = E.Solver.from_case(c, store=store)
        h = []
        for _ in range(12):
            g.step(50)
            s = g.turbulence_stats()
            h.append((s["K"], s["theta_rms"]))
        hist[store] = np.array(h)
        g.close()
    ref = hist["f64"]
    assert ref[-1, 0] < 0.8 * ref[0, 0]          # the turbulence decays
    for store in ("f32", "f16dev"):
        dev = np.abs(hist[store] / ref - 1.0)
        assert dev.max() <= 0.01, (store, dev.max(axis=0))
