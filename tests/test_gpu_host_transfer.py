"""GPU tests of the host transfers: fields (elbm_set_fields / elbm_get_fields) and the
asynchronous step totals (elbm_step_totals_async).

Host arrays in page-locked memory that the device maps are read by the initialisation
kernel and written by the field kernel directly, over the host link; pageable arrays go
through the auxiliary staging area with copies.  Both paths run the same kernels on the
same values, so the states they produce and the fields they return are equal bit for
bit, for the ping-pong stores and the single (AA) store, including arrays that start
inside a larger page-locked allocation.
"""
import numpy as np
import pytest

from paper_2102_09512_gb300 import cases as C

pytestmark = pytest.mark.gpu

U0 = {2: (0.08, -0.06, 0.0), 3: (0.08, -0.06, 0.05)}


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2102_09512_gb300 import build as B
    B.build()
    from paper_2102_09512_gb300 import elbm
    return elbm


def pinned_copy(torch, a, lead=0):
    """a (FP64) in page-locked memory, `lead` elements into a larger allocation."""
    flat = np.ascontiguousarray(a, dtype=np.float64).reshape(-1)
    buf = torch.empty(flat.size + lead + 7, dtype=torch.float64).pin_memory()
    buf[lead:lead + flat.size] = torch.from_numpy(flat)
    return buf, buf[lead:lead + flat.size]


def pinned_fields(E, torch, g, lead):
    bufs = [torch.zeros(n + lead + 5, dtype=torch.float64).pin_memory() for n in (g.N, g.D * g.N, g.N)]
    views = [b[lead:lead + n] for b, n in zip(bufs, (g.N, g.D * g.N, g.N))]
    E._check(E.elbm_get_fields(g.h, *views), "elbm_get_fields")
    return [v.numpy().copy() for v in views]


@pytest.mark.parametrize("layout", ["pingpong", "aa"])
@pytest.mark.parametrize("store", ["f64", "f32", "f16dev"])
@pytest.mark.parametrize("D", [2, 3])
def test_page_locked_transfers_equal_staged_ones(E, D, store, layout):
    import torch
    c = C.random_smooth(D, 41, 23, 13 if D == 3 else 1, seed=171 + D, mu0=0.01, du=0.05, u0=U0[D])
    kw = {"layout": E.ELBM_LAYOUT_AA} if layout == "aa" else {}
    staged = E.Solver.from_case(c, store=store, **kw)     # numpy (pageable) fields
    direct = E.Solver.from_case(c, store=store, **kw)
    lead = 3 if D == 3 else 0
    keep = [pinned_copy(torch, a, lead) for a in (c.rho, c.u, c.T)]
    E._check(E.elbm_set_fields(direct.h, *[v for _, v in keep]), "elbm_set_fields")
    for g in (staged, direct):
        g.step(5)
    a = staged.fields()
    b = pinned_fields(E, torch, direct, lead)
    b2 = direct.fields()
    for x, y, z in zip(a, b, b2):
        assert np.array_equal(np.ravel(x), np.ravel(y)), (D, store, layout)
        assert np.array_equal(np.ravel(x), np.ravel(z)), (D, store, layout)
    assert np.array_equal(staged.conservation(), direct.conservation())
    staged.close()
    direct.close()


def test_bench_size_transfer_round_trip(E):
    """At the bench's 256^3 D3Q27 size (0.67 GB of FP64 fields each way) the page-locked
    path returns the fields the staged path returns."""
    import torch
    c = C.hit(256)
    N = c.N
    g = E.Solver.from_case(c, store="f32")
    ref = g.fields()
    rho = torch.empty(N, dtype=torch.float64).pin_memory()
    u = torch.empty(3 * N, dtype=torch.float64).pin_memory()
    T = torch.empty(N, dtype=torch.float64).pin_memory()
    E._check(E.elbm_get_fields(g.h, rho, u, T), "elbm_get_fields")
    assert np.array_equal(ref[0], rho.numpy())
    assert np.array_equal(ref[1].reshape(-1), u.numpy())
    assert np.array_equal(ref[2], T.numpy())
    E._check(E.elbm_set_fields(g.h, rho, u, T), "elbm_set_fields")   # equilibria of the same fields
    rho2, u2, T2 = g.fields()
    assert np.max(np.abs(rho2 - ref[0])) <= 1e-6 * np.max(np.abs(ref[0]))
    g.close()
    del rho, u, T
    torch.cuda.empty_cache()


def test_async_step_totals_equal_synchronous_ones(E):
    """Totals enqueued after each of several steps without synchronising (into page-locked
    and into pageable buffers) equal those the synchronising call returns after the same
    steps; before the first step the call is refused."""
    import torch
    c = C.random_smooth(3, 41, 23, 13, seed=181, mu0=0.01, du=0.05, u0=U0[3])
    a = E.Solver.from_case(c, store="f32")
    b = E.Solver.from_case(c, store="f32")
    pinned = [torch.full((5,), np.nan, dtype=torch.float64).pin_memory() for _ in range(4)]
    pageable = np.full(5, np.nan)
    assert E.elbm_step_totals_async(a.h, pinned[0]) == E.ELBM_ERR_ARG
    for k in range(4):
        a.step(1)
        E._check(E.elbm_step_totals_async(a.h, pinned[k]), "elbm_step_totals_async")
    E._check(E.elbm_step_totals_async(a.h, pageable), "elbm_step_totals_async")
    a.sync()
    for k in range(4):
        b.step(1)
        assert np.array_equal(pinned[k].numpy(), b.step_totals()), k
    assert np.array_equal(pageable, pinned[3].numpy())
    a.close()
    b.close()
