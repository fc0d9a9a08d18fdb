"""GPU tests of graph-replayed stepping (elbm_set_step_graph).

Whole groups of G steps run as one replay of a CUDA graph captured on first use; the
replays launch the same kernels with the same arguments as single steps, so the states,
step totals, step counts and launch counts equal those of single steps bit for bit, in
every schedule and layout, with a remainder of single steps after the last whole group,
and after a change of schedule (which drops the graphs).
"""
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


U2, U3 = (0.08, -0.06, 0.0), (0.08, -0.06, 0.05)
CASES = {
    "sod-800x4-f64": (lambda: C.sod(), "f64", {}),
    "d2-march-f16": (lambda: C.random_smooth(2, 300, 96, 1, seed=201, mu0=0.01, du=0.05, u0=U2), "f16dev", {"tz": 16}),
    "d3-fused-f32": (lambda: C.random_smooth(3, 40, 27, 30, seed=202, mu0=0.01, du=0.05, u0=U3), "f32", {}),
    "d3-twopass-f64": (lambda: C.random_smooth(3, 24, 16, 12, seed=203, mu0=0.01, du=0.05, u0=U3), "f64",
                       {"kernel": 1}),
    "d3-aa-f32": (lambda: C.random_smooth(3, 24, 16, 12, seed=204, mu0=0.01, du=0.05, u0=U3), "f32", {"aa": True}),
}


def make(E, c, store, opt):
    g = E.Solver.from_case(c, store=store, **({"layout": E.ELBM_LAYOUT_AA} if opt.get("aa") else {}))
    if "kernel" in opt:
        g.set_kernel(opt["kernel"])
    if "tz" in opt:
        E._check(E.lib().elbm_set_tile_z(g.h, opt["tz"]), "elbm_set_tile_z")
    return g


@pytest.mark.parametrize("name", list(CASES))
def test_graph_steps_equal_single_steps(E, name):
    build, store, opt = CASES[name]
    c = build()
    a = make(E, c, store, opt)
    b = make(E, c, store, opt)
    b.set_step_graph(8)
    l0a, l0b = a.launches, b.launches
    for n in (29, 1, 16):   # groups of 8 plus remainders, from either store parity
        a.step(n)
        b.step(n)
        assert b.steps_done == a.steps_done
        assert b.launches - l0b == a.launches - l0a
        assert np.array_equal(a.step_totals(), b.step_totals()), (name, n)
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y), (name, n)
    a.close()
    b.close()


def test_graphs_follow_a_change_of_schedule(E):
    c = C.random_smooth(3, 40, 27, 30, seed=205, mu0=0.01, du=0.05, u0=U3)
    a = make(E, c, "f32", {})
    b = make(E, c, "f32", {})
    b.set_step_graph(4)
    for kernel in (0, 1, 2, 0):
        a.set_kernel(kernel)
        b.set_kernel(kernel)
        a.step(9)
        b.step(9)
        for x, y in zip(a.fields(), b.fields()):
            assert np.array_equal(x, y), kernel
    b.set_step_graph(0)   # replays off again
    a.step(3)
    b.step(3)
    for x, y in zip(a.fields(), b.fields()):
        assert np.array_equal(x, y)
    a.close()
    b.close()
