"""elbm_step_noalloc: the entry point for callers that cannot allocate device memory
(an application that owns the device memory pool and lends the library only the
population stores).  Its scratch lives in a fixed static device array instead of the
handle's auxiliary buffer.  The test calls it through the C ABI twice in a row
(A -> B, then B -> A) and compares the result with the existing handle API running
the same two-pass schedule for two steps.  The test itself allocates its buffers
with PyTorch; the entry point allocates nothing.

The rejection of grids beyond the static scratch is checked without a GPU, before any
launch could happen (tests/test_host_logic.py): a test of a size guard should not rely
on that guard to keep a kernel inside its buffers.

This file is named to be collected last, so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

from paper_2102_09512_gb300 import cases as C

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def E():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2102_09512_gb300 import build as B
    B.build()
    from paper_2102_09512_gb300 import elbm
    return elbm


def rel_l2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("D,store", [(3, "f64"), (3, "f32"), (2, "f32")])
def test_noalloc_step_matches_handle_api(E, D, store):
    import torch
    shape = (29, 17, 11) if D == 3 else (45, 23, 1)
    c = C.random_smooth(D, *shape, seed=91, mu0=0.01, du=0.05, u0=(0.09, -0.07, 0.06))

    # existing entry points: handle API, two-pass schedule, two steps
    ref = E.Solver.from_case(c, store=store)
    ref.set_kernel(E.ELBM_KERNEL_TWOPASS)
    start = ref.get_populations()
    ref.step(2)
    ref_pops = ref.get_populations()
    ref_fields = ref.fields()
    params = ref.params

    # the allocation-free entry point on caller-owned stores, two calls in a row
    stream = torch.cuda.current_stream()
    a = torch.from_numpy(start).cuda()
    b = torch.empty_like(a)
    assert a.data_ptr() % 256 == 0 and b.data_ptr() % 256 == 0
    assert E.elbm_step_noalloc(params, a.data_ptr(), b.data_ptr(), stream.cuda_stream) == E.ELBM_OK
    assert E.elbm_step_noalloc(params, b.data_ptr(), a.data_ptr(), stream.cuda_stream) == E.ELBM_OK
    torch.cuda.synchronize()
    got_pops = a.cpu().numpy()

    # same kernels, same scratch contents: identical populations
    assert np.array_equal(got_pops, ref_pops)
    # and, through the handle's field extraction, the same fields within the parity tolerance
    chk = E.Solver(params)
    chk.set_populations(got_pops)
    for x, y in zip(chk.fields(), ref_fields):
        assert rel_l2(x, y) <= TOL[store]
    ref.close()
    chk.close()

