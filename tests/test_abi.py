"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
symbol that include/elbm.h declares, and validates parameters on the host
(elbm_create and elbm_bytes_required make no CUDA call)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2102_09512_gb300 import build as B
    B.build()
    from paper_2102_09512_gb300 import elbm as E
    return E


def declared_symbols():
    with open(os.path.join(ROOT, "include", "elbm.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(elbm_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 20
    lib = L.lib()
    for n in names:
        assert hasattr(lib, n), n
    # and the binding wraps each of them under the same name
    for n in names:
        assert hasattr(L, n), n


def test_status_strings(L):
    for code in (0, -1, -2, -3, -4, -5):
        assert L.elbm_status_str(code)


def test_velocity_table(L):
    for lat, Q in ((L.ELBM_D2Q9, 9), (L.ELBM_D3Q27, 27)):
        cs = {L.elbm_velocity(lat, i) for i in range(Q)}
        assert len(cs) == Q
        for i in range(Q):
            c = L.elbm_velocity(lat, i)
            assert i == (c[0] + 1) + 3 * (c[1] + 1) + (9 * (c[2] + 1) if Q == 27 else 0)


def test_create_and_sizes(L):
    p = L.make_params(3, 64, 48, 40, store="f32")
    h = L.elbm_create(p)
    pop, aux = L.elbm_bytes_required(h)
    assert pop == 2 * 27 * 64 * 48 * 40 * 4
    assert aux >= 3 * 64 * 48 * 40 * 4 + 5 * 64 * 48 * 40 * 8
    L.elbm_destroy(h)
    p = L.make_params(2, 100, 30, 1, store="f16dev")
    h = L.elbm_create(p)
    pop, _ = L.elbm_bytes_required(h)
    assert pop == 2 * 9 * 3000 * 2
    L.elbm_destroy(h)


@pytest.mark.parametrize("field,value", [
    ("lattice", 19), ("nx", 0), ("nz", 2), ("gamma", 1.0), ("Pr", 0.0), ("mu0", -1.0),
    ("T0", 0.0), ("store", 7), ("deriv", 3),
])
def test_create_rejects_bad_arguments(L, field, value):
    p = L.make_params(2, 16, 16, 1)
    setattr(p, field, value)
    with pytest.raises(L.ElbmError) as ei:
        L.elbm_create(p)
    assert ei.value.code == L.ELBM_ERR_ARG


def test_create_rejects_mixed_axis_bc(L):
    p = L.make_params(2, 16, 16, 1, bc=(0, 1, 0, 0, 0, 0))
    with pytest.raises(L.ElbmError):
        L.elbm_create(p)


def test_unbound_handle_is_rejected(L):
    h = L.elbm_create(L.make_params(2, 16, 16, 1))
    assert L.elbm_step(h, 1) == L.ELBM_ERR_ARG
    L.elbm_destroy(h)


def test_fixed_state_faces_are_validated(L):
    fixed = (1.0, 0.3, 0.0, 0.0, 0.05)
    h = L.elbm_create(L.make_params(2, 32, 16, 1, bc=(2, 1, 0, 0, 0, 0), fixed=fixed))
    L.elbm_destroy(h)
    with pytest.raises(L.ElbmError) as ei:   # the fixed state must be physical
        L.elbm_create(L.make_params(2, 32, 16, 1, bc=(2, 1, 0, 0, 0, 0), fixed=(0.0, 0.3, 0.0, 0.0, 0.05)))
    assert ei.value.code == L.ELBM_ERR_ARG
    with pytest.raises(L.ElbmError) as ei:   # D2Q9 only
        L.elbm_create(L.make_params(3, 16, 16, 16, bc=(2, 1, 0, 0, 0, 0), fixed=fixed))
    assert ei.value.code == L.ELBM_ERR_UNSUPPORTED
    with pytest.raises(L.ElbmError):          # a fixed face cannot pair with a periodic one
        L.elbm_create(L.make_params(2, 32, 16, 1, bc=(2, 0, 0, 0, 0, 0), fixed=fixed))


def test_caloric_eos_is_validated(L):
    h = L.elbm_create(L.make_params(3, 16, 16, 16, cv=(1.0, 4.0, -4.0, 5.0)))
    L.elbm_destroy(h)
    for cv in ((0.0, 1.0, 0.0, 0.0), (1.0, float("nan"), 0.0, 0.0)):
        with pytest.raises(L.ElbmError) as ei:
            L.elbm_create(L.make_params(2, 16, 16, 1, cv=cv))
        assert ei.value.code == L.ELBM_ERR_ARG
    p = L.make_params(2, 16, 16, 1)
    p.eos = 7
    with pytest.raises(L.ElbmError) as ei:
        L.elbm_create(p)
    assert ei.value.code == L.ELBM_ERR_ARG


def test_tma_schedule_eligibility(L):
    """The TMA-staged D3Q27 schedule needs FP32/FP16/BF16 pairs and nx a multiple of 2
    (FP32) or 4 (FP16/BF16), the tensor map's row pitch being a multiple of 16 bytes; any
    boundary types (host-only check in elbm_set_kernel)."""
    ok = [(64, "f32", (0,) * 6), (38, "f32", (1,) * 6), (6, "f32", (0,) * 6), (40, "f16dev", (1, 1, 0, 0, 1, 1)),
          (48, "bf16dev", (0,) * 6)]
    bad = [(37, "f32"), (42, "f16dev"), (38, "bf16dev"), (64, "f64")]
    for nx, store, bc in ok:
        h = L.elbm_create(L.make_params(3, nx, 12, 10, store=store, bc=bc))
        L.elbm_set_kernel(h, L.ELBM_KERNEL_FUSED_TMA)
        L.elbm_destroy(h)
    for nx, store in bad:
        h = L.elbm_create(L.make_params(3, nx, 12, 10, store=store))
        with pytest.raises(L.ElbmError) as ei:
            L.elbm_set_kernel(h, L.ELBM_KERNEL_FUSED_TMA)
        assert ei.value.code == L.ELBM_ERR_UNSUPPORTED, (nx, store)
        L.elbm_destroy(h)
    h = L.elbm_create(L.make_params(2, 64, 12, 1, store="f32"))
    with pytest.raises(L.ElbmError) as ei:
        L.elbm_set_kernel(h, L.ELBM_KERNEL_FUSED_TMA)
    assert ei.value.code == L.ELBM_ERR_UNSUPPORTED
    L.elbm_destroy(h)


def test_wait_timeout_injection_arguments(L):
    h = L.elbm_create(L.make_params(3, 64, 24, 8, store="f32"))
    L.elbm_inject_wait_timeout(h, 1)
    L.elbm_inject_wait_timeout(h, 0)
    with pytest.raises(L.ElbmError) as ei:
        L.elbm_inject_wait_timeout(h, 2)
    assert ei.value.code == L.ELBM_ERR_ARG
    L.elbm_destroy(h)


def test_grid_size_limit(L):
    """Node indices are 32-bit: N = 2^31 nodes is the largest grid a handle accepts."""
    h = L.elbm_create(L.make_params(3, 2048, 1024, 1024, store="f16dev"))
    L.elbm_destroy(h)
    with pytest.raises(L.ElbmError) as ei:
        L.elbm_create(L.make_params(3, 2048, 1024, 1025, store="f16dev"))
    assert ei.value.code == L.ELBM_ERR_UNSUPPORTED


def test_aa_layout_host_checks(L):
    """The single-store (AA) layout: periodic grids only, selected before binding, the
    two-pass schedule only, and a staging area of at most 2^25 nodes for host transfers."""
    p = L.make_params(3, 64, 48, 40, store="f32")
    h = L.elbm_create(p)
    L.elbm_set_layout(h, L.ELBM_LAYOUT_AA)
    pop, aux = L.elbm_bytes_required(h)
    assert pop == 2 * 27 * 64 * 48 * 40 * 4   # the size of one store
    assert L.lib().elbm_set_kernel(h, L.ELBM_KERNEL_FUSED) == L.ELBM_ERR_UNSUPPORTED
    assert L.lib().elbm_set_kernel(h, L.ELBM_KERNEL_FUSED_REREAD) == L.ELBM_ERR_UNSUPPORTED
    assert L.lib().elbm_set_kernel(h, L.ELBM_KERNEL_TWOPASS) == L.ELBM_OK
    assert L.lib().elbm_set_layout(h, 7) == L.ELBM_ERR_ARG
    L.elbm_destroy(h)
    # a zero-gradient axis: two nodes would read a slot that one of them writes
    for bc in [(1, 1, 0, 0, 0, 0), (0, 0, 0, 0, 1, 1)]:
        h = L.elbm_create(L.make_params(3, 16, 16, 16, bc=bc, store="f64"))
        assert L.lib().elbm_set_layout(h, L.ELBM_LAYOUT_AA) == L.ELBM_ERR_UNSUPPORTED
        L.elbm_destroy(h)
    # 1024^3 FP32: one store of 232 GB and a small auxiliary buffer (Q~ field and a
    # chunk-sized staging area) fit a GB300, where ping-pong stores would not
    h = L.elbm_create(L.make_params(3, 1024, 1024, 1024, store="f32"))
    pp_pop, pp_aux = L.elbm_bytes_required(h)
    L.elbm_set_layout(h, L.ELBM_LAYOUT_AA)
    pop, aux = L.elbm_bytes_required(h)
    n = 1024 ** 3
    assert pop == pp_pop == 27 * n * 8
    assert aux < 3 * n * 4 + (5 * 8 << 25) + (1 << 30)
    assert pop + aux < 260e9 < 2 * pp_pop
    L.elbm_destroy(h)


def test_step_graph_host_checks(L):
    """Graph-replayed steps: an even group size of at most 1024 (0 turns replays off);
    nothing is captured before the handle is bound (no CUDA call here)."""
    h = L.elbm_create(L.make_params(2, 800, 4, 1, store="f64"))
    for bad in (-2, 1, 3, 1026):
        assert L.lib().elbm_set_step_graph(h, bad) == L.ELBM_ERR_ARG
    for ok in (0, 2, 8, 1024):
        assert L.lib().elbm_set_step_graph(h, ok) == L.ELBM_OK
    assert L.lib().elbm_step(h, 4) == L.ELBM_ERR_ARG   # not bound
    L.elbm_destroy(h)
