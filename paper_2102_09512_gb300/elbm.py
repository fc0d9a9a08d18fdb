"""Thin ctypes binding of ``libelbm.so`` (C ABI in ``include/elbm.h``).

The module-level functions carry the C names and only marshal arguments; every
step of the method runs in the library's CUDA kernels.  :class:`Solver` is a
convenience wrapper that allocates the caller-owned device buffers with PyTorch
(device memory and streams only) and binds them.

There is no CPU fallback: if the library has not been built, or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libelbm.so")

ELBM_OK, ELBM_ERR_ARG, ELBM_ERR_UNSUPPORTED, ELBM_ERR_CUDA, ELBM_ERR_NONPHYSICAL, ELBM_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
ELBM_D2Q9, ELBM_D3Q27 = 9, 27
ELBM_BC_PERIODIC, ELBM_BC_ZEROGRAD, ELBM_BC_FIXED = 0, 1, 2
ELBM_EOS_GAMMA, ELBM_EOS_CV_POLY = 0, 1
ELBM_F64, ELBM_F32, ELBM_F16DEV, ELBM_BF16DEV = 0, 1, 2, 3
ELBM_DERIV_UPWIND, ELBM_DERIV_CENTRAL = 0, 1
ELBM_KERNEL_FUSED, ELBM_KERNEL_TWOPASS, ELBM_KERNEL_FUSED_REREAD, ELBM_KERNEL_FUSED_TMA = 0, 1, 2, 3
ELBM_ENSEMBLE_PERSISTENT, ELBM_ENSEMBLE_PER_INSTANCE = 0, 1
ELBM_LAYOUT_PINGPONG, ELBM_LAYOUT_AA = 0, 1

STORES = {"f64": ELBM_F64, "f32": ELBM_F32, "f16dev": ELBM_F16DEV, "bf16dev": ELBM_BF16DEV}
VALUE_BYTES = {ELBM_F64: 8, ELBM_F32: 4, ELBM_F16DEV: 2, ELBM_BF16DEV: 2}


class ElbmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {elbm_status_str(code)} ({code})")


class elbm_params(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
        ("mu0", ctypes.c_double), ("T0", ctypes.c_double), ("mu_exp", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("store", ctypes.c_int),
        ("deriv", ctypes.c_int),
        ("rho_ref", ctypes.c_double), ("T_ref", ctypes.c_double),
        ("fix_rho", ctypes.c_double), ("fix_u", ctypes.c_double * 3), ("fix_T", ctypes.c_double),
        ("eos", ctypes.c_int), ("cv", ctypes.c_double * 4),
    ]


_lib = None
_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes)
_SIGS = {
    "elbm_create": (ctypes.c_int, [ctypes.POINTER(elbm_params), ctypes.POINTER(_vp)]),
    "elbm_bytes_required": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "elbm_bind": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "elbm_set_fields": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "elbm_set_fields_device": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "elbm_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "elbm_get_fields": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "elbm_get_fields_device": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "elbm_conservation": (ctypes.c_int, [_vp, _dp]),
    "elbm_step_totals": (ctypes.c_int, [_vp, _dp]),
    "elbm_step_totals_async": (ctypes.c_int, [_vp, ctypes.c_void_p]),
    "elbm_set_step_graph": (ctypes.c_int, [_vp, ctypes.c_int]),
    "elbm_turbulence_stats": (ctypes.c_int, [_vp, _dp]),
    "elbm_set_kernel": (ctypes.c_int, [_vp, ctypes.c_int]),
    "elbm_set_layout": (ctypes.c_int, [_vp, ctypes.c_int]),
    "elbm_inject_wait_timeout": (ctypes.c_int, [_vp, ctypes.c_int]),
    "elbm_set_tile_z": (ctypes.c_int, [_vp, ctypes.c_int]),
    "elbm_get_populations": (ctypes.c_int, [_vp, _vp]),
    "elbm_set_populations": (ctypes.c_int, [_vp, _vp]),
    "elbm_sync": (ctypes.c_int, [_vp]),
    "elbm_steps_done": (ctypes.c_longlong, [_vp]),
    "elbm_launch_count": (ctypes.c_longlong, [_vp]),
    "elbm_velocity": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "elbm_destroy": (ctypes.c_int, [_vp]),
    "elbm_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "elbm_step_noalloc": (ctypes.c_int, [ctypes.POINTER(elbm_params), _vp, _vp, _vp]),
    "elbm_ensemble_create": (ctypes.c_int, [ctypes.POINTER(elbm_params), ctypes.c_int, ctypes.POINTER(_vp)]),
    "elbm_ensemble_bytes_required": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t),
                                                    ctypes.POINTER(ctypes.c_size_t)]),
    "elbm_ensemble_bind": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "elbm_ensemble_set_fields": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "elbm_ensemble_get_fields": (ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, _vp]),
    "elbm_ensemble_set_mode": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "elbm_ensemble_set_schedule": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "elbm_ensemble_get_schedule": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                  ctypes.POINTER(ctypes.c_int)]),
    "elbm_ensemble_tune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int]),
    "elbm_ensemble_step": (ctypes.c_int, [_vp, ctypes.c_int]),
    "elbm_ensemble_sync": (ctypes.c_int, [_vp]),
    "elbm_ensemble_launch_count": (ctypes.c_longlong, [_vp]),
    "elbm_ensemble_nodes": (ctypes.c_longlong, [_vp]),
    "elbm_ensemble_destroy": (ctypes.c_int, [_vp]),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libelbm.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                               "or python paper_2102_09512_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != ELBM_OK:
        raise ElbmError(rc, where)


def _ptr(a) -> int:
    """Raw pointer of a numpy array (host) or torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


# ---------------------------------------------------------------------------
# C-named thin wrappers
# ---------------------------------------------------------------------------
def elbm_status_str(code: int) -> str:
    return lib().elbm_status_str(int(code)).decode()


def elbm_create(params: elbm_params) -> int:
    h = _vp()
    _check(lib().elbm_create(ctypes.byref(params), ctypes.byref(h)), "elbm_create")
    return h.value


def elbm_bytes_required(h: int):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().elbm_bytes_required(h, ctypes.byref(a), ctypes.byref(b)), "elbm_bytes_required")
    return a.value, b.value


def elbm_bind(h: int, pop_a: int, pop_b: int, aux: int, stream: int):
    _check(lib().elbm_bind(h, pop_a, pop_b, aux, stream), "elbm_bind")


def elbm_set_fields(h, rho, u, T):
    return lib().elbm_set_fields(h, _ptr(rho), _ptr(u), _ptr(T))


def elbm_set_fields_device(h, rho, u, T):
    return lib().elbm_set_fields_device(h, _ptr(rho), _ptr(u), _ptr(T))


def elbm_step(h: int, nsteps: int):
    return lib().elbm_step(h, int(nsteps))


def elbm_get_fields(h, rho, u, T):
    return lib().elbm_get_fields(h, _ptr(rho), _ptr(u), _ptr(T))


def elbm_get_fields_device(h, rho, u, T):
    return lib().elbm_get_fields_device(h, _ptr(rho), _ptr(u), _ptr(T))


def elbm_conservation(h) -> np.ndarray:
    out = np.zeros(5)
    _check(lib().elbm_conservation(h, out.ctypes.data_as(_dp)), "elbm_conservation")
    return out


def elbm_set_step_graph(h, steps_per_graph: int):
    return lib().elbm_set_step_graph(h, int(steps_per_graph))


def elbm_step_totals_async(h, out):
    """Enqueues the step totals' copy into out (a 5-element FP64 host tensor or array,
    page-locked for an asynchronous copy); returns the status code."""
    return lib().elbm_step_totals_async(h, _ptr(out))


def elbm_step_totals(h) -> np.ndarray:
    out = np.zeros(5)
    _check(lib().elbm_step_totals(h, out.ctypes.data_as(_dp)), "elbm_step_totals")
    return out


STATS_KEYS = ("rho_mean", "rho_rms", "K", "u_rms", "theta_rms", "T_mean", "T_rms", "dudx2", "omega_rms",
              "enstrophy", "dissipation", "lambda", "Re_lambda")


def elbm_turbulence_stats(h) -> dict:
    out = np.zeros(len(STATS_KEYS))
    _check(lib().elbm_turbulence_stats(h, out.ctypes.data_as(_dp)), "elbm_turbulence_stats")
    return dict(zip(STATS_KEYS, out.tolist()))


def elbm_set_kernel(h, kernel: int):
    _check(lib().elbm_set_kernel(h, int(kernel)), "elbm_set_kernel")


def elbm_set_layout(h, layout: int):
    _check(lib().elbm_set_layout(h, int(layout)), "elbm_set_layout")


def elbm_inject_wait_timeout(h, on: int):
    _check(lib().elbm_inject_wait_timeout(h, int(on)), "elbm_inject_wait_timeout")


def elbm_set_tile_z(h, tz: int):
    _check(lib().elbm_set_tile_z(h, int(tz)), "elbm_set_tile_z")


def elbm_get_populations(h, host_dst):
    return lib().elbm_get_populations(h, _ptr(host_dst))


def elbm_set_populations(h, host_src):
    return lib().elbm_set_populations(h, _ptr(host_src))


def elbm_sync(h) -> int:
    return lib().elbm_sync(h)


def elbm_steps_done(h) -> int:
    return int(lib().elbm_steps_done(h))


def elbm_launch_count(h) -> int:
    return int(lib().elbm_launch_count(h))


def elbm_velocity(lattice: int, i: int):
    c = (ctypes.c_int * 3)()
    _check(lib().elbm_velocity(int(lattice), int(i), c), "elbm_velocity")
    return tuple(c)


def elbm_destroy(h):
    return lib().elbm_destroy(h)


def elbm_step_noalloc(params: elbm_params, src: int, dst: int, stream: int) -> int:
    """One two-pass step src -> dst without any device allocation (static scratch)."""
    return lib().elbm_step_noalloc(ctypes.byref(params), src, dst, stream)


def elbm_ensemble_create(params_list) -> int:
    arr = (elbm_params * len(params_list))(*params_list)
    h = _vp()
    _check(lib().elbm_ensemble_create(arr, len(params_list), ctypes.byref(h)), "elbm_ensemble_create")
    return h.value


def elbm_ensemble_bytes_required(e):
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().elbm_ensemble_bytes_required(e, ctypes.byref(a), ctypes.byref(b)), "elbm_ensemble_bytes_required")
    return a.value, b.value


def elbm_ensemble_bind(e, pop_a, pop_b, aux, stream):
    _check(lib().elbm_ensemble_bind(e, pop_a, pop_b, aux, stream), "elbm_ensemble_bind")


def elbm_ensemble_set_fields(e, k, rho, u, T):
    return lib().elbm_ensemble_set_fields(e, int(k), _ptr(rho), _ptr(u), _ptr(T))


def elbm_ensemble_get_fields(e, k, rho, u, T):
    return lib().elbm_ensemble_get_fields(e, int(k), _ptr(rho), _ptr(u), _ptr(T))


def elbm_ensemble_set_mode(e, mode, use_graph=1):
    _check(lib().elbm_ensemble_set_mode(e, int(mode), int(use_graph)), "elbm_ensemble_set_mode")


def elbm_ensemble_set_schedule(e, tile_y, ctas_per_sm):
    _check(lib().elbm_ensemble_set_schedule(e, int(tile_y), int(ctas_per_sm)), "elbm_ensemble_set_schedule")


def elbm_ensemble_get_schedule(e):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().elbm_ensemble_get_schedule(e, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "elbm_ensemble_get_schedule")
    return a.value, b.value, c.value


def elbm_ensemble_tune(e, trial_steps=3, use_cache=0):
    _check(lib().elbm_ensemble_tune(e, int(trial_steps), int(use_cache)), "elbm_ensemble_tune")


def elbm_ensemble_step(e, nsteps):
    return lib().elbm_ensemble_step(e, int(nsteps))


def elbm_ensemble_sync(e):
    return lib().elbm_ensemble_sync(e)


def elbm_ensemble_launch_count(e):
    return int(lib().elbm_ensemble_launch_count(e))


def elbm_ensemble_nodes(e):
    return int(lib().elbm_ensemble_nodes(e))


def elbm_ensemble_destroy(e):
    return lib().elbm_ensemble_destroy(e)


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
def make_params(lattice, nx, ny, nz=1, gamma=1.4, Pr=0.71, mu0=1e-3, T0=0.15, mu_exp=0.0,
                bc=(0, 0, 0, 0, 0, 0), store=ELBM_F32, deriv=ELBM_DERIV_UPWIND,
                rho_ref=1.0, T_ref=None, fixed=(0.0, 0.0, 0.0, 0.0, 0.0), cv=None) -> elbm_params:
    """elbm_params of a problem; fixed = (rho, u_x, u_y, u_z, T) of the ELBM_BC_FIXED faces;
    cv = None for constant Cv = 1/(gamma-1), else the coefficients of a cubic Cv(T)."""
    p = elbm_params()
    p.lattice = ELBM_D3Q27 if lattice in (3, 27, ELBM_D3Q27) else ELBM_D2Q9
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.gamma, p.Pr, p.mu0, p.T0, p.mu_exp = gamma, Pr, mu0, T0, mu_exp
    for k in range(6):
        p.bc[k] = int(bc[k])
    p.store = STORES[store] if isinstance(store, str) else int(store)
    p.deriv = int(deriv)
    p.rho_ref = rho_ref
    p.T_ref = T0 if T_ref is None else T_ref
    p.fix_rho = float(fixed[0])
    for a in range(3):
        p.fix_u[a] = float(fixed[1 + a])
    p.fix_T = float(fixed[4])
    p.eos = ELBM_EOS_GAMMA if cv is None else ELBM_EOS_CV_POLY
    for k in range(4):
        p.cv[k] = 0.0 if cv is None else float(cv[k])
    return p


class Solver:
    """One lattice with caller-owned (torch) device buffers bound to a stream."""

    def __init__(self, params: elbm_params, device="cuda", stream=None, layout=ELBM_LAYOUT_PINGPONG):
        import torch

        self.torch = torch
        self.params = params
        self.layout = layout
        self.D = 3 if params.lattice == ELBM_D3Q27 else 2
        self.N = params.nx * params.ny * params.nz
        self.h = elbm_create(params)
        try:
            if layout != ELBM_LAYOUT_PINGPONG:
                elbm_set_layout(self.h, layout)
            self.pop_bytes, self.aux_bytes = elbm_bytes_required(self.h)
            dev = torch.device(device)
            self.pop_a = torch.empty(self.pop_bytes, dtype=torch.uint8, device=dev)
            # the AA layout updates one store in place
            self.pop_b = None if layout == ELBM_LAYOUT_AA else torch.empty(self.pop_bytes, dtype=torch.uint8,
                                                                             device=dev)
            self.aux = torch.empty(self.aux_bytes, dtype=torch.uint8, device=dev)
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            elbm_bind(self.h, self.pop_a.data_ptr(), 0 if self.pop_b is None else self.pop_b.data_ptr(),
                      self.aux.data_ptr(), self.stream.cuda_stream)
        except Exception:
            elbm_destroy(self.h)
            self.h = None
            raise

    @classmethod
    def from_case(cls, case, store="f32", deriv=ELBM_DERIV_UPWIND, rho_ref=None, T_ref=None, **kw):
        rho_ref = float(np.mean(case.rho)) if rho_ref is None else rho_ref
        T_ref = float(np.mean(case.T)) if T_ref is None else T_ref
        p = make_params(case.D, case.nx, case.ny, case.nz, case.gamma, case.Pr, case.mu0, case.T0,
                        case.mu_exp, case.bc, store, deriv, rho_ref, T_ref, getattr(case, "fixed", (0,) * 5),
                        getattr(case, "cv", None))
        s = cls(p, **kw)
        s.set_fields(case.rho, case.u, case.T)
        return s

    # -- state -------------------------------------------------------------
    def set_fields(self, rho, u, T):
        if isinstance(rho, np.ndarray):
            rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(self.N)
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.D * self.N)
            T = np.ascontiguousarray(T, dtype=np.float64).reshape(self.N)
            _check(elbm_set_fields(self.h, rho, u, T), "elbm_set_fields")
        else:
            for t in (rho, u, T):
                assert t.is_cuda and t.dtype == self.torch.float64 and t.is_contiguous()
            _check(elbm_set_fields_device(self.h, rho, u, T), "elbm_set_fields_device")

    def step(self, n: int = 1):
        _check(elbm_step(self.h, n), "elbm_step")

    def set_step_graph(self, steps_per_graph: int):
        _check(elbm_set_step_graph(self.h, steps_per_graph), "elbm_set_step_graph")

    def fields(self):
        """(rho (N,), u (D, N), T (N,)) as numpy FP64 (synchronises)."""
        rho = np.empty(self.N)
        u = np.empty((self.D, self.N))
        T = np.empty(self.N)
        _check(elbm_get_fields(self.h, rho, u, T), "elbm_get_fields")
        return rho, u, T

    def fields_device(self, rho, u, T):
        _check(elbm_get_fields_device(self.h, rho, u, T), "elbm_get_fields_device")

    def conservation(self) -> np.ndarray:
        return elbm_conservation(self.h)

    def step_totals(self) -> np.ndarray:
        return elbm_step_totals(self.h)

    def turbulence_stats(self) -> dict:
        return elbm_turbulence_stats(self.h)

    def set_kernel(self, k: int):
        elbm_set_kernel(self.h, k)

    def set_tile_z(self, tz: int):
        elbm_set_tile_z(self.h, tz)

    def get_populations(self) -> np.ndarray:
        out = np.empty(self.pop_bytes, dtype=np.uint8)
        _check(elbm_get_populations(self.h, out), "elbm_get_populations")
        return out

    def set_populations(self, buf: np.ndarray):
        assert buf.dtype == np.uint8 and buf.size == self.pop_bytes
        _check(elbm_set_populations(self.h, np.ascontiguousarray(buf)), "elbm_set_populations")

    def sync(self):
        _check(elbm_sync(self.h), "elbm_sync")

    @property
    def steps_done(self) -> int:
        return elbm_steps_done(self.h)

    @property
    def launches(self) -> int:
        return elbm_launch_count(self.h)

    def close(self):
        if self.h is not None:
            elbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Independent D2Q9 lattices of uneven sizes stepped together (caller-owned
    buffers allocated with PyTorch)."""

    def __init__(self, params_list, device="cuda", stream=None):
        import torch

        self.params = list(params_list)
        self.sizes = [(p.nx, p.ny) for p in self.params]
        self.e = elbm_ensemble_create(self.params)
        try:
            pop, aux = elbm_ensemble_bytes_required(self.e)
            dev = torch.device(device)
            self.pop_a = torch.empty(pop, dtype=torch.uint8, device=dev)
            self.pop_b = torch.empty(pop, dtype=torch.uint8, device=dev)
            self.aux = torch.empty(aux, dtype=torch.uint8, device=dev)
            self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
            elbm_ensemble_bind(self.e, self.pop_a.data_ptr(), self.pop_b.data_ptr(), self.aux.data_ptr(),
                               self.stream.cuda_stream)
        except Exception:
            elbm_ensemble_destroy(self.e)
            self.e = None
            raise

    @classmethod
    def from_cases(cls, cases, store="f32", **kw):
        ps = []
        for c in cases:
            ps.append(make_params(2, c.nx, c.ny, 1, c.gamma, c.Pr, c.mu0, c.T0, c.mu_exp, c.bc, store, 0,
                                  float(np.mean(c.rho)), float(np.mean(c.T)), getattr(c, "fixed", (0,) * 5),
                                  getattr(c, "cv", None)))
        ens = cls(ps, **kw)
        for k, c in enumerate(cases):
            ens.set_fields(k, c.rho, c.u, c.T)
        return ens

    def set_fields(self, k, rho, u, T):
        nx, ny = self.sizes[k]
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(nx * ny)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(2 * nx * ny)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(nx * ny)
        _check(elbm_ensemble_set_fields(self.e, k, rho, u, T), "elbm_ensemble_set_fields")

    def fields(self, k):
        nx, ny = self.sizes[k]
        rho, u, T = np.empty(nx * ny), np.empty((2, nx * ny)), np.empty(nx * ny)
        _check(elbm_ensemble_get_fields(self.e, k, rho, u, T), "elbm_ensemble_get_fields")
        return rho, u, T

    def set_mode(self, mode, use_graph=True):
        elbm_ensemble_set_mode(self.e, mode, 1 if use_graph else 0)

    def set_schedule(self, tile_y, ctas_per_sm):
        elbm_ensemble_set_schedule(self.e, tile_y, ctas_per_sm)

    def schedule(self):
        return elbm_ensemble_get_schedule(self.e)

    def tune(self, trial_steps=3, use_cache=False):
        elbm_ensemble_tune(self.e, trial_steps, 1 if use_cache else 0)
        return self.schedule()

    def step(self, n=1):
        _check(elbm_ensemble_step(self.e, n), "elbm_ensemble_step")

    def sync(self):
        _check(elbm_ensemble_sync(self.e), "elbm_ensemble_sync")

    @property
    def nodes(self):
        return elbm_ensemble_nodes(self.e)

    @property
    def launches(self):
        return elbm_ensemble_launch_count(self.e)

    def close(self):
        if self.e is not None:
            elbm_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
