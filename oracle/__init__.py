"""FP64 CPU oracle of the two-population compressible lattice Boltzmann model
(arXiv:2102.09512, Sec. II and Sec. III.A).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the bench's
CPU-baseline leg load it; the product package never imports it.  The arithmetic
lives in ``elbm_oracle.c`` (plain C, FP64); this module builds it with gcc and
marshals numpy arrays through ctypes.  It shares no code with the CUDA library.

State layout here is node-major: ``f[n, i]`` with ``n = x + nx*(y + ny*z)`` and
direction ``i`` with components ``c_a = ((i // 3**a) % 3) - 1``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over nodes) into oracle/_build."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("D", ctypes.c_int),
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("gamma", ctypes.c_double), ("Pr", ctypes.c_double),
        ("mu0", ctypes.c_double), ("T0", ctypes.c_double), ("mu_exp", ctypes.c_double),
        ("bc", ctypes.c_int * 6),
        ("deriv", ctypes.c_int),
        ("correction", ctypes.c_int),
        ("fix_rho", ctypes.c_double), ("fix_u", ctypes.c_double * 3), ("fix_T", ctypes.c_double),
        ("eos", ctypes.c_int), ("cv", ctypes.c_double * 4),
    ]


@dataclass
class Params:
    """Problem statement of the method: lattice, grid, gamma, Pr, mu law, BCs."""
    D: int = 2
    nx: int = 8
    ny: int = 8
    nz: int = 1
    gamma: float = 1.4
    Pr: float = 0.71
    mu0: float = 1e-3
    T0: float = 0.15
    mu_exp: float = 0.0
    bc: tuple = (0, 0, 0, 0, 0, 0)
    deriv: int = 0
    correction: int = 1
    fixed: tuple = (0.0, 0.0, 0.0, 0.0, 0.0)   # (rho, u_x, u_y, u_z, T) of fixed-state faces (bc 2)
    cv: tuple = None   # None: constant Cv = 1/(gamma-1); else Cv(T) = cv[0] + cv[1] T + cv[2] T^2 + cv[3] T^3

    @property
    def Q(self) -> int:
        return 27 if self.D == 3 else 9

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    def c_struct(self) -> _Params:
        s = _Params()
        s.D, s.nx, s.ny, s.nz = self.D, self.nx, self.ny, self.nz
        s.gamma, s.Pr, s.mu0, s.T0, s.mu_exp = self.gamma, self.Pr, self.mu0, self.T0, self.mu_exp
        for k in range(6):
            s.bc[k] = int(self.bc[k])
        s.deriv = self.deriv
        s.correction = self.correction
        s.fix_rho = float(self.fixed[0])
        for a in range(3):
            s.fix_u[a] = float(self.fixed[1 + a])
        s.fix_T = float(self.fixed[4])
        s.eos = 0 if self.cv is None else 1
        for k in range(4):
            s.cv[k] = 0.0 if self.cv is None else float(self.cv[k])
        return s


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        L = _lib
        L.orc_init.argtypes = [pp, dp, dp, dp, dp, dp]
        L.orc_step.argtypes = [pp, dp, dp, ctypes.c_int]
        L.orc_fields.argtypes = [pp, dp, dp, dp, dp, dp]
        L.orc_conservation.argtypes = [pp, dp, dp, dp]
        L.orc_fex.argtypes = [pp, ctypes.c_double, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_geq.argtypes = [pp, ctypes.c_double, dp, ctypes.c_double, dp]
        L.orc_energy_moments.argtypes = [pp, ctypes.c_double, dp, ctypes.c_double, dp]
        L.orc_rates.argtypes = [pp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_collide_node.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_velocity.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.orc_set_threads.argtypes = [ctypes.c_int]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps the current one); returns it."""
    return int(lib().orc_set_threads(int(n)))


def velocities(D: int) -> np.ndarray:
    """The oracle's velocity set, shape (Q, 3) (Eq. d3q27vel and its 2D analogue)."""
    Q = 27 if D == 3 else 9
    out = np.zeros((Q, 3), dtype=np.int64)
    c3 = (ctypes.c_int * 3)()
    for i in range(Q):
        lib().orc_velocity(D, i, c3)
        out[i] = list(c3)
    return out


def _vec3(u) -> np.ndarray:
    v = np.zeros(3, dtype=np.float64)
    v[: len(u)] = u
    return v


def feq(p: Params, rho: float, u, T: float) -> np.ndarray:
    """Product-form equilibrium f^eq (Eq. 27eq)."""
    out = np.zeros(p.Q)
    lib().orc_fex(ctypes.byref(p.c_struct()), rho, _dp(_vec3(u)), T, 1.0, None, _dp(out))
    return out


def fex(p: Params, rho: float, u, T: float, omega: float, dQ) -> np.ndarray:
    """Extended equilibrium f^ex (Eqs. extf, Pa_star) for derivative values dQ_a."""
    out = np.zeros(p.Q)
    lib().orc_fex(ctypes.byref(p.c_struct()), rho, _dp(_vec3(u)), T, omega, _dp(_vec3(dQ)), _dp(out))
    return out


def geq(p: Params, rho: float, u, T: float) -> np.ndarray:
    """Operator product-form energy equilibrium g^eq (Eq. geq_i)."""
    out = np.zeros(p.Q)
    lib().orc_geq(ctypes.byref(p.c_struct()), rho, _dp(_vec3(u)), T, _dp(out))
    return out


def energy_moments(p: Params, rho: float, u, T: float) -> np.ndarray:
    """G_lmn = rho O_x^l O_y^m O_z^n E for l,m,n <= 2 (Eq. Ecompact), shape (3,3,3)."""
    out = np.zeros(27)
    lib().orc_energy_moments(ctypes.byref(p.c_struct()), rho, _dp(_vec3(u)), T, _dp(out))
    return out.reshape(3, 3, 3)


def rates(p: Params, rho: float, T: float):
    """(omega, omega_1) from mu and Pr (Eqs. mu, Pr)."""
    w = ctypes.c_double()
    w1 = ctypes.c_double()
    lib().orc_rates(ctypes.byref(p.c_struct()), rho, T, ctypes.byref(w), ctypes.byref(w1))
    return w.value, w1.value


def collide_node(p: Params, f: np.ndarray, g: np.ndarray, dQ):
    """One collision at one node; returns dict with f_post, g_post, fex, geq, gstar."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = {k: np.zeros(p.Q) for k in ("f_post", "g_post", "fex", "geq", "gstar")}
    lib().orc_collide_node(ctypes.byref(p.c_struct()), _dp(f), _dp(g), _dp(_vec3(dQ)),
                           _dp(out["f_post"]), _dp(out["g_post"]), _dp(out["fex"]),
                           _dp(out["geq"]), _dp(out["gstar"]))
    return out


@dataclass
class State:
    p: Params
    f: np.ndarray = field(repr=False)
    g: np.ndarray = field(repr=False)


def init(p: Params, rho: np.ndarray, u: np.ndarray, T: np.ndarray) -> State:
    """f = f^eq, g = g^eq of the given fields.  rho, T: (N,); u: (D, N); node order
    n = x + nx*(y + ny*z) (arrays shaped (nz, ny, nx) flatten to it)."""
    N, Q = p.N, p.Q
    rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(N)
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(N)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(p.D, N)
    f = np.zeros((N, Q))
    g = np.zeros((N, Q))
    lib().orc_init(ctypes.byref(p.c_struct()), _dp(rho), _dp(u), _dp(T), _dp(f), _dp(g))
    return State(p, f, g)


def step(s: State, nsteps: int = 1) -> State:
    rc = lib().orc_step(ctypes.byref(s.p.c_struct()), _dp(s.f), _dp(s.g), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle step could not allocate its work arrays")
    return s


def fields(s: State):
    """(rho (N,), u (D, N), T (N,)) of the current populations."""
    p = s.p
    rho = np.zeros(p.N)
    u = np.zeros((p.D, p.N))
    T = np.zeros(p.N)
    lib().orc_fields(ctypes.byref(p.c_struct()), _dp(s.f), _dp(s.g), _dp(rho), _dp(u), _dp(T))
    return rho, u, T


def conservation(s: State) -> np.ndarray:
    """[sum rho, sum rho u_x, sum rho u_y, sum rho u_z, sum rho E], compensated FP64."""
    out = np.zeros(5)
    lib().orc_conservation(ctypes.byref(s.p.c_struct()), _dp(s.f), _dp(s.g), _dp(out))
    return out
