"""ctypes wrapper of the FP64 CPU oracle (oracle/hydro_oracle.{hpp,cpp}).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product package.  The oracle shares
no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "hydro_oracle.cpp")]
_HDR = [os.path.join(_HERE, "hydro_oracle.hpp")]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NVAR = 5
NG = 2


class Config(ctypes.Structure):
    """Mirror of ho::Config."""
    _fields_ = [
        ("nx", ctypes.c_int32 * 3),
        ("nb", ctypes.c_int32 * 3),
        ("xmin", ctypes.c_double * 3),
        ("xmax", ctypes.c_double * 3),
        ("max_level", ctypes.c_int32),
        ("adaptive", ctypes.c_int32),
        ("gamma", ctypes.c_double),
        ("cfl", ctypes.c_double),
        ("dfloor", ctypes.c_double),
        ("pfloor", ctypes.c_double),
        ("refine_tol", ctypes.c_double),
        ("derefine_tol", ctypes.c_double),
        ("derefine_count", ctypes.c_int32),
        ("static_region", ctypes.c_int32),
        ("static_lo", ctypes.c_double * 3),
        ("static_hi", ctypes.c_double * 3),
        ("bc", ctypes.c_int32 * 6),
        ("nscalars", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


BC = {"periodic": 0, "outflow": 1, "reflect": 2}


def make_config(nx, nb, xmin=(-0.5, -0.5, -0.5), xmax=(0.5, 0.5, 0.5), gamma=5.0 / 3.0, cfl=0.3,
                max_level=0, adaptive=0, dfloor=1e-12, pfloor=1e-12, refine_tol=0.05,
                derefine_tol=0.0125, derefine_count=10, static_region=0,
                static_lo=(-0.2, -0.2, -0.2), static_hi=(0.2, 0.2, 0.2), bc=None,
                nscalars=0) -> Config:
    """bc: None (all periodic) or 6 entries, names or codes, for the faces
    x1 inner, x1 outer, x2 inner, x2 outer, x3 inner, x3 outer."""
    c = Config()
    c.nx[:] = list(nx)
    c.nb[:] = list(nb)
    c.xmin[:] = list(xmin)
    c.xmax[:] = list(xmax)
    c.max_level = max_level
    c.adaptive = adaptive
    c.gamma = gamma
    c.cfl = cfl
    c.dfloor = dfloor
    c.pfloor = pfloor
    c.refine_tol = refine_tol
    c.derefine_tol = derefine_tol
    c.derefine_count = derefine_count
    c.static_region = static_region
    c.static_lo[:] = list(static_lo)
    c.static_hi[:] = list(static_hi)
    c.bc[:] = [BC[b] if isinstance(b, str) else int(b) for b in (bc or ["periodic"] * 6)]
    c.nscalars = int(nscalars)
    return c


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, -O2 -ffp-contract=off: no contraction)."""
    newest = max(os.path.getmtime(p) for p in _SRC + _HDR)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + _SRC
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            i8p = ctypes.POINTER(ctypes.c_int8)
            cfgp = ctypes.POINTER(Config)
            sig = {
                "or_create": (P, [cfgp]),
                "or_destroy": (None, [P]),
                "or_num_blocks": (ctypes.c_int, [P]),
                "or_tree": (None, [P, i64p]),
                "or_set_state": (None, [P, dp]),
                "or_get_state": (None, [P, dp]),
                "or_get_full": (None, [P, dp]),
                "or_fill_ghosts": (None, [P]),
                "or_compute_dt": (ctypes.c_double, [P]),
                "or_step": (None, [P, ctypes.c_int, dp]),
                "or_step_dt": (None, [P, ctypes.c_int, dp]),
                "or_stage": (None, [P, ctypes.c_int, dp, ctypes.c_double]),
                "or_get_time": (None, [P, dp, dp, i64p]),
                "or_totals": (None, [P, dp]),
                "or_floor_hits": (ctypes.c_long, [P]),
                "or_tag": (None, [P, i8p, dp]),
                "or_remesh": (ctypes.c_int, [P, i8p, ctypes.c_int]),
                "or_composite": (None, [P, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_int64, dp]),
                "or_cons_to_prim": (None, [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
                "or_vanleer": (ctypes.c_double, [ctypes.c_double] * 3),
                "or_minmod": (ctypes.c_double, [ctypes.c_double] * 2),
                "or_hlle": (None, [dp, dp, ctypes.c_int, ctypes.c_double, dp]),
                "or_morton": (ctypes.c_uint64, [ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                ctypes.c_int64, ctypes.c_int]),
                "or_jvp": (None, [cfgp, dp, dp, ctypes.c_double, dp, ctypes.c_int, dp,
                                  ctypes.c_double, dp, dp]),
                "or_jvp_state": (None, [cfgp, dp, dp, ctypes.c_double, ctypes.c_int, dp,
                                        ctypes.c_double, dp, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class OracleMesh:
    """One oracle mesh (uniform or multi-level) with its state."""

    def __init__(self, cfg: Config):
        if not 0 <= cfg.nscalars <= 2:
            raise ValueError("0 .. 2 passive scalars")
        self.cfg = cfg
        self.L = lib()
        self.h = self.L.or_create(ctypes.byref(cfg))
        self.nx = tuple(cfg.nx)
        self.nv = NVAR + int(cfg.nscalars)   # conserved variables per cell

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.or_destroy(h)
            self.h = None

    @property
    def nblocks(self) -> int:
        return self.L.or_num_blocks(self.h)

    def tree(self) -> np.ndarray:
        out = np.zeros((self.nblocks, 4), dtype=np.int64)
        self.L.or_tree(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return out

    def state_shape(self):
        return (self.nblocks, self.nv, self.nx[2], self.nx[1], self.nx[0])

    def set_state(self, U: np.ndarray):
        U = np.ascontiguousarray(U, dtype=np.float64)
        assert U.shape == self.state_shape(), (U.shape, self.state_shape())
        self.L.or_set_state(self.h, _dp(U))

    def get_state(self) -> np.ndarray:
        U = np.zeros(self.state_shape(), dtype=np.float64)
        self.L.or_get_state(self.h, _dp(U))
        return U

    def get_full(self) -> np.ndarray:
        S = [n + 2 * NG for n in self.nx]
        U = np.zeros((self.nblocks, self.nv, S[2], S[1], S[0]), dtype=np.float64)
        self.L.or_get_full(self.h, _dp(U))
        return U

    def fill_ghosts(self):
        self.L.or_fill_ghosts(self.h)

    def compute_dt(self) -> float:
        return self.L.or_compute_dt(self.h)

    def step(self, n: int) -> np.ndarray:
        dts = np.zeros(max(n, 1), dtype=np.float64)
        self.L.or_step(self.h, n, _dp(dts))
        return dts[:n]

    def step_dt(self, dts):
        dts = np.ascontiguousarray(dts, dtype=np.float64)
        self.L.or_step_dt(self.h, len(dts), _dp(dts))

    def stage(self, which: int, U0: np.ndarray, dt: float):
        U0 = np.ascontiguousarray(U0, dtype=np.float64)
        self.L.or_stage(self.h, which, _dp(U0), dt)

    def time(self):
        t = np.zeros(1)
        dt = np.zeros(1)
        cyc = np.zeros(1, dtype=np.int64)
        self.L.or_get_time(self.h, _dp(t), _dp(dt), cyc.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
        return float(t[0]), float(dt[0]), int(cyc[0])

    def totals(self) -> np.ndarray:
        out = np.zeros(NVAR + 2)
        self.L.or_totals(self.h, _dp(out))
        return out[:self.nv]

    def floor_hits(self) -> int:
        return int(self.L.or_floor_hits(self.h))

    def tag(self):
        flags = np.zeros(self.nblocks, dtype=np.int8)
        mb = np.zeros(self.nblocks, dtype=np.float64)
        self.L.or_tag(self.h, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), _dp(mb))
        return flags, mb

    def remesh(self, flags, check_age: bool = True) -> bool:
        flags = np.ascontiguousarray(flags, dtype=np.int8)
        assert flags.shape == (self.nblocks,)
        return bool(self.L.or_remesh(self.h, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                                     1 if check_age else 0))

    def composite(self, level, I, J, K) -> np.ndarray:
        out = np.zeros(NVAR + 2)
        self.L.or_composite(self.h, level, I, J, K, _dp(out))
        return out[:self.nv]


def cons_to_prim(u, gamma, dfloor=1e-12, pfloor=1e-12):
    u = np.ascontiguousarray(u, dtype=np.float64)
    w = np.zeros(NVAR)
    lib().or_cons_to_prim(_dp(u), _dp(w), gamma, dfloor, pfloor)
    return w


def vanleer(a, b, c) -> float:
    return lib().or_vanleer(a, b, c)


def minmod(a, b) -> float:
    return lib().or_minmod(a, b)


def hlle(wl, wr, direction: int, gamma: float) -> np.ndarray:
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(NVAR)
    lib().or_hlle(_dp(wl), _dp(wr), direction, gamma, _dp(f))
    return f


def morton(level, l1, l2, l3, max_level) -> int:
    return int(lib().or_morton(level, l1, l2, l3, max_level))


def jvp_state(cfg: Config, U0, V, dgamma, dts, h=1e-30):
    """Complex-step tangent J V of the final state (and the final state itself)."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    Uo = np.zeros_like(U0)
    JV = np.zeros_like(U0)
    lib().or_jvp_state(ctypes.byref(cfg), _dp(U0), _dp(V), dgamma, len(dts), _dp(dts), h, _dp(Uo),
                       _dp(JV))
    return Uo, JV


def jvp(cfg: Config, U0, V, dgamma, rho_target, dts, h=1e-30):
    """Complex-step directional derivative of J = sum (rho_final - rho_target)^2."""
    U0 = np.ascontiguousarray(U0, dtype=np.float64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    rt = np.ascontiguousarray(rho_target, dtype=np.float64)
    dts = np.ascontiguousarray(dts, dtype=np.float64)
    J = np.zeros(1)
    dJ = np.zeros(1)
    lib().or_jvp(ctypes.byref(cfg), _dp(U0), _dp(V), dgamma, _dp(rt), len(dts), _dp(dts), h,
                 _dp(J), _dp(dJ))
    return float(J[0]), float(dJ[0])
