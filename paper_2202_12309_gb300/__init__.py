"""Python binding of libphhydro.so (include/ph_hydro.h): argument marshalling only.

Every step of the hydro cycle runs in the library's CUDA kernels; this module
only converts Python arguments into the C ABI's plain pointers and sizes.
PyTorch is used for device memory (its caching allocator backs the library's
allocations) and streams.  There is no CPU fallback: if the shared library is
missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libphhydro.so")

PH_OK = 0
PH_ERR = {-1: "PH_ERR_INVALID", -2: "PH_ERR_OOM", -3: "PH_ERR_NONPHYSICAL", -4: "PH_ERR_TIMEOUT",
          -5: "PH_ERR_CUDA", -6: "PH_ERR_STATE", -7: "PH_ERR_IO"}
PH_FP64 = 0
PH_FP32 = 1

EXPORTS = [
    "ph_set_allocator", "ph_last_error", "ph_create", "ph_destroy", "ph_num_blocks", "ph_tree",
    "ph_set_state", "ph_get_state", "ph_get_full", "ph_step", "ph_get_dt", "ph_get_next_dt",
    "ph_get_time", "ph_totals", "ph_tag", "ph_refine_where", "ph_refine_by_density", "ph_status",
    "ph_fill_ghosts", "ph_launches_per_cycle", "ph_get_tile", "ph_profile_cycles",
    "ph_totals_noalloc",
    "ph_batch_create", "ph_batch_destroy", "ph_batch_num_blocks", "ph_batch_set_state",
    "ph_batch_get_state", "ph_batch_step", "ph_batch_get_dt", "ph_batch_get_time",
    "ph_batch_status", "ph_batch_get_launch", "ph_batch_set_launch", "ph_batch_autotune",
    "ph_debug_barrier_timeout", "ph_step_dt", "ph_adjoint", "ph_debug_math", "ph_debug_fma_rate",
    "ph_save", "ph_load", "ph_set_state_async", "ph_get_state_async",
    "ph_create_shard", "ph_shard_halo", "ph_shard_stage", "ph_shard_pack", "ph_shard_unpack",
    "ph_shard_rate", "ph_shard_finish", "ph_shards_sync", "ph_shards_step", "ph_shard_plan",
]


class PhError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (PH_ERR.get(code, "PH_ERR"), code, msg))
        self.code = code


class Config(ctypes.Structure):
    """Mirror of ph_config."""
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
        ("precision", ctypes.c_int32),
        ("tile", ctypes.c_int32 * 3),
        ("bc", ctypes.c_int32 * 6),
        ("nscalars", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


BC = {"periodic": 0, "outflow": 1, "reflect": 2}


def make_config(nx, nb, xmin=(-0.5, -0.5, -0.5), xmax=(0.5, 0.5, 0.5), gamma=5.0 / 3.0, cfl=0.3,
                max_level=0, adaptive=0, dfloor=None, pfloor=None, refine_tol=0.05,
                derefine_tol=0.0125, derefine_count=10, static_region=0,
                static_lo=(-0.2, -0.2, -0.2), static_hi=(0.2, 0.2, 0.2), precision="fp64",
                tile=(0, 0, 0), bc=None, nscalars=0) -> Config:
    """bc: None (periodic everywhere) or 6 entries, names ("periodic",
    "outflow", "reflect") or PH_BC_* codes, for the faces x1 inner, x1 outer,
    x2 inner, x2 outer, x3 inner, x3 outer."""
    prec = PH_FP32 if precision in ("fp32", PH_FP32) else PH_FP64
    if dfloor is None:
        dfloor = 1e-7 if prec == PH_FP32 else 1e-12
    if pfloor is None:
        pfloor = 1e-7 if prec == PH_FP32 else 1e-12
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
    c.precision = prec
    c.tile[:] = list(tile)
    c.bc[:] = [BC[b] if isinstance(b, str) else int(b) for b in (bc or ["periodic"] * 6)]
    c.nscalars = int(nscalars)
    return c


_lib = None
_alloc_refs = None


def lib():
    """Load libphhydro.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libphhydro.so is missing: run paper_2202_12309_gb300/build.py "
                              "(or __graft_entry__.build()) first")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.c_void_p
        i32, i64 = ctypes.c_int32, ctypes.c_int64
        dp = ctypes.POINTER(ctypes.c_double)
        sig = {
            "ph_set_allocator": [P, P, P],
            "ph_create": [ctypes.POINTER(Config), P, ctypes.POINTER(P)],
            "ph_destroy": [P],
            "ph_num_blocks": [P, ctypes.POINTER(i32)],
            "ph_tree": [P, ctypes.POINTER(i64), i32],
            "ph_set_state": [P, P, i64, i32],
            "ph_get_state": [P, P, i64, i32],
            "ph_get_full": [P, P, i64, i32],
            "ph_step": [P, i32],
            "ph_get_dt": [P, dp],
            "ph_get_next_dt": [P, dp],
            "ph_get_time": [P, dp, ctypes.POINTER(i64)],
            "ph_totals": [P, dp],
            "ph_tag": [P, ctypes.POINTER(ctypes.c_int8), dp, i32],
            "ph_refine_where": [P, ctypes.POINTER(ctypes.c_int8), i32, i32, ctypes.POINTER(i32)],
            "ph_refine_by_density": [P, ctypes.POINTER(i32)],
            "ph_status": [P, ctypes.POINTER(i64), ctypes.POINTER(i32)],
            "ph_fill_ghosts": [P],
            "ph_launches_per_cycle": [P, ctypes.POINTER(i32)],
            "ph_get_tile": [P, ctypes.POINTER(i32)],
            "ph_profile_cycles": [P, i32, dp, i32],
            "ph_totals_noalloc": [P, i32, ctypes.POINTER(i32), i32, i32, P, dp, i32, P, P],
            "ph_batch_create": [ctypes.POINTER(Config), i32, P, ctypes.POINTER(P)],
            "ph_batch_destroy": [P],
            "ph_batch_num_blocks": [P, i32, ctypes.POINTER(i32)],
            "ph_batch_set_state": [P, i32, P, i64, i32],
            "ph_batch_get_state": [P, i32, P, i64, i32],
            "ph_batch_step": [P, i32],
            "ph_batch_get_dt": [P, dp],
            "ph_batch_get_time": [P, dp, ctypes.POINTER(i64)],
            "ph_batch_status": [P, ctypes.POINTER(i64), ctypes.POINTER(i32)],
            "ph_batch_get_launch": [P, ctypes.POINTER(i32)],
            "ph_batch_set_launch": [P, ctypes.POINTER(i32)],
            "ph_batch_autotune": [P, i32, ctypes.POINTER(i32)],
            "ph_debug_barrier_timeout": [P, i32, i64, ctypes.POINTER(i32)],
            "ph_step_dt": [P, i32, dp],
            "ph_adjoint": [P, P, i32, i32, dp, P, P, dp, i32],
            "ph_debug_math": [i32, i32, P, P, i64, P],
            "ph_debug_fma_rate": [i32, i32, i64, P, P],
            "ph_save": [P, ctypes.c_char_p, i32],
            "ph_set_state_async": [P, P, i64, i32],
            "ph_get_state_async": [P, P, i64, i32],
            "ph_load": [ctypes.c_char_p, P, ctypes.POINTER(P)],
            "ph_create_shard": [ctypes.POINTER(Config), i32, i32, P, ctypes.POINTER(P)],
            "ph_shard_halo": [P, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64),
                              ctypes.POINTER(i64), ctypes.POINTER(i64)],
            "ph_shard_stage": [P, i32],
            "ph_shard_pack": [P, i32, P],
            "ph_shard_unpack": [P, i32, P],
            "ph_shard_rate": [P, i32, P],
            "ph_shard_finish": [P, i32, P],
            "ph_shards_sync": [ctypes.POINTER(P), i32],
            "ph_shards_step": [ctypes.POINTER(P), i32, i32],
            "ph_shard_plan": [ctypes.POINTER(Config), i32, i32, i32, ctypes.POINTER(i64), ctypes.POINTER(i64),
                              ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.ph_last_error.restype = ctypes.c_char_p
        L.ph_last_error.argtypes = []
        _lib = L
    return _lib


def check(rc: int):
    if rc != PH_OK:
        raise PhError(rc, lib().ph_last_error().decode())


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_refs
    import torch

    ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
    FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

    def _alloc(nbytes, stream, ctx):
        return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream or 0)))

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = ALLOC(_alloc), FREE(_free)
    check(lib().ph_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None))
    _alloc_refs = (a, f)


def totals_noalloc(U, nx, nblocks, out, precision="fp64", nvar=5, level=None, vol=(1.0,),
                   stream: Optional[int] = None):
    """ph_totals_noalloc on caller-owned device tensors (U packed interior
    state of nvar variables per cell, out nvar doubles, level int8 per block
    or None); vol[l] is the cell volume of level l.  The library allocates
    nothing for this call."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    n3 = (ctypes.c_int32 * 3)(*nx)
    prec = PH_FP32 if precision in ("fp32", PH_FP32) else PH_FP64
    vols = np.ascontiguousarray(vol, dtype=np.float64)
    if 0 <= int(nblocks) <= 16384 and 5 <= int(nvar) <= 7:  # else rejected by the library itself
        _check_buffer(U, int(nblocks) * int(nvar) * nx[0] * nx[1] * nx[2], 4 if prec == PH_FP32 else 8, "U")
        _check_buffer(out, int(nvar), 8, "out")
        if level is not None:
            _check_buffer(level, int(nblocks), 1, "level")
    if not (U.is_cuda and out.is_cuda) or (level is not None and not level.is_cuda):
        raise ValueError("U, out and level must be device tensors")
    lvl = ctypes.c_void_p(level.data_ptr()) if level is not None else None
    check(lib().ph_totals_noalloc(ctypes.c_void_p(U.data_ptr()), prec, n3, int(nvar), int(nblocks), lvl,
                                  vols.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(vols),
                                  ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream)))


def _ptr(x):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr(), (1 if x.is_cuda else 0)


def _count(x) -> int:
    """Number of elements actually held by x (passed to the C ABI, which
    rejects a count that does not match the mesh)."""
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


def _itemsize(x) -> int:
    return int(x.itemsize) if isinstance(x, np.ndarray) else int(x.element_size())


def _check_buffer(x, count: int, itemsize: int, what: str):
    if _count(x) != count or _itemsize(x) != itemsize:
        raise ValueError("%s: expected %d elements of %d bytes, got %d of %d"
                         % (what, count, itemsize, _count(x), _itemsize(x)))


class Mesh:
    """A GPU mesh (uniform or two-level) with its conserved state."""

    def __init__(self, cfg: Config, stream: Optional[int] = None, shard: Optional[Tuple[int, int]] = None):
        """shard = (nshards, s): shard s of the uniform mesh cfg (ph_create_shard)."""
        if stream is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the GB300 hydro library has no CPU path")
            stream = torch.cuda.current_stream().cuda_stream
        self.L = lib()
        self.cfg = cfg
        self.h = ctypes.c_void_p()
        if shard is None:
            check(self.L.ph_create(ctypes.byref(cfg), ctypes.c_void_p(stream), ctypes.byref(self.h)))
        else:
            check(self.L.ph_create_shard(ctypes.byref(cfg), int(shard[0]), int(shard[1]), ctypes.c_void_p(stream),
                                         ctypes.byref(self.h)))
        self.nx = tuple(cfg.nx)
        self.nvar = 5 + int(cfg.nscalars)
        self.dtype = np.float32 if cfg.precision == PH_FP32 else np.float64

    @classmethod
    def load(cls, path: str, stream: Optional[int] = None) -> "Mesh":
        """ph_load: a new mesh from a file written by save()."""
        if stream is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the GB300 hydro library has no CPU path")
            stream = torch.cuda.current_stream().cuda_stream
        L = lib()
        h = ctypes.c_void_p()
        check(L.ph_load(os.fsencode(path), ctypes.c_void_p(stream), ctypes.byref(h)))
        self = cls.__new__(cls)
        self.L = L
        self.h = h
        cfg = Config()
        # the configuration lives in the file's header, after magic, version
        # and precision (8 + 4 + 4 bytes)
        with open(path, "rb") as f:
            f.seek(16)
            f.readinto(cfg)
        self.cfg = cfg
        self.nx = tuple(cfg.nx)
        self.nvar = 5 + int(cfg.nscalars)
        self.dtype = np.float32 if cfg.precision == PH_FP32 else np.float64
        return self

    def save(self, path: str, precision: Optional[str] = None):
        """ph_save: restart file (default: the mesh's own precision) or an
        output of the given precision ("fp64" / "fp32")."""
        if precision is None:
            prec = self.cfg.precision
        else:
            prec = PH_FP32 if precision == "fp32" else PH_FP64
        check(self.L.ph_save(self.h, os.fsencode(path), prec))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.ph_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nblocks(self) -> int:
        n = ctypes.c_int32()
        check(self.L.ph_num_blocks(self.h, ctypes.byref(n)))
        return n.value

    def tree(self) -> np.ndarray:
        n = self.nblocks
        out = np.zeros((n, 4), dtype=np.int64)
        check(self.L.ph_tree(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n))
        return out

    def state_shape(self):
        return (self.nblocks, self.nvar, self.nx[2], self.nx[1], self.nx[0])

    def count(self) -> int:
        return int(np.prod(self.state_shape()))

    def set_state(self, U, sync: bool = True):
        """Copy a state in.  sync=False queues it on the mesh's stream
        (ph_set_state_async): U must then stay alive and unchanged until the
        stream has passed the copy (page-locked memory for overlap)."""
        if isinstance(U, np.ndarray):
            if not sync and not (U.flags.c_contiguous and U.dtype == self.dtype):
                raise ValueError("an asynchronous copy needs a contiguous array of the mesh's dtype")
            U = np.ascontiguousarray(U, dtype=self.dtype)
        p, dev = _ptr(U)
        # the element count of the buffer itself: the ABI rejects a mismatch
        fn = self.L.ph_set_state if sync else self.L.ph_set_state_async
        check(fn(self.h, ctypes.c_void_p(p), _count(U), dev))

    def get_state(self, out=None, sync: bool = True):
        """Copy the state out.  sync=False queues the copy on the mesh's
        stream (ph_get_state_async); read `out` after synchronising it."""
        if out is None:
            out = np.zeros(self.state_shape(), dtype=self.dtype)
        p, dev = _ptr(out)
        fn = self.L.ph_get_state if sync else self.L.ph_get_state_async
        check(fn(self.h, ctypes.c_void_p(p), _count(out), dev))
        return out

    def get_full(self) -> np.ndarray:
        S = [n + 4 for n in self.nx]
        out = np.zeros((self.nblocks, self.nvar, S[2], S[1], S[0]), dtype=self.dtype)
        check(self.L.ph_get_full(self.h, ctypes.c_void_p(out.ctypes.data), out.size, 0))
        return out

    def step(self, n: int = 1):
        check(self.L.ph_step(self.h, int(n)))

    def dt(self) -> float:
        v = ctypes.c_double()
        check(self.L.ph_get_dt(self.h, ctypes.byref(v)))
        return v.value

    def next_dt(self) -> float:
        v = ctypes.c_double()
        check(self.L.ph_get_next_dt(self.h, ctypes.byref(v)))
        return v.value

    def time(self):
        t = ctypes.c_double()
        c = ctypes.c_int64()
        check(self.L.ph_get_time(self.h, ctypes.byref(t), ctypes.byref(c)))
        return t.value, c.value

    def totals(self) -> np.ndarray:
        out = np.zeros(self.nvar)
        check(self.L.ph_totals(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def tag(self):
        n = self.nblocks
        flags = np.zeros(n, dtype=np.int8)
        mb = np.zeros(n, dtype=np.float64)
        check(self.L.ph_tag(self.h, flags.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)),
                            mb.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n))
        return flags, mb

    def refine_where(self, flags: Sequence[int], check_age: bool = True) -> bool:
        f = np.ascontiguousarray(flags, dtype=np.int8)
        ch = ctypes.c_int32()
        check(self.L.ph_refine_where(self.h, f.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)), len(f),
                                     1 if check_age else 0, ctypes.byref(ch)))
        return bool(ch.value)

    def refine_by_density(self) -> bool:
        ch = ctypes.c_int32()
        check(self.L.ph_refine_by_density(self.h, ctypes.byref(ch)))
        return bool(ch.value)

    def status(self):
        fh = ctypes.c_int64()
        nf = ctypes.c_int32()
        rc = self.L.ph_status(self.h, ctypes.byref(fh), ctypes.byref(nf))
        return rc, fh.value, nf.value

    def fill_ghosts(self):
        check(self.L.ph_fill_ghosts(self.h))

    def launches_per_cycle(self) -> int:
        n = ctypes.c_int32()
        check(self.L.ph_launches_per_cycle(self.h, ctypes.byref(n)))
        return n.value

    def profile(self, ncycles: int) -> np.ndarray:
        """Summed device ms per launch slot over ncycles (stage1, ghost, stage2, ghost, dt)."""
        ms = np.zeros(5)
        check(self.L.ph_profile_cycles(self.h, int(ncycles),
                                       ms.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 5))
        return ms

    def step_dt(self, dts):
        """Cycles with prescribed dts (host array)."""
        d = np.ascontiguousarray(dts, dtype=np.float64)
        check(self.L.ph_step_dt(self.h, len(d), d.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def adjoint(self, U0, dLdU, ncycles: int, ckpt_every: int = 5, dts=None, out=None):
        """(dL/dU0, dL/dgamma) for a loss of the state after ncycles from U0.
        U0, dLdU (and out) are numpy arrays or CUDA tensors in the interior
        layout; dts fixes the dt schedule (None: the forward run's CFL dts)."""
        if isinstance(U0, np.ndarray):
            U0 = np.ascontiguousarray(U0, dtype=self.dtype)
            dLdU = np.ascontiguousarray(dLdU, dtype=self.dtype)
            if out is None:
                out = np.zeros_like(U0)
        elif out is None:
            import torch
            out = torch.empty_like(U0)
        isz = np.dtype(self.dtype).itemsize
        for buf, what in ((U0, "U0"), (dLdU, "dLdU"), (out, "out")):
            _check_buffer(buf, self.count(), isz, what)
        p0, dev = _ptr(U0)
        pg, dev2 = _ptr(dLdU)
        po, dev3 = _ptr(out)
        if not dev == dev2 == dev3:
            raise ValueError("U0, dLdU and out must all be host arrays or all device tensors")
        dptr = None
        if dts is not None:
            dts = np.ascontiguousarray(dts, dtype=np.float64)
            assert len(dts) == ncycles
            dptr = dts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        g = ctypes.c_double()
        check(self.L.ph_adjoint(self.h, ctypes.c_void_p(p0), int(ncycles), int(ckpt_every), dptr,
                                ctypes.c_void_p(pg), ctypes.c_void_p(po), ctypes.byref(g), dev))
        return out, g.value

    def tile(self):
        t = (ctypes.c_int32 * 3)()
        check(self.L.ph_get_tile(self.h, t))
        return tuple(t)


class Batch:
    """Independent uniform meshes advanced together by one persistent launch per cycle."""

    def __init__(self, cfgs, stream: Optional[int] = None):
        if stream is None:
            import torch
            if not torch.cuda.is_available():
                raise RuntimeError("no CUDA device: the GB300 hydro library has no CPU path")
            stream = torch.cuda.current_stream().cuda_stream
        self.L = lib()
        arr = (Config * len(cfgs))(*cfgs)
        self.cfgs = list(cfgs)
        self.nsim = len(cfgs)
        self.h = ctypes.c_void_p()
        check(self.L.ph_batch_create(arr, self.nsim, ctypes.c_void_p(stream), ctypes.byref(self.h)))
        self.dtype = np.float32 if cfgs[0].precision == PH_FP32 else np.float64

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            self.L.ph_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nblocks(self, sim: int) -> int:
        n = ctypes.c_int32()
        check(self.L.ph_batch_num_blocks(self.h, sim, ctypes.byref(n)))
        return n.value

    def state_shape(self, sim: int):
        nx = tuple(self.cfgs[sim].nx)
        return (self.nblocks(sim), 5, nx[2], nx[1], nx[0])

    def set_state(self, sim: int, U):
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=self.dtype)
        p, dev = _ptr(U)
        check(self.L.ph_batch_set_state(self.h, sim, ctypes.c_void_p(p), _count(U), dev))

    def get_state(self, sim: int, out=None):
        if out is None:
            out = np.zeros(self.state_shape(sim), dtype=self.dtype)
        p, dev = _ptr(out)
        check(self.L.ph_batch_get_state(self.h, sim, ctypes.c_void_p(p), _count(out), dev))
        return out

    def step(self, n: int = 1):
        check(self.L.ph_batch_step(self.h, int(n)))

    def dt(self) -> np.ndarray:
        out = np.zeros(self.nsim)
        check(self.L.ph_batch_get_dt(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def time(self):
        t = np.zeros(self.nsim)
        c = np.zeros(self.nsim, dtype=np.int64)
        check(self.L.ph_batch_get_time(self.h, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       c.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
        return t, c

    def status(self):
        fh = ctypes.c_int64()
        nf = ctypes.c_int32()
        rc = self.L.ph_batch_status(self.h, ctypes.byref(fh), ctypes.byref(nf))
        return rc, fh.value, nf.value

    def launch(self):
        c = (ctypes.c_int32 * 4)()
        check(self.L.ph_batch_get_launch(self.h, c))
        return tuple(c)

    def set_launch(self, choice):
        c = (ctypes.c_int32 * 4)(*choice)
        check(self.L.ph_batch_set_launch(self.h, c))

    def autotune(self, trial_cycles: int = 2):
        c = (ctypes.c_int32 * 4)()
        check(self.L.ph_batch_autotune(self.h, int(trial_cycles), c))
        return tuple(c)


def debug_barrier_timeout(nctas: int = 4, spin_limit: int = 1 << 16, stream: Optional[int] = None):
    """Run the barrier self test; returns (return code, CTAs that gave up)."""
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    g = ctypes.c_int32()
    rc = lib().ph_debug_barrier_timeout(ctypes.c_void_p(stream), int(nctas), int(spin_limit),
                                        ctypes.byref(g))
    return rc, g.value


MATH_FN = {"rcp": 0, "rsqrt": 1, "sqrt": 2, "rcp_approx": 3, "rsqrt_approx": 4}


def debug_math(fn: str, x):
    """Evaluate the stage kernels' reciprocal / root routine `fn` on the CUDA
    tensor x (float64 or float32); returns a new tensor on x's stream."""
    import torch
    if not (x.is_cuda and x.is_contiguous() and x.dtype in (torch.float64, torch.float32)):
        raise ValueError("x must be a contiguous float64/float32 CUDA tensor")
    y = torch.empty_like(x)
    prec = PH_FP64 if x.dtype == torch.float64 else PH_FP32
    check(lib().ph_debug_math(MATH_FN[fn], prec, ctypes.c_void_p(x.data_ptr()),
                              ctypes.c_void_p(y.data_ptr()), x.numel(),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return y


FMA_KIND = {"fp64": 0, "fp32": 1, "fp32x2": 2}


def debug_fma_rate(kind: str, ctas: int, iters: int, out, stream: Optional[int] = None):
    """Queue the multiply-add throughput probe (ph_debug_fma_rate) on the
    stream: `out` is a CUDA tensor of ctas * 256 elements (float64 for
    "fp64", float32 otherwise).  Returns the flops the launch performs."""
    import torch
    k = FMA_KIND[kind]
    want = torch.float64 if k == 0 else torch.float32
    if not (out.is_cuda and out.is_contiguous() and out.dtype == want and out.numel() == ctas * 256):
        raise ValueError("out must be a contiguous %s CUDA tensor of %d elements" % (want, ctas * 256))
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    check(lib().ph_debug_fma_rate(k, int(ctas), int(iters), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(stream)))
    return ctas * 256 * iters * 16 * (2 if k == 2 else 1)


def _hydro_run_function():
    import torch

    class HydroRun(torch.autograd.Function):
        """U_final = hydro(U0, gamma) over `ncycles` cycles of a uniform mesh.

        forward: set_state + ncycles cycles (the CFL dts are recorded);
        backward: ph_adjoint with that dt schedule (frozen) and
        checkpoint-every-k recomputation: gradients w.r.t. U0 and gamma."""

        @staticmethod
        def forward(ctx, U0, gamma, cfg, ncycles, ckpt_every):
            import copy
            c = copy.copy(cfg)
            c.gamma = float(gamma)
            m = Mesh(c)
            U0c = U0.detach().contiguous()
            m.set_state(U0c)
            dts = []
            for _ in range(int(ncycles)):
                m.step(1)
                dts.append(m.dt())
            out = torch.empty_like(U0c)
            m.get_state(out)
            ctx.save_for_backward(U0c)
            ctx.cfg = c
            ctx.ncycles = int(ncycles)
            ctx.ckpt = int(ckpt_every)
            ctx.dts = np.asarray(dts)
            m.close()
            return out

        @staticmethod
        def backward(ctx, gout):
            (U0,) = ctx.saved_tensors
            m = Mesh(ctx.cfg)
            gU0, gg = m.adjoint(U0, gout.contiguous(), ctx.ncycles, ctx.ckpt, dts=ctx.dts)
            m.close()
            return gU0, torch.tensor(gg, dtype=torch.float64), None, None, None

    return HydroRun


def hydro_run(U0, gamma, cfg: Config, ncycles: int, ckpt_every: int = 5):
    """Differentiable hydro run: see HydroRun (torch.autograd.Function)."""
    global _HydroRun
    if "_HydroRun" not in globals():
        _HydroRun = _hydro_run_function()
    return _HydroRun.apply(U0, gamma, cfg, ncycles, ckpt_every)


# ---------------------------------------------------------------------------
# Domain decomposition (ph_create_shard and the ph_shard_* calls): argument
# marshalling for shards of one process (ShardedMesh) and for one shard per
# process over torch.distributed (DistShard).
# ---------------------------------------------------------------------------

def shard_plan(cfg: Config, nshards: int, shard: int, peer: int):
    """ph_shard_plan (host only, no GPU needed): the receiving-cell keys that
    `shard` sends to and receives from `peer`, and its global leaf range."""
    L = lib()
    i64p = ctypes.POINTER(ctypes.c_int64)
    ns, nr = ctypes.c_int64(0), ctypes.c_int64(0)
    rng = (ctypes.c_int64 * 2)()
    check(L.ph_shard_plan(ctypes.byref(cfg), nshards, shard, peer, None, ctypes.byref(ns), None,
                          ctypes.byref(nr), rng))
    send = np.zeros(ns.value, dtype=np.int64)
    recv = np.zeros(nr.value, dtype=np.int64)
    check(L.ph_shard_plan(ctypes.byref(cfg), nshards, shard, peer, send.ctypes.data_as(i64p), ctypes.byref(ns),
                          recv.ctypes.data_as(i64p), ctypes.byref(nr), rng))
    return send, recv, (int(rng[0]), int(rng[1]))


class Shard(Mesh):
    """Shard s of nshards of a uniform mesh: a mesh of its own leaves."""

    def __init__(self, cfg: Config, nshards: int, s: int, stream: Optional[int] = None):
        super().__init__(cfg, stream=stream, shard=(nshards, s))
        self.nshards, self.shard = int(nshards), int(s)

    def halo(self, peer: int):
        """(send entries, send offset, recv entries, recv offset) with peer,
        and the shard's global leaf range."""
        v = [ctypes.c_int64() for _ in range(4)]
        rng = (ctypes.c_int64 * 2)()
        check(self.L.ph_shard_halo(self.h, peer, *[ctypes.byref(x) for x in v], rng))
        return tuple(x.value for x in v), (int(rng[0]), int(rng[1]))

    def stage(self, stage: int):
        check(self.L.ph_shard_stage(self.h, stage))

    def pack(self, pool: int, buf):
        check(self.L.ph_shard_pack(self.h, pool, ctypes.c_void_p(buf.data_ptr())))

    def unpack(self, pool: int, buf):
        check(self.L.ph_shard_unpack(self.h, pool, ctypes.c_void_p(buf.data_ptr())))

    def rate(self, recompute: int, d_rate):
        check(self.L.ph_shard_rate(self.h, recompute, ctypes.c_void_p(d_rate.data_ptr())))

    def finish(self, first: int, d_rate):
        check(self.L.ph_shard_finish(self.h, first, ctypes.c_void_p(d_rate.data_ptr())))


class ShardedMesh:
    """All shards of a uniform mesh in this process (ph_shards_sync /
    ph_shards_step), with the global state in the layout of Mesh (blocks in
    Z-order) split by the shards' leaf ranges."""

    def __init__(self, cfg: Config, nshards: int, devices: Optional[Sequence[int]] = None):
        import torch
        self.cfg = cfg
        self.shards: List[Shard] = []
        self.streams = []
        for s in range(nshards):
            dev = devices[s] if devices else torch.cuda.current_device()
            with torch.cuda.device(dev):
                st = torch.cuda.Stream(device=dev)
                self.streams.append(st)
                self.shards.append(Shard(cfg, nshards, s, stream=st.cuda_stream))
        self.ranges = [sh.halo(0)[1] for sh in self.shards] if nshards > 1 else [(0, self.shards[0].nblocks)]
        self._handles = (ctypes.c_void_p * nshards)(*[sh.h.value for sh in self.shards])

    @property
    def nblocks(self) -> int:
        return self.ranges[-1][1]

    def tree(self) -> np.ndarray:
        return np.concatenate([sh.tree() for sh in self.shards])

    def set_state(self, U: np.ndarray):
        for sh, (a, b) in zip(self.shards, self.ranges):
            sh.set_state(np.ascontiguousarray(U[a:b]))
        check(lib().ph_shards_sync(self._handles, len(self.shards)))

    def step(self, n: int = 1):
        check(lib().ph_shards_step(self._handles, len(self.shards), int(n)))

    def get_state(self) -> np.ndarray:
        return np.concatenate([sh.get_state() for sh in self.shards])

    def dt(self) -> float:
        return self.shards[0].dt()

    def time(self):
        return self.shards[0].time()

    def close(self):
        for sh in self.shards:
            sh.close()


def reduce_rate_max(r, dist):
    """Max of one signal rate (a one-element float64 tensor) over the ranks
    of the default process group, in place.  A NaN rate (a non-finite state
    on some rank) becomes +inf first: the max of floating-point values with
    a NaN among them depends on the backend, +inf wins on all of them, and
    dt = cfl / inf = 0 is reported as non-finite by the dt bookkeeping."""
    import torch
    r.copy_(torch.where(torch.isnan(r), torch.full_like(r, float("inf")), r))
    dist.all_reduce(r, op=dist.ReduceOp.MAX)
    return r


class DistShard:
    """One shard per process of a torch.distributed group: shard `rank` of
    `world` on the current device, with the halo exchange as point-to-point
    messages (device buffers with NCCL, host-staged with gloo) and the dt as
    an all-reduce max."""

    def __init__(self, cfg: Config):
        import torch
        import torch.distributed as dist
        self.dist, self.torch = dist, torch
        self.rank, self.world = dist.get_rank(), dist.get_world_size()
        self.host = dist.get_backend() == "gloo"
        self.m = Shard(cfg, self.world, self.rank)
        self.nvar = self.m.nvar
        tdt = torch.float32 if cfg.precision == PH_FP32 else torch.float64
        self.peers = []
        nsend = nrecv = 0
        for p in range(self.world):
            if p == self.rank:
                continue
            (ns, so, nr, ro), self.range = self.m.halo(p)
            self.peers.append((p, ns, so, nr, ro))
            nsend, nrecv = max(nsend, so + ns), max(nrecv, ro + nr)
        dev = torch.device("cuda", torch.cuda.current_device())
        self.send = torch.empty(max(nsend, 1) * self.nvar, dtype=tdt, device=dev)
        self.recv = torch.empty(max(nrecv, 1) * self.nvar, dtype=tdt, device=dev)
        self.rate_d = torch.zeros(1, dtype=torch.float64, device=dev)

    def _exchange(self, pool: int):
        torch, dist, nv = self.torch, self.dist, self.nvar
        self.m.pack(pool, self.send)
        torch.cuda.current_stream().synchronize()
        send = self.send.cpu() if self.host else self.send
        recv = torch.empty_like(self.recv, device="cpu") if self.host else self.recv
        ops = []
        for p, ns, so, nr, ro in self.peers:
            if ns:
                ops.append(dist.P2POp(dist.isend, send[so * nv:(so + ns) * nv], p))
            if nr:
                ops.append(dist.P2POp(dist.irecv, recv[ro * nv:(ro + nr) * nv], p))
        if ops:
            for w in dist.batch_isend_irecv(ops):
                w.wait()
        if self.host:
            self.recv.copy_(recv)
        self.m.unpack(pool, self.recv)

    def _dt(self, recompute: int, first: int):
        torch, dist = self.torch, self.dist
        self.m.rate(recompute, self.rate_d)
        torch.cuda.current_stream().synchronize()
        r = self.rate_d.cpu() if self.host else self.rate_d
        reduce_rate_max(r, dist)
        if self.host:
            self.rate_d.copy_(r)
        self.m.finish(first, self.rate_d)

    def set_state(self, U_local: np.ndarray):
        """This shard's blocks (global leaves self.range) of the state."""
        self.m.set_state(U_local)
        self._exchange(0)
        self._dt(1, 1)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.m.stage(1)
            self._exchange(1)
            self.m.stage(2)
            self._exchange(0)
            self._dt(0, 0)

    def get_state(self) -> np.ndarray:
        return self.m.get_state()
