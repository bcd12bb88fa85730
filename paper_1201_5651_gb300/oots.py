"""Thin Python binding of the C ABI in include/oots.h (ctypes; argument
marshalling only -- every step of the path runs in the CUDA library).

The functions below keep the C names (``oots_create``, ``oots_advance`` ...);
``Context`` and ``Batch`` wrap them for convenience.  Loading fails loudly if
the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import _build

OOTS_OK = 0
OOTS_E_INVAL = -1
OOTS_E_STATE = -2
OOTS_E_NOMEM = -3
OOTS_E_CUDA = -4
OOTS_E_DEVICE_TIMEOUT = -5
OOTS_E_UNSUPPORTED = -6

OOTS_FP64 = 0
OOTS_MIXED = 1
OOTS_A1, OOTS_A2, OOTS_A3 = 1, 2, 3
OOTS_MONO, OOTS_BLACKBODY = 0, 1

# every symbol include/oots.h declares
EXPORTS = [
    "oots_create", "oots_destroy", "oots_set_stream", "oots_last_error", "oots_reset_error",
    "oots_set_grid", "oots_set_density", "oots_set_neutral_fraction", "oots_set_physics",
    "oots_add_source", "oots_clear_sources", "oots_set_scheme", "oots_dtcrit_preset",
    "oots_compute_dt", "oots_step", "oots_advance", "oots_get_neutral_fraction",
    "oots_get_column_density", "oots_get_budget", "oots_reset_budget", "oots_get_time", "oots_set_time",
    "oots_set_neutral_fraction_device", "oots_get_neutral_fraction_device", "oots_synchronize",
    "oots_batch_create", "oots_batch_advance", "oots_batch_destroy", "oots_set_tile_shape",
    "oots_tile_shape_info", "oots_debug_set", "oots_version", "oots_run_substeps", "oots_profile_substep",
    "oots_trace_noalloc", "oots_add_plane_source", "oots_batch_run_substeps",
    "oots_set_partition", "oots_run_phase", "oots_array_device",
]
OOTS_PH_TRACE1, OOTS_PH_DT, OOTS_PH_STEP1, OOTS_PH_TRACE2, OOTS_PH_FULL = 0, 1, 2, 3, 4
KERNEL_KINDS = {1: "sweep1", 2: "ratedt", 3: "final0", 4: "half", 5: "sweep2", 6: "full", 7: "final1", 8: "implicit",
                9: "half_general", 10: "full_general", 11: "plane_trace", 12: "plane_implicit",
                13: "pack", 14: "ratedt_verify"}


class OotsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"oots error {code}: {msg}")
        self.code = code


class dtcrit(ctypes.Structure):
    _fields_ = [("K1", ctypes.c_double), ("K2", ctypes.c_double), ("K3", ctypes.c_double),
                ("K4", ctypes.c_double), ("dt_fixed", ctypes.c_double)]


class budget(ctypes.Structure):
    _fields_ = [("emitted", ctypes.c_double), ("absorbed", ctypes.c_double), ("ions", ctypes.c_double),
                ("recombinations", ctypes.c_double)]


_lib = None


def library_path() -> str:
    return _build.lib_path()


def load(build_if_missing: bool = True):
    """Load the compiled library (building it in-tree if it is missing and a
    CUDA toolkit is present).  Raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path) or _build._stale(path):
        if not build_if_missing:
            raise ImportError(f"CUDA library not built: {path}")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "oots_create": ([P(vp), ip, ip], ip),
        "oots_destroy": ([vp], ip),
        "oots_set_stream": ([vp, vp], ip),
        "oots_last_error": ([vp], ctypes.c_char_p),
        "oots_reset_error": ([vp], ip),
        "oots_set_grid": ([vp, ip, ip, ip, dp], ip),
        "oots_set_density": ([vp, vp, dp], ip),
        "oots_set_neutral_fraction": ([vp, vp, dp], ip),
        "oots_set_physics": ([vp, dp, dp, dp, dp], ip),
        "oots_add_source": ([vp, P(dp), dp, ip, dp, P(ip)], ip),
        "oots_add_plane_source": ([vp, ip, ip, dp, ip, dp, P(ip)], ip),
        "oots_clear_sources": ([vp], ip),
        "oots_set_scheme": ([vp, ip, P(dtcrit)], ip),
        "oots_dtcrit_preset": ([ip, ip, P(dtcrit)], ip),
        "oots_compute_dt": ([vp, P(dp)], ip),
        "oots_step": ([vp, dp], ip),
        "oots_advance": ([vp, dp, P(dp), P(ctypes.c_longlong)], ip),
        "oots_get_neutral_fraction": ([vp, vp], ip),
        "oots_get_column_density": ([vp, ip, vp], ip),
        "oots_get_budget": ([vp, P(budget)], ip),
        "oots_reset_budget": ([vp], ip),
        "oots_get_time": ([vp, P(dp), P(ctypes.c_longlong)], ip),
        "oots_set_time": ([vp, dp], ip),
        "oots_set_neutral_fraction_device": ([vp, vp, ip], ip),
        "oots_get_neutral_fraction_device": ([vp, vp, ip], ip),
        "oots_synchronize": ([vp], ip),
        "oots_batch_create": ([P(vp), P(vp), ip], ip),
        "oots_batch_advance": ([vp, P(dp), P(ctypes.c_longlong)], ip),
        "oots_batch_destroy": ([vp], ip),
        "oots_batch_run_substeps": ([vp, ctypes.c_longlong, P(dp)], ip),
        "oots_set_partition": ([vp, ctypes.c_ulonglong, ip, ip], ip),
        "oots_run_phase": ([vp, ip, P(dp)], ip),
        "oots_array_device": ([vp, ip, ip, P(vp), P(ctypes.c_ulonglong)], ip),
        "oots_set_tile_shape": ([vp, ip], ip),
        "oots_tile_shape_info": ([ip, P(ip)], ip),
        "oots_debug_set": ([vp, ip, ctypes.c_longlong], ip),
        "oots_version": ([], ctypes.c_char_p),
        "oots_run_substeps": ([vp, ctypes.c_longlong, dp], ip),
        "oots_profile_substep": ([vp, P(ip), P(dp), ip, P(ip)], ip),
        "oots_trace_noalloc": ([ip, ip, ip, ip, ip, dp, vp, dp, vp, P(dp), dp, dp, vp, vp, P(ip)], ip),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(rc: int, ctx=None):
    if rc != OOTS_OK:
        raise OotsError(rc, load().oots_last_error(ctx).decode())
    return rc


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------- C-named wrappers
def oots_create(device: int = 0, precision: int = OOTS_FP64):
    h = ctypes.c_void_p()
    _check(load().oots_create(ctypes.byref(h), device, precision))
    return h


def oots_destroy(ctx):
    return _check(load().oots_destroy(ctx))


def oots_version() -> str:
    return load().oots_version().decode()


def oots_dtcrit_preset(id: int, scheme: int) -> dtcrit:
    c = dtcrit()
    _check(load().oots_dtcrit_preset(id, scheme, ctypes.byref(c)))
    return c


def oots_trace_noalloc(device: int, precision: int, nx: int, ny: int, nz: int, dx: float, n_ptr, uniform_n: float,
                       x_ptr: int, pos, sigma0: float, tau0: float, nin_ptr: int, stream_ptr=None):
    """Column trace into caller-owned device buffers without any allocation
    (pointers are device addresses, e.g. torch tensors' data_ptr())."""
    p = (ctypes.c_double * 3)(*[float(v) for v in pos])
    detail = ctypes.c_int(0)
    rc = load().oots_trace_noalloc(int(device), int(precision), int(nx), int(ny), int(nz), float(dx),
                                   ctypes.c_void_p(n_ptr) if n_ptr else None, float(uniform_n), ctypes.c_void_p(x_ptr),
                                   p, float(sigma0), float(tau0), ctypes.c_void_p(nin_ptr),
                                   ctypes.c_void_p(stream_ptr) if stream_ptr else None, ctypes.byref(detail))
    if rc != OOTS_OK:
        raise OotsError(rc, load().oots_last_error(None).decode() + f" (detail {detail.value})")
    return rc


def oots_tile_shape_info(shape: int):
    d = (ctypes.c_int * 3)()
    n = load().oots_tile_shape_info(shape, d)
    if n < 0:
        raise OotsError(n, load().oots_last_error(None).decode())
    return n, tuple(d)


class Context:
    """One grid with its sources and scheme (wraps an oots_ctx)."""

    def __init__(self, device: int = 0, precision: str = "fp64"):
        self.lib = load()
        self.precision = OOTS_FP64 if precision in ("fp64", OOTS_FP64) else OOTS_MIXED
        self.h = oots_create(device, self.precision)
        self.shape = None

    def close(self):
        if self.h is not None:
            self.lib.oots_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        return _check(rc, self.h)

    # grid and state
    def set_grid(self, nx, ny, nz, dx):
        self.shape = (int(nz), int(ny), int(nx))
        return self._c(self.lib.oots_set_grid(self.h, int(nx), int(ny), int(nz), float(dx)))

    def set_density(self, n):
        if np.isscalar(n):
            return self._c(self.lib.oots_set_density(self.h, None, float(n)))
        a = np.ascontiguousarray(n, np.float64)
        return self._c(self.lib.oots_set_density(self.h, _dptr(a), 0.0))

    def set_neutral_fraction(self, x):
        if np.isscalar(x):
            return self._c(self.lib.oots_set_neutral_fraction(self.h, None, float(x)))
        a = np.ascontiguousarray(x, np.float64)
        return self._c(self.lib.oots_set_neutral_fraction(self.h, _dptr(a), 0.0))

    def set_physics(self, alpha_B=2.59e-13, sigma0=6.3e-18, tau0=0.6, T=1e4):
        return self._c(self.lib.oots_set_physics(self.h, alpha_B, sigma0, tau0, T))

    def add_source(self, pos, Q, spectrum="mono", T=0.0):
        p = (ctypes.c_double * 3)(*[float(v) for v in pos])
        i = ctypes.c_int()
        sp = OOTS_MONO if spectrum in ("mono", OOTS_MONO) else OOTS_BLACKBODY
        self._c(self.lib.oots_add_source(self.h, p, float(Q), sp, float(T), ctypes.byref(i)))
        return i.value

    def add_plane_source(self, axis, direction, F, spectrum="mono", T=0.0):
        """Plane-parallel source: rays along +axis (direction 1) or -axis (-1), flux F [cm^-2 s^-1]."""
        i = ctypes.c_int()
        sp = OOTS_MONO if spectrum in ("mono", OOTS_MONO) else OOTS_BLACKBODY
        self._c(self.lib.oots_add_plane_source(self.h, int(axis), int(direction), float(F), sp, float(T),
                                               ctypes.byref(i)))
        return i.value

    def clear_sources(self):
        return self._c(self.lib.oots_clear_sources(self.h))

    def set_scheme(self, scheme=OOTS_A3, K1=0.0, K3=0.0, K4=0.0, dt_fixed=0.0, preset=None):
        if preset is not None:
            c = oots_dtcrit_preset(preset, scheme)
        else:
            c = dtcrit(K1, 0.0, K3, K4, dt_fixed)
        return self._c(self.lib.oots_set_scheme(self.h, int(scheme), ctypes.byref(c)))

    def set_tile_shape(self, shape: int):
        return self._c(self.lib.oots_set_tile_shape(self.h, int(shape)))

    def debug_set(self, key: int, value: int):
        return self._c(self.lib.oots_debug_set(self.h, int(key), int(value)))

    def set_cell_block(self, threads: int):
        """Threads per block of the closed-form per-cell passes: 128, 256 or 0 (default)."""
        return self.debug_set(5, threads)

    def set_stream(self, stream_ptr):
        return self._c(self.lib.oots_set_stream(self.h, ctypes.c_void_p(stream_ptr) if stream_ptr else None))

    # stepping
    def compute_dt(self) -> float:
        d = ctypes.c_double()
        self._c(self.lib.oots_compute_dt(self.h, ctypes.byref(d)))
        return d.value

    def step(self, dt: float):
        return self._c(self.lib.oots_step(self.h, float(dt)))

    def advance(self, t_end: float):
        t = ctypes.c_double()
        n = ctypes.c_longlong()
        self._c(self.lib.oots_advance(self.h, float(t_end), ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def synchronize(self):
        return self._c(self.lib.oots_synchronize(self.h))

    def run_substeps(self, n: int, t_end: float):
        """Enqueue exactly n substeps (asynchronous; pair with synchronize())."""
        return self._c(self.lib.oots_run_substeps(self.h, int(n), float(t_end)))

    def profile_substep(self):
        """One eager substep; returns [(kernel kind, milliseconds)] per launch."""
        kinds = (ctypes.c_int * 32)()
        ms = (ctypes.c_double * 32)()
        n = ctypes.c_int()
        self._c(self.lib.oots_profile_substep(self.h, kinds, ms, 32, ctypes.byref(n)))
        return [(KERNEL_KINDS.get(kinds[i], str(kinds[i])), ms[i]) for i in range(n.value)]

    def reset_error(self):
        return self._c(self.lib.oots_reset_error(self.h))

    # read-back
    def get_neutral_fraction(self) -> np.ndarray:
        out = np.empty(self.shape, np.float64)
        self._c(self.lib.oots_get_neutral_fraction(self.h, _dptr(out)))
        return out

    def get_neutral_fraction_into(self, out: np.ndarray) -> np.ndarray:
        """oots_get_neutral_fraction into a caller-owned contiguous float64 host array."""
        if out.dtype != np.float64 or not out.flags.c_contiguous or out.size != int(np.prod(self.shape)):
            raise ValueError("out must be a contiguous float64 array of one value per cell")
        self._c(self.lib.oots_get_neutral_fraction(self.h, _dptr(out)))
        return out

    def get_column_density(self, source: int = 0) -> np.ndarray:
        out = np.empty(self.shape, np.float64)
        self._c(self.lib.oots_get_column_density(self.h, int(source), _dptr(out)))
        return out

    def get_budget(self):
        b = budget()
        self._c(self.lib.oots_get_budget(self.h, ctypes.byref(b)))
        return np.array([b.emitted, b.absorbed, b.ions, b.recombinations])

    def reset_budget(self):
        return self._c(self.lib.oots_reset_budget(self.h))

    def get_time(self):
        t = ctypes.c_double()
        n = ctypes.c_longlong()
        self._c(self.lib.oots_get_time(self.h, ctypes.byref(t), ctypes.byref(n)))
        return t.value, n.value

    def set_time(self, t: float):
        return self._c(self.lib.oots_set_time(self.h, float(t)))

    # partitioned runs (one process per GPU)
    def set_partition(self, src_mask: int = (1 << 64) - 1, z0: int = 0, z1: int = 0):
        return self._c(self.lib.oots_set_partition(self.h, ctypes.c_ulonglong(src_mask), int(z0), int(z1)))

    def run_phase(self, phase: int, value: float = 0.0) -> float:
        v = ctypes.c_double(value)
        self._c(self.lib.oots_run_phase(self.h, int(phase), ctypes.byref(v)))
        return v.value

    def array_device(self, kind: int, source: int = 0):
        """(device address, bytes) of x (0), x_half (1), first (2) or second (3) columns of a source."""
        p = ctypes.c_void_p()
        n = ctypes.c_ulonglong()
        self._c(self.lib.oots_array_device(self.h, int(kind), int(source), ctypes.byref(p), ctypes.byref(n)))
        return p.value, n.value

    # caller-owned device memory (e.g. torch tensors' data_ptr())
    def set_neutral_fraction_device(self, ptr: int, float32: bool):
        return self._c(self.lib.oots_set_neutral_fraction_device(self.h, ctypes.c_void_p(ptr), 1 if float32 else 0))

    def get_neutral_fraction_device(self, ptr: int, float32: bool):
        return self._c(self.lib.oots_get_neutral_fraction_device(self.h, ctypes.c_void_p(ptr), 1 if float32 else 0))

    @classmethod
    def from_workload(cls, w, precision="fp64", device=0, scheme=OOTS_A3, **crit):
        c = cls(device, precision)
        c.set_grid(w.nx, w.ny, w.nz, w.dx)
        c.set_physics(w.alpha, w.sigma0, w.tau0)
        if w.uniform_n is not None:
            c.set_density(w.uniform_n)
        else:
            c.set_density(w.nH)
        c.set_neutral_fraction(w.x0)
        for s in w.sources:
            code = getattr(s, "plane", -1)
            if code >= 0:
                c.add_plane_source(code // 2, -1 if code & 1 else 1, s.Q, s.spectrum, s.T)
            else:
                c.add_source(s.pos, s.Q, s.spectrum, s.T)
        if crit:
            c.set_scheme(scheme, **crit)
        return c


class Batch:
    """Many contexts advanced together in one persistent launch per pass."""

    def __init__(self, ctxs: Sequence[Context]):
        self.lib = load()
        self.ctxs = list(ctxs)
        arr = (ctypes.c_void_p * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = ctypes.c_void_p()
        _check(self.lib.oots_batch_create(ctypes.byref(h), arr, len(self.ctxs)))
        self.h = h

    def advance(self, t_end_each: Sequence[float]):
        te = (ctypes.c_double * len(self.ctxs))(*[float(t) for t in t_end_each])
        ns = (ctypes.c_longlong * len(self.ctxs))()
        _check(self.lib.oots_batch_advance(self.h, te, ns))
        return list(ns)

    def run_substeps(self, n: int, t_end_each: Sequence[float]):
        """Enqueue exactly n substeps of every grid (asynchronous; pair with the
        first context's synchronize())."""
        te = (ctypes.c_double * len(self.ctxs))(*[float(t) for t in t_end_each])
        _check(self.lib.oots_batch_run_substeps(self.h, int(n), te))

    def close(self):
        if self.h is not None:
            self.lib.oots_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
