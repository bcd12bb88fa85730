"""Python access to the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: used by tests/, by ``__graft_entry__.smoke()`` and
by the CPU-baseline leg of ``bench.py``.  The product path never imports it.
The C source is compiled on first use (or by ``build()``) into a library named
for the machine architecture, next to this file.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")

# table layout used by every tabulated source: 512 nodes, 1e10 .. 1e24 cm^-2
TAB_K = 512
TAB_LNN_LO = 10.0 * math.log(10.0)
TAB_LNN_HI = 24.0 * math.log(10.0)
NU_MAX = 40.0          # blackbody spectrum on [nu0, 40 nu0]


def lib_path() -> str:
    return os.path.join(_HERE, f"_liboracle_{platform.machine()}.so")


def build(force: bool = False) -> str:
    out = lib_path()
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(_SRC):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("alpha", ctypes.c_double), ("sigma0", ctypes.c_double),
                ("tau0", ctypes.c_double), ("nH", ctypes.c_void_p), ("nsrc", ctypes.c_int),
                ("vtx", ctypes.c_void_p), ("Q", ctypes.c_void_p), ("kind", ctypes.c_void_p),
                ("tabL", ctypes.c_void_p), ("tabD1", ctypes.c_void_p), ("tabD2", ctypes.c_void_p),
                ("K", ctypes.c_int), ("lnN_lo", ctypes.c_double), ("lnN_hi", ctypes.c_double),
                ("plane", ctypes.c_void_p)]


class _Scheme(ctypes.Structure):
    _fields_ = [("scheme", ctypes.c_int), ("K1", ctypes.c_double), ("K3", ctypes.c_double),
                ("K4", ctypes.c_double), ("dt_fixed", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        dp = ctypes.c_void_p
        lib.or_table_build.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, dp, dp]
        lib.or_table_build.restype = ctypes.c_int
        lib.or_lnp.argtypes = [P, ctypes.c_int, ctypes.c_double]
        lib.or_lnp.restype = ctypes.c_double
        lib.or_dlnp.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.or_dlnp.restype = ctypes.c_double
        lib.or_trace.argtypes = [P, ctypes.c_int, dp, dp, dp]
        lib.or_trace.restype = None
        lib.or_rates.argtypes = [P, dp, dp, dp, dp]
        lib.or_rates.restype = None
        lib.or_integrate.argtypes = [ctypes.c_int, dp, dp, dp, dp, dp, P, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, dp]
        lib.or_integrate.restype = None
        lib.or_substep.argtypes = [P, ctypes.POINTER(_Scheme), dp, dp, ctypes.c_double, dp, dp]
        lib.or_substep.restype = ctypes.c_double
        lib.or_long_char.argtypes = [P, ctypes.c_int, dp, dp]
        lib.or_integrate_cells.argtypes = [P, ctypes.c_long, ctypes.c_void_p, dp, dp, ctypes.c_double, dp]
        lib.or_integrate_cells.restype = None
        lib.or_long_char.restype = None
        lib.or_compute_dt.argtypes = [P, ctypes.POINTER(_Scheme), dp]
        lib.or_compute_dt.restype = ctypes.c_double
        lib.or_crit_dt_range.argtypes = [P, ctypes.POINTER(_Scheme), dp, dp, ctypes.c_long, ctypes.c_long]
        lib.or_crit_dt_range.restype = ctypes.c_double
        lib.or_snap.argtypes = [ctypes.c_double, ctypes.c_int]
        lib.or_snap.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def table_build(spectrum: str, T: float = 0.0, sigma0: float = 6.3e-18, K: int = TAB_K,
                lnN_lo: float = TAB_LNN_LO, lnN_hi: float = TAB_LNN_HI, nu_max: float = NU_MAX):
    """(L, D1, D2): ln(P/Q) and its first two derivatives in ln N at the K nodes.
    spectrum "delta" (all photons at nu0) or "bb" (blackbody at T)."""
    lib = _load()
    L = np.zeros(K); D1 = np.zeros(K); D2 = np.zeros(K)
    kind = 0 if spectrum == "delta" else 1
    rc = lib.or_table_build(kind, T, sigma0, nu_max, K, lnN_lo, lnN_hi, _ptr(L), _ptr(D1), _ptr(D2))
    if rc != 0:
        raise ValueError("or_table_build failed")
    return L, D1, D2


def snap(pos: float, n: int) -> int:
    return _load().or_snap(pos, n)


class Problem:
    """A grid, its density and its sources, in the oracle's own layout
    (arrays of shape (nz, ny, nx), x fastest)."""

    def __init__(self, nx, ny, nz, dx, nH, sources, alpha=2.59e-13, sigma0=6.3e-18, tau0=0.6,
                 tables=None):
        """sources: list of (pos(3 floats), Q, spectrum "mono"|"bb", T[, plane]).
        plane (default -1, a point source at the vertex nearest pos) = 2*axis + back
        makes a plane-parallel source whose rays run along +axis (back 0) or
        -axis (back 1); its Q is a photon flux [cm^-2 s^-1] and pos is unused.
        tables: optional per-source (L, D1, D2) overriding the built table."""
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.ncell = self.nx * self.ny * self.nz
        self.nH = np.ascontiguousarray(np.broadcast_to(np.asarray(nH, np.float64), (nz, ny, nx)), np.float64).copy()
        self.nsrc = len(sources)
        ns = max(self.nsrc, 1)
        self.vtx = np.zeros(3 * ns, np.int32)
        self.Q = np.zeros(ns)
        self.kind = np.zeros(ns, np.int32)
        self.plane = np.full(ns, -1, np.int32)
        self.tabL = np.zeros(ns * TAB_K); self.tabD1 = np.zeros(ns * TAB_K); self.tabD2 = np.zeros(ns * TAB_K)
        n3 = (self.nx, self.ny, self.nz)
        for s, src in enumerate(sources):
            pos, Q, spec, T = src[:4]
            self.plane[s] = int(src[4]) if len(src) > 4 else -1
            if not -1 <= self.plane[s] <= 5:
                raise ValueError(f"plane code {self.plane[s]}")
            if self.plane[s] < 0:
                for q in range(3):
                    self.vtx[3 * s + q] = snap(pos[q], n3[q])
            self.Q[s] = Q
            if spec != "mono":
                self.kind[s] = 1
                if tables is not None and tables[s] is not None:
                    L, D1, D2 = tables[s]
                else:
                    L, D1, D2 = table_build("bb" if spec == "bb" else spec, T, sigma0)
                self.tabL[s * TAB_K:(s + 1) * TAB_K] = L
                self.tabD1[s * TAB_K:(s + 1) * TAB_K] = D1
                self.tabD2[s * TAB_K:(s + 1) * TAB_K] = D2
        self.st = _Problem(self.nx, self.ny, self.nz, float(dx), float(alpha), float(sigma0), float(tau0),
                           self.nH.ctypes.data, self.nsrc, self.vtx.ctypes.data, self.Q.ctypes.data,
                           self.kind.ctypes.data, self.tabL.ctypes.data, self.tabD1.ctypes.data,
                           self.tabD2.ctypes.data, TAB_K, TAB_LNN_LO, TAB_LNN_HI, self.plane.ctypes.data)
        self.dx = float(dx)
        self.alpha = float(alpha)
        self.sigma0 = float(sigma0)

    @classmethod
    def from_workload(cls, w, **kw):
        srcs = [(s.pos, s.Q, s.spectrum, s.T, getattr(s, "plane", -1)) for s in w.sources]
        return cls(w.nx, w.ny, w.nz, w.dx, w.nH, srcs, alpha=w.alpha, sigma0=w.sigma0, tau0=w.tau0, **kw)

    # ---------------------------------------------------------------- trace
    def trace(self, s: int, x: np.ndarray, want_dtau: bool = False):
        x = np.ascontiguousarray(x, np.float64).reshape(self.nz, self.ny, self.nx)
        Nin = np.zeros_like(x)
        dtau = np.zeros_like(x) if want_dtau else None
        _load().or_trace(ctypes.byref(self.st), s, _ptr(x), _ptr(Nin), _ptr(dtau))
        return (Nin, dtau) if want_dtau else Nin

    def long_char(self, s: int, x: np.ndarray):
        x = np.ascontiguousarray(x, np.float64).reshape(self.nz, self.ny, self.nx)
        N = np.zeros_like(x)
        _load().or_long_char(ctypes.byref(self.st), s, _ptr(x), _ptr(N))
        return N

    def rates(self, x: np.ndarray, Nin: np.ndarray):
        """F (photoionisations per H atom per s) and dx/dt for entry columns Nin (nsrc, nz, ny, nx)."""
        x = np.ascontiguousarray(x, np.float64).reshape(self.nz, self.ny, self.nx)
        Nin = np.ascontiguousarray(Nin, np.float64)
        F = np.zeros_like(x); xd = np.zeros_like(x)
        _load().or_rates(ctypes.byref(self.st), _ptr(x), _ptr(Nin), _ptr(F), _ptr(xd))
        return F, xd

    def integrate_cells(self, idx: np.ndarray, x0: np.ndarray, Nin: np.ndarray, h: float) -> np.ndarray:
        """x(h) of the cells with flat indices idx from x0, entry columns Nin (nsrc, nz, ny, nx) frozen."""
        idx = np.ascontiguousarray(idx, np.int64)
        x0 = np.ascontiguousarray(x0, np.float64)
        Nin = np.ascontiguousarray(Nin, np.float64)
        assert Nin.size == max(self.nsrc, 1) * self.ncell and x0.size == idx.size
        out = np.zeros(idx.size)
        _load().or_integrate_cells(ctypes.byref(self.st), idx.size, idx.ctypes.data, _ptr(x0), _ptr(Nin), float(h),
                                   _ptr(out))
        return out

    def lnp(self, s: int, N: float) -> float:
        return _load().or_lnp(ctypes.byref(self.st), s, N)

    def dlnp(self, s: int, Na: float, dN: float) -> float:
        return _load().or_dlnp(ctypes.byref(self.st), s, Na, dN)

    # ---------------------------------------------------------------- schemes
    def substep(self, x: np.ndarray, t: float, t_end: float, scheme: int = 3, K1=0.0, K3=0.0, K4=0.0,
                dt_fixed=0.0, want_N1: bool = False):
        """Advance x (modified in place, float64 (nz,ny,nx)) by one substep.
        Returns (t_new, dt, budget[emitted, absorbed, ions, recombinations], N1 or None)."""
        assert x.dtype == np.float64 and x.flags.c_contiguous and x.size == self.ncell
        sc = _Scheme(int(scheme), float(K1), float(K3), float(K4), float(dt_fixed))
        tt = np.array([t], np.float64)
        bud = np.zeros(4)
        N1 = np.zeros((max(self.nsrc, 1), self.nz, self.ny, self.nx)) if want_N1 else None
        dt = _load().or_substep(ctypes.byref(self.st), ctypes.byref(sc), _ptr(x), _ptr(tt), float(t_end),
                                _ptr(bud), _ptr(N1))
        return float(tt[0]), dt, bud, N1

    def compute_dt(self, x: np.ndarray, scheme: int = 3, K1=0.0, K3=0.0, K4=0.0) -> float:
        """Eq. 4 minimum over all cells for the state x (trace included)."""
        x = np.ascontiguousarray(x, np.float64).reshape(self.nz, self.ny, self.nx)
        sc = _Scheme(int(scheme), float(K1), float(K3), float(K4), 0.0)
        return _load().or_compute_dt(ctypes.byref(self.st), ctypes.byref(sc), _ptr(x))

    def crit_dt_range(self, x: np.ndarray, Nin: np.ndarray, lo: int, hi: int, scheme: int = 3, K1=0.0, K3=0.0,
                      K4=0.0) -> float:
        """Eq. 4 minimum over the cells [lo, hi) (flat indices) for x and entry columns Nin (nsrc, nz, ny, nx)."""
        x = np.ascontiguousarray(x, np.float64).reshape(self.nz, self.ny, self.nx)
        Nin = np.ascontiguousarray(Nin, np.float64)
        sc = _Scheme(int(scheme), float(K1), float(K3), float(K4), 0.0)
        return _load().or_crit_dt_range(ctypes.byref(self.st), ctypes.byref(sc), _ptr(x), _ptr(Nin), int(lo), int(hi))

    def run(self, x: np.ndarray, t: float, t_end: float, scheme: int = 3, max_steps: int = 10 ** 9,
            callback=None, **crit):
        """Substeps until t >= t_end (or max_steps). Returns (t, nsteps, summed budget)."""
        tot = np.zeros(4)
        n = 0
        while t < t_end and n < max_steps:
            t, dt, bud, _ = self.substep(x, t, t_end, scheme=scheme, **crit)
            tot += bud
            n += 1
            if callback is not None:
                callback(t, x)
            if dt <= 0:
                break
        return t, n, tot


def integrate(x0: float, h: float, c: float, rates, b0: float = 0.0, problem: Optional[Problem] = None):
    """Integrate one cell: rates = list of (kind, A, b, Nin, table_source_index).
    Returns (x(h), int F dt, int c(1-x)^2 dt, ln <exp(-b0 x)>)."""
    ns = len(rates)
    kind = np.array([r[0] for r in rates] or [0], np.int32)
    A = np.array([r[1] for r in rates] or [0.0])
    b = np.array([r[2] for r in rates] or [0.0])
    Nin = np.array([r[3] for r in rates] or [0.0])
    tabsrc = np.array([r[4] if len(r) > 4 else 0 for r in rates] or [0], np.int32)
    out = np.zeros(4)
    pst = ctypes.byref(problem.st) if problem is not None else None
    _load().or_integrate(ns, _ptr(kind), _ptr(A), _ptr(b), _ptr(Nin), _ptr(tabsrc), pst, float(c), float(b0),
                         float(x0), float(h), _ptr(out))
    return tuple(out)
