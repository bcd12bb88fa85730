"""The library's cell integrator (the __host__ __device__ code of
integrator.cuh) built for the host and checked on the CPU against
the oracle and against photon conservation.  This runs the product's
arithmetic without a GPU; the GPU tests check the kernels around it.

- Single monochromatic cells over the regimes of Eq. 2 (thin, opaque, stiff,
  near equilibrium, recombination-dominated, no recombinations): x(h) against
  the oracle's integration, FP64 to 1e-10 and FP32 to 1e-4.
- The blackbody rate table (built by the library's own tables.cpp, read by
  its interpolation) against the oracle's independently built table, and
  blackbody cells against the oracle's integration.
- A1 on a row lit by a plane-parallel flux with no recombinations (Sect. 3.1):
  ions per unit area = F t; FP64 to 1e-11, FP32 to 1e-5.  A subnormal rate
  deep in the row once moved x by 1% here.
"""
import ctypes
import os
import platform
import shutil
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "host", "integrator_host.cu")
SIG, ALPHA = 6.3e-18, 2.59e-13


@pytest.fixture(scope="module")
def lib():
    # host code only: the host compiler with the CUDA headers (the device half
    # of an nvcc build is not needed and takes a minute)
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    cxx = shutil.which("g++")
    if nvcc is None or cxx is None:
        pytest.skip("no CUDA headers or host compiler")
    cuda_inc = os.path.join(os.path.dirname(os.path.realpath(nvcc)), "..", "include")
    out = os.path.join(HERE, "host", f"_libintegrator_host_{platform.machine()}.so")
    csrc = os.path.join(HERE, "..", "paper_1201_5651_gb300", "csrc")
    deps = [SRC] + [os.path.join(csrc, f) for f in ("common.cuh", "integrator.cuh", "oots_internal.h", "tables.h",
                                                    "tables.cpp")]
    if not os.path.exists(out) or os.path.getmtime(out) < max(os.path.getmtime(d) for d in deps):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call([cxx, "-std=c++17", "-O2", "-shared", "-fPIC", "-I", cuda_inc, "-o", tmp,
                               "-x", "c++", SRC, "-x", "none", os.path.join(csrc, "tables.cpp")])
        os.replace(tmp, out)
    L = ctypes.CDLL(out)
    d = ctypes.c_double
    L.oots_host_integrate_mono.argtypes = [ctypes.c_int, d, d, d, d, d, d, d, d, ctypes.c_void_p]
    L.oots_host_integrate_mono.restype = None
    L.oots_host_a1_row.argtypes = [ctypes.c_int, ctypes.c_int, d, d, d, d, ctypes.c_void_p, ctypes.c_void_p, d,
                                   ctypes.c_int]
    L.oots_host_a1_row.restype = d
    L.oots_host_table_lnp.argtypes = [ctypes.c_int, d, d, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.oots_host_table_lnp.restype = None
    L.oots_host_integrate_bb.argtypes = [ctypes.c_int, d, d, d, d, d, d, d, d, ctypes.c_void_p]
    L.oots_host_integrate_bb.restype = None
    return L


def _cell(L, precision, A, b, c, x0, h, b0=0.0):
    out = np.zeros(3)
    L.oots_host_integrate_mono(precision, A, b, 0.0, c, b0, SIG, x0, h, out.ctypes.data)
    return out


CASES = [  # (A [1/s], b, c [1/s], x0, h [s])
    (1e-9, 0.05, ALPHA * 100, 1 - 1e-6, 3e8),      # optically thin, slow
    (1e-8, 300.0, ALPHA * 100, 1 - 1e-6, 1e9),     # opaque front cell
    (1e-6, 10.0, ALPHA * 100, 0.9, 1e9),           # stiff
    (3e-10, 2.0, ALPHA * 100, 0.02, 5e9),          # near equilibrium
    (1e-14, 5.0, ALPHA * 1000, 0.3, 2e9),          # recombination-dominated
    (2e-9, 8.0, 0.0, 1 - 1e-6, 4e8),               # no recombinations
]


@pytest.mark.parametrize("case", CASES)
def test_host_integrator_matches_oracle(lib, case):
    A, b, c, x0, h = case
    xo, IF, IR, _ = oracle.integrate(x0, h, c, [(0, A, b, 0.0)])
    for precision, tol in ((0, 1e-10), (1, 1e-4)):
        x, ir, _ = _cell(lib, precision, A, b, c, x0, h)
        assert abs(x - xo) <= tol, (precision, x, xo)
        assert abs(ir - IR) <= tol * max(1.0, abs(IR)) + 1e-12, (precision, ir, IR)


def test_host_a1_row_conserves_photons(lib):
    n_cells, F, n, dtau = 100, 1e9, 100.0, 10.0
    dx = dtau / (SIG * n)
    tc = n * dx / F
    dt, steps = 0.7 * tc, 57
    for precision, tol in ((0, 1e-11), (1, 1e-5)):
        nn = np.full(n_cells, n)
        x = np.full(n_cells, 1 - 1e-6)
        ions = lib.oots_host_a1_row(precision, n_cells, F, SIG, 0.0, dx, nn.ctypes.data, x.ctypes.data, dt, steps)
        assert abs(ions / (F * dt * steps) - 1) <= tol, (precision, ions / (F * dt * steps) - 1)
        # the front stands where F t / n puts it, the rest of the row is untouched
        front = F * dt * steps / (n * dx)
        assert np.all(x[: int(front) - 2] < 1e-3) and np.all(x[int(front) + 3:] > 1 - 2e-6)


def test_host_blackbody_table_matches_oracle(lib):
    T = 4e4
    P = oracle.Problem(1, 1, 1, 1e16, 100.0, [((0, 0, 0), 1e48, "bb", T)])
    N = np.concatenate([[0.0, 1e5], np.logspace(8, 25, 400)])
    ref = np.array([P.lnp(0, v) for v in N])
    # ln P to 1e-12 (FP64) or 1e-5 relative (FP32: the interpolation runs in float) where P > e^-60 Q
    for precision, tol in ((0, 1e-12), (1, 1e-5)):
        out = np.zeros(N.size)
        lib.oots_host_table_lnp(precision, T, SIG, N.ctypes.data, N.size, out.ctypes.data)
        fin = np.isfinite(ref) & (ref > -60)
        err = np.abs(out[fin] - ref[fin]) / np.maximum(1.0, np.abs(ref[fin]))
        assert float(err.max()) <= tol, (precision, float(err.max()))
        assert np.all(out[~np.isfinite(ref)] == -np.inf)


@pytest.mark.parametrize("Nin", [0.0, 3e16, 4e17, 2e18])
def test_host_blackbody_cell_matches_oracle(lib, Nin):
    T, Q, n, ds = 4e4, 1e48, 100.0, 2e16
    P = oracle.Problem(1, 1, 1, 1e16, 100.0, [((0, 0, 0), Q, "bb", T)])
    V = 4 * np.pi * (3e17) ** 2 * ds
    A = Q / (n * V)
    for x0, h in [(1 - 1e-6, 2e8), (0.4, 1e9), (0.01, 3e9)]:
        xo, IF, IR, _ = oracle.integrate(x0, h, ALPHA * n, [(1, A, n * ds, Nin, 0)], problem=P)
        for precision, tol in ((0, 1e-9), (1, 2e-4)):
            out = np.zeros(3)
            lib.oots_host_integrate_bb(precision, T, A, n * ds, Nin, ALPHA * n, SIG, x0, h, out.ctypes.data)
            assert abs(out[0] - xo) <= tol, (precision, x0, h, out[0], xo)


def test_host_integrator_random_cells_match_oracle(lib):
    """300 random monochromatic cells, log-uniform over rates, optical depths,
    recombination rates, starting states and steps (including cells lit too
    faintly to move, cells at and near their equilibrium, and A1's attenuation
    average): x(h) and ln<exp(-b0 x)> against the oracle, FP64 to 1e-10; x(h)
    in FP32 to 2e-6."""
    rng = np.random.default_rng(2024)
    worst_x = worst_f = 0.0
    for k in range(300):
        A = 10 ** rng.uniform(-16, -5)
        b = 10 ** rng.uniform(-3, 3)
        c = ALPHA * 10 ** rng.uniform(0, 4) if k % 5 else 0.0
        x0 = float(np.clip(10 ** rng.uniform(-9, 0), 0, 1 - 1e-6))
        h = 10 ** rng.uniform(6, 11)
        b0 = b if k % 3 == 0 else 0.0
        xo, IF, IR, lnf = oracle.integrate(x0, h, c, [(0, A, b, 0.0)], b0=b0)
        x, ir, lnfav = _cell(lib, 0, A, b, c, x0, h, b0=b0)
        worst_x = max(worst_x, abs(x - xo))
        assert abs(x - xo) <= 1e-10, (k, A, b, c, x0, h, b0, x, xo)
        xf = _cell(lib, 1, A, b, c, x0, h, b0=b0)[0]
        assert abs(xf - xo) <= 2e-6, (k, A, b, c, x0, h, b0, xf, xo)
        if b0 > 0:
            worst_f = max(worst_f, abs(lnfav - lnf))
            assert abs(lnfav - lnf) <= 1e-9 * max(1.0, abs(lnf)), (k, A, b, c, x0, h, lnfav, lnf)


def test_host_table_difference_matches_oracle(lib):
    """The stable table difference ln P(Na + dN) - ln P(Na), which carries a
    cell's absorbed fraction without cancellation, against the oracle's own
    table difference: from steps 1e-12 of the column up to steps of 1e24."""
    lib.oots_host_table_dlnp.argtypes = [ctypes.c_int] + [ctypes.c_double] * 2 + [ctypes.c_void_p] * 2 + \
        [ctypes.c_int, ctypes.c_void_p]
    T = 4e4
    P = oracle.Problem(1, 1, 1, 1e16, 100.0, [((0, 0, 0), 1e48, "bb", T)])
    rng = np.random.default_rng(5)
    Na = np.concatenate([[0.0, 0.0], 10 ** rng.uniform(8, 23.5, 300)])
    dN = np.concatenate([[1e10, 1e20], Na[2:] * 10 ** rng.uniform(-12, 1.5, 300)])
    ref = np.array([P.dlnp(0, a, d) for a, d in zip(Na, dN)])
    out = np.zeros(Na.size)
    lib.oots_host_table_dlnp(0, T, SIG, Na.ctypes.data, dN.ctypes.data, Na.size, out.ctypes.data)
    fin = np.isfinite(ref) & (ref > -60)
    err = np.abs(out[fin] - ref[fin]) / np.maximum(np.abs(ref[fin]), 1e-300)
    assert fin.sum() > 250 and float(err.max()) <= 1e-8, float(err.max())


def test_host_float_float_column_sum(lib):
    """The mixed path's float-float column accumulation keeps about 44 bits:
    a running sum of 10^5 positive float increments spanning six decades,
    against the exactly rounded sum."""
    import math
    lib.oots_host_ff_sum.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.oots_host_ff_sum.restype = ctypes.c_double
    rng = np.random.default_rng(6)
    v = (10 ** rng.uniform(14, 20, 100000)).astype(np.float32)
    exact = math.fsum(float(a) for a in v)
    got = lib.oots_host_ff_sum(v.ctypes.data, v.size)
    assert abs(got / exact - 1) <= 1e-12, got / exact - 1
    assert abs(float(np.cumsum(v, dtype=np.float32)[-1]) / exact - 1) > 1e-6   # a running float sum loses this


def test_host_rate_geometry_matches_oracle(lib):
    """The library's per-cell rate (src_rate: shell volume 4 pi r^2 ds of a
    point source, volume per unit face area dx of a plane source) against the
    oracle's rates on a ragged grid with random density, state and columns."""
    lib.oots_host_rate_mono.argtypes = [ctypes.c_int, ctypes.c_void_p] + [ctypes.c_double] * 4 + \
        [ctypes.c_int] * 3 + [ctypes.c_double] * 2
    lib.oots_host_rate_mono.restype = ctypes.c_double
    rng = np.random.default_rng(8)
    nx, ny, nz, dx = 7, 5, 6, 3e16
    nH = 100 * np.exp(rng.standard_normal((nz, ny, nx)))
    x = rng.uniform(0, 1, (nz, ny, nx))
    for src in [((2.0, 3.0, 1.0), 1e48, "mono", 0.0), ((0.0, 0.0, 0.0), 3e10, "mono", 0.0, 3)]:
        P = oracle.Problem(nx, ny, nz, dx, nH, [src])
        N = 10 ** rng.uniform(15, 18.5, (1, nz, ny, nx))
        F, _ = P.rates(x, N)
        plane = len(src) > 4
        v = (ctypes.c_int * 3)(*[int(c) for c in src[0]])
        for Z in range(nz):
            for Y in range(ny):
                for X in range(nx):
                    g = lib.oots_host_rate_mono(int(plane), v, src[1], SIG, dx, nH[Z, Y, X], X, Y, Z, N[0, Z, Y, X],
                                                x[Z, Y, X])
                    assert abs(g / F[Z, Y, X] - 1) <= 1e-12, (plane, X, Y, Z, g, F[Z, Y, X])
