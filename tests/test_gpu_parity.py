"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

FP64 path: per-cell neutral fraction within 1e-9 (the tolerance of the
FP64 plain method), columns and dt within 1e-10 relative.  Mixed path:
checked on the error metrics (front radius, ionised volume, max |dx|).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import inputs, oots

pytestmark = pytest.mark.gpu

XTOL = 1e-9


def _ctx(w, precision="fp64", **kw):
    return oots.Context.from_workload(w, precision, **kw)


def _rel(a, b, floor=1.0):
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


# --------------------------------------------------------------------------- trace
@pytest.mark.parametrize("shape", range(9))
def test_trace_columns_every_tile_shape(shape):
    """Ragged non-cubic grid, two sources (one on the grid corner vertex),
    every tile shape: columns equal the oracle's to 1e-12 relative."""
    w = inputs.small_random(n=21, ny=13, nz=17, seed=11 + shape, nsrc=2)
    w.sources[0].pos = (0.0, 13.0, 5.0)          # on the grid boundary: four octants are empty
    c = _ctx(w)
    c.set_tile_shape(shape)
    c.set_scheme(oots.OOTS_A3, K4=0.25)
    try:
        c.compute_dt()
    except oots.OotsError as e:
        # a shape that does not fit this device's shared memory is refused cleanly
        assert e.code == oots.OOTS_E_UNSUPPORTED
        pytest.skip(f"tile shape {shape} does not fit at FP64")
    P = oracle.Problem.from_workload(w)
    for s in range(2):
        N = c.get_column_density(s)
        Nr = P.trace(s, w.x0)
        assert _rel(N, Nr, floor=1e10) <= 1e-12, (shape, s)


@pytest.mark.parametrize("vtx", [(0, 0, 0), (16, 16, 16), (8, 8, 8), (16, 0, 7), (3, 16, 0)])
def test_trace_source_positions(vtx):
    w = inputs.small_random(n=16, seed=3)
    w.sources[0].pos = tuple(float(v) for v in vtx)
    c = _ctx(w)
    c.compute_dt()
    Nr = oracle.Problem.from_workload(w).trace(0, w.x0)
    assert _rel(c.get_column_density(0), Nr, floor=1e10) <= 1e-12


def test_degenerate_grids():
    """One-cell-thick and single-cell grids."""
    for (nx, ny, nz, vtx) in [(9, 7, 1, (4, 3, 0)), (1, 1, 1, (0, 0, 0)), (1, 1, 1, (1, 1, 1)), (5, 1, 1, (2, 0, 1))]:
        w = inputs.small_random(n=nx, ny=ny, nz=nz, seed=nx * 7 + nz)
        w.sources[0].pos = tuple(float(v) for v in vtx)
        c = _ctx(w)
        c.compute_dt()
        Nr = oracle.Problem.from_workload(w).trace(0, w.x0)
        assert _rel(c.get_column_density(0), Nr, floor=1e10) <= 1e-12


# --------------------------------------------------------------------------- timestep
@pytest.mark.parametrize("crit", [dict(K4=0.25), dict(K3=0.125), dict(K1=0.1), dict(K3=0.5, K4=0.5)])
def test_dt_criterion(crit):
    w = inputs.small_random(n=12, seed=5, nsrc=2)
    c = _ctx(w, scheme=oots.OOTS_A3, **crit)
    dt = c.compute_dt()
    dtr = oracle.Problem.from_workload(w).compute_dt(w.x0, **crit)
    assert abs(dt / dtr - 1) <= 1e-10


# --------------------------------------------------------------------------- substeps
@pytest.mark.parametrize("scheme", [3, 2, 1])
def test_substeps_fp64(scheme):
    """Random state (every regime: thin, opaque, near equilibrium), fixed dt,
    three substeps: per-cell x within 1e-9 and the photon budget within 1e-8."""
    w = inputs.small_random(n=11, ny=9, nz=10, seed=21 + scheme, nsrc=1)
    dt = 0.01 * w.t_rec
    c = _ctx(w, scheme=scheme, dt_fixed=dt)
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    t = 0.0
    tot = np.zeros(4)
    for k in range(3):
        c.step(dt)
        t, _, bud, _ = P.substep(x, t, t + dt, scheme=scheme, dt_fixed=dt)
        tot += bud
        xg = c.get_neutral_fraction()
        assert np.max(np.abs(xg - x)) <= XTOL, (scheme, k, np.max(np.abs(xg - x)))
    b = c.get_budget()
    assert abs(b[0] / tot[0] - 1) <= 1e-12
    for q in (1, 2, 3):
        assert abs(b[q] - tot[q]) <= 1e-8 * abs(tot[1]), (q, b, tot)


def test_multisource_blackbody_fp64():
    """Three sources (two blackbody tables, one monochromatic), A3."""
    w = inputs.small_random(n=10, seed=31, nsrc=3, spectrum="bb")
    w.sources[2].spectrum = "mono"
    dt = 0.02 * w.t_rec
    c = _ctx(w, scheme=3, dt_fixed=dt)
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    t = 0.0
    for k in range(2):
        c.step(dt)
        t, *_ = P.substep(x, t, t + dt, scheme=3, dt_fixed=dt)
        assert np.max(np.abs(c.get_neutral_fraction() - x)) <= XTOL


def test_stromgren_run_fp64_adaptive():
    """A3-dt02 (K4 = 1/4) from a neutral start through the R-type phase:
    same substep count and per-cell x within 1e-9 after the whole run."""
    n, Q, nH = 12, 1e44, 1.0
    L = 1.5 * inputs.stromgren_radius(Q, nH)
    w = inputs.Workload("strom_mod", n, n, n, L / n, np.full((n, n, n), nH), np.full((n, n, n), 1 - 1e-6),
                        [inputs.Source((0.0, 0.0, 0.0), Q, "mono")], uniform_n=nH)
    w.t_rec = 1.0 / (inputs.ALPHA_B * nH)
    tend = 0.3 * w.t_rec
    c = _ctx(w, scheme=3, K4=0.25)
    t, nsub = c.advance(tend)
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    tr, nr, _ = P.run(x, 0.0, tend, scheme=3, K4=0.25)
    assert nsub == nr
    assert abs(t - tr) <= 1e-12 * tr
    assert np.max(np.abs(c.get_neutral_fraction() - x)) <= XTOL


# --------------------------------------------------------------------------- mixed precision
def test_mixed_precision_error_metrics():
    """FP32 state and rates with float-float columns against the FP64 oracle
    on the 16^3 Stromgren problem to one recombination time: front radius and
    ionised volume within 0.5%, max per-cell |dx| reported."""
    w = inputs.stromgren_corner(16)
    dt = w.t_rec / 250
    c = _ctx(w, "mixed", scheme=3, dt_fixed=dt)
    c.advance(w.t_rec)
    P = oracle.Problem.from_workload(w)
    x = w.x0.copy()
    P.run(x, 0.0, w.t_rec, scheme=3, dt_fixed=dt)
    xg = c.get_neutral_fraction()
    V = w.dx ** 3
    vi, vr = ((1 - xg) * V).sum(), ((1 - x) * V).sum()
    assert abs(vi / vr - 1) < 0.005
    assert abs((vi / vr) ** (1 / 3) - 1) < 0.005
    assert np.max(np.abs(xg - x)) < 0.02


# --------------------------------------------------------------------------- batch, device pointers, faults
def test_batch_matches_individual_runs():
    ws = inputs.batch(count=4, seed=9, sides=(12, 16, 20))
    solo = []
    for w in ws:
        c = _ctx(w, "fp64", scheme=3, K4=0.25)
        c.advance(0.05 * w.t_rec)
        solo.append(c.get_neutral_fraction())
    ctxs = [_ctx(w, "fp64", scheme=3, K4=0.25) for w in ws]
    b = oots.Batch(ctxs)
    b.advance([0.05 * w.t_rec for w in ws])
    b.close()
    for c, xs in zip(ctxs, solo):
        assert np.max(np.abs(c.get_neutral_fraction() - xs)) == 0.0


def test_device_pointer_roundtrip():
    torch = pytest.importorskip("torch")
    w = inputs.small_random(n=8, seed=2)
    c = _ctx(w, "mixed")
    src = torch.rand(w.ncell, dtype=torch.float64, device="cuda")
    c.set_neutral_fraction_device(src.data_ptr(), False)
    dst = torch.zeros(w.ncell, dtype=torch.float32, device="cuda")
    c.get_neutral_fraction_device(dst.data_ptr(), True)
    c.synchronize()
    assert torch.max(torch.abs(dst.double() - src)).item() < 1e-7
    assert np.max(np.abs(c.get_neutral_fraction().ravel() - src.cpu().numpy())) < 1e-7


def test_bounded_wait_times_out_and_recovers():
    """A tile that never publishes makes its downstream waits run out: the call
    returns OOTS_E_DEVICE_TIMEOUT (no fault) and the context keeps working."""
    w = inputs.small_random(n=40, ny=20, nz=20, seed=4)
    w.sources[0].pos = (0.0, 0.0, 0.0)   # one octant of 3 x 3 x 3 tiles: tile 0 has downstream tiles
    c = _ctx(w, scheme=3, K4=0.25)
    c.debug_set(1, 2000)      # short spin limit
    c.debug_set(2, 0)         # the first tile never publishes
    with pytest.raises(oots.OotsError) as e:
        c.compute_dt()
    assert e.value.code == oots.OOTS_E_DEVICE_TIMEOUT
    c.debug_set(2, -1)
    c.debug_set(1, 1 << 22)
    c.reset_error()
    dt = c.compute_dt()
    assert abs(dt / oracle.Problem.from_workload(w).compute_dt(w.x0, K4=0.25) - 1) <= 1e-10


def test_argument_errors():
    w = inputs.small_random(n=4, seed=1)
    c = _ctx(w)
    with pytest.raises(oots.OotsError):
        c.set_neutral_fraction(np.full(w.ncell, 1.5))
    with pytest.raises(oots.OotsError):
        c.set_density(np.zeros(w.ncell))
    with pytest.raises(oots.OotsError):
        c.step(-1.0)
    with pytest.raises(oots.OotsError):
        c.add_source((1, 1, 1), -5.0)
    c.add_source((2, 2, 2), 1e48)
    c.set_scheme(oots.OOTS_A1, K1=0.1)
    with pytest.raises(oots.OotsError) as e:
        c.step(1e6)
    assert e.value.code == oots.OOTS_E_UNSUPPORTED


def test_mixed_budget_and_dt_against_fp64():
    """The mixed path forms the Eq. 4 criterion and the photon budget in FP32
    (warp sums scaled to FP64): dt within 1e-5 and every budget term within
    1e-4 of the absorbed total, against the FP64 path on the same state."""
    w = inputs.small_random(n=24, ny=20, nz=22, seed=77, nsrc=1, spectrum="bb", x_lo=0.5)
    cm = _ctx(w, "mixed", scheme=3, K4=0.25)
    cf = _ctx(w, "fp64", scheme=3, K4=0.25)
    dm, df = cm.compute_dt(), cf.compute_dt()
    assert abs(dm / df - 1) <= 1e-5, (dm, df)
    for c in (cm, cf):
        c.step(df)
    bm, bf = cm.get_budget(), cf.get_budget()
    assert abs(bm[0] / bf[0] - 1) <= 1e-6
    for q in (1, 2, 3):
        assert abs(bm[q] - bf[q]) <= 1e-4 * abs(bf[1]), (q, bm, bf)
