"""More parity of the CUDA path against the FP64 CPU oracle.

- A1 (Sect. 2.1, Eq. 3) with a blackbody point source: FP64 per cell within
  1e-9 of the oracle; the mixed path's front radius, ionised volume and
  largest per-cell difference against the oracle.
- A batch of uneven FP64 grids advanced in one persistent launch per pass:
  each grid against the oracle's own run of that grid, within 1e-9.
- The 32^3 Stromgren workload (Sect. 3.2) on the plain FP64 path: 4000 A3
  substeps of t_rec/1000; the front radius follows the closed form
  R_S (1 - e^{-t/t_rec})^(1/3) within 2% from t_rec to 4 t_rec.
- The autotuner's choice for a small grid keeps parity with the oracle.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import autotune, inputs, oots

pytestmark = pytest.mark.gpu
XTOL = 1e-9


def _reff(x, dx, n_oct=8):
    return (3.0 * float((1.0 - x).sum()) * dx ** 3 * (8.0 / n_oct) / (4.0 * math.pi)) ** (1.0 / 3.0)


@pytest.mark.parametrize("crit", [dict(dt_fixed=0.02), dict(K1=0.1)])
def test_A1_blackbody_point_source_fp64(crit):
    """A1 on a random state with a 4e4 K blackbody point source: three substeps,
    fixed step or the K1 criterion (t_rec of the densest cell)."""
    w = inputs.small_random(n=12, ny=11, nz=10, seed=61, nsrc=1, spectrum="bb")
    kw = dict(crit)
    if "dt_fixed" in kw:
        kw["dt_fixed"] *= w.t_rec
    c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A1, **kw)
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.astype(np.float64))
    t = 0.0
    for k in range(3):
        if "dt_fixed" in kw:
            c.step(kw["dt_fixed"])
            t, *_ = P.substep(x, t, t + kw["dt_fixed"], scheme=1, dt_fixed=kw["dt_fixed"])
        else:
            dt_g = c.compute_dt()
            t_new, dt, _, _ = P.substep(x, t, 1e300, scheme=1, K1=kw["K1"])
            assert abs(dt_g / dt - 1.0) <= 1e-10, (k, dt_g, dt)
            c.step(dt_g)
            t = t_new
        err = float(np.max(np.abs(c.get_neutral_fraction() - x)))
        assert err <= XTOL, (crit, k, err)


def test_A1_blackbody_point_source_mixed_error_metrics():
    """The mixed path of A1 with a blackbody point source against the oracle,
    from a neutral start over 0.3 t_rec (K1 = 0.03): ionised volume and front
    radius within 0.5%, largest per-cell |dx| below 0.02."""
    n = 16
    Q, nH = 1e48, 100.0
    L = 1.5 * inputs.stromgren_radius(Q, nH)
    w = inputs.Workload("a1_bb", n, n, n, L / n, np.full((n, n, n), nH), np.full((n, n, n), inputs.X_NEUTRAL),
                        [inputs.Source((0.0, 0.0, 0.0), Q, "bb", 4e4)], uniform_n=nH)
    w.t_rec = 1.0 / (inputs.ALPHA_B * nH)
    tend = 0.3 * w.t_rec
    c = oots.Context.from_workload(w, "mixed", scheme=oots.OOTS_A1, K1=0.03)
    c.advance(tend)
    xg = c.get_neutral_fraction()
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.astype(np.float64))
    P.run(x, 0.0, tend, scheme=1, K1=0.03)
    vg, vr = float((1 - xg).sum()), float((1 - x).sum())
    assert vr > 10.0                                            # a front has formed
    assert abs(vg / vr - 1.0) <= 0.005, (vg, vr)
    assert abs(_reff(xg, w.dx, 1) / _reff(x, w.dx, 1) - 1.0) <= 0.005
    assert float(np.max(np.abs(xg - x))) <= 0.02


def test_fp64_batch_against_the_oracle():
    """Four uneven grids (sides 12-20, densities 10-1000, rates 1e47-1e50) in one
    batch, A3-dt02 with a per-grid step: every grid equals the oracle's own
    run of that grid (same substep count, x within 1e-9)."""
    ws = inputs.batch(count=4, seed=17, sides=(12, 16, 20))
    tend = [0.03 * w.t_rec for w in ws]
    ctxs = [oots.Context.from_workload(w, "fp64", scheme=3, K4=0.25) for w in ws]
    b = oots.Batch(ctxs)
    nsub = b.advance(tend)
    b.close()
    for g, (c, w, te) in enumerate(zip(ctxs, ws, tend)):
        P = oracle.Problem.from_workload(w)
        x = np.ascontiguousarray(w.x0.astype(np.float64))
        tr, nr, _ = P.run(x, 0.0, te, scheme=3, K4=0.25)
        assert nsub[g] == nr, (g, nsub[g], nr)
        assert float(np.max(np.abs(c.get_neutral_fraction() - x))) <= XTOL, g


def test_stromgren_32_cube_fp64_front_follows_the_closed_form():
    """The plain FP64 path on the full 32^3 Stromgren workload (n = 100,
    Q = 1e48, corner source, box 1.5 R_S, dt = t_rec/1000; Sect. 3.2)."""
    w = inputs.stromgren_corner(32)
    c = oots.Context.from_workload(w, "fp64", scheme=3, dt_fixed=w.t_rec / 1000)
    R_S = inputs.stromgren_radius(w.sources[0].Q, 100.0)
    for f in (1.0, 2.0, 3.0, 4.0):
        t, _ = c.advance(f * w.t_rec)
        x = c.get_neutral_fraction()
        ratio = _reff(x, w.dx, 1) / (R_S * (1.0 - math.exp(-t / w.t_rec)) ** (1.0 / 3.0))
        assert abs(ratio - 1.0) <= 0.02, (f, ratio)
    assert 4000 <= c.get_time()[1] <= 4004


def test_autotuned_shape_keeps_parity(tmp_path):
    """Whatever shape the tuner picks for a small three-source grid, the columns
    and one A3 substep equal the oracle's."""
    import torch
    w = inputs.small_random(n=26, ny=21, nz=19, seed=88, nsrc=3)
    c = oots.Context.from_workload(w, "fp64", scheme=3, K4=0.25)
    shape = autotune.tune(c, torch.cuda.get_device_name(0), 3, use_cache=False, path=str(tmp_path / "t.json"))
    assert shape is not None
    c.set_neutral_fraction(w.x0)
    c.set_time(0.0)
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.astype(np.float64))
    dt_g = c.compute_dt()
    for s in range(3):
        Nr = P.trace(s, x)
        assert float(np.max(np.abs(c.get_column_density(s) - Nr) / np.maximum(Nr, 1e10))) <= 1e-12, (shape, s)
    _, dt, _, _ = P.substep(x, 0.0, 1e300, scheme=3, K4=0.25)
    assert abs(dt_g / dt - 1.0) <= 1e-10
    c.step(dt_g)
    assert float(np.max(np.abs(c.get_neutral_fraction() - x))) <= XTOL, shape


@pytest.mark.parametrize("nsrc", [1, 3])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cell_block_sizes_agree(nsrc, precision):
    """The closed-form passes give every cell the same result with 128- and
    256-thread blocks (tuning key 5): the same steps, x bit for bit; the FP64
    path also equals the oracle."""
    w = inputs.small_random(n=26, ny=21, nz=19, seed=91 + nsrc, nsrc=nsrc, spectrum="bb")
    out = {}
    for bs in (128, 256):
        c = oots.Context.from_workload(w, precision, scheme=3, K4=0.25)
        c.set_cell_block(bs)
        dts = []
        for _ in range(3):
            dts.append(c.compute_dt())
            c.step(dts[-1])
        out[bs] = (dts, c.get_neutral_fraction())
    assert out[128][0] == out[256][0]
    assert np.array_equal(out[128][1], out[256][1])
    if precision == "fp64":
        P = oracle.Problem.from_workload(w)
        x = np.ascontiguousarray(w.x0.astype(np.float64))
        t = 0.0
        for _ in range(3):
            t, *_ = P.substep(x, t, 1e300, scheme=3, K4=0.25)
        assert float(np.max(np.abs(out[256][1] - x))) <= XTOL
