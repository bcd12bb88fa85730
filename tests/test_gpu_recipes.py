"""Parity on the recipes of the clumpy and many-source workloads, at sizes the
oracle integrates whole in seconds.

Clumpy: a lognormal density with sigma_ln 1.5 times overdense spheres, a
monochromatic source at the centre vertex.  It runs each scheme with its
criterion: A2-dt12 (K3 = 1/16), A3-dt02 (K4 = 1/4) and A1 with K1 = 0.1.
Each run takes three adaptive substeps; dt and x per cell match the oracle.

Many sources: sixteen blackbody sources (T 3e4-5e4 K, Q 1e47-1e49) at random
vertices of a lognormal grid.  The checks are the columns of every source,
dt and x per cell after two A3-dt02 substeps (FP64), and the mixed path's
front metrics against FP64.
"""
import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import inputs, oots

pytestmark = pytest.mark.gpu

XTOL = 1e-9

CRIT = {1: dict(K1=0.1), 2: dict(K3=1.0 / 16), 3: dict(K4=0.25)}


@pytest.fixture(scope="module")
def clumpy40():
    w = inputs.clumpy(40, 1.5, 1203, 1303, 30, Q=1e48, box_rs=2.5, spectrum="mono")
    # a partly ionised state (every regime: ionised, front, neutral), seeded
    w.x0 = (np.random.default_rng(7).uniform(0.0, 1.0, w.ncell) ** 3).reshape(w.x0.shape)
    return w


@pytest.mark.parametrize("scheme", [1, 2, 3])
def test_clumpy_adaptive_substeps_fp64(clumpy40, scheme):
    w = clumpy40
    c = oots.Context.from_workload(w, "fp64", scheme=scheme, **CRIT[scheme])
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.reshape(w.nz, w.ny, w.nx).astype(np.float64))
    t = 0.0
    for k in range(3):
        dt_g = c.compute_dt()
        t_new, dt, _, _ = P.substep(x, t, 1e300, scheme=scheme, **CRIT[scheme])
        assert abs(dt_g / dt - 1.0) <= 1e-10, (k, dt_g, dt)
        c.step(dt_g)
        t = t_new
        err = np.max(np.abs(c.get_neutral_fraction().ravel() - x.ravel()))
        assert err <= XTOL, (scheme, k, err)


@pytest.fixture(scope="module")
def many_sources():
    return inputs.multisource(24, 1.0, 1205, nsrc=16, box_rs=2.0)


def test_sixteen_sources_columns_dt_and_substeps_fp64(many_sources):
    w = many_sources
    c = oots.Context.from_workload(w, "fp64", scheme=3, K4=0.25)
    P = oracle.Problem.from_workload(w)
    x = np.ascontiguousarray(w.x0.reshape(w.nz, w.ny, w.nx).astype(np.float64))
    t = 0.0
    for k in range(2):
        dt_g = c.compute_dt()
        for s in range(len(w.sources)):
            N = c.get_column_density(s).reshape(w.nz, w.ny, w.nx)
            Nref = P.trace(s, x)
            assert float(np.max(np.abs(N - Nref) / np.maximum(Nref, 1e10))) <= 1e-10, (k, s)
        t_new, dt, _, _ = P.substep(x, t, 1e300, scheme=3, K4=0.25)
        assert abs(dt_g / dt - 1.0) <= 1e-10, (k, dt_g, dt)
        c.step(dt_g)
        t = t_new
        err = np.max(np.abs(c.get_neutral_fraction().ravel() - x.ravel()))
        assert err <= XTOL, (k, err)


def test_sixteen_sources_mixed_against_fp64(many_sources):
    w = many_sources
    t_end = 0.05 * w.t_rec
    cm = oots.Context.from_workload(w, "mixed", scheme=3, K4=0.25)
    cf = oots.Context.from_workload(w, "fp64", scheme=3, K4=0.25)
    cm.advance(t_end)
    cf.advance(t_end)
    xm, xf = cm.get_neutral_fraction(), cf.get_neutral_fraction()
    vm, vf = float((1 - xm).sum()), float((1 - xf).sum())
    assert abs(vm / vf - 1.0) <= 1e-3            # ionised volume (R_eff to a third of that)
    assert float(np.abs(xm - xf).max()) <= 1e-3
