"""Parity at full size: the 128^3 lognormal blackbody workload that bench.py
times, through the same C ABI and launch path (persistent sweep, closed-form
and general integration passes, captured substeps).

The oracle integrates a whole 128^3 grid in about a minute, so the checks use
what it computes quickly at this size:
- the whole column field of a trace;
- the dt criterion;
- x^{n+1} of sampled cells, integrated one by one from the GPU's own state
  and entry columns.
The samples include the cells that moved most, which are the front cells the
general pass integrates.  The mixed path is checked on the front-radius
metrics against the FP64 path.
"""
import numpy as np
import pytest

import oracle
from paper_1201_5651_gb300 import inputs, oots

pytestmark = pytest.mark.gpu


def _reff(x, dx):
    # eight octants around a centre source: R_eff = (3 V_ion / 4 pi)^(1/3)
    return (3.0 * float((1.0 - x).sum()) * dx ** 3 / (4.0 * np.pi)) ** (1.0 / 3.0)


@pytest.fixture(scope="module")
def workload():
    return inputs.lognormal_bb(128, 1.0, 1202, Q=1e48, T=4e4, box_rs=2.5)


def test_fullsize_fp64_columns_dt_and_sampled_cells(workload):
    w = workload
    c = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A2, K4=0.25)
    c.advance(0.01 * w.t_rec)                      # a front has formed
    x = c.get_neutral_fraction().reshape(w.nz, w.ny, w.nx).astype(np.float64)
    P = oracle.Problem.from_workload(w)
    dt = c.compute_dt()
    dt_ref = P.compute_dt(x, scheme=2, K4=0.25)
    assert abs(dt / dt_ref - 1.0) <= 1e-10, (dt, dt_ref)
    c.step(dt)
    N = c.get_column_density(0).reshape(w.nz, w.ny, w.nx)
    Nref = P.trace(0, x)
    rel = np.abs(N - Nref) / np.maximum(Nref, 1e10)
    assert float(rel.max()) <= 1e-10, float(rel.max())
    xn = c.get_neutral_fraction().ravel()
    moved = np.abs(xn - x.ravel())
    rng = np.random.default_rng(1)
    idx = np.unique(np.concatenate([np.argsort(moved)[-400:], rng.choice(x.size, 400, replace=False)]))
    assert moved[idx].max() > 1e-3                 # the sample holds cells the step really moves
    xo = P.integrate_cells(idx, x.ravel()[idx], Nref[None], dt)
    err = np.abs(xn[idx] - xo)
    assert float(err.max()) <= 1e-9, (float(err.max()), int(idx[np.argmax(err)]))


def test_fullsize_mixed_front_against_fp64(workload):
    w = workload
    t_end = 0.02 * w.t_rec
    cm = oots.Context.from_workload(w, "mixed", scheme=oots.OOTS_A3, K4=0.25)
    cf = oots.Context.from_workload(w, "fp64", scheme=oots.OOTS_A3, K4=0.25)
    cm.advance(t_end)
    cf.advance(t_end)
    xm = cm.get_neutral_fraction()
    xf = cf.get_neutral_fraction()
    rm, rf = _reff(xm, w.dx), _reff(xf, w.dx)
    assert abs(rm / rf - 1.0) <= 5e-3 * 0.1          # a tenth of the 0.5% gate
    vm, vf = float((1 - xm).sum()), float((1 - xf).sum())
    assert abs(vm / vf - 1.0) <= 1e-3
    assert float(np.abs(xm - xf).max()) <= 1e-3
